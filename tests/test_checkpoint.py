"""Checkpoint / resume (lbhpde_batch_save / lbhpde_batch_load, lbhpde_save / lbhpde_load) through
the C ABI.

A batch of mixed members (D1Q5 and D1Q7, resident and windowed, periodic and bounded) takes n
steps, is saved, and takes m more; a second batch of the same members loads the checkpoint and
takes the same m steps.  The two results must be equal bit for bit, in FP32 and FP64, and the
loaded batch's step count continues.  Loading a checkpoint of another layout or precision, or a
truncated one, is refused and changes nothing.
"""
import numpy as np
import pytest

from paper_0907_1720_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0907_1720_gb300 import build as B
    B.build()
    from paper_0907_1720_gb300 import lbhpde
    lbhpde.lib()
    return lbhpde


def members():
    kdv = W.kdv_config(N=400, t_end=0.01)
    kaw = W.kawahara_config(N=600, dt=1e-3, tau=2.53, t_end=0.05)
    wide = W.kdv_burgers_ensemble(count=1, n_lo=9000, n_hi=9000, nsteps=50)[0]  # windows
    bnd = W.bounded_config("4.1", 1e-3, 2.05, 0.05, scheme=1 | 0x100)
    bnd.meta["depth"] = 2
    return [kdv, kaw, wide, bnd]


def step(L, b, probs, n, done):
    bounded = [i for i, p in enumerate(probs) if getattr(p, "boundary", "periodic") == "nee"]
    if not bounded:
        b.step(n)
        return
    pb = W.boundary_values(probs[bounded[0]], 2, done, n)  # one bounded member: a shared array
    b.step_nee(n, pb, 0)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_resume_is_bitwise(L, precision):
    P = L.FP32_DEV if precision == "fp32" else L.FP64
    probs = members()
    n, m = 37, 45
    a = L.Batch(probs, precision=P)
    a.set_phi(np.concatenate([p.phi0 for p in probs]))
    step(L, a, probs, n, 0)
    ck = a.save()
    step(L, a, probs, m, n)
    want = a.read_phi()
    d_want = a.diagnostics()
    a.close()

    b = L.Batch(probs, precision=P)
    b.load(ck)
    step(L, b, probs, m, n)
    got = b.read_phi()
    d_got = b.diagnostics()
    b.close()
    assert np.array_equal(got, want)
    assert [d["steps"] for d in d_got] == [d["steps"] for d in d_want] == [n + m] * len(probs)


def test_single_instance_and_refusals(L):
    p = W.kdv_config(N=400, t_end=0.01)
    s = L.Solver.for_problem(p, precision=L.FP32_DEV)
    s.set_phi(p.phi0).step(20)
    ck = s.save()
    want = s.step(30).read_phi()
    s2 = L.Solver.for_problem(p, precision=L.FP32_DEV)
    got = s2.load(ck).step(30).read_phi()
    assert np.array_equal(got, want)
    # another precision, another size, a truncated buffer: refused, the state unchanged
    s64 = L.Solver.for_problem(p, precision=L.FP64)
    q = W.kdv_config(N=401, t_end=0.01)
    s401 = L.Solver.for_problem(q, precision=L.FP32_DEV)
    for h, buf in ((s64, ck), (s401, ck), (s2, ck[: len(ck) // 2])):
        with pytest.raises(L.LbhpdeError) as ei:
            h.load(buf)
        assert ei.value.code == L.ERR_ARG
    assert np.array_equal(s2.read_phi(), got)
    # a batch whose phi was never set has nothing to save
    fresh = L.Solver.for_problem(p, precision=L.FP32_DEV)
    with pytest.raises(L.LbhpdeError) as ei:
        fresh.save()
    assert ei.value.code == L.ERR_ARG
    for h in (s, s2, s64, s401, fresh):
        h.close()

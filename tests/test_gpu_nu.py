"""Real-exponent flux functions on the GPU (class (1) of Sec. III C with u^n u_x, real n)
against the oracle, through the C ABI.  Such models take the run-time degree paths of the
streaming and on-chip kernels (w = phi^nu once per node, then a Horner evaluation in phi and w).

FP64 tolerance 1e-12 normwise on problems whose rounding growth the oracle measures below 2
(a 1e-13 perturbation of phi0). Where n < 1, phi stays away from 0: phi^n has an infinite
slope there, and two roundings on either side of zero would differ by far more than an ulp.
"""
import numpy as np
import pytest

import oracle
from paper_0907_1720_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
FP64_TOL = 1e-12
N, DX = 600, 0.1
X = W.grid(-30.0, N, DX)
LEN = N * DX


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0907_1720_gb300 import build as B
    B.build()
    from paper_0907_1720_gb300 import lbhpde
    lbhpde.lib()
    return lbhpde


def normwise(a, b):
    assert np.all(np.isfinite(b)), "the oracle diverged"
    return float(np.abs(a - b).max() / np.abs(b).max())


def oracle_periodic(p):
    eq = p.eq
    M = oracle.Model(eq.alpha, eq.pi, p.dx, p.dt, p.tau, lattice=eq.lattice, scheme=p.scheme, nu=eq.nu,
                     pi_nu=eq.pi_nu)
    f = M.init(p.phi0)
    M.step(f, p.nsteps)
    return M.phi(f)


def problems():
    return {
        "gkdv_1.5_soliton": W.Problem(W.gkdv(1.5), N, DX, 1e-4, 1.3, 2000, W.gkdv_soliton(X, 0.0, 1.5, L=LEN),
                                      xl=-30.0),
        "gkdv_0.5_offset": W.Problem(W.gkdv(0.5), N, DX, 1e-4, 1.3, 2000, 0.8 + 0.4 * W.sech(X / 2.0) ** 2,
                                     xl=-30.0),
        "ks_real_d1q5": W.Problem(W.class1_real(1.0, 0.6, 2.3, (0.05, 0.8, 0.2)), N, DX, 1e-4, 1.3, 2000,
                                  0.6 + 0.3 * np.cos(2 * np.pi * X / LEN), xl=-30.0),
        "kawahara_real_d1q7": W.Problem(W.class1_real(1.0, -0.4, 1.7, (0.0, 1.0, 0.0, -1.0)), N, DX, 1e-4, 2.02,
                                        1000, 0.5 + 0.3 * W.sech(X / 3.0) ** 2, xl=-30.0),
    }


KERNELS = {"auto": 0, "stream": 1, "onchip": 2, "halo": 3, "onchip_k2": 2}


@pytest.mark.parametrize("name", list(problems()))
@pytest.mark.parametrize("kernel", list(KERNELS))
def test_fp64_matches_oracle(L, name, kernel):
    """Every kernel: the streaming step, the resident and windowed on-chip variants with the
    real-exponent evaluation, and 2 nodes a thread (which real exponents take by streaming)."""
    p = problems()[name]
    want = oracle_periodic(p)
    s = L.Solver.for_problem(p, precision=L.FP64)
    K = 2 if kernel == "onchip_k2" else 0
    if kernel == "onchip_k2" and p.eq.lattice == 7:
        pytest.skip("D1Q7 needs at least 3 nodes a thread")
    s.set_kernel(KERNELS[kernel], K)
    got = s.set_phi(p.phi0).step(p.nsteps).read_phi()
    s.close()
    assert normwise(got, want) <= FP64_TOL


@pytest.mark.parametrize("kernel", ["onchip", "halo"])
def test_fp32_onchip_matches_fp64(L, kernel):
    """FP32 on the on-chip variants stays within the FP32 bound of the parity tests (64 eps32
    sqrt(steps) + 1e-6, a random walk of per-step roundings) of the FP64 oracle: gKdV soliton,
    2000 steps, with phi^nu by the FP32 intrinsic."""
    p = problems()["gkdv_1.5_soliton"]
    want = oracle_periodic(p)
    s = L.Solver.for_problem(p, precision=L.FP32_DEV)
    s.set_kernel(KERNELS[kernel])
    got = s.set_phi(p.phi0).step(p.nsteps).read_phi()
    s.close()
    assert normwise(got, want) <= 64 * np.finfo(np.float32).eps * np.sqrt(p.nsteps) + 1e-6


def test_batch_with_real_exponent_and_polynomial_members(L):
    """A real-exponent member sends its lattice group to the streaming kernel; every member,
    ordinary ones included, still matches its own oracle run."""
    ps = problems()
    kdv = W.kdv_config(N=400, dt=1e-4, tau=1.3, t_end=0.1)
    probs = [ps["gkdv_1.5_soliton"], kdv, ps["kawahara_real_d1q7"], W.kawahara_config(N=600, t_end=0.05)]
    n = 500
    for p in probs:
        p.nsteps = n
    b = L.Batch(probs, precision=L.FP64)
    b.set_phi(np.concatenate([p.phi0 for p in probs])).step(n)
    got = b.split(b.read_phi())
    b.close()
    for p, g in zip(probs, got):
        want = oracle_periodic(p) if p.eq.pi_nu is not None else oracle.run_problem(p)
        assert normwise(g, want) <= FP64_TOL, p.eq.name


def _bounded_real_problems():
    """Real-exponent models on bounded grids with boundary values from a known profile: the gKdV
    soliton (n = 1.5, D1Q5) with its exact solution, and a D1Q7 class (1) model whose boundary
    holds its initial values (a slowly varying profile whose ends stay at the background)."""
    n, dt, tau = 1.5, 1e-4, 1.3
    ex = lambda x, t: W.gkdv_soliton(x, t, n, x0=-5.0)  # noqa: E731
    x = W.grid(-30.0, 601, DX)
    gk = W.Problem(W.gkdv(n), 601, DX, dt, tau, 1500, ex(x, 0.0), xl=-30.0, exact=lambda t: ex(x, t),
                   boundary="nee", exact_xt=ex, meta={"depth": 2})
    prof = lambda x, t: 0.5 + 0.3 * W.sech(x / 3.0) ** 2 + 0.0 * t  # noqa: E731
    kw = W.Problem(W.class1_real(1.0, -0.4, 1.7, (0.0, 1.0, 0.0, -1.0)), 601, DX, 1e-4, 2.02, 600, prof(x, 0.0),
                   xl=-30.0, exact=lambda t: prof(x, t), boundary="nee", exact_xt=prof, meta={"depth": 2})
    return {"gkdv_1.5_soliton_q5": gk, "kawahara_real_q7": kw}


def _oracle_bounded(p, phi0=None):
    M = oracle.Model(p.eq.alpha, p.eq.pi, p.dx, p.dt, p.tau, lattice=p.eq.lattice, scheme=p.scheme, nu=p.eq.nu,
                     pi_nu=p.eq.pi_nu)
    f = M.init(p.phi0 if phi0 is None else phi0)
    return M.phi(M.step_nee(f, W.boundary_values(p, (M.b - 1) // 2, 0, p.nsteps), p.meta["depth"]))


def _gpu_bounded(L, p, precision, kernel):
    s = L.Solver.for_problem(p, precision=precision)
    s.set_kernel(kernel)
    Wd = (s.model().b - 1) // 2
    s.set_phi(p.phi0)
    done = 0
    for m in (p.nsteps // 3, p.nsteps - p.nsteps // 3):  # two launches: the boundary rows' offset
        s.step_nee(m, W.boundary_values(p, Wd, done, m))
        done += m
    got = s.read_phi()
    s.close()
    return got


@pytest.mark.parametrize("name", list(_bounded_real_problems()))
@pytest.mark.parametrize("kernel", ["resident", "stream"])
def test_bounded_real_exponent(L, name, kernel):
    """Real exponents on bounded grids: the resident bounded kernel's variant with the
    generalised f^eq (in the relaxation, at x_f and at the boundary values), and the streaming
    step with the outer-node rebuild, against the oracle's bounded step."""
    p = _bounded_real_problems()[name]
    want = _oracle_bounded(p)
    got = _gpu_bounded(L, p, L.FP64, L.KERNEL_STREAM if kernel == "stream" else L.KERNEL_AUTO)
    assert normwise(got, want) <= FP64_TOL


@pytest.mark.parametrize("name", list(_bounded_real_problems()))
def test_fp32_bounded_real_exponent(L, name):
    """FP32 on the resident bounded kernel with real exponents: within one FP32 rounding of phi
    and of the stored deviations a step, added like a random walk, times the growth of a
    perturbation of phi0 that the oracle measures on the problem."""
    p = _bounded_real_problems()[name]
    want = _oracle_bounded(p)
    rng = np.random.default_rng(0)
    pert = _oracle_bounded(p, p.phi0 * (1 + 1e-6 * rng.standard_normal(p.N)))
    growth = max(1.0, normwise(pert, want) / 1e-6)
    eps = 2.0 ** -24
    got = _gpu_bounded(L, p, L.FP32_DEV, L.KERNEL_AUTO)
    assert normwise(got, want) <= (16 * eps * np.sqrt(p.nsteps) + 4 * eps) * growth


def test_fp32_accuracy(L):
    """FP32 on the gKdV soliton: error against the exact solution within twice the FP64 path's."""
    p = problems()["gkdv_1.5_soliton"]
    p.nsteps = 10000
    ex = W.gkdv_soliton(X, 1.0, 1.5, L=LEN)
    errs = {}
    for prec in (L.FP64, L.FP32_DEV):
        s = L.Solver.for_problem(p, precision=prec)
        errs[prec] = oracle.error_E(s.set_phi(p.phi0).step(p.nsteps).read_phi(), ex)
        s.close()
    assert errs[L.FP64] < 0.05
    assert errs[L.FP32_DEV] <= 2.0 * errs[L.FP64]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_server_serves_real_exponent_requests(L, precision):
    """Real-exponent requests mixed with polynomial ones in the server: each result equals, bit
    for bit, the same request solved alone on the on-chip kernels, and matches the oracle."""
    P = L.FP32_DEV if precision == "fp32" else L.FP64
    ps = problems()
    xw = W.grid(-450.0, 9000, DX)  # longer than a resident CTA holds: windows
    wide = W.Problem(W.gkdv(1.5), 9000, DX, 1e-4, 1.3, 0, W.gkdv_soliton(xw, 0.0, 1.5, L=900.0), xl=-450.0)
    reqs = [ps["gkdv_1.5_soliton"], W.kdv_config(N=400, dt=1e-4, tau=1.3, t_end=0.0), ps["ks_real_d1q5"],
            ps["kawahara_real_d1q7"], ps["gkdv_0.5_offset"], wide]
    for i, p in enumerate(reqs):
        p.nsteps = 300 + 37 * i
    srv = L.Server(precision=P, device_bytes=64 << 20, max_active=16, steps_per_block=128)
    ids = [srv.submit_problem(p) for p in reqs]
    got = [srv.wait(i, 120.0) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["error"] == 0
    for (rc, phi, info), p in zip(got, reqs):
        assert rc == L.OK, (p.eq.name, rc)
        s = L.Solver.for_problem(p, precision=P).set_kernel(L.KERNEL_ONCHIP)
        alone = s.set_phi(p.phi0).step(p.nsteps).read_phi()
        s.close()
        assert np.array_equal(phi, alone), p.eq.name
        want = oracle_periodic(p) if p.eq.pi_nu is not None else oracle.run_problem(p)
        tol = FP64_TOL if P == L.FP64 else 64 * np.finfo(np.float32).eps * np.sqrt(p.nsteps) + 1e-6
        assert normwise(phi, want) <= tol, p.eq.name


def test_replan_discards_captured_graphs(L):
    """Re-planning between long streaming runs (lbhpde_batch_set_kernel, which rebuilds the
    captured graphs) keeps every member of a mixed batch on its oracle trajectory: a
    real-exponent member and an ordinary D1Q7 member, 200 steps, a re-plan, 200 more."""
    ps = problems()
    gk = ps["gkdv_1.5_soliton"]
    kaw = W.kawahara_config(N=600, dt=1e-4, tau=2.02, t_end=0.0)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        b = L.Batch([gk, kaw], precision=L.FP64)
        b.set_phi(np.concatenate([gk.phi0, kaw.phi0])).step(200)
        b.set_kernel(L.KERNEL_STREAM)
        b.step(200)
        got = b.split(b.read_phi())
        b.close()
    gk.nsteps = kaw.nsteps = 400
    assert normwise(got[0], oracle_periodic(gk)) <= FP64_TOL
    assert normwise(got[1], oracle.run_problem(kaw)) <= FP64_TOL

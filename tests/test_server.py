"""The continuous-batching request server (lbhpde_server_*) through the C ABI.

Requests of different equations, lattices and sizes (resident instances and temporally
blocked windows) are submitted while others are running; every result must be identical,
bit for bit, to the same request solved alone with the single-instance API, and agree with
the oracle.  Also: bounded waits, unknown ids, requests larger than the arena, bad arguments.
"""
import copy
import time

import numpy as np
import pytest

import oracle
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


def bump(N, dx, seed):
    rng = np.random.default_rng(seed)
    Lx = N * dx
    x = W.grid(-0.5 * Lx, N, dx)
    return rng.uniform(0.4, 0.9) * W.sech((x - rng.uniform(-0.1, 0.1) * Lx) / max(3 * dx, 0.08 * Lx)) ** 2


def mixed_requests(n, seed=0):
    # (equation, dt, tau): stable choices from the oracle scans
    menu = [(W.kdv_burgers(2.0, 0.05, 0.9), 1e-4, 1.3), (W.kdv(), 1e-4, 1.3), (W.ks(), 1e-4, 1.3),
            (W.kawahara(), 1e-3, 2.5), (W.mkdv(), 1e-4, 1.2), (W.k22(), 1e-4, 1.5)]
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        eq, dt, tau = menu[i % len(menu)]
        N = int(np.exp(rng.uniform(np.log(8), np.log(9000))))
        steps = int(rng.integers(0, 600))
        out.append(W.Problem(eq, N, 0.1, dt, tau, steps, bump(N, 0.1, seed * 1000 + i)))
    return out


def alone(L, p, precision):
    s = L.Solver.for_problem(p, precision=precision)
    s.set_phi(p.phi0).step(p.nsteps)
    out = s.read_phi(check=False)
    s.close()
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_results_identical_alone_and_in_the_mix(L, precision):
    P = L.FP32_DEV if precision == "fp32" else L.FP64
    t_start = time.time()
    srv = L.Server(precision=P, device_bytes=64 << 20, max_active=64, steps_per_block=128)
    first = mixed_requests(20, seed=1)
    ids = [srv.submit_problem(p) for p in first]
    # more requests arrive while the first ones run
    time.sleep(0.01)
    late = mixed_requests(20, seed=2)
    ids += [srv.submit_problem(p) for p in late]
    probs = first + late
    results = {}
    deadline = time.time() + 120
    while len(results) < len(ids) and time.time() < deadline:
        for rid in ids:
            if rid in results:
                continue
            rc, phi, info = srv.poll(rid)
            if rc != L.PENDING:
                results[rid] = (rc, phi, info)
        time.sleep(0.002)
    st = srv.stats()
    srv.close()
    assert len(results) == len(ids), st
    assert st["error"] == 0 and st["completed"] == len(ids)
    # the scheduler's phase times (one thread, so they add up to at most the wall time)
    phases = [st[k] for k in ("host_admit_s", "host_setup_s", "host_plan_s", "host_launch_s", "host_wait_s",
                              "host_retire_s")]
    assert min(phases) >= 0 and st["gpu_busy_s"] > 0
    assert sum(phases) <= time.time() - t_start
    for rid, p in zip(ids, probs):
        rc, phi, info = results[rid]
        assert rc == L.OK, (p.eq.name, p.N, rc)
        assert info["steps_done"] == p.nsteps
        assert info["finish_s"] >= info["admit_s"] >= info["submit_s"] >= 0
        assert np.array_equal(phi, alone(L, p, P)), (p.eq.name, p.N, p.nsteps)
    tol = 1e-12 if P == L.FP64 else 64 * 2.0 ** -24 * np.sqrt(600) + 1e-6
    for rid, p in list(zip(ids, probs))[::7]:
        want = oracle.run_problem(p)
        got = results[rid][1]
        assert np.abs(got - want).max() <= tol * np.abs(want).max()


def _bounded_requests(n, seed):
    """Bounded requests (Sec. IV examples on D1Q5 and D1Q7, depths 1-3, grids of 601-2001
    nodes, and the gKdV soliton with the real exponent 1.5) with random step counts, each with
    its boundary values from the exact solution."""
    menu = [("4.1", 1e-3, 1.989, 1 | oracle.NO_AUX_CORRECTION, 2), ("4.2", 1e-2, 4.569, 1 | oracle.NO_AUX_CORRECTION, 2),
            ("4.5", 1e-4, 2.02, 1, 1), ("4.6", 1e-2, 4.04, 2, 3), ("4.7", 1e-3, 3.31, 1, 2)]
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        ex, dt, tau, scheme, depth = menu[i % len(menu)]
        steps = int(rng.integers(0, 400))
        if i % 6 == 5:
            ex_ = lambda x, t: W.gkdv_soliton(x, t, 1.5, x0=-5.0)  # noqa: E731
            x = W.grid(-30.0, 601, 0.1)
            p = W.Problem(W.gkdv(1.5), 601, 0.1, 1e-4, 1.3, steps, ex_(x, 0.0), xl=-30.0,
                          exact=lambda t, x=x: ex_(x, t), boundary="nee", exact_xt=ex_, meta={"depth": 2})
        else:
            p = W.bounded_config(ex, dt, tau, steps * dt, scheme=scheme)
            p.meta["depth"] = depth
        out.append(p)
    return out


def _bounded_alone(L, p, precision, phib):
    """The same bounded request solved alone on the one-instance-per-CTA bounded kernel."""
    s = L.Solver.for_problem(p, precision=precision)
    s.set_kernel(L.KERNEL_ONCHIP, 4)
    s.set_phi(p.phi0)
    if p.nsteps:
        s.step_nee(p.nsteps, phib)
    out = s.read_phi(check=False)
    s.close()
    return out


def _wd(p):
    """max|e_j| of p's lattice (the columns of its boundary rows are 2 max|e_j|)."""
    M = oracle.Model(p.eq.alpha, p.eq.pi, p.dx, p.dt, p.tau, lattice=p.eq.lattice, scheme=p.scheme, nu=p.eq.nu,
                     pi_nu=p.eq.pi_nu)
    return (M.b - 1) // 2


def _oracle_nee(p):
    M = oracle.Model(p.eq.alpha, p.eq.pi, p.dx, p.dt, p.tau, lattice=p.eq.lattice, scheme=p.scheme, nu=p.eq.nu,
                     pi_nu=p.eq.pi_nu)
    f = M.init(p.phi0)
    if p.nsteps:
        M.step_nee(f, W.boundary_values(p, (M.b - 1) // 2, 0, p.nsteps), p.meta["depth"])
    return M.phi(f)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_bounded_requests_in_the_mix(L, precision):
    """Bounded requests among periodic ones, over several step blocks whose launches end where a
    request's steps end: each result equals, bit for bit, the request solved alone on the bounded
    kernel, and agrees with the oracle's bounded step."""
    P = L.FP32_DEV if precision == "fp32" else L.FP64
    srv = L.Server(precision=P, device_bytes=64 << 20, max_active=64, steps_per_block=128)
    bnd = _bounded_requests(10, seed=3)
    per = mixed_requests(10, seed=4)
    ids = []
    for i in range(10):
        p = bnd[i]
        Wd = _wd(p)
        ids.append((srv.submit_problem(p, phib=W.boundary_values(p, Wd, 0, p.nsteps)), p, True))
        ids.append((srv.submit_problem(per[i]), per[i], False))
    results = {rid: srv.wait(rid, timeout=120) for rid, _, _ in ids}
    st = srv.stats()
    srv.close()
    assert st["error"] == 0 and st["completed"] == len(ids)
    for rid, p, is_bnd in ids:
        rc, phi, info = results[rid]
        assert rc == L.OK and info["steps_done"] == p.nsteps, (p.N, rc)
        if is_bnd:
            Wd = _wd(p)
            want = _bounded_alone(L, p, P, W.boundary_values(p, Wd, 0, p.nsteps))
        else:
            want = alone(L, p, P)
        assert np.array_equal(phi, want), (p.eq.name, p.N, p.nsteps, is_bnd)
    for rid, p, is_bnd in ids[::3]:
        if not is_bnd or p.nsteps == 0:
            continue
        want = _oracle_nee(p)
        got = results[rid][1]
        if P == L.FP64:
            tol = 1e-12
        else:
            # one FP32 rounding of phi and of the stored deviations a step, added like a random
            # walk, times the growth of a perturbation of phi0 that the oracle measures on p
            q = copy.copy(p)
            q.phi0 = p.phi0 * (1 + 1e-6 * np.random.default_rng(0).standard_normal(p.N))
            growth = np.abs(_oracle_nee(q) - want).max() / np.abs(want).max() / 1e-6
            tol = (16 * 2.0 ** -24 * np.sqrt(p.nsteps) + 4 * 2.0 ** -24) * max(1.0, growth)
        assert np.abs(got - want).max() <= tol * np.abs(want).max(), (p.meta, p.nsteps)


def test_bounded_request_arguments(L):
    srv = L.Server(precision=L.FP32_DEV, device_bytes=8 << 20, max_active=4)
    p = W.bounded_config("4.1", 1e-3, 1.989, 0.01, scheme=1 | oracle.NO_AUX_CORRECTION)
    with pytest.raises(L.LbhpdeError) as ei:  # boundary values missing
        srv.submit(p.eq, p.N, p.dx, p.dt, p.tau, p.nsteps, p.phi0, p.scheme, boundary=L.NEE, phib=None)
    assert ei.value.code == L.ERR_ARG
    with pytest.raises(L.LbhpdeError) as ei:  # N < 2 (W + depth)
        srv.submit(p.eq, 7, p.dx, p.dt, p.tau, 1, p.phi0[:7], p.scheme, boundary=L.NEE, phib=np.zeros((1, 4)))
    assert ei.value.code == L.ERR_ARG
    big = W.bounded_config("4.1", 1e-3, 1.989, 0.001, scheme=1, dx=0.02)  # 3001 nodes: over one CTA
    with pytest.raises(L.LbhpdeError) as ei:
        srv.submit_problem(big, phib=W.boundary_values(big, 2, 0, big.nsteps))
    assert ei.value.code == L.ERR_UNSUPPORTED
    rid = srv.submit_problem(p, phib=W.boundary_values(p, 2, 0, p.nsteps))
    rc, phi, info = srv.wait(rid, timeout=60)
    assert rc == L.OK and info["steps_done"] == p.nsteps
    srv.close()


def test_admission_is_bounded_by_memory(L):
    """With an arena that holds only a few requests at a time, all still complete."""
    srv = L.Server(precision=L.FP32_DEV, device_bytes=2 << 20, max_active=8, steps_per_block=64)
    probs = [W.Problem(W.kdv_burgers(2.0, 0.05, 0.9), 4000, 0.1, 1e-4, 1.3, 200, bump(4000, 0.1, i))
             for i in range(12)]
    ids = [srv.submit_problem(p) for p in probs]
    for rid, p in zip(ids, probs):
        rc, phi, info = srv.wait(rid, timeout=60)
        assert rc == L.OK
        assert np.array_equal(phi, alone(L, p, L.FP32_DEV))
    st = srv.stats()
    assert st["bytes_in_use"] == 0 and st["queued"] == 0
    srv.close()


def test_wait_timeout_poll_unknown_and_oversize(L):
    srv = L.Server(precision=L.FP32_DEV, device_bytes=4 << 20, max_active=4)
    p = W.Problem(W.kawahara(), 3000, 0.1, 1e-3, 2.5, 200000, bump(3000, 0.1, 3))
    rid = srv.submit_problem(p)
    rc, phi, info = srv.wait(rid, timeout=0.0)
    assert rc == L.ERR_TIMEOUT and phi is None and info["status"] == L.PENDING
    rc, _, _ = srv.poll(rid)
    assert rc == L.PENDING
    with pytest.raises(L.LbhpdeError) as ei:
        srv.poll(rid + 1000)
    assert ei.value.code == L.ERR_NOT_FOUND
    big = W.Problem(W.kdv(), 1 << 20, 0.1, 1e-4, 1.3, 1, np.zeros(1 << 20))
    with pytest.raises(L.LbhpdeError) as ei:
        srv.submit_problem(big)  # 2 buffers x 5 rows x 4 MiB > 4 MiB arena
    assert ei.value.code == L.ERR_OOM
    bad = W.Problem(W.kdv(), 3, 0.1, 1e-4, 1.3, 1, np.zeros(3))  # N < 2 max|e|
    with pytest.raises(L.LbhpdeError) as ei:
        srv.submit_problem(bad)
    assert ei.value.code == L.ERR_ARG
    srv.close()  # drops the long request still running


def test_divergent_request_is_reported(L):
    srv = L.Server(precision=L.FP32_DEV, device_bytes=8 << 20, max_active=4)
    phi0 = bump(500, 0.1, 4)
    phi0[7] = np.nan
    rid = srv.submit(W.kdv(), 500, 0.1, 1e-4, 1.3, 10, phi0)
    ok = srv.submit(W.kdv(), 500, 0.1, 1e-4, 1.3, 10, bump(500, 0.1, 5))
    rc, phi, info = srv.wait(rid, timeout=60)
    assert rc == L.ERR_DIVERGED and info["nonfinite"] > 0
    rc, phi, info = srv.wait(ok, timeout=60)
    assert rc == L.OK and info["nonfinite"] == 0
    srv.close()

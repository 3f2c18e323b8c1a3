"""GPU path vs the CPU oracle, element by element, through the C ABI.

Tolerances (normwise: max_x |phi_gpu - phi_oracle| / max_x |phi_oracle|):
* FP64: 1e-12, the stated bound.  Both sides round every operation in IEEE double; they
  differ only in evaluation order (Horner with omega folded in, flux-difference update of
  phi, fused multiply-add on the GPU), a few ulp per step.
* FP32 deviation storage: FP32_TOL(n) = 16 * eps32 * sqrt(n) + 4 * eps32 (eps32 = 2^-24,
  relative to max|phi|).  Model: each step rounds phi and the stored deviations once in
  float, and these roundings add up like a random walk over the n steps (sqrt(n)); the second
  term is the one-time rounding of the initial state.  Measured on GB300 over every case
  below and every kernel, the FP32-minus-oracle gap is at most 4.0 eps32 sqrt(n) (scheme-2
  KdV) and at most 1.5 eps32 sqrt(n) on the ensemble members at 1000 steps, so the bound is
  4x the worst measured case and about 10x the ensemble's: an encoding slip or a lost
  rounding step costing 10x the honest error fails it.  The accuracy bar of the FP32 path
  (error against the exact solution within twice the FP64 path's) is checked on full runs.
"""
import math
import os
import zlib

import numpy as np
import pytest

import oracle
from paper_0907_1720_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
FP64_TOL = 1e-12


def FP32_TOL(n):
    return 16 * 2.0 ** -24 * math.sqrt(max(n, 1)) + 4 * 2.0 ** -24


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
    assert np.all(np.isfinite(b)), "the oracle diverged: the test problem is unstable"
    return float(np.abs(a - b).max() / np.abs(b).max())


def problem(eq, N, dx, dt, tau, nsteps, scheme=1, width=None, seed=0):
    """A soliton-like bump on a periodic grid (random amplitude/offset from the seed)."""
    rng = np.random.default_rng(seed)
    L_ = N * dx
    x = W.grid(-0.5 * L_, N, dx)
    w = width or max(3 * dx, 0.08 * L_)
    amp = rng.uniform(0.5, 1.0)
    phi0 = amp * W.sech((x - rng.uniform(-0.1, 0.1) * L_) / w) ** 2 + 0.05 * np.cos(2 * np.pi * x / L_)
    return W.Problem(eq, N, dx, dt, tau, nsteps, phi0, xl=-0.5 * L_, scheme=scheme)


def run_gpu(L, p, precision, kernel, K=0, spl=0, nsteps=None):
    s = L.Solver.for_problem(p, precision=precision)
    s.set_kernel(kernel, K, spl)
    s.set_phi(p.phi0)
    s.step(p.nsteps if nsteps is None else nsteps)
    out = s.read_phi()
    s.close()
    return out


CASES = [
    # name, equation, N, dx, dt, tau, steps, scheme
    ("kdv_400", W.kdv(), 400, 0.1, 2e-5, 1.07, 1500, 1),
    ("ks_1024", W.ks(), 1024, 32 * math.pi / 1024, 1e-4, 1.3, 1500, 1),
    ("kawahara_q7_600", W.kawahara(), 600, 0.1, 1e-4, 2.02, 1500, 1),
    ("kawahara_q7_s2_601", W.kawahara(), 601, 0.1, 1e-3, 2.55, 800, 2),
    ("mod_kawahara_q7_D13", W.modified_kawahara(), 300, 0.1, 1e-2, 4.54, 200, 1),
    ("mkdv_D9_515", W.mkdv(), 515, 0.1, 1e-4, 1.2, 800, 1),
    ("k22_333", W.k22(), 333, 0.1, 1e-4, 1.5, 600, 1),
    ("kdv_burgers_1025", W.kdv_burgers(3.0, 0.07, 0.8), 1025, 0.1, 1e-4, 1.15, 600, 1),
    ("kdv_s2_777", W.kdv(), 777, 0.1, 1e-4, 1.3, 600, 2),
    ("gks_cubic_q7_250", W.gks_cubic(lattice=7), 250, 0.1, 1e-3, 3.0, 300, 1),
    ("sixth_q7_96", W.Equation("sixth", (1.0, 0.0, 0.5, 0.3, -1.0, 0.2),
                               ((0, 0, 0.5), (), (0, 1), (0, 1), (0, 1), (0, 1))), 96, 0.1, 1e-4, 3.0, 300, 1),
]


KERNELS = ["stream", "onchip", "halo"]


def kernel_id(L, name):
    return {"stream": L.KERNEL_STREAM, "onchip": L.KERNEL_ONCHIP, "halo": L.KERNEL_HALO}[name]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kernel", KERNELS)
def test_fp64_matches_oracle(L, case, kernel):
    name, eq, N, dx, dt, tau, n, scheme = case
    p = problem(eq, N, dx, dt, tau, n, scheme, seed=zlib.crc32(name.encode()) % 1000)
    want = oracle.run_problem(p)
    K = kernel_id(L, kernel)
    got = run_gpu(L, p, L.FP64, K)
    assert normwise(got, want) <= FP64_TOL


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kernel", KERNELS)
def test_fp32_matches_oracle(L, case, kernel):
    name, eq, N, dx, dt, tau, n, scheme = case
    p = problem(eq, N, dx, dt, tau, n, scheme, seed=zlib.crc32(name.encode()) % 1000)
    want = oracle.run_problem(p)
    K = kernel_id(L, kernel)
    got = run_gpu(L, p, L.FP32_DEV, K)
    assert normwise(got, want) <= FP32_TOL(n)


# ragged and extreme sizes: minimum N (2 max|e|), one node past a tile, thread counts that
# leave the last thread 1..K-1 nodes, several 1024-node tiles
SIZES = [(5, 4), (5, 5), (5, 9), (5, 17), (5, 33), (5, 255), (5, 1023), (5, 1025), (5, 2049), (5, 4095),
         (7, 6), (7, 7), (7, 13), (7, 31), (7, 250), (7, 1021), (7, 2047), (7, 3073)]


@pytest.mark.parametrize("b,N", SIZES, ids=[f"q{b}_N{N}" for b, N in SIZES])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sizes_both_kernels(L, b, N, prec):
    eq = W.kdv_burgers(2.0, 0.05, 0.9) if b == 5 else W.kawahara()
    p = problem(eq, N, 0.1, 1e-4 if b == 5 else 1e-3, 1.3 if b == 5 else 2.3, 97, seed=N)
    want = oracle.run_problem(p)
    P = L.FP64 if prec == "fp64" else L.FP32_DEV
    tol = FP64_TOL if prec == "fp64" else FP32_TOL(97)
    got_s = run_gpu(L, p, P, L.KERNEL_STREAM)
    assert normwise(got_s, want) <= tol
    for kern, K, spl in [(k, K, spl) for k in (L.KERNEL_ONCHIP, L.KERNEL_HALO)
                         for K in ((2, 4, 8, 16) if b == 5 else (4, 8)) for spl in (0, 13)]:
        s = L.Solver.for_problem(p, precision=P)
        try:
            s.set_kernel(kern, K, spl)
        except L.LbhpdeError as e:
            assert e.code == L.ERR_UNSUPPORTED
            s.close()
            continue
        s.set_phi(p.phi0).step(p.nsteps)
        got = s.read_phi()
        s.close()
        assert normwise(got, want) <= tol, (kern, K, spl)


def test_onchip_step_chunks_are_seamless(L):
    """Steps split over several launches give the same bits as one launch."""
    p = problem(W.ks(), 700, 0.1, 1e-4, 1.3, 333, seed=3)
    a = run_gpu(L, p, L.FP64, L.KERNEL_ONCHIP, 0, 0)
    b = run_gpu(L, p, L.FP64, L.KERNEL_ONCHIP, 0, 50)
    assert np.array_equal(a, b)


def test_resident_launch_longer_than_a_window_allows(L):
    """Resident-only batches accept a steps-per-launch whose halo would not fit a window (it
    only chunks the resident launches); a batch that needs windows refuses it."""
    p = problem(W.kdv_burgers(2.0, 0.05, 0.9), 1800, 0.1, 1e-4, 1.3, 300, seed=8)
    for P, K in ((L.FP32_DEV, 8), (L.FP64, 4)):
        got = run_gpu(L, p, P, L.KERNEL_ONCHIP, K, 1000)
        assert normwise(got, oracle.run_problem(p)) <= (FP64_TOL if P == L.FP64 else FP32_TOL(300))
    s = L.Solver.for_problem(p, precision=L.FP32_DEV)
    with pytest.raises(L.LbhpdeError) as e:
        s.set_kernel(L.KERNEL_HALO, 8, 1000)
    assert e.value.code == L.ERR_UNSUPPORTED
    s.close()


def test_step_zero_and_incremental(L):
    p = problem(W.kdv(), 128, 0.1, 1e-4, 1.3, 40, seed=9)
    s = L.Solver.for_problem(p, precision=L.FP64)
    s.set_phi(p.phi0)
    s.step(0)
    assert np.allclose(s.read_phi(), p.phi0, rtol=0, atol=0)
    for _ in range(4):
        s.step(10)
    got = s.read_phi()
    s.close()
    assert normwise(got, oracle.run_problem(p)) <= FP64_TOL


def test_conservation_and_diagnostics(L):
    p = W.kdv_config(t_end=0.02)
    s = L.Solver.for_problem(p, precision=L.FP64)
    s.set_phi(p.phi0)
    d0 = s.diagnostics()
    s.step(p.nsteps)
    ps = torch.tensor(p.exact(p.t_end), device="cuda", dtype=torch.float64)
    d1 = s.diagnostics(ps)
    phi = s.read_phi()
    s.close()
    assert d1["nonfinite"] == 0 and d1["steps"] == p.nsteps
    assert abs(d1["sum_phi"] - d0["sum_phi"]) <= 1e-12 * np.abs(p.phi0).sum()
    assert d1["err_E"] == pytest.approx(oracle.error_E(phi, p.exact(p.t_end)), rel=1e-12)
    ex = p.exact(p.t_end)
    assert d1["err_L2"] == pytest.approx(np.linalg.norm(phi - ex) / np.linalg.norm(ex), rel=1e-10)
    assert d1["max_abs_phi"] == pytest.approx(np.abs(phi).max(), rel=1e-15)


def test_uniform_state_is_fixed_point(L):
    for kernel in (L.KERNEL_STREAM, L.KERNEL_ONCHIP):
        p = W.Problem(W.kawahara(), 300, 0.1, 1e-3, 2.1, 50, np.full(300, 0.37))
        got = run_gpu(L, p, L.FP64, kernel)
        assert got.max() == got.min() and abs(got[0] - 0.37) < 1e-14


def test_nan_input_reports_divergence(L):
    """Host-side fault injection: a poisoned initial profile is reported, not trapped."""
    p = problem(W.kdv(), 256, 0.1, 1e-4, 1.3, 5)
    phi0 = p.phi0.copy()
    phi0[17] = np.nan
    for kernel in (L.KERNEL_STREAM, L.KERNEL_ONCHIP):
        s = L.Solver.for_problem(p, precision=L.FP32_DEV).set_kernel(kernel)
        s.set_phi(phi0).step(5)
        with pytest.raises(L.LbhpdeError) as ei:
            s.read_phi()
        assert ei.value.code == L.ERR_DIVERGED
        assert s.diagnostics()["nonfinite"] > 0
        s.close()


def test_unsupported_nodes_per_thread(L):
    p = problem(W.kawahara(), 1000, 0.1, 1e-3, 2.3, 1)
    s = L.Solver.for_problem(p, precision=L.FP32_DEV)
    with pytest.raises(L.LbhpdeError) as ei:
        s.set_kernel(L.KERNEL_ONCHIP, 2)  # D1Q7 needs at least 3 nodes per thread
    assert ei.value.code == L.ERR_UNSUPPORTED
    s.set_phi(p.phi0).step(1)  # the previous (automatic) choice still works
    s.close()


def test_batch_members_match_alone_bitwise(L):
    """Each instance gives the same bits alone and packed with others (both precisions)."""
    probs = []
    rng = np.random.default_rng(11)
    # (equation, dt, tau) with perturbation growth below 10 over 120 steps (oracle scan)
    eqs = [(W.kdv_burgers(2.0, 0.05, 0.9), 1e-4, 1.3), (W.kdv(), 1e-4, 1.3), (W.ks(), 1e-4, 1.3),
           (W.kawahara(), 1e-3, 2.5), (W.mkdv(), 1e-4, 1.2), (W.k22(), 1e-4, 1.5)]
    for i in range(14):
        eq, dt, tau = eqs[i % len(eqs)]
        N = int(rng.integers(6, 1500))
        probs.append(problem(eq, N, 0.1, dt, tau, 120, seed=i))
    for P in (L.FP64, L.FP32_DEV):
        for kernel in (L.KERNEL_AUTO, L.KERNEL_STREAM):
            bt = L.Batch(probs, precision=P).set_kernel(kernel)
            bt.set_phi(np.concatenate([p.phi0 for p in probs])).step(120)
            outs = bt.split(bt.read_phi())
            bt.close()
            for p, o in zip(probs, outs):
                s = L.Solver.for_problem(p, precision=P).set_kernel(kernel)
                s.set_phi(p.phi0).step(120)
                alone = s.read_phi()
                s.close()
                assert np.array_equal(o, alone), (p.eq.name, p.N, P, kernel)
                tol = FP64_TOL if P == L.FP64 else FP32_TOL(120)
                assert normwise(o, oracle.run_problem(p)) <= tol


def _window_oracle(p, x, n):
    """Oracle value of phi(x) after n steps, from a periodic window wide enough that the
    wrap-around cannot reach x (the scheme moves information at most 3 nodes per step)."""
    h = 3 * n + 8
    idx = (np.arange(x - h, x + h + 1)) % p.N
    sub = W.Problem(p.eq, idx.size, p.dx, p.dt, p.tau, n, p.phi0[idx], scheme=p.scheme)
    return oracle.run_problem(sub)[h]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_long_grid_full_size_sampled(L, prec):
    """The 2^24-node Kawahara grid in the launch configuration the benchmark times, checked
    at sampled nodes against windowed oracle runs."""
    p = W.long_grid_config(nsteps=12)
    P = L.FP64 if prec == "fp64" else L.FP32_DEV
    got = run_gpu(L, p, P, L.KERNEL_AUTO)
    rng = np.random.default_rng(5)
    xs = list(rng.integers(0, p.N, 10)) + [0, 1, 2, p.N - 1, p.N - 3, p.N // 2]
    c = np.argmax(np.abs(p.phi0))
    xs += [c - 5, c, c + 7]
    scale = np.abs(p.phi0).max()
    tol = FP64_TOL if prec == "fp64" else FP32_TOL(p.nsteps)
    for x in xs:
        want = _window_oracle(p, int(x), p.nsteps)
        assert abs(got[x] - want) <= tol * scale, x


ENSEMBLE_CLASSES = ((0, 2048), (2048, 4096), (4096, 8192))  # nodes held by 128-, 256-, 512-thread CTAs


@pytest.fixture(scope="module")
def ensemble_full(L):
    """The 4096-member KdV-Burgers ensemble of the benchmark, 1000 steps, and the oracle's phi for
    sampled members: the smallest, the largest, one from each resident CTA size class and seeded
    random picks.  The oracle runs one member per thread."""
    from concurrent.futures import ThreadPoolExecutor
    probs = W.kdv_burgers_ensemble()
    Ns = np.array([p.N for p in probs])
    pick = [int(np.argmin(Ns)), int(np.argmax(Ns))]
    for lo, hi in ENSEMBLE_CLASSES:
        pick.append(int(np.where((Ns > lo) & (Ns <= hi))[0][0]))
    rng = np.random.default_rng(1)
    pick += [int(i) for i in rng.choice(len(probs), 7, replace=False)]
    pick = sorted(set(pick))
    with ThreadPoolExecutor(max(1, min(len(pick), os.cpu_count() or 1))) as ex:
        want = dict(zip(pick, ex.map(lambda i: oracle.run_problem(probs[i]), pick)))
    return probs, want


@pytest.mark.parametrize("plan", ["bench", "windows"])
def test_ensemble_full_depth_vs_oracle(L, ensemble_full, plan):
    """The benchmark's ensemble at its full 1000 steps in the launch configuration the benchmark
    times (the on-chip pair the autotuner picks on GB300, K = 8 and 32 steps per window,
    recorded without timing; every member of up to 8192 nodes resident in the split-barrier
    kernel), and again with every member cut into those temporally blocked windows.  Sampled
    members against the oracle, normwise, within FP32_TOL(1000) = 16 eps32 sqrt(1000) + 4 eps32
    = 3.0e-5 (about 10x the gap measured on these members)."""
    probs, want = ensemble_full
    L.set_tuning(L.FP32_DEV, 5, 5, 8, 32)
    bt = L.Batch(probs, precision=L.FP32_DEV)
    if plan == "windows":
        bt.set_kernel(L.KERNEL_HALO, 8, 32)
    bt.set_phi(np.concatenate([p.phi0 for p in probs])).step(W.ENSEMBLE_STEPS)
    outs = bt.split(bt.read_phi())
    d = bt.diagnostics()
    bt.close()
    assert all(r["nonfinite"] == 0 for r in d)
    for i, w in want.items():
        assert normwise(outs[i], w) <= FP32_TOL(W.ENSEMBLE_STEPS), (i, probs[i].N)


def test_autotune_then_parity(L):
    """The autotuner's choice is a compiled configuration, and batches built after it (which
    use the tuned nodes per thread and window steps) still match the oracle."""
    K, T, rate = L.autotune(L.FP32_DEV, 5, 5)
    assert K in (2, 4, 8) and T in (16, 32, 64, 96, 128) and rate > 0
    K7, T7, _ = L.autotune(L.FP64, 7, 7)
    assert K7 == 4
    probs = [problem(W.kdv_burgers(2.0, 0.05, 0.9), N, 0.1, 1e-4, 1.3, 150, seed=N) for N in (300, 5000, 9001)]
    probs += [problem(W.kawahara(), N, 0.1, 1e-3, 2.5, 150, seed=N) for N in (700, 2500)]
    for P, tol in ((L.FP32_DEV, FP32_TOL(150)), (L.FP64, FP64_TOL)):
        bt = L.Batch(probs, precision=P)
        bt.set_phi(np.concatenate([p.phi0 for p in probs])).step(150)
        for p, got in zip(probs, bt.split(bt.read_phi())):
            assert normwise(got, oracle.run_problem(p)) <= tol, (P, p.N)
        bt.close()


def test_kernel_launch_count(L):
    """lbhpde_kernel_launches counts every kernel: graph replays count the kernels they hold."""
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        p = problem(W.kawahara(), 2049, 0.1, 1e-3, 2.5, 200, seed=21)
        s = L.Solver.for_problem(p, precision=L.FP32_DEV).set_kernel(L.KERNEL_STREAM)
        n0 = s.kernel_launches()
        s.set_phi(p.phi0).step(200)  # initialisation, then 3 replays of a 64-step graph + 8 launches
        assert s.kernel_launches() - n0 == 1 + 200
        s.read_phi()
        s.diagnostics()
        assert s.kernel_launches() - n0 == 1 + 200 + 1 + 2
        s.close()
        q = problem(W.kdv(), 400, 0.1, 2e-5, 1.07, 100)
        r = L.Solver.for_problem(q, precision=L.FP32_DEV).set_kernel(L.KERNEL_ONCHIP)
        m0 = r.kernel_launches()
        r.set_phi(q.phi0).step(100)  # initialisation and one resident launch
        assert r.kernel_launches() - m0 == 2
        r.close()


def test_stream_graph_replay_matches_single_launches(L):
    """On a non-default stream, long streaming runs replay a captured graph of 64 one-step
    launches; the result equals 200 individual launches bit for bit and matches the oracle."""
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        for P in (L.FP32_DEV, L.FP64):
            p = problem(W.kawahara(), 2049, 0.1, 1e-3, 2.5, 200, seed=21)
            a = L.Solver.for_problem(p, precision=P).set_kernel(L.KERNEL_STREAM)
            a.set_phi(p.phi0).step(200)  # 3 graph replays + 8 launches
            a.step(130)                  # graph for the other buffer parity
            ga = a.read_phi()
            b = L.Solver.for_problem(p, precision=P).set_kernel(L.KERNEL_STREAM)
            b.set_phi(p.phi0)
            for _ in range(330):
                b.step(1)
            gb = b.read_phi()
            a.close()
            b.close()
            assert np.array_equal(ga, gb)
            p2 = problem(W.kawahara(), 2049, 0.1, 1e-3, 2.5, 330, seed=21)
            tol = FP64_TOL if P == L.FP64 else FP32_TOL(330)
            assert normwise(ga, oracle.run_problem(p2)) <= tol

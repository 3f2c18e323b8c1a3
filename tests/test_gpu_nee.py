"""Bounded grids on the GPU (non-equilibrium extrapolation boundary of Sec. IV) against the
oracle, through the C ABI: the resident kernel (one CTA per instance), the streaming step with
the outer-node rebuild, batches that mix bounded and periodic members, and the printed errors of
Tables I, II, V, VI and VII.

Tolerances: FP64 normwise 1e-12 on problems whose perturbation growth over the run is below
~500 (measured with the oracle: a 1e-13 relative perturbation of phi0 grows to < 5e-11); the
table rows compare the global error E with the printed value at the golden file's tolerance.
FP32: the error against the exact solution stays within twice the FP64 path's.
"""
import os

import numpy as np
import pytest

import oracle
from paper_0907_1720_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
FP64_TOL = 1e-12
NOA = oracle.NO_AUX_CORRECTION


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


def bounded(example, dt, tau, nsteps, scheme=1, depth=2):
    p = W.bounded_config(example, dt, tau, nsteps * dt, scheme=scheme)
    p.meta["depth"] = depth
    return p


def oracle_run(p, nsteps=None):
    n = p.nsteps if nsteps is None else nsteps
    M = oracle.Model(p.eq.alpha, p.eq.pi, p.dx, p.dt, p.tau, lattice=p.eq.lattice, scheme=p.scheme)
    Wd = (M.b - 1) // 2
    f = M.init(p.phi0)
    M.step_nee(f, W.boundary_values(p, Wd, 0, n), p.meta.get("depth", 2))
    return M.phi(f)


def gpu_run(L, p, precision=0, kernel=0, chunks=None, device_phib=False):
    s = L.Solver.for_problem(p, precision=precision)
    s.set_kernel(kernel)
    s.set_phi(p.phi0)
    Wd = (s.model().b - 1) // 2
    done = 0
    for n in chunks or [p.nsteps]:
        pb = W.boundary_values(p, Wd, done, n)
        if device_phib:
            pb = torch.from_numpy(pb).cuda()
        s.step_nee(n, pb)
        done += n
    torch.cuda.synchronize()
    out = s.read_phi()
    s.close()
    return out


# (name, example, dt, tau, scheme, depth, steps): D1Q5 and D1Q7, both compile-time degree
# variants' lattices, depths 1-3, N up to 2001, runs longer than one resident launch
CASES = [
    ("ks_4.1_c100", "4.1", 1e-3, 1.989, 1 | NOA, 2, 1100),
    ("ks2_4.2_c10", "4.2", 1e-2, 4.569, 1 | NOA, 2, 600),
    ("kawahara_4.5_c1000_d1", "4.5", 1e-4, 2.02, 1, 1, 1100),
    ("mkawahara_4.6_s2_d3", "4.6", 1e-2, 4.04, 2, 3, 200),
    ("kdv_kawahara_4.7_c100", "4.7", 1e-3, 3.31, 1, 2, 1000),
    ("kdv_kawahara_4.7_c10", "4.7", 1e-2, 5.01, 1, 2, 100),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kernel", ["resident", "stream"])
def test_fp64_matches_oracle(L, case, kernel):
    name, ex, dt, tau, scheme, depth, n = case
    p = bounded(ex, dt, tau, n, scheme, depth)
    want = oracle_run(p)
    k = L.KERNEL_STREAM if kernel == "stream" else L.KERNEL_AUTO
    got = gpu_run(L, p, L.FP64, k, chunks=[n // 3, n - n // 3])
    assert normwise(got, want) <= FP64_TOL


def long_bounded_kawahara(n, N=3001):
    """Example 4.5's soliton on a bounded grid of N nodes (over the resident limit of 2048)."""
    dx, dt, tau = 0.1, 1e-4, 2.02
    xl = -0.5 * (N - 1) * dx
    x = W.grid(xl, N, dx)
    return W.Problem(W.kawahara(), N, dx, dt, tau, n, W.kawahara_soliton(x, 0.0), xl=xl,
                     exact=lambda t, x=x: W.kawahara_soliton(x, t), boundary="nee",
                     exact_xt=W.kawahara_soliton, meta={"depth": 1})


def test_grid_longer_than_one_cta_streams(L):
    """A bounded grid of 3001 nodes takes the streaming step plus the rebuild kernel."""
    p = long_bounded_kawahara(300)
    want = oracle_run(p)
    got = gpu_run(L, p, L.FP64)
    assert normwise(got, want) <= FP64_TOL


def test_device_boundary_values(L):
    p = bounded("4.1", 1e-3, 1.989, 300, 1 | NOA)
    want = oracle_run(p)
    got = gpu_run(L, p, L.FP64, device_phib=True, chunks=[100, 200])
    assert normwise(got, want) <= FP64_TOL


def _mixed_members():
    per = W.kawahara_config(N=600, dx=0.1, dt=1e-4, tau=2.02, t_end=0.0)
    per_long = W.kawahara_config(N=9000, dx=0.1, dt=1e-4, tau=2.02, t_end=0.0)
    return [
        bounded("4.1", 1e-3, 1.989, 0, 1 | NOA),
        per,
        bounded("4.7", 1e-3, 3.31, 0, 1),
        bounded("4.5", 1e-4, 2.02, 0, 1, depth=1),
        per_long,
        long_bounded_kawahara(0),
    ]


@pytest.mark.parametrize("kernel", ["auto", "stream", "halo"])
@pytest.mark.parametrize("nsteps", [257, 300])
def test_batch_mixes_bounded_and_periodic_members(L, kernel, nsteps):
    """Every member of a mixed batch equals its own oracle run, whichever kernels the members
    take and whichever buffer the step count ends in; member i's boundary values start at
    phib + i * stride."""
    probs = _mixed_members()
    for p in probs:
        p.nsteps = nsteps
    want = []
    for p in probs:
        if p.boundary == "nee":
            want.append(oracle_run(p))
        else:
            want.append(oracle.run_problem(p))
    b = L.Batch(probs, precision=L.FP64)
    b.set_kernel({"auto": L.KERNEL_AUTO, "stream": L.KERNEL_STREAM, "halo": L.KERNEL_HALO}[kernel])
    b.set_phi(np.concatenate([p.phi0 for p in probs]))
    stride = nsteps * 6 + 10
    phib = np.full(len(probs) * stride, np.nan)
    for i, p in enumerate(probs):
        if p.boundary == "nee":
            Wd = 2 if p.eq.lattice != 7 and p.eq.m <= 4 else 3
            blk = W.boundary_values(p, Wd, 0, nsteps).ravel()
            phib[i * stride: i * stride + blk.size] = blk
    b.step_nee(nsteps, phib, stride)
    got = b.read_phi()
    for i, p in enumerate(probs):
        seg = got[b.offsets[i]: b.offsets[i + 1]]
        assert normwise(seg, want[i]) <= FP64_TOL, (i, kernel)


def test_tau_sweep_shares_one_boundary_array(L):
    """Bounded members that differ only in tau share their boundary data (stride 0); each
    matches its own oracle run.  This is how a batch scans tau for the smallest error."""
    # tau >= 1.989: below it rounding grows fast (x5e6 at 1.97 over 500 steps; 1.95 diverges)
    taus = [1.989, 2.0, 2.05, 2.1, 2.2, 2.4]
    probs = [bounded("4.1", 1e-3, t, 500, 1 | NOA) for t in taus]
    b = L.Batch(probs, precision=L.FP64)
    b.set_phi(np.concatenate([p.phi0 for p in probs]))
    b.step_nee(500, W.boundary_values(probs[0], 2, 0, 500), 0)
    got = b.read_phi()
    for i, p in enumerate(probs):
        assert normwise(got[b.offsets[i]: b.offsets[i + 1]], oracle_run(p)) <= FP64_TOL


def _golden_rows():
    import test_oracle_nee as T
    return [r for r in T.nee_rows("pin") if r["c"] <= 100]


@pytest.mark.parametrize("row", _golden_rows(),
                         ids=lambda r: f"{r['table']}-s{r['scheme']}-c{int(r['c'])}-t{r['t']}")
def test_gpu_reproduces_printed_errors(L, row):
    """The FP64 GPU path reproduces the printed errors that the oracle reproduces."""
    p = bounded(row["example"], 0.1 / row["c"], row["tau"], int(round(row["t"] * row["c"] / 0.1)),
                row["scheme"] | (NOA if row["noA"] else 0), row["depth"])
    got = gpu_run(L, p, L.FP64)
    E = oracle.error_E(got, p.exact(p.t_end))
    assert E == pytest.approx(row["E"], rel=row["tol"])


@pytest.mark.parametrize("ex,dt,tau,scheme,n", [("4.1", 1e-3, 1.989, 1 | NOA, 1000), ("4.7", 1e-3, 3.31, 1, 1000)])
def test_fp32_bounded_accuracy(L, ex, dt, tau, scheme, n):
    """FP32 deviation storage on a bounded grid: error against the exact solution within twice
    the FP64 path's."""
    p = bounded(ex, dt, tau, n, scheme)
    e64 = oracle.error_E(gpu_run(L, p, L.FP64), p.exact(p.t_end))
    e32 = oracle.error_E(gpu_run(L, p, L.FP32_DEV), p.exact(p.t_end))
    assert e32 <= 2.0 * e64


def test_bounded_instance_needs_boundary_values(L):
    p = bounded("4.1", 1e-3, 1.989, 10, 1 | NOA)
    s = L.Solver.for_problem(p, precision=L.FP64)
    s.set_phi(p.phi0)
    with pytest.raises(L.LbhpdeError) as e:
        s.step(1)
    assert e.value.code == L.ERR_ARG
    with pytest.raises(L.LbhpdeError) as e:
        s.step_nee(1, None)
    assert e.value.code == L.ERR_ARG
    s.close()
    probs = [bounded("4.1", 1e-3, 1.989, 10, 1 | NOA), bounded("4.5", 1e-4, 2.02, 10)]
    b = L.Batch(probs, precision=L.FP64)
    b.set_phi(np.concatenate([p.phi0 for p in probs]))
    with pytest.raises(L.LbhpdeError) as e:  # shared array, but W differs (2 and 3)
        b.step_nee(10, np.zeros(10 * 6), 0)
    assert e.value.code == L.ERR_ARG
    with pytest.raises(L.LbhpdeError) as e:  # stride shorter than a member's block
        b.step_nee(10, np.zeros(200), 30)
    assert e.value.code == L.ERR_ARG


def test_tau_sweep_helper(L):
    """lbhpde.tau_sweep: E for every tau from one batch equals the oracle's E for that tau."""
    p = bounded("4.1", 1e-3, 2.0, 300, 1 | NOA)
    taus, E = L.tau_sweep(p, [1.989, 2.1, 2.3], precision=L.FP64)
    for t, e in zip(taus, E):
        q = bounded("4.1", 1e-3, float(t), 300, 1 | NOA)
        assert e == pytest.approx(oracle.error_E(oracle_run(q), q.exact(q.t_end)), rel=1e-9)


# ---------------------------------------------------------------- FP32: the 16-node kernel
EPS32 = 2.0 ** -24


def _growth(p, rel=1e-6, seed=0):
    """Growth of a relative perturbation of phi0 over p's steps, measured with the oracle: the
    factor by which the scheme amplifies errors made along the way on this problem."""
    rng = np.random.default_rng(seed)
    a = oracle_run(p)
    q = W.Problem(p.eq, p.N, p.dx, p.dt, p.tau, p.nsteps, p.phi0 * (1 + rel * rng.standard_normal(p.N)),
                  xl=p.xl, scheme=p.scheme, boundary=p.boundary, exact=p.exact, exact_xt=p.exact_xt, meta=p.meta)
    b = oracle_run(q)
    return normwise(b, a) / rel


def fp32_bound(p):
    """The FP32 parity bound of the periodic tests, 16 eps32 sqrt(n) + 4 eps32 (one rounding of
    phi and of the stored deviations a step, added like a random walk, plus the initial
    rounding), times the perturbation growth G >= 1 the oracle measures on the problem."""
    return (16 * EPS32 * np.sqrt(p.nsteps) + 4 * EPS32) * max(1.0, _growth(p))


# (name, example, dt, tau, scheme, depth, steps, dx): D1Q5, depths 1-4 and 20 (x_f in the second
# thread of 16 nodes), grids of 484, 486, 501, 601 and 1001 nodes, tau at the paper's tau_opt (growth ~30)
# and above it (growth < 1)
FP32_CASES = [
    ("ks_4.1_tauopt", "4.1", 1e-3, 1.989, 1 | NOA, 2, 1100, 0.1),
    ("ks2_4.2_tauopt", "4.2", 1e-2, 4.569, 1 | NOA, 2, 600, 0.1),
    ("ks_4.1_d1", "4.1", 1e-3, 2.05, 1 | NOA, 1, 600, 0.1),
    ("ks_4.1_d3", "4.1", 1e-3, 2.05, 1 | NOA, 3, 600, 0.1),
    ("ks_4.1_d4", "4.1", 1e-3, 2.05, 1 | NOA, 4, 600, 0.1),
    ("ks_4.1_d20", "4.1", 1e-3, 2.1, 1 | NOA, 20, 400, 0.1),
    ("ks_4.1_N501", "4.1", 1.2e-3, 2.05, 1 | NOA, 2, 500, 0.12),
    # 16 r + 2 and 16 r interior nodes: the right end's x_f at the first and the last position
    # where the depth-2 variant of the 16-node kernel finds it in the last thread
    ("ks_4.1_N486", "4.1", 1.2e-3, 2.05, 1 | NOA, 2, 500, 60.0 / 485),
    ("ks_4.1_N484", "4.1", 1.2e-3, 2.05, 1 | NOA, 2, 500, 60.0 / 483),
]


def _bounded_dx(ex, dt, tau, n, scheme, depth, dx):
    p = W.bounded_config(ex, dt, tau, n * dt, scheme=scheme, dx=dx)
    p.meta["depth"] = depth
    return p


@pytest.mark.parametrize("case", FP32_CASES, ids=[c[0] for c in FP32_CASES])
@pytest.mark.parametrize("kernel", ["auto", "resident4", "stream"])
def test_fp32_matches_oracle(L, case, kernel):
    """FP32 deviation storage on bounded grids, each kernel: the 16-node resident kernel (the
    automatic choice for FP32 D1Q5), the one-instance-per-CTA kernel at 4 nodes a thread, and the
    streaming step with the rebuild; launches split in two to cover the step offset of the
    boundary rows.  Bound: fp32_bound."""
    name, ex, dt, tau, scheme, depth, n, dx = case
    p = _bounded_dx(ex, dt, tau, n, scheme, depth, dx)
    want = oracle_run(p)
    s = L.Solver.for_problem(p, precision=L.FP32_DEV)
    if kernel == "resident4":
        s.set_kernel(L.KERNEL_ONCHIP, 4)
    elif kernel == "stream":
        s.set_kernel(L.KERNEL_STREAM)
    s.set_phi(p.phi0)
    done = 0
    for m in (n // 3, n - n // 3):
        s.step_nee(m, W.boundary_values(p, 2, done, m))
        done += m
    got = s.read_phi()
    s.close()
    assert normwise(got, want) <= fp32_bound(p), kernel


def test_fp32_bounded_batch_matches_alone_bitwise(L):
    """Bounded FP32 members of different grids and depths packed into shared CTAs of the 16-node
    kernel give the same bits as each alone, and each matches its oracle run."""
    cases = [c for c in FP32_CASES if c[0] != "ks2_4.2_tauopt"]
    probs = [_bounded_dx(ex, dt, tau, 300, scheme, depth, dx) for _, ex, dt, tau, scheme, depth, _, dx in cases]
    stride = 300 * 4
    phib = np.concatenate([W.boundary_values(p, 2, 0, 300).ravel() for p in probs])
    b = L.Batch(probs, precision=L.FP32_DEV)
    b.set_phi(np.concatenate([p.phi0 for p in probs])).step_nee(300, phib, stride)
    got = b.read_phi()
    b.close()
    for i, p in enumerate(probs):
        s = L.Solver.for_problem(p, precision=L.FP32_DEV)
        alone = s.set_phi(p.phi0).step_nee(300, W.boundary_values(p, 2, 0, 300)).read_phi()
        s.close()
        seg = got[b.offsets[i]: b.offsets[i + 1]]
        assert np.array_equal(seg, alone), (i, p.N, p.meta["depth"])
        assert normwise(seg, oracle_run(p)) <= fp32_bound(p)


@pytest.mark.parametrize("depths", [(2,), (1, 2, 3)], ids=["depth2", "mixed_depths"])
def test_fp32_tiny_bounded_grids_share_ctas(L, depths):
    """Bounded FP32 grids of 8 to 100 nodes (one or a few threads of the 16-node kernel, many
    instances a CTA: more helper roles than interior threads), 100 steps: each member matches its
    oracle run within fp32_bound and equals, bit for bit, the same member solved alone."""
    sizes = (8, 9, 12, 20, 21, 37, 100)
    probs = []
    for i, n in enumerate(sizes * 3):
        p = W.bounded_config("4.1", 1e-3, 2.05 + 0.01 * i, 0.1, scheme=1 | NOA, dx=60.0 / (n - 1))
        p.meta["depth"] = depths[i % len(depths)]
        if p.N < 2 * (2 + p.meta["depth"]):
            p.meta["depth"] = 2
        probs.append(p)
    steps = probs[0].nsteps
    phib = np.concatenate([W.boundary_values(p, 2, 0, steps).ravel() for p in probs])
    b = L.Batch(probs, precision=L.FP32_DEV)
    b.set_phi(np.concatenate([p.phi0 for p in probs])).step_nee(steps, phib, steps * 4)
    got = b.read_phi()
    b.close()
    for i, p in enumerate(probs):
        seg = got[b.offsets[i]: b.offsets[i + 1]]
        s = L.Solver.for_problem(p, precision=L.FP32_DEV)
        alone = s.set_phi(p.phi0).step_nee(steps, W.boundary_values(p, 2, 0, steps)).read_phi()
        s.close()
        assert np.array_equal(seg, alone), (i, p.N, p.meta["depth"])
        assert normwise(seg, oracle_run(p)) <= fp32_bound(p), (i, p.N, p.meta["depth"])

"""Full-size runs of the small configurations and the FP32 accuracy bar.

* KdV soliton (N = 400, 50 000 steps) and Kuramoto-Sivashinsky (N = 1024, 100 000 steps):
  the FP64 GPU path matches the oracle element by element (1e-12 normwise) at full size.
* The FP32 deviation-storage path stays within twice the FP64 path's error against the
  exact solution (KdV soliton, Kawahara Table V case) or the spectral ETDRK4 reference (KS).
"""
import math

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


def run(L, p, precision, kernel=None):
    s = L.Solver.for_problem(p, precision=precision)
    if kernel is not None:
        s.set_kernel(kernel)
    s.set_phi(p.phi0).step(p.nsteps)
    out = s.read_phi()
    s.close()
    return out


def err_E(phi, ref):
    return float(np.abs(phi - ref).sum() / np.abs(ref).sum())


@pytest.fixture(scope="module")
def kdv(L):
    p = W.kdv_config()
    return p, oracle.run_problem(p)


@pytest.fixture(scope="module")
def ks(L):
    p = W.ks_config()
    return p, oracle.run_problem(p), W.ks_spectral_reference(t_end=p.t_end)


@pytest.mark.parametrize("kernel", ["auto", "stream"])
def test_kdv_config_full_size_fp64_parity(L, kdv, kernel):
    p, want = kdv
    got = run(L, p, L.FP64, None if kernel == "auto" else L.KERNEL_STREAM)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_kdv_config_fp32_within_twice_fp64_error(L, kdv):
    p, want = kdv
    ex = p.exact(p.t_end)
    e64 = err_E(run(L, p, L.FP64), ex)
    e32 = err_E(run(L, p, L.FP32_DEV), ex)
    assert e64 == pytest.approx(err_E(want, ex), rel=1e-9)
    assert e32 <= 2.0 * e64


def test_ks_config_full_size_fp64_parity(L, ks):
    p, want, _ = ks
    got = run(L, p, L.FP64)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_ks_config_fp32_within_twice_fp64_error(L, ks):
    p, want, ref = ks
    e64 = err_E(run(L, p, L.FP64), ref)
    e32 = err_E(run(L, p, L.FP32_DEV), ref)
    assert e32 <= 2.0 * e64


@pytest.mark.parametrize("dt,tau,E_paper", [(1e-3, 2.53, 2.6928e-3), (1e-4, 2.02, 1.5361e-3)])
def test_kawahara_table_v_on_gpu(L, dt, tau, E_paper):
    """Table V (Example 4.5, scheme 1, t = 1) on the GPU: FP64 reproduces the printed error and
    FP32 stays within twice the FP64 error."""
    p = W.kawahara_config(N=600, dx=0.1, dt=dt, tau=tau, t_end=1.0)
    ex = p.exact(p.t_end)
    e64 = err_E(run(L, p, L.FP64), ex)
    e32 = err_E(run(L, p, L.FP32_DEV), ex)
    assert e64 == pytest.approx(E_paper, rel=3e-4)
    assert e32 <= 2.0 * e64


def test_observed_order_on_the_gpu(L):
    """The joint refinement of the oracle test (dt = 1e-2 dx^3, tau = 1.1, KdV soliton, t = 0.1)
    on the GPU (FP64, resident kernel): E at dx = 0.1 and 0.05 equals the oracle's and gives the
    same order (> 1.7).  One level further (dx = 0.025, c = 1.6e5, 640 000 steps) the scheme
    itself amplifies a 1e-13 perturbation 8e10-fold in the oracle, so that level measures
    rounding, not the method, and is left out."""
    from test_oracle_pins import kdv_refinement_error
    Es = {}
    for dx in (0.1, 0.05):
        N = int(round(40.0 / dx))
        dt = 1e-2 * dx ** 3
        n = int(round(0.1 / dt))
        x = W.grid(-20.0, N, dx)
        p = W.Problem(W.kdv(), N, dx, dt, 1.1, n, W.kdv_soliton(x, 0.0, L=40.0), xl=-20.0)
        s = L.Solver.for_problem(p, precision=L.FP64)
        phi = s.set_phi(p.phi0).step(n).read_phi()
        s.close()
        Es[dx] = oracle.error_E(phi, W.kdv_soliton(x, n * dt, L=40.0))
        assert Es[dx] == pytest.approx(kdv_refinement_error(dx), rel=1e-9)
    assert math.log2(Es[0.1] / Es[0.05]) > 1.7, Es

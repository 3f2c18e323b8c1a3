"""The diagnostics entry point that allocates nothing (lbhpde_phi_diagnostics_noalloc).

Some callers cannot let a library allocate device memory: applications that hand all of
the GPU's memory to their own pool up front, or latency-critical loops where the
device-wide synchronisation of cudaMalloc/cudaFree is not acceptable.  For them the
library offers a diagnostics reduction whose scratch is a file-scope device array.

This test calls it through the C ABI on a phi array the test owns and checks its result
against lbhpde_diagnostics of the same solver, with the tolerance of the FP64 parity tests,
on two calls in a row (the shared scratch array must not carry anything over).  The file
is named so that pytest collects it last; it must also pass when run alone.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-12  # the FP64 parity tolerance


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0907_1720_gb300 import build as B
    B.build()
    from paper_0907_1720_gb300 import lbhpde
    lbhpde.lib()
    return lbhpde


def _noalloc(L, phi_dev, phistar_dev, stream):
    d = L.lbhpde_diag()
    rc = L.lib().lbhpde_phi_diagnostics_noalloc(ctypes.c_void_p(phi_dev.data_ptr()), phi_dev.numel(),
                                                ctypes.c_void_p(phistar_dev.data_ptr()) if phistar_dev is not None
                                                else None, ctypes.byref(d), ctypes.c_void_p(stream))
    return rc, d.as_dict()


def _close(a, b):
    for k in ("sum_phi", "max_abs_phi", "err_E", "err_L2"):
        assert abs(a[k] - b[k]) <= TOL * max(abs(b[k]), 1e-300), (k, a[k], b[k])
    assert a["nonfinite"] == b["nonfinite"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_matches_diagnostics_twice(L, precision):
    from paper_0907_1720_gb300 import workloads as W

    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        p = W.kawahara_config(N=3000, dt=1e-3, tau=2.53, t_end=0.2)
        prec = L.FP32_DEV if precision == "fp32" else L.FP64
        s = L.Solver.for_problem(p, precision=prec)
        s.set_phi(p.phi0)
        phi = torch.empty(p.N, dtype=torch.float64, device="cuda")
        for call in range(2):
            s.step(p.nsteps // 2)
            t = (call + 1) * (p.nsteps // 2) * p.dt
            ex = torch.tensor(p.exact(t), dtype=torch.float64, device="cuda")
            want = s.diagnostics(ex)
            s.read_phi(phi)
            rc, got = _noalloc(L, phi, ex, st.cuda_stream)
            assert rc == L.OK
            _close(got, want)
            rc, got0 = _noalloc(L, phi, None, st.cuda_stream)
            assert rc == L.OK and got0["err_E"] == 0.0
            assert abs(got0["sum_phi"] - want["sum_phi"]) <= TOL * abs(want["sum_phi"])
        s.close()


def test_noalloc_rejects_oversize_and_reports_nonfinite(L):
    st = torch.cuda.Stream()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    d = L.lbhpde_diag()
    lim = 16777216
    assert L.lib().lbhpde_phi_diagnostics_noalloc(ctypes.c_void_p(x.data_ptr()), lim + 1, None, ctypes.byref(d),
                                                  ctypes.c_void_p(st.cuda_stream)) == L.ERR_ARG
    assert L.lib().lbhpde_phi_diagnostics_noalloc(None, 4, None, ctypes.byref(d),
                                                  ctypes.c_void_p(st.cuda_stream)) == L.ERR_ARG
    y = torch.tensor([1.0, float("nan"), 2.0, 3.0], dtype=torch.float64, device="cuda")
    rc, got = _noalloc(L, y, None, st.cuda_stream)
    assert rc == L.ERR_DIVERGED and got["nonfinite"] == 1 and got["sum_phi"] == 6.0

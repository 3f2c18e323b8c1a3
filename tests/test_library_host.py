"""Host-side checks of the CUDA library that need no GPU.

* the shared library builds here (nvcc cross-compiles for sm_103a) and exports every entry
  point that include/lbhpde.h declares, with the binding naming the same set;
* step a0 (lbhpde_model, pure host code) agrees with the oracle: tau_k, beta_k, A_k0,
  the inexact-recovery flag and f^eq_j(phi) at random phi;
* the library's set-up, on its own, satisfies the dispersion pin of the oracle tests;
* argument validation returns the documented status codes.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_0907_1720_gb300 import build as B
from paper_0907_1720_gb300 import lbhpde as L
from paper_0907_1720_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbhpde.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbhpde_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(L.EXPORTED) == names


EQUATIONS = [
    ("kdv", W.kdv(), 1e-4, 1.3, 1),
    ("kdv_s2", W.kdv(), 1e-4, 1.3, 2),
    ("mkdv", W.mkdv(), 1e-4, 1.2, 1),
    ("kdv_burgers", W.kdv_burgers(3.0, 0.07, 0.8), 1e-4, 1.15, 1),
    ("k22", W.k22(), 1e-3, 1.6, 1),
    ("ks", W.ks(), 1e-4, 1.3, 1),
    ("gks_cubic_q7", W.gks_cubic(lattice=7), 1e-3, 1.4, 1),
    ("kawahara", W.kawahara(), 1e-4, 2.02, 1),
    ("kawahara_s2", W.kawahara(), 1e-3, 2.55, 2),
    ("modified_kawahara", W.modified_kawahara(), 1e-2, 4.54, 1),
    ("kdv_kawahara", W.kdv_kawahara(), 1e-3, 3.31, 1),
    ("sixth", W.Equation("sixth", (1.0, 0.0, 0.5, 0.3, -1.0, 0.2),
                         ((0, 0, 0.5), (), (0, 1), (0, 1), (0, 1), (0, 1))), 1e-3, 2.2, 1),
    # A_40, A_50, A_60 left out (LBHPDE_NO_AUX_CORRECTION)
    ("ks_noA", W.ks(), 1e-2, 5.99, 1 | 0x100),
    ("kdv_burgers_noA", W.kdv_burgers(3.0, 0.07, 0.8), 1e-4, 1.15, 1 | 0x100),
    ("kawahara_noA", W.kawahara(), 1e-4, 2.02, 1 | 0x100),
]


@pytest.mark.parametrize("name,eq,dt,tau,scheme", EQUATIONS, ids=[e[0] for e in EQUATIONS])
def test_model_matches_oracle(lib, name, eq, dt, tau, scheme):
    info = L.lbhpde_model(eq.alpha, eq.pi, 0.1, dt, tau, lattice=eq.lattice, scheme=scheme)
    M = oracle.Model(eq.alpha, eq.pi, 0.1, dt, tau, lattice=eq.lattice, scheme=scheme)
    assert info.b == M.b
    assert bool(info.inexact) == M.inexact
    assert np.allclose(list(info.tk)[2:], M.taus[2:], rtol=1e-14, atol=0)
    assert np.allclose(list(info.beta), M.beta, rtol=1e-13, atol=0)
    assert np.allclose(list(info.A), M.A, rtol=1e-12, atol=0)
    feq, coef = L.model_coeffs(info)
    rng = np.random.default_rng(3)
    for phi in np.concatenate([rng.uniform(-1.5, 1.5, 20), [0.0, 1.0, -1.0]]):
        want = M.feq(phi)
        got = np.polynomial.polynomial.polyval(phi, feq.T)
        scale = np.abs(want).max() + 1e-300
        assert np.abs(got - want).max() <= 1e-13 * scale + 1e-300, phi
        assert np.allclose(coef, feq / tau, rtol=1e-15, atol=0)


@pytest.mark.parametrize("case", [c for c in __import__("test_oracle_pins").DISPERSION_CASES],
                         ids=[c[0] for c in __import__("test_oracle_pins").DISPERSION_CASES])
def test_model_dispersion_pin(lib, case):
    """The library's own a0 set-up passes the recovered-equation pin (Eqs. (NPDE3)-(NPDE6))."""
    from test_oracle_pins import E7, expected_dispersion
    name, eq, dx, dt, tau, scheme, phibar, n_exact = case
    info = L.lbhpde_model(eq.alpha, eq.pi, dx, dt, tau, lattice=eq.lattice, scheme=scheme)
    feq, _ = L.model_coeffs(info)
    b = info.b
    dfeq = np.array([np.polynomial.polynomial.polyval(phibar, np.polynomial.polynomial.polyder(feq[j]))
                     for j in range(b)])
    w = 1.0 / tau
    C = (1 - w) * np.eye(b) + w * np.outer(dfeq, np.ones(b))
    r, Q = 1.0, 128
    th = 2 * np.pi * np.arange(Q) / Q
    g = []
    for q in range(Q):
        kap = r * np.exp(1j * th[q])
        ev = np.linalg.eigvals(np.diag(np.exp(-1j * kap * E7[:b] * dx)) @ C)
        g.append(np.log(ev[np.argmin(np.abs(ev - 1))]) / dt)
    g = np.array(g)
    a = np.array([np.mean(g * np.exp(-1j * n * th)) / r ** n for n in range(n_exact + 1)])
    want = expected_dispersion(eq.alpha, eq.pi, phibar, n_exact)
    assert np.all(np.abs(a - want) <= 1e-7 * (1 + np.abs(want)))


def _pis(pi):
    return (L.lbhpde_pi * len(pi))(*[L.make_pi(r) for r in pi])


def test_model_argument_errors(lib):
    eq = W.kdv_burgers(1.0, 0.05, 1.0)
    info = L.lbhpde_model_info()
    a = (ctypes.c_double * 3)(*eq.alpha)
    P = _pis(eq.pi)
    f = lib.lbhpde_model
    assert f(3, a, P, 0.1, 1e-3, 1.3, 0, 1, ctypes.byref(info)) == L.OK
    assert f(0, a, P, 0.1, 1e-3, 1.3, 0, 1, ctypes.byref(info)) == L.ERR_ARG
    assert f(7, a, P, 0.1, 1e-3, 1.3, 0, 1, ctypes.byref(info)) == L.ERR_ARG
    assert f(3, a, P, -0.1, 1e-3, 1.3, 0, 1, ctypes.byref(info)) == L.ERR_ARG
    assert f(3, a, P, 0.1, float("nan"), 1.3, 0, 1, ctypes.byref(info)) == L.ERR_ARG
    assert f(3, a, P, 0.1, 1e-3, 1.3, 6, 1, ctypes.byref(info)) == L.ERR_ARG
    assert f(3, a, P, 0.1, 1e-3, 1.3, 0, 3, ctypes.byref(info)) == L.ERR_ARG
    assert f(3, a, P, 0.1, 1e-3, 0.5, 0, 1, ctypes.byref(info)) == L.ERR_TAU_SINGULAR
    assert f(3, a, P, 0.1, 1e-3, 0.5 + 3 ** 0.5 / 6, 0, 1, ctypes.byref(info)) == L.ERR_TAU_SINGULAR
    ks = W.ks()
    a4 = (ctypes.c_double * 4)(*ks.alpha)
    assert f(4, a4, _pis(ks.pi), 0.1, 1e-3, 1.3, 0, 2, ctypes.byref(info)) == L.ERR_ARG  # scheme 2 needs m < b-1
    assert f(3, a, P, 0.1, 1e-3, 1.3, 0, 1, None) == L.ERR_ARG
    bad = L.lbhpde_pi()
    bad.kind = 9
    P2 = (L.lbhpde_pi * 3)(P[0], bad, P[2])
    assert f(3, a, P2, 0.1, 1e-3, 1.3, 0, 1, ctypes.byref(info)) == L.ERR_ARG


def test_degree_limit(lib):
    """f^eq degree above 31 is rejected: Pi_1 = phi^7 on D1Q7 gives degree 6*6+1 = 37."""
    eq = W.Equation("deg", (1.0, 0.0, 1.0, 0.0, 1.0), ((0,) * 7 + (1.0,), (), (0, 1), (), (0, 1)), lattice=7)
    with pytest.raises(L.LbhpdeError) as ei:
        L.lbhpde_model(eq.alpha, eq.pi, 0.1, 1e-3, 2.0, lattice=7)
    assert ei.value.code == L.ERR_ARG


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    eq = W.kdv()
    a = (ctypes.c_double * 3)(*eq.alpha)
    P = _pis(eq.pi)
    h = ctypes.c_void_p()
    assert lib.lbhpde_create(None, 3, a, P, 100, 0.1, 1e-3, 1.3, 0, 1, L.FP64, 0, None, None) == L.ERR_ARG
    # unknown boundary kind; bounded grid too short for the extrapolation node; periodic with a
    # depth; negative code: all rejected before any device memory is touched
    assert lib.lbhpde_create(ctypes.byref(h), 3, a, P, 100, 0.1, 1e-3, 1.3, 0, 1, L.FP64, 2, None, None) == \
        L.ERR_UNSUPPORTED
    assert lib.lbhpde_create(ctypes.byref(h), 3, a, P, 7, 0.1, 1e-3, 1.3, 0, 1, L.FP64, L.NEE, None, None) == \
        L.ERR_ARG
    assert lib.lbhpde_create(ctypes.byref(h), 3, a, P, 100, 0.1, 1e-3, 1.3, 0, 1, L.FP64, L.nee_depth(49),
                             None, None) == L.ERR_ARG
    assert lib.lbhpde_create(ctypes.byref(h), 3, a, P, 100, 0.1, 1e-3, 1.3, 0, 1, L.FP64, 1 << 8, None, None) == \
        L.ERR_ARG
    assert lib.lbhpde_create(ctypes.byref(h), 3, a, P, 100, 0.1, 1e-3, 1.3, 0, 1, L.FP64, -1, None, None) == \
        L.ERR_ARG
    assert lib.lbhpde_step_nee(None, 1, None, 0) == L.ERR_ARG
    assert lib.lbhpde_batch_step_nee(None, 1, None, 0, 0) == L.ERR_ARG
    assert lib.lbhpde_step(None, 1) == L.ERR_ARG
    assert lib.lbhpde_destroy(None) == L.ERR_ARG
    assert lib.lbhpde_strerror(L.ERR_DIVERGED).decode().startswith("non-finite")


NU_EQUATIONS = [
    # (name, equation, dt, tau): class (1) with a real exponent n on D1Q5 and D1Q7
    ("gkdv_1.5", W.gkdv(1.5), 1e-4, 1.3),
    ("gkdv_0.5", W.gkdv(0.5), 1e-4, 1.3),
    ("ks_real", W.class1_real(1.0, 0.6, 2.3, (1.0, 0.0, 1.0)), 1e-4, 1.3),
    ("kawahara_real", W.class1_real(1.0, -0.4, 1.7, (0.0, 1.0, 0.0, -1.0)), 1e-4, 2.02),
    ("sixth_real", W.class1_real(0.5, 0.3, 0.8, (0.2, 0.5, 0.3, -1.0, 0.2)), 1e-3, 2.2),
]


@pytest.mark.parametrize("name,eq,dt,tau", NU_EQUATIONS, ids=[e[0] for e in NU_EQUATIONS])
def test_real_exponent_model_matches_oracle(lib, name, eq, dt, tau):
    """The library's generalised f^eq tables (sum_a (phi^nu)^a sum_i g[j][a][i] phi^i) against
    the oracle's f^eq at positive phi, and zero real-exponent terms at phi <= 0."""
    info = L.lbhpde_model(eq.alpha, eq.pi, 0.1, dt, tau, lattice=eq.lattice, nu=eq.nu, pi_nu=eq.pi_nu)
    M = oracle.Model(eq.alpha, eq.pi, 0.1, dt, tau, lattice=eq.lattice, nu=eq.nu, pi_nu=eq.pi_nu)
    assert info.b == M.b and info.nu_rows > 1 and info.nu == eq.nu
    assert bool(info.inexact) == M.inexact
    assert np.allclose(list(info.beta), M.beta, rtol=1e-13, atol=0)
    assert np.allclose(list(info.A), M.A, rtol=1e-12, atol=0)
    g, gc = L.model_coeffs(info)
    assert np.allclose(gc, g / tau, rtol=1e-15, atol=0)
    rng = np.random.default_rng(5)
    for phi in np.concatenate([rng.uniform(0.01, 2.0, 16), [1.0, -0.3, 0.0]]):
        w = phi ** eq.nu if phi > 0 else 0.0
        got = np.array([sum(w ** a * np.polynomial.polynomial.polyval(phi, g[j, a]) for a in range(g.shape[1]))
                        for j in range(info.b)])
        want = M.feq(phi)
        assert np.abs(got - want).max() <= 1e-12 * (np.abs(want).max() + 1e-300), phi


def test_real_exponent_argument_errors(lib):
    eq = W.gkdv(1.5)
    bad_nu = [L.make_pi(eq.pi[0], -1.0, eq.pi_nu[0])] + [L.make_pi(r) for r in eq.pi[1:]]
    a = (ctypes.c_double * 3)(*eq.alpha)
    info = L.lbhpde_model_info()
    P = (L.lbhpde_pi * 3)(*bad_nu)
    assert lib.lbhpde_model(3, a, P, 0.1, 1e-4, 1.3, 0, 1, ctypes.byref(info)) == L.ERR_ARG
    p0 = L.make_pi((0.0, 0.0, 0.5), 1.5, (0.0, 1.0))
    p0.coef_nu[0] = 1.0  # a phi^nu term with no derivative of the form
    P = (L.lbhpde_pi * 3)(p0, L.make_pi(eq.pi[1]), L.make_pi(eq.pi[2]))
    assert lib.lbhpde_model(3, a, P, 0.1, 1e-4, 1.3, 0, 1, ctypes.byref(info)) == L.ERR_ARG
    # two different real exponents in one equation
    P = (L.lbhpde_pi * 3)(L.make_pi((0, 0, 0.5), 1.5, (0, 1.0)), L.make_pi((0, 1.0)),
                          L.make_pi((0, 0.0), 2.5, (0, 1.0)))
    assert lib.lbhpde_model(3, a, P, 0.1, 1e-4, 1.3, 0, 1, ctypes.byref(info)) == L.ERR_ARG


def test_set_tuning_argument_checks(lib):
    """lbhpde_set_tuning records a pair on the host only; it rejects what the autotuner would
    never choose."""
    f = lib.lbhpde_set_tuning
    assert f(7, 5, 5, 8, 128) == L.ERR_ARG             # precision
    assert f(L.FP32_DEV, 6, 5, 8, 128) == L.ERR_ARG     # lattice
    assert f(L.FP32_DEV, 5, 0, 8, 128) == L.ERR_ARG     # degree
    assert f(L.FP32_DEV, 5, 5, 8, 0) == L.ERR_ARG       # steps per window
    assert f(L.FP32_DEV, 5, 5, 3, 128) == L.ERR_UNSUPPORTED   # not a compiled width
    assert f(L.FP64, 7, 7, 8, 16) == L.ERR_UNSUPPORTED        # FP64 D1Q7 has K = 4 only
    assert f(L.FP32_DEV, 5, 5, 8, 600) == L.ERR_UNSUPPORTED   # halo 2400 nodes: more than half a window
    # a run-time-degree FP64 D1Q7 pair (valid for every model of that class)
    assert f(L.FP64, 7, 9, 4, 16) == L.OK

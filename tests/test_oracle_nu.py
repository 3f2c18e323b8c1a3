"""Pins of the oracle's real-exponent terms: equations of class (1) of Sec. III C,
u_t + a u u_x + b u^n u_x + sum_k alpha_k d_x^k u = 0, with a real n > 0, so that
Pi_1 = a u^2 / 2 + b u^(n+1) / (n+1) and the auxiliary moments carry powers u^(i + j n).

Pins: the closed forms the paper prints for this class (Eq. (Pi30t60) with Eq. (intPi1k), and
Eq. (3Pi20t40) for class (2)), which hold for real n; the recovered-equation (dispersion) pin at
a positive base state; a whole-number exponent against the ordinary polynomial model; the
generalised-KdV solitary wave; planted mistakes in the generalised algebra.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_0907_1720_gb300 import workloads as W

from test_oracle_pins import _int_pi1k, dispersion_coeffs


def _model(eq, dx=0.1, dt=1e-3, tau=1.7, lattice=None, scheme=1, lib=None):
    return oracle.Model(eq.alpha, eq.pi, dx, dt, tau, lattice=eq.lattice if lattice is None else lattice,
                        scheme=scheme, lib=lib, nu=eq.nu, pi_nu=eq.pi_nu)


def class1_error(seed, lib=None):
    """Largest relative deviation of Pi_20..Pi_60 from Eq. (Pi30t60) + Eq. (intPi1k)."""
    rng = np.random.default_rng(300 + seed)
    a, bb = rng.uniform(-2, 2), rng.uniform(-2, 2)
    n = float(rng.uniform(0.2, 3.5))
    al = rng.uniform(0.2, 1.0, size=5) * rng.choice([-1, 1], size=5)
    eq = W.class1_real(a, bb, n, tuple(al), lattice=7)
    M = _model(eq, lattice=7, lib=lib)
    be, (A40, A50, A60) = M.beta, M.A
    worst = 0.0
    for u in rng.uniform(0.05, 1.5, size=6):
        P1 = a / 2 * u ** 2 + bb / (n + 1) * u ** (n + 1)
        I = {k: _int_pi1k(u, a, bb, n, k) for k in range(2, 7)}
        want = {
            2: I[2],
            3: I[3] + 3 * be[2] * P1,
            4: I[4] + 6 * be[2] * I[2] + 4 * be[3] * P1 + A40 * u,
            5: I[5] + 10 * be[2] * I[3] + 10 * be[3] * I[2] + 5 * be[4] * P1 + A50 * u,
            6: I[6] + 15 * be[2] * I[4] + 20 * be[3] * I[3] + 15 * be[4] * I[2] + 6 * be[5] * P1 + A60 * u,
        }
        for k in range(2, 7):
            scale = max(abs(want[k]), abs(I[k]), 1e-300) + abs(A60 * u) + 1e-12
            worst = max(worst, abs(M.aux_moment(k, u) - want[k]) / scale)
    return worst


@pytest.mark.parametrize("seed", range(6))
def test_class1_real_exponent_closed_forms(seed):
    """Eq. (Pi30t60) with Eq. (intPi1k) for a real n: every auxiliary moment Pi_20..Pi_60."""
    assert class1_error(seed) <= 1e-12


@pytest.mark.parametrize("seed", range(4))
def test_class2_real_exponent_closed_forms(seed):
    """Eq. (3Pi20t40): u_t + a u u_x + b u^n u_x + alpha_2 (u^p)_xx + alpha_3 (u^q)_xxx = 0 with a
    real n and whole p, q (D1Q5)."""
    rng = np.random.default_rng(400 + seed)
    a, bb = rng.uniform(-2, 2), rng.uniform(-2, 2)
    n, p, q = float(rng.uniform(0.2, 3.5)), int(rng.integers(1, 4)), int(rng.integers(1, 4))
    a2, a3 = rng.uniform(0.1, 0.5), rng.uniform(0.5, 1.0)
    pi1 = (0.0, 0.0, a / 2.0)
    eq = W.Equation("class2_real", (1.0, a2, a3), (pi1, (0.0,) * p + (1.0,), (0.0,) * q + (1.0,)), 5, n,
                    ((0.0, bb / (n + 1)), (), ()))
    M = _model(eq, dt=1e-3, tau=1.3, lattice=5)
    be, A40 = M.beta, M.A[0]
    for u in rng.uniform(0.05, 1.5, size=6):
        I2, I3, I4 = (_int_pi1k(u, a, bb, n, k) for k in (2, 3, 4))
        want = {
            2: I2,
            3: I3 + 3 * be[2] * p * u ** p * (a * u / (p + 1) + bb * u ** n / (p + n)),
            4: I4 + 6 * be[2] * p * u ** p * ((a * u) ** 2 / (p + 2) + 2 * a * u * bb * u ** n / (p + n + 1)
                                              + (bb * u ** n) ** 2 / (p + 2 * n))
            + 4 * be[3] * q * u ** q * (a * u / (q + 1) + bb * u ** n / (q + n)) + A40 * u,
        }
        for k in (2, 3, 4):
            assert M.aux_moment(k, u) == pytest.approx(want[k], rel=1e-12, abs=1e-12 * (abs(I2) + 1)), (k, u)


def dispersion_error(n, lattice, lib=None):
    """Largest deviation of the Taylor coefficients of log(lambda)/dt from the recovered
    equation's -sum_k alpha_k Pi_k'(phibar) (i kappa)^k, through kappa^m."""
    a, bb, phibar = 0.8, 1.3, 0.6
    if lattice == 5:
        eq = W.class1_real(a, bb, n, (0.05, 0.7, 0.2), lattice=5)  # KdV-Burgers-KS with u^n u_x
        tau = 1.3
    else:
        eq = W.class1_real(a, bb, n, (0.0, 1.0, 0.0, -1.0), lattice=7)  # Kawahara with u^n u_x
        tau = 2.0
    M = _model(eq, dx=0.1, dt=1e-3, tau=tau, lib=lib)
    got = dispersion_coeffs(M, phibar)
    want = np.zeros(eq.m + 1, dtype=complex)
    d1 = a * phibar + bb * phibar ** n
    want[1] = -d1 * 1j
    for k in range(2, eq.m + 1):
        want[k] = -eq.alpha[k - 1] * (1j) ** k
    return float(np.max(np.abs(got[: eq.m + 1] - want) / (1.0 + np.abs(want))))


@pytest.mark.parametrize("n", [0.5, 1.5, 2.7])
@pytest.mark.parametrize("lattice", [5, 7])
def test_real_exponent_recovers_the_equation(n, lattice):
    """Linearised about phibar > 0 the scheme recovers -sum_k alpha_k Pi_k'(phibar) (i kappa)^k
    through kappa^m (Eqs. (NPDE3)-(NPDE6)), with Pi_1' = a phibar + b phibar^n."""
    assert dispersion_error(n, lattice) <= 1e-7


@pytest.mark.parametrize("n", [1, 2, 3])
def test_whole_exponent_equals_the_polynomial_model(n):
    """nu = n with the term phi^(1 + nu) gives the model of the ordinary polynomial phi^(n + 1)."""
    a, bb = 0.7, -0.4
    eq = W.class1_real(a, bb, n, (0.1, 0.8, 0.3), lattice=5)
    M1 = _model(eq, lattice=5)
    pi1 = [0.0] * (n + 2)
    pi1[2] += a / 2
    pi1[n + 1] += bb / (n + 1)
    M2 = oracle.Model(eq.alpha, (tuple(pi1),) + eq.pi[1:], 0.1, 1e-3, 1.7, lattice=5)
    for phi in (0.1, 0.5, 1.3):
        assert np.allclose(M1.feq(phi), M2.feq(phi), rtol=1e-12, atol=1e-13)


def test_gkdv_soliton_accuracy():
    """u_t + u^1.5 u_x + u_xxx = 0: the solitary wave (c = 1) on a periodic grid of N = 600,
    t = 1, stays within 5% (E) of the exact one; a scheme that recovered another equation would
    be O(1) off."""
    n, N, dx, dt, tau = 1.5, 600, 0.1, 1e-4, 1.3
    eq = W.gkdv(n)
    x = W.grid(-30.0, N, dx)
    L = N * dx
    phi0 = W.gkdv_soliton(x, 0.0, n, L=L)
    M = _model(eq, dx=dx, dt=dt, tau=tau)
    f = M.init(phi0)
    M.step(f, 10000)
    E = oracle.error_E(M.phi(f), W.gkdv_soliton(x, 1.0, n, L=L))
    assert E < 0.05


def test_gkdv_solitary_wave_solves_its_equation():
    """The solitary wave used as the yardstick of the real-exponent path solves
    u_t + b u^n u_x + u_xxx = 0 (symbolic substitution at rational n, b, c)."""
    sp = pytest.importorskip("sympy")
    x, t = sp.symbols("x t", real=True)
    for n, b, c in ((sp.Rational(3, 2), 1, 1), (sp.Rational(7, 10), 2, sp.Rational(1, 2))):
        u = (c * (n + 1) * (n + 2) / (2 * b) * sp.sech(n * sp.sqrt(c) * (x - c * t) / 2) ** 2) ** (1 / n)
        r = sp.diff(u, t) + b * u ** n * sp.diff(u, x) + sp.diff(u, x, 3)
        for xv, tv in ((sp.Rational(3, 10), sp.Rational(1, 5)), (-1, 2)):
            assert abs(float(sp.N(r.subs({x: xv, t: tv}), 30))) < 1e-20
        # and the workloads' numeric version agrees with the closed form
        xs = np.linspace(-5.0, 5.0, 7)
        got = W.gkdv_soliton(xs, 0.3, float(n), b=float(b), c=float(c))
        want = [float(u.subs({x: xv, t: sp.Rational(3, 10)})) for xv in xs]
        assert np.allclose(got, want, rtol=1e-13)


def test_real_exponent_argument_checks():
    eq = W.class1_real(1.0, 1.0, 1.5, (0.0, 1.0))
    with pytest.raises(oracle.OracleError):  # nu must be positive
        oracle.Model(eq.alpha, eq.pi, 0.1, 1e-3, 1.3, nu=-0.5, pi_nu=eq.pi_nu)
    with pytest.raises(oracle.OracleError):  # a phi^nu term (p = 0) has no derivative of the form
        oracle.Model(eq.alpha, eq.pi, 0.1, 1e-3, 1.3, nu=1.5, pi_nu=((1.0, 1.0), (), ()))


NU_MUTATIONS = [
    ("integral exponent", "x->c[a][i] / ((double)(i + 1) + (double)a * nu)", "x->c[a][i] / ((double)(i + 1))"),
    ("derivative exponent", "((double)i + (double)a * nu) * x->c[a][i]", "((double)i) * x->c[a][i]"),
    ("product exponent", "t.c[a + b][i + j] += x->c[a][i] * y->c[b][j];", "t.c[a][i + j] += x->c[a][i] * y->c[b][j];"),
    ("power of phi^nu", "wa *= w;", "wa *= phi;"),
]


@pytest.mark.parametrize("mut", NU_MUTATIONS, ids=[m[0] for m in NU_MUTATIONS])
def test_planted_real_exponent_mistakes_fail(mut, tmp_path):
    """Each plausible mistake in the generalised algebra fails a closed-form or dispersion pin."""
    name, old, new = mut
    src = open(oracle.SOURCE).read()
    assert src.count(old) == 1, name
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    lib = oracle.bind(oracle.compile_source(str(path), str(tmp_path / "libmut.so")))
    failed = False
    try:
        failed = class1_error(0, lib=lib) > 1e-12 or dispersion_error(1.5, 5, lib=lib) > 1e-7
    except Exception:
        failed = True
    assert failed, name

"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's own formulas.  Each one compares the
oracle with an independent fact:

* the written-out EDFs of Eq. (EDF5)/(EDF7) against the moment constraints of
  Eq. (moments5)/(moments7), i.e. against the Vandermonde matrix of the velocities;
* the tau_k of Eq. (taus) against the Taylor coefficients of
  (e^z - 1) / (1 + tau (e^z - 1)), which the Taylor expansion of Eq. (LBE) yields;
* the auxiliary moments of Sec. II against the closed forms the paper derives
  for its two equation classes, Eqs. (Pi30t60), (intPi1k) and (3Pi20t40);
* the whole set-up (beta_k, A_k0, Pi_k0, M^-1) against the recovered equations
  (NPDE3)-(NPDE6): the linearised LBGK update must have the dispersion relation
  of the PDE through order kappa^m;
* the whole scheme against the global relative errors printed in Tables V and VI;
* conservation of sum(phi) and the uniform fixed point, which hold for any
  correct LBGK scheme on a periodic grid.

``pin_battery`` runs a fast subset of all of them; ``test_planted_mistakes_fail``
compiles copies of the oracle with one plausible mistake each and checks that
every copy fails at least one pin.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_0907_1720_gb300 import workloads as W

E7 = np.array([0, 1, -1, 2, -2, 3, -3])
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")


# ----------------------------------------------------------------- helpers

def moment_matrix(b):
    e = E7[:b].astype(float)
    return np.array([e ** k for k in range(b)])


def taus_series(tau: Fraction, order=6):
    """[z^k] of u/(1 + tau u), u = e^z - 1, exactly in rationals."""
    u = [Fraction(0)] + [Fraction(1, math.factorial(k)) for k in range(1, order + 1)]

    def mul(a, b):
        r = [Fraction(0)] * (order + 1)
        for i, x in enumerate(a):
            if x:
                for j, y in enumerate(b[: order + 1 - i]):
                    r[i + j] += x * y
        return r

    g = [Fraction(0)] * (order + 1)
    un = u[:]
    for n in range(1, order + 1):
        g = [gi + (-tau) ** (n - 1) * ui for gi, ui in zip(g, un)]
        un = mul(un, u)
    return g


def dispersion_coeffs(M, phibar, r=1.0, Q=128):
    """Taylor coefficients a_n of log(lambda(kappa)) / dt, lambda = principal eigenvalue of the
    linearised update G = S(kappa) [(1 - w) I + w dfeq 1^T], S = diag(exp(-i kappa e_j dx)),
    by the Cauchy integral on |kappa| = r."""
    b = M.b
    d = M.dfeq(phibar)
    w = 1.0 / M.tau
    C = (1.0 - w) * np.eye(b) + w * np.outer(d, np.ones(b))
    e = E7[:b]
    th = 2.0 * np.pi * np.arange(Q) / Q
    g = np.empty(Q, dtype=complex)
    for q in range(Q):
        kap = r * np.exp(1j * th[q])
        ev = np.linalg.eigvals(np.diag(np.exp(-1j * kap * e * M.dx)) @ C)
        g[q] = np.log(ev[np.argmin(np.abs(ev - 1.0))]) / M.dt
    return np.array([np.mean(g * np.exp(-1j * n * th)) / r ** n for n in range(Q // 2)])


def expected_dispersion(alpha, pi, phibar, nmax):
    """a_n of the linearised PDE: -alpha_n Pi_n'(phibar) i^n (alpha_1 folded into Pi_1)."""
    out = np.zeros(nmax + 1, dtype=complex)
    for k in range(1, len(alpha) + 1):
        coef = pi[k - 1]
        dpi = sum(p * c * phibar ** (p - 1) for p, c in enumerate(coef) if p >= 1)
        if k <= nmax:
            out[k] = -alpha[k - 1] * dpi * (1j) ** k
    return out


DISPERSION_CASES = [
    # (name, equation, dx, dt, tau, scheme, phibar, exact_through)
    ("kdv_d1q5", W.kdv(), 0.1, 1e-3, 1.3, 1, 0.7, 4),
    ("kdv_d1q5_scheme2", W.kdv(), 0.1, 1e-3, 1.3, 2, 0.7, 3),
    ("kdv_burgers_d1q5_A40", W.kdv_burgers(2.0, 0.05, 0.7), 0.1, 1e-3, 1.3, 1, 0.4, 4),
    ("ks_d1q5_A40", W.ks(), 0.1, 1e-3, 1.3, 1, 0.3, 4),
    ("gks_d1q5", W.ks(1.0, 4.0, 1.0), 0.1, 1e-3, 1.4, 1, -0.2, 4),
    ("gks_cubic_d1q5", W.gks_cubic(), 0.1, 1e-3, 1.4, 1, 0.5, 4),
    ("k22_d1q5", W.k22(), 0.1, 1e-3, 1.5, 1, 0.6, 4),
    ("kawahara_d1q7_A60", W.kawahara(), 0.1, 1e-3, 2.0, 1, 0.5, 6),
    ("kawahara_d1q7_scheme2", W.kawahara(), 0.1, 1e-3, 2.0, 2, 0.5, 5),
    ("modified_kawahara_d1q7", W.modified_kawahara(), 0.1, 1e-3, 2.1, 1, -0.4, 6),
    ("sixth_order_d1q7", W.Equation("sixth", (1.0, 0.0, 0.5, 0.3, -1.0, 0.2),
                                    ((0, 0, 0.5), (), (0, 1), (0, 1), (0, 1), (0, 1))),
     0.1, 1e-3, 2.2, 1, 0.3, 6),
]


def check_dispersion(case, lib=None):
    name, eq, dx, dt, tau, scheme, phibar, n_exact = case
    M = oracle.Model(eq.alpha, eq.pi, dx, dt, tau, lattice=eq.lattice, scheme=scheme, lib=lib)
    a = dispersion_coeffs(M, phibar)
    want = expected_dispersion(eq.alpha, eq.pi, phibar, n_exact)
    err = np.abs(a[: n_exact + 1] - want)
    tol = 1e-7 * (1.0 + np.abs(want))
    return bool(np.all(err <= tol)), a, want


def a50_cross_residual(lib=None, phibar=0.5, tau=2.0, dt=1e-3):
    """kappa^5 coefficient with alpha_2 and alpha_3 both on, minus the two one-term runs.  A_50
    (Sec. II E) is built to cancel exactly the beta_2 beta_3 cross terms of Eq. (Oeps5E1), so the
    kappa^5 residual that alpha_2 alone leaves on D1Q7 must add up with no cross part."""
    def a5(a2, a3):
        eq = W.Equation("x", (1.0, a2, a3, 0.0, 0.0), ((0, 0, 0.5), (0, 1), (0, 1), (0, 1), ()), lattice=7)
        M = oracle.Model(eq.alpha, eq.pi, 0.1, dt, tau, lattice=7, lib=lib)
        return dispersion_coeffs(M, phibar)[5]
    return abs(a5(0.3, 0.5) - a5(0.3, 0.0) - a5(0.0, 0.5) + a5(0.0, 0.0))


def table_rows(use=None):
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tab, ex, scheme, c, tau, t, E, kind, tol = line.split()
            if use and kind != use:
                continue
            rows.append(dict(table=tab, scheme=int(scheme), c=float(c), tau=float(tau), t=int(t),
                             E=float(E), tol=None if tol == "-" else float(tol)))
    return rows


def table_error(row, lib=None):
    dt = 0.1 / row["c"]
    if row["table"] == "V":
        p = W.kawahara_config(N=600, dx=0.1, dt=dt, tau=row["tau"], t_end=row["t"], scheme=row["scheme"])
    else:
        p = W.modified_kawahara_config(N=600, dx=0.1, dt=dt, tau=row["tau"], t_end=row["t"],
                                       scheme=row["scheme"])
    phi = oracle.run_problem(p, lib=lib)
    return oracle.error_E(phi, p.exact(p.t_end))


def pin_battery(lib=None):
    """Fast subset of every pin; returns the names of the pins that fail."""
    failed = []
    rng = np.random.default_rng(7)
    for b in (5, 7):
        Mm = moment_matrix(b)
        for _ in range(3):
            P = rng.normal(size=b)
            if not np.allclose(Mm @ oracle.edf(b, P, lib=lib), P, rtol=0, atol=1e-12 * (1 + np.abs(P).max())):
                failed.append(f"edf{b}")
                break
    for tau in (Fraction(13, 10), Fraction(202, 100)):
        M = oracle.Model((1.0,), ((0, 1),), 0.1, 1e-3, float(tau), lattice=7, lib=lib)
        want = [float(v) for v in taus_series(tau)]
        if not np.allclose(M.taus[2:7], want[2:7], rtol=1e-13, atol=1e-15):
            failed.append("taus")
            break
    for case in DISPERSION_CASES:
        try:
            ok, _, _ = check_dispersion(case, lib=lib)
        except Exception:
            ok = False
        if not ok:
            failed.append("dispersion:" + case[0])
    if not a50_cross_residual(lib=lib) < 1e-10:
        failed.append("a50_cross")
    p = W.kdv_config(dt=2e-5, tau=1.07, t_end=0.01)
    M = oracle.Model(p.eq.alpha, p.eq.pi, p.dx, p.dt, p.tau, lib=lib)
    f = M.init(p.phi0)
    s0 = M.phi(f).sum()
    M.step(f, 200)
    s1 = M.phi(f).sum()
    if abs(s1 - s0) > 1e-12 * np.abs(p.phi0).sum():
        failed.append("conservation")
    for row in table_rows("pin"):
        if row["c"] == 10.0 and row["t"] == 1:
            E = table_error(row, lib=lib)
            if not abs(E / row["E"] - 1.0) <= row["tol"]:
                failed.append(f"table{row['table']}_s{row['scheme']}_c10")
    return failed


# ------------------------------------------------------------------- tests

@pytest.mark.parametrize("b", [5, 7])
def test_edf_satisfies_moment_constraints(b):
    """Eq. (moments5)/(moments7): sum_j e_j^k f^eq_j = Pibar_k for k < b."""
    rng = np.random.default_rng(b)
    Mm = moment_matrix(b)
    for _ in range(20):
        P = rng.normal(size=b) * 10.0 ** rng.uniform(-3, 3, size=b)
        f = oracle.edf(b, P)
        assert np.allclose(Mm @ f, P, rtol=0, atol=1e-13 * np.abs(P).max())


@pytest.mark.parametrize("b", [5, 7])
def test_edf_columns_are_inverse_of_vandermonde(b):
    """The EDF maps unit moment vectors onto the columns of M^-1 (numpy's inverse of M)."""
    Minv = np.linalg.inv(moment_matrix(b))
    cols = np.array([oracle.edf(b, np.eye(b)[k]) for k in range(b)]).T
    assert np.allclose(cols, Minv, rtol=0, atol=1e-14)


@pytest.mark.parametrize("tau", [Fraction(1, 2) + Fraction(1, 7), Fraction(13, 10), Fraction(202, 100),
                                 Fraction(3777, 100)])
def test_taus_are_taylor_coefficients(tau):
    """Eq. (taus): tau_k = [z^k] (e^z - 1)/(1 + tau (e^z - 1))."""
    M = oracle.Model((1.0,), ((0, 1),), 0.1, 1e-3, float(tau), lattice=7)
    want = taus_series(tau)
    for k in range(2, 7):
        assert M.taus[k] == pytest.approx(float(want[k]), rel=1e-12, abs=1e-14)


def _int_pi1k(u, a, bb, n, k):
    """Eq. (intPi1k): int (Pi_1')^k du for Pi_1' = a u + b u^n."""
    return u * sum(math.comb(k, j) * (a * u) ** (k - j) * (bb * u ** n) ** j / (j * n + k + 1 - j)
                   for j in range(k + 1))


@pytest.mark.parametrize("seed", range(4))
def test_aux_moments_class1_closed_forms(seed):
    """Eq. (Pi30t60) with Eq. (intPi1k): u_t + a u u_x + b u^n u_x + sum_k alpha_k d^k u = 0."""
    rng = np.random.default_rng(100 + seed)
    a, bb = rng.uniform(-2, 2), rng.uniform(-2, 2)
    n = int(rng.integers(0, 4))
    al = rng.uniform(0.2, 1.0, size=5) * rng.choice([-1, 1], size=5)
    pi1 = [0.0] * max(3, n + 2)
    pi1[2] += a / 2.0
    pi1[n + 1] += bb / (n + 1)
    eq = W.Equation("class1", (1.0,) + tuple(al), (tuple(pi1),) + ((0, 1),) * 5, lattice=7)
    M = oracle.Model(eq.alpha, eq.pi, 0.1, 1e-3, 1.7, lattice=7)
    be, (A40, A50, A60) = M.beta, M.A
    for u in rng.uniform(-1.5, 1.5, size=6):
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
            assert abs(M.aux_moment(k, u) - want[k]) <= 1e-12 * scale, (k, u)


@pytest.mark.parametrize("seed", range(4))
def test_aux_moments_class2_closed_forms(seed):
    """Eq. (3Pi20t40): u_t + a u u_x + b u^n u_x + alpha_2 (u^p)_xx + alpha_3 (u^q)_xxx = 0."""
    rng = np.random.default_rng(200 + seed)
    a, bb = rng.uniform(-2, 2), rng.uniform(-2, 2)
    n, p, q = int(rng.integers(0, 4)), int(rng.integers(1, 4)), int(rng.integers(1, 4))
    a2, a3 = rng.uniform(0.1, 0.5), rng.uniform(0.5, 1.0)
    pi1 = [0.0] * max(3, n + 2)
    pi1[2] += a / 2.0
    pi1[n + 1] += bb / (n + 1)
    pi2 = [0.0] * p + [1.0]
    pi3 = [0.0] * q + [1.0]
    eq = W.Equation("class2", (1.0, a2, a3), (tuple(pi1), tuple(pi2), tuple(pi3)), lattice=5)
    M = oracle.Model(eq.alpha, eq.pi, 0.1, 1e-3, 1.3, lattice=5)
    be, A40 = M.beta, M.A[0]
    for u in rng.uniform(0.1, 1.5, size=6):
        I2, I3, I4 = (_int_pi1k(u, a, bb, n, k) for k in (2, 3, 4))
        want3 = I3 + 3 * be[2] * p * u ** p * (a * u / (p + 1) + bb * u ** n / (p + n))
        want4 = (I4 + 6 * be[2] * p * u ** p * ((a * u) ** 2 / (p + 2) + 2 * (a * u) * (bb * u ** n) / (p + n + 1)
                                               + (bb * u ** n) ** 2 / (p + 2 * n))
                 + 4 * be[3] * q * u ** q * (a * u / (q + 1) + bb * u ** n / (q + n)) + A40 * u)
        for k, want in ((2, I2), (3, want3), (4, want4)):
            assert M.aux_moment(k, u) == pytest.approx(want, rel=1e-11, abs=1e-12), (k, u)


@pytest.mark.parametrize("case", DISPERSION_CASES, ids=[c[0] for c in DISPERSION_CASES])
def test_linear_dispersion_matches_recovered_equation(case):
    """Eqs. (NPDE3)-(NPDE6): the linearised update reproduces the PDE's dispersion relation
    exactly through order kappa^m (through kappa^{b-1} for scheme 1 when the remarks hold)."""
    ok, a, want = check_dispersion(case)
    n = case[-1]
    assert ok, np.c_[a[: n + 1], want]


def test_d1q7_with_alpha2_is_flagged_and_inexact_at_fifth_order():
    """Remark 5 requires alpha_2 = 0 on D1Q7.  With alpha_2 != 0 the printed A_50/A_60 leave a
    kappa^5 residual (the paper's Sec. II E derivation omits it); the model flags the case."""
    eq = W.Equation("d1q7_alpha2", (1.0, 0.3, 0.0, 0.0, 0.0), ((0, 0, 0.5), (0, 1), (), (), ()), lattice=7)
    M = oracle.Model(eq.alpha, eq.pi, 0.1, 1e-3, 2.0, lattice=7)
    assert M.inexact
    a = dispersion_coeffs(M, 0.5)
    want = expected_dispersion(eq.alpha, eq.pi, 0.5, 4)
    assert np.allclose(a[:5], want, rtol=0, atol=1e-7)
    assert abs(a[5]) > 1e-9  # residual, three orders above the 1e-13 rounding level of the Cauchy sum


@pytest.mark.parametrize("phibar,tau,dt", [(0.5, 2.0, 1e-3), (0.2, 1.6, 1e-2), (-0.7, 2.5, 1e-3)])
def test_a50_cancels_cross_terms(phibar, tau, dt):
    """A_50 = (4 tau_2 tau_4 + 3 tau_3^2 - 2 tau_2^2 tau_3) beta_2 beta_3 / tau_5 removes every
    beta_2 beta_3 term at kappa^5: the residual is the sum of the one-coefficient residuals
    (rounding of the Cauchy sum is about 1e-13)."""
    assert a50_cross_residual(phibar=phibar, tau=tau, dt=dt) < 1e-10


def test_flags_inexact_when_pi2_is_not_phi():
    """A_40 is derived for Pi_2 = phi (Sec. II D); Eq. (3Pi20t40) keeps A_40 u for Pi_2 = u^p."""
    eq = W.Equation("burgers_p2", (1.0, 0.2, 1.0), ((0, 0, 0.5), (0, 0, 1), (0, 1)), lattice=5)
    assert oracle.Model(eq.alpha, eq.pi, 0.1, 1e-3, 1.3).inexact
    assert not oracle.Model(W.kdv_burgers(1, 0.1, 1).alpha, W.kdv_burgers(1, 0.1, 1).pi, 0.1, 1e-3, 1.3).inexact


@pytest.mark.parametrize("tau", [0.5, 0.5 + math.sqrt(3) / 6])
def test_singular_tau_rejected(tau):
    """tau_2 = 0 at tau = 1/2 and tau_3 = 0 at tau = 1/2 + sqrt(3)/6: beta_k would be infinite."""
    eq = W.kdv_burgers(1.0, 0.05, 1.0)
    with pytest.raises(oracle.OracleError):
        oracle.Model(eq.alpha, eq.pi, 0.1, 1e-3, tau)


def test_conservation_periodic():
    """sum_x phi is invariant: streaming permutes f, and sum_j f^eq_j = phi (Eq. (moments))."""
    p = W.ks_config(t_end=0.2)
    M = oracle.Model(p.eq.alpha, p.eq.pi, p.dx, p.dt, p.tau)
    f = M.init(p.phi0)
    s0 = M.phi(f).sum()
    M.step(f, p.nsteps)
    phi = M.phi(f)
    assert abs(phi.sum() - s0) <= 50 * np.finfo(float).eps * np.abs(phi).sum() * math.sqrt(p.nsteps)


@pytest.mark.parametrize("eq", [W.kdv(), W.kawahara(), W.ks()], ids=["kdv", "kawahara", "ks"])
def test_uniform_state_is_fixed_point(eq):
    M = oracle.Model(eq.alpha, eq.pi, 0.1, 1e-3, 1.5, lattice=eq.lattice)
    f = M.init(np.full(37, 0.37))
    M.step(f, 50)
    phi = M.phi(f)
    assert phi.max() == phi.min()
    assert abs(phi[0] - 0.37) < 1e-14


@pytest.mark.parametrize("row", table_rows("pin"),
                         ids=lambda r: f"T{r['table']}_s{r['scheme']}_c{int(r['c'])}_t{r['t']}")
def test_paper_tables_reproduced(row):
    """Global relative errors of Tables V and VI (Examples 4.5, 4.6), periodic N = 600."""
    if row["c"] >= 1000 and row["t"] > 1:
        pytest.skip("long run")
    E = table_error(row)
    assert E == pytest.approx(row["E"], rel=row["tol"])


def test_kdv_soliton_accuracy():
    """The KdV soliton (c = 4) on N = 400 at t = 1 (dt = 1e-5, tau = 1.1, 100 000 steps): the
    error against the exact solution is E = 0.0994 (relative L2 0.059).  The pin holds E to
    within 2.5% of that value on both sides: a scheme that recovered another equation would be
    O(1) off, and a dropped or mis-scaled term of the equilibria moves E by more than 2.5%."""
    p = W.kdv_config()
    phi = oracle.run_problem(p)
    E = oracle.error_E(phi, p.exact(p.t_end))
    assert 0.097 < E < 0.102


def test_error_decreases_with_dt():
    """Observed convergence under dt refinement at fixed dx (the protocol of Tables I-VII);
    the paper states no order, so only monotone decrease is asserted (parity unpinned)."""
    Es = []
    for c, tau in ((10, 3.37), (100, 2.53), (1000, 2.02)):
        p = W.kawahara_config(N=600, dx=0.1, dt=0.1 / c, tau=tau, t_end=0.5)
        Es.append(oracle.error_E(oracle.run_problem(p), p.exact(p.t_end)))
    assert Es[0] > Es[1] > Es[2]


def kdv_refinement_error(dx, t_end=0.1, C=1e-2, tau=1.1):
    """E of the KdV soliton (c = 4, periodic [-20, 20)) at t_end with dt = C dx^3 and fixed tau:
    the joint refinement under which the recovered equation's error terms shrink together (dt
    scaled like dx^m for the m = 3 equation, c = dx/dt growing like 1/dx^2)."""
    N = int(round(40.0 / dx))
    dt = C * dx ** 3
    x = W.grid(-20.0, N, dx)
    n = int(round(t_end / dt))
    phi = oracle.run(W.kdv().alpha, W.kdv().pi, dx, dt, tau, W.kdv_soliton(x, 0.0, L=40.0), n)
    return oracle.error_E(phi, W.kdv_soliton(x, n * dt, L=40.0))


def test_observed_order_under_joint_refinement():
    """Observed convergence order of the whole scheme (the paper states none): halving dx with
    dt = 1e-2 dx^3 and tau = 1.1 gives orders 1.63 and 1.88 on the KdV soliton at t = 0.1,
    approaching second order in dx (parity unpinned: measured, not derived)."""
    E = [kdv_refinement_error(dx) for dx in (0.2, 0.1, 0.05)]
    orders = [math.log2(E[i] / E[i + 1]) for i in range(2)]
    assert orders[0] > 1.4 and orders[1] > 1.7, (E, orders)


def test_exact_solutions_satisfy_their_equations():
    """Substitute the closed forms used as yardsticks into their PDEs (symbolically)."""
    sp = pytest.importorskip("sympy")
    x, t = sp.symbols("x t", real=True)
    c = sp.Rational(4)
    checks = []
    u = c / 2 * sp.sech(sp.sqrt(c) / 2 * (x - c * t)) ** 2
    checks.append(sp.diff(u, t) + 6 * u * sp.diff(u, x) + sp.diff(u, x, 3))
    c = sp.Rational(3, 2)
    u = sp.sqrt(c) * sp.sech(sp.sqrt(c) * (x - c * t))
    checks.append(sp.diff(u, t) + 6 * u ** 2 * sp.diff(u, x) + sp.diff(u, x, 3))
    lam = sp.Rational(5, 4)
    u = 4 * lam / 3 * sp.cos((x - lam * t) / 4) ** 2
    checks.append(sp.diff(u, t) + sp.diff(u ** 2, x) + sp.diff(u ** 2, x, 3))
    A, B, C = sp.Rational(105, 169), 1 / (2 * sp.sqrt(13)), sp.Rational(36, 169)
    u = A * sp.sech(B * (x - C * t)) ** 4
    checks.append(sp.diff(u, t) + u * sp.diff(u, x) + sp.diff(u, x, 3) - sp.diff(u, x, 5))
    A, B, C = -3 / sp.sqrt(10), sp.sqrt(sp.Rational(1, 5)) / 2, sp.Rational(4, 25)
    u = A * sp.sech(B * (x - C * t)) ** 2
    checks.append(sp.diff(u, t) + u ** 2 * sp.diff(u, x) + sp.diff(u, x, 3) - sp.diff(u, x, 5))
    u = sp.Rational(105, 169) * sp.sech((x - sp.Rational(205, 169) * t) / (2 * sp.sqrt(13))) ** 4
    checks.append(sp.diff(u, t) + u * sp.diff(u, x) + sp.diff(u, x) + sp.diff(u, x, 3) - sp.diff(u, x, 5))
    for r in checks:
        f = sp.lambdify((x, t), r, "mpmath")
        for xv, tv in ((0.3, 0.1), (-1.7, 0.4), (2.9, 1.3)):
            assert abs(f(xv, tv)) < 1e-12
    # the workloads module evaluates the same closed forms
    xs = np.linspace(-5, 5, 11)
    assert np.allclose(W.kdv_soliton(xs, 0.3), [float(4 / 2 * sp.sech(1 * (v - 4 * 0.3)) ** 2) for v in xs])
    assert np.allclose(W.kawahara_soliton(xs, 0.3),
                       [float(sp.Rational(105, 169) * sp.sech((v - 36 / 169 * 0.3) / (2 * sp.sqrt(13))) ** 4)
                        for v in xs])


def test_ks_spectral_reference_converged():
    """The ETDRK4 yardstick of the KS run agrees with itself at half the step."""
    a = W.ks_spectral_reference(t_end=2.0, h=2e-3)
    b = W.ks_spectral_reference(t_end=2.0, h=1e-3)
    assert np.abs(a - b).max() < 1e-9 * np.abs(b).max()


def test_pin_battery_passes():
    assert pin_battery() == []


MUTATIONS = [
    ("drop A60", "op_axpy(&g, M->A60, &one);", ""),
    ("drop A40", "op_axpy(&g, M->A40, &one);", ""),
    ("A60 sign", "(4.0 * t4 - t2 * t3)", "(4.0 * t4 + t2 * t3)"),
    ("tau3 sign", "tk[3] = t2 - tau + 1.0 / 6.0;", "tk[3] = t2 + tau + 1.0 / 6.0;"),
    ("beta power", "pow(dt, (double)(k - 1))", "pow(dt, (double)k)"),
    ("Pi50 10 beta3", "op_axpy(&g, 10.0 * b3, &t)", "op_axpy(&g, 5.0 * b3, &t)"),
    ("Pi30 drop beta2", "op_axpy(&g, 3.0 * b2, &t)", "op_axpy(&g, 0.0 * b2, &t)"),
    ("EDF7 f3 index", "feq[3] = (-18.0 * P[1]", "feq[3] = (-18.0 * P[2]"),
    ("EDF5 f1 denominator", "feq[1] = (4.0 * (P[1] + P[2]) - P[3] - P[4]) / 6.0;",
     "feq[1] = (4.0 * (P[1] + P[2]) - P[3] - P[4]) / 8.0;"),
    ("moment scaling", "double ck = pow(M->c, (double)k);", "double ck = pow(M->c, (double)(k - 1));"),
    ("stream direction", "long dst = ((i + E7[j]) % N + N) % N;", "long dst = ((i - E7[j]) % N + N) % N;"),
    ("relaxation", "fstar[j] = fj - (fj - feq[j]) / M->tau;", "fstar[j] = fj - (fj - feq[j]) * M->tau;"),
    ("A50 coefficient", "(4.0 * t2 * t4 + 3.0 * t3 * t3", "(4.0 * t2 * t4 + 2.0 * t3 * t3"),
]


@pytest.mark.parametrize("mut", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistakes_fail(mut, tmp_path):
    """Each plausible mistake planted in a copy of the oracle fails at least one pin."""
    name, old, new = mut
    src = open(oracle.SOURCE).read()
    assert src.count(old) == 1, name
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    lib = oracle.bind(oracle.compile_source(str(path), str(tmp_path / "libmut.so")))
    assert pin_battery(lib=lib), name

"""Seeded synthetic inputs: equations, grids, initial data and exact solutions.

This module is shared by the tests, the benchmark and the smoke check.  It holds
none of the lattice Boltzmann arithmetic: it only says WHICH problem to solve
(the coefficients alpha_k and the polynomials Pi_k of Eq. (NPDE)), on which
grid, from which initial profile, and what the exact solution is where one is
known.  Both the CUDA library and the CPU oracle consume these descriptions.

An equation is ``Equation(name, alpha, pi)``: ``alpha[k-1]`` is alpha_k and
``pi[k-1]`` lists the coefficients of Pi_k(phi) = sum_p pi[k-1][p] * phi**p.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED = 20090717


@dataclass(frozen=True)
class Equation:
    name: str
    alpha: tuple
    pi: tuple
    lattice: int = 0  # 0 = the smallest lattice that carries order m (5 for m <= 4, else 7)
    nu: float = 0.0   # real exponent of the phi^(p + nu) terms (0: none)
    pi_nu: tuple = None  # pi_nu[k-1][p]: coefficient of phi^(p + nu) in Pi_k (p >= 1)

    @property
    def m(self) -> int:
        return len(self.alpha)


def _eq(name, m, terms, pi1, lattice=0):
    """terms: {k: (alpha_k, Pi_k coefficients)} for k >= 2; pi1: coefficients of Pi_1."""
    alpha = [1.0] + [0.0] * (m - 1)
    pi = [tuple(pi1)] + [()] * (m - 1)
    for k, (a, p) in terms.items():
        alpha[k - 1] = float(a)
        pi[k - 1] = tuple(float(v) for v in p)
    return Equation(name, tuple(alpha), tuple(tuple(float(v) for v in r) for r in pi), lattice)


# ----------------------------------------------------------------- equations

def kdv(lattice=0):
    """phi_t + 6 phi phi_x + phi_xxx = 0:  Pi_1 = 3 phi^2, alpha_3 = 1, Pi_3 = phi."""
    return _eq("kdv", 3, {3: (1.0, (0, 1))}, (0, 0, 3.0), lattice)


def mkdv(lattice=0):
    """u_t + 6 u^2 u_x + u_xxx = 0:  Pi_1 = 2 u^3, alpha_3 = 1, Pi_3 = u."""
    return _eq("mkdv", 3, {3: (1.0, (0, 1))}, (0, 0, 0, 2.0), lattice)


def kdv_burgers(a, b, d, lattice=0):
    """u_t + a u u_x - b u_xx + d u_xxx = 0 (Example 4.8 with alpha = a, gamma = b, delta = d)."""
    return _eq("kdv_burgers", 3, {2: (-b, (0, 1)), 3: (d, (0, 1))}, (0, 0, 0.5 * a), lattice)


def k22(lattice=0):
    """K(2,2): u_t + (u^2)_x + (u^2)_xxx = 0:  Pi_1 = u^2, alpha_3 = 1, Pi_3 = u^2."""
    return _eq("k22", 3, {3: (1.0, (0, 0, 1))}, (0, 0, 1.0), lattice)


def ks(a2=1.0, a3=0.0, a4=1.0, lattice=0):
    """Kuramoto-Sivashinsky family u_t + u u_x + a2 u_xx + a3 u_xxx + a4 u_xxxx = 0."""
    terms = {2: (a2, (0, 1)), 4: (a4, (0, 1))}
    if a3:
        terms[3] = (a3, (0, 1))
    return _eq("ks", 4, terms, (0, 0, 0.5), lattice)


def gks_cubic(a=1.0, b=1.0, lattice=0):
    """Example 4.4: u_t + 3 u^3 u_x + a u_xx - b u_xxx + u_xxxx = 0 (Pi_1 = 3 u^4 / 4)."""
    return _eq("gks_cubic", 4, {2: (a, (0, 1)), 3: (-b, (0, 1)), 4: (1.0, (0, 1))},
               (0, 0, 0, 0, 0.75), lattice)


def kawahara(alpha=1.0, beta=1.0, gamma=-1.0, lattice=0):
    """Example 4.5: u_t + alpha u u_x + beta u_xxx + gamma u_xxxxx = 0."""
    return _eq("kawahara", 5, {3: (beta, (0, 1)), 5: (gamma, (0, 1))}, (0, 0, 0.5 * alpha), lattice)


def modified_kawahara(a=1.0, b=1.0, k=1.0, lattice=0):
    """Example 4.6: u_t + a u^2 u_x + b u_xxx - k u_xxxxx = 0 (Pi_1 = a u^3 / 3)."""
    return _eq("modified_kawahara", 5, {3: (b, (0, 1)), 5: (-k, (0, 1))}, (0, 0, 0, a / 3.0), lattice)


def class1_real(a, b, n, alphas, lattice=0):
    """Class (1) of Sec. III C with a real exponent n > 0:
    u_t + a u u_x + b u^n u_x + sum_{k>=2} alpha_k d_x^k u = 0, i.e. Pi_1 = a u^2 / 2 +
    b u^(n+1) / (n+1), Pi_k = u.  alphas = (alpha_2, ..., alpha_m)."""
    m = 1 + len(alphas)
    alpha = (1.0,) + tuple(float(x) for x in alphas)
    pi = ((0.0, 0.0, a / 2.0),) + ((0.0, 1.0),) * (m - 1)
    pi_nu = ((0.0, b / (n + 1.0)),) + ((),) * (m - 1)
    return Equation(f"class1_n{n:g}", alpha, pi, lattice, float(n), pi_nu)


def gkdv(n, b=1.0, lattice=0):
    """Generalised KdV u_t + b u^n u_x + u_xxx = 0 with a real exponent n (class (1))."""
    return class1_real(0.0, b, n, (0.0, 1.0), lattice)


def kdv_kawahara(lattice=0):
    """Example 4.7: u_t + u u_x + u_x + u_xxx - u_xxxxx = 0 (Pi_1 = u^2/2 + u)."""
    return _eq("kdv_kawahara", 5, {3: (1.0, (0, 1)), 5: (-1.0, (0, 1))}, (0, 1.0, 0.5), lattice)


# ------------------------------------------------------------ exact solutions

def sech(z):
    with np.errstate(over="ignore"):
        return 1.0 / np.cosh(z)


def kdv_soliton(x, t, c=4.0, x0=0.0, L=None):
    """(c/2) sech^2(sqrt(c)/2 (x - c t - x0)); with L, the nearest periodic image."""
    z = x - c * t - x0
    if L is not None:
        z = (z + 0.5 * L) % L - 0.5 * L
    return 0.5 * c * sech(0.5 * math.sqrt(c) * z) ** 2


def mkdv_soliton(x, t, c=1.0, x0=0.0, L=None):
    """sqrt(c) sech(sqrt(c) (x - c t - x0)) solves u_t + 6 u^2 u_x + u_xxx = 0."""
    z = x - c * t - x0
    if L is not None:
        z = (z + 0.5 * L) % L - 0.5 * L
    return math.sqrt(c) * sech(math.sqrt(c) * z)


def k22_compacton(x, t, lam=1.0, x0=0.0, L=None):
    """(4 lam / 3) cos^2((x - lam t - x0) / 4) on |x - lam t - x0| <= 2 pi, else 0."""
    z = x - lam * t - x0
    if L is not None:
        z = (z + 0.5 * L) % L - 0.5 * L
    return np.where(np.abs(z) <= 2.0 * np.pi, (4.0 * lam / 3.0) * np.cos(z / 4.0) ** 2, 0.0)


def kawahara_soliton(x, t, alpha=1.0, beta=1.0, gamma=-1.0, x0=0.0, L=None):
    """Example 4.5: A sech^4(B (x - C t)), A = -105 beta^2/(169 alpha gamma),
    B = sqrt(-beta / (13 gamma)) / 2, C = -36 beta^2 / (169 gamma)."""
    A = -105.0 * beta ** 2 / (169.0 * alpha * gamma)
    B = 0.5 * math.sqrt(-beta / (13.0 * gamma))
    C = -36.0 * beta ** 2 / (169.0 * gamma)
    z = x - C * t - x0
    if L is not None:
        z = (z + 0.5 * L) % L - 0.5 * L
    return A * sech(B * z) ** 4


def modified_kawahara_soliton(x, t, a=1.0, b=1.0, k=1.0, x0=0.0, L=None):
    """Example 4.6: A sech^2(B (x - C t)), A = -3 b / sqrt(10 a k), B = sqrt(b / (5 k)) / 2,
    C = 4 b^2 / (25 k)."""
    A = -3.0 * b / math.sqrt(10.0 * a * k)
    B = 0.5 * math.sqrt(b / (5.0 * k))
    C = 4.0 * b ** 2 / (25.0 * k)
    z = x - C * t - x0
    if L is not None:
        z = (z + 0.5 * L) % L - 0.5 * L
    return A * sech(B * z) ** 2


def gkdv_soliton(x, t, n, b=1.0, c=1.0, x0=0.0, L=None):
    """Solitary wave of u_t + b u^n u_x + u_xxx = 0 (real n > 0, b > 0, speed c > 0):
    [c (n + 1)(n + 2) / (2 b) sech^2(n sqrt(c) (x - c t - x0) / 2)]^(1/n)."""
    z = x - c * t - x0
    if L is not None:
        z = (z + 0.5 * L) % L - 0.5 * L
    return (c * (n + 1.0) * (n + 2.0) / (2.0 * b) * sech(0.5 * n * math.sqrt(c) * z) ** 2) ** (1.0 / n)


def kdv_kawahara_soliton(x, t, x0=20.0, L=None):
    """Example 4.7: (105/169) sech^4((x - 205 t / 169 - x0) / (2 sqrt(13)))."""
    z = x - 205.0 / 169.0 * t - x0
    if L is not None:
        z = (z + 0.5 * L) % L - 0.5 * L
    return 105.0 / 169.0 * sech(z / (2.0 * math.sqrt(13.0))) ** 4


def kdv_burgers_soliton_ic(x, a, d, c, x0=0.0):
    """KdV soliton (3c/a) sech^2(sqrt(c/d)/2 (x - x0)) of u_t + a u u_x + d u_xxx = 0, used as
    the initial profile of the KdV-Burgers ensemble (no exact solution once b > 0)."""
    return (3.0 * c / a) * sech(0.5 * math.sqrt(c / d) * (x - x0)) ** 2


def ks_shock(x, t, b=5.0, k=0.5 * math.sqrt(11.0 / 19.0), x0=-12.0):
    """Example 4.1: b + (15/19) sqrt(11/19) (-9 z + 11 z^3), z = tanh(k (x - b t - x0)), solves
    u_t + u u_x + u_xx + u_xxxx = 0 for k = sqrt(11/19) / 2."""
    z = np.tanh(k * (x - b * t - x0))
    return b + 15.0 / 19.0 * math.sqrt(11.0 / 19.0) * (-9.0 * z + 11.0 * z ** 3)


def ks_shock2(x, t, b=5.0, k=1.0 / (2.0 * math.sqrt(19.0)), x0=-25.0):
    """Example 4.2: b + 15/(19 sqrt 19) (-3 z + z^3), z = tanh(k (x - b t - x0)), solves
    u_t + u u_x - u_xx + u_xxxx = 0 for k = 1 / (2 sqrt 19)."""
    z = np.tanh(k * (x - b * t - x0))
    return b + 15.0 / (19.0 * math.sqrt(19.0)) * (-3.0 * z + z ** 3)


def ks_initial(x):
    """u0 = cos(x/16) (1 + sin(x/16)) on [0, 32 pi)."""
    return np.cos(x / 16.0) * (1.0 + np.sin(x / 16.0))


# --------------------------------------------------------------------- grids

def grid(xl, N, dx):
    """x_i = xl + i dx, i = 0..N-1; periodic with period N dx."""
    return xl + dx * np.arange(N, dtype=np.float64)


# ------------------------------------------------------------------- problems

@dataclass
class Problem:
    """One solve: equation, grid, relaxation, steps, initial profile, exact solution."""
    eq: Equation
    N: int
    dx: float
    dt: float
    tau: float
    nsteps: int
    phi0: np.ndarray
    xl: float = 0.0
    scheme: int = 1
    exact: object = None          # callable t -> phi*(x, t) on the grid, or None
    meta: dict = field(default_factory=dict)
    boundary: str = "periodic"    # or "nee": bounded grid, prescribed phi at both ends
    exact_xt: object = None       # callable (x, t) -> phi*(x, t) (bounded problems)

    @property
    def x(self):
        return grid(self.xl, self.N, self.dx)

    @property
    def t_end(self):
        return self.nsteps * self.dt


def kdv_config(N=400, dt=1e-5, tau=1.1, t_end=1.0):
    """KdV single soliton, c = 4, x0 = 0, periodic x in [-20, 20), N = 400 (dx = 0.1)."""
    L = 40.0
    dx = L / N
    x = grid(-20.0, N, dx)
    nsteps = int(round(t_end / dt))
    return Problem(kdv(), N, dx, dt, tau, nsteps, kdv_soliton(x, 0.0, L=L), xl=-20.0,
                   exact=lambda t, x=x: kdv_soliton(x, t, L=L), meta={"c": 4.0})


def ks_config(N=1024, dt=1e-4, tau=1.3, t_end=10.0):
    """Kuramoto-Sivashinsky u_t + u u_x + u_xx + u_xxxx = 0, x in [0, 32 pi), N = 1024."""
    L = 32.0 * math.pi
    dx = L / N
    x = grid(0.0, N, dx)
    nsteps = int(round(t_end / dt))
    return Problem(ks(), N, dx, dt, tau, nsteps, ks_initial(x), xl=0.0, exact=None)


def kawahara_config(N=600, dx=0.1, dt=1e-4, tau=2.02, t_end=1.0, scheme=1, centre=0.0):
    """Example 4.5 (alpha = beta = -gamma = 1) on a periodic grid centred on the soliton."""
    L = N * dx
    xl = centre - 0.5 * L
    x = grid(xl, N, dx)
    nsteps = int(round(t_end / dt))
    return Problem(kawahara(), N, dx, dt, tau, nsteps, kawahara_soliton(x, 0.0, L=L), xl=xl,
                   scheme=scheme, exact=lambda t, x=x: kawahara_soliton(x, t, L=L))


def modified_kawahara_config(N=600, dx=0.1, dt=1e-2, tau=4.54, t_end=1.0, scheme=1):
    """Example 4.6 (a = b = k = 1), periodic on [-N dx / 2, N dx / 2)."""
    L = N * dx
    x = grid(-0.5 * L, N, dx)
    nsteps = int(round(t_end / dt))
    return Problem(modified_kawahara(), N, dx, dt, tau, nsteps, modified_kawahara_soliton(x, 0.0, L=L),
                   xl=-0.5 * L, scheme=scheme,
                   exact=lambda t, x=x: modified_kawahara_soliton(x, t, L=L))


# Examples of Sec. IV solved on a bounded grid [x_L, x_R] with exact boundary data:
# equation, x_L, x_R, exact solution phi*(x, t).
PAPER_EXAMPLES = {
    "4.1": (ks, -30.0, 30.0, ks_shock),
    "4.2": (lambda: ks(a2=-1.0), -50.0, 50.0, ks_shock2),
    "4.5": (kawahara, -30.0, 30.0, kawahara_soliton),
    "4.6": (modified_kawahara, -30.0, 30.0, modified_kawahara_soliton),
    "4.7": (kdv_kawahara, 0.0, 200.0, kdv_kawahara_soliton),
}


def bounded_config(example, dt, tau, t_end, scheme=1, dx=0.1):
    """Example 4.x on the nodes x_L, x_L + dx, ..., x_R, phi0 = phi*(x, 0); the boundary data
    are phi* at the outer nodes (``boundary_values``)."""
    make, xl, xr, ex = PAPER_EXAMPLES[example]
    N = int(round((xr - xl) / dx)) + 1
    x = grid(xl, N, dx)
    nsteps = int(round(t_end / dt))
    return Problem(make(), N, dx, dt, tau, nsteps, ex(x, 0.0), xl=xl, scheme=scheme,
                   exact=lambda t, x=x: ex(x, t), boundary="nee", exact_xt=ex,
                   meta={"example": example})


def boundary_values(p, W, n0, n):
    """[n, 2W] array: phi* at the W first then the W last nodes at times (n0 + 1..n0 + n) dt."""
    x = p.x
    xb = np.concatenate([x[:W], x[p.N - W:]])
    t = (n0 + 1 + np.arange(n, dtype=np.float64))[:, None] * p.dt
    return np.ascontiguousarray(p.exact_xt(xb[None, :], t), dtype=np.float64)


def long_grid_config(N=1 << 24, dx=0.1, dt=1e-4, tau=2.02, nsteps=1000):
    """Single long grid: Kawahara (Example 4.5) sech^4 wave, periodic, N nodes, D1Q7 scheme 1."""
    L = N * dx
    x = grid(-0.5 * L, N, dx)
    return Problem(kawahara(), N, dx, dt, tau, nsteps, kawahara_soliton(x, 0.0, L=L), xl=-0.5 * L,
                   exact=lambda t, x=x: kawahara_soliton(x, t, L=L))


# Batched KdV-Burgers ensemble: fixed dx, dt, tau for every member (chosen by an oracle
# stability scan over the sampled coefficient ranges).
def gkdv_grid_config(N=1 << 24, dx=0.1, dt=1e-4, tau=1.3, nsteps=1000, n=1.5):
    """Periodic grid of N nodes for u_t + u^n u_x + u_xxx = 0 (real n): a train of solitary
    waves (c = 1, one per 60 length units) on a background that keeps u > 0."""
    x = grid(0.0, N, dx)
    period = 60.0
    z = (x % period) - 0.5 * period
    phi0 = 0.05 + gkdv_soliton(z, 0.0, n)
    return Problem(gkdv(n), N, dx, dt, tau, nsteps, phi0, xl=0.0, meta={"n": n})


ENSEMBLE_DX = 0.1
ENSEMBLE_DT = 1e-4
ENSEMBLE_TAU = 1.15
ENSEMBLE_STEPS = 1000


def kdv_burgers_ensemble(count=4096, n_lo=256, n_hi=8192, seed=SEED, dx=ENSEMBLE_DX,
                         dt=ENSEMBLE_DT, tau=ENSEMBLE_TAU, nsteps=ENSEMBLE_STEPS):
    """``count`` independent KdV-Burgers u_t + a u u_x - b u_xx + d u_xxx = 0 problems with
    N ~ U{n_lo..n_hi}, a ~ U[1,6], b ~ U[0,0.1], d ~ U[0.5,1] and a single-soliton initial
    profile of speed c ~ U[1,4] centred in its periodic domain."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.integers(n_lo, n_hi + 1))
        a = float(rng.uniform(1.0, 6.0))
        b = float(rng.uniform(0.0, 0.1))
        d = float(rng.uniform(0.5, 1.0))
        c = float(rng.uniform(1.0, 4.0))
        L = N * dx
        x = grid(-0.5 * L, N, dx)
        phi0 = kdv_burgers_soliton_ic(x, a, d, c)
        out.append(Problem(kdv_burgers(a, b, d), N, dx, dt, tau, nsteps, phi0, xl=-0.5 * L,
                           meta={"a": a, "b": b, "d": d, "c": c, "index": i}))
    return out


def ks_spectral_reference(N=1024, t_end=10.0, h=1e-3, L=32.0 * math.pi, u0=None):
    """Reference solution of u_t + u u_x + u_xx + u_xxxx = 0 on the periodic grid of ``ks_config``:
    Fourier pseudo-spectral in x with the fourth-order exponential time differencing scheme
    ETDRK4 (Cox and Matthews 2002), its phi-function coefficients taken by contour integrals
    (Kassam and Trefethen 2005).  Used as the yardstick of discretisation error for the KS run,
    which has no closed-form solution."""
    x = grid(0.0, N, L / N)
    u = ks_initial(x) if u0 is None else np.asarray(u0, dtype=np.float64)
    v = np.fft.fft(u)
    k = 2.0 * np.pi / L * np.fft.fftfreq(N, d=1.0 / N)
    Lop = k ** 2 - k ** 4
    E = np.exp(h * Lop)
    E2 = np.exp(h * Lop / 2.0)
    M = 64
    r = np.exp(1j * np.pi * (np.arange(1, M + 1) - 0.5) / M)
    LR = h * Lop[:, None] + r[None, :]
    Q = h * np.real(np.mean((np.exp(LR / 2.0) - 1.0) / LR, axis=1))
    f1 = h * np.real(np.mean((-4.0 - LR + np.exp(LR) * (4.0 - 3.0 * LR + LR ** 2)) / LR ** 3, axis=1))
    f2 = h * np.real(np.mean((2.0 + LR + np.exp(LR) * (-2.0 + LR)) / LR ** 3, axis=1))
    f3 = h * np.real(np.mean((-4.0 - 3.0 * LR - LR ** 2 + np.exp(LR) * (4.0 - LR)) / LR ** 3, axis=1))
    g = -0.5j * k
    g[N // 2] = 0.0  # drop the odd derivative of the Nyquist mode

    def nl(w):
        return g * np.fft.fft(np.real(np.fft.ifft(w)) ** 2)

    nsteps = int(round(t_end / h))
    for _ in range(nsteps):
        Nv = nl(v)
        a = E2 * v + Q * Nv
        Na = nl(a)
        b = E2 * v + Q * Na
        Nb = nl(b)
        c = E2 * a + Q * (2.0 * Nb - Nv)
        Nc = nl(c)
        v = E * v + Nv * f1 + 2.0 * (Na + Nb) * f2 + Nc * f3
    return np.real(np.fft.ifft(v))


# Serving mix: (equation factory, dt, tau, initial profile) per request type, with (dt, tau)
# chosen by oracle scans so that every type stays bounded for 1e5 steps on dx = 0.1.
SERVING_DX = 0.1


def _serving_request(kind, N, steps, rng):
    dx = SERVING_DX
    L = N * dx
    x = grid(-0.5 * L, N, dx)
    if kind == "kdv":
        c = float(rng.uniform(1.0, 4.0))
        return Problem(kdv(), N, dx, 1e-5, 1.1, steps, kdv_soliton(x, 0.0, c=c, L=L), xl=-0.5 * L,
                       meta={"kind": kind, "c": c})
    if kind == "mkdv":
        c = float(rng.uniform(0.5, 2.0))
        return Problem(mkdv(), N, dx, 1e-5, 1.2, steps, mkdv_soliton(x, 0.0, c=c, L=L), xl=-0.5 * L,
                       meta={"kind": kind, "c": c})
    if kind == "k22":
        lam = float(rng.uniform(0.5, 1.5))
        return Problem(k22(), N, dx, 1e-4, 3.0, steps, k22_compacton(x, 0.0, lam=lam, L=L), xl=-0.5 * L,
                       meta={"kind": kind, "lam": lam})
    if kind == "ks":
        a2 = float(rng.uniform(0.5, 1.5))
        u0 = np.cos(2 * np.pi * x / L) * (1.0 + np.sin(2 * np.pi * x / L))
        return Problem(ks(a2=a2), N, dx, 1e-4, 1.3, steps, u0, xl=-0.5 * L, meta={"kind": kind, "a2": a2})
    b = float(rng.uniform(0.5, 1.0))
    return Problem(kawahara(1.0, b, -1.0), N, dx, 1e-4, 3.0, steps, kawahara_soliton(x, 0.0, 1.0, b, -1.0, L=L),
                   xl=-0.5 * L, meta={"kind": "kawahara", "beta": b})


SERVING_KINDS = ("kdv", "mkdv", "k22", "ks", "kawahara")


def serving_requests(count, rate=2000.0, seed=SEED, n_lo=128, n_hi=65536, s_lo=1000, s_hi=100000):
    """``count`` requests with Poisson arrivals of mean ``rate`` per second: (arrival time,
    Problem).  Equation ~ uniform over KdV, mKdV, K(2,2) compacton, KS and Kawahara; N
    log-uniform in [n_lo, n_hi]; steps uniform in [s_lo, s_hi]; coefficients and soliton or
    compacton parameters drawn from the seed."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate))
        kind = SERVING_KINDS[int(rng.integers(0, len(SERVING_KINDS)))]
        N = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        steps = int(rng.integers(s_lo, s_hi + 1))
        out.append((t, _serving_request(kind, N, steps, rng)))
    return out

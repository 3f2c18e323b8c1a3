"""Plain FP64 CPU oracle of the LBGK model of Shi, He and Guo (arXiv:0907.1720).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline leg and ``--impl reference``) may import this
package.  The CUDA library never calls it and shares no code with it.

The arithmetic lives in ``lbhpde_oracle.c`` (compiled with ``-ffp-contract=off``
so that every operation is a separately rounded IEEE double operation); this
module only marshals numpy arrays through ctypes.

An equation is given as ``(alpha, pi)``: ``alpha[k-1]`` is the coefficient
alpha_k of Eq. (NPDE) and ``pi[k-1][p]`` is the coefficient of phi**p in
Pi_k(phi).  ``alpha[0]`` multiplies Pi_1 (the paper fixes alpha_1 = 1).

Parity status of each function: every function is pinned by a test in
``tests/test_oracle_pins.py`` except the observed convergence order, which the
paper does not state ("parity unpinned").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "lbhpde_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbhpde_oracle.so")

OK, ERR_ARG, ERR_TAU_SINGULAR, ERR_DEGREE = 0, 1, 2, 3
NO_AUX_CORRECTION = 0x100  # scheme flag: leave A_40, A_50, A_60 out
_ERRORS = {ERR_ARG: "invalid argument", ERR_TAU_SINGULAR: "tau_k = 0 (singular relaxation time)",
           ERR_DEGREE: "polynomial degree too high"}

_lock = threading.Lock()
_lib = None


class OracleError(ValueError):
    def __init__(self, code):
        super().__init__(_ERRORS.get(code, f"oracle error {code}"))
        self.code = code


def compile_source(src_path: str, out_path: str) -> str:
    """Compile an oracle source file with plain -O2 and no FMA contraction."""
    tmp = out_path + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, src_path, "-lm"])
    os.replace(tmp, out_path)
    return out_path


def build(force: bool = False) -> str:
    """Compile the oracle (once; again only when the source is newer)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(SOURCE):
        compile_source(SOURCE, _LIB_PATH)
    return _LIB_PATH


def bind(path: str):
    """Load a compiled oracle and declare its C signatures."""
    lib = ctypes.CDLL(path)
    D = ctypes.POINTER(ctypes.c_double)
    V = ctypes.c_void_p
    i, l, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
    lib.oracle_model_size.restype = ctypes.c_size_t
    lib.oracle_model_init.argtypes = [V, i, D, D, i, d, d, d, i, i]
    lib.oracle_model_init.restype = i
    lib.oracle_model_init_nu.argtypes = [V, i, D, D, D, i, d, d, d, d, i, i]
    lib.oracle_model_init_nu.restype = i
    lib.oracle_moments.argtypes = [V, d, D]
    lib.oracle_feq.argtypes = [V, d, D]
    lib.oracle_dfeq.argtypes = [V, d, D]
    lib.oracle_edf.argtypes = [i, D, D]
    lib.oracle_init.argtypes = [V, l, D, D]
    lib.oracle_step.argtypes = [V, l, D, D, l]
    lib.oracle_step_nee.argtypes = [V, l, D, D, l, D, i]
    lib.oracle_phi.argtypes = [V, l, D, D]
    lib.oracle_error_E.argtypes = [l, D, D]
    lib.oracle_error_E.restype = d
    lib.oracle_model_b.argtypes = [V]
    lib.oracle_model_inexact.argtypes = [V]
    lib.oracle_model_params.argtypes = [V, D, D, D]
    lib.oracle_aux_moment.argtypes = [V, i, d]
    lib.oracle_aux_moment.restype = d
    lib.oracle_run.argtypes = [i, D, D, i, d, d, d, i, i, l, D, l, D]
    lib.oracle_run.restype = i
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
        return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pack(alpha, pi):
    alpha = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).ravel())
    m = alpha.size
    rows = [list(map(float, r)) for r in pi]
    if len(rows) != m:
        raise ValueError("need one Pi_k per alpha_k")
    ncoef = max(1, max(len(r) for r in rows))
    P = np.zeros((m, ncoef), dtype=np.float64)
    for k, r in enumerate(rows):
        P[k, :len(r)] = r
    return m, alpha, np.ascontiguousarray(P), ncoef


def edf(b: int, pibar, lib=None) -> np.ndarray:
    """f^eq from the scaled moments by the written-out Eq. (EDF5)/(EDF7)."""
    lib = lib or _load()
    P = np.ascontiguousarray(np.asarray(pibar, dtype=np.float64))
    out = np.zeros(b)
    lib.oracle_edf(b, _dp(P), _dp(out))
    return out


class Model:
    """One LBGK model (lattice, moments, relaxation) built by the oracle.  With ``nu`` and
    ``pi_nu`` (``pi_nu[k-1][p]`` = coefficient of phi**(p + nu) in Pi_k, p >= 1) the Pi_k carry
    terms with the real exponent nu as well."""

    def __init__(self, alpha, pi, dx, dt, tau, lattice=0, scheme=1, lib=None, nu=0.0, pi_nu=None):
        self._lib = lib = lib or _load()
        self._buf = ctypes.create_string_buffer(lib.oracle_model_size())
        if pi_nu is not None:
            rows = [list(r) for r in pi]
            rows_nu = [list(r) for r in pi_nu]
            ncoef = max(1, max(len(r) for r in rows + rows_nu))
            pi = [r + [0.0] * (ncoef - len(r)) for r in rows]
            pi_nu = [r + [0.0] * (ncoef - len(r)) for r in rows_nu]
        m, a, P, ncoef = _pack(alpha, pi)
        if pi_nu is not None:
            _, _, Pn, _ = _pack(alpha, pi_nu)
            rc = lib.oracle_model_init_nu(self._buf, m, _dp(a), _dp(P), _dp(Pn), ncoef, float(nu), float(dx),
                                          float(dt), float(tau), int(lattice), int(scheme))
        else:
            rc = lib.oracle_model_init(self._buf, m, _dp(a), _dp(P), ncoef, float(dx), float(dt),
                                       float(tau), int(lattice), int(scheme))
        if rc != OK:
            raise OracleError(rc)
        self.b = lib.oracle_model_b(self._buf)
        self.inexact = bool(lib.oracle_model_inexact(self._buf))
        tk, beta, A = np.zeros(7), np.zeros(7), np.zeros(3)
        lib.oracle_model_params(self._buf, _dp(tk), _dp(beta), _dp(A))
        self.taus, self.beta, self.A = tk, beta, A
        self.dx, self.dt, self.tau = float(dx), float(dt), float(tau)
        self.c = self.dx / self.dt

    def moments(self, phi: float) -> np.ndarray:
        out = np.zeros(self.b)
        self._lib.oracle_moments(self._buf, float(phi), _dp(out))
        return out

    def feq(self, phi: float) -> np.ndarray:
        out = np.zeros(self.b)
        self._lib.oracle_feq(self._buf, float(phi), _dp(out))
        return out

    def dfeq(self, phi: float) -> np.ndarray:
        out = np.zeros(self.b)
        self._lib.oracle_dfeq(self._buf, float(phi), _dp(out))
        return out

    def aux_moment(self, k: int, phi: float) -> float:
        return self._lib.oracle_aux_moment(self._buf, int(k), float(phi))

    def init(self, phi0) -> np.ndarray:
        phi0 = np.ascontiguousarray(np.asarray(phi0, dtype=np.float64))
        f = np.zeros((self.b, phi0.size))
        self._lib.oracle_init(self._buf, phi0.size, _dp(phi0), _dp(f))
        return f

    def step(self, f: np.ndarray, nsteps: int) -> np.ndarray:
        assert f.flags.c_contiguous and f.dtype == np.float64 and f.shape[0] == self.b
        tmp = np.empty_like(f)
        self._lib.oracle_step(self._buf, f.shape[1], _dp(f), _dp(tmp), int(nsteps))
        return f

    def step_nee(self, f: np.ndarray, phib, depth: int = 2) -> np.ndarray:
        """len(phib) steps with the non-equilibrium extrapolation boundary; phib[n] holds the
        prescribed phi at time (n + 1) dt at the W left then the W right boundary nodes, and
        the outer nodes extrapolate from the node ``depth`` places inside them."""
        assert f.flags.c_contiguous and f.dtype == np.float64 and f.shape[0] == self.b
        pb = np.ascontiguousarray(np.asarray(phib, dtype=np.float64))
        W = (self.b - 1) // 2
        assert pb.ndim == 2 and pb.shape[1] == 2 * W
        if depth < 1 or f.shape[1] < 2 * (W + depth):
            raise OracleError(ERR_ARG)
        tmp = np.empty_like(f)
        self._lib.oracle_step_nee(self._buf, f.shape[1], _dp(f), _dp(tmp), pb.shape[0], _dp(pb), int(depth))
        return f

    def phi(self, f: np.ndarray) -> np.ndarray:
        out = np.zeros(f.shape[1])
        self._lib.oracle_phi(self._buf, f.shape[1], _dp(f), _dp(out))
        return out


def run(alpha, pi, dx, dt, tau, phi0, nsteps, lattice=0, scheme=1, lib=None) -> np.ndarray:
    """phi after ``nsteps`` steps from f = f^eq(phi0) on a periodic grid."""
    lib = lib or _load()
    m, a, P, ncoef = _pack(alpha, pi)
    phi0 = np.ascontiguousarray(np.asarray(phi0, dtype=np.float64))
    out = np.zeros(phi0.size)
    rc = lib.oracle_run(m, _dp(a), _dp(P), ncoef, float(dx), float(dt), float(tau), int(lattice),
                        int(scheme), phi0.size, _dp(phi0), int(nsteps), _dp(out))
    if rc != OK:
        raise OracleError(rc)
    return out


def run_problem(p, nsteps=None, lib=None) -> np.ndarray:
    """Run a ``workloads.Problem``-like object (eq, dx, dt, tau, scheme, phi0, nsteps)."""
    return run(p.eq.alpha, p.eq.pi, p.dx, p.dt, p.tau, p.phi0,
               p.nsteps if nsteps is None else nsteps, lattice=p.eq.lattice, scheme=p.scheme, lib=lib)


def error_E(phi, phistar) -> float:
    """Global relative error E of Sec. IV: sum |phi - phi*| / sum |phi*|."""
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64))
    ps = np.ascontiguousarray(np.asarray(phistar, dtype=np.float64))
    return _load().oracle_error_E(phi.size, _dp(phi), _dp(ps))


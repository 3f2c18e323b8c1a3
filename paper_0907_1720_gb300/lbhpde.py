"""Python binding of the C ABI in ``include/lbhpde.h`` (ctypes; argument marshalling only).

Every step of the solver runs in the CUDA library ``_build/liblbhpde.so``; this module
only converts Python/numpy/torch arguments into the C structures and pointers.  If the
library has not been built, :func:`lib` raises ``RuntimeError`` -- there is no fallback.

Low-level functions carry the C names (``lbhpde_model``, ``lbhpde_create`` ...).  The
classes :class:`Solver` and :class:`Batch` wrap a handle for convenience; device memory
is obtained through torch's caching allocator and work runs on the torch stream current
at creation time.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbhpde.so")

OK, ERR_ARG, ERR_TAU_SINGULAR, ERR_OOM, ERR_DIVERGED, PENDING, ERR_TIMEOUT, ERR_CUDA, ERR_NOT_FOUND, \
    ERR_UNSUPPORTED = range(10)
FP64, FP32_DEV = 0, 1
PERIODIC = 0
NEE = 1  # bounded grid, non-equilibrium extrapolation boundary (depth 2)


def nee_depth(d):
    """Boundary code of the non-equilibrium extrapolation boundary with extrapolation depth d."""
    return NEE | (int(d) << 8)

NO_AUX_CORRECTION = 0x100  # or-ed into scheme: leave A_40, A_50, A_60 out
PI_ZERO, PI_PHI, PI_POWER, PI_POLY, PI_POLY_NU = 0, 1, 2, 3, 4
PI_NCOEF = 8
MAX_DEG = 31
NU_TERMS = 64
KERNEL_AUTO, KERNEL_STREAM, KERNEL_ONCHIP, KERNEL_HALO = 0, 1, 2, 3


class lbhpde_pi(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("power", ctypes.c_int), ("coef", ctypes.c_double * PI_NCOEF),
                ("nu", ctypes.c_double), ("coef_nu", ctypes.c_double * PI_NCOEF)]


class lbhpde_model_info(ctypes.Structure):
    _fields_ = [("b", ctypes.c_int), ("m", ctypes.c_int), ("scheme", ctypes.c_int), ("D", ctypes.c_int),
                ("inexact", ctypes.c_int), ("c", ctypes.c_double), ("omega", ctypes.c_double),
                ("tk", ctypes.c_double * 7), ("beta", ctypes.c_double * 7), ("A", ctypes.c_double * 3),
                ("feq", (ctypes.c_double * (MAX_DEG + 1)) * 7), ("coef", (ctypes.c_double * (MAX_DEG + 1)) * 7),
                ("nu", ctypes.c_double), ("nu_rows", ctypes.c_int), ("nu_deg", ctypes.c_int),
                ("gfeq", (ctypes.c_double * NU_TERMS) * 7), ("gcoef", (ctypes.c_double * NU_TERMS) * 7)]


class lbhpde_allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)),
                ("release", ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                             ctypes.c_void_p)),
                ("user", ctypes.c_void_p)]


class lbhpde_diag(ctypes.Structure):
    _fields_ = [("sum_phi", ctypes.c_double), ("max_abs_phi", ctypes.c_double), ("nonfinite", ctypes.c_long),
                ("err_E", ctypes.c_double), ("err_L2", ctypes.c_double), ("steps", ctypes.c_long)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class lbhpde_instance(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("alpha", ctypes.c_double * 6), ("pi", lbhpde_pi * 6), ("N", ctypes.c_long),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("tau", ctypes.c_double),
                ("lattice", ctypes.c_int), ("scheme", ctypes.c_int), ("boundary", ctypes.c_int)]


class lbhpde_request(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("alpha", ctypes.c_double * 6), ("pi", lbhpde_pi * 6), ("N", ctypes.c_long),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("tau", ctypes.c_double),
                ("lattice", ctypes.c_int), ("scheme", ctypes.c_int), ("nsteps", ctypes.c_long),
                ("phi0", ctypes.POINTER(ctypes.c_double))]


class lbhpde_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("steps_done", ctypes.c_long), ("submit_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("finish_s", ctypes.c_double), ("sum_phi", ctypes.c_double),
                ("nonfinite", ctypes.c_long)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class lbhpde_server_info(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_long), ("in_flight", ctypes.c_long), ("completed", ctypes.c_long),
                ("node_updates", ctypes.c_double), ("bytes_in_use", ctypes.c_size_t),
                ("bytes_total", ctypes.c_size_t), ("launches", ctypes.c_long), ("error", ctypes.c_int),
                ("gpu_busy_s", ctypes.c_double), ("host_admit_s", ctypes.c_double), ("host_setup_s", ctypes.c_double),
                ("host_plan_s", ctypes.c_double), ("host_launch_s", ctypes.c_double), ("host_wait_s", ctypes.c_double),
                ("host_retire_s", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class LbhpdeError(RuntimeError):
    def __init__(self, code, where=""):
        msg = lib().lbhpde_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes)
_V, _I, _L, _D, _S = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_size_t
_P = ctypes.POINTER
_SIGS = {
    "lbhpde_model": (_I, [_I, _P(_D), _P(lbhpde_pi), _D, _D, _D, _I, _I, _P(lbhpde_model_info)]),
    "lbhpde_create": (_I, [_P(_V), _I, _P(_D), _P(lbhpde_pi), _L, _D, _D, _D, _I, _I, _I, _I, _V,
                           _P(lbhpde_allocator)]),
    "lbhpde_set_phi": (_I, [_V, _V, _I]),
    "lbhpde_step": (_I, [_V, _L]),
    "lbhpde_step_nee": (_I, [_V, _L, _V, _I]),
    "lbhpde_read_phi": (_I, [_V, _V, _I]),
    "lbhpde_diagnostics": (_I, [_V, _V, _P(lbhpde_diag)]),
    "lbhpde_kernel_launches": (_I, [_V, _P(ctypes.c_longlong)]),
    "lbhpde_set_kernel": (_I, [_V, _I, _I, _I]),
    "lbhpde_get_model": (_I, [_V, _P(lbhpde_model_info)]),
    "lbhpde_autotune": (_I, [_I, _I, _I, _P(_I), _P(_I), _P(_D)]),
    "lbhpde_set_tuning": (_I, [_I, _I, _I, _I, _I]),
    "lbhpde_destroy": (_I, [_V]),
    "lbhpde_strerror": (ctypes.c_char_p, [_I]),
    "lbhpde_batch_create": (_I, [_P(_V), _I, _P(lbhpde_instance), _I, _V, _P(lbhpde_allocator)]),
    "lbhpde_batch_set_phi": (_I, [_V, _V, _I]),
    "lbhpde_batch_step": (_I, [_V, _L]),
    "lbhpde_batch_step_nee": (_I, [_V, _L, _V, _L, _I]),
    "lbhpde_batch_read_phi": (_I, [_V, _V, _I]),
    "lbhpde_batch_diagnostics": (_I, [_V, _V, _P(lbhpde_diag)]),
    "lbhpde_batch_kernel_launches": (_I, [_V, _P(ctypes.c_longlong)]),
    "lbhpde_batch_set_kernel": (_I, [_V, _I, _I, _I]),
    "lbhpde_batch_size": (_I, [_V, _P(_L), _P(_S)]),
    "lbhpde_batch_destroy": (_I, [_V]),
    "lbhpde_batch_checkpoint_size": (_I, [_V, _P(_S)]),
    "lbhpde_batch_save": (_I, [_V, _V, _S]),
    "lbhpde_batch_load": (_I, [_V, _V, _S]),
    "lbhpde_checkpoint_size": (_I, [_V, _P(_S)]),
    "lbhpde_save": (_I, [_V, _V, _S]),
    "lbhpde_load": (_I, [_V, _V, _S]),
    "lbhpde_phi_diagnostics_noalloc": (_I, [_V, _L, _V, _P(lbhpde_diag), _V]),
    "lbhpde_server_create": (_I, [_P(_V), _I, _S, _I, _I, _I]),
    "lbhpde_submit": (_I, [_V, _P(lbhpde_request), _P(ctypes.c_uint64)]),
    "lbhpde_submit_nee": (_I, [_V, _P(lbhpde_request), _I, _V, _P(ctypes.c_uint64)]),
    "lbhpde_poll": (_I, [_V, ctypes.c_uint64, _V, _P(lbhpde_result)]),
    "lbhpde_wait": (_I, [_V, ctypes.c_uint64, _D, _V, _P(lbhpde_result)]),
    "lbhpde_server_stats": (_I, [_V, _P(lbhpde_server_info)]),
    "lbhpde_server_destroy": (_I, [_V]),
}
EXPORTED = tuple(_SIGS)


def lib():
    """The loaded CUDA library; raises RuntimeError when it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run __graft_entry__.build() or python -m paper_0907_1720_gb300.build)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype, fn.argtypes = res, args
            _lib = L
        return _lib


def _check(code, where):
    if code != OK:
        raise LbhpdeError(code, where)


# ------------------------------------------------------------------ marshalling

def make_pi(coefs, nu=0.0, coefs_nu=None) -> lbhpde_pi:
    """A Pi_k from polynomial coefficients (coef[p] of phi**p), plus coefs_nu[p] of phi**(p + nu)
    when the equation has a real exponent nu; uses the menu's closed forms."""
    cn = [float(v) for v in (coefs_nu or ())]
    while cn and cn[-1] == 0.0:
        cn.pop()
    if cn:
        if len(coefs) > PI_NCOEF or len(cn) > PI_NCOEF:
            raise ValueError("Pi_k degree above 7")
        p = lbhpde_pi()
        p.kind, p.nu = PI_POLY_NU, float(nu)
        for i, v in enumerate(coefs):
            p.coef[i] = float(v)
        for i, v in enumerate(cn):
            p.coef_nu[i] = v
        return p
    c = [float(v) for v in coefs]
    while c and c[-1] == 0.0:
        c.pop()
    p = lbhpde_pi()
    if not c:
        p.kind = PI_ZERO
    elif c == [0.0, 1.0]:
        p.kind = PI_PHI
    elif len(c) > 1 and all(v == 0.0 for v in c[:-1]) and c[-1] == 1.0:
        p.kind, p.power = PI_POWER, len(c) - 1
    else:
        if len(c) > PI_NCOEF:
            raise ValueError("Pi_k degree above 7")
        p.kind = PI_POLY
        for i, v in enumerate(c):
            p.coef[i] = v
    return p


def _pis(pi, nu=0.0, pi_nu=None):
    rows_nu = pi_nu if pi_nu is not None else [()] * len(pi)
    return [make_pi(r, nu, rn) for r, rn in zip(pi, rows_nu)]


def _eq_args(alpha, pi, nu=0.0, pi_nu=None):
    m = len(alpha)
    a = (ctypes.c_double * m)(*[float(v) for v in alpha])
    P = (lbhpde_pi * m)(*_pis(pi, nu, pi_nu))
    return m, a, P


def lbhpde_model(alpha, pi, dx, dt, tau, lattice=0, scheme=1, nu=0.0, pi_nu=None) -> lbhpde_model_info:
    """Step a0 on the host: the model the library builds for one equation (with nu and pi_nu,
    pi_nu[k-1][p] the coefficient of phi**(p + nu) in Pi_k)."""
    m, a, P = _eq_args(alpha, pi, nu, pi_nu)
    out = lbhpde_model_info()
    _check(lib().lbhpde_model(m, a, P, dx, dt, tau, lattice, scheme, ctypes.byref(out)), "lbhpde_model")
    return out


def model_coeffs(info: lbhpde_model_info):
    """(feq[b][D+1], coef[b][D+1]) as numpy arrays; for a real-exponent model (nu_rows > 1)
    (gfeq[b][A+1][Dg+1], gcoef[b][A+1][Dg+1]) with f^eq_j = sum_a (phi**nu)**a sum_i g[j][a][i] phi**i."""
    b, D = info.b, info.D
    if info.nu_rows > 1:
        R, Dg = info.nu_rows, info.nu_deg
        g = np.array([[info.gfeq[j][p] for p in range(R * (Dg + 1))] for j in range(b)]).reshape(b, R, Dg + 1)
        gc = np.array([[info.gcoef[j][p] for p in range(R * (Dg + 1))] for j in range(b)]).reshape(b, R, Dg + 1)
        return g, gc
    feq = np.array([[info.feq[j][p] for p in range(D + 1)] for j in range(b)])
    coef = np.array([[info.coef[j][p] for p in range(D + 1)] for j in range(b)])
    return feq, coef


def make_instance(eq, N, dx, dt, tau, scheme=1, boundary=PERIODIC) -> lbhpde_instance:
    I = lbhpde_instance()
    I.m = eq.m
    pis = _pis(eq.pi, getattr(eq, "nu", 0.0), getattr(eq, "pi_nu", None))
    for k in range(eq.m):
        I.alpha[k] = float(eq.alpha[k])
        I.pi[k] = pis[k]
    I.N, I.dx, I.dt, I.tau, I.lattice, I.scheme = int(N), float(dx), float(dt), float(tau), int(eq.lattice), int(scheme)
    I.boundary = int(boundary)
    return I


def _boundary_code(p):
    """Boundary code of a workloads.Problem: periodic, or NEE with meta['depth'] (default 2)."""
    if getattr(p, "boundary", "periodic") == "nee":
        return nee_depth(p.meta.get("depth", 2))
    return PERIODIC


def _on_device(x):
    return hasattr(x, "data_ptr") and bool(getattr(x, "is_cuda", False))


def _host_array(x):
    """A C-contiguous float64 view of host data (a CPU tensor's own memory, so page-locked memory
    stays page-locked), copied only when its layout or type requires it."""
    if hasattr(x, "data_ptr"):
        x = x.detach().numpy()
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _in_arg(x, n=None):
    """(pointer, on_device, keep-alive) for a double input: a CUDA tensor is passed as device
    memory, anything else as host memory."""
    if x is None:
        return None, 0, None
    if _on_device(x):
        return ctypes.c_void_p(x.data_ptr()), 1, x
    a = _host_array(x)
    if n is not None and a.size != n:
        raise ValueError(f"input of {a.size} values, {n} expected")
    return a.ctypes.data_as(ctypes.c_void_p), 0, a


def _out_arg(out, n):
    """(pointer, on_device, result, host array) for a [n] double output: a CUDA tensor (device),
    a float64 host array or CPU tensor written in place, or a new array."""
    if out is None:
        a = np.empty(n)
        return a.ctypes.data_as(ctypes.c_void_p), 0, a, a
    if _on_device(out):
        return ctypes.c_void_p(out.data_ptr()), 1, out, None
    a = out.detach().numpy() if hasattr(out, "data_ptr") else out
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.size == n):
        raise ValueError(f"output: a contiguous float64 buffer of {n} values expected")
    return a.ctypes.data_as(ctypes.c_void_p), 0, out, a


def _phib_arg(phib):
    """(pointer, on_device, keep-alive) for boundary values given as a tensor or array."""
    return _in_arg(phib)


def autotune(precision, lattice, degree):
    """lbhpde_autotune: (nodes per thread, steps per window, node-updates/s) of the fastest
    on-chip configuration; later batches use it."""
    K, T, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().lbhpde_autotune(int(precision), int(lattice), int(degree), ctypes.byref(K), ctypes.byref(T),
                                 ctypes.byref(r)), "lbhpde_autotune")
    return K.value, T.value, r.value


def set_tuning(precision, lattice, degree, nodes_per_thread, steps_per_launch):
    """lbhpde_set_tuning: record a tuned on-chip pair without timing (later batches use it)."""
    _check(lib().lbhpde_set_tuning(int(precision), int(lattice), int(degree), int(nodes_per_thread),
                                   int(steps_per_launch)), "lbhpde_set_tuning")


def tau_sweep(problem, taus, precision=FP64, nsteps=None, phib=None):
    """The global relative error E (Sec. IV) of ``problem`` for every tau in ``taus``, all solved
    in one batch: one member per tau, the same grid, initial profile and boundary data.  Sec. IV
    picks tau_opt per lattice speed as the tau with the smallest error; this scans for it.
    problem: a workloads.Problem with ``exact`` (phi* at t_end) and, for a bounded grid,
    ``boundary == "nee"`` and ``exact_xt``; phib: [nsteps, 2W] boundary values (default: phi*
    at the outer nodes).  Returns (taus, E) as numpy arrays."""
    import copy

    import torch

    from . import workloads as W

    n = problem.nsteps if nsteps is None else int(nsteps)
    members = []
    for t in taus:
        q = copy.copy(problem)
        q.tau, q.nsteps = float(t), n
        members.append(q)
    b = Batch(members, precision=precision)
    try:
        b.set_phi(np.tile(np.asarray(problem.phi0, dtype=np.float64), len(members)))
        if problem.boundary == "nee":
            if phib is None:
                Wd = 3 if (problem.eq.lattice == 7 or problem.eq.m > 4) else 2
                phib = W.boundary_values(problem, Wd, 0, n)
            b.step_nee(n, phib, 0)
        else:
            b.step(n)
        ex = np.tile(np.asarray(problem.exact(n * problem.dt), dtype=np.float64), len(members))
        d = b.diagnostics(torch.tensor(ex, device="cuda", dtype=torch.float64))
        return np.asarray(taus, dtype=np.float64), np.array(d["err_E"])
    finally:
        b.close()


# ------------------------------------------------------------ torch plumbing

_torch_alloc_keep = []


def torch_allocator():
    """An lbhpde_allocator that draws device memory from torch's caching allocator."""
    import torch

    dev = torch.cuda.current_device()

    @ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream if stream else None)
        except Exception:
            return None

    @ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    def _release(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a = lbhpde_allocator(_alloc, _release, None)
    _torch_alloc_keep.append((a, _alloc, _release))
    return a


def _current_stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ----------------------------------------------------------------- handles

def _save(h, size_fn, save_fn, where):
    n = ctypes.c_size_t()
    _check(size_fn(h, ctypes.byref(n)), where)
    buf = np.empty(n.value, dtype=np.uint8)
    _check(save_fn(h, buf.ctypes.data_as(ctypes.c_void_p), buf.size), where)
    return buf


def _load(h, buf, load_fn, where):
    a = np.ascontiguousarray(np.frombuffer(buf, dtype=np.uint8) if isinstance(buf, (bytes, bytearray)) else buf,
                             dtype=np.uint8)
    _check(load_fn(h, a.ctypes.data_as(ctypes.c_void_p), a.size), where)


class Solver:
    """One instance (lbhpde_create ... lbhpde_destroy), periodic or bounded (boundary=NEE)."""

    def __init__(self, eq, N, dx, dt, tau, scheme=1, precision=FP64, stream=None, use_torch=True,
                 boundary=PERIODIC):
        m, a, P = _eq_args(eq.alpha, eq.pi, getattr(eq, "nu", 0.0), getattr(eq, "pi_nu", None))
        self._alloc = torch_allocator() if use_torch else None
        st = stream if stream is not None else (_current_stream() if use_torch else None)
        h = ctypes.c_void_p()
        _check(lib().lbhpde_create(ctypes.byref(h), m, a, P, int(N), float(dx), float(dt), float(tau),
                                   int(eq.lattice), int(scheme), int(precision), int(boundary), st,
                                   ctypes.byref(self._alloc) if self._alloc else None), "lbhpde_create")
        self.h, self.N = h, int(N)

    @classmethod
    def for_problem(cls, p, precision=FP64, **kw):
        kw.setdefault("boundary", _boundary_code(p))
        return cls(p.eq, p.N, p.dx, p.dt, p.tau, scheme=p.scheme, precision=precision, **kw)

    def set_kernel(self, kernel=KERNEL_AUTO, nodes_per_thread=0, steps_per_launch=0):
        _check(lib().lbhpde_set_kernel(self.h, kernel, nodes_per_thread, steps_per_launch), "lbhpde_set_kernel")
        return self

    def set_phi(self, phi0):
        """phi0: [N] doubles, a CUDA tensor (device) or host memory (array or CPU tensor)."""
        ptr, dev, keep = _in_arg(phi0, self.N)
        _check(lib().lbhpde_set_phi(self.h, ptr, dev), "lbhpde_set_phi")
        return self

    def step(self, nsteps):
        _check(lib().lbhpde_step(self.h, int(nsteps)), "lbhpde_step")
        return self

    def step_nee(self, nsteps, phib):
        """nsteps bounded steps; phib: [nsteps, 2W] boundary values (array or device tensor)."""
        ptr, dev, keep = _phib_arg(phib)
        _check(lib().lbhpde_step_nee(self.h, int(nsteps), ptr, dev), "lbhpde_step_nee")
        return self

    def read_phi(self, out=None, check=True):
        """phi into out ([N] doubles: a CUDA tensor, a host array or CPU tensor; None: a new array)."""
        ptr, dev, res, keep = _out_arg(out, self.N)
        rc = lib().lbhpde_read_phi(self.h, ptr, dev)
        if check or rc != ERR_DIVERGED:
            _check(rc, "lbhpde_read_phi")
        return res

    def diagnostics(self, phistar_device=None) -> dict:
        d = lbhpde_diag()
        ptr = ctypes.c_void_p(phistar_device.data_ptr()) if phistar_device is not None else None
        rc = lib().lbhpde_diagnostics(self.h, ptr, ctypes.byref(d))
        if rc not in (OK, ERR_DIVERGED):
            _check(rc, "lbhpde_diagnostics")
        return d.as_dict()

    def kernel_launches(self) -> int:
        """lbhpde_kernel_launches: kernels launched since the handle was made."""
        n = ctypes.c_longlong()
        _check(lib().lbhpde_kernel_launches(self.h, ctypes.byref(n)), "lbhpde_kernel_launches")
        return n.value

    def model(self) -> lbhpde_model_info:
        out = lbhpde_model_info()
        _check(lib().lbhpde_get_model(self.h, ctypes.byref(out)), "lbhpde_get_model")
        return out

    def save(self) -> np.ndarray:
        """lbhpde_save: the instance's checkpoint as a byte array."""
        return _save(self.h, lib().lbhpde_checkpoint_size, lib().lbhpde_save, "lbhpde_save")

    def load(self, buf):
        """lbhpde_load: restore a checkpoint made by save() on an instance of the same layout."""
        _load(self.h, buf, lib().lbhpde_load, "lbhpde_load")
        return self

    def close(self):
        if self.h:
            lib().lbhpde_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many instances stepped together (lbhpde_batch_*); bounded members come from problems
    with boundary == "nee"."""

    def __init__(self, problems, precision=FP32_DEV, stream=None, use_torch=True):
        members = (lbhpde_instance * len(problems))(
            *[make_instance(p.eq, p.N, p.dx, p.dt, p.tau, p.scheme, _boundary_code(p)) for p in problems])
        self._alloc = torch_allocator() if use_torch else None
        st = stream if stream is not None else (_current_stream() if use_torch else None)
        h = ctypes.c_void_p()
        _check(lib().lbhpde_batch_create(ctypes.byref(h), len(problems), members, int(precision), st,
                                         ctypes.byref(self._alloc) if self._alloc else None), "lbhpde_batch_create")
        self.h = h
        self.sizes = [int(p.N) for p in problems]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.total = int(self.offsets[-1])

    def set_kernel(self, kernel=KERNEL_AUTO, nodes_per_thread=0, steps_per_launch=0):
        _check(lib().lbhpde_batch_set_kernel(self.h, kernel, nodes_per_thread, steps_per_launch),
               "lbhpde_batch_set_kernel")
        return self

    def set_phi(self, phi0):
        """phi0: [sum N] doubles, a CUDA tensor (device) or host memory (array or CPU tensor)."""
        ptr, dev, keep = _in_arg(phi0, self.total)
        _check(lib().lbhpde_batch_set_phi(self.h, ptr, dev), "lbhpde_batch_set_phi")
        return self

    def step(self, nsteps):
        _check(lib().lbhpde_batch_step(self.h, int(nsteps)), "lbhpde_batch_step")
        return self

    def step_nee(self, nsteps, phib, member_stride=0):
        """nsteps steps; member i's boundary values are the [nsteps, 2W_i] doubles at
        phib + i * member_stride (0: one array shared by all bounded members)."""
        ptr, dev, keep = _phib_arg(phib)
        _check(lib().lbhpde_batch_step_nee(self.h, int(nsteps), ptr, int(member_stride), dev),
               "lbhpde_batch_step_nee")
        return self

    def read_phi(self, out=None, check=True):
        """phi into out ([sum N] doubles: a CUDA tensor, a host array or CPU tensor; None: a new
        array)."""
        ptr, dev, res, keep = _out_arg(out, self.total)
        rc = lib().lbhpde_batch_read_phi(self.h, ptr, dev)
        if check or rc != ERR_DIVERGED:
            _check(rc, "lbhpde_batch_read_phi")
        return res

    def split(self, flat):
        return [flat[self.offsets[i]:self.offsets[i + 1]] for i in range(len(self.sizes))]

    def diagnostics(self, phistar_device=None):
        """One record per member (numpy structured array over the C records, no copy):
        r["sum_phi"], r["max_abs_phi"], r["nonfinite"], r["err_E"], r["err_L2"], r["steps"]."""
        out = (lbhpde_diag * len(self.sizes))()
        ptr = ctypes.c_void_p(phistar_device.data_ptr()) if phistar_device is not None else None
        rc = lib().lbhpde_batch_diagnostics(self.h, ptr, out)
        if rc not in (OK, ERR_DIVERGED):
            _check(rc, "lbhpde_batch_diagnostics")
        return np.ctypeslib.as_array(out)

    def kernel_launches(self) -> int:
        """lbhpde_batch_kernel_launches: kernels launched since the batch was made."""
        n = ctypes.c_longlong()
        _check(lib().lbhpde_batch_kernel_launches(self.h, ctypes.byref(n)), "lbhpde_batch_kernel_launches")
        return n.value

    def size(self):
        n, b = ctypes.c_long(), ctypes.c_size_t()
        _check(lib().lbhpde_batch_size(self.h, ctypes.byref(n), ctypes.byref(b)), "lbhpde_batch_size")
        return n.value, b.value

    def save(self) -> np.ndarray:
        """lbhpde_batch_save: the batch's checkpoint as a byte array."""
        return _save(self.h, lib().lbhpde_batch_checkpoint_size, lib().lbhpde_batch_save, "lbhpde_batch_save")

    def load(self, buf):
        """lbhpde_batch_load: restore a checkpoint made by save() on a batch of the same layout."""
        _load(self.h, buf, lib().lbhpde_batch_load, "lbhpde_batch_load")
        return self

    def close(self):
        if self.h:
            lib().lbhpde_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (lbhpde_server_*)."""

    def __init__(self, precision=FP32_DEV, device_bytes=1 << 30, max_active=4096, steps_per_block=256, device=None):
        if device is None:
            import torch
            device = torch.cuda.current_device()
        h = ctypes.c_void_p()
        _check(lib().lbhpde_server_create(ctypes.byref(h), int(precision), int(device_bytes), int(max_active),
                                          int(steps_per_block), int(device)), "lbhpde_server_create")
        self.h = h
        self.sizes = {}

    def submit(self, eq, N, dx, dt, tau, nsteps, phi0, scheme=1, boundary=PERIODIC, phib=None) -> int:
        """A request; a bounded one (boundary NEE or nee_depth(d)) with its [nsteps][2W] boundary
        values phib (host, copied)."""
        q = lbhpde_request()
        q.m = eq.m
        pis = _pis(eq.pi, getattr(eq, "nu", 0.0), getattr(eq, "pi_nu", None))
        for k in range(eq.m):
            q.alpha[k] = float(eq.alpha[k])
            q.pi[k] = pis[k]
        a = _host_array(phi0)
        if a.size != N:
            raise ValueError(f"phi0 of {a.size} values, N = {N}")
        q.N, q.dx, q.dt, q.tau, q.lattice, q.scheme, q.nsteps = int(N), float(dx), float(dt), float(tau), \
            int(eq.lattice), int(scheme), int(nsteps)
        q.phi0 = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        rid = ctypes.c_uint64()
        if boundary == PERIODIC:
            _check(lib().lbhpde_submit(self.h, ctypes.byref(q), ctypes.byref(rid)), "lbhpde_submit")
        else:
            pb = None if phib is None else np.ascontiguousarray(np.asarray(phib, dtype=np.float64))
            ptr = None if pb is None else pb.ctypes.data_as(ctypes.c_void_p)
            _check(lib().lbhpde_submit_nee(self.h, ctypes.byref(q), int(boundary), ptr, ctypes.byref(rid)),
                   "lbhpde_submit_nee")
        self.sizes[rid.value] = int(N)
        return rid.value

    def submit_problem(self, p, nsteps=None, phib=None) -> int:
        """p's request; a bounded p needs its [nsteps][2W] boundary values phib."""
        return self.submit(p.eq, p.N, p.dx, p.dt, p.tau, p.nsteps if nsteps is None else nsteps, p.phi0, p.scheme,
                           boundary=_boundary_code(p), phib=phib)

    def poll(self, rid):
        """(status, phi or None, info dict); phi only once finished."""
        info = lbhpde_result()
        out = np.empty(max(self.sizes.get(rid, 0), 1))
        rc = lib().lbhpde_poll(self.h, ctypes.c_uint64(rid), out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(info))
        if rc == PENDING:
            return rc, None, info.as_dict()
        if rc == ERR_NOT_FOUND:
            _check(rc, "lbhpde_poll")
        self.sizes.pop(rid, None)
        return rc, out, info.as_dict()

    def wait(self, rid, timeout=60.0):
        info = lbhpde_result()
        out = np.empty(max(self.sizes.get(rid, 0), 1))
        rc = lib().lbhpde_wait(self.h, ctypes.c_uint64(rid), float(timeout), out.ctypes.data_as(ctypes.c_void_p),
                               ctypes.byref(info))
        if rc in (PENDING, ERR_TIMEOUT):
            return rc, None, info.as_dict()
        if rc == ERR_NOT_FOUND:
            _check(rc, "lbhpde_wait")
        self.sizes.pop(rid, None)
        return rc, out, info.as_dict()

    def stats(self) -> dict:
        st = lbhpde_server_info()
        _check(lib().lbhpde_server_stats(self.h, ctypes.byref(st)), "lbhpde_server_stats")
        return st.as_dict()

    def close(self):
        if self.h:
            lib().lbhpde_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Thin Python binding of libhpt's C ABI (include/hpt.h).

Argument marshalling only: every step of the path runs in libhpt's CUDA
kernels.  PyTorch provides device memory (tensors) and streams.  There is no
CPU fallback: if ``libhpt.so`` is missing the import of this module fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhpt.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libhpt.so not built ({LIB_PATH}); run paper_2111_14317_gb300.build.build()")
_lib = ctypes.CDLL(LIB_PATH)

HPT_FP64, HPT_MIXED = 0, 1
CELL_PAIRS, CELL_EXPLICIT, CELL_LOWER = 0, 1, 2
ACTIVE, CONVERGED, DIVERGED, UNDERFLOW, SINGULAR, MAX_STEPS = range(6)
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error",
                4: "value out of range", 5: "not a cell", 6: "device wait timed out",
                7: "not supported"}

EXPORTS = ["hpt_default_params", "hpt_status_string", "hpt_last_error", "hpt_lift_exponents",
           "hpt_binomial_start",
           "hpt_create_system", "hpt_destroy", "hpt_get_info", "hpt_get_texp", "hpt_eval",
           "hpt_paths_init", "hpt_step", "hpt_step_static", "hpt_track", "hpt_polish", "hpt_adjoint",
           "hpt_device_error", "hpt_profile_enable", "hpt_profile_read", "hpt_binomial_points",
           "hpt_batch_create", "hpt_batch_destroy", "hpt_batch_get_tuning", "hpt_batch_set_tuning",
           "hpt_batch_track", "hpt_batch_autotune", "hpt_batch_stats", "hpt_homogenize", "hpt_get_nvars",
           "hpt_euler_newton", "hpt_binomial_start_device", "hpt_mixed_cells", "hpt_check_bounded_wait"]


class HptError(RuntimeError):
    def __init__(self, code, where):
        msg = _lib.hpt_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)} ({msg})")
        self.code = code


class _Cell(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pairs", ctypes.c_void_p),
                ("alpha_num", ctypes.c_void_p), ("beta_num", ctypes.c_void_p),
                ("denom", ctypes.c_int64)]


class Params(ctypes.Structure):
    """hpt_params; defaults from hpt_default_params."""
    _fields_ = [("tol_accept", ctypes.c_double), ("dtau_init", ctypes.c_double),
                ("dtau_min", ctypes.c_double), ("dtau_max", ctypes.c_double),
                ("grow", ctypes.c_double), ("shrink", ctypes.c_double),
                ("grow_after", ctypes.c_int32), ("max_steps", ctypes.c_int32),
                ("div_bound", ctypes.c_double), ("polish_tol", ctypes.c_double),
                ("polish_iters", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("cond_max", ctypes.c_double), ("eps0", ctypes.c_double),
                ("predictor", ctypes.c_int32), ("pad_", ctypes.c_int32)]

    def __init__(self, **kw):
        super().__init__()
        _lib.hpt_default_params(ctypes.byref(self))
        for k, v in kw.items():
            setattr(self, k, v)


class _Paths(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in
                ("y", "tau", "dtau", "y_acc", "tau_acc", "dE_acc", "status", "steps", "accepts",
                 "rejects", "streak", "y_prev", "tau_prev", "dE_prev", "hermite")]


class Tuning(ctypes.Structure):
    """hpt_batch_tuning."""
    _fields_ = [("steps_per_round", ctypes.c_int32), ("eval_ctas_per_sm", ctypes.c_int32),
                ("solve_lanes_n17_24", ctypes.c_int32)]

    def as_tuple(self):
        return (int(self.steps_per_round), int(self.eval_ctas_per_sm), int(self.solve_lanes_n17_24))


_VP, _I64, _I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
_lib.hpt_status_string.restype = ctypes.c_char_p
_lib.hpt_last_error.restype = ctypes.c_char_p
for _name, _args in {
    "hpt_lift_exponents": [_I32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "hpt_binomial_start": [_I32, _VP, _VP, _VP, _VP, _I64, _I64, _VP, _VP],
    "hpt_create_system": [_I32, _VP, _VP, _VP, _VP, _VP, _I32, _VP],
    "hpt_destroy": [_VP],
    "hpt_get_info": [_VP, _VP, _VP, _VP, ctypes.c_double, _VP],
    "hpt_get_texp": [_VP, _VP, _VP, _VP, _VP],
    "hpt_eval": [_VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP],
    "hpt_paths_init": [_VP, _I64, _VP, _VP, _VP, _VP],
    "hpt_step": [_VP, _I64, _VP, _I32, _VP, _VP],
    "hpt_step_static": [_VP, _I64, _VP, _I32, _VP, _VP],
    "hpt_track": [_VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP],
    "hpt_polish": [_VP, _I64, _VP, _VP, _VP, _VP],
    "hpt_adjoint": [_VP, _I64, _VP, _VP, _VP, _VP],
    "hpt_device_error": [_VP],
    "hpt_profile_enable": [_VP, _I32],
    "hpt_profile_read": [_VP, _I32, _VP, _VP, _VP, _VP],
    "hpt_binomial_points": [_I32, _VP, _VP, _VP, _VP, _I64, _VP, _VP],
    "hpt_batch_create": [_I32, _VP, _VP],
    "hpt_batch_destroy": [_VP],
    "hpt_batch_get_tuning": [_VP, _VP],
    "hpt_batch_set_tuning": [_VP, _VP],
    "hpt_batch_track": [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "hpt_batch_autotune": [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP],
    "hpt_batch_stats": [_VP, _VP, _VP, _VP],
    "hpt_homogenize": [_VP, _VP],
    "hpt_get_nvars": [_VP, _VP, _VP, _VP],
    "hpt_euler_newton": [_VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP],
    "hpt_binomial_start_device": [_I32, _VP, _VP, _VP, _VP, _I64, _I64, _VP, _VP, _VP],
    "hpt_mixed_cells": [_I32, _VP, _VP, _VP, _I64, _VP, _VP, _VP],
    "hpt_check_bounded_wait": [_VP, _VP],
}.items():
    getattr(_lib, _name).argtypes = _args
    getattr(_lib, _name).restype = ctypes.c_int


def _check(rc, where):
    if rc != 0:
        raise HptError(rc, where)


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _t_ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need(t, name, dtype, shape):
    """The library sees a pointer only: refuse (ValueError) a tensor it would
    read or write with another layout, size or device."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} must be a tensor on the current CUDA device")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)}, "
                         f"got {t.dtype} {tuple(t.shape)}")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _cell_struct(cell, keep):
    c = _Cell()
    kind = cell["kind"]
    if kind == "pairs":
        pr = np.ascontiguousarray(np.asarray(cell["pairs"], dtype=np.int32).reshape(-1))
        keep.append(pr)
        c.kind, c.pairs = CELL_PAIRS, pr.ctypes.data
    elif kind in ("explicit", "lower"):
        al = np.ascontiguousarray(np.asarray(cell["alpha_num"], dtype=np.int64))
        keep.append(al)
        c.alpha_num, c.denom = al.ctypes.data, int(cell["denom"])
        if kind == "explicit":
            be = np.ascontiguousarray(np.asarray(cell["beta_num"], dtype=np.int64))
            keep.append(be)
            c.kind, c.beta_num = CELL_EXPLICIT, be.ctypes.data
        else:
            c.kind = CELL_LOWER
    else:
        raise ValueError(kind)
    return c


def _arrays(n, m, exponents, coeffs, lifting):
    msz = np.ascontiguousarray(np.asarray(m, dtype=np.int32).reshape(-1))
    ex = np.ascontiguousarray(np.asarray(exponents, dtype=np.int32))
    M = int(msz.sum())
    if msz.shape != (n,) or ex.shape != (M, n) or (msz < 0).any():
        raise ValueError(f"support sizes must be n = {n} non-negative counts and exponents an (M, n) = "
                         f"({M}, {n}) integer array, got {msz.shape} and {ex.shape}")
    co = np.asarray(coeffs, dtype=np.complex128).reshape(M)
    co = np.ascontiguousarray(np.stack([co.real, co.imag], -1).reshape(-1))
    li = np.ascontiguousarray(np.asarray(lifting, dtype=np.int64).reshape(M))
    return msz, ex, co, li, M


def lift_exponents(n, m, exponents, lifting, cell):
    """Host-only exact t-exponents: dict(e, D, alpha_num, beta_num)."""
    msz, ex, _, li, M = _arrays(n, m, exponents, np.zeros(sum(np.atleast_1d(m))), lifting)
    keep = []
    c = _cell_struct(cell, keep)
    e = np.zeros(M, np.int64)
    D = ctypes.c_int64(0)
    al = np.zeros(n, np.int64)
    be = np.zeros(n, np.int64)
    _check(_lib.hpt_lift_exponents(n, _np_ptr(msz), _np_ptr(ex), _np_ptr(li), ctypes.byref(c),
                                   _np_ptr(e), ctypes.byref(D), _np_ptr(al), _np_ptr(be)),
           "hpt_lift_exponents")
    return dict(e=e.tolist(), D=int(D.value), alpha_num=al.tolist(), beta_num=be.tolist())


def binomial_start(n, m, exponents, coeffs, pairs, first=0, count=None):
    """Host-only start points of a cell given by pairs: (y0 (count, n)
    complex128 numpy, |det V|)."""
    msz, ex, co, _, M = _arrays(n, m, exponents, coeffs, np.zeros(sum(np.atleast_1d(m))))
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1))
    tot = ctypes.c_int64(0)
    _check(_lib.hpt_binomial_start(n, _np_ptr(msz), _np_ptr(ex), _np_ptr(co), _np_ptr(pr), 0, 0, None,
                                   ctypes.byref(tot)), "hpt_binomial_start")
    if count is None:
        count = int(tot.value) - first
    y0 = np.zeros((count, n), np.complex128)
    _check(_lib.hpt_binomial_start(n, _np_ptr(msz), _np_ptr(ex), _np_ptr(co), _np_ptr(pr), int(first),
                                   int(count), _np_ptr(y0), ctypes.byref(tot)), "hpt_binomial_start")
    return y0, int(tot.value)


def mixed_cells(n, m, exponents, lifting, cap=1 << 16):
    """Host-only fine mixed cells (hpt_mixed_cells): (pairs (count, n, 2)
    int32 numpy, mixed volume)."""
    msz, ex, _, li, M = _arrays(n, m, exponents, np.zeros(sum(np.atleast_1d(m)), np.complex128), lifting)
    out = np.zeros((cap, n, 2), np.int32)
    cnt, vol = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(_lib.hpt_mixed_cells(n, _np_ptr(msz), _np_ptr(ex), _np_ptr(li), cap, _np_ptr(out), ctypes.byref(cnt),
                                ctypes.byref(vol)), "hpt_mixed_cells")
    return out[:min(cnt.value, cap)].copy(), int(vol.value)


def binomial_start_device(n, m, exponents, coeffs, pairs, first=0, count=None, device="cuda", stream=None):
    """The same start points computed on the device (hpt_binomial_start_device):
    (y0 (count, n) complex128 tensor on `device`, |det V|)."""
    msz, ex, co, _, M = _arrays(n, m, exponents, coeffs, np.zeros(sum(np.atleast_1d(m))))
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1))
    tot = ctypes.c_int64(0)
    _check(_lib.hpt_binomial_start(n, _np_ptr(msz), _np_ptr(ex), _np_ptr(co), _np_ptr(pr), 0, 0, None,
                                   ctypes.byref(tot)), "hpt_binomial_start")
    if count is None:
        count = int(tot.value) - first
    y0 = torch.empty(count, n, dtype=torch.complex128, device=device)
    _check(_lib.hpt_binomial_start_device(n, _np_ptr(msz), _np_ptr(ex), _np_ptr(co), _np_ptr(pr), int(first),
                                          int(count), _t_ptr(y0), ctypes.byref(tot), _stream(stream)),
           "hpt_binomial_start_device")
    return y0, int(tot.value)


def binomial_points(n, m, exponents, coeffs, pairs, k):
    """Host-only start points y = exp(V^-1 (log b + 2 pi i k)) for the integer
    rows of k (count, n): (count, n) complex128 numpy."""
    msz, ex, co, _, M = _arrays(n, m, exponents, coeffs, np.zeros(sum(np.atleast_1d(m))))
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1))
    kv = np.ascontiguousarray(np.asarray(k, dtype=np.int64).reshape(-1, n))
    y0 = np.zeros((kv.shape[0], n), np.complex128)
    _check(_lib.hpt_binomial_points(n, _np_ptr(msz), _np_ptr(ex), _np_ptr(co), _np_ptr(pr), kv.shape[0],
                                    _np_ptr(kv), _np_ptr(y0)), "hpt_binomial_points")
    return y0


class PathState:
    """Caller-owned structure-of-arrays path state on a device (or in pinned
    host memory with device="cpu", pin=True): every field is a view into one
    contiguous byte arena, so the whole state moves between host and device
    in one copy (`arena`).  hermite=True adds the previous accepted point
    (y_prev, tau_prev, dE_prev) and the pending-prediction flag (hermite)
    that the cubic Hermite predictor needs."""

    BASE = ("y", "tau", "dtau", "y_acc", "tau_acc", "dE_acc", "status", "steps", "accepts",
            "rejects", "streak")
    PREV = ("y_prev", "tau_prev", "dE_prev", "hermite")

    def __init__(self, p, n, precision, device="cuda", pin=False, hermite=False):
        cdt = torch.complex128 if precision == HPT_FP64 else torch.complex64
        self.p, self.n, self.precision = p, n, precision
        self.FIELDS = self.BASE + (self.PREV if hermite else ())
        shapes = {"y": ((p, n), cdt), "y_acc": ((p, n), cdt), "dE_acc": ((p, n), cdt),
                  "tau": ((p,), torch.float64), "dtau": ((p,), torch.float64), "tau_acc": ((p,), torch.float64),
                  "status": ((p,), torch.int32), "steps": ((p,), torch.int32), "accepts": ((p,), torch.int32),
                  "rejects": ((p,), torch.int32), "streak": ((p,), torch.int32),
                  "y_prev": ((p, n), cdt), "tau_prev": ((p,), torch.float64), "dE_prev": ((p, n), cdt),
                  "hermite": ((p,), torch.int32)}
        offs, off = {}, 0
        for k in self.FIELDS:
            shp, dt = shapes[k]
            nb = int(np.prod(shp)) * torch.empty((), dtype=dt).element_size()
            offs[k] = (off, nb)
            off += (nb + 255) // 256 * 256
        self.arena = torch.zeros(max(off, 256), dtype=torch.uint8, device=device)
        if pin:
            self.arena = self.arena.pin_memory()
        for k in self.FIELDS:
            shp, dt = shapes[k]
            o, nb = offs[k]
            setattr(self, k, self.arena[o:o + nb].view(dt).view(*shp))

    def _c(self):
        return _Paths(*[getattr(self, k).data_ptr() if hasattr(self, k) else None
                        for k in self.BASE + self.PREV])

    def to_host(self):
        return {k: getattr(self, k).cpu() for k in self.FIELDS}

    def load(self, host):
        for k, v in host.items():
            getattr(self, k).copy_(v)


class System:
    """A Laurent system with a cell on the current CUDA device (hpt_system)."""

    def __init__(self, n, m, exponents, coeffs, lifting, cell, precision=HPT_FP64):
        self.n = int(n)
        self.precision = int(precision)
        msz, ex, co, li, M = _arrays(self.n, m, exponents, coeffs, lifting)
        self.M = M
        keep = []
        c = _cell_struct(cell, keep)
        h = ctypes.c_void_p()
        _check(_lib.hpt_create_system(self.n, _np_ptr(msz), _np_ptr(ex), _np_ptr(co), _np_ptr(li),
                                      ctypes.byref(c), self.precision, ctypes.byref(h)),
               "hpt_create_system")
        self._h = h
        self.cdtype = torch.complex128 if self.precision == HPT_FP64 else torch.complex64
        self.nv, self.projective, self.degrees = self.n, False, None

    @classmethod
    def from_laurent(cls, sysm, cell, precision=HPT_FP64):
        return cls(sysm.n, sysm.m, sysm.exponents, sysm.coeffs, sysm.lifting, cell, precision)

    def homogenize(self):
        """The projective form of this system (hpt_homogenize): n equations in
        nv = n + 1 homogeneous coordinates, the homogenizing one last."""
        h = ctypes.c_void_p()
        _check(_lib.hpt_homogenize(self._h, ctypes.byref(h)), "hpt_homogenize")
        o = System.__new__(System)
        o._h, o.n, o.M, o.precision, o.cdtype = h, self.n, self.M, self.precision, self.cdtype
        nv, pj = ctypes.c_int32(0), ctypes.c_int32(0)
        deg = np.zeros(self.n, np.int64)
        _check(_lib.hpt_get_nvars(h, ctypes.byref(nv), ctypes.byref(pj), _np_ptr(deg)), "hpt_get_nvars")
        o.nv, o.projective, o.degrees = int(nv.value), bool(pj.value), deg
        return o

    def new_state(self, p, device="cuda", pin=False, hermite=False):
        """A PathState for p paths of this system (nv entries per path)."""
        return PathState(p, self.nv, self.precision, device=device, pin=pin, hermite=hermite)

    def close(self):
        if getattr(self, "_h", None):
            _lib.hpt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------- host data
    def tau0(self, eps0=1e-10):
        t = ctypes.c_double(0)
        _check(_lib.hpt_get_info(self._h, None, None, None, ctypes.c_double(eps0), ctypes.byref(t)),
               "hpt_get_info")
        return float(t.value)

    def texp(self):
        e = np.zeros(self.M, np.int64)
        D = ctypes.c_int64(0)
        al = np.zeros(self.n, np.int64)
        be = np.zeros(self.n, np.int64)
        _check(_lib.hpt_get_texp(self._h, _np_ptr(e), ctypes.byref(D), _np_ptr(al), _np_ptr(be)),
               "hpt_get_texp")
        return dict(e=e.tolist(), D=int(D.value), alpha_num=al.tolist(), beta_num=be.tolist())

    def check_bounded_wait(self, stream=None):
        """Enqueue the bounded-wait probe (times out after ~2 s, sets the error flag)."""
        _check(_lib.hpt_check_bounded_wait(self._h, _stream(stream)), "hpt_check_bounded_wait")

    def device_error(self):
        rc = _lib.hpt_device_error(self._h)
        return rc

    # ----------------------------------------------------------- device work
    def _need_state(self, state):
        if state.n != self.nv or state.precision != self.precision or not state.y.is_cuda:
            raise ValueError(f"state must be a device PathState with {self.nv} variables per path in "
                             f"precision {self.precision}")

    def eval(self, y, t, stream=None, out=None):
        """H (p,n), H_y (p,n,nv), H_t (p,n) at y (p,nv) complex, t (p,) float64."""
        p = y.shape[0]
        _need(y, "y", self.cdtype, (p, self.nv))
        _need(t, "t", torch.float64, (p,))
        if out is None:
            out = (torch.empty(p, self.n, dtype=self.cdtype, device=y.device),
                   torch.empty(p, self.n, self.nv, dtype=self.cdtype, device=y.device),
                   torch.empty(p, self.n, dtype=self.cdtype, device=y.device))
        H, Hy, Ht = out
        for a, nm, shp in ((H, "H", (p, self.n)), (Hy, "Hy", (p, self.n, self.nv)), (Ht, "Ht", (p, self.n))):
            if a is not None:
                _need(a, nm, self.cdtype, shp)
        _check(_lib.hpt_eval(self._h, p, _t_ptr(y), _t_ptr(t), _t_ptr(H), _t_ptr(Hy), _t_ptr(Ht),
                             _stream(stream)), "hpt_eval")
        return H, Hy, Ht

    def euler_newton(self, y, tau, stream=None):
        """Algorithm 3 at y (p,nv) complex, tau (p,) float64: the Euler and
        Newton directions (p,nv) each and ok (p,) int32."""
        p = y.shape[0]
        tau = tau.contiguous()
        _need(y, "y", self.cdtype, (p, self.nv))
        _need(tau, "tau", torch.float64, (p,))
        dE = torch.empty(p, self.nv, dtype=self.cdtype, device=y.device)
        dN = torch.empty(p, self.nv, dtype=self.cdtype, device=y.device)
        ok = torch.empty(p, dtype=torch.int32, device=y.device)
        _check(_lib.hpt_euler_newton(self._h, p, _t_ptr(y), _t_ptr(tau), _t_ptr(dE), _t_ptr(dN),
                                     _t_ptr(ok), _stream(stream)), "hpt_euler_newton")
        return dE, dN, ok

    def paths_init(self, state, y0, params=None, stream=None):
        params = params or Params()
        self._need_state(state)
        _need(y0, "y0", torch.complex128, (state.p, self.n))
        c = state._c()
        _check(_lib.hpt_paths_init(self._h, state.p, _t_ptr(y0), ctypes.byref(params), ctypes.byref(c),
                                   _stream(stream)), "hpt_paths_init")
        return state

    def step(self, state, nsteps=1, params=None, stream=None):
        params = params or Params()
        self._need_state(state)
        c = state._c()
        _check(_lib.hpt_step(self._h, state.p, ctypes.byref(c), int(nsteps), ctypes.byref(params),
                             _stream(stream)), "hpt_step")
        return state

    def step_static(self, state, nsteps=1, params=None, stream=None):
        """hpt_step without device-memory allocation: scratch from the library's
        fixed 32 MiB array (see hpt_step_static in include/hpt.h for the path
        limit and the sharing rules)."""
        params = params or Params()
        self._need_state(state)
        c = state._c()
        _check(_lib.hpt_step_static(self._h, state.p, ctypes.byref(c), int(nsteps), ctypes.byref(params),
                                    _stream(stream)), "hpt_step_static")
        return state

    def track(self, y0, params=None, stream=None):
        """Returns (x (p,n) complex128, status (p,) int32, steps (p,) int32)."""
        params = params or Params()
        p = y0.shape[0]
        _need(y0, "y0", torch.complex128, (p, self.n))
        x = torch.empty(p, self.n, dtype=torch.complex128, device=y0.device)
        st = torch.empty(p, dtype=torch.int32, device=y0.device)
        sp = torch.empty(p, dtype=torch.int32, device=y0.device)
        _check(_lib.hpt_track(self._h, p, _t_ptr(y0), ctypes.byref(params), _t_ptr(x), _t_ptr(st),
                              _t_ptr(sp), _stream(stream)), "hpt_track")
        return x, st, sp

    def polish(self, x, status=None, params=None, stream=None):
        params = params or Params()
        _need(x, "x", torch.complex128, (x.shape[0], self.n))
        if status is not None:
            _need(status, "status", torch.int32, (x.shape[0],))
        _check(_lib.hpt_polish(self._h, x.shape[0], _t_ptr(x), _t_ptr(status), ctypes.byref(params),
                               _stream(stream)), "hpt_polish")
        return x

    def adjoint(self, x, gx, stream=None):
        """Coefficient gradient (M,) complex128 of a real loss with gx = dL/dx."""
        x, gx = x.contiguous(), gx.contiguous()
        _need(x, "x", torch.complex128, (x.shape[0], self.n))
        _need(gx, "gx", torch.complex128, (x.shape[0], self.n))
        gc = torch.empty(self.M, dtype=torch.complex128, device=x.device)
        _check(_lib.hpt_adjoint(self._h, x.shape[0], _t_ptr(x), _t_ptr(gx),
                                _t_ptr(gc), _stream(stream)), "hpt_adjoint")
        return gc

    def profile(self, enable=True):
        _check(_lib.hpt_profile_enable(self._h, int(bool(enable))), "hpt_profile_enable")

    def profile_read(self):
        cap = 32
        names = (ctypes.c_char_p * cap)()
        launches = np.zeros(cap, np.int64)
        ms = np.zeros(cap)
        cnt = ctypes.c_int32(0)
        _check(_lib.hpt_profile_read(self._h, cap, names, _np_ptr(launches), _np_ptr(ms),
                                     ctypes.byref(cnt)), "hpt_profile_read")
        return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(cnt.value, cap))}


class Batch:
    """Many HPT_MIXED systems tracked together (hpt_batch).  Keeps the System
    objects alive for its own lifetime."""

    def __init__(self, systems):
        self.systems = list(systems)
        self.n = [s.n for s in self.systems]
        arr = (ctypes.c_void_p * len(self.systems))(*[s._h.value for s in self.systems])
        h = ctypes.c_void_p()
        _check(_lib.hpt_batch_create(len(self.systems), arr, ctypes.byref(h)), "hpt_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.hpt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def tuning(self):
        t = Tuning()
        _check(_lib.hpt_batch_get_tuning(self._h, ctypes.byref(t)), "hpt_batch_get_tuning")
        return t.as_tuple()

    @tuning.setter
    def tuning(self, kv):
        """(K, eval CTAs/SM[, solve lanes for 17 <= n <= 24]); omitted entries keep their value."""
        cur = self.tuning
        kv = tuple(kv) + cur[len(kv):]
        t = Tuning(int(kv[0]), int(kv[1]), int(kv[2]))
        _check(_lib.hpt_batch_set_tuning(self._h, ctypes.byref(t)), "hpt_batch_set_tuning")

    def _check_y0(self, y0, paths):
        """The library cannot see buffer sizes: the start points must hold
        exactly sum_s paths[s] n_s values for the batch's systems."""
        p = np.ascontiguousarray(np.asarray(paths, dtype=np.int64).reshape(-1))
        if len(p) != len(self.systems) or (p < 0).any():
            raise ValueError(f"paths must list {len(self.systems)} non-negative counts")
        need = int(sum(int(c) * h.n for c, h in zip(p, self.systems)))
        if y0.dtype != torch.complex128 or not y0.is_contiguous() or y0.numel() != need:
            raise ValueError(f"y0 must be a contiguous complex128 tensor of {need} values")
        return p

    def track(self, y0, paths, params=None, stream=None):
        """y0: (sum p_s n_s,) complex128 device tensor (systems concatenated,
        path-major); paths: per-system path counts.  Returns (x like y0,
        status (P,) int32, steps (P,) int32)."""
        params = params or Params()
        p = self._check_y0(y0, paths)
        x = torch.empty_like(y0)
        P = int(p.sum())
        st = torch.empty(P, dtype=torch.int32, device=y0.device)
        sp = torch.empty(P, dtype=torch.int32, device=y0.device)
        _check(_lib.hpt_batch_track(self._h, _np_ptr(p), _t_ptr(y0), ctypes.byref(params), _t_ptr(x),
                                    _t_ptr(st), _t_ptr(sp), _stream(stream)), "hpt_batch_track")
        return x, st, sp

    def autotune(self, y0, paths, params=None, stream=None):
        """Coordinate-descent autotuner (hpt_batch_autotune).  Returns
        (best (K, ctas, lanes), {(K, ctas, lanes): ms})."""
        params = params or Params()
        p = self._check_y0(y0, paths)
        x = torch.empty_like(y0)
        cap = 16
        cand = (Tuning * cap)()
        ms = np.zeros(cap)
        nc = ctypes.c_int32(cap)
        best = Tuning()
        _check(_lib.hpt_batch_autotune(self._h, _np_ptr(p), _t_ptr(y0), ctypes.byref(params), _t_ptr(x),
                                       _stream(stream), ctypes.byref(best), cand, _np_ptr(ms),
                                       ctypes.byref(nc)), "hpt_batch_autotune")
        return best.as_tuple(), {cand[i].as_tuple(): float(ms[i]) for i in range(nc.value)}

    def stats(self):
        r, ps, k = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int32(0)
        _check(_lib.hpt_batch_stats(self._h, ctypes.byref(r), ctypes.byref(ps), ctypes.byref(k)),
               "hpt_batch_stats")
        return dict(rounds=int(r.value), position_steps=int(ps.value), kernels_per_round=int(k.value))

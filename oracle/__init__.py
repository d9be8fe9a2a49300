"""CPU oracle of the polyhedral-homotopy path tracker -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The CUDA library never does,
and the oracle shares no code with it.

The numerical core is plain C99 complex128 (``hpt_oracle.c``, built with gcc
into ``oracle/_build/liboracle.so``); the exact integer bookkeeping is Python
(``cells.py``).  Parity status of every function is stated in those files.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

from . import cells  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hpt_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

ACTIVE, CONVERGED, DIVERGED, UNDERFLOW, SINGULAR, MAX_STEPS = range(6)


def build(force=False):
    """Compile the C core (gcc, -O2, IEEE semantics, OpenMP over paths)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.ora_eval.restype = ctypes.c_int
        _lib.ora_scale.restype = ctypes.c_int
        _lib.ora_solve.restype = ctypes.c_int64
        _lib.ora_directions.restype = ctypes.c_int
        _lib.ora_step.restype = ctypes.c_int
        _lib.ora_track.restype = ctypes.c_int
        _lib.ora_polish.restype = ctypes.c_int
        _lib.ora_adjoint.restype = ctypes.c_int64
        _lib.ora_num_threads.restype = ctypes.c_int
    return _lib


def num_threads() -> int:
    return int(_load().ora_num_threads())


def set_threads(k: int) -> None:
    _load().ora_set_threads(ctypes.c_int(int(k)))


class _Sys(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("M", ctypes.c_int32),
                ("msz", ctypes.c_void_p), ("off", ctypes.c_void_p),
                ("exps", ctypes.c_void_p), ("coef", ctypes.c_void_p),
                ("texp", ctypes.c_void_p), ("D", ctypes.c_int64)]


class _Params(ctypes.Structure):
    _fields_ = [("tol_accept", ctypes.c_double), ("dtau_init", ctypes.c_double),
                ("dtau_min", ctypes.c_double), ("dtau_max", ctypes.c_double),
                ("grow", ctypes.c_double), ("shrink", ctypes.c_double),
                ("grow_after", ctypes.c_int32), ("max_steps", ctypes.c_int32),
                ("div_bound", ctypes.c_double), ("polish_tol", ctypes.c_double),
                ("polish_iters", ctypes.c_int32), ("predictor", ctypes.c_int32)]


@dataclass
class Params:
    """Step-size control constants (a stated reading; the paper gives none)."""
    tol_accept: float = 1e-3
    dtau_init: float = 0.05
    dtau_min: float = 1e-8
    dtau_max: float = 0.5
    grow: float = 2.0
    shrink: float = 0.5
    grow_after: int = 3
    max_steps: int = 10000
    div_bound: float = 1e8
    polish_tol: float = 1e-13
    polish_iters: int = 8
    predictor: int = 0          # 0: Euler; 1: cubic Hermite (two accepted points)

    def _c(self):
        return _Params(self.tol_accept, self.dtau_init, self.dtau_min, self.dtau_max,
                       self.grow, self.shrink, self.grow_after, self.max_steps,
                       self.div_bound, self.polish_tol, self.polish_iters, self.predictor)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


class System:
    """A Laurent system with its t-exponents, as the oracle sees it."""

    def __init__(self, sysm, texp, D):
        self.sysm = sysm
        self.n = sysm.n
        self.M = sysm.M
        self.msz = np.ascontiguousarray(sysm.m, dtype=np.int32)
        self.off = np.ascontiguousarray(sysm.offsets, dtype=np.int32)
        self.exps = np.ascontiguousarray(sysm.exponents, dtype=np.int32)
        self.coef = np.ascontiguousarray(np.stack([sysm.coeffs.real, sysm.coeffs.imag], -1).reshape(-1))
        self.texp = np.ascontiguousarray(texp, dtype=np.int64)
        self.D = int(D)
        assert self.texp.shape == (self.M,)
        self._c = _Sys(self.n, self.M, self.msz.ctypes.data, self.off.ctypes.data,
                       self.exps.ctypes.data, self.coef.ctypes.data, self.texp.ctypes.data,
                       self.D)

    @classmethod
    def from_cell(cls, sysm, cell):
        te = cells.t_exponents(sysm, cell)
        return cls(sysm, te["e"], te["D"])

    # ------------------------------------------------------------ evaluation
    def eval(self, y, tau):
        """H (p,n), H_y (p,n,n) [k,j], H_tau (p,n) at points y (p,n), tau (p,)."""
        y = np.ascontiguousarray(y, dtype=np.complex128)
        tau = np.ascontiguousarray(np.broadcast_to(tau, (y.shape[0],)), dtype=np.float64)
        p, n = y.shape
        assert n == self.n
        H = np.zeros((p, n), np.complex128)
        Hy = np.zeros((p, n, n), np.complex128)
        Ht = np.zeros((p, n), np.complex128)
        rc = _load().ora_eval(ctypes.byref(self._c), ctypes.c_int64(p), _ptr(y), _ptr(tau),
                              _ptr(H), _ptr(Hy), _ptr(Ht))
        assert rc == 0
        return H, Hy, Ht

    def scale(self, y, tau):
        """Sums of term magnitudes matching eval's outputs (tolerance scales)."""
        y = np.ascontiguousarray(y, dtype=np.complex128)
        tau = np.ascontiguousarray(np.broadcast_to(tau, (y.shape[0],)), dtype=np.float64)
        p, n = y.shape
        SH = np.zeros((p, n))
        SHy = np.zeros((p, n, n))
        SHt = np.zeros((p, n))
        rc = _load().ora_scale(ctypes.byref(self._c), ctypes.c_int64(p), _ptr(y), _ptr(tau),
                               _ptr(SH), _ptr(SHy), _ptr(SHt))
        assert rc == 0
        return SH, SHy, SHt

    def directions(self, y, tau):
        """Euler and Newton directions (p,n) each, and a regularity flag."""
        y = np.ascontiguousarray(y, dtype=np.complex128)
        tau = np.ascontiguousarray(np.broadcast_to(tau, (y.shape[0],)), dtype=np.float64)
        p, n = y.shape
        dE = np.zeros((p, n), np.complex128)
        dN = np.zeros((p, n), np.complex128)
        ok = np.zeros(p, np.int32)
        _load().ora_directions(ctypes.byref(self._c), ctypes.c_int64(p), _ptr(y), _ptr(tau),
                               _ptr(dE), _ptr(dN), _ptr(ok))
        return dE, dN, ok.astype(bool)

    # -------------------------------------------------------------- tracking
    def step(self, params, state, nsteps=1):
        """Advance a PathState in place by nsteps Euler-Newton steps."""
        s = state
        _load().ora_step(ctypes.byref(self._c), ctypes.byref(params._c()), ctypes.c_int64(s.p),
                         ctypes.c_int32(nsteps), _ptr(s.y), _ptr(s.tau), _ptr(s.dtau),
                         _ptr(s.yacc), _ptr(s.tauacc), _ptr(s.dEacc), _ptr(s.status),
                         _ptr(s.steps), _ptr(s.accepts), _ptr(s.rejects), _ptr(s.streak),
                         _ptr(s.yprev), _ptr(s.tauprev), _ptr(s.dEprev), _ptr(s.hflag))
        return state

    def track(self, params, y0, tau0):
        """Track every start point from tau0 to 0 and polish; returns
        (x (p,n), status (p,), steps (p,), polish_err (p,))."""
        y0 = np.ascontiguousarray(y0, dtype=np.complex128)
        p, n = y0.shape
        x = np.zeros((p, n), np.complex128)
        st = np.zeros(p, np.int32)
        steps = np.zeros(p, np.int32)
        perr = np.zeros(p)
        _load().ora_track(ctypes.byref(self._c), ctypes.byref(params._c()), ctypes.c_int64(p),
                          _ptr(y0), ctypes.c_double(tau0), _ptr(x), _ptr(st), _ptr(steps),
                          _ptr(perr))
        return x, st, steps, perr

    def polish(self, params, y):
        y = np.array(y, dtype=np.complex128, copy=True, order="C")
        err = np.zeros(y.shape[0])
        _load().ora_polish(ctypes.byref(self._c), ctypes.byref(params._c()),
                           ctypes.c_int64(y.shape[0]), _ptr(y), _ptr(err))
        return y, err

    def adjoint(self, x, gx):
        """Gradient of a real loss w.r.t. the coefficients (M,) complex, given
        x (p,n) solutions at t = 1 and gx = dL/dRe x + i dL/dIm x."""
        x = np.ascontiguousarray(x, dtype=np.complex128)
        gx = np.ascontiguousarray(gx, dtype=np.complex128)
        gc = np.zeros(2 * self.M)
        ns = _load().ora_adjoint(ctypes.byref(self._c), ctypes.c_int64(x.shape[0]), _ptr(x),
                                 _ptr(gx), _ptr(gc))
        assert ns == 0, f"{ns} singular Jacobians"
        return gc[0::2] + 1j * gc[1::2]


def solve(A, B):
    """Batched LU solve A X = B; A (p,n,n), B (p,n,r) complex; returns
    (X, n_singular)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    B = np.ascontiguousarray(B, dtype=np.complex128)
    p, n, _ = A.shape
    r = B.shape[2]
    X = np.zeros((p, n, r), np.complex128)
    ns = _load().ora_solve(ctypes.c_int(n), ctypes.c_int(r), ctypes.c_int64(p), _ptr(A), _ptr(B),
                           _ptr(X))
    return X, int(ns)


@dataclass
class PathState:
    """Structure-of-arrays tracker state (oracle side)."""
    y: np.ndarray
    tau: np.ndarray
    dtau: np.ndarray
    yacc: np.ndarray
    tauacc: np.ndarray
    dEacc: np.ndarray
    status: np.ndarray
    steps: np.ndarray
    accepts: np.ndarray
    rejects: np.ndarray
    streak: np.ndarray
    yprev: np.ndarray = None      # the accepted point before the last one (Hermite predictor)
    tauprev: np.ndarray = None
    dEprev: np.ndarray = None
    hflag: np.ndarray = None      # 1 while the pending prediction is a cubic Hermite one
    p: int = field(init=False)

    def __post_init__(self):
        self.p = self.y.shape[0]
        if self.yprev is None:
            self.yprev = np.zeros_like(self.y)
            self.dEprev = np.zeros_like(self.y)
            self.tauprev = np.zeros(self.p)
        if self.hflag is None:
            self.hflag = np.zeros(self.p, np.int32)

    @classmethod
    def start(cls, y0, tau0, dtau0):
        """State before the first step: predicted point = start point."""
        y0 = np.array(y0, dtype=np.complex128, copy=True, order="C")
        p, n = y0.shape
        return cls(y=y0, tau=np.full(p, float(tau0)), dtau=np.full(p, float(dtau0)),
                   yacc=y0.copy(), tauacc=np.full(p, float(tau0)),
                   dEacc=np.zeros((p, n), np.complex128), status=np.zeros(p, np.int32),
                   steps=np.zeros(p, np.int32), accepts=np.zeros(p, np.int32),
                   rejects=np.zeros(p, np.int32), streak=np.zeros(p, np.int32))

    def copy(self):
        return PathState(**{k: getattr(self, k).copy() for k in
                            ("y", "tau", "dtau", "yacc", "tauacc", "dEacc", "status", "steps",
                             "accepts", "rejects", "streak", "yprev", "tauprev", "dEprev", "hflag")})

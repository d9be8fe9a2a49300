"""Projective formulation and Algorithm 3 -- TEST INFRASTRUCTURE (oracle).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may use this module; the CUDA library never does and shares no code with it.

What it computes (T. Chen, "GPU-accelerated path tracker for polyhedral
homotopy"):

* Section 2.2, eq. (3) (projective formulation): every monomial y^a of equation k
  becomes y^{a_hat} with a_hat = (a, d_k - 1^T a) in n + 1 homogeneous
  coordinates (the homogenizing coordinate last), so that every h_k is
  homogeneous of degree d_k.  Reading: d_k is the largest 1^T a over S_k
  (the total degree deg f_k for a polynomial system; for a Laurent support it
  is the smallest choice that leaves the new exponent non-negative).
* Section 6, Algorithm 3 (EulerNewton): the consolidated matrix
      J = [[dH/dy, dH/dtau, H], [y^*, 0, 0]]        (N x (N+2), N = n + 1)
  is factored as J^T = Q [R; 0] (a library Householder QR, numpy/LAPACK, is
  the QR step); the rows of V = [e_{N+1}; e_{N+2}] Q^* span the null space of
  J; row reduction makes the rightmost 2 x 2 block of V the identity, and the
  leftmost N columns of its two rows are the Euler direction (eq. (4): dH/dy
  dE + dH/dtau = 0, y^* dE = 0) and the Newton direction (eq. (5): dH/dy dN
  + H = 0, y^* dN = 0).  The same steps with no y^* row give the affine
  directions (N = n).
* Tracking in homogeneous coordinates.  The paper gives the directions, not a
  projective step rule; the rule here is the affine tracker's (one
  prediction, one Newton correction, Section 8, with the same step-size
  control and the same predictor choice) plus two readings: after every
  Newton correction the point is scaled back to unit Euclidean norm (and the
  stored Euler direction by the same factor), and a path is divergent when a
  dehomogenized coordinate |y_j / y_n| leaves (1/div_bound, div_bound), the
  affine test on x = y'/y_n, checked before the end-of-path test (a path can
  reach tau = 0 at infinity: y_n = 0 is an ordinary point of projective
  space).  Start
  points are (x0, 1)/|(x0, 1)|; end points are dehomogenized and then
  polished by the affine oracle.

The homotopy itself is evaluated by the affine oracle's C core (monomials by
repeated multiplication, derivatives by direct differentiation) on the square
system made of the n homogenized equations and the chart equation y_n - 1 = 0,
whose last row is dropped.

Parity: pinned by tests/test_oracle_projective.py (homogeneity and Euler's
identity, agreement with the affine oracle on the chart y_n = 1, the defining
equations of both directions checked through the Pythagorean relation and an
independent LU solve of the bordered system, the projective tracker reaching
the affine tracker's end points and the BKK root count, and the known point
at infinity of a system without finite solutions).
"""
from __future__ import annotations

import numpy as np

from . import (ACTIVE, CONVERGED, DIVERGED, MAX_STEPS, SINGULAR, UNDERFLOW, PathState,
               System)


def degrees(sysm):
    """d_k = max over S_k of 1^T a (the homogenization degree, Section 2.2)."""
    off = sysm.offsets
    return np.array([int(sysm.exponents[off[k]:off[k] + sysm.m[k]].sum(axis=1).max())
                     for k in range(sysm.n)], np.int64)


def homogenize(sysm):
    """Exponents a_hat = (a, d_k - 1^T a) (M, n+1) and the degrees d (n,)."""
    d = degrees(sysm)
    eq = np.repeat(np.arange(sysm.n), sysm.m)
    last = d[eq] - sysm.exponents.sum(axis=1)
    return np.concatenate([sysm.exponents, last[:, None]], axis=1).astype(np.int32), d


class _Square:
    """Plain container the affine oracle reads (n+1 equations and variables)."""

    def __init__(self, n, m, exponents, coeffs):
        self.n, self.m, self.exponents, self.coeffs = n, m, exponents, coeffs
        self.M = int(sum(m))
        off, acc = [], 0
        for v in m:
            off.append(acc)
            acc += v
        self.offsets = off


def homogeneous_start(x0):
    """(x0, 1) / |(x0, 1)|_2 for start points x0 (p, n)."""
    x0 = np.asarray(x0, np.complex128)
    y = np.concatenate([x0, np.ones((x0.shape[0], 1), np.complex128)], axis=1)
    return y / np.linalg.norm(y, axis=1, keepdims=True)


def dehomogenize(y):
    y = np.asarray(y, np.complex128)
    return y[:, :-1] / y[:, -1:]


def null_directions(J):
    """Algorithm 3 on a batch of consolidated matrices J (p, N, N+2): QR of
    J^T, the two null vectors, the 2 x 2 reduction.  Returns dE, dN (p, N)
    and ok (p,) (finite and the 2 x 2 block invertible)."""
    J = np.asarray(J, np.complex128)
    p, N, C = J.shape
    assert C == N + 2
    dE = np.full((p, N), np.nan + 0j)
    dN = np.full((p, N), np.nan + 0j)
    ok = np.isfinite(J).all(axis=(1, 2))
    if ok.any():
        Q, _ = np.linalg.qr(np.swapaxes(J[ok], 1, 2), mode="complete")   # J^T = Q [R; 0]
        V = np.conj(np.swapaxes(Q[:, :, N:], 1, 2))                     # [e_{N+1}; e_{N+2}] Q^*
        Mb = V[:, :, N:]                                                  # rightmost 2 x 2 block
        det = Mb[:, 0, 0] * Mb[:, 1, 1] - Mb[:, 0, 1] * Mb[:, 1, 0]
        good = (det != 0) & np.isfinite(det)
        Vr = np.full_like(V, np.nan)
        Vr[good] = np.linalg.solve(Mb[good], V[good])                     # row reduction
        idx = np.flatnonzero(ok)
        dE[idx] = Vr[:, 0, :N]
        dN[idx] = Vr[:, 1, :N]
        fin = good & np.isfinite(Vr[:, :, :N]).all(axis=(1, 2))
        ok[idx] = fin
    return dE, dN, ok


def _predict(P, s, q, h, cubic):
    """Euler, or (cubic set: not the Euler retry of a rejected cubic
    prediction) the cubic Hermite interpolant through the last two accepted
    points (values and Euler directions) evaluated at tau_acc + h; hflag
    records the choice.  In
    homogeneous coordinates the corrector leaves a point's phase free (y and
    e^{i theta} y are one point), so the previous point and its direction are
    first turned into the phase of the last one (y_acc^* y_prev real and
    positive); otherwise the extrapolation amplifies phase differences."""
    d = s.tauacc[q] - s.tauprev[q]
    s.hflag[q] = 0
    if cubic and P.predictor == 1 and s.accepts[q] >= 2 and d > 0:
        s.hflag[q] = 1
        t = 1.0 + h / d
        h00, h10 = 2 * t**3 - 3 * t**2 + 1, t**3 - 2 * t**2 + t
        h01, h11 = -2 * t**3 + 3 * t**2, t**3 - t**2
        dot = np.vdot(s.yacc[q], s.yprev[q])
        u = np.conj(dot) / abs(dot) if dot != 0 else 1.0
        return h00 * u * s.yprev[q] + h10 * d * u * s.dEprev[q] + h01 * s.yacc[q] + h11 * d * s.dEacc[q]
    return s.yacc[q] + h * s.dEacc[q]


class ProjectiveSystem:
    """The homogenized homotopy of a Laurent system with its t-exponents."""

    def __init__(self, sysm, texp, D):
        self.sysm = sysm
        self.n = sysm.n
        self.nv = sysm.n + 1
        self.exps_hat, self.deg = homogenize(sysm)
        self.affine = System(sysm, texp, D)
        n = self.n
        # the chart equation y_n - 1 = 0 makes the system square; its row is dropped
        chart = np.zeros((2, n + 1), np.int32)
        chart[0, n] = 1
        sq = _Square(n + 1, list(sysm.m) + [2], np.concatenate([self.exps_hat, chart]),
                     np.concatenate([sysm.coeffs, [1.0, -1.0]]))
        self._sq = System(sq, np.concatenate([np.asarray(texp, np.int64), [0, 0]]), D)

    @classmethod
    def from_cell(cls, sysm, cell):
        from . import cells
        te = cells.t_exponents(sysm, cell)
        return cls(sysm, te["e"], te["D"])

    def eval(self, y, tau):
        """H (p,n), H_y (p,n,n+1) [k,j], H_tau (p,n) of the homogenized
        homotopy at y (p, n+1)."""
        H, Hy, Ht = self._sq.eval(y, tau)
        n = self.n
        return H[:, :n], Hy[:, :n, :], Ht[:, :n]

    def scale(self, y, tau):
        """Sums of term magnitudes matching eval's outputs (tolerance scales)."""
        SH, SHy, SHt = self._sq.scale(y, tau)
        n = self.n
        return SH[:, :n], SHy[:, :n, :], SHt[:, :n]

    def consolidated(self, y, tau):
        """J = [[H_y, H_tau, H], [y^*, 0, 0]] (p, n+1, n+3) (Section 6)."""
        y = np.asarray(y, np.complex128)
        p = y.shape[0]
        H, Hy, Ht = self.eval(y, tau)
        top = np.concatenate([Hy, Ht[:, :, None], H[:, :, None]], axis=2)
        bottom = np.concatenate([np.conj(y), np.zeros((p, 2), np.complex128)], axis=1)
        return np.concatenate([top, bottom[:, None, :]], axis=1)

    def directions(self, y, tau):
        """Euler and Newton directions (p, n+1) by Algorithm 3, and ok (p,)."""
        return null_directions(self.consolidated(y, tau))

    # ------------------------------------------------------------- tracking
    def step(self, params, s: PathState, nsteps=1):
        """nsteps projective Euler-Newton steps of every ACTIVE path, in place."""
        P = params
        n = self.n
        for _ in range(nsteps):
            act = np.flatnonzero(s.status == ACTIVE)
            if act.size == 0:
                break
            dE, dN, ok = self.directions(s.y[act], s.tau[act])
            for r, q in enumerate(act):
                s.steps[q] += 1
                err = np.abs(dN[r]).max() / max(1.0, np.abs(s.y[q]).max()) if ok[r] else np.inf
                accepted = bool(ok[r] and err <= P.tol_accept)
                if accepted:
                    if P.predictor == 1 and s.accepts[q] >= 1:   # keep the point being replaced
                        s.yprev[q], s.dEprev[q], s.tauprev[q] = s.yacc[q], s.dEacc[q], s.tauacc[q]
                    w = s.y[q] + dN[r]
                    nw = np.linalg.norm(w)
                    s.yacc[q] = w / nw
                    s.dEacc[q] = dE[r] / nw
                    s.tauacc[q] = s.tau[q]
                    s.accepts[q] += 1
                    s.streak[q] += 1
                    # divergence first: a path may reach tau = 0 at infinity
                    m = np.abs(s.yacc[q, :n]) / np.abs(s.yacc[q, n])
                    if (~(m < P.div_bound) | ~(m > 1.0 / P.div_bound)).any():
                        s.status[q] = DIVERGED
                        continue
                    if s.tauacc[q] == 0.0:
                        s.status[q] = CONVERGED
                        continue
                    if s.streak[q] >= P.grow_after:
                        s.dtau[q] = min(s.dtau[q] * P.grow, P.dtau_max)
                        s.streak[q] = 0
                else:
                    s.rejects[q] += 1
                    s.streak[q] = 0
                    if s.accepts[q] == 0:
                        # no accepted point yet: keep correcting at the start parameter
                        if not ok[r]:
                            s.status[q] = SINGULAR
                            continue
                        w = s.y[q] + dN[r]
                        s.y[q] = w / np.linalg.norm(w)
                        s.yacc[q] = s.y[q]
                        if s.steps[q] >= P.max_steps:
                            s.status[q] = MAX_STEPS
                        continue
                    # a rejected cubic prediction is retried with Euler at the
                    # same step size; a rejected Euler prediction shrinks the step
                    retry = P.predictor == 1 and bool(s.hflag[q])
                    if not retry:
                        s.dtau[q] *= P.shrink
                        if s.dtau[q] < P.dtau_min:
                            s.status[q] = UNDERFLOW
                            continue
                h = min(s.dtau[q], -s.tauacc[q])
                s.y[q] = _predict(P, s, q, h, accepted or not retry)
                s.tau[q] = s.tauacc[q] + h
                if s.steps[q] >= P.max_steps:
                    s.status[q] = MAX_STEPS
        return s

    def start(self, params, x0, tau0):
        return PathState.start(homogeneous_start(x0), tau0, params.dtau_init)

    def track(self, params, x0, tau0):
        """Track affine start points x0 (p, n) in homogeneous coordinates from
        tau0 to 0, dehomogenize, polish the converged ones with the affine
        oracle.  Returns (x (p,n), status, steps, polish_err, y_end (p,n+1))."""
        s = self.start(params, x0, tau0)
        while (s.status == ACTIVE).any():
            self.step(params, s, 16)
        x = dehomogenize(s.yacc)
        perr = np.full(s.p, np.nan)
        conv = np.flatnonzero(s.status == CONVERGED)
        if conv.size:
            xp, e = self.affine.polish(params, x[conv])
            x[conv] = xp
            perr[conv] = e
        return x, s.status.copy(), s.steps.copy(), perr, s.yacc.copy()


def affine_directions(osys, y, tau):
    """Algorithm 3 applied to the affine extended Jacobian [H_y, H_tau, H]
    (n x (n+2), no y^* row): the affine Euler and Newton directions."""
    H, Hy, Ht = osys.eval(y, tau)
    J = np.concatenate([Hy, Ht[:, :, None], H[:, :, None]], axis=2)
    return null_directions(J)

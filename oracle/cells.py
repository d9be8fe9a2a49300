"""Exact integer and rational bookkeeping of the oracle -- TEST INFRASTRUCTURE.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg use
this module; the CUDA library has its own independent implementation.

Contents (polyhedral homotopy of Huber and Sturmfels as reviewed in Section 2
of T. Chen, "GPU-accelerated path tracker for polyhedral homotopy"):

* ``t_exponents`` -- the lifted t-exponents of the cell-transformed homotopy
  H_k(y,t) = sum c y^a t^{<a,alpha> + w(a) - beta_k}, as integer numerators
  over a common denominator D (Python integers and ``fractions.Fraction``).
  The change of variables x = y t^alpha applied to eq. (1) gives these
  exponents; the paper defers the cell step to Huber and Sturmfels.
* ``mixed_cells`` -- brute-force enumeration of fine mixed cells for tiny n
  (one pair of points per support, strict lower-facet test); the mixed
  volume is the sum of |det V| over the cells (Bernshtein's theorem, the
  root count the paper's Section 2 relies on for generic coefficients).
* ``diagonalize`` / ``binomial_solutions`` / ``start_points`` -- all
  |det V| solutions of the binomial start system y^V = b of a cell, through
  an integer diagonal (Smith-type) form U V W = S.
* ``tau0`` -- the starting value of the logarithmic path parameter
  (Section 2.1): tau0 = ln(eps0) / s_min with s_min the smallest positive
  t-exponent, so that every non-cell term starts at most eps0.

Definitions shared with the library by specification only (not by code):

* cell kind "pairs": alpha solves V alpha = (w_{k,p0} - w_{k,p1})_k with
  V_k = a_{k,p1} - a_{k,p0}; D is the least positive common denominator of
  the entries of alpha; alpha_num = D alpha; beta_num_k = <a_{k,p0},
  alpha_num> + D w_{k,p0}.
* cell kind "explicit": alpha_num, beta_num, D given as they are.
* cell kind "lower": alpha_num, D given; beta_num_k = min over S_k of
  <a, alpha_num> + D w(a).
* e_{k,i} = <a_{k,i}, alpha_num> + D w_{k,i} - beta_num_k.

Parity: pinned by the CPU tests (closed-form 2-D mixed volume, Bezout count
for simplex supports, independence of the lifting, brute-force enumeration of
binomial solutions, residuals of the start systems).
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np


class NotACell(ValueError):
    """The pair choice is singular or is not a lower facet."""


class NonGeneric(ValueError):
    """A lifting attains a cell's lower facet at more than two points."""


def _supports(sysm):
    off = sysm.offsets
    return [[tuple(int(v) for v in sysm.exponents[off[k] + i]) for i in range(sysm.m[k])]
            for k in range(sysm.n)]


def _liftings(sysm):
    off = sysm.offsets
    return [[int(sysm.lifting[off[k] + i]) for i in range(sysm.m[k])] for k in range(sysm.n)]


def det_int(V):
    """Exact determinant of an integer matrix (fraction-free elimination)."""
    A = [[Fraction(int(x)) for x in row] for row in V]
    n = len(A)
    det = Fraction(1)
    for j in range(n):
        piv = next((i for i in range(j, n) if A[i][j] != 0), None)
        if piv is None:
            return 0
        if piv != j:
            A[j], A[piv] = A[piv], A[j]
            det = -det
        det *= A[j][j]
        for i in range(j + 1, n):
            f = A[i][j] / A[j][j]
            if f:
                for c in range(j, n):
                    A[i][c] -= f * A[j][c]
    assert det.denominator == 1
    return int(det)


def solve_rational(V, rhs):
    """Exact solution of V x = rhs over the rationals (V nonsingular)."""
    n = len(V)
    A = [[Fraction(int(x)) for x in row] + [Fraction(r)] for row, r in zip(V, rhs)]
    for j in range(n):
        piv = next((i for i in range(j, n) if A[i][j] != 0), None)
        if piv is None:
            raise NotACell("singular pair matrix")
        A[j], A[piv] = A[piv], A[j]
        for i in range(n):
            if i != j and A[i][j] != 0:
                f = A[i][j] / A[j][j]
                for c in range(j, n + 1):
                    A[i][c] -= f * A[j][c]
    return [A[i][n] / A[i][i] for i in range(n)]


def _lcm(a, b):
    return a * b // math.gcd(a, b)


def pair_matrix(sysm, pairs):
    S = _supports(sysm)
    return [[S[k][int(pairs[k][1])][j] - S[k][int(pairs[k][0])][j] for j in range(sysm.n)]
            for k in range(sysm.n)]


def t_exponents(sysm, cell):
    """Integer t-exponent numerators for a cell.

    ``cell`` is a dict: {"kind": "pairs", "pairs": (n,2)},
    {"kind": "explicit", "alpha_num", "beta_num", "denom"} or
    {"kind": "lower", "alpha_num", "denom"}.

    Returns dict(e=list[int] (M), D=int, alpha_num=list[int], beta_num=list[int]).
    Raises NotACell for a singular pair matrix or a pair that is not a lower
    facet, NonGeneric when a non-pair point also attains the facet.
    """
    n = sysm.n
    S = _supports(sysm)
    W = _liftings(sysm)
    kind = cell["kind"]
    if kind == "pairs":
        pairs = [(int(p[0]), int(p[1])) for p in cell["pairs"]]
        V = pair_matrix(sysm, pairs)
        rhs = [W[k][pairs[k][0]] - W[k][pairs[k][1]] for k in range(n)]
        if det_int(V) == 0:
            raise NotACell("singular pair matrix")
        alpha = solve_rational(V, rhs)
        D = 1
        for a in alpha:
            D = _lcm(D, a.denominator)
        alpha_num = [int(a * D) for a in alpha]
        beta_num = [sum(S[k][pairs[k][0]][j] * alpha_num[j] for j in range(n)) + D * W[k][pairs[k][0]]
                    for k in range(n)]
    elif kind == "explicit":
        alpha_num = [int(v) for v in cell["alpha_num"]]
        beta_num = [int(v) for v in cell["beta_num"]]
        D = int(cell["denom"])
    elif kind == "lower":
        alpha_num = [int(v) for v in cell["alpha_num"]]
        D = int(cell["denom"])
        beta_num = [min(sum(a[j] * alpha_num[j] for j in range(n)) + D * w for a, w in zip(S[k], W[k]))
                    for k in range(n)]
    else:
        raise ValueError(kind)
    if D <= 0:
        raise ValueError("denominator must be positive")
    e = []
    for k in range(n):
        for i, (a, w) in enumerate(zip(S[k], W[k])):
            e.append(sum(a[j] * alpha_num[j] for j in range(n)) + D * w - beta_num[k])
    if kind == "pairs":
        off = sysm.offsets
        for k in range(n):
            for i in range(sysm.m[k]):
                v = e[off[k] + i]
                on_pair = i in pairs[k]
                if on_pair and v != 0:
                    raise AssertionError("pair off its own facet")  # cannot happen
                if not on_pair and v < 0:
                    raise NotACell("pair is not a lower facet")
                if not on_pair and v == 0:
                    raise NonGeneric("lifting is not generic for this cell")
    return dict(e=e, D=D, alpha_num=alpha_num, beta_num=beta_num)


def mixed_cells(sysm):
    """All fine mixed cells by brute force over one pair per support.

    Returns (cells, mixed_volume); each cell is dict(pairs, det).  Raises
    NonGeneric when the lifting is not generic (a facet with a third point).
    Exponential in n: for tiny systems only.
    """
    n = sysm.n
    cells, mv = [], 0
    pair_lists = [list(itertools.combinations(range(sysm.m[k]), 2)) for k in range(n)]
    for choice in itertools.product(*pair_lists):
        V = pair_matrix(sysm, choice)
        d = det_int(V)
        if d == 0:
            continue
        try:
            t_exponents(sysm, {"kind": "pairs", "pairs": choice})
        except NotACell:
            continue
        cells.append(dict(pairs=[list(p) for p in choice], det=abs(d)))
        mv += abs(d)
    return cells, mv


def diagonalize(V):
    """Integer matrices U, W (unimodular) and the diagonal d with
    U V W = diag(d).  Plain pivot-and-reduce elimination on integers."""
    n = len(V)
    A = [[int(x) for x in row] for row in V]
    U = [[int(i == j) for j in range(n)] for i in range(n)]
    W = [[int(i == j) for j in range(n)] for i in range(n)]

    def swap_rows(M, a, b):
        M[a], M[b] = M[b], M[a]

    def swap_cols(M, a, b):
        for row in M:
            row[a], row[b] = row[b], row[a]

    for t in range(n):
        while True:
            cand = [(abs(A[i][j]), i, j) for i in range(t, n) for j in range(t, n) if A[i][j] != 0]
            if not cand:
                raise NotACell("singular matrix")
            _, pi, pj = min(cand)
            if pi != t:
                swap_rows(A, pi, t)
                swap_rows(U, pi, t)
            if pj != t:
                swap_cols(A, pj, t)
                swap_cols(W, pj, t)
            done = True
            for i in range(t + 1, n):          # rows: row_i -= q row_t
                q = A[i][t] // A[t][t]
                if q:
                    for c in range(n):
                        A[i][c] -= q * A[t][c]
                        U[i][c] -= q * U[t][c]
                if A[i][t] != 0:
                    done = False
            for j in range(t + 1, n):          # cols: col_j -= q col_t
                q = A[t][j] // A[t][t]
                if q:
                    for r in range(n):
                        A[r][j] -= q * A[r][t]
                        W[r][j] -= q * W[r][t]
                if A[t][j] != 0:
                    done = False
            if done:
                break
    return U, [A[i][i] for i in range(n)], W


def binomial_solutions(V, b, limit=None):
    """All solutions y in (C*)^n of prod_j y_j^{V[k][j]} = b_k, k = 0..n-1.

    With U V W = diag(d) (U, W unimodular), V^{-1} = W diag(1/d) U, and the
    solutions are log y = V^{-1} log b + 2 pi i W diag(1/d) m for
    m_j = 0..|d_j|-1: |det V| of them.  The first term comes from a linear
    solve with V itself (numpy.linalg.solve); the rational vector
    W diag(1/d) m is reduced modulo 1 exactly (integers), since only its
    fractional part changes y.  (Forming W zeta in floating point instead
    cancels badly when W has large entries.)
    """
    n = len(V)
    U, d, W = diagonalize(V)
    logb = np.log(np.asarray(b, dtype=np.complex128))
    z0 = np.linalg.solve(np.array(V, dtype=np.float64), logb)
    L = 1
    for dj in d:
        L = _lcm(L, abs(int(dj)))
    sols = []
    for m in itertools.product(*[range(abs(dj)) for dj in d]):
        if limit is not None and len(sols) >= limit:
            break
        # numerators over L of (W diag(1/d) m)_r, reduced mod L
        num = [sum(int(W[r][j]) * int(m[j]) * (L // int(d[j])) for j in range(n)) % L for r in range(n)]
        frac = np.array([v / L for v in num])
        sols.append(np.exp(z0 + 2j * np.pi * frac))
    return np.array(sols, dtype=np.complex128).reshape(len(sols), n)


def start_points(sysm, pairs, limit=None):
    """Solutions of the cell's binomial start system H(y, t=0) = 0:
    c_{k,p0} y^{a_{k,p0}} + c_{k,p1} y^{a_{k,p1}} = 0 (the first `limit` of
    them in the enumeration order when a limit is given)."""
    off = sysm.offsets
    V = pair_matrix(sysm, pairs)
    b = [-sysm.coeffs[off[k] + int(pairs[k][0])] / sysm.coeffs[off[k] + int(pairs[k][1])]
         for k in range(sysm.n)]
    return binomial_solutions(V, b, limit)


def binomial_points(V, b, ks):
    """The solutions log y = V^{-1} (log b + 2 pi i k) of the binomial system
    prod_j y_j^{V[k][j]} = b_k for the integer vectors k (rows of ks): every
    solution has this form, and k, k' give the same y exactly when k - k' is
    in V Z^n.  A plain linear solve per k (numpy.linalg.solve), usable at any
    |det V|."""
    Vf = np.array(V, dtype=np.float64)
    logb = np.log(np.asarray(b, dtype=np.complex128))
    ks = np.asarray(ks, dtype=np.int64).reshape(-1, len(V))
    out = np.empty(ks.shape, dtype=np.complex128)
    for i, k in enumerate(ks):
        out[i] = np.exp(np.linalg.solve(Vf, logb + 2j * np.pi * k))
    return out


def start_points_at(sysm, pairs, ks):
    """Start points of the cell's binomial start system for chosen lattice
    vectors k (see binomial_points)."""
    off = sysm.offsets
    V = pair_matrix(sysm, pairs)
    b = [-sysm.coeffs[off[k] + int(pairs[k][0])] / sysm.coeffs[off[k] + int(pairs[k][1])]
         for k in range(sysm.n)]
    return binomial_points(V, b, ks)


def tau0(e, D, eps0=1e-10):
    """tau0 = ln(eps0) / s_min, s_min = min over e > 0 of e / D."""
    pos = [v for v in e if v > 0]
    if not pos:
        return math.log(eps0)
    return math.log(eps0) / (min(pos) / D)

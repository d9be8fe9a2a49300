"""Pins of the oracle's exact cell bookkeeping and start systems (CPU only).

* hand-derived t-exponents of two cells (tests/golden/cells_hand.json);
* the mixed volume of two plane polygons in closed form,
  MV(P1, P2) = area(P1 + P2) - area(P1) - area(P2) (scipy's convex hull);
* Bezout's count prod d_k for full simplex supports {0, d e_1, ..., d e_n};
* the mixed volume does not depend on the (generic) lifting;
* the diagonal form U V W = diag(d) with unimodular U, W;
* binomial start solutions: count |det V|, residuals, and the same set as a
  brute-force enumeration of V^{-1}(log b + 2 pi i m) over a box of m.
"""
import itertools
import json
import os

import numpy as np
import pytest
from scipy.spatial import ConvexHull, QhullError

import workloads as W
from oracle import cells

GOLD = os.path.join(os.path.dirname(__file__), "golden", "cells_hand.json")


def _system_from(supports, lifting):
    n = len(supports)
    exps = np.array([a for S in supports for a in S], dtype=np.int32)
    M = exps.shape[0]
    return W.LaurentSystem(n, [len(S) for S in supports], exps, np.ones(M, complex),
                           np.array([w for L in lifting for w in L], dtype=np.int64))


def test_hand_derived_cells():
    for case in json.load(open(GOLD))["cases"]:
        s = _system_from(case["supports"], case["lifting"])
        te = cells.t_exponents(s, {"kind": "pairs", "pairs": case["pairs"]})
        assert te["e"] == case["e"]
        assert te["D"] == case["denom"]
        assert te["alpha_num"] == case["alpha_num"]
        assert te["beta_num"] == case["beta_num"]
        assert abs(cells.det_int(cells.pair_matrix(s, case["pairs"]))) == case["det"]
        ex = cells.t_exponents(s, {"kind": "explicit", "alpha_num": case["alpha_num"],
                                   "beta_num": case["beta_num"], "denom": case["denom"]})
        assert ex["e"] == case["e"]
        lo = cells.t_exponents(s, {"kind": "lower", "alpha_num": case["alpha_num"],
                                   "denom": case["denom"]})
        assert lo["e"] == case["e"]


def test_not_a_cell_rejected():
    case = json.load(open(GOLD))["cases"][0]
    s = _system_from(case["supports"], case["lifting"])
    # pairs (1,0),(0,1) and (0,0),(2,1): alpha = (-2/3, 1/3), D = 3,
    # beta_num_1 = -2 + 3*2 = 4, so the point (0,0) of S_1 gets e = -4 < 0
    with pytest.raises(cells.NotACell):
        cells.t_exponents(s, {"kind": "pairs", "pairs": [[1, 2], [0, 1]]})


def _area(pts):
    pts = np.unique(np.asarray(pts, dtype=float), axis=0)
    if len(pts) < 3:
        return 0.0
    try:
        return ConvexHull(pts).volume
    except QhullError:
        return 0.0


def _generic_mv(s, seed0):
    for att in range(50):
        lift = np.random.default_rng([seed0, att]).integers(0, 1000, size=s.M)
        try:
            return cells.mixed_cells(s.with_lifting(lift))[1]
        except cells.NonGeneric:
            continue
    raise RuntimeError("no generic lifting found")


@pytest.mark.parametrize("seed", range(12))
def test_mixed_volume_closed_form_2d(seed):
    rng = np.random.default_rng(seed)
    s = W.laurent_system(seed, 2, [int(rng.integers(3, 6)), int(rng.integers(3, 6))], -2, 2, 0)
    P1, P2 = s.support(0), s.support(1)
    mink = [p + q for p in P1 for q in P2]
    closed = _area(mink) - _area(P1) - _area(P2)
    assert _generic_mv(s, seed) == round(closed)


@pytest.mark.parametrize("degs", [(1, 1), (2, 3), (3, 2), (1, 2, 2), (2, 2, 2)])
def test_bezout_simplex_supports(degs):
    n = len(degs)
    supports = []
    for d in degs:
        S = [[0] * n]
        for j in range(n):
            v = [0] * n
            v[j] = d
            S.append(v)
        supports.append(S)
    s = _system_from(supports, [[0] * (n + 1)] * n)
    assert _generic_mv(s, 99) == int(np.prod(degs))


@pytest.mark.parametrize("seed", range(4))
def test_mixed_volume_independent_of_lifting(seed):
    s = W.laurent_system(40 + seed, 3, 4, -1, 2, 0)
    assert _generic_mv(s, 1) == _generic_mv(s, 2)


@pytest.mark.parametrize("seed", range(8))
def test_diagonal_form(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 6))
    while True:
        V = rng.integers(-4, 5, size=(n, n))
        if cells.det_int(V.tolist()) != 0:
            break
    U, d, Wm = cells.diagonalize(V.tolist())
    U, Wm = np.array(U, dtype=object), np.array(Wm, dtype=object)
    assert (U.dot(np.array(V, dtype=object)).dot(Wm) == np.diag(np.array(d, dtype=object))).all()
    assert abs(cells.det_int(U.tolist())) == 1 and abs(cells.det_int(Wm.tolist())) == 1
    assert abs(int(np.prod(d))) == abs(cells.det_int(V.tolist()))


@pytest.mark.parametrize("seed", range(6))
def test_binomial_solutions_2d_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    while True:
        V = rng.integers(-3, 4, size=(2, 2))
        det = cells.det_int(V.tolist())
        if det != 0:
            break
    b = np.exp(1j * rng.uniform(0, 2 * np.pi, 2)) * rng.uniform(0.5, 2, 2)
    sols = cells.binomial_solutions(V.tolist(), b)
    assert len(sols) == abs(det)
    res = np.prod(sols[:, None, :] ** V[None, :, :], axis=2) - b[None, :]
    assert np.abs(res).max() < 1e-12
    # brute force: z = V^{-1}(log b + 2 pi i m) over a box of m, dedup
    Vinv = np.linalg.inv(V.astype(float))
    found = []
    for m in itertools.product(range(-abs(det), abs(det) + 1), repeat=2):
        y = np.exp(Vinv @ (np.log(b) + 2j * np.pi * np.array(m)))
        if not any(np.abs(y - f).max() < 1e-9 for f in found):
            found.append(y)
    assert len(found) == abs(det)
    for f in found:
        assert np.min(np.abs(sols - f[None, :]).max(axis=1)) < 1e-9


def test_start_points_solve_the_cell_system(oracle_mod):
    s = W.config2(0)
    for att in range(20):
        try:
            cl, mv = cells.mixed_cells(W.config2(att))
            s = W.config2(att)
            break
        except cells.NonGeneric:
            continue
    assert mv == sum(c["det"] for c in cl)
    for c in cl[:3]:
        te = cells.t_exponents(s, {"kind": "pairs", "pairs": c["pairs"]})
        y0 = cells.start_points(s, c["pairs"])
        assert len(y0) == c["det"]
        osys = oracle_mod.System(s, te["e"], te["D"])
        H, _, _ = osys.eval(y0, np.full(len(y0), -1e4))
        SH, _, _ = osys.scale(y0, np.full(len(y0), -1e4))
        assert np.max(np.abs(H) / SH) < 1e-13


def test_start_points_large_determinant():
    """A planted n=8 cell with |det V| ~ 1e5, whose unimodular factors have
    entries ~1e8: the start points still solve y^V = b to rounding level."""
    import _util
    s, pairs, _, d = _util.planted_case(W.config5, 4096)
    V = np.array(cells.pair_matrix(s, pairs))
    off = s.offsets
    b = np.array([-s.coeffs[off[k] + pairs[k][0]] / s.coeffs[off[k] + pairs[k][1]] for k in range(s.n)])
    y = cells.start_points(s, pairs, limit=2000)
    res = np.abs(np.prod(y[:, None, :] ** V[None, :, :], axis=2) / b[None, :] - 1).max()
    assert res < 1e-12
    # distinct points
    assert _util.min_separation(y) > 1e-8


def _pair_data(s, pairs):
    V = np.array(cells.pair_matrix(s, pairs))
    off = s.offsets
    b = np.array([-s.coeffs[off[k] + pairs[k][0]] / s.coeffs[off[k] + pairs[k][1]] for k in range(s.n)])
    return V, b


def _powprod(y, V):
    """prod_j y_j^{V[k][j]} by repeated multiplication (complex128)."""
    out = np.ones((y.shape[0], V.shape[0]), dtype=np.complex128)
    for k in range(V.shape[0]):
        for j in range(V.shape[1]):
            e = int(V[k, j])
            f = y[:, j] if e >= 0 else 1.0 / y[:, j]
            for _ in range(abs(e)):
                out[:, k] *= f
    return out


def test_binomial_points_cover_the_exact_enumeration():
    """Small |det V|: points for k over a box that meets every coset of
    V Z^n are exactly the |det V| solutions of the exact enumeration."""
    import _util

    def small(att):
        s = W.laurent_system(7, 2, 4, -2, 2, 0, attempt=att)
        lift, pairs = W.planted_lifting(7, s.m, 16, attempt=att)
        return s.with_lifting(lift), pairs

    s, pairs, _, d = _util.planted_case(small, 3, 12)
    V, b = _pair_data(s, pairs)
    exact = cells.start_points(s, pairs)
    assert exact.shape[0] == d
    # d e_j lies in V Z^n (d V^{-1} is integral), so [0, d)^n meets every coset
    ks = np.array(list(itertools.product(*([range(d)] * s.n))), dtype=np.int64)
    ys = cells.binomial_points(V, b, ks)
    # distinct points of ys
    reps = []
    for y in ys:
        if not any(np.abs(y - r).max() < 1e-9 for r in reps):
            reps.append(y)
    assert len(reps) == d
    for r in reps:
        assert np.abs(exact - r).max(axis=1).min() < 1e-10


def test_binomial_points_large_determinant():
    """Many-systems workload systems (n up to 24, |det V| far beyond 2^62):
    points for k = j e_1 solve y^V = b (checked by repeated multiplication)
    and are distinct."""
    import _util
    for idx in (0, 3, 7):
        s, pairs = W.config4_system(idx)
        V, b = _pair_data(s, pairs)
        ks = np.zeros((24, s.n), np.int64)
        ks[:, 0] = np.arange(24)
        y = cells.binomial_points(V, b, ks)
        res = np.abs(_powprod(y, V) / b[None, :] - 1).max()
        assert res < 1e-9, (idx, s.n, res)
        assert _util.min_separation(y) > 1e-8

"""The C ABI library loads and exports every entry point declared in
include/hpt.h, and its host-only exact integer bookkeeping (no device work)
is bit-identical to the oracle's (CPU only)."""
import json
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import cells

import _util

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hpt():
    from paper_2111_14317_gb300 import build
    build.build()
    from paper_2111_14317_gb300 import hpt as mod
    return mod


def test_exports_every_declared_symbol(hpt):
    import ctypes
    hdr = open(os.path.join(ROOT, "include", "hpt.h")).read()
    declared = set(re.findall(r"^\s*(?:hpt_status|void|const char\*)\s+(hpt_\w+)\s*\(", hdr, re.M))
    assert len(declared) >= 15
    lib = ctypes.CDLL(hpt.LIB_PATH)
    missing = [d for d in declared if not hasattr(lib, d)]
    assert not missing, missing
    assert declared == set(hpt.EXPORTS)


def _cmp(hpt, s, cell):
    ref = cells.t_exponents(s, cell)
    got = hpt.lift_exponents(s.n, s.m, s.exponents, s.lifting, cell)
    assert got["e"] == ref["e"] and got["D"] == ref["D"]
    assert got["alpha_num"] == ref["alpha_num"] and got["beta_num"] == ref["beta_num"]


def test_lift_golden(hpt):
    for case in json.load(open(os.path.join(ROOT, "tests", "golden", "cells_hand.json")))["cases"]:
        exps = np.array([a for S in case["supports"] for a in S], dtype=np.int32)
        s = W.LaurentSystem(len(case["supports"]), [len(S) for S in case["supports"]], exps,
                            np.ones(len(exps), complex),
                            np.array([w for L in case["lifting"] for w in L], dtype=np.int64))
        got = hpt.lift_exponents(s.n, s.m, s.exponents, s.lifting, {"kind": "pairs", "pairs": case["pairs"]})
        assert got["e"] == case["e"] and got["D"] == case["denom"]


@pytest.mark.parametrize("cfg", [W.config1, W.config2])
def test_lift_every_brute_force_cell(hpt, cfg):
    s, cl, _ = _util.first_generic(cfg)
    for c in cl:
        _cmp(hpt, s, {"kind": "pairs", "pairs": c["pairs"]})


@pytest.mark.parametrize("name", ["n16", "n7_ragged", "n24"])
def test_lift_lower_envelope(hpt, name):
    s, cell = _util.eval_case(name)
    _cmp(hpt, s, cell)
    _cmp(hpt, s, {"kind": "explicit", "alpha_num": cell["alpha_num"],
                  "beta_num": cells.t_exponents(s, cell)["beta_num"], "denom": cell["denom"]})


def test_lift_errors(hpt):
    case = json.load(open(os.path.join(ROOT, "tests", "golden", "cells_hand.json")))["cases"][0]
    exps = np.array([a for S in case["supports"] for a in S], dtype=np.int32)
    lift = np.array([w for L in case["lifting"] for w in L], dtype=np.int64)
    with pytest.raises(hpt.HptError) as e:
        hpt.lift_exponents(2, [3, 3], exps, lift, {"kind": "pairs", "pairs": [[1, 2], [0, 1]]})
    assert e.value.code == 5
    lift2 = lift.copy()
    lift2[2] = 0            # (0,1) lands on the facet of the first cell: not generic
    lift2[1] = 0
    with pytest.raises(hpt.HptError) as e:
        hpt.lift_exponents(2, [3, 3], exps, lift2, {"kind": "pairs", "pairs": [[0, 1], [0, 1]]})
    assert e.value.code == 5
    # singular pair matrix: both pair differences are multiples of (1, 0)
    bad = np.array([[0, 0], [1, 0], [2, 0], [0, 0], [2, 0], [1, 2]], np.int32)
    with pytest.raises(hpt.HptError) as e:
        hpt.lift_exponents(2, [3, 3], bad, lift, {"kind": "pairs", "pairs": [[0, 1], [0, 1]]})
    assert e.value.code == 5


@pytest.mark.parametrize("cfg", [W.config1, W.config2])
def test_binomial_start_matches_oracle(hpt, cfg):
    """The library's start points (its own integer diagonal form) are the
    oracle's start set: same count |det V|, same points up to order."""
    s, cl, _ = _util.first_generic(cfg)
    for c in cl[:8]:
        y_lib, tot = hpt.binomial_start(s.n, s.m, s.exponents, s.coeffs, c["pairs"])
        assert tot == c["det"]
        assert _util.match_solutions(y_lib, cells.start_points(s, c["pairs"])) < 1e-9


def test_binomial_start_large_determinant(hpt):
    """n=8 planted cell with |det V| ~ 1e5 (unimodular factors with entries
    ~1e8): the library's start points solve y^V = b to rounding level and are
    distinct."""
    s, pairs, _, d = _util.planted_case(W.config5, 4096)
    y, tot = hpt.binomial_start(s.n, s.m, s.exponents, s.coeffs, pairs, 1000, 3000)
    assert tot == d
    V = np.array(cells.pair_matrix(s, pairs))
    off = s.offsets
    b = np.array([-s.coeffs[off[k] + pairs[k][0]] / s.coeffs[off[k] + pairs[k][1]] for k in range(s.n)])
    res = np.abs(np.prod(y[:, None, :] ** V[None, :, :], axis=2) / b[None, :] - 1).max()
    assert res < 1e-12
    assert _util.min_separation(y) > 1e-8


def test_binomial_points_match_oracle(hpt):
    """hpt_binomial_points equals the oracle's linear-solve start points
    (FP64 rounding only) on many-systems workload systems."""
    for idx in (0, 1, 5):
        s, pairs = W.config4_system(idx)
        V = np.array(cells.pair_matrix(s, pairs))
        off = s.offsets
        b = np.array([-s.coeffs[off[k] + pairs[k][0]] / s.coeffs[off[k] + pairs[k][1]] for k in range(s.n)])
        rng = np.random.default_rng(idx)
        ks = rng.integers(-50, 50, size=(16, s.n))
        got = hpt.binomial_points(s.n, s.m, s.exponents, s.coeffs, pairs, ks)
        want = cells.binomial_points(V, b, ks)
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err < 1e-9, (idx, err)


def test_binomial_points_singular(hpt):
    s, pairs = W.config4_system(0)
    pr = np.array(pairs).copy()
    pr[1] = pr[0] if s.m[1] > max(pr[0]) else pr[1]
    # a pair matrix with two equal rows: copy equation 0's support into 1's pairs
    ex = np.array(s.exponents).copy()
    off = s.offsets
    ex[off[1] + pr[1][0]] = ex[off[0] + pr[0][0]]
    ex[off[1] + pr[1][1]] = ex[off[0] + pr[0][1]]
    with pytest.raises(hpt.HptError) as ei:
        hpt.binomial_points(s.n, s.m, ex, s.coeffs, pr, np.zeros((1, s.n), np.int64))
    assert ei.value.code == 5


def test_lift_large_planted_cells_bit_exact(hpt):
    """Planted pair cells of the many-systems workload (n up to 24, |det V|
    beyond 64-bit range): the library's exact lift equals the oracle's."""
    for idx in (1, 3, 4, 5):
        s, pairs = W.config4_system(idx)
        cell = {"kind": "pairs", "pairs": pairs}
        want = cells.t_exponents(s, cell)
        got = hpt.lift_exponents(s.n, s.m, s.exponents, s.lifting, cell)
        assert got["e"] == [int(v) for v in want["e"]]
        assert got["D"] == want["D"]


def test_lift_singular_planted_cell(hpt):
    """A planted cell whose pair matrix has two equal rows is refused
    (HPT_ENOTCELL) by the exact modular determinant check."""
    s, pairs = W.config4_system(4)
    ex = np.array(s.exponents).copy()
    off = s.offsets
    ex[off[1] + pairs[1][0]] = ex[off[0] + pairs[0][0]]
    ex[off[1] + pairs[1][1]] = ex[off[0] + pairs[0][1]]
    with pytest.raises(hpt.HptError) as ei:
        hpt.lift_exponents(s.n, s.m, ex, s.lifting, {"kind": "pairs", "pairs": pairs})
    assert ei.value.code == 5


@pytest.mark.timeout(60)
def test_binomial_start_singular_pairs_cell(hpt):
    """A pairs cell whose pair matrix is singular although no row is zero
    (rows (1, 0) and (2, 0)) is refused with HPT_ENOTCELL; every prime the
    exact determinant tries divides 0, so the search for a usable prime has to
    stop once det V = 0 is certain."""
    exps = np.array([[0, 0], [1, 0], [0, 1],
                     [0, 0], [2, 0], [1, 1]], dtype=np.int32)
    coeffs = np.ones(6, complex)
    with pytest.raises(hpt.HptError) as ei:
        hpt.binomial_start(2, [3, 3], exps, coeffs, [[0, 1], [0, 1]])
    assert ei.value.code == 5

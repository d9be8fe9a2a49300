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

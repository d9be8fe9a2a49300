"""The library's mixed-cell search (hpt_mixed_cells, host code; CPU tests).

* On configs 1 and 2 and on dozens of small random systems it finds exactly
  the oracle's brute-force cells (same pairs, same mixed volume, and the BKK
  root counts of those configs).
* Beyond brute force (n = 6 and 8) the mixed volume it reports does not
  depend on the lifting (two independent generic liftings agree), every cell
  passes the exact cell test, and no two cells coincide.
* cap bounds the cells written while the count and volume stay complete.
"""
import numpy as np
import pytest

import workloads as W
from oracle import cells

import _util


def _canon(cl):
    return sorted(tuple(tuple(sorted(int(v) for v in p)) for p in c) for c in cl)


@pytest.fixture(scope="module")
def hpt_host():
    from paper_2111_14317_gb300 import build
    build.build()
    from paper_2111_14317_gb300 import hpt
    return hpt


@pytest.mark.parametrize("cfg", [W.config1, W.config2])
def test_cells_equal_brute_force_on_configs(hpt_host, cfg):
    s, cl, mv = _util.first_generic(cfg)
    pc, vol = hpt_host.mixed_cells(s.n, s.m, s.exponents, s.lifting)
    assert vol == mv
    assert _canon(pc) == _canon([c["pairs"] for c in cl])


@pytest.mark.parametrize("n,m,seed", [(3, 4, 11), (4, 4, 12), (5, 4, 13)])
def test_cells_equal_brute_force_random(hpt_host, n, m, seed):
    for att in range(10):
        s = W.laurent_system(seed, n, m, -2, 2, 64, attempt=att)
        try:
            cl, mv = cells.mixed_cells(s)
        except cells.NonGeneric:
            continue
        pc, vol = hpt_host.mixed_cells(s.n, s.m, s.exponents, s.lifting)
        assert vol == mv and _canon(pc) == _canon([c["pairs"] for c in cl])
        return
    pytest.skip("no generic sample")


@pytest.mark.parametrize("n,m", [(2, 4), (3, 4), (3, 5), (4, 4)])
def test_cells_equal_brute_force_sweep(hpt_host, n, m):
    """Many generic random systems per shape (lifting up to 2^12): the same
    cells and mixed volume as brute force every time."""
    checked = 0
    for seed in range(10):
        s = W.laurent_system(900 + seed, n, m, -2, 2, 1 << 12, attempt=seed)
        try:
            cl, mv = cells.mixed_cells(s)
        except cells.NonGeneric:
            continue
        pc, vol = hpt_host.mixed_cells(s.n, s.m, s.exponents, s.lifting)
        assert vol == mv and _canon(pc) == _canon([c["pairs"] for c in cl]), seed
        checked += 1
    assert checked >= 5


@pytest.mark.parametrize("n,m", [(6, 5), (8, 5)])
def test_volume_is_independent_of_the_lifting(hpt_host, n, m):
    s = W.laurent_system(40 + n, n, m, -2, 2, 64)
    vols = []
    for seed in (1, 2):
        lift = np.random.default_rng(seed).integers(0, 1 << 20, size=s.M).astype(np.int64)
        pc, vol = hpt_host.mixed_cells(s.n, s.m, s.exponents, lift)
        assert len(_canon(pc)) == len(set(map(tuple, _canon(pc))))
        for c in pc[:50]:
            hpt_host.lift_exponents(s.n, s.m, s.exponents, lift, {"kind": "pairs", "pairs": c})
        vols.append(vol)
    assert vols[0] == vols[1] > 0


def test_cap_and_count(hpt_host):
    s, cl, mv = _util.first_generic(W.config2)
    pc, vol = hpt_host.mixed_cells(s.n, s.m, s.exponents, s.lifting, cap=3)
    assert pc.shape[0] == 3 and vol == mv
    full, _ = hpt_host.mixed_cells(s.n, s.m, s.exponents, s.lifting)
    assert _canon(pc) == sorted(_canon(full[:3]))


def test_cells_refuse_a_lifting_beyond_the_exact_range(hpt_host):
    """A lifting value outside [-2^40, 2^40] is refused up front (HPT_ERANGE),
    not dropped cell by cell."""
    s, _, _ = _util.first_generic(W.config2)
    lift = s.lifting.copy()
    lift[3] = (1 << 40) + 1
    with pytest.raises(hpt_host.HptError) as ei:
        hpt_host.mixed_cells(s.n, s.m, s.exponents, lift)
    assert ei.value.code == 4


def test_cells_report_a_non_generic_lifting(hpt_host):
    """A lifting with an exact tie (a non-cell point lifted onto a cell's lower
    facet) is reported (HPT_ENOTCELL, 'not generic') instead of returning a
    short mixed volume; the oracle's brute force calls the same lifting
    non-generic."""
    s, cl, _ = _util.first_generic(W.config2)
    pairs = cl[0]["pairs"]
    D = cells.t_exponents(s, {"kind": "pairs", "pairs": pairs})["D"]
    lift = s.lifting * D          # the cell's inner normal becomes integral
    s2 = W.LaurentSystem(s.n, s.m, s.exponents, s.coeffs, lift)
    te = cells.t_exponents(s2, {"kind": "pairs", "pairs": pairs})
    assert te["D"] == 1
    o = s.offsets[0]
    i = [q for q in range(s.m[0]) if q not in pairs[0]][0]
    lift[o + i] = te["beta_num"][0] - int(np.asarray(s.exponents[o + i], np.int64) @ np.asarray(te["alpha_num"]))
    s3 = W.LaurentSystem(s.n, s.m, s.exponents, s.coeffs, lift)
    with pytest.raises(cells.NonGeneric):
        cells.mixed_cells(s3)
    with pytest.raises(hpt_host.HptError) as ei:
        hpt_host.mixed_cells(s3.n, s3.m, s3.exponents, s3.lifting)
    assert ei.value.code == 5 and "not generic" in str(ei.value)

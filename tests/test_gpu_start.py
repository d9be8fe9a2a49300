"""Start points of a cell on the device (GPU).

hpt_binomial_start_device equals the host enumeration hpt_binomial_start
(relative 1e-13: only the device exp/sincos differ) and, for small cells,
the oracle's exact start points as a set; the points solve the binomial start
system (the cell's two monomials per equation) to rounding; ranges at the
end of a large enumeration, count 0 and out-of-range requests behave as on
the host.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cells

import _util

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


def _binomial_residual(s, pairs, y):
    """max_k |c0 y^a0 + c1 y^a1| / (|c0 y^a0| + |c1 y^a1|) (numpy powers)."""
    off = s.offsets
    worst = 0.0
    for k in range(s.n):
        i0, i1 = off[k] + pairs[k][0], off[k] + pairs[k][1]
        t0 = s.coeffs[i0] * np.prod(y ** s.exponents[i0][None, :], axis=1)
        t1 = s.coeffs[i1] * np.prod(y ** s.exponents[i1][None, :], axis=1)
        worst = max(worst, float(np.max(np.abs(t0 + t1) / (np.abs(t0) + np.abs(t1)))))
    return worst


def test_device_start_points_small_cells(hpt):
    s, cl, mv = _util.first_generic(W.config2)
    for c in cl:
        y_h, tot = hpt.binomial_start(s.n, s.m, s.exponents, s.coeffs, c["pairs"])
        y_d, tot_d = hpt.binomial_start_device(s.n, s.m, s.exponents, s.coeffs, c["pairs"])
        assert tot == tot_d == c["det"]
        y_d = y_d.cpu().numpy()
        assert _rel(y_d, y_h) < 1e-13
        assert _util.match_solutions(y_d, cells.start_points(s, c["pairs"])) < 1e-12


@pytest.mark.parametrize("shape", [(14, 184), (24, 324)], ids=["n14", "n24"])
def test_device_start_points_large_cells(hpt, shape):
    s, pairs = W.paper_shape(*shape)
    _, tot = hpt.binomial_start(s.n, s.m, s.exponents, s.coeffs, pairs, 0, 0)
    assert tot == abs(cells.det_int(cells.pair_matrix(s, pairs)))
    for first, count in ((0, 4096), (tot - 1000, 1000), (tot // 3, 777)):
        y_h, _ = hpt.binomial_start(s.n, s.m, s.exponents, s.coeffs, pairs, first, count)
        y_d, _ = hpt.binomial_start_device(s.n, s.m, s.exponents, s.coeffs, pairs, first, count)
        y_d = y_d.cpu().numpy()
        assert _rel(y_d, y_h) < 1e-13
        assert _binomial_residual(s, [tuple(p) for p in pairs], y_d) < 1e-11
    # a million points at once, sampled against the host
    count = min(tot, 1 << 20)
    y_d, _ = hpt.binomial_start_device(s.n, s.m, s.exponents, s.coeffs, pairs, 0, count)
    idx = np.concatenate([np.random.default_rng(1).choice(count, 200, replace=False), [0, count - 1]])
    for i in idx[:40]:
        y_h, _ = hpt.binomial_start(s.n, s.m, s.exponents, s.coeffs, pairs, int(i), 1)
        assert _rel(y_d[int(i)].cpu().numpy()[None, :], y_h) < 1e-13


def test_device_start_points_edges(hpt):
    s, cl, mv = _util.first_generic(W.config2)
    c = cl[0]
    y_d, tot = hpt.binomial_start_device(s.n, s.m, s.exponents, s.coeffs, c["pairs"], 0, 0)
    assert y_d.shape == (0, s.n) and tot == c["det"]
    with pytest.raises(hpt.HptError) as ei:
        hpt.binomial_start_device(s.n, s.m, s.exponents, s.coeffs, c["pairs"], 1, tot)
    assert ei.value.code == 4

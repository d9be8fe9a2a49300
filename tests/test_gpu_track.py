"""Whole tracks on the GPU (GPU).

For configs 1 and 2 every mixed cell's start points are tracked to t = 1 in
the FP64 form and in the mixed split-BF16 form, each followed by the FP64
polish: every path converges, the number of distinct solutions is the
mixed volume (BKK), and the solutions match the oracle's one to one within
relative 1e-9."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cells

import _util

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("cfg", [W.config1, W.config2], ids=["config1", "config2"])
def test_track_bkk_and_parity(hpt, oracle_mod, cfg, prec):
    s, cl, mv = _util.first_generic(cfg)
    P = oracle_mod.Params()
    gx, ox = [], []
    for c in cl:
        cell = {"kind": "pairs", "pairs": c["pairs"]}
        te = cells.t_exponents(s, cell)
        osys = oracle_mod.System(s, te["e"], te["D"])
        y0 = cells.start_points(s, c["pairs"])
        x_o, st_o, _, _ = osys.track(P, y0, cells.tau0(te["e"], te["D"]))
        assert (st_o == oracle_mod.CONVERGED).all()
        h = hpt.System.from_laurent(s, cell, prec)
        prm = hpt.Params(tol_accept=1e-3 if prec == 0 else 3e-3)
        x, st, steps = h.track(torch.from_numpy(y0).cuda(), prm)
        assert h.device_error() == 0
        st = st.cpu().numpy()
        assert (st == hpt.CONVERGED).all(), np.bincount(st)
        gx.append(x.cpu().numpy())
        ox.append(x_o)
        h.close()
    gx, ox = np.concatenate(gx), np.concatenate(ox)
    assert len(gx) == mv
    d = np.abs(gx[:, None, :] - gx[None, :, :]).max(-1)
    np.fill_diagonal(d, np.inf)
    assert d.min() > 1e-6
    assert _util.match_solutions(gx, ox) < 1e-9


def _large_exponent_case():
    """n = 3, one monomial per equation with sum |a_j| between 66 and 120
    beside four with exponents in [-2, 2]; lifting 0 on monomials 0 and 1 of
    every equation and U{1..16} elsewhere, so those pairs form a planted cell
    (|det V| = 32 start points)."""
    s = W.large_exponent_system(61, 3, 5, 1, 22, 40, lift_hi=16)
    lift = np.random.default_rng(11).integers(1, 17, size=s.M).astype(np.int64)
    for k in range(3):
        lift[5 * k] = lift[5 * k + 1] = 0
    return W.LaurentSystem(3, s.m, s.exponents, s.coeffs, lift), [[0, 1]] * 3


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_track_large_exponents(hpt, oracle_mod, prec):
    """Monomials with sum |a_j| above 64, whose phase the mixed form
    accumulates in 32-bit fixed point (exactly modulo one revolution) instead
    of by the FP32 exponent GEMM: every start point of the planted cell is
    tracked to t = 1 and polished, every path converges, and the solutions
    match the oracle's one to one within relative 1e-9."""
    s, pairs = _large_exponent_case()
    assert (np.abs(s.exponents).sum(1) > 64).sum() == 3
    cell = {"kind": "pairs", "pairs": pairs}
    te = cells.t_exponents(s, cell)
    osys = oracle_mod.System(s, te["e"], te["D"])
    y0 = cells.start_points(s, pairs)
    assert len(y0) == 32
    x_o, st_o, _, _ = osys.track(oracle_mod.Params(), y0, cells.tau0(te["e"], te["D"]))
    assert (st_o == oracle_mod.CONVERGED).all()
    h = hpt.System.from_laurent(s, cell, prec)
    x, st, _ = h.track(torch.from_numpy(y0).cuda(), hpt.Params(tol_accept=1e-3 if prec == 0 else 3e-3))
    assert h.device_error() == 0
    st = st.cpu().numpy()
    assert (st == hpt.CONVERGED).all(), np.bincount(st)
    assert _util.match_solutions(x.cpu().numpy(), x_o) < 1e-9
    h.close()

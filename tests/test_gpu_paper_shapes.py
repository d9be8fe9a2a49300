"""The stand-ins of the paper's test-system shapes on the GPU (GPU).

n = 14 with 184 monomials and n = 24 with 324 (Section 8, Tables 1-2, the
shapes of cyclic-14 and chandra-24; synthetic systems, planted cells):
evaluation within 1e-11 (FP64) / 2e-4 (mixed) of the oracle, and polished
end points of tracked paths within 1e-9 of the oracle's tracker.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cells

import _util

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(14, 184), (24, 324)], ids=["n14_m184", "n24_m324"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_paper_shape_eval_and_tracks(hpt, oracle_mod, shape, prec):
    n, M = shape
    s, pairs = W.paper_shape(n, M)
    assert s.M == M
    cell = {"kind": "pairs", "pairs": pairs}
    te = cells.t_exponents(s, cell)
    osys = oracle_mod.System(s, te["e"], te["D"])
    h = hpt.System.from_laurent(s, cell, prec)
    y, t = W.random_points(3, 200, n)
    H, Hy, Ht = (a.cpu().numpy() for a in h.eval(torch.from_numpy(y).to("cuda", h.cdtype), torch.from_numpy(t).cuda()))
    Ho, Hyo, Hto = osys.eval(y, np.log(t))
    SH, SHy, SHt = osys.scale(y, np.log(t))
    tol, floor = (1e-11, 0.0) if prec == 0 else (2e-4, 1e-30)
    assert _util.scaled_err(H, Ho, np.maximum(SH, floor)) <= tol
    assert _util.scaled_err(Hy, Hyo, np.maximum(SHy, floor)) <= tol
    ks = np.zeros((24, n), np.int64)
    ks[:, 0] = np.arange(24)
    x0 = cells.start_points_at(s, pairs, ks)
    prm = hpt.Params(tol_accept=3e-3 if prec == 1 else 1e-3)
    x, st, _ = (a.cpu().numpy() for a in h.track(torch.from_numpy(x0).cuda(), prm))
    xo, sto, _, _ = osys.track(oracle_mod.Params(), x0, cells.tau0(te["e"], te["D"]))
    both = (st == hpt.CONVERGED) & (sto == oracle_mod.CONVERGED)
    assert both.mean() > 0.9, (np.bincount(st), np.bincount(sto))
    rel = np.abs(x[both] - xo[both]).max(1) / np.maximum(1, np.abs(xo[both]).max(1))
    assert (rel < 1e-9).mean() > 0.95, np.sort(rel)[-3:]

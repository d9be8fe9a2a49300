"""Adjoint form (GPU): gradient of L = sum |x|^2 over 4,096 solutions of the
n=8, 12-monomial workload with respect to the complex coefficients, through
torch.autograd (HptSolve), against the oracle's adjoint gradient (relative
1e-9) and against central finite differences of re-polished solutions."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cells

import _util

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case(oracle_mod):
    s, pairs, te, d = _util.planted_case(W.config5, 4096)
    y0 = cells.start_points(s, pairs, limit=4096)
    osys = oracle_mod.System(s, te["e"], te["D"])
    x_o, st_o, _, _ = osys.track(oracle_mod.Params(), y0, cells.tau0(te["e"], te["D"]))
    return s, pairs, te, y0, osys, x_o, st_o


def test_adjoint_matches_oracle(hpt, oracle_mod, case):
    from paper_2111_14317_gb300.autograd import solve
    s, pairs, te, y0, osys, x_o, st_o = case
    spec = dict(n=s.n, m=s.m, exponents=s.exponents, lifting=s.lifting,
                cell={"kind": "pairs", "pairs": pairs})
    c = torch.tensor(s.coeffs, dtype=torch.complex128, requires_grad=True)
    x, status = solve(c, spec, torch.from_numpy(y0).cuda())
    conv = (status == hpt.CONVERGED)
    assert conv.float().mean().item() > 0.99
    L = (x[conv].abs() ** 2).sum()
    L.backward()
    g = c.grad.numpy()
    st = status.cpu().numpy()
    both = (st == hpt.CONVERGED) & (st_o == oracle_mod.CONVERGED)
    xg = x.detach().cpu().numpy()
    assert _util.match_solutions(xg[both], x_o[both]) < 1e-9
    keep = st == hpt.CONVERGED
    g_o = osys.adjoint(xg[keep], 2 * xg[keep])
    assert np.max(np.abs(g - g_o)) <= 1e-9 * np.abs(g_o).max()


def test_adjoint_finite_differences(hpt, oracle_mod, case):
    s, pairs, te, y0, osys, x_o, st_o = case
    cell = {"kind": "pairs", "pairs": pairs}
    keep = st_o == oracle_mod.CONVERGED
    x = torch.from_numpy(x_o[keep][:512]).cuda()
    h0 = hpt.System.from_laurent(s, cell, hpt.HPT_FP64)
    g = h0.adjoint(x, 2 * x).cpu().numpy()

    def loss(coeffs):
        h = hpt.System.from_laurent(s.with_coeffs(coeffs), cell, hpt.HPT_FP64)
        xp = h.polish(x.clone())
        torch.cuda.synchronize()
        v = float((xp.abs() ** 2).sum())
        h.close()
        return v

    eps = 1e-6
    for i in (0, 5, 17, 40, 95):
        fd = 0j
        for unit in (1.0, 1j):
            cp, cm = s.coeffs.copy(), s.coeffs.copy()
            cp[i] += eps * unit
            cm[i] -= eps * unit
            d = (loss(cp) - loss(cm)) / (2 * eps)
            fd += d if unit == 1.0 else 1j * d
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, np.abs(g).max()), (i, fd, g[i])

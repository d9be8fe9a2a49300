"""Pins of the oracle's tracker (CPU only).

* BKK: for generic coefficients the number of distinct solutions reached
  from all mixed cells equals the brute-force mixed volume (configs 1, 2).
* Every endpoint solves F(x) = H(x, t=1) = 0 to rounding level (scaled
  residual), and no two paths end at the same solution (no path jumping).
* A closed-form path: h = c1 y - c0 - c2 t is tracked to (c0 + c2)/c1.
* Stepping k then k more steps equals stepping 2k at once (the state is
  the whole checkpoint).
"""
import numpy as np
import pytest

import workloads as W
from oracle import cells


def _first_generic(cfg):
    for att in range(40):
        s = cfg(att)
        try:
            cl, mv = cells.mixed_cells(s)
        except cells.NonGeneric:
            continue
        if mv >= 2:
            return s, cl, mv
    raise RuntimeError("no generic sample")


def _track_all(oracle_mod, s, cl, params):
    xs, sts = [], []
    for c in cl:
        te = cells.t_exponents(s, {"kind": "pairs", "pairs": c["pairs"]})
        osys = oracle_mod.System(s, te["e"], te["D"])
        y0 = cells.start_points(s, c["pairs"])
        x, st, _, _ = osys.track(params, y0, cells.tau0(te["e"], te["D"]))
        xs.append(x)
        sts.append(st)
    return np.concatenate(xs), np.concatenate(sts), osys


@pytest.mark.parametrize("cfg", [W.config1, W.config2])
def test_bkk_root_count(oracle_mod, cfg):
    s, cl, mv = _first_generic(cfg)
    x, st, osys = _track_all(oracle_mod, s, cl, oracle_mod.Params())
    assert len(x) == mv
    assert (st == oracle_mod.CONVERGED).all()
    H, _, _ = osys.eval(x, np.zeros(len(x)))
    SH, _, _ = osys.scale(x, np.zeros(len(x)))
    assert np.max(np.abs(H) / SH) < 1e-12
    d = np.abs(x[:, None, :] - x[None, :, :]).max(-1)
    np.fill_diagonal(d, np.inf)
    assert d.min() > 1e-6


def test_closed_form_path(oracle_mod):
    c1, c0, c2 = 2 - 1j, 0.5 + 0.25j, -1.5 + 2j
    s = W.LaurentSystem(1, [3], np.array([[1], [0], [0]]), np.array([c1, -c0, -c2]),
                        np.zeros(3, np.int64))
    osys = oracle_mod.System(s, np.array([0, 0, 1]), 1)
    tau0 = -20.0
    y0 = np.array([[(c0 + c2 * np.exp(tau0)) / c1 + 1e-3]])
    x, st, steps, _ = osys.track(oracle_mod.Params(), y0, tau0)
    assert st[0] == oracle_mod.CONVERGED
    assert abs(x[0, 0] - (c0 + c2) / c1) < 1e-14


def test_step_resume(oracle_mod):
    s, cl, _ = _first_generic(W.config1)
    c = cl[0]
    te = cells.t_exponents(s, {"kind": "pairs", "pairs": c["pairs"]})
    osys = oracle_mod.System(s, te["e"], te["D"])
    y0 = cells.start_points(s, c["pairs"])
    P = oracle_mod.Params()
    a = oracle_mod.PathState.start(y0, cells.tau0(te["e"], te["D"]), P.dtau_init)
    b = a.copy()
    osys.step(P, a, 14)
    osys.step(P, b, 7)
    b = b.copy()
    osys.step(P, b, 7)
    for f in ("y", "tau", "dtau", "yacc", "tauacc", "dEacc", "status", "steps", "accepts"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f

"""Pins of the oracle's predictors (CPU only).

* Order of accuracy on a closed-form path (h = c1 y - c0 - c2 t, so
  y(tau) = (c0 + c2 e^tau) / c1): from two exact accepted points tau1 - h
  and tau1 the prediction at tau1 + h errs by O(h^2) with the Euler
  predictor and by O(h^4) with the cubic Hermite predictor, so halving h
  divides the error by about 4 and 16.  The predictors' formulas are not
  restated here; only the convergence order of what the tracker predicts.
* Tracks with the Hermite predictor reach the Euler tracker's end points
  (BKK configs 1 and 2, affine and projective) in fewer steps.
"""
import numpy as np

import workloads as W
from oracle import cells
from oracle import projective as PJ

C1, C0, C2 = 2 - 1j, 0.5 + 0.25j, -1.5 + 2j


def _closed_form(oracle_mod):
    s = W.LaurentSystem(1, [3], np.array([[1], [0], [0]]), np.array([C1, -C0, -C2]), np.zeros(3, np.int64))
    return oracle_mod.System(s, np.array([0, 0, 1]), 1)


def _path(tau):
    return (C0 + C2 * np.exp(tau)) / C1


def _dpath(tau):
    return C2 * np.exp(tau) / C1


def _prediction_error(oracle_mod, osys, predictor, h, tau1=-1.0):
    """One step from accepted point tau1 - h with the current point exactly
    on the path at tau1: the step accepts it and predicts at tau1 + h."""
    P = oracle_mod.Params(predictor=predictor, dtau_init=h)
    t0 = tau1 - h
    st = oracle_mod.PathState.start(np.array([[_path(t0)]]), t0, h)
    st.dEacc[:] = _dpath(t0)
    st.accepts[:] = 1
    st.y[:] = _path(tau1)
    st.tau[:] = tau1
    osys.step(P, st, 1)
    assert st.accepts[0] == 2 and abs(st.tau[0] - (tau1 + h)) < 1e-15
    return abs(st.y[0, 0] - _path(tau1 + h))


def test_predictor_order_of_accuracy(oracle_mod):
    osys = _closed_form(oracle_mod)
    for predictor, order in ((0, 2), (1, 4)):
        e = [_prediction_error(oracle_mod, osys, predictor, h) for h in (0.2, 0.1, 0.05)]
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert abs(np.log2(r1) - order) < 0.35 and abs(np.log2(r2) - order) < 0.25, (predictor, e)
    # the cubic is far closer at the same step
    assert _prediction_error(oracle_mod, osys, 1, 0.1) < 0.05 * _prediction_error(oracle_mod, osys, 0, 0.1)


def _generic(cfg):
    for att in range(40):
        s = cfg(att)
        try:
            cl, mv = cells.mixed_cells(s)
        except cells.NonGeneric:
            continue
        if mv >= 2:
            return s, cl, mv
    raise RuntimeError("no generic sample")


def test_hermite_tracks_reach_the_same_solutions_in_fewer_steps(oracle_mod):
    for cfg in (W.config1, W.config2):
        s, cl, mv = _generic(cfg)
        res = {}
        for pred in (0, 1):
            P = oracle_mod.Params(predictor=pred)
            xs, steps, xsp, stepsp = [], 0, [], 0
            for c in cl:
                te = cells.t_exponents(s, {"kind": "pairs", "pairs": c["pairs"]})
                osys = oracle_mod.System(s, te["e"], te["D"])
                x0 = cells.start_points(s, c["pairs"])
                t0 = cells.tau0(te["e"], te["D"])
                x, st, sp, _ = osys.track(P, x0, t0)
                assert (st == oracle_mod.CONVERGED).all()
                xs.append(x)
                steps += int(sp.sum())
                ps = PJ.ProjectiveSystem(s, te["e"], te["D"])
                x, st, sp, _, _ = ps.track(P, x0, t0)
                assert (st == oracle_mod.CONVERGED).all()
                xsp.append(x)
                stepsp += int(sp.sum())
            res[pred] = (np.concatenate(xs), steps, np.concatenate(xsp), stepsp)
        (xe, se, xpe, spe), (xh, sh, xph, sph) = res[0], res[1]
        for a, b in ((xh, xe), (xph, xe), (xpe, xe)):
            assert np.max(np.abs(a - b).max(1) / np.maximum(1, np.abs(b).max(1))) < 1e-9
        assert sh < se and sph < spe, (sh, se, sph, spe)

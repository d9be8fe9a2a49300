"""The cubic Hermite predictor on the GPU (GPU).

* One FP64 step from a mid-track oracle state (affine and projective, with
  the previous accepted point in the state) gives the oracle's accept
  decisions and new state within 1e-10 / 1e-9.
* Whole tracks with the Hermite predictor (FP64 and mixed, affine and
  projective, one system and the many-systems batch) reach the Euler
  tracker's polished solutions (1e-9) in fewer steps.
* Stepping is resumable from the state arrays (prev arrays included), and
  predictor = 1 without them is refused.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cells
from oracle import projective as PJ

import _util

pytestmark = pytest.mark.gpu
OF = [("y", "y"), ("tau", "tau"), ("dtau", "dtau"), ("yacc", "y_acc"), ("tauacc", "tau_acc"),
      ("dEacc", "dE_acc"), ("status", "status"), ("steps", "steps"), ("accepts", "accepts"),
      ("rejects", "rejects"), ("streak", "streak"), ("yprev", "y_prev"), ("tauprev", "tau_prev"),
      ("dEprev", "dE_prev"), ("hflag", "hermite")]


def _to_gpu(ost, g):
    for a, b in OF:
        getattr(g, b).copy_(torch.from_numpy(np.ascontiguousarray(getattr(ost, a))).to(getattr(g, b).dtype))
    return g


def _compare(g, ost, tol):
    gh = g.to_host()
    same = gh["accepts"].numpy() == ost.accepts
    assert same.mean() >= 0.98
    assert np.array_equal(gh["status"].numpy()[same], ost.status[same])
    assert np.array_equal(gh["hermite"].numpy()[same], ost.hflag[same])
    for a, b in (("y", "y"), ("yacc", "y_acc"), ("dEacc", "dE_acc"), ("yprev", "y_prev")):
        ref = getattr(ost, a)[same]
        got = gh[b].numpy()[same]
        assert np.max(np.abs(got - ref) / (1 + np.abs(ref))) < tol, a
    assert np.allclose(gh["tau"].numpy()[same], ost.tau[same], rtol=0, atol=1e-12)


@pytest.mark.parametrize("nsteps", [3, 12, 30])
def test_hermite_step_matches_oracle(hpt, oracle_mod, nsteps):
    s, cl, _ = _util.first_generic(W.config2)
    P = oracle_mod.Params(predictor=1)
    prm = hpt.Params(predictor=1)
    for c in cl[:5]:
        cell = {"kind": "pairs", "pairs": c["pairs"]}
        te = cells.t_exponents(s, cell)
        x0 = cells.start_points(s, c["pairs"])
        t0 = cells.tau0(te["e"], te["D"])
        # affine
        osys = oracle_mod.System(s, te["e"], te["D"])
        ost = oracle_mod.PathState.start(x0, t0, P.dtau_init)
        osys.step(P, ost, nsteps)
        h = hpt.System.from_laurent(s, cell, 0)
        g = _to_gpu(ost, hpt.PathState(ost.p, s.n, 0, hermite=True))
        h.step(g, 1, prm)
        osys.step(P, ost, 1)
        _compare(g, ost, 1e-10)
        # projective
        ps = PJ.ProjectiveSystem(s, te["e"], te["D"])
        ost = ps.start(P, x0, t0)
        ps.step(P, ost, nsteps)
        hp = h.homogenize()
        g = _to_gpu(ost, hp.new_state(ost.p, hermite=True))
        hp.step(g, 1, prm)
        ps.step(P, ost, 1)
        _compare(g, ost, 1e-9)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_hermite_tracks_fewer_steps_same_solutions(hpt, prec):
    """Tolerance 1e-3 for both forms: at the mixed form's default 3e-3 the
    oracle itself sees one of the 878 projective Hermite paths jump to a
    neighbour (the cubic allows longer steps; the accept test is the same)."""
    s, cl, mv = _util.first_generic(W.config2)
    tol = 1e-3
    out = {}
    for pred in (0, 1):
        prm = hpt.Params(tol_accept=tol, predictor=pred)
        xs, steps, xps, stepsp = [], 0, [], 0
        for c in cl:
            cell = {"kind": "pairs", "pairs": c["pairs"]}
            h = hpt.System.from_laurent(s, cell, prec)
            x0 = torch.from_numpy(cells.start_points(s, c["pairs"])).cuda()
            x, st, sp = h.track(x0, prm)
            assert (st.cpu().numpy() == hpt.CONVERGED).all()
            xs.append(x.cpu().numpy())
            steps += int(sp.sum())
            x, st, sp = h.homogenize().track(x0, prm)
            assert (st.cpu().numpy() == hpt.CONVERGED).all()
            xps.append(x.cpu().numpy())
            stepsp += int(sp.sum())
        out[pred] = (np.concatenate(xs), steps, np.concatenate(xps), stepsp)
    (xe, se, xpe, spe), (xh, sh, xph, sph) = out[0], out[1]
    for a in (xh, xph, xpe):
        assert np.max(np.abs(a - xe).max(1) / np.maximum(1, np.abs(xe).max(1))) < 1e-9
    # (the oracle: config 2 at tol 1e-3 takes 0.59x / 0.75x the Euler steps)
    fa, fp = 0.75, 0.85
    assert sh < fa * se and sph < fp * spe, (sh, se, sph, spe)


def test_hermite_batch_equals_per_system_track(hpt):
    """The batch with the Hermite predictor: the same statuses and polished
    solutions as hpt_track per system (n from 4 to 16), and fewer steps
    than with the Euler predictor."""
    idx = []
    for i in range(400):
        s, _ = W.config4_system(i)
        if 4 <= s.n <= 16:
            idx.append(i)
        if len(idx) == 4:
            break
    systems = []
    for i in idx:
        s, pairs = W.config4_system(i)
        systems.append((s, pairs, hpt.System.from_laurent(s, {"kind": "pairs", "pairs": pairs}, hpt.HPT_MIXED)))
    paths = [100, 64, 129, 40]
    y0 = []
    for (s, pairs, _), p in zip(systems, paths):
        ks = np.zeros((p, s.n), np.int64)
        ks[:, 0] = np.arange(p)
        y0.append(cells.start_points_at(s, pairs, ks))
    flat = torch.from_numpy(np.concatenate([y.reshape(-1) for y in y0])).cuda()
    b = hpt.Batch([h for _, _, h in systems])
    res = {}
    for pred in (0, 1):
        prm = hpt.Params(tol_accept=1e-3, predictor=pred)
        x, st, sp = b.track(flat, paths, prm)
        res[pred] = (x.cpu().numpy(), st.cpu().numpy(), sp.cpu().numpy())
    xb, stb, spb = res[1]
    vo = po = 0
    for (s, pairs, h), p, y in zip(systems, paths, y0):
        xt, stt, spt = (a.cpu().numpy() for a in h.track(torch.from_numpy(y).cuda(),
                                                         hpt.Params(tol_accept=1e-3, predictor=1)))
        assert np.array_equal(stb[po:po + p], stt) and np.array_equal(spb[po:po + p], spt)
        assert np.array_equal(xb[vo:vo + p * s.n].reshape(p, s.n), xt)
        vo += p * s.n
        po += p
    conv = (res[0][1] == hpt.CONVERGED) & (stb == hpt.CONVERGED)
    assert conv.mean() > 0.9
    assert spb[conv].sum() < res[0][2][conv].sum()


def test_hermite_resume_and_refusal(hpt, oracle_mod):
    s, cl, _ = _util.first_generic(W.config2)
    c = max(cl, key=lambda c: c["det"])
    cell = {"kind": "pairs", "pairs": c["pairs"]}
    x0 = torch.from_numpy(cells.start_points(s, c["pairs"])).cuda()
    prm = hpt.Params(predictor=1)
    for prec in (0, 1):
        for h in (hpt.System.from_laurent(s, cell, prec), hpt.System.from_laurent(s, cell, prec).homogenize()):
            a = h.new_state(x0.shape[0], hermite=True)
            b = h.new_state(x0.shape[0], hermite=True)
            h.paths_init(a, x0, prm)
            h.paths_init(b, x0, prm)
            h.step(a, 24, prm)
            h.step(b, 12, prm)
            saved = b.to_host()
            b2 = h.new_state(x0.shape[0], hermite=True)
            b2.load(saved)
            h.step(b2, 12, prm)
            ha, hb = a.to_host(), b2.to_host()
            for k in ha:
                assert torch.equal(ha[k], hb[k]), k
            plain = h.new_state(x0.shape[0])
            with pytest.raises(hpt.HptError) as ei:
                h.paths_init(plain, x0, prm)
            assert ei.value.code == 1

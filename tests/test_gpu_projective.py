"""Projective formulation and Algorithm 3 by QR on the GPU (GPU).

* Evaluation of the homogenized homotopy (n equations in n + 1 coordinates):
  FP64 form within 1e-11 and mixed form within 2e-4 of the oracle, scaled by
  the sum of term magnitudes (the tolerances of the affine evaluation).
* hpt_euler_newton: the FP64 QR null-space directions equal the oracle's
  Algorithm 3 (relative 1e-10 per point), for every lane-group shape
  (N = nv rows: <= 8, <= 16, <= 32), on projective and on affine handles
  (where they equal the LU directions).  The FP32 factorisation of the mixed
  form: relative error within 5e-4 times the condition number of J (the
  stated evaluation error amplified by the conditioning of the null-space
  problem), checked per point, on sampled points of the 65,536-point n = 16
  workload as well.
* The projective step: one FP64 step from a mid-track oracle state gives the
  oracle's accept decisions and new state within 1e-9.
* Tracks: the projective tracker's polished end points equal the oracle's
  projective tracker and the affine GPU tracker (1e-9), FP64 and mixed; two
  parallel lines end DIVERGED at the point at infinity [1 : -1 : 0].
* Edge cases: p = 0, ragged p, refusals (twice homogenized, batch, static
  step).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cells
from oracle import projective as PJ

import _util

pytestmark = pytest.mark.gpu
TOL = {0: 1e-11, 1: 2e-4}
FLOOR = {0: 0.0, 1: 1e-30}


def _proj_case(name):
    s, cell = _util.eval_case(name)
    te = cells.t_exponents(s, cell)
    return s, cell, PJ.ProjectiveSystem(s, te["e"], te["D"])


def _hom_points(seed, p, nv):
    rng = np.random.default_rng(seed)
    y = np.exp(rng.normal(0, 0.5, (p, nv))) * np.exp(2j * np.pi * rng.random((p, nv)))
    return y / np.linalg.norm(y, axis=1, keepdims=True)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", ["n4", "n7_ragged", "n16"])
def test_projective_eval_parity(hpt, oracle_mod, name, prec):
    s, cell, ps = _proj_case(name)
    h = hpt.System.from_laurent(s, cell, prec).homogenize()
    assert h.projective and h.nv == s.n + 1 and np.array_equal(h.degrees, ps.deg)
    p = 333
    y = _hom_points(5, p, h.nv)
    t = np.random.default_rng(6).uniform(0.05, 1.0, p)
    H, Hy, Ht = (a.cpu().numpy() for a in h.eval(torch.from_numpy(y).to("cuda", h.cdtype),
                                                 torch.from_numpy(t).cuda()))
    assert h.device_error() == 0
    Ho, Hyo, Hto = ps.eval(y, np.log(t))
    SH, SHy, SHt = ps.scale(y, np.log(t))
    f = FLOOR[prec]
    errs = (_util.scaled_err(H, Ho, np.maximum(SH, f)), _util.scaled_err(Hy, Hyo, np.maximum(SHy, f)),
            _util.scaled_err(Ht, Hto / t[:, None], np.maximum(SHt, f) / t[:, None]))
    assert max(errs) <= TOL[prec], errs


def _rel(a, b):
    return np.abs(a - b).max(1) / np.abs(b).max(1)


def _cond(J):
    sv = np.linalg.svd(J, compute_uv=False)
    return sv[:, 0] / sv[:, J.shape[1] - 1]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", ["n4", "n7_ragged", "n16", "n24"])
def test_euler_newton_projective(hpt, oracle_mod, name, prec):
    """N = nv = 5, 8, 17, 25: the (8,1), (8,1), (8,3)/(32,1) and (32,1) shapes."""
    s, cell, ps = _proj_case(name)
    if name == "n24" and prec == 1:
        # homogenized exponent sums reach 79 > 64: refused for the mixed form
        with pytest.raises(hpt.HptError) as ei:
            hpt.System.from_laurent(s, cell, prec).homogenize()
        assert ei.value.code == 4
        return
    h = hpt.System.from_laurent(s, cell, prec).homogenize()
    p = 301
    y = _hom_points(7, p, h.nv)
    tau = -np.random.default_rng(8).uniform(0.0, 2.0, p)
    dE, dN, ok = (a.cpu().numpy() for a in h.euler_newton(torch.from_numpy(y).to("cuda", h.cdtype),
                                                          torch.from_numpy(tau).cuda()))
    dEo, dNo, oko = ps.directions(y, tau)
    assert oko.all() and (ok == 1).all()
    if prec == 0:
        assert _rel(dE, dEo).max() < 1e-10 and _rel(dN, dNo).max() < 1e-10
    else:
        kappa = _cond(ps.consolidated(y, tau))
        assert (_rel(dE, dEo) <= 5e-4 * kappa).all(), np.max(_rel(dE, dEo) / kappa)
        assert (_rel(dN, dNo) <= 5e-4 * kappa).all(), np.max(_rel(dN, dNo) / kappa)
        assert np.median(_rel(dE, dEo)) < 1e-4


@pytest.mark.parametrize("name", ["n4", "n16", "n24"])
def test_euler_newton_affine_equals_lu(hpt, oracle_mod, name):
    """Algorithm 3 on an affine handle (no y^* row): the affine directions."""
    s, cell = _util.eval_case(name)
    te = cells.t_exponents(s, cell)
    osys = oracle_mod.System(s, te["e"], te["D"])
    h = hpt.System.from_laurent(s, cell, 0)
    y, t = W.random_points(9, 200, s.n)
    tau = np.log(t)
    dE, dN, ok = (a.cpu().numpy() for a in h.euler_newton(torch.from_numpy(y).cuda(), torch.from_numpy(tau).cuda()))
    dEo, dNo, oko = osys.directions(y, tau)
    good = oko & (ok == 1)
    assert good.mean() > 0.99
    assert _rel(dE[good], dEo[good]).max() < 1e-9 and _rel(dN[good], dNo[good]).max() < 1e-9


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_euler_newton_full_size_sampled(hpt, oracle_mod, prec):
    """The 65,536-point n = 16 workload in projective form, sampled points."""
    s, cell, ps = _proj_case("n16")
    h = hpt.System.from_laurent(s, cell, prec).homogenize()
    p = 65536
    y = _hom_points(10, p, h.nv)
    tau = -np.random.default_rng(11).uniform(0.0, 2.0, p)
    dE, dN, ok = (a.cpu().numpy() for a in h.euler_newton(torch.from_numpy(y).to("cuda", h.cdtype),
                                                          torch.from_numpy(tau).cuda()))
    idx = np.concatenate([np.random.default_rng(12).choice(p, 250, replace=False), [0, 127, 128, p - 1]])
    dEo, dNo, oko = ps.directions(y[idx], tau[idx])
    assert oko.all() and (ok[idx] == 1).all()
    if prec == 0:
        assert _rel(dE[idx], dEo).max() < 1e-10 and _rel(dN[idx], dNo).max() < 1e-10
    else:
        kappa = _cond(ps.consolidated(y[idx], tau[idx]))
        assert (_rel(dE[idx], dEo) <= 5e-4 * kappa).all()
        assert (_rel(dN[idx], dNo) <= 5e-4 * kappa).all()


def test_euler_newton_edges(hpt):
    s, cell = _util.eval_case("n4")
    h = hpt.System.from_laurent(s, cell, 0).homogenize()
    z = torch.zeros(0, h.nv, dtype=torch.complex128, device="cuda")
    dE, dN, ok = h.euler_newton(z, torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert dE.shape == (0, h.nv)
    with pytest.raises(hpt.HptError):
        h.homogenize()
    hm = hpt.System.from_laurent(s, cell, 1).homogenize()
    with pytest.raises(hpt.HptError) as ei:
        hpt.Batch([hm])
    assert ei.value.code == 7
    st = hm.new_state(4)
    with pytest.raises(hpt.HptError) as ei:
        hm.step_static(st, 1)
    assert ei.value.code == 7


def _proj_state_to_gpu(hpt, ost, h):
    g = h.new_state(ost.p)
    for a, b in (("y", "y"), ("tau", "tau"), ("dtau", "dtau"), ("yacc", "y_acc"), ("tauacc", "tau_acc"),
                 ("dEacc", "dE_acc"), ("status", "status"), ("steps", "steps"), ("accepts", "accepts"),
                 ("rejects", "rejects"), ("streak", "streak")):
        getattr(g, b).copy_(torch.from_numpy(np.ascontiguousarray(getattr(ost, a))).to(getattr(g, b).dtype))
    return g


@pytest.mark.parametrize("nsteps", [0, 4, 20])
def test_projective_step_matches_oracle(hpt, oracle_mod, nsteps):
    s, cl, _ = _util.first_generic(W.config2)
    P = oracle_mod.Params()
    for c in cl[:5]:
        cell = {"kind": "pairs", "pairs": c["pairs"]}
        te = cells.t_exponents(s, cell)
        ps = PJ.ProjectiveSystem(s, te["e"], te["D"])
        ost = ps.start(P, cells.start_points(s, c["pairs"]), cells.tau0(te["e"], te["D"]))
        ps.step(P, ost, nsteps)
        h = hpt.System.from_laurent(s, cell, 0).homogenize()
        g = _proj_state_to_gpu(hpt, ost, h)
        h.step(g, 1)
        ps.step(P, ost, 1)
        gh = g.to_host()
        same = gh["accepts"].numpy() == ost.accepts
        assert same.mean() >= 0.98
        assert np.array_equal(gh["status"].numpy()[same], ost.status[same])
        for a, b in (("y", "y"), ("yacc", "y_acc"), ("dEacc", "dE_acc")):
            ref = getattr(ost, a)[same]
            got = gh[b].numpy()[same]
            assert np.max(np.abs(got - ref) / (1 + np.abs(ref))) < 1e-9, a
        assert np.allclose(gh["tau"].numpy()[same], ost.tau[same], rtol=0, atol=1e-12)


def test_projective_paths_init(hpt):
    s, cl, _ = _util.first_generic(W.config2)
    cell = {"kind": "pairs", "pairs": cl[0]["pairs"]}
    x0 = cells.start_points(s, cl[0]["pairs"])
    for prec in (0, 1):
        h = hpt.System.from_laurent(s, cell, prec).homogenize()
        g = h.new_state(len(x0))
        h.paths_init(g, torch.from_numpy(x0).cuda())
        y = g.y.cpu().numpy()
        ref = PJ.homogeneous_start(x0)
        assert np.abs(y - ref).max() < (1e-15 if prec == 0 else 1e-6)
        assert (g.status.cpu().numpy() == hpt.ACTIVE).all()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_projective_track_matches_oracle_and_affine(hpt, oracle_mod, prec):
    for cfg in (W.config1, W.config2):
        s, cl, mv = _util.first_generic(cfg)
        P = oracle_mod.Params()
        prm = hpt.Params(tol_accept=3e-3) if prec == 1 else hpt.Params()
        xs, xo, xa = [], [], []
        for c in cl:
            cell = {"kind": "pairs", "pairs": c["pairs"]}
            te = cells.t_exponents(s, cell)
            ps = PJ.ProjectiveSystem(s, te["e"], te["D"])
            x0 = cells.start_points(s, c["pairs"])
            ha = hpt.System.from_laurent(s, cell, prec)
            h = ha.homogenize()
            x, st, _ = h.track(torch.from_numpy(x0).cuda(), prm)
            assert (st.cpu().numpy() == hpt.CONVERGED).all()
            xs.append(x.cpu().numpy())
            xo.append(ps.track(P, x0, cells.tau0(te["e"], te["D"]))[0])
            xa.append(ha.track(torch.from_numpy(x0).cuda(), prm)[0].cpu().numpy())
        xs, xo, xa = np.concatenate(xs), np.concatenate(xo), np.concatenate(xa)
        assert len(xs) == mv
        assert _util.match_solutions(xs, xo) < 1e-9
        assert np.max(np.abs(xs - xa).max(1) / np.maximum(1, np.abs(xa).max(1))) < 1e-9


def test_projective_track_larger_systems(hpt, oracle_mod):
    """FP64 projective tracks of many-systems workload systems (n in [9, 16]
    and [17, 24]): the polished end points of the paths that converge in both
    equal the affine tracker's."""
    for lo, hi in ((9, 16), (17, 24)):
        for idx in range(400):
            s, pairs = W.config4_system(idx)
            if lo <= s.n <= hi:
                break
        cell = {"kind": "pairs", "pairs": pairs}
        ks = np.zeros((64, s.n), np.int64)
        ks[:, 0] = np.arange(64)
        x0 = cells.start_points_at(s, pairs, ks)
        ha = hpt.System.from_laurent(s, cell, 0)
        h = ha.homogenize()
        x, st, _ = (a.cpu().numpy() for a in h.track(torch.from_numpy(x0).cuda()))
        xa, sta, _ = (a.cpu().numpy() for a in ha.track(torch.from_numpy(x0).cuda()))
        both = (st == hpt.CONVERGED) & (sta == hpt.CONVERGED)
        assert both.mean() > 0.9, (np.bincount(st), np.bincount(sta))
        rel = np.abs(x[both] - xa[both]).max(1) / np.maximum(1, np.abs(xa[both]).max(1))
        assert (rel < 1e-9).mean() > 0.97, np.sort(rel)[-4:]


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_parallel_lines_diverge_to_infinity(hpt, prec):
    ex = np.array([[1, 0], [0, 1], [0, 0]] * 2)
    s = W.LaurentSystem(2, [3, 3], ex, np.array([1, 1, 1, 2, 2, 5], np.complex128),
                        np.array([0, 3, 7, 5, 1, 2]))
    cl, mv = cells.mixed_cells(s)
    assert mv == 1
    cell = {"kind": "pairs", "pairs": cl[0]["pairs"]}
    h = hpt.System.from_laurent(s, cell, prec).homogenize()
    x0 = cells.start_points(s, cl[0]["pairs"])
    prm = hpt.Params(tol_accept=3e-3) if prec == 1 else hpt.Params()
    g = h.new_state(1)
    h.paths_init(g, torch.from_numpy(x0).cuda(), prm)
    for _ in range(100):
        h.step(g, 32, prm)
        if int(g.status[0]) != hpt.ACTIVE:
            break
    assert int(g.status[0]) == hpt.DIVERGED
    y = g.y_acc[0].cpu().numpy().astype(np.complex128)
    y = y / np.linalg.norm(y)
    assert abs(y[2]) <= abs(y[0]) / prm.div_bound * 1.01
    assert abs(y[0] + y[1]) < (1e-6 if prec == 0 else 1e-4) * abs(y[0])


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("n,M", [(12, 150), (20, 260), (24, 300)], ids=["nv13", "nv21", "nv25"])
def test_euler_newton_every_qr_shape(hpt, oracle_mod, n, M, prec):
    """nv = 13, 21, 25: the (8,2,18), (8,3,26) / (32,1,26) and (32,1,34)
    lane shapes of the FP32 and FP64 factorisations, on projective handles of
    paper-shape systems, against the oracle's Algorithm 3."""
    s, pairs = W.paper_shape(n, M)
    cell = {"kind": "pairs", "pairs": pairs}
    te = cells.t_exponents(s, cell)
    ps = PJ.ProjectiveSystem(s, te["e"], te["D"])
    h = hpt.System.from_laurent(s, cell, prec).homogenize()
    assert h.nv == n + 1
    p = 200
    y = _hom_points(13, p, h.nv)
    tau = -np.random.default_rng(14).uniform(0.0, 2.0, p)
    dE, dN, ok = (a.cpu().numpy() for a in h.euler_newton(torch.from_numpy(y).to("cuda", h.cdtype),
                                                          torch.from_numpy(tau).cuda()))
    dEo, dNo, oko = ps.directions(y, tau)
    assert oko.all() and (ok == 1).all()
    if prec == 0:
        assert _rel(dE, dEo).max() < 1e-10 and _rel(dN, dNo).max() < 1e-10
    else:
        kappa = _cond(ps.consolidated(y, tau))
        assert (_rel(dE, dEo) <= 5e-4 * kappa).all(), np.max(_rel(dE, dEo) / kappa)
        assert (_rel(dN, dNo) <= 5e-4 * kappa).all(), np.max(_rel(dN, dNo) / kappa)

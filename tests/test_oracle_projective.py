"""Pins of the oracle's projective formulation and Algorithm 3 (CPU only).

* Homogenization (Section 2.2, eq. (3)): h_k(lambda y) = lambda^{d_k} h_k(y)
  for complex lambda, Euler's identity sum_j y_j dh_k/dy_j = d_k h_k, and on
  the chart y_n = 1 the homogenized homotopy, its y' derivatives and its
  tau derivative equal the affine oracle's.
* Algorithm 3: the Euler and Newton directions are orthogonal to y
  (Pythagoras for real and imaginary step lengths: |y + h d|^2 = |y|^2 +
  |h|^2 |d|^2 only when y^* d = 0) and equal an LU solve of the bordered
  square system [H_y; y^*] (the oracle's batched LU, a different routine);
  the dehomogenized Euler direction satisfies the chain-rule identity with
  the affine oracle's homotopy (and is the affine direction on the path);
  both directions scale with y; on the affine extended Jacobian (no y^*
  row) the algorithm gives the affine LU directions.
* Tracking: the projective tracker reaches the affine tracker's end points,
  as many as the mixed volume (BKK), and follows the one path of two
  parallel lines to their common point at infinity [1 : -1 : 0].
"""
import numpy as np

import workloads as W
from oracle import cells
from oracle import projective as PJ


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


def _psys(oracle_mod, s, pairs):
    te = cells.t_exponents(s, {"kind": "pairs", "pairs": pairs})
    return PJ.ProjectiveSystem(s, te["e"], te["D"]), te


def _points(rng, p, nv):
    r = np.exp(rng.normal(0, 0.5, (p, nv)))
    return r * np.exp(2j * np.pi * rng.random((p, nv)))


def test_homogeneous_of_degree_d_and_euler_identity(oracle_mod):
    s, cl, _ = _generic(W.config2)
    ps, _ = _psys(oracle_mod, s, cl[0]["pairs"])
    rng = np.random.default_rng(1)
    y = _points(rng, 12, ps.nv)
    tau = -rng.random(12) * 2
    lam = 0.7 * np.exp(1j * 1.1)
    H, Hy, Ht = ps.eval(y, tau)
    H2, _, _ = ps.eval(lam * y, tau)
    scale = np.abs(H).max() + 1e-300
    assert np.abs(H2 - lam ** ps.deg[None, :] * H).max() < 1e-12 * scale * max(1, abs(lam) ** ps.deg.max())
    euler = np.einsum("pkj,pj->pk", Hy, y)
    assert np.abs(euler - ps.deg[None, :] * H).max() < 1e-12 * np.abs(Hy).max() * np.abs(y).max() * ps.nv
    assert (ps.exps_hat[:, -1] >= 0).all() and (ps.exps_hat[:, -1] == 0).any()


def test_chart_is_the_affine_homotopy(oracle_mod):
    s, cl, _ = _generic(W.config2)
    ps, _ = _psys(oracle_mod, s, cl[0]["pairs"])
    rng = np.random.default_rng(2)
    x = _points(rng, 10, s.n)
    tau = -rng.random(10)
    y = np.concatenate([x, np.ones((10, 1))], axis=1)
    H, Hy, Ht = ps.eval(y, tau)
    Ha, Hya, Hta = ps.affine.eval(x, tau)
    tol = 1e-13 * max(1.0, np.abs(Hya).max())
    assert np.abs(H - Ha).max() < tol and np.abs(Ht - Hta).max() < tol
    assert np.abs(Hy[:, :, :s.n] - Hya).max() < tol


def test_directions_are_orthogonal_to_y(oracle_mod):
    s, cl, _ = _generic(W.config2)
    ps, _ = _psys(oracle_mod, s, cl[0]["pairs"])
    rng = np.random.default_rng(3)
    y = _points(rng, 16, ps.nv)
    tau = -rng.random(16)
    dE, dN, ok = ps.directions(y, tau)
    assert ok.all()
    ny2 = (np.abs(y) ** 2).sum(1)
    for d in (dE, dN):
        nd2 = (np.abs(d) ** 2).sum(1)
        for h in (0.3, 0.3j):
            lhs = (np.abs(y + h * d) ** 2).sum(1)
            assert np.abs(lhs - ny2 - abs(h) ** 2 * nd2).max() < 1e-12 * (ny2 + nd2).max()


def test_directions_equal_bordered_lu_solve(oracle_mod):
    s, cl, _ = _generic(W.config2)
    ps, _ = _psys(oracle_mod, s, cl[0]["pairs"])
    rng = np.random.default_rng(4)
    p = 20
    y = _points(rng, p, ps.nv)
    tau = -rng.random(p)
    dE, dN, ok = ps.directions(y, tau)
    H, Hy, Ht = ps.eval(y, tau)
    A = np.concatenate([Hy, np.conj(y)[:, None, :]], axis=1)
    B = np.zeros((p, ps.nv, 2), np.complex128)
    B[:, :s.n, 0] = -Ht
    B[:, :s.n, 1] = -H
    X, nsing = oracle_mod.solve(A, B)
    assert nsing == 0 and ok.all()
    rel = lambda a, b: np.abs(a - b).max(1) / np.abs(b).max(1)
    assert rel(dE, X[:, :, 0]).max() < 1e-10
    assert rel(dN, X[:, :, 1]).max() < 1e-10


def test_dehomogenized_euler_direction(oracle_mod):
    """With h_k(y) = y_n^{d_k} f_k(y'/y_n) (f = the affine homotopy) the chain
    rule along y + s dE, tau + s turns eq. (4) into
        f_x dx + f_tau = -d_k (dE_n / y_n) f_k,
    dx = (dE' y_n - y' dE_n) / y_n^2 the dehomogenized direction, at any point
    and for any representative lambda (x, 1); on the path (f = 0) dx is the
    affine Euler direction."""
    s, cl, _ = _generic(W.config2)
    ps, _ = _psys(oracle_mod, s, cl[0]["pairs"])
    rng = np.random.default_rng(5)
    x = _points(rng, 15, s.n)
    tau = -rng.random(15)
    lam = _points(rng, 15, 1)
    y = lam * np.concatenate([x, np.ones((15, 1))], axis=1)
    dE, _, ok = ps.directions(y, tau)
    assert ok.all()
    Ha, Hya, Hta = ps.affine.eval(x, tau)
    yn, En = y[:, -1:], dE[:, -1:]
    dx = (dE[:, :-1] * yn - y[:, :-1] * En) / yn ** 2
    lhs = np.einsum("pkj,pj->pk", Hya, dx) + Hta + ps.deg[None, :] * (En / yn) * Ha
    scale = np.abs(Hya).max((1, 2)) * np.abs(dx).max(1) + np.abs(Hta).max(1)
    assert (np.abs(lhs).max(1) / scale).max() < 1e-12
    # at the end points of the affine tracker f = 0 and the two directions agree
    x0 = cells.start_points(s, cl[0]["pairs"])
    te = cells.t_exponents(s, {"kind": "pairs", "pairs": cl[0]["pairs"]})
    xe, st, _, _ = ps.affine.track(oracle_mod.Params(), x0, cells.tau0(te["e"], te["D"]))
    z = np.zeros(len(xe))
    ye = np.concatenate([xe, np.ones((len(xe), 1))], axis=1) * 0.6j
    dE, _, _ = ps.directions(ye, z)
    dEa, _, _ = ps.affine.directions(xe, z)
    dx = (dE[:, :-1] * ye[:, -1:] - ye[:, :-1] * dE[:, -1:]) / ye[:, -1:] ** 2
    assert (np.abs(dx - dEa).max(1) / np.abs(dEa).max(1)).max() < 1e-9


def test_directions_scale_with_y(oracle_mod):
    s, cl, _ = _generic(W.config1)
    ps, _ = _psys(oracle_mod, s, cl[0]["pairs"])
    rng = np.random.default_rng(6)
    y = _points(rng, 10, ps.nv)
    tau = -rng.random(10)
    lam = 1.9 * np.exp(-0.4j)
    dE, dN, _ = ps.directions(y, tau)
    dE2, dN2, _ = ps.directions(lam * y, tau)
    assert np.abs(dE2 - lam * dE).max() < 1e-11 * np.abs(lam * dE).max()
    assert np.abs(dN2 - lam * dN).max() < 1e-11 * np.abs(lam * dN).max()


def test_affine_algorithm3_equals_lu(oracle_mod):
    s, cl, _ = _generic(W.config2)
    te = cells.t_exponents(s, {"kind": "pairs", "pairs": cl[0]["pairs"]})
    osys = oracle_mod.System(s, te["e"], te["D"])
    rng = np.random.default_rng(7)
    x = _points(rng, 20, s.n)
    tau = -rng.random(20)
    dE, dN, ok = PJ.affine_directions(osys, x, tau)
    dEa, dNa, oka = osys.directions(x, tau)
    assert ok.all() and oka.all()
    assert (np.abs(dE - dEa).max(1) / np.abs(dEa).max(1)).max() < 1e-10
    assert (np.abs(dN - dNa).max(1) / np.abs(dNa).max(1)).max() < 1e-10


def test_projective_track_matches_affine_and_bkk(oracle_mod):
    for cfg in (W.config1, W.config2):
        s, cl, mv = _generic(cfg)
        P = oracle_mod.Params()
        xs_p, xs_a = [], []
        for c in cl:
            ps, te = _psys(oracle_mod, s, c["pairs"])
            x0 = cells.start_points(s, c["pairs"])
            t0 = cells.tau0(te["e"], te["D"])
            x, st, _, perr, yend = ps.track(P, x0, t0)
            assert (st == oracle_mod.CONVERGED).all(), st
            assert np.allclose(np.linalg.norm(yend, axis=1), 1.0, atol=1e-14)
            xa, sta, _, _ = ps.affine.track(P, x0, t0)
            assert (sta == oracle_mod.CONVERGED).all()
            xs_p.append(x)
            xs_a.append(xa)
        xp, xa = np.concatenate(xs_p), np.concatenate(xs_a)
        assert len(xp) == mv
        rel = np.abs(xp - xa).max(1) / np.maximum(1.0, np.abs(xa).max(1))
        assert rel.max() < 1e-9
        d = np.abs(xp[:, None, :] - xp[None, :, :]).max(-1)
        np.fill_diagonal(d, np.inf)
        assert d.min() > 1e-6


def test_parallel_lines_reach_the_point_at_infinity(oracle_mod):
    """x1 + x2 + 1 = 0 and 2 x1 + 2 x2 + 5 = 0 have no finite solution; the
    mixed volume of the two standard triangles is 1, and the one path goes to
    [1 : -1 : 0]."""
    ex = np.array([[1, 0], [0, 1], [0, 0]] * 2)
    coef = np.array([1, 1, 1, 2, 2, 5], np.complex128)
    s = W.LaurentSystem(2, [3, 3], ex, coef, np.array([0, 3, 7, 5, 1, 2]))
    cl, mv = cells.mixed_cells(s)
    assert mv == 1
    ps, te = _psys(oracle_mod, s, cl[0]["pairs"])
    x0 = cells.start_points(s, cl[0]["pairs"])
    P = oracle_mod.Params()
    x, st, _, _, y = ps.track(P, x0, cells.tau0(te["e"], te["D"]))
    assert st[0] == oracle_mod.DIVERGED
    y = y[0] / np.linalg.norm(y[0])
    assert abs(y[2]) <= abs(y[0]) / P.div_bound * 1.0001
    assert abs(y[0] + y[1]) < 1e-6 * abs(y[0])

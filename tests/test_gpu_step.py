"""Euler-Newton step parity and checkpoint/resume (GPU).

FP64 form: one step from a mid-track state gives the oracle's accept
decisions and the same new state (relative 1e-10).  The state arrays are the
whole checkpoint: 2k steps equal k steps, a host round trip and k more."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cells

import _util

pytestmark = pytest.mark.gpu
FIELDS = [("y", "y"), ("tau", "tau"), ("dtau", "dtau"), ("yacc", "y_acc"), ("tauacc", "tau_acc"),
          ("dEacc", "dE_acc"), ("status", "status"), ("steps", "steps"), ("accepts", "accepts"),
          ("rejects", "rejects"), ("streak", "streak")]


def _cell_state(oracle_mod, s, c, nsteps):
    te = cells.t_exponents(s, {"kind": "pairs", "pairs": c["pairs"]})
    osys = oracle_mod.System(s, te["e"], te["D"])
    P = oracle_mod.Params()
    st = oracle_mod.PathState.start(cells.start_points(s, c["pairs"]), cells.tau0(te["e"], te["D"]),
                                    P.dtau_init)
    osys.step(P, st, nsteps)
    return osys, st, P


def _to_gpu(hpt, ost, prec):
    g = hpt.PathState(ost.p, ost.y.shape[1], prec)
    for a, b in FIELDS:
        getattr(g, b).copy_(torch.from_numpy(np.ascontiguousarray(getattr(ost, a))).to(getattr(g, b).dtype))
    return g


@pytest.mark.parametrize("nsteps", [0, 3, 25])
def test_fp64_step_matches_oracle(hpt, oracle_mod, nsteps):
    s, cl, _ = _util.first_generic(W.config2)
    for c in cl[:6]:
        osys, ost, P = _cell_state(oracle_mod, s, c, nsteps)
        h = hpt.System.from_laurent(s, {"kind": "pairs", "pairs": c["pairs"]}, 0)
        g = _to_gpu(hpt, ost, 0)
        h.step(g, 1)
        osys.step(P, ost, 1)
        torch.cuda.synchronize()
        gh = g.to_host()
        same = gh["accepts"].numpy() == ost.accepts
        assert same.mean() >= 0.98
        assert np.array_equal(gh["status"].numpy()[same], ost.status[same])
        for a, b in (("y", "y"), ("yacc", "y_acc"), ("dEacc", "dE_acc")):
            ref = getattr(ost, a)[same]
            got = gh[b].numpy()[same]
            assert np.max(np.abs(got - ref) / (1 + np.abs(ref))) < 1e-10, a
        assert np.allclose(gh["tau"].numpy()[same], ost.tau[same], rtol=0, atol=1e-12)
        h.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_step_resume_is_exact(hpt, oracle_mod, prec):
    s, cl, _ = _util.first_generic(W.config2)
    c = max(cl, key=lambda c: c["det"])
    _, ost, _ = _cell_state(oracle_mod, s, c, 0)
    h = hpt.System.from_laurent(s, {"kind": "pairs", "pairs": c["pairs"]}, prec)
    a = _to_gpu(hpt, ost, prec)
    b = _to_gpu(hpt, ost, prec)
    h.step(a, 20)
    h.step(b, 10)
    saved = b.to_host()
    b2 = hpt.PathState(b.p, b.n, prec)
    b2.load(saved)
    h.step(b2, 10)
    torch.cuda.synchronize()
    ha, hb = a.to_host(), b2.to_host()
    for k in ha:
        assert torch.equal(ha[k], hb[k]), k
    h.close()


@pytest.mark.parametrize("n,m", [(6, 10), (16, 32), (24, 40)])
def test_fp64_resolve_path(hpt, n, m):
    """The mixed form's FP64 re-solve (redo_fp64_kernel): with cond_max = 1
    every FP32 solve is redone in FP64 from the same FP32 Jacobian; the step
    agrees with the all-FP32 step (cond_max = 1e30) to FP32 solve accuracy."""
    sysm = W.laurent_system(40 + n, n, m, -3, 3, 64, nnz=min(4, n))
    alpha = W.random_alpha(40 + n, n)
    cell = {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 1}
    h = hpt.System.from_laurent(sysm, cell, hpt.HPT_MIXED)
    y, t = W.random_points(9, 2000, n)
    out = []
    for cmax in (1.0, 1e30):
        st = hpt.PathState(2000, n, hpt.HPT_MIXED)
        yd = torch.from_numpy(y).cuda().to(torch.complex64)
        st.y.copy_(yd)
        st.y_acc.copy_(yd)
        st.tau.copy_(torch.from_numpy(np.log(t)))
        st.tau_acc.copy_(st.tau)
        st.dtau.fill_(1e-3)
        st.accepts.fill_(1)
        h.step(st, 1, hpt.Params(tol_accept=3e-3, cond_max=cmax))
        torch.cuda.synchronize()
        out.append(st.to_host())
    a, b = out
    same = (a["accepts"] == b["accepts"]) & (a["status"] == b["status"])
    assert same.float().mean() > 0.97
    ya, yb = a["y_acc"].numpy()[same.numpy()], b["y_acc"].numpy()[same.numpy()]
    rel = np.abs(ya - yb).max(-1) / np.maximum(1.0, np.abs(yb).max(-1))
    assert np.median(rel) < 1e-5 and (rel < 1e-3).mean() > 0.97
    h.close()


def _config4_in(lo, hi):
    for idx in range(400):
        s, pairs = W.config4_system(idx)
        if lo <= s.n <= hi:
            return s, pairs
    raise RuntimeError("no system")


@pytest.mark.parametrize("band", [(4, 8), (9, 16), (17, 24)], ids=["n<=8", "n<=16", "n<=24"])
def test_fp64_step_matches_oracle_larger_n(hpt, oracle_mod, band):
    """Every FP64 solve shape (8 lanes x 1 row, 8 x 2, 32 x 1) on real paths of
    many-systems workload systems: after 6 oracle steps from the start
    points, one more step on the GPU gives the oracle's accept decisions and
    new state (relative 1e-10) on the paths where the decisions agree."""
    s, pairs = _config4_in(*band)
    cell = {"kind": "pairs", "pairs": pairs}
    te = cells.t_exponents(s, cell)
    osys = oracle_mod.System(s, te["e"], te["D"])
    P = oracle_mod.Params()
    ks = np.zeros((96, s.n), np.int64)
    ks[:, 0] = np.arange(96)
    ost = oracle_mod.PathState.start(cells.start_points_at(s, pairs, ks), cells.tau0(te["e"], te["D"]),
                                     P.dtau_init)
    osys.step(P, ost, 6)
    h = hpt.System.from_laurent(s, cell, 0)
    g = _to_gpu(hpt, ost, 0)
    h.step(g, 1)
    osys.step(P, ost, 1)
    torch.cuda.synchronize()
    gh = g.to_host()
    same = (gh["accepts"].numpy() == ost.accepts) & (gh["status"].numpy() == ost.status)
    assert same.mean() >= 0.97
    assert (ost.accepts[same] > 1).mean() > 0.5      # real steps, not only rejections
    for a, b in (("y", "y"), ("yacc", "y_acc"), ("dEacc", "dE_acc")):
        ref = getattr(ost, a)[same]
        got = gh[b].numpy()[same]
        err = np.abs(got - ref).max(-1) / np.maximum(1.0, np.abs(ref).max(-1))
        assert err.max() < 1e-10, (a, np.sort(err)[-3:])
    h.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_step_over_several_chunks(hpt, prec):
    """More paths than one evaluate/solve round takes (65,536): the step over
    66,000 paths equals the steps of its first 65,536 and last 464 paths
    taken separately, bit for bit."""
    sysm, alpha = W.config3(6, 8)
    cell = {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 1}
    h = hpt.System.from_laurent(sysm, cell, prec)
    y, t = W.random_points(13, 66000, 6)

    def state(lo, hi):
        st = hpt.PathState(hi - lo, 6, prec)
        yd = torch.from_numpy(y[lo:hi]).cuda().to(st.y.dtype)
        st.y.copy_(yd)
        st.y_acc.copy_(yd)
        st.tau.copy_(torch.from_numpy(np.log(t[lo:hi])))
        st.tau_acc.copy_(st.tau)
        st.dtau.fill_(1e-3)
        st.accepts.fill_(1)
        return st

    whole, a, b = state(0, 66000), state(0, 65536), state(65536, 66000)
    for st in (whole, a, b):
        h.step(st, 2)
    torch.cuda.synchronize()
    hw, ha, hb = whole.to_host(), a.to_host(), b.to_host()
    for k in hw:
        assert torch.equal(hw[k], torch.cat([ha[k], hb[k]])), k
    h.close()


def _bench_like_state(hpt, y, t, prec, accepts):
    st = hpt.PathState(y.shape[0], y.shape[1], prec)
    yd = torch.from_numpy(y).cuda().to(st.y.dtype)
    st.y.copy_(yd)
    st.y_acc.copy_(yd)
    st.tau.copy_(torch.from_numpy(np.log(t)))
    st.tau_acc.copy_(st.tau)
    st.dtau.fill_(0.01)
    st.accepts.fill_(accepts)
    return st


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_step_full_size_sampled(hpt, oracle_mod, prec):
    """The throughput step at its full size and launch shape: n = 16, 32
    monomials per equation, 65,536 random points (seed 1), one hpt_step, the
    tolerance of the form (1e-3 FP64, 3e-3 mixed).  400 sampled paths (and
    both ends of the first and last tiles) are stepped by the oracle from the
    same state, cast to the form's precision.

    (A) One accepted point and dE_acc = 0: the same accept decisions and, where
        they agree, the same new state.
    (B) No accepted point: every path's new y_acc is y + d_N (accepted or not),
        so the Newton direction of every sampled path is compared.  FP64:
        relative 1e-10 on 99% of the paths.  Mixed: the evaluation is good to
        about 2e-4 of the term magnitudes and the solve factors the row- and
        column-equilibrated D_z H = H_y diag(y), which turns that into a
        relative error of at most about kappa_eq times as much, so
        |d_N - d_N(oracle)| <= 1e-3 kappa_eq |d_N(oracle)| on every sampled
        path, the worst e / kappa_eq below 1e-4 (kappa_eq of the oracle's
        D_z H, equilibrated; at these random points its median is about 50),
        the median error below 1e-3, and at most two decisions differing."""
    sysm, alpha = W.config3(16, 32)
    cell = {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 1}
    te = cells.t_exponents(sysm, cell)
    osys = oracle_mod.System(sysm, te["e"], te["D"])
    P = oracle_mod.Params(tol_accept=3e-3 if prec else 1e-3)
    prm = hpt.Params(tol_accept=P.tol_accept)
    p = 65536
    y, t = W.random_points(1, p, 16)
    if prec:
        y = y.astype(np.complex64).astype(np.complex128)
    idx = np.concatenate([[0, 127, 128, p - 128, p - 1],
                          np.random.default_rng(3).choice(p, 400, replace=False)])
    idx = np.unique(idx)
    h = hpt.System.from_laurent(sysm, cell, prec)
    got = {}
    for acc in (1, 0):
        st = _bench_like_state(hpt, y, t, prec, acc)
        h.step(st, 1, prm)
        torch.cuda.synchronize()
        got[acc] = {k: v.numpy()[idx] for k, v in st.to_host().items()}
    ost = {}
    for acc in (1, 0):
        o = oracle_mod.PathState.start(y[idx], 0.0, 0.01)
        o.tau[:] = np.log(t[idx])
        o.tauacc[:] = o.tau
        o.accepts[:] = acc
        osys.step(P, o, 1)
        ost[acc] = o

    def rel(a, b):
        return np.abs(a - b).max(-1) / np.maximum(1.0, np.abs(b).max(-1))

    # (A) the bench's state
    g, o = got[1], ost[1]
    same = (g["accepts"] == o.accepts) & (g["status"] == o.status)
    assert same.mean() >= 0.97, same.mean()
    assert np.allclose(g["tau"][same], o.tau[same], rtol=0, atol=1e-12)
    assert np.allclose(g["dtau"][same], o.dtau[same], rtol=0, atol=1e-15)
    rej = same & (o.accepts == 1)    # rejected: the predicted point is y_acc again
    assert np.array_equal(g["y"][rej], y[idx][rej].astype(g["y"].dtype))
    if prec == 0:
        for a, b in (("y", "y"), ("yacc", "y_acc"), ("dEacc", "dE_acc")):
            assert rel(g[b][same], getattr(o, a)[same]).max() < 1e-10, a
    # (B) every path's Newton direction
    g, o = got[0], ost[0]
    same = g["status"] == o.status
    assert same.mean() >= 0.97, same.mean()
    act = same & (o.status == oracle_mod.ACTIVE)
    assert act.mean() > 0.9
    dg = g["y_acc"][act] - y[idx][act]
    do = o.yacc[act] - y[idx][act]
    if prec == 0:
        e = rel(g["y_acc"][act], o.yacc[act])
        assert np.quantile(e, 0.99) < 1e-10 and e.max() < 1e-6, np.sort(e)[-5:]
    else:
        _, Hy, _ = osys.eval(y[idx][act], np.log(t[idx][act]))
        A = Hy * y[idx][act][:, None, :]
        A = A / np.max(np.abs(A), axis=2, keepdims=True)
        A = A / np.max(np.abs(A), axis=1, keepdims=True)
        kappa = np.linalg.cond(A)
        e = np.abs(dg - do).max(-1) / np.abs(do).max(-1)
        ok = e <= 1e-3 * kappa
        q = np.quantile(e, [0.5, 0.9, 0.99])
        worst = float(np.max(e / kappa))
        print(f"mixed Newton directions: {int((~ok).sum())} of {ok.size} sampled paths beyond 1e-3 kappa_eq; "
              f"worst e/kappa_eq {worst:.3e}; decisions differ on {int((~same).sum())}; "
              f"e quantiles {q}")
        # counted, not a fraction: no sampled path may miss the bound (the
        # worst measured e/kappa_eq is about 4e-6), and at most two
        # decisions may differ from the oracle's
        assert int((~ok).sum()) == 0 and worst < 1e-4 and q[0] < 1e-3, (int((~ok).sum()), worst, q)
        assert int((~same).sum()) <= 2, int((~same).sum())


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_step_control_schedule(hpt, prec):
    """The GPU step control on the path y(tau) = (c0 + c2 e^tau) / c1 of
    h = c1 y - c0 - c2 t, accepting every step (tol_accept = 1e30) from
    tau = -3 with dtau 0.05: the Newton points are at the hand-worked tau
    values (the step doubles after every third accept up to 0.5 and the last
    one lands on tau = 0 exactly), y_acc is on the path (FP64 1e-14, mixed
    1e-5) and the 14th step ends the path as converged -- the same schedule
    the oracle's pins check."""
    c1, c0, c2 = 2 - 1j, 0.5 + 0.25j, -1.5 + 2j
    yx = lambda tau: (c0 + c2 * np.exp(tau)) / c1
    h = hpt.System(1, [3], np.array([[1], [0], [0]]), np.array([c1, -c0, -c2]), np.array([0, 0, 1]),
                   {"kind": "explicit", "alpha_num": [0], "beta_num": [0], "denom": 1}, prec)
    st = h.new_state(1)
    y0 = torch.tensor([[yx(-3.0)]], dtype=st.y.dtype, device="cuda")
    st.y.copy_(y0)
    st.y_acc.copy_(y0)
    st.tau.fill_(-3.0)
    st.tau_acc.fill_(-3.0)
    st.dtau.fill_(0.05)
    taus = [-3, -2.95, -2.90, -2.80, -2.70, -2.60, -2.40, -2.20, -2.00, -1.60, -1.20, -0.80, -0.30, 0.0]
    dts = [0.05, 0.05, 0.1, 0.1, 0.1, 0.2, 0.2, 0.2, 0.4, 0.4, 0.4, 0.5, 0.5]
    tol = 1e-14 if prec == 0 else 1e-5
    for k in range(14):
        h.step(st, 1, hpt.Params(tol_accept=1e30))
        r = {f: v.numpy() for f, v in st.to_host().items()}
        assert r["accepts"][0] == k + 1 and r["rejects"][0] == 0
        assert abs(r["tau_acc"][0] - taus[k]) < 1e-12
        assert abs(r["y_acc"][0, 0] - yx(taus[k])) < tol * max(1.0, abs(yx(taus[k])))
        if k < 13:
            assert r["status"][0] == hpt.ACTIVE and abs(r["dtau"][0] - dts[k]) < 1e-15 and r["tau"][0] <= 0.0
    assert r["status"][0] == hpt.CONVERGED and r["tau_acc"][0] == 0.0
    assert h.device_error() == 0


@pytest.mark.parametrize("n,m", [(1, 3), (3, 6), (8, 12), (9, 14), (13, 20), (16, 32)])
def test_mixed_step_newton_directions(hpt, oracle_mod, n, m):
    """The FP32 step of one system for each lane-group shape of its solve
    (n <= 8: 8 lanes, n <= 16: 16 lanes, one row per lane) on 3,000 random
    points (23 full tiles and a ragged tail): from a state with no accepted
    point every active path's new y_acc is y + d_N, so its Newton direction is
    compared with the oracle's from the same (complex64) point, within
    1e-3 kappa_eq (kappa_eq: condition number of the oracle's row- and
    column-equilibrated D_z H), and the statuses agree."""
    sysm = W.laurent_system(70 + n, n, m, -3, 3, 64, nnz=min(4, n))
    alpha = W.random_alpha(70 + n, n)
    cell = {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 1}
    y, t = W.random_points(11, 3000, n)
    _newton_direction_check(hpt, oracle_mod, sysm, cell, y, t, f"n={n}")


def test_mixed_step_large_exponents(hpt, oracle_mod):
    """The pipelined evaluation's fixed-point phase (monomials with sum |a_j|
    > 64, here 160..820) inside a whole FP32 step: n = 6, 8 monomials per
    equation, 3,000 points near the unit torus (23 full tiles and a ragged
    tail), Newton directions as in test_mixed_step_newton_directions."""
    s = W.large_exponent_system(31, 6, 8, 3, 40, 250)
    assert (np.abs(s.exponents).sum(1) > 64).sum() == 18
    cell = {"kind": "lower", "alpha_num": [0] * 6, "denom": 1}
    y, t = W.torus_points(8, 3000, 6, 0.005)
    _newton_direction_check(hpt, oracle_mod, s, cell, y, t, "large exponents")


def _newton_direction_check(hpt, oracle_mod, sysm, cell, y, t, label):
    te = cells.t_exponents(sysm, cell)
    osys = oracle_mod.System(sysm, te["e"], te["D"])
    p, n = y.shape
    y = y.astype(np.complex64).astype(np.complex128)
    h = hpt.System.from_laurent(sysm, cell, hpt.HPT_MIXED)
    st = _bench_like_state(hpt, y, t, 1, 0)
    h.profile(True)
    h.step(st, 1, hpt.Params(tol_accept=3e-3))
    torch.cuda.synchronize()
    h.profile(False)
    assert "eval_pipe_tc" in h.profile_read()   # n <= 16: the pipelined evaluation
    g = {k: v.numpy() for k, v in st.to_host().items()}
    o = oracle_mod.PathState.start(y, 0.0, 0.01)
    o.tau[:] = np.log(t)
    o.tauacc[:] = o.tau
    osys.step(oracle_mod.Params(tol_accept=3e-3), o, 1)
    same = g["status"] == o.status
    assert int((~same).sum()) <= 3, int((~same).sum())
    act = same & (o.status == oracle_mod.ACTIVE)
    assert act.mean() > 0.9
    dg = g["y_acc"][act] - y[act]
    do = o.yacc[act] - y[act]
    _, Hy, _ = osys.eval(y[act], np.log(t[act]))
    A = Hy * y[act][:, None, :]
    A = A / np.max(np.abs(A), axis=2, keepdims=True)
    A = A / np.max(np.abs(A), axis=1, keepdims=True)
    kappa = np.linalg.cond(A)
    e = np.abs(dg - do).max(-1) / np.abs(do).max(-1)
    miss = int((e > 1e-3 * kappa).sum())
    print(f"{label}: {miss} of {e.size} paths beyond 1e-3 kappa_eq, worst e/kappa_eq "
          f"{float(np.max(e / kappa)):.3e}, median e {float(np.median(e)):.2e}")
    assert miss == 0 and float(np.median(e)) < 1e-3
    h.close()

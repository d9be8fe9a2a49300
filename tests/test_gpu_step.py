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

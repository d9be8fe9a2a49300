"""The largest systems the library takes (GPU).

n = 32 variables is the library's bound: 36 monomials per equation
(M = 1,152), exponent vectors with 8 nonzeros in [-2, 2] (so the sum of
|a_j| stays inside the mixed form's exponent limit), a lower cell.

* Evaluation parity with the oracle (FP64 1e-11, mixed 2e-4 of the term
  magnitudes) on 300 points -- two full tiles and a ragged third -- in the
  32-variable shapes of both evaluation kernels.
* One step from a state with no accepted point, so that every path's new
  y_acc is y + d_N: FP64 within 1e-10 of the oracle on 99% of the paths
  (the 32-lane solve); mixed within 1e-3 kappa_eq of it on 97%, kappa_eq the
  condition number of the equilibrated D_z H that the solve factors.
* The projective form at n = 31 (32 homogeneous coordinates): evaluation
  parity.  n = 32 has no projective form (HPT_ENOTSUP) and n = 33 no handle
  (HPT_EINVAL).
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


def _case(n):
    s = W.laurent_system(320 + n, n, 36, -2, 2, 8, nnz=8)
    alpha = W.random_alpha(321 + n, n, -1, 1)
    return s, {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 1}


def _points(seed, p, n):
    y, t = W.random_points(seed, p, n)
    return y, np.ascontiguousarray(0.05 + 0.95 * t)


def _errs(got, ref, scale, t, f):
    (H, Hy, Ht), (Ho, Hyo, Hto), (SH, SHy, SHt) = got, ref, scale
    # the library returns dH/dt = (dH/dtau) / t; the oracles return dH/dtau
    return (_util.scaled_err(H, Ho, np.maximum(SH, f)), _util.scaled_err(Hy, Hyo, np.maximum(SHy, f)),
            _util.scaled_err(Ht, Hto / t[:, None], np.maximum(SHt, f) / t[:, None]))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_n32_eval_parity(hpt, oracle_mod, prec):
    s, cell = _case(32)
    te = cells.t_exponents(s, cell)
    osys = oracle_mod.System(s, te["e"], te["D"])
    h = hpt.System.from_laurent(s, cell, prec)
    y, t = _points(32, 300, 32)
    got = [a.cpu().numpy() for a in h.eval(torch.from_numpy(y).to("cuda", h.cdtype), torch.from_numpy(t).cuda())]
    assert h.device_error() == 0
    errs = _errs(got, osys.eval(y, np.log(t)), osys.scale(y, np.log(t)), t, FLOOR[prec])
    assert max(errs) <= TOL[prec], errs


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_n32_newton_directions(hpt, oracle_mod, prec):
    s, cell = _case(32)
    te = cells.t_exponents(s, cell)
    osys = oracle_mod.System(s, te["e"], te["D"])
    P = oracle_mod.Params(tol_accept=3e-3 if prec else 1e-3)
    h = hpt.System.from_laurent(s, cell, prec)
    p = 300
    y, t = _points(33, p, 32)
    if prec:
        y = y.astype(np.complex64).astype(np.complex128)
    st = h.new_state(p)
    yd = torch.from_numpy(y).to("cuda", st.y.dtype)
    st.y.copy_(yd)
    st.y_acc.copy_(yd)
    st.tau.copy_(torch.from_numpy(np.log(t)))
    st.tau_acc.copy_(st.tau)
    st.dtau.fill_(0.01)
    h.step(st, 1, hpt.Params(tol_accept=P.tol_accept))
    g = {k: v.numpy() for k, v in st.to_host().items()}
    assert h.device_error() == 0
    o = oracle_mod.PathState.start(y, 0.0, 0.01)
    o.tau[:] = np.log(t)
    o.tauacc[:] = o.tau
    osys.step(P, o, 1)
    same = g["status"] == o.status
    assert same.mean() >= 0.97, np.bincount(g["status"])
    act = same & (o.status == oracle_mod.ACTIVE)
    assert act.mean() > 0.9
    if prec == 0:
        e = np.abs(g["y_acc"][act] - o.yacc[act]).max(-1) / np.maximum(1.0, np.abs(o.yacc[act]).max(-1))
        assert np.quantile(e, 0.99) < 1e-10 and e.max() < 1e-6, np.sort(e)[-5:]
    else:
        _, Hy, _ = osys.eval(y[act], np.log(t[act]))
        A = Hy * y[act][:, None, :]
        A = A / np.max(np.abs(A), axis=2, keepdims=True)
        A = A / np.max(np.abs(A), axis=1, keepdims=True)
        kappa = np.linalg.cond(A)
        dg, do = g["y_acc"][act] - y[act], o.yacc[act] - y[act]
        e = np.abs(dg - do).max(-1) / np.abs(do).max(-1)
        ok = e <= 1e-3 * kappa
        assert ok.mean() >= 0.97, (ok.mean(), np.quantile(e, [0.5, 0.9, 0.99]), np.quantile(kappa, [0.5, 0.99]))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_n31_projective_eval_parity(hpt, prec):
    s, cell = _case(31)
    te = cells.t_exponents(s, cell)
    ps = PJ.ProjectiveSystem(s, te["e"], te["D"])
    h = hpt.System.from_laurent(s, cell, prec).homogenize()
    assert h.nv == 32 and np.array_equal(h.degrees, ps.deg)
    rng = np.random.default_rng(31)
    y = np.exp(rng.normal(0, 0.5, (300, 32))) * np.exp(2j * np.pi * rng.random((300, 32)))
    y = np.ascontiguousarray(y / np.linalg.norm(y, axis=1, keepdims=True))
    t = np.ascontiguousarray(rng.uniform(0.05, 1.0, 300))
    got = [a.cpu().numpy() for a in h.eval(torch.from_numpy(y).to("cuda", h.cdtype), torch.from_numpy(t).cuda())]
    assert h.device_error() == 0
    errs = _errs(got, ps.eval(y, np.log(t)), ps.scale(y, np.log(t)), t, FLOOR[prec])
    assert max(errs) <= TOL[prec], errs


def test_size_limits_refused(hpt):
    s, cell = _case(32)
    h = hpt.System.from_laurent(s, cell, 0)
    with pytest.raises(hpt.HptError) as ei:
        h.homogenize()                       # 33 homogeneous coordinates
    assert ei.value.code == 7
    s33 = W.laurent_system(353, 33, 3, -1, 1, 4, nnz=2)
    with pytest.raises(hpt.HptError) as ei:
        hpt.System.from_laurent(s33, {"kind": "lower", "alpha_num": [0] * 33, "denom": 1}, 0)
    assert ei.value.code == 1

"""Failure detection without a device fault (GPU).

Faults are made on the host, and every test ends by checking that the GPU
context is still usable (an evaluation that matches the oracle):

* a bounded device-side wait that nothing completes gives up after about
  2 s and is reported as HPT_ETIMEOUT (then cleared);
* non-finite coefficients and out-of-range step parameters are refused
  with status codes; tensors whose shape, dtype or device the library
  would misread (a state of the other precision or width, points with the
  affine width on a projective handle, host memory) and mismatched batch
  inputs are refused by the binding before any device work;
* on a system whose two equations coincide (singular Jacobian everywhere)
  every path stops within its step budget; non-finite start points end as
  HPT_PATH_SINGULAR; both forms, affine and projective.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cells

import _util

pytestmark = pytest.mark.gpu


def _usable(hpt, oracle_mod):
    s, cl, _ = _util.first_generic(W.config2)
    cell = {"kind": "pairs", "pairs": cl[0]["pairs"]}
    te = cells.t_exponents(s, cell)
    osys = oracle_mod.System(s, te["e"], te["D"])
    h = hpt.System.from_laurent(s, cell, 0)
    y, t = W.random_points(2, 64, s.n)
    H, _, _ = h.eval(torch.from_numpy(y).cuda(), torch.from_numpy(t).cuda())
    Ho, _, _ = osys.eval(y, np.log(t))
    SH, _, _ = osys.scale(y, np.log(t))
    assert _util.scaled_err(H.cpu().numpy(), Ho, SH) < 1e-11
    assert h.device_error() == 0


def test_bounded_wait_times_out_and_context_survives(hpt, oracle_mod):
    s, cl, _ = _util.first_generic(W.config1)
    h = hpt.System.from_laurent(s, {"kind": "pairs", "pairs": cl[0]["pairs"]}, 1)
    assert h.device_error() == 0
    h.check_bounded_wait()
    assert h.device_error() == 6          # HPT_ETIMEOUT
    assert h.device_error() == 0          # read and cleared
    _usable(hpt, oracle_mod)


def test_refusals(hpt, oracle_mod):
    s, cl, _ = _util.first_generic(W.config2)
    cell = {"kind": "pairs", "pairs": cl[0]["pairs"]}
    bad = s.coeffs.copy()
    bad[3] = np.nan
    with pytest.raises(hpt.HptError) as ei:
        hpt.System.from_laurent(s.with_coeffs(bad), cell, 0)
    assert ei.value.code == 1
    bad[3] = np.inf
    with pytest.raises(hpt.HptError):
        hpt.System.from_laurent(s.with_coeffs(bad), cell, 1)
    h = hpt.System.from_laurent(s, cell, 0)
    x0 = torch.from_numpy(cells.start_points(s, cl[0]["pairs"])).cuda()
    for kw in (dict(shrink=1.5), dict(dtau_min=1.0, dtau_max=0.1), dict(tol_accept=-1.0), dict(predictor=3),
               dict(max_steps=0), dict(div_bound=0.5)):
        with pytest.raises(hpt.HptError) as ei:
            h.track(x0, hpt.Params(**kw))
        assert ei.value.code == 1, kw
    hm = hpt.System.from_laurent(s, cell, 1)
    b = hpt.Batch([hm])
    # the library cannot see buffer sizes; the binding refuses before any device work
    with pytest.raises(ValueError):
        b.track(x0[:3].reshape(-1).contiguous(), [4], hpt.Params(tol_accept=3e-3))   # 3 paths of data, 4 announced
    with pytest.raises(ValueError):
        b.track(x0.reshape(-1).contiguous(), [x0.shape[0], 1], hpt.Params(tol_accept=3e-3))   # two counts, one system
    # tensors the library would read with another layout or size
    hp = h.homogenize()
    t = torch.rand(x0.shape[0], dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        hp.eval(x0, t)                                    # n columns where the projective form reads n + 1
    with pytest.raises(ValueError):
        h.eval(x0, t[:-1])                                # one t short
    with pytest.raises(ValueError):
        h.step(hm.new_state(x0.shape[0]), 1)              # a mixed-form state on an FP64 handle
    with pytest.raises(ValueError):
        h.step(hp.new_state(x0.shape[0]), 1)              # n + 1 variables per path on an affine handle
    with pytest.raises(ValueError):
        h.track(x0.to(torch.complex64))                   # start points are complex128
    with pytest.raises(ValueError):
        h.track(x0.cpu())                                 # host memory
    with pytest.raises(ValueError):
        h.polish(x0[:, :-1].contiguous())
    _usable(hpt, oracle_mod)


def _duplicate_equation_system(hpt, prec):
    """config 2 with equation 1 replaced by a copy of equation 0 (same
    support, coefficients and t-exponents through an explicit cell)."""
    s, cl, _ = _util.first_generic(W.config2)
    cell = {"kind": "pairs", "pairs": cl[0]["pairs"]}
    te = cells.t_exponents(s, cell)
    off = s.offsets
    m = list(s.m)
    rows = [s.support(k) for k in range(s.n)]
    co = [s.coeffs[off[k]:off[k] + m[k]] for k in range(s.n)]
    li = [s.lifting[off[k]:off[k] + m[k]] for k in range(s.n)]
    rows[1], co[1], li[1], m[1] = rows[0], co[0], li[0], m[0]
    s2 = W.LaurentSystem(s.n, m, np.concatenate(rows), np.concatenate(co), np.concatenate(li))
    beta = list(te["beta_num"])
    beta[1] = beta[0]
    ecell = {"kind": "explicit", "alpha_num": list(te["alpha_num"]), "beta_num": beta, "denom": te["D"]}
    return s2, hpt.System.from_laurent(s2, ecell, prec)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_singular_and_nonfinite_paths(hpt, oracle_mod, prec):
    """Two equal equations: every path stops within the step budget with a
    status (elimination may leave a rounding-size pivot instead of an exact
    zero, so which status depends on rounding) and the device reports no
    error; non-finite start points on a regular system: SINGULAR."""
    s2, h = _duplicate_equation_system(hpt, prec)
    rng = np.random.default_rng(5)
    x0 = np.exp(rng.normal(0, 0.3, (40, s2.n)) + 2j * np.pi * rng.random((40, s2.n)))
    prm = hpt.Params(tol_accept=3e-3 if prec else 1e-3, max_steps=200)
    for hh in (h, h.homogenize()):
        g = hh.new_state(40)
        hh.paths_init(g, torch.from_numpy(x0).cuda(), prm)
        hh.step(g, 210, prm)
        st = g.status.cpu().numpy()
        assert not (st == hpt.ACTIVE).any(), np.bincount(st)
        assert hh.device_error() == 0
    s, cl, _ = _util.first_generic(W.config2)
    c = max(cl, key=lambda c: c["det"])
    hr = hpt.System.from_laurent(s, {"kind": "pairs", "pairs": c["pairs"]}, prec)
    x1 = cells.start_points(s, c["pairs"])[:32].copy()
    x1[5, 2] = np.nan
    x1[9, 0] = np.inf
    for hh in (hr, hr.homogenize()):
        g = hh.new_state(32)
        hh.paths_init(g, torch.from_numpy(x1).cuda(), prm)
        hh.step(g, 3, prm)
        st = g.status.cpu().numpy()
        assert st[5] == hpt.SINGULAR and st[9] == hpt.SINGULAR, st
        assert (np.delete(st, [5, 9]) != hpt.SINGULAR).all()
        assert hh.device_error() == 0
    _usable(hpt, oracle_mod)

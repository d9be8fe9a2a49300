"""Evaluation parity, CUDA path vs the CPU oracle (GPU).

Tolerance (componentwise, scaled by the sum of term magnitudes the oracle
returns): FP64 form <= 1e-11, mixed split-BF16 form <= 2e-4 per evaluation.
The mixed form holds FP32/BF16 values, whose normal range ends at 1.2e-38
(BF16 low parts sit 2^-8 lower), so its scale has an absolute floor of 1e-30:
entries whose whole magnitude sum lies below it (terms with large t-exponents
at small t, down to 1e-291 here) are compared absolutely.  For H_t = H_tau / t
the floor applies to H_tau, the FP32 value the kernel accumulates before its
exact division by t (at t = 2.4e-4 an H_tau of 7e-38 is still an FP32 sum
of flushed terms, while H_t = 3e-34 would clear a floor applied after the
division).
Sizes span several 128-point tiles and a ragged tail; the full 65,536-point
throughput workload is checked on sampled points.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cells

import _util

pytestmark = pytest.mark.gpu
TOL = {0: 1e-11, 1: 2e-4}
FLOOR = {0: 0.0, 1: 1e-30}


def _run(hpt, oracle_mod, s, cell, prec, y, t, sample=None):
    te = cells.t_exponents(s, cell)
    osys = oracle_mod.System(s, te["e"], te["D"])
    h = hpt.System.from_laurent(s, cell, prec)
    assert h.texp()["e"] == te["e"]
    yd = torch.from_numpy(y).to("cuda", h.cdtype)
    td = torch.from_numpy(t).cuda()
    H, Hy, Ht = (a.cpu().numpy() for a in h.eval(yd, td))
    torch.cuda.synchronize()
    assert h.device_error() == 0
    if sample is not None:
        y, t, H, Hy, Ht = y[sample], t[sample], H[sample], Hy[sample], Ht[sample]
    Ho, Hyo, Hto = osys.eval(y, np.log(t))
    SH, SHy, SHt = osys.scale(y, np.log(t))
    h.close()
    # the library returns dH/dt = (dH/dtau) / t; the oracle returns dH/dtau
    f = FLOOR[prec]
    return (_util.scaled_err(H, Ho, np.maximum(SH, f)), _util.scaled_err(Hy, Hyo, np.maximum(SHy, f)),
            _util.scaled_err(Ht, Hto / t[:, None], np.maximum(SHt, f) / t[:, None]))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name", ["n2", "n4", "n7_ragged", "n16", "n24"])
@pytest.mark.parametrize("p", [1, 333])
def test_eval_parity(hpt, oracle_mod, name, prec, p):
    s, cell = _util.eval_case(name)
    y, t = W.random_points(7, p, s.n)
    errs = _run(hpt, oracle_mod, s, cell, prec, y, t)
    assert max(errs) <= TOL[prec], errs


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_eval_full_size_sampled(hpt, oracle_mod, prec):
    s, cell = _util.eval_case("n16")
    y, t = W.random_points(1, 65536, 16)
    sample = np.random.default_rng(0).choice(65536, 384, replace=False)
    sample = np.concatenate([sample, [0, 127, 128, 65535]])
    errs = _run(hpt, oracle_mod, s, cell, prec, y, t, sample)
    assert max(errs) <= TOL[prec], errs


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_eval_tile_edges(hpt, oracle_mod, prec):
    s, cell = _util.eval_case("n4")
    for p in (127, 128, 129, 256):
        y, t = W.random_points(p, p, s.n)
        assert max(_run(hpt, oracle_mod, s, cell, prec, y, t)) <= TOL[prec]


def test_eval_empty_is_noop(hpt):
    s, cell = _util.eval_case("n4")
    h = hpt.System.from_laurent(s, cell, 0)
    y = torch.zeros(0, 4, dtype=torch.complex128, device="cuda")
    t = torch.zeros(0, dtype=torch.float64, device="cuda")
    H, Hy, Ht = h.eval(y, t)
    assert H.shape == (0, 4) and Hy.shape == (0, 4, 4)


def test_mixed_rejects_inexact_exponents(hpt):
    s = W.laurent_system(3, 3, 4, -2, 2, 8)
    e = s.exponents.copy()
    e[0, 0] = 300
    s2 = W.LaurentSystem(3, s.m, e, s.coeffs, s.lifting)
    cell = {"kind": "lower", "alpha_num": [0, 0, 0], "denom": 1}
    with pytest.raises(hpt.HptError) as err:
        hpt.System.from_laurent(s2, cell, 1)
    assert err.value.code == 4
    hpt.System.from_laurent(s2, cell, 0).close()   # FP64 form takes it


def test_mixed_refuses_shapes_beyond_on_chip_memory(hpt):
    """n = 24 with 128 monomials per equation does not fit the evaluation
    kernel's shared memory: HPT_ENOTSUP at creation, not a failing launch."""
    s = W.laurent_system(31, 24, 128, -1, 1, 8, nnz=4)
    alpha = W.random_alpha(31, 24, -1, 1)
    with pytest.raises(hpt.HptError) as ei:
        hpt.System.from_laurent(s, {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 1}, hpt.HPT_MIXED)
    assert ei.value.code == 7


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_eval_parity_large_exponents(hpt, oracle_mod, prec):
    """Three monomials per equation with sum |a_j| between about 160 and 820
    (four coordinates of magnitude 40..250) at points near the unit torus,
    where such monomials stay in range: the mixed form takes their phase
    sum_j a_j arg(y_j) in 32-bit fixed point, exact modulo one revolution,
    instead of from the FP32 exponent GEMM, and meets the same 2e-4 (333
    points, three tiles with a ragged tail)."""
    s = W.large_exponent_system(31, 6, 8, 3, 40, 250)
    assert (np.abs(s.exponents).sum(1) > 64).sum() == 18
    cell = {"kind": "lower", "alpha_num": [0] * 6, "denom": 1}
    y, t = W.torus_points(8, 333, 6, 0.005)
    errs = _run(hpt, oracle_mod, s, cell, prec, y, t)
    print("large exponents", ["fp64", "mixed"][prec], errs)
    assert max(errs) <= TOL[prec], errs

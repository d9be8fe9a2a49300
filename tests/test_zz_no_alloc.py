"""hpt_step_static, the step without device-memory allocation (GPU).

Some callers cannot let a library call cudaMalloc while they run: they give
all device memory to their own allocator or pool, keep a fixed device-memory
budget, or cannot afford the synchronisation of an allocation inside their
loop.  hpt_step_static serves them with scratch from a fixed 32 MiB array in
the library.  This file is collected last so that a stop at the first failure
has already run every other test; it passes alone in a fresh process and after
the others.  Checked through the C ABI: two calls in a row give the same
states as hpt_step (bit for bit: same kernels on the same inputs), in both
forms, at n = 16 within one round and at n = 2 over two rounds of 65,536
paths, and a batch over the array's limit is refused with HPT_ERANGE.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cells

pytestmark = pytest.mark.gpu
FIELDS = ("y", "tau", "dtau", "y_acc", "tau_acc", "dE_acc", "status", "steps", "accepts",
          "rejects", "streak")


def _state(hpt, h, y, t, prec):
    st = hpt.PathState(y.shape[0], y.shape[1], prec)
    yd = torch.from_numpy(y).to("cuda", h.cdtype)
    st.y.copy_(yd)
    st.y_acc.copy_(yd)
    st.tau.copy_(torch.from_numpy(np.log(t)))
    st.tau_acc.copy_(st.tau)
    st.dtau.fill_(0.01)
    st.accepts.fill_(1)
    return st


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_static_step_matches_step(hpt, prec):
    sysm, alpha = W.config3(16, 32)
    cell = {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 1}
    h = hpt.System.from_laurent(sysm, cell, prec)
    y, t = W.random_points(5, 4000, 16)      # 31 tiles and a ragged tail
    prm = hpt.Params(tol_accept=1e-3 if prec == 0 else 3e-3)
    ref = _state(hpt, h, y, t, prec)
    got = _state(hpt, h, y, t, prec)
    for _ in range(2):                       # two calls in a row
        h.step(ref, 1, prm)
        h.step_static(got, 1, prm)
        torch.cuda.synchronize()
        for f in FIELDS:
            a, b = getattr(ref, f), getattr(got, f)
            assert torch.equal(a, b), f
    assert h.device_error() == 0
    h.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_static_step_matches_step_beyond_one_round(hpt, prec):
    """At n = 2 the array holds far more than the 65,536 paths of one round
    of hpt_step; 70,001 paths run as two rounds, exactly as in hpt_step."""
    s = W.config1(0)
    cl, _ = cells.mixed_cells(s)
    h = hpt.System.from_laurent(s, {"kind": "pairs", "pairs": cl[0]["pairs"]}, prec)
    y, t = W.random_points(6, 70001, 2)
    prm = hpt.Params(tol_accept=1e-3 if prec == 0 else 3e-3)
    ref = _state(hpt, h, y, t, prec)
    got = _state(hpt, h, y, t, prec)
    for _ in range(2):
        h.step(ref, 1, prm)
        h.step_static(got, 1, prm)
        torch.cuda.synchronize()
        for f in FIELDS:
            assert torch.equal(getattr(ref, f), getattr(got, f)), f
    assert h.device_error() == 0
    h.close()


def test_static_step_rejects_oversized_batch(hpt):
    s = W.config2(1)
    cl, _ = cells.mixed_cells(s)
    h = hpt.System.from_laurent(s, {"kind": "pairs", "pairs": cl[0]["pairs"]}, 0)
    jac = 4 * 6 * 16
    limit = ((32 << 20) - 511 - 127 * jac) // (jac + 8)
    st = hpt.PathState(limit + 1, 4, 0)       # a real state of the refused size
    with pytest.raises(hpt.HptError) as err:
        h.step_static(st, 1)
    assert err.value.code == 4 and "static scratch limit" in str(err.value)
    h.close()

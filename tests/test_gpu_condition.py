"""The FP32 solve's condition proxy on the GPU against the oracle (GPU).

The mixed form's solve redoes in FP64 every path whose pivot ratio
max |u_jj| / min |u_jj| (after power-of-two row and column equilibration)
exceeds params.cond_max.  Here the paths it flags at a bound T are read off
the GPU: the same step from the same state with cond_max = T and with
cond_max = 1e30 (every path accepted, so each one stores both solutions)
differs exactly on the paths re-solved in FP64.  They are compared with the
oracle's pivot ratio of the same equilibrated D_z H (oracle.condest, from
the oracle's FP64 Jacobian): every path whose ratio is more than 25% from T
is flagged exactly when its ratio exceeds T.  The Hager-Higham kappa_1 of the
same matrices is printed beside (the proxy's calibration against it is a CPU
test, tests/test_oracle_condest.py).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cells, condest

pytestmark = pytest.mark.gpu


def test_condition_proxy_flags(hpt, oracle_mod):
    sysm, alpha = W.config3(16, 32)
    cell = {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 1}
    te = cells.t_exponents(sysm, cell)
    osys = oracle_mod.System(sysm, te["e"], te["D"])
    p = 4000
    y, t = W.random_points(21, p, 16)
    y = y.astype(np.complex64).astype(np.complex128)
    h = hpt.System.from_laurent(sysm, cell, hpt.HPT_MIXED)

    def step(cmax):
        st = hpt.PathState(p, 16, hpt.HPT_MIXED)
        yd = torch.from_numpy(y).cuda().to(torch.complex64)
        st.y.copy_(yd)
        st.y_acc.copy_(yd)
        st.tau.copy_(torch.from_numpy(np.log(t)))
        st.tau_acc.copy_(st.tau)
        st.dtau.fill_(0.01)
        st.accepts.fill_(1)
        h.step(st, 1, hpt.Params(tol_accept=1e30, cond_max=cmax))
        torch.cuda.synchronize()
        return st.to_host()

    ref = step(1e30)
    acc = ref["accepts"].numpy() == 2   # accepted: both solutions stored
    assert acc.mean() > 0.99
    _, Hy, _ = osys.eval(y, np.log(t))
    D = Hy * y[:, None, :]
    ratio = np.array([condest.pivot_ratio(a) for a in D])[acc]
    kappa = np.array([condest.cond1_estimate(a) for a in condest.pow2_equilibrate(D)])[acc]
    for T in (10.0, 30.0, 100.0):
        got = step(T)
        fl = ~(torch.all(got["y_acc"] == ref["y_acc"], dim=1) & torch.all(got["dE_acc"] == ref["dE_acc"], dim=1))
        fl = fl.numpy()[acc]
        clear = np.abs(np.log(ratio / T)) > np.log(1.25)
        print(f"T={T:g}: flagged {int(fl.sum())}, oracle ratio above {int((ratio > T).sum())}, "
              f"disagreeing outside the band {int((fl != (ratio > T))[clear].sum())}; kappa_1 of the flagged "
              f"paths: min {kappa[fl].min() if fl.any() else float('nan'):.3g}")
        assert fl.any() and (~fl).any()
        assert np.array_equal(fl[clear], (ratio > T)[clear])
    h.close()

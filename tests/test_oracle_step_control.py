"""Pins of the oracle's step control (CPU only).

The control rule is a stated reading (the paper gives none): accept when
|d_N|_inf / max(1, |y|_inf) <= tol_accept; after grow_after = 3 accepts in a
row the step doubles, up to dtau_max = 0.5; a reject halves it and predicts
again from the last accepted point, with STEP_UNDERFLOW below dtau_min =
1e-8; the step never passes tau = 0, and an accept at tau = 0 ends the path.

The system is h = c1 y - c0 - c2 t (t-exponent 1 on the last term), whose
path is y(tau) = (c0 + c2 e^tau) / c1.  The equation is linear in y, so one
Newton step lands exactly on the path, and the Euler direction at a path
point is y'(tau) = c2 e^tau / c1.  The expected values below come from that
closed form and from the rule worked by hand, not from the oracle.
"""
import numpy as np

import workloads as W

C1, C0, C2 = 2 - 1j, 0.5 + 0.25j, -1.5 + 2j


def _y(tau):
    return (C0 + C2 * np.exp(tau)) / C1


def _dy(tau):
    return C2 * np.exp(tau) / C1


def _system(oracle_mod):
    s = W.LaurentSystem(1, [3], np.array([[1], [0], [0]]), np.array([C1, -C0, -C2]), np.zeros(3, np.int64))
    return oracle_mod.System(s, np.array([0, 0, 1]), 1)


def _run(oracle_mod, P, st, k):
    osys = _system(oracle_mod)
    rec = []
    for _ in range(k):
        osys.step(P, st, 1)
        rec.append({f: getattr(st, f).copy() for f in ("y", "tau", "dtau", "yacc", "tauacc", "dEacc", "status",
                                                       "steps", "accepts", "rejects", "streak")})
    return rec


def test_always_accept_schedule(oracle_mod):
    """tol_accept = 1e30 accepts every step.  From tau0 = -3 with dtau 0.05:
    the Newton points are at tau = -3, -2.95, -2.90 (then the step doubles to
    0.1), -2.80, -2.70, -2.60 (0.2), -2.40, -2.20, -2.00 (0.4), -1.60,
    -1.20, -0.80 (0.5, the cap), -0.30, and then 0 exactly (the last step is
    0.30, not 0.5), where the 14th step ends the path as converged."""
    P = oracle_mod.Params(tol_accept=1e30)
    st = oracle_mod.PathState.start(np.array([[_y(-3.0)]]), -3.0, 0.05)
    rec = _run(oracle_mod, P, st, 16)
    taus = [-3, -2.95, -2.90, -2.80, -2.70, -2.60, -2.40, -2.20, -2.00, -1.60, -1.20, -0.80, -0.30, 0.0]
    dts = [0.05, 0.05, 0.1, 0.1, 0.1, 0.2, 0.2, 0.2, 0.4, 0.4, 0.4, 0.5, 0.5]
    for k, r in enumerate(rec[:14]):
        assert r["accepts"][0] == k + 1 and r["rejects"][0] == 0 and r["steps"][0] == k + 1
        assert abs(r["tauacc"][0] - taus[k]) < 1e-12
        assert abs(r["yacc"][0, 0] - _y(taus[k])) < 1e-14 * max(1.0, abs(_y(taus[k])))
        assert abs(r["dEacc"][0, 0] - _dy(taus[k])) < 1e-13
        if k < 13:
            assert r["status"][0] == oracle_mod.ACTIVE
            assert abs(r["dtau"][0] - dts[k]) < 1e-15
            assert r["streak"][0] == (k + 1) % 3
            assert -1e-15 < r["tau"][0] - r["tauacc"][0] <= r["dtau"][0] + 1e-15 and r["tau"][0] <= 0.0
            assert abs(r["y"][0, 0] - (r["yacc"][0, 0] + (r["tau"][0] - r["tauacc"][0]) * r["dEacc"][0, 0])) < 1e-14
    assert rec[12]["tau"][0] == 0.0                     # the last step lands on tau = 0 exactly
    assert rec[13]["status"][0] == oracle_mod.CONVERGED and rec[13]["tauacc"][0] == 0.0
    assert rec[15]["steps"][0] == 14                    # a finished path is not stepped again


def test_always_reject_underflow(oracle_mod):
    """tol_accept = -1 rejects every step.  After one accepted step the
    prediction is redone from the same accepted point with the step halved
    each time: 0.05 / 2^22 = 1.19e-8 is still >= 1e-8, 0.05 / 2^23 = 5.96e-9
    is not, so the 23rd reject ends the path with STEP_UNDERFLOW."""
    P = oracle_mod.Params(tol_accept=1e30)
    st = oracle_mod.PathState.start(np.array([[_y(-3.0)]]), -3.0, 0.05)
    _run(oracle_mod, P, st, 1)
    ya, ta, da = st.yacc.copy(), st.tauacc.copy(), st.dEacc.copy()
    P = oracle_mod.Params(tol_accept=-1.0)
    rec = _run(oracle_mod, P, st, 25)
    for k, r in enumerate(rec):
        assert r["accepts"][0] == 1 and r["streak"][0] == 0
        assert np.array_equal(r["yacc"], ya) and np.array_equal(r["tauacc"], ta) and np.array_equal(r["dEacc"], da)
        if k < 22:
            assert r["status"][0] == oracle_mod.ACTIVE and r["rejects"][0] == k + 1
            h = 0.05 * 0.5 ** (k + 1)
            assert r["dtau"][0] == h
            assert r["tau"][0] == ta[0] + h
            assert abs(r["y"][0, 0] - (ya[0, 0] + h * da[0, 0])) < 1e-15
    assert rec[22]["status"][0] == oracle_mod.UNDERFLOW and rec[22]["rejects"][0] == 23
    assert rec[24]["rejects"][0] == 23


def test_start_phase_corrects_in_place(oracle_mod):
    """Before the first accept a reject does not move tau or the step: the
    point is Newton-corrected where it is (here onto the path in one step,
    the equation being linear), and max_steps ends the path."""
    P = oracle_mod.Params(tol_accept=-1.0, max_steps=5)
    st = oracle_mod.PathState.start(np.array([[_y(-3.0) + 0.3 - 0.2j]]), -3.0, 0.05)
    rec = _run(oracle_mod, P, st, 6)
    for k, r in enumerate(rec[:5]):
        assert r["accepts"][0] == 0 and r["rejects"][0] == k + 1
        assert r["tau"][0] == -3.0 and r["dtau"][0] == 0.05
        assert abs(r["y"][0, 0] - _y(-3.0)) < 1e-15 and np.array_equal(r["y"], r["yacc"])
    assert rec[3]["status"][0] == oracle_mod.ACTIVE and rec[4]["status"][0] == oracle_mod.MAX_STEPS


def test_decisions_follow_the_closed_form_error(oracle_mod):
    """With tol_accept = 1e-3 along the whole path: before each step the
    Newton correction at the predicted point (y, tau) is y(tau) - y exactly,
    so the oracle must accept exactly when |y(tau) - y| / max(1, |y|) <=
    1e-3; an accept doubles the step after three in a row or keeps it, a
    reject halves it.  Both kinds occur on this path."""
    P = oracle_mod.Params(tol_accept=1e-3)
    st = oracle_mod.PathState.start(np.array([[_y(-3.0)]]), -3.0, 0.05)
    osys = _system(oracle_mod)
    seen = {True: 0, False: 0}
    for _ in range(400):
        if st.status[0] != oracle_mod.ACTIVE:
            break
        y, tau, dt, acc = st.y[0, 0], st.tau[0], st.dtau[0], st.accepts[0]
        err = abs(_y(tau) - y) / max(1.0, abs(y))
        osys.step(P, st, 1)
        accepted = st.accepts[0] == acc + 1
        if abs(err - P.tol_accept) > 1e-9 * P.tol_accept:
            assert accepted == (err <= P.tol_accept), (tau, err)
        seen[bool(accepted)] += 1
        if st.status[0] == oracle_mod.ACTIVE and acc > 0:
            assert st.dtau[0] in ((dt, min(2 * dt, 0.5)) if accepted else (dt / 2,))
    assert st.status[0] == oracle_mod.CONVERGED and abs(st.yacc[0, 0] - _y(0.0)) < 1e-14
    assert seen[True] > 10 and seen[False] > 0, seen

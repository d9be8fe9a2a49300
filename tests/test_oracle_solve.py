"""Pins of the oracle's consolidated Euler+Newton solve (CPU only).

* The batched LU with partial pivoting against numpy.linalg.solve (LAPACK).
* The Euler and Newton directions against the residuals of their defining
  equations, Section 2.3: H_y E + H_tau = 0 and H_y N + H = 0.
* A closed-form path (one variable, linear in y) where both directions are
  known exactly.
"""
import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("n", [1, 2, 5, 16, 24])
def test_lu_matches_lapack(oracle_mod, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((40, n, n)) + 1j * rng.standard_normal((40, n, n))
    B = rng.standard_normal((40, n, 2)) + 1j * rng.standard_normal((40, n, 2))
    X, ns = oracle_mod.solve(A, B)
    assert ns == 0
    ref = np.linalg.solve(A, B)
    assert np.allclose(X, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())


def test_lu_needs_pivoting(oracle_mod):
    # zero leading entries: elimination without row exchanges breaks down
    A = np.array([[[0, 1, 2], [3, 0, 1], [1, 1, 0]]], dtype=complex)
    B = np.array([[[1, 0], [0, 1], [1, 1]]], dtype=complex)
    X, ns = oracle_mod.solve(A, B)
    assert ns == 0
    assert np.allclose(X, np.linalg.solve(A, B), atol=1e-14)


def test_singular_flagged(oracle_mod):
    A = np.ones((1, 3, 3), complex)
    B = np.ones((1, 3, 2), complex)
    _, ns = oracle_mod.solve(A, B)
    assert ns == 1


def test_direction_residuals(oracle_mod):
    s = W.laurent_system(3, 6, 8, -2, 2, 16)
    texp = np.random.default_rng(3).integers(0, 9, size=s.M)
    osys = oracle_mod.System(s, texp, 1)
    y, t = W.random_points(2, 50, 6)
    tau = np.log(t)
    dE, dN, ok = osys.directions(y, tau)
    assert ok.all()
    H, Hy, Ht = osys.eval(y, tau)
    rE = np.einsum("pkj,pj->pk", Hy, dE) + Ht
    rN = np.einsum("pkj,pj->pk", Hy, dN) + H
    nrm = np.abs(Hy).max(axis=(1, 2))[:, None]
    assert np.max(np.abs(rE) / (nrm * (1 + np.abs(dE).max(1, keepdims=True)))) < 1e-12
    assert np.max(np.abs(rN) / (nrm * (1 + np.abs(dN).max(1, keepdims=True)))) < 1e-12


def test_closed_form_line(oracle_mod):
    """h(y, t) = c1 y - c0 - c2 t: the path is y(tau) = (c0 + c2 e^tau)/c1,
    E = c2 e^tau / c1, and Newton from any y lands on the path: N = y(tau) - y."""
    c1, c0, c2 = 2 - 1j, 0.5 + 0.25j, -1.5 + 2j
    s = W.LaurentSystem(1, [3], np.array([[1], [0], [0]]), np.array([c1, -c0, -c2]),
                        np.zeros(3, np.int64))
    osys = oracle_mod.System(s, np.array([0, 0, 1]), 1)
    tau = np.array([-3.0, -1.0, -0.25, 0.0])
    ypath = (c0 + c2 * np.exp(tau)) / c1
    y = ypath + np.array([0.1, -0.2j, 0.3 + 0.1j, 0.0])
    dE, dN, ok = osys.directions(y[:, None], tau)
    assert ok.all()
    assert np.allclose(dE[:, 0], c2 * np.exp(tau) / c1, rtol=1e-14, atol=1e-15)
    assert np.allclose(dN[:, 0], ypath - y, rtol=1e-13, atol=1e-15)

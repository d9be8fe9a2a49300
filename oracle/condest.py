"""1-norm condition estimate -- TEST INFRASTRUCTURE (part of the oracle).

Section 6 of the paper remarks that the consolidated linear systems can be
ill-conditioned; the library's FP32 solve redoes in FP64 the paths whose
condition proxy (the pivot ratio max |u_jj| / min |u_jj| after power-of-two
row and column equilibration) exceeds a bound.  The oracle's reference for
that proxy is a condition estimate by the published method of W. W. Hager
(1984, "Condition estimates", SIAM J. Sci. Stat. Comput. 5) with N. J.
Higham's refinements (1988, "FORTRAN codes for estimating the one-norm of a
real or complex matrix", ACM TOMS 14): a few solves with A and A^H on
vectors of unit 1-norm give a lower bound of ||A^{-1}||_1 that is exact or
close for most matrices; kappa_1 = ||A||_1 times that bound.  The solves
use the LU factorisation of scipy (a library step).

pivot_ratio restates the library's proxy from its definition, so that the
GPU's choice of paths can be checked against it and the proxy calibrated
against kappa_1.

Parity status: pinned by tests/test_oracle_condest.py (lower bound of and
closeness to numpy.linalg.cond(A, 1); exact on diagonal matrices; the
equilibration's scales are powers of two that put every row's and column's
largest entry in [1/2, 1); the pivot ratio of a diagonal matrix is the
ratio of its equilibrated entries).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def norm1_inv_estimate(A, itmax=5):
    """Lower bound of ||A^{-1}||_1 (A square, complex or real, nonsingular)."""
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    lu = scipy.linalg.lu_factor(A)
    x = np.full(n, 1.0 / n, np.complex128)
    est = 0.0
    for it in range(itmax):
        y = scipy.linalg.lu_solve(lu, x)                      # A^{-1} x, ||x||_1 = 1
        e = float(np.abs(y).sum())
        if it > 0 and e <= est:
            break
        est = e
        ay = np.abs(y)
        xi = np.where(ay > 0, y / np.where(ay > 0, ay, 1.0), 1.0)   # the subgradient of ||.||_1 at y
        z = scipy.linalg.lu_solve(lu, xi, trans=2)            # A^{-H} xi
        j = int(np.argmax(np.abs(z)))
        # stationary: no unit vector improves on the current x
        if it > 0 and np.abs(z[j]) <= np.real(np.vdot(z, x)):
            break
        x = np.zeros(n, np.complex128)
        x[j] = 1.0
    # Higham's extra vector of alternating signs and growing magnitudes
    if n > 1:
        b = np.array([(-1.0) ** i * (1.0 + i / (n - 1)) for i in range(n)], np.complex128)
        est = max(est, 2.0 * float(np.abs(scipy.linalg.lu_solve(lu, b)).sum()) / (3.0 * n))
    return est


def cond1_estimate(A, itmax=5):
    """Estimate of kappa_1(A) = ||A||_1 ||A^{-1}||_1 (a lower bound)."""
    A = np.asarray(A, dtype=np.complex128)
    return float(np.abs(A).sum(axis=0).max()) * norm1_inv_estimate(A, itmax)


def pow2_equilibrate(A):
    """Rows, then columns, scaled by the exact powers of two that bring their
    largest max(|re|, |im|) into [1/2, 1) (zero rows and columns unscaled).
    A is (..., n, n)."""
    A = np.array(A, dtype=np.complex128, copy=True)

    def scale(m):
        with np.errstate(divide="ignore"):
            e = np.floor(np.log2(m))
        return np.where(m > 0, 2.0 ** (-e - 1), 1.0)

    cm = np.maximum(np.abs(A.real), np.abs(A.imag))
    A *= scale(cm.max(axis=-1, keepdims=True))
    cm = np.maximum(np.abs(A.real), np.abs(A.imag))
    A *= scale(cm.max(axis=-2, keepdims=True))
    return A


def lu_pivots(A):
    """The pivots u_jj of Gaussian elimination with partial pivoting on A,
    the pivot of a column being its largest |a|^2 among the remaining rows
    (ties to the lowest row), as the oracle's solve chooses it.  (LAPACK's
    complex LU compares |re| + |im| instead, which can pick other rows.)"""
    U = np.array(A, dtype=np.complex128, copy=True)
    n = U.shape[0]
    piv = np.zeros(n, np.complex128)
    for j in range(n):
        m2 = np.abs(U[j:, j]) ** 2
        p = j + int(np.argmax(m2))          # the first maximum: ties to the lowest row
        U[[j, p]] = U[[p, j]]
        piv[j] = U[j, j]
        if U[j, j] != 0:
            U[j + 1:, j:] -= np.outer(U[j + 1:, j] / U[j, j], U[j, j:])
    return piv


def pivot_ratio(A):
    """max |u_jj| / min |u_jj| of lu_pivots after pow2_equilibrate: the
    library's cheaper condition proxy, restated from its definition."""
    d = np.abs(lu_pivots(pow2_equilibrate(A)))
    return float(d.max() / d.min()) if d.min() > 0 else float("inf")

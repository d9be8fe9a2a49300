"""Seeded synthetic inputs for the polyhedral-homotopy path tracker.

This module only draws random numbers and arranges them into the input
format shared by the CUDA library and by the CPU oracle: exponent supports,
complex coefficients, integer liftings, cell parameters and sample points.
It performs none of the method's arithmetic (no t-exponents, no monomials,
no mixed volumes, no start solutions); where a workload must satisfy such a
condition (for example "mixed volume at least 2"), the caller computes it
and asks for the next ``attempt``.

Workload recipes (shapes and distributions of the paper's Laurent systems,
Section 2, eq. (1); the paper's own test systems are not used):

* ``config1`` -- n=2, 3 monomials/equation, exponents uniform in [-2,2],
  unit-modulus coefficients e^{i theta}, lifting uniform in {0..16}.
* ``config2`` -- n=4, 5 monomials/equation, exponents in [-2,2], lifting
  in {0..64}.
* ``config3`` -- n=16, 32 monomials/equation, every exponent vector has 4
  nonzero coordinates drawn from {+-1,+-2,+-3}, alpha in [-8,8]^16, lifting
  in {0..64}; points y_j = exp(g + i phi), g ~ N(0,1), phi ~ U[0,2pi),
  t ~ U(0,1).
* ``config4`` -- many systems, n in [4,24], monomials/equation in
  [n+1, 4n], exponents in [-3,3], planted cell.
* ``config5`` -- n=8, 12 monomials/equation, exponents in [-2,2], planted
  cell.

A "planted cell" lifting puts lifting value 0 on two chosen monomials of
every equation and a value in {1..delta_hi} on every other monomial; the
chosen pairs then form a mixed cell with inner normal (0, 1) whenever their
difference vectors are linearly independent (checked by the caller).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "LaurentSystem",
    "laurent_system",
    "random_points",
    "torus_points",
    "large_exponent_system",
    "random_alpha",
    "planted_lifting",
    "config1",
    "config2",
    "config3",
    "config4_system",
    "config5",
    "paper_shape",
]


class LaurentSystem:
    """A square Laurent system with lifting (plain container, no arithmetic).

    Attributes
    ----------
    n : int
        number of variables and equations.
    m : list[int]
        support sizes m_k, k = 0..n-1.
    exponents : ndarray int32 (M, n)
        exponent vectors, grouped by equation (rows off[k] .. off[k]+m[k]-1).
    coeffs : ndarray complex128 (M,)
    lifting : ndarray int64 (M,)
    """

    def __init__(self, n, m, exponents, coeffs, lifting):
        self.n = int(n)
        self.m = [int(v) for v in m]
        self.exponents = np.ascontiguousarray(exponents, dtype=np.int32)
        self.coeffs = np.ascontiguousarray(coeffs, dtype=np.complex128)
        self.lifting = np.ascontiguousarray(lifting, dtype=np.int64)
        assert self.exponents.shape == (sum(self.m), self.n)
        assert self.coeffs.shape == (sum(self.m),)
        assert self.lifting.shape == (sum(self.m),)

    @property
    def M(self) -> int:
        return int(sum(self.m))

    @property
    def offsets(self) -> list[int]:
        off, acc = [], 0
        for v in self.m:
            off.append(acc)
            acc += v
        return off

    def support(self, k: int) -> np.ndarray:
        o = self.offsets[k]
        return self.exponents[o:o + self.m[k]]

    def with_coeffs(self, coeffs) -> "LaurentSystem":
        return LaurentSystem(self.n, self.m, self.exponents, coeffs, self.lifting)

    def with_lifting(self, lifting) -> "LaurentSystem":
        return LaurentSystem(self.n, self.m, self.exponents, self.coeffs, lifting)


def _rng(*key) -> np.random.Generator:
    return np.random.default_rng([int(k) & 0xFFFFFFFF for k in key])


def _draw_exponent(rng, n, lo, hi, nnz):
    if nnz is None:
        return rng.integers(lo, hi + 1, size=n)
    vals = np.array([v for v in range(lo, hi + 1) if v != 0])
    a = np.zeros(n, dtype=np.int64)
    idx = rng.choice(n, size=nnz, replace=False)
    a[idx] = rng.choice(vals, size=nnz)
    return a


def laurent_system(seed, n, m, exp_lo, exp_hi, lift_hi, nnz=None, attempt=0):
    """Random Laurent system with distinct exponent vectors in each support.

    ``m`` is an int (same support size for every equation) or a list.
    Coefficients are e^{i theta}, theta ~ U[0, 2 pi); lifting ~ U{0..lift_hi}.
    """
    rng = _rng(seed, attempt, n, 0x5157)
    ms = [int(m)] * n if np.isscalar(m) else [int(v) for v in m]
    rows = []
    for k in range(n):
        seen = set()
        while len(seen) < ms[k]:
            a = _draw_exponent(rng, n, exp_lo, exp_hi, nnz)
            key = tuple(int(v) for v in a)
            if key in seen:
                continue
            seen.add(key)
            rows.append(a)
    M = sum(ms)
    exps = np.array(rows, dtype=np.int32).reshape(M, n)
    theta = rng.uniform(0.0, 2.0 * np.pi, size=M)
    coeffs = np.exp(1j * theta)
    lifting = rng.integers(0, lift_hi + 1, size=M).astype(np.int64)
    return LaurentSystem(n, ms, exps, coeffs, lifting)


def random_points(seed, p, n):
    """Points y in (C*)^n and t in (0,1): y_j = exp(g + i phi), g ~ N(0,1),
    phi ~ U[0, 2 pi), t ~ U(0,1) (t = 0 excluded)."""
    rng = _rng(seed, p, n, 0x9017)
    g = rng.standard_normal((p, n))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=(p, n))
    y = np.exp(g + 1j * phi)
    t = rng.uniform(0.0, 1.0, size=p)
    t = np.where(t <= 0.0, 0.5, t)
    return np.ascontiguousarray(y, dtype=np.complex128), np.ascontiguousarray(t)


def torus_points(seed, p, n, sigma):
    """Points near the unit torus: y_j = exp(g + i phi), g ~ N(0, sigma^2),
    phi ~ U[0, 2 pi), t ~ U(0,1) -- for systems with large exponents, whose
    monomials y^a stay in floating-point range only where |y_j| is near 1."""
    rng = _rng(seed, p, n, 0x7085)
    g = sigma * rng.standard_normal((p, n))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=(p, n))
    y = np.exp(g + 1j * phi)
    t = rng.uniform(0.0, 1.0, size=p)
    t = np.where(t <= 0.0, 0.5, t)
    return np.ascontiguousarray(y, dtype=np.complex128), np.ascontiguousarray(t)


def large_exponent_system(seed, n, m, n_big, big_lo, big_hi, lift_hi=64, attempt=0):
    """A Laurent system whose equations each have n_big monomials with large
    exponents (min(4, n) nonzero coordinates of magnitude in [big_lo,
    big_hi], random signs) beside m - n_big monomials with exponents in
    [-2, 2]; coefficients e^{i theta}, lifting U{0..lift_hi}."""
    rng = _rng(seed, attempt, n, 0xB16E)
    rows = []
    for k in range(n):
        seen = set()
        while len(seen) < m:
            big = len(seen) >= m - n_big
            if big:
                a = np.zeros(n, dtype=np.int64)
                idx = rng.choice(n, size=min(4, n), replace=False)
                a[idx] = rng.integers(big_lo, big_hi + 1, size=len(idx)) * rng.choice([-1, 1], size=len(idx))
            else:
                a = rng.integers(-2, 3, size=n)
            key = tuple(int(v) for v in a)
            if key in seen:
                continue
            seen.add(key)
            rows.append(a)
    M = n * m
    exps = np.array(rows, dtype=np.int32).reshape(M, n)
    coeffs = np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, size=M))
    lifting = rng.integers(0, lift_hi + 1, size=M).astype(np.int64)
    return LaurentSystem(n, [m] * n, exps, coeffs, lifting)


def random_alpha(seed, n, lo=-8, hi=8):
    """Integer cell normal alpha in [lo, hi]^n."""
    rng = _rng(seed, n, 0xA1FA)
    return rng.integers(lo, hi + 1, size=n).astype(np.int64)


def planted_lifting(seed, m, delta_hi, attempt=0):
    """Lifting with value 0 on a random pair of each support and a value in
    {1..delta_hi} elsewhere.  Returns (lifting (M,), pairs (n, 2) local
    indices)."""
    rng = _rng(seed, attempt, len(m), 0x91A7)
    lift, pairs = [], []
    for mk in m:
        pr = np.sort(rng.choice(mk, size=2, replace=False))
        w = rng.integers(1, delta_hi + 1, size=mk)
        w[pr] = 0
        lift.append(w)
        pairs.append(pr)
    return (np.concatenate(lift).astype(np.int64),
            np.array(pairs, dtype=np.int32))


def config1(attempt=0):
    """n=2 tracking workload (seed 0)."""
    return laurent_system(0, 2, 3, -2, 2, 16, attempt=attempt)


def config2(attempt=0):
    """n=4 tracking workload (seed 0)."""
    return laurent_system(0, 4, 5, -2, 2, 64, attempt=attempt)


def config3(n=16, m=32):
    """Throughput workload: system (seed 0) and alpha; points come from
    ``random_points(1, p, n)``."""
    sysm = laurent_system(0, n, m, -3, 3, 64, nnz=min(4, n))
    alpha = random_alpha(0, n)
    return sysm, alpha


def config4_system(index, attempt=0):
    """One system of the many-systems workload: n ~ U{4..24},
    m_k ~ U{n+1..4n}, exponents in [-3,3], planted-cell lifting."""
    rng = _rng(4, index, attempt, 0xC04)
    n = int(rng.integers(4, 25))
    m = [int(v) for v in rng.integers(n + 1, 4 * n + 1, size=n)]
    sysm = laurent_system(1000 + index, n, m, -3, 3, 0, attempt=attempt)
    lift, pairs = planted_lifting(2000 + index, m, 16, attempt=attempt)
    return sysm.with_lifting(lift), pairs


def paper_shape(n, total_m, attempt=0):
    """A stand-in of the paper's test-system shapes (Section 8, Tables 1-2:
    n equations and `total_m` monomials in all, about total_m / n per
    equation, no monomial shared between equations): exponents in [-2,2]
    with 4 nonzeros, coefficients e^{i theta}, planted-cell lifting.
    Returns (system, pairs)."""
    m = [total_m // n + (1 if k < total_m % n else 0) for k in range(n)]
    sysm = laurent_system(7000 + n, n, m, -2, 2, 0, nnz=min(4, n), attempt=attempt)
    lift, pairs = planted_lifting(7100 + n, m, 16, attempt=attempt)
    return sysm.with_lifting(lift), pairs


def config5(attempt=0):
    """Adjoint workload: n=8, 12 monomials/equation, exponents in [-2,2],
    planted-cell lifting."""
    sysm = laurent_system(5, 8, 12, -2, 2, 0, attempt=attempt)
    lift, pairs = planted_lifting(5, sysm.m, 16, attempt=attempt)
    return sysm.with_lifting(lift), pairs

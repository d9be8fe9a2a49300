"""Pins of the oracle's 1-norm condition estimate (Hager 1984, Higham 1988;
CPU only), against numpy.linalg.cond(A, 1):
* it never exceeds the exact kappa_1 (it is a lower bound);
* it is exact on diagonal matrices (the first solve finds the largest 1/|d|);
* on random complex matrices, and on matrices scaled towards singularity, it
  is within a factor 3 of kappa_1 on at least 95% of them and its median ratio
  is at least 0.9;
* two planted slips (a start vector of the wrong 1-norm, the infinity norm of
  A for its 1-norm) break these pins.
"""
import numpy as np
import pytest

from oracle import condest


def _rand(rng, n):
    return rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16])
def test_lower_bound_and_close(n):
    rng = np.random.default_rng(100 + n)
    ratios = []
    for q in range(300):
        A = _rand(rng, n)
        if q % 3 == 1:   # graded columns
            A = A * np.logspace(0, rng.uniform(0, 8), n)[None, :]
        elif q % 3 == 2:   # near a singular matrix
            u, s, vh = np.linalg.svd(A)
            s[-1] = s[0] * 10.0 ** -rng.uniform(2, 10)
            A = (u * s) @ vh
        k = np.linalg.cond(A, 1)
        e = condest.cond1_estimate(A)
        assert e <= k * (1 + 1e-10), (e, k)
        ratios.append(e / k)
    ratios = np.array(ratios)
    assert (ratios >= 1 / 3).mean() >= 0.95, np.quantile(ratios, [0.01, 0.05, 0.5])
    assert np.median(ratios) >= 0.9


def test_exact_on_diagonal():
    rng = np.random.default_rng(7)
    for n in (1, 3, 16):
        d = np.exp(rng.uniform(-5, 5, n)) * np.exp(2j * np.pi * rng.uniform(size=n))
        A = np.diag(d)
        assert condest.cond1_estimate(A) == pytest.approx(np.abs(d).max() / np.abs(d).min(), rel=1e-12)


def _pins_hold(est):
    rng = np.random.default_rng(5)
    ratios = []
    for q in range(200):
        A = _rand(rng, 8)
        if q % 2:
            A = A * np.logspace(0, 6, 8)[None, :]
        k = np.linalg.cond(A, 1)
        e = est(A)
        if e > k * (1 + 1e-10):
            return False
        ratios.append(e / k)
    ratios = np.array(ratios)
    return (ratios >= 1 / 3).mean() >= 0.95 and np.median(ratios) >= 0.9


def test_pins_reject_planted_mistakes():
    """Two plausible slips each break a pin: a start vector of 1-norm n
    instead of 1 (overestimates by n), and the infinity norm (row sums) of A
    in place of its 1-norm."""
    assert _pins_hold(condest.cond1_estimate)
    assert not _pins_hold(lambda A: A.shape[0] * condest.cond1_estimate(A))
    assert not _pins_hold(lambda A: float(np.abs(A).sum(axis=1).max()) * condest.norm1_inv_estimate(A))


def test_pow2_equilibration_and_pivot_ratio_definitions():
    rng = np.random.default_rng(11)
    A = _rand(rng, 6) * np.logspace(-3, 5, 6)[:, None] * np.logspace(2, -4, 6)[None, :]
    E = condest.pow2_equilibrate(A)
    cm = np.maximum(np.abs(E.real), np.abs(E.imag))
    assert np.all(cm.max(axis=0) >= 0.5) and np.all(cm.max(axis=0) < 1.0)
    assert np.all(cm.max(axis=1) < 1.0)
    ratio = E / A   # a rank-one array of powers of two
    lg = np.log2(np.abs(ratio))
    assert np.allclose(lg, np.round(lg), atol=0) and np.allclose(np.angle(ratio), 0)
    # a diagonal matrix equilibrates to entries in [1/2, 1): its pivot ratio is
    # the ratio of its largest to smallest equilibrated entry, below 2
    d = np.exp(rng.uniform(-5, 5, 5))
    m = d * 2.0 ** (-np.floor(np.log2(d)) - 1)
    assert condest.pivot_ratio(np.diag(d)) == pytest.approx(m.max() / m.min()) and m.max() / m.min() < 2


def test_pivot_ratio_calibration_on_the_throughput_workload():
    """The library's FP32 solve re-solves in FP64 the paths whose pivot ratio
    exceeds params.cond_max.  On 4,000 random points of the n = 16 throughput
    workload (the oracle's D_z H = H_y diag(y)) kappa_1 / pivot ratio has a
    median between 10 and 100 (about 33) and never exceeds 1,000 (the largest
    of 20,000 points measured was 539): the default cond_max of 3e4 flags
    the typical path whose kappa_1 exceeds 1e6, and every one above 3e7."""
    import workloads as W
    import oracle
    from oracle import cells
    sysm, alpha = W.config3(16, 32)
    cell = {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 1}
    te = cells.t_exponents(sysm, cell)
    osys = oracle.System(sysm, te["e"], te["D"])
    y, t = W.random_points(23, 4000, 16)
    _, Hy, _ = osys.eval(y, np.log(t))
    A = condest.pow2_equilibrate(Hy * y[:, None, :])
    f = np.array([condest.cond1_estimate(a) / condest.pivot_ratio(a) for a in A])
    assert 10 <= np.median(f) <= 100 and f.max() <= 1000, (np.median(f), f.max())

"""Shared helpers of the test suite (inputs and comparisons only)."""
import numpy as np

import workloads as W
from oracle import cells


def first_generic(cfg, min_mv=2):
    """First attempt of a workload whose lifting is generic and whose mixed
    volume is at least min_mv: (system, cells, mixed volume)."""
    for att in range(60):
        s = cfg(att)
        try:
            cl, mv = cells.mixed_cells(s)
        except cells.NonGeneric:
            continue
        if mv >= min_mv:
            return s, cl, mv
    raise RuntimeError("no generic sample")


def min_separation(y):
    """Smallest Euclidean distance between two rows of a complex point set
    (k-d tree over the real coordinates, O(N log N) memory-light)."""
    from scipy.spatial import cKDTree
    pts = np.concatenate([np.real(y), np.imag(y)], axis=1)
    d, _ = cKDTree(pts).query(pts, k=2)
    return float(d[:, 1].min())


def scaled_err(got, ref, scale):
    return float(np.max(np.abs(np.asarray(got) - ref) / np.maximum(scale, 1e-300)))


def match_solutions(a, b):
    """Greedy one-to-one nearest matching of two solution sets (rows); returns
    the largest relative distance max|a_i - b_j| / max(1, |b_j|)."""
    a = np.asarray(a)
    b = np.asarray(b)
    assert a.shape == b.shape
    d = np.abs(a[:, None, :] - b[None, :, :]).max(-1) / np.maximum(1.0, np.abs(b).max(-1))[None, :]
    used = np.zeros(len(b), bool)
    worst = 0.0
    for i in np.argsort(d.min(1)):
        cand = np.where(used, np.inf, d[i])
        j = int(np.argmin(cand))
        used[j] = True
        worst = max(worst, float(cand[j]))
    return worst


def eval_case(name):
    """(system, cell dict) for the evaluation parity cases."""
    if name == "n2":
        s, cl, _ = first_generic(W.config1)
        return s, {"kind": "pairs", "pairs": cl[0]["pairs"]}
    if name == "n4":
        s, cl, _ = first_generic(W.config2)
        return s, {"kind": "pairs", "pairs": cl[-1]["pairs"]}
    if name == "n16":
        s, alpha = W.config3(16, 32)
        return s, {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 1}
    if name == "n7_ragged":
        s = W.laurent_system(11, 7, [5, 9, 17, 3, 12, 8, 20], -3, 3, 40)
        alpha = W.random_alpha(3, 7, -4, 4)
        return s, {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 3}
    if name == "n24":
        rng = np.random.default_rng(24)
        m = [int(v) for v in rng.integers(25, 97, size=24)]
        s = W.laurent_system(24, 24, m, -2, 2, 16)
        alpha = W.random_alpha(24, 24, -2, 2)
        return s, {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 1}
    raise KeyError(name)


def planted_case(cfg, min_det, max_det=400000):
    """First attempt of a planted-cell workload whose pair matrix has
    min_det <= |det V| <= max_det and passes the cell test:
    (system, pairs, t-exponent dict, |det V|)."""
    for att in range(200):
        s, pairs = cfg(att)
        d = abs(cells.det_int(cells.pair_matrix(s, pairs)))
        if not (min_det <= d <= max_det):
            continue
        try:
            te = cells.t_exponents(s, {"kind": "pairs", "pairs": pairs})
        except (cells.NotACell, cells.NonGeneric):
            continue
        return s, pairs, te, d
    raise RuntimeError("no planted cell found")

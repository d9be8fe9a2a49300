"""The batching form (many systems in one tracker) on the GPU (GPU).

* Same results as tracking each system alone: systems whose sizes share one
  lane-group shape give bit-identical solutions, statuses and step counts
  to hpt_track per system (the batch runs the same per-path arithmetic);
  mixed shapes agree after the FP64 polish.
* Parity with the oracle's tracker on sampled paths of the many-systems
  workload (n up to 24): endpoints within relative 1e-9.
* Edge cases: a system with no paths, one path, ragged tiles (127, 129),
  the autotuner's candidates, tuning bounds, and an FP64 handle refused.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cells

pytestmark = pytest.mark.gpu


def _systems(hpt, indices):
    out = []
    for idx in indices:
        s, pairs = W.config4_system(idx)
        cell = {"kind": "pairs", "pairs": pairs}
        out.append((s, pairs, hpt.System.from_laurent(s, cell, hpt.HPT_MIXED)))
    return out


def _starts(s, pairs, p):
    """p start points y = exp(V^-1 (log b + 2 pi i j e_1)), j = 0..p-1 (oracle)."""
    ks = np.zeros((p, s.n), np.int64)
    ks[:, 0] = np.arange(p)
    return cells.start_points_at(s, pairs, ks)


def _indices(lo, hi, count):
    """The first `count` workload systems with lo <= n <= hi."""
    out = []
    for idx in range(400):
        s, _ = W.config4_system(idx)
        if lo <= s.n <= hi:
            out.append(idx)
            if len(out) == count:
                return out
    raise RuntimeError("not enough systems")


def _run_batch(hpt, systems, paths, prm):
    y0 = [_starts(s, pr, p) for (s, pr, _), p in zip(systems, paths)]
    flat = np.concatenate([y.reshape(-1) for y in y0]) if sum(paths) else np.zeros(0, np.complex128)
    b = hpt.Batch([h for _, _, h in systems])
    x, st, sp = b.track(torch.from_numpy(flat).cuda(), paths, prm)
    return b, y0, x.cpu().numpy(), st.cpu().numpy(), sp.cpu().numpy()


def _track_by_steps(hpt, h, y0, prm):
    """The paths of one system stepped together with hpt_step until none is
    active, then the FP64 polish of the converged ones (hpt_polish): a track
    without the batch machinery (no compaction, no graph)."""
    p, n = y0.shape
    st = hpt.PathState(p, n, hpt.HPT_MIXED)
    h.paths_init(st, torch.from_numpy(np.ascontiguousarray(y0)).cuda(), prm)
    done = 0
    while done <= prm.max_steps + 32:
        h.step(st, 32, prm)
        done += 32
        if int((st.status == hpt.ACTIVE).sum().item()) == 0:
            break
    x = st.y_acc.to(torch.complex128)
    h.polish(x, st.status, prm)
    return x.cpu().numpy(), st.status.cpu().numpy(), st.steps.cpu().numpy()


def _split(systems, paths, x, st, sp):
    out, vo, po = [], 0, 0
    for (s, _, _), p in zip(systems, paths):
        out.append((x[vo:vo + p * s.n].reshape(p, s.n), st[po:po + p], sp[po:po + p]))
        vo += p * s.n
        po += p
    return out


def test_batch_equals_per_system_track_one_shape(hpt):
    """n in [9, 16] (one solve shape): bit-identical to stepping each system's
    paths with hpt_step and polishing them (no batch machinery), and to
    hpt_track (which runs as a one-system batch)."""
    systems = _systems(hpt, _indices(9, 16, 5))
    paths = [130, 0, 127, 1, 256]
    prm = hpt.Params(tol_accept=3e-3)
    b, y0, x, st, sp = _run_batch(hpt, systems, paths, prm)
    for (s, pr, h), p, y, (xb, stb, spb) in zip(systems, paths, y0, _split(systems, paths, x, st, sp)):
        if p == 0:
            continue
        xs, sts, sps = _track_by_steps(hpt, h, y, prm)
        assert np.array_equal(stb, sts)
        assert np.array_equal(spb, sps)
        assert np.array_equal(xb, xs)
        xt, stt, spt = h.track(torch.from_numpy(y).cuda(), prm)
        assert np.array_equal(xb, xt.cpu().numpy()) and np.array_equal(stb, stt.cpu().numpy())
    st_all = st
    assert (st_all == hpt.CONVERGED).mean() > 0.9, np.bincount(st_all)
    r = b.stats()
    assert r["rounds"] >= 1 and r["kernels_per_round"] > 0


def test_batch_mixed_shapes_match_per_system(hpt):
    """n from 4 to 24 (three solve shapes): statuses and polished solutions
    agree with hpt_track per system."""
    idx = _indices(4, 8, 2) + _indices(9, 16, 2) + _indices(17, 24, 2)
    systems = _systems(hpt, idx)
    paths = [64, 200, 96, 33, 128, 70]
    prm = hpt.Params(tol_accept=3e-3)
    _, y0, x, st, sp = _run_batch(hpt, systems, paths, prm)
    same_status = total = 0
    for (s, pr, h), p, y, (xb, stb, spb) in zip(systems, paths, y0, _split(systems, paths, x, st, sp)):
        xs, sts, _ = h.track(torch.from_numpy(y).cuda(), prm)
        xs, sts = xs.cpu().numpy(), sts.cpu().numpy()
        same_status += int((stb == sts).sum())
        total += p
        both = (stb == hpt.CONVERGED) & (sts == hpt.CONVERGED)
        if both.any():
            rel = np.abs(xb[both] - xs[both]).max(-1) / np.maximum(1.0, np.abs(xs[both]).max(-1))
            assert rel.max() < 1e-9, (s.n, rel.max())
    assert same_status >= total - 2


def test_batch_matches_oracle_on_sampled_paths(hpt, oracle_mod):
    """Endpoints of sampled paths of the many-systems workload (one system of
    each size band, 64 paths each) agree with the oracle's tracker."""
    idx = _indices(4, 8, 1) + _indices(9, 16, 1) + _indices(17, 24, 1)
    systems = _systems(hpt, idx)
    paths = [64] * len(systems)
    prm = hpt.Params(tol_accept=3e-3)
    _, y0, x, st, _ = _run_batch(hpt, systems, paths, prm)
    P = oracle_mod.Params()
    checked = mismatched = 0
    for (s, pr, _), y, (xb, stb, _) in zip(systems, y0, _split(systems, paths, x, st, st)):
        te = cells.t_exponents(s, {"kind": "pairs", "pairs": pr})
        osys = oracle_mod.System(s, te["e"], te["D"])
        sample = np.arange(0, 64, 8)
        xo, sto, _, _ = osys.track(P, y[sample], cells.tau0(te["e"], te["D"]))
        for i, q in enumerate(sample):
            if sto[i] != oracle_mod.CONVERGED or stb[q] != hpt.CONVERGED:
                continue
            checked += 1
            rel = np.abs(xb[q] - xo[i]).max() / max(1.0, np.abs(xo[i]).max())
            mismatched += rel > 1e-9
    assert checked >= 18
    assert mismatched <= 1


def test_batch_autotune_and_tuning(hpt):
    systems = _systems(hpt, _indices(4, 12, 3))
    paths = [100, 60, 140]
    y0 = np.concatenate([_starts(s, pr, p).reshape(-1) for (s, pr, _), p in zip(systems, paths)])
    b = hpt.Batch([h for _, _, h in systems])
    best, ms = b.autotune(torch.from_numpy(y0).cuda(), paths, hpt.Params(tol_accept=3e-3))
    assert best in ms and len(ms) >= 5
    assert b.tuning == best
    b.tuning = (8, 1, 32)
    assert b.tuning == (8, 1, 32)
    with pytest.raises(hpt.HptError):
        b.tuning = (0, 1, 8)
    with pytest.raises(hpt.HptError):
        b.tuning = (8, 3, 8)
    with pytest.raises(hpt.HptError):
        b.tuning = (8, 1, 16)


def test_batch_solve_shapes_agree(hpt):
    """Systems with 17 <= n <= 24 solved by 8-lane x 3-row and by 32-lane
    groups: same statuses, solutions within 1e-9 after polish."""
    systems = _systems(hpt, _indices(17, 24, 3))
    paths = [96, 130, 64]
    y0 = np.concatenate([_starts(s, pr, p).reshape(-1) for (s, pr, _), p in zip(systems, paths)])
    b = hpt.Batch([h for _, _, h in systems])
    prm = hpt.Params(tol_accept=3e-3)
    out = {}
    for lanes in (8, 32):
        b.tuning = (8, 1, lanes)
        x, st, _ = b.track(torch.from_numpy(y0).cuda(), paths, prm)
        out[lanes] = (x.cpu().numpy(), st.cpu().numpy())
    (x8, s8), (x32, s32) = out[8], out[32]
    assert (s8 == s32).mean() > 0.98
    both = np.repeat((s8 == hpt.CONVERGED) & (s32 == hpt.CONVERGED),
                     [s.n for (s, _, _), p in zip(systems, paths) for _ in range(p)])
    rel = np.abs(x8[both] - x32[both]) / np.maximum(1.0, np.abs(x32[both]))
    assert rel.max() < 1e-9


def test_batch_refuses_fp64_handles(hpt):
    s, pairs = W.config4_system(0)
    h = hpt.System.from_laurent(s, {"kind": "pairs", "pairs": pairs}, hpt.HPT_FP64)
    with pytest.raises(hpt.HptError) as ei:
        hpt.Batch([h])
    assert ei.value.code == 7


def test_batch_fp64_resolve_everything(hpt):
    """Every FP32 solve of a mixed-shape batch redone in FP64 (cond_max = 1,
    the warp solves with its largest n, identity rows pad smaller systems):
    the polished solutions equal those of the FP32 solves."""
    idx = _indices(4, 8, 1) + _indices(9, 16, 1) + _indices(17, 24, 1)
    systems = _systems(hpt, idx)
    paths = [64, 64, 64]
    _, _, x1, st1, _ = _run_batch(hpt, systems, paths, hpt.Params(tol_accept=3e-3, cond_max=1.0))
    _, _, x2, st2, _ = _run_batch(hpt, systems, paths, hpt.Params(tol_accept=3e-3))
    assert (st1 == st2).mean() > 0.97
    for (s, _, _), (xa, sa, _), (xb, sb, _) in zip(systems, _split(systems, paths, x1, st1, st1),
                                                    _split(systems, paths, x2, st2, st2)):
        both = (sa == hpt.CONVERGED) & (sb == hpt.CONVERGED)
        rel = np.abs(xa[both] - xb[both]).max(-1) / np.maximum(1.0, np.abs(xb[both]).max(-1))
        assert (rel < 1e-9).mean() > 0.97, (s.n, np.sort(rel)[-5:])

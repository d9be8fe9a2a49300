#!/usr/bin/env python3
"""Benchmark: Euler+Newton path-steps/s of hpt_step at n=16, 65,536 paths.

One "step" is one hpt_step call with nsteps=1 over all 65,536 paths of the
throughput workload (random Laurent system, n=16, 32 monomials/equation,
4 nonzero exponents in [-3,3] per monomial, alpha in [-8,8]^16, lifting in
{0..64}, beta the lower envelope; points y_j = exp(g + i phi), g ~ N(0,1),
phi ~ U[0,2pi), t ~ U(0,1)): evaluation of H, H_y, H_tau (log, exponent
GEMM, complex exp, coefficient GEMM, diag(1/y) scaling), the consolidated
Euler+Newton LU solve and the step control, for every path.  The state is
restored before every timed step (so every step does the same work on all
paths) and L2 is flushed by a 256 MiB write between timed steps.

The headline value is the mixed split-BF16/FP32 tensor-core form; the plain
FP64 form is measured in the same run.  --impl reference times the CPU
oracle (complex128, OpenMP over paths) on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_VARS, M_PER_EQ, PATHS = 16, 32, 65536
WORKLOAD = ("random Laurent system n=16, 32 monomials/equation (M=512), 4 nonzero exponents "
            "in [-3,3] per monomial, alpha in [-8,8]^16, lifting {0..64}; 65,536 paths; one "
            "hpt_step (evaluate + consolidated Euler/Newton solve + step control) per step")
METRIC = "Euler+Newton steps/s at n=16, 64K paths: mixed vs FP64 form, % of roofline"
UNIT = "path-steps/s"

# algorithmic work per path-step (dense within each equation's block)
FLOP_EXP_GEMM = 2 * (2 * N_VARS + 1) * N_VARS * M_PER_EQ          # 33,792
FLOP_COEF_GEMM = 8 * (N_VARS + 2) * N_VARS * M_PER_EQ             # 73,728
CEXP = N_VARS * M_PER_EQ                                           # 512
n = N_VARS
FLOP_LU = 8 * (n - 1) * n * (2 * n - 1) // 6 + 6 * n * (n - 1) // 2   # 10,640
FLOP_SOLVE = 16 * n * n + 16 * n                                     # 4,352
# path state read and written by a step (mixed form, complex64): y, y_acc,
# dE_acc (n complex each), tau, dtau, tau_acc (FP64), five int32 counters
STATE_BYTES = 2 * (3 * N_VARS * 8 + 3 * 8 + 5 * 4)                  # 856
# MUFU issue slots per SM and clock (derived): ex2 32 (the doubled
# special-function rate of this part), sin and cos 16 each
MUFU_EX2_PER_CLK, MUFU_SINCOS_PER_CLK, FP32_LANES = 32, 16, 128


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_seed(rank: int) -> int:
    """Weak scaling: every rank tracks its own 65,536 paths (seed 1 + rank)."""
    return 1 + rank


def max_over_ranks(value: float, device) -> float:
    """The largest of every rank's value (the slowest rank's time); the value
    itself without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, seconds: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank / seconds


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._proc = None

    def __enter__(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self._proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self._proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        time.sleep(0.2)
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _workload():
    import workloads as W
    sysm, alpha = W.config3(N_VARS, M_PER_EQ)
    cell = {"kind": "lower", "alpha_num": alpha.tolist(), "denom": 1}
    return sysm, cell


def _traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, valid only while
    the kernel's source is unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    srcs = rec["source"] if isinstance(rec["source"], list) else [rec["source"]]
    h = hashlib.sha256()
    for f in srcs:
        h.update(open(os.path.join(ROOT, "paper_2111_14317_gb300", "csrc", f), "rb").read())
    if h.hexdigest()[:16] != rec["source_sha"]:
        return None
    return rec["bytes_per_launch_full"]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2111_14317_gb300 import build as hbuild
    hbuild.build()
    from paper_2111_14317_gb300 import hpt
    import workloads as W

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    sysm, cell = _workload()
    y_np, t_np = W.random_points(shard_seed(rank), PATHS, N_VARS)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = {}
    for form, prec in (("mixed", hpt.HPT_MIXED), ("fp64", hpt.HPT_FP64)):
        h = hpt.System.from_laurent(sysm, cell, prec)
        prm = hpt.Params(tol_accept=3e-3 if prec == hpt.HPT_MIXED else 1e-3)
        st = hpt.PathState(PATHS, N_VARS, prec, device=dev)
        yd = torch.from_numpy(y_np).to(dev, h.cdtype)
        st.y.copy_(yd)
        st.y_acc.copy_(yd)
        st.tau.copy_(torch.from_numpy(np.log(t_np)))
        st.tau_acc.copy_(st.tau)
        st.dtau.fill_(0.01)
        st.accepts.fill_(1)
        pristine = {k: v.clone() for k, v in st.to_host().items()}
        pristine_dev = {k: v.to(dev) for k, v in pristine.items()}

        def restore():
            for k, v in pristine_dev.items():
                getattr(st, k).copy_(v)

        steps = args.steps if form == "mixed" else max(3, min(args.steps, args.fp64_steps))
        for _ in range(args.warmup):
            restore()
            h.step(st, 1, prm)
        torch.cuda.synchronize()

        def timed(profile):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            h.profile(profile)
            if ws > 1:
                dist.barrier()
            torch.cuda.synchronize()
            for i in range(steps):
                restore()
                flush.zero_()
                ev[i][0].record()
                h.step(st, 1, prm)
                ev[i][1].record()
            torch.cuda.synchronize()
            if ws > 1:
                dist.barrier()
            h.profile(False)
            return [a.elapsed_time(b) for a, b in ev]

        # headline pass (no per-kernel events), clocks sampled meanwhile
        with ClockSampler(local) as clk:
            ms = timed(False)
        tot = max_over_ranks(sum(ms), dev)
        # second pass: CUDA events around every kernel on the launching stream
        timed(True)
        kern = h.profile_read()
        # end-to-end through the C ABI: every step copies the whole state (one
        # contiguous arena) from pinned host memory to the device, steps it and
        # copies it back.  Three device states rotate, with the copies in on
        # one stream, the steps on another and the copies out on a third, so
        # step i runs while step i+1's input arrives and step i-1's result
        # leaves, and a state's copy out and next copy in have two steps'
        # time (each direction is ordered against the others by events).
        e2e_steps = max(6, steps // 2)
        NB = 3
        hin = [hpt.PathState(PATHS, N_VARS, prec, device="cpu", pin=True) for _ in range(NB)]
        hout = [hpt.PathState(PATHS, N_VARS, prec, device="cpu", pin=True) for _ in range(NB)]
        for hh in hin:
            hh.load(pristine)
        dev2 = [st] + [hpt.PathState(PATHS, N_VARS, prec, device=dev) for _ in range(NB - 1)]
        h2d = hin[0].arena.numel()
        s_in, s_run, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(NB)]
        ev_run = [torch.cuda.Event() for _ in range(NB)]
        ev_out = [torch.cuda.Event() for _ in range(NB)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            b = i % NB
            with torch.cuda.stream(s_in):
                if i >= NB:
                    s_in.wait_event(ev_out[b])          # step i-NB's result has left dev2[b]
                dev2[b].arena.copy_(hin[b].arena, non_blocking=True)
                ev_in[b].record(s_in)
            s_run.wait_event(ev_in[b])
            h.step(dev2[b], 1, prm, stream=s_run)
            ev_run[b].record(s_run)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_run[b])
                hout[b].arena.copy_(dev2[b].arena, non_blocking=True)
                ev_out[b].record(s_out)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        out[form] = dict(steps=steps, ms_per_step=tot / steps, ms_list=ms, kernels=kern,
                         clocks=clk.summary(), e2e_s=e2e_s, h2d=h2d, d2h=h2d,
                         launches=sum(v[0] for v in kern.values()))
        assert h.device_error() == 0, "device-side wait timed out"
        h.close()
        del st, pristine_dev
        torch.cuda.empty_cache()
    if args.batch_systems > 0:
        out["batch"] = run_batch(args, dev)
    out["sms"] = torch.cuda.get_device_properties(dev).multi_processor_count
    if args.workload == "all":
        out["track_adjoint"] = run_track_adjoint(args, dev)
        out["projective"] = run_projective(args, dev)
        out["paper_shapes"] = run_paper_shapes(args, dev)
        out["start_points"] = run_start_points(args, dev)
        out["step100"] = run_step100(args, dev)
    if ws > 1:
        dist.destroy_process_group()
    return out, ws, rank


BATCH_WORKLOAD = ("many-systems batch: 256 random Laurent systems, n ~ U{4..24}, m_k ~ U{n+1..4n}, "
                  "exponents in [-3,3], coefficients e^{i theta}, planted pair cell (lifting 0 on one pair "
                  "per support, U{1..16} elsewhere); 512 paths per system from the start points "
                  "exp(V^-1 (log b + 2 pi i j e_1)), j < 512; tracked t: 0 -> 1 and polished")


def run_batch(args, dev):
    """The batching form on the many-systems workload: autotune, then time
    whole hpt_batch_track calls (device-resident start points) and one
    end-to-end call with the start points copied from pinned host memory and
    the solutions copied back inside the timed region."""
    import torch
    from paper_2111_14317_gb300 import hpt
    import workloads as W
    nsys, npaths = args.batch_systems, args.batch_paths
    t0 = time.perf_counter()
    systems, y0s, gemm_flop = [], [], []
    for idx in range(nsys):
        s, pairs = W.config4_system(idx)
        M = int(sum(s.m))
        gemm_flop.append(2 * (2 * s.n + 1) * M + 8 * (s.n + 2) * M)   # per path-step, as for n=16
        systems.append(hpt.System.from_laurent(s, {"kind": "pairs", "pairs": pairs}, hpt.HPT_MIXED))
        ks = np.zeros((npaths, s.n), np.int64)
        ks[:, 0] = np.arange(npaths)
        y0s.append(hpt.binomial_points(s.n, s.m, s.exponents, s.coeffs, pairs, ks).reshape(-1))
    setup_s = time.perf_counter() - t0
    paths = [npaths] * nsys
    y0_host = torch.from_numpy(np.concatenate(y0s))
    y0 = y0_host.to(dev)
    b = hpt.Batch(systems)
    prm = hpt.Params(tol_accept=3e-3)
    if args.no_autotune:
        best, cand = b.tuning, {}
    else:
        best, cand = b.autotune(y0, paths, prm)
    for _ in range(max(1, min(args.warmup, 2))):
        b.track(y0, paths, prm)
    reps = max(1, args.batch_reps)
    with ClockSampler(dev.index or 0) as clk:
        ms = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, st, sp = b.track(y0, paths, prm)
            torch.cuda.synchronize()
            ms.append((time.perf_counter() - t0) * 1e3)
    stats = b.stats()
    # the same track with the cubic Hermite predictor at tol_accept 1e-3 (the
    # tolerance the predictor is used with), and the Euler predictor at 1e-3
    # for a like-for-like step count
    pred = {}
    for name, kw in (() if args.skip_predictors else
                     (("euler_tol1e-3", dict(predictor=0)), ("hermite_tol1e-3", dict(predictor=1)))):
        prm_p = hpt.Params(tol_accept=1e-3, **kw)
        b.track(y0, paths, prm_p)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st_p, sp_p = b.track(y0, paths, prm_p)
        torch.cuda.synchronize()
        ms_p = (time.perf_counter() - t0) * 1e3
        st_n_p, sp_n_p = st_p.cpu().numpy(), sp_p.cpu().numpy()
        pred[name] = {"ms_per_track": ms_p, "path_steps": int(sp_n_p.sum()),
                      "converged": int((st_n_p == hpt.CONVERGED).sum()),
                      "paths_per_s": nsys * npaths / (ms_p * 1e-3)}
    # end to end: pinned host start points in, solutions and statuses out
    pinned = y0_host.pin_memory()
    x_host = torch.empty_like(y0_host).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    yd = pinned.to(dev, non_blocking=True)
    x, st, sp = b.track(yd, paths, prm)
    x_host.copy_(x, non_blocking=True)
    st_h = st.cpu()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3
    sp_h = sp.cpu().numpy()
    st_n = st_h.numpy()
    total_steps = int(sp_h.sum())
    t_ms = statistics.median(ms)
    conv = sp_h[st_n == hpt.CONVERGED]
    # algorithmic GEMM work of every path-step taken, over the whole track time
    steps_per_sys = sp_h.reshape(nsys, npaths).sum(axis=1)
    flop = float(np.dot(steps_per_sys, np.array(gemm_flop, dtype=np.float64)))
    peaks, peak_kind = _peaks()
    ach = flop / (t_ms * 1e-3) / 1e12
    out = {
        "workload": BATCH_WORKLOAD, "systems": nsys, "paths": nsys * npaths,
        "ms_per_track": t_ms, "ms_list": ms,
        "value": total_steps / (t_ms * 1e-3), "unit": "path-steps/s",
        "paths_per_s": nsys * npaths / (t_ms * 1e-3),
        "e2e": {"ms_per_track": e2e_ms, "value": total_steps / (e2e_ms * 1e-3), "unit": "path-steps/s",
                "h2d_bytes": int(y0_host.numel() * 16), "d2h_bytes": int(y0_host.numel() * 16 + st_n.size * 4)},
        "path_steps": total_steps, "position_steps": stats["position_steps"],
        "lane_efficiency": total_steps / max(stats["position_steps"], 1),
        "rounds": stats["rounds"], "kernels_per_round": stats["kernels_per_round"],
        "gpu_launches_rounds": stats["rounds"] * stats["kernels_per_round"],
        "tuning": {"steps_per_round": best[0], "eval_ctas_per_sm": best[1], "solve_lanes_n17_24": best[2],
                   "candidates_ms": {f"K={k},ctas={c},lanes={ln}": v for (k, c, ln), v in cand.items()}},
        "status_counts": {int(k): int(v) for k, v in zip(*np.unique(st_n, return_counts=True))},
        "steps_per_path": {"min": int(conv.min()) if conv.size else None,
                           "median": float(np.median(conv)) if conv.size else None,
                           "max": int(conv.max()) if conv.size else None},
        "predictors": pred,
        "setup_s": setup_s, "clocks": clk.summary(),
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops_sustained"],
                     "unit": "TFLOP/s", "frac": ach / peaks["bf16_tflops_sustained"],
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json, sustained)",
                     "note": "algorithmic exponent + coefficient GEMM flops of all path-steps over the whole "
                             "track time (evaluation, solves, compaction and polish included)"},
    }
    b.close()
    for h in systems:
        h.close()
    return out


ADJ_WORKLOAD = ("adjoint workload: n=8, 12 monomials/equation, exponents in [-2,2], planted pair cell "
                "with |det V| >= 4096; 4,096 start points tracked to t = 1 (mixed form + FP64 polish), "
                "then the implicit-function coefficient gradient at the converged solutions")
FP64_PEAK_TFLOPS = 1.25   # nominal FP64 (non-tensor) rate of the part


def run_track_adjoint(args, dev):
    """hpt_track on the adjoint workload's 4,096 paths (whole tracks with the
    FP64 polish), then hpt_adjoint at the converged solutions."""
    import torch
    from paper_2111_14317_gb300 import hpt
    import workloads as W
    n_sol = 4096
    for att in range(200):
        s, pairs = W.config5(att)
        try:
            y0, tot = hpt.binomial_start(s.n, s.m, s.exponents, s.coeffs, pairs, 0, 1)
            if tot < n_sol:
                continue
            y0, _ = hpt.binomial_start(s.n, s.m, s.exponents, s.coeffs, pairs, 0, n_sol)
            h = hpt.System.from_laurent(s, {"kind": "pairs", "pairs": pairs}, hpt.HPT_MIXED)
            break
        except hpt.HptError:
            continue
    prm = hpt.Params(tol_accept=3e-3)
    yd = torch.from_numpy(y0).to(dev)
    h.track(yd, prm)
    reps = 3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        x, st, sp = h.track(yd, prm)
    torch.cuda.synchronize()
    track_ms = (time.perf_counter() - t0) * 1e3 / reps
    conv = st == hpt.CONVERGED
    xc = x[conv].contiguous()
    gx = (2.0 * xc).contiguous()             # gradient of sum |x|^2
    for _ in range(3):
        h.adjoint(xc, gx)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(10):
        gc = h.adjoint(xc, gx)
    ev[1].record()
    torch.cuda.synchronize()
    adj_ms = ev[0].elapsed_time(ev[1]) / 10
    nconv = int(conv.sum().item())
    n, M = s.n, h.M
    # FP64 work per solution: evaluation (dot products, coefficient sums),
    # LU with one right-hand side and the contributions; exp/sincos not counted
    flop = M * (2 * n + 8 * (n + 2)) + 8 * (n - 1) * n * (2 * n - 1) // 6 + 8 * n * n + M * (2 * n + 8)
    achieved = nconv * flop / (adj_ms * 1e-3) / 1e12
    out = {
        "workload": ADJ_WORKLOAD, "attempt": att, "det_V": int(tot),
        "track": {"paths": n_sol, "ms": track_ms, "paths_per_s": n_sol / (track_ms * 1e-3),
                  "path_steps_per_s": float(sp.sum().item()) / (track_ms * 1e-3),
                  "converged": nconv, "median_steps": float(sp.float().median().item())},
        "adjoint": {"solutions": nconv, "ms": adj_ms, "value": nconv / (adj_ms * 1e-3), "unit": "solutions/s",
                    "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                 "frac": achieved / FP64_PEAK_TFLOPS, "peak_source": "nominal FP64 rate",
                                 "flop_per_solution": flop}},
    }
    h.close()
    return out


PROJ_WORKLOAD = ("projective form (Section 2.2) of the n=16 throughput workload: 16 equations in 17 homogeneous "
                 "coordinates, exponents (a, deg_k - 1^T a); 65,536 paths at (x, 1)/|(x, 1)|; one hpt_step "
                 "(evaluation + Algorithm 3 by QR + projective step control) per step")
# bytes one projective QR step moves per path: the extended Jacobian (16 rows x
# 19 complex64), y, y_acc, dE_acc (17 complex64 each, read and written), three
# doubles and five int32 (read and written)
QR_BYTES_PATH = 16 * 19 * 8 + 3 * 17 * 8 * 2 + 3 * 8 * 2 + 5 * 4 * 2


def run_projective(args, dev):
    """hpt_step on projective handles of the n=16 workload, both forms, timed as
    the headline step (state restored, L2 flushed before every timed step)."""
    import torch
    from paper_2111_14317_gb300 import hpt
    import workloads as W
    sysm, cell = _workload()
    x_np, t_np = W.random_points(shard_seed(0), PATHS, N_VARS)
    y_np = np.concatenate([x_np, np.ones((PATHS, 1))], axis=1)
    y_np /= np.linalg.norm(y_np, axis=1, keepdims=True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peaks, peak_kind = _peaks()
    out = {"workload": PROJ_WORKLOAD}
    for form, prec in (("mixed", hpt.HPT_MIXED), ("fp64", hpt.HPT_FP64)):
        ha = hpt.System.from_laurent(sysm, cell, prec)
        h = ha.homogenize()
        prm = hpt.Params(tol_accept=3e-3 if prec == hpt.HPT_MIXED else 1e-3)
        st = h.new_state(PATHS, device=dev)
        yd = torch.from_numpy(y_np).to(dev, h.cdtype)
        st.y.copy_(yd)
        st.y_acc.copy_(yd)
        st.tau.copy_(torch.from_numpy(np.log(t_np)))
        st.tau_acc.copy_(st.tau)
        st.dtau.fill_(0.01)
        st.accepts.fill_(1)
        pristine = st.arena.clone()
        steps = args.steps if form == "mixed" else max(3, min(args.steps, args.fp64_steps))
        for _ in range(args.warmup):
            st.arena.copy_(pristine)
            h.step(st, 1, prm)
        torch.cuda.synchronize()
        res = {}
        for profile in (False, True):
            h.profile(profile)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            for i in range(steps):
                st.arena.copy_(pristine)
                flush.zero_()
                ev[i][0].record()
                h.step(st, 1, prm)
                ev[i][1].record()
            torch.cuda.synchronize()
            h.profile(False)
            if not profile:
                res["ms_per_step"] = sum(a.elapsed_time(b) for a, b in ev) / steps
        kern = h.profile_read()
        assert h.device_error() == 0, "device-side wait timed out"
        res["value"] = PATHS / (res["ms_per_step"] * 1e-3)
        res["unit"] = UNIT
        res["kernels"] = {k: {"launches": v[0], "ms_avg": v[1] / max(v[0], 1)} for k, v in kern.items()}
        qr = kern.get("qr_step")
        if qr:
            avg_s = qr[1] / max(qr[0], 1) * 1e-3
            ach = PATHS * QR_BYTES_PATH / avg_s / 1e9
            res["roofline_qr"] = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                  "frac": ach / peaks["hbm_gbs"], "bytes_per_path": QR_BYTES_PATH,
                                  "peak_source": f"{peak_kind} (MEASURED_PEAKS.json)",
                                  "traffic": _traffic("qr_step") if form == "mixed" else None}
        out[form] = res
        h.close()
        ha.close()
        del st, pristine
        torch.cuda.empty_cache()
    out["mixed_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


PAPER_SHAPES = {
    # stand-ins for the paper's Table 1 (cyclic-14: 14 equations, 184 monomials)
    # and Table 2 (chandra-24: 24 equations, 324 monomials); the systems
    # themselves are not available, only their shapes are matched
    "n14_m184": (14, 184, (10, 50, 250, 500, 1000), {10: 0.0222, 50: 0.0274, 250: 0.0296, 500: 0.0313, 1000: 0.0355}),
    "n24_m324": (24, 324, (250, 500, 1000), {250: 0.0728, 500: 0.0757, 1000: 0.0852}),
}


def run_paper_shapes(args, dev):
    """The protocol of the paper's Tables 1-2 on synthetic systems of the same
    shapes: 100 consecutive Euler-Newton steps (one hpt_step call with
    nsteps = 100) on p paths, wall-clock time with the start points copied
    from pinned host memory and the accepted points copied back inside the
    timed region (median of 3 runs), plus the device time of the steps."""
    import torch
    from paper_2111_14317_gb300 import hpt
    import workloads as W
    out = {"protocol": "100 consecutive Euler-Newton steps per call on p paths of a planted cell (start "
                       "points exp(V^-1(log b + 2 pi i j e_1))); wall = H2D of the start points + init + "
                       "100 steps + D2H of y_acc, median of 3; paper_v100_s = the paper's V100 column "
                       "(other hardware, other systems of the same shape: context only)"}
    for name, (n, M, ps, paper) in PAPER_SHAPES.items():
        s, pairs = W.paper_shape(n, M)
        rec = {"n": n, "monomials": M, "paper_v100_s": {str(k): v for k, v in paper.items()}}
        pmax = max(ps)
        ks = np.zeros((pmax, n), np.int64)
        ks[:, 0] = np.arange(pmax)
        x0_all = hpt.binomial_points(n, s.m, s.exponents, s.coeffs, pairs, ks)
        for form, prec in (("mixed", hpt.HPT_MIXED), ("fp64", hpt.HPT_FP64)):
            h = hpt.System.from_laurent(s, {"kind": "pairs", "pairs": pairs}, prec)
            prm = hpt.Params(tol_accept=3e-3 if prec == hpt.HPT_MIXED else 1e-3)
            res = {}
            for p in ps:
                host = torch.from_numpy(np.ascontiguousarray(x0_all[:p])).pin_memory()
                st = hpt.PathState(p, n, prec, device=dev)
                back = torch.empty(st.y_acc.shape, dtype=st.y_acc.dtype).pin_memory()
                walls, devs = [], []
                for rep in range(4):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    x0 = host.to(dev, non_blocking=True)
                    h.paths_init(st, x0, prm)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    h.step(st, 100, prm)
                    e1.record()
                    back.copy_(st.y_acc, non_blocking=True)
                    torch.cuda.synchronize()
                    if rep:   # the first run warms up
                        walls.append(time.perf_counter() - t0)
                        devs.append(e0.elapsed_time(e1) * 1e-3)
                active = int((st.status == hpt.ACTIVE).sum().item())
                done = int(st.steps.sum().item())
                res[str(p)] = {"wall_s": statistics.median(walls), "device_s": statistics.median(devs),
                               "path_steps": done, "active_after": active}
            rec[form] = res
            h.close()
        out[name] = rec
    return out


def run_step100(args, dev):
    """The paper's protocol (100 consecutive Euler-Newton steps in one call)
    at the throughput size: 65,536 paths of a system of the same shape
    (n = 16, 32 monomials per equation, exponent vectors with 4 nonzeros, here
    in [-2, 2]) whose planted cell gives real homotopy paths, started at
    exp(V^-1 (log b + 2 pi i j e_1)), j < 65,536 (j taken modulo |det V| by
    the lattice: a repeated start point costs the same).  One hpt_step call
    with nsteps = 100 per run, CUDA events around it, median of 3 after a
    warm-up; path-steps are the steps the paths actually took (accepts and
    rejects alike; a path that finishes stops)."""
    import torch
    from paper_2111_14317_gb300 import hpt
    import workloads as W
    n = N_VARS
    s, pairs = W.paper_shape(n, N_VARS * M_PER_EQ)
    _, det = hpt.binomial_start(s.n, s.m, s.exponents, s.coeffs, pairs, 0, 0)
    ks = np.zeros((PATHS, n), np.int64)
    ks[:, 0] = np.arange(PATHS)
    x0 = torch.from_numpy(np.ascontiguousarray(hpt.binomial_points(n, s.m, s.exponents, s.coeffs, pairs, ks)))
    x0 = x0.to(dev)
    out = {"workload": f"planted-cell system n={n}, {M_PER_EQ} monomials/equation, |det V| = {det}; "
                       f"{PATHS} paths from the start points; hpt_step(nsteps=100) per call",
           "det_V": int(det)}
    for form, prec in (("mixed", hpt.HPT_MIXED), ("fp64", hpt.HPT_FP64)):
        h = hpt.System.from_laurent(s, {"kind": "pairs", "pairs": pairs}, prec)
        prm = hpt.Params(tol_accept=3e-3 if prec == hpt.HPT_MIXED else 1e-3)
        st = hpt.PathState(PATHS, n, prec, device=dev)
        ms = []
        for rep in range(4):
            h.paths_init(st, x0, prm)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            h.step(st, 100, prm)
            e1.record()
            torch.cuda.synchronize()
            if rep:   # the first run warms up
                ms.append(e0.elapsed_time(e1))
        med = statistics.median(ms)
        steps = int(st.steps.sum().item())
        out[form] = {"ms_per_call": med, "path_steps": steps, "value": steps / (med * 1e-3), "unit": UNIT,
                     "active_after": int((st.status == hpt.ACTIVE).sum().item()),
                     "converged_after": int((st.status == hpt.CONVERGED).sum().item())}
        assert h.device_error() == 0, "device-side wait timed out"
        h.close()
        del st
        torch.cuda.empty_cache()
    out["mixed_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def run_start_points(args, dev):
    """Start points of a large cell (the n = 24, 324-monomial stand-in):
    hpt_binomial_start_device for 2^20 solutions (CUDA events) against the
    host enumeration hpt_binomial_start for 2^16."""
    import torch
    from paper_2111_14317_gb300 import hpt
    import workloads as W
    s, pairs = W.paper_shape(24, 324)
    _, tot = hpt.binomial_start(s.n, s.m, s.exponents, s.coeffs, pairs, 0, 0)
    nd, nh = min(tot, 1 << 20), min(tot, 1 << 16)
    hpt.binomial_start_device(s.n, s.m, s.exponents, s.coeffs, pairs, 0, nd)   # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    hpt.binomial_start_device(s.n, s.m, s.exponents, s.coeffs, pairs, 0, nd)
    e1.record()
    torch.cuda.synchronize()
    dms = e0.elapsed_time(e1)
    t0 = time.perf_counter()
    hpt.binomial_start(s.n, s.m, s.exponents, s.coeffs, pairs, 0, nh)
    hms = (time.perf_counter() - t0) * 1e3
    return {"cell": "n=24, 324 monomials, planted pairs cell", "det_V": int(tot),
            "device": {"points": int(nd), "ms": dms, "points_per_s": nd / (dms * 1e-3)},
            "host_one_core": {"points": int(nh), "ms": hms, "points_per_s": nh / (hms * 1e-3)}}


def alu_peaks(sms, clk_mhz):
    """Derived ALU rates at the maximum SM clock: FP32 FMA (TFLOP/s) and the
    MUFU time of one path's complex exponentials (seconds per path, ex2 at
    MUFU_EX2_PER_CLK and sin, cos at MUFU_SINCOS_PER_CLK per SM and clock)."""
    hz = clk_mhz * 1e6
    fp32 = sms * FP32_LANES * 2 * hz / 1e12
    mufu_s_per_path = (CEXP / MUFU_EX2_PER_CLK + 2 * CEXP / MUFU_SINCOS_PER_CLK) / (sms * hz)
    return fp32, mufu_s_per_path


def step_roofline(mx, peaks, peak_kind, sms):
    """Per-kernel and whole-step rooflines of the mixed step from the
    algorithmic work of one path-step (dense within each equation's block):
    GEMM flops on the tensor pipe, 3 MUFU operations per complex exponential,
    LU + two solves + update on the FP32 pipe, the path state in HBM.  The
    bound of a kernel is the pipe whose time is the largest; frac = that
    time / the measured kernel time (achieved / peak of that pipe).  The
    extended-Jacobian scratch between the kernels is not algorithmic work:
    the DRAM bytes ncu measured are reported beside it as traffic_ratio."""
    clk = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak, mufu_path = alu_peaks(sms, clk)
    bf16 = peaks["bf16_tflops"]
    hbm = peaks["hbm_gbs"]
    src = f"{peak_kind} (MEASURED_PEAKS.json, burst)"
    derived = f"derived: {sms} SMs x {clk:.0f} MHz"
    kinfo = {}
    for name, (launches, msum) in mx["kernels"].items():
        avg = msum / max(launches, 1) * 1e-3
        ppl = PATHS * mx["steps"] / max(launches, 1)
        rec = {"ms_avg": avg * 1e3, "launches": launches, "share": msum}
        if name.startswith("eval_mixed"):
            gemm = (FLOP_EXP_GEMM + FLOP_COEF_GEMM) * ppl
            ops = 3 * CEXP * ppl                       # ex2, sin, cos per exponential
            mufu_peak = 3 * CEXP / mufu_path / 1e12    # the mix's rate at the derived unit counts
            rec.update({"bound": "alu", "pipe": "MUFU", "achieved": ops / avg / 1e12, "peak": mufu_peak,
                        "unit": "Tops/s", "frac": ops / avg / 1e12 / mufu_peak,
                        "peak_source": derived + f", ex2 {MUFU_EX2_PER_CLK}/clk/SM, sin/cos "
                                                 f"{MUFU_SINCOS_PER_CLK}/clk/SM",
                        "tensor": {"achieved": gemm / avg / 1e12, "peak": bf16, "unit": "TFLOP/s",
                                   "frac": gemm / avg / 1e12 / bf16, "peak_source": src}})
        elif name.startswith("redo"):
            # re-solves a device-side list of a few paths: no per-path figure
            rec.update({"bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None})
        else:
            fl = (FLOP_LU + FLOP_SOLVE) * ppl
            ach = fl / avg / 1e12
            rec.update({"bound": "alu", "pipe": "FP32 FMA", "achieved": ach, "peak": fp32_peak,
                        "unit": "TFLOP/s", "frac": ach / fp32_peak, "peak_source": derived + ", 128 FP32 lanes"})
        tr = _traffic(name)
        rec["traffic"] = tr
        if tr is not None:
            rec["traffic_ratio"] = tr / (STATE_BYTES * ppl)
        kinfo[name] = rec
    total_k = sum(v["share"] for v in kinfo.values()) or 1.0
    for v in kinfo.values():
        v["share"] = v["share"] / total_k
    dom = max(kinfo, key=lambda k: kinfo[k]["share"])
    roof = {k: kinfo[dom].get(k) for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
    roof["kernel"] = dom
    roof["pipe"] = kinfo[dom].get("pipe")
    roof["peak_source"] = kinfo[dom].get("peak_source")
    # whole step: T_roof = max over pipes of the step's algorithmic work / peak
    t_pipe = {"tensor": (FLOP_EXP_GEMM + FLOP_COEF_GEMM) * PATHS / (bf16 * 1e12),
              "MUFU": mufu_path * PATHS,
              "FP32 FMA": (FLOP_LU + FLOP_SOLVE) * PATHS / (fp32_peak * 1e12),
              "HBM": STATE_BYTES * PATHS / (hbm * 1e9)}
    bind = max(t_pipe, key=t_pipe.get)
    t_step = mx["ms_per_step"] * 1e-3
    traffic = [v["traffic"] for v in kinfo.values() if v.get("traffic") is not None]
    step_roof = {"t_roof_us": t_pipe[bind] * 1e6, "binding_pipe": bind,
                 "t_pipe_us": {k: v * 1e6 for k, v in t_pipe.items()},
                 "t_measured_us": t_step * 1e6, "frac": t_pipe[bind] / t_step,
                 "algorithmic_bytes": STATE_BYTES * PATHS,
                 "traffic_ratio": (sum(traffic) / (STATE_BYTES * PATHS)
                                   if len(traffic) == len([v for v in kinfo.values() if v["bound"] != "latency"])
                                   else None)}
    return kinfo, roof, step_roof


def cpu_baseline(seconds=12.0, max_paths=PATHS):
    """Times the oracle's step (as it stands) on growing slices of the same
    workload until about `seconds` of work is done."""
    import oracle
    import workloads as W
    from oracle import cells
    sysm, cell = _workload()
    te = cells.t_exponents(sysm, cell)
    osys = oracle.System(sysm, te["e"], te["D"])
    y, t = W.random_points(1, PATHS, N_VARS)
    P = oracle.Params()
    done, el, q0, chunk = 0, 0.0, 0, 256
    while el < seconds and done < max_paths:
        cnt = min(chunk, PATHS - q0)
        st = oracle.PathState.start(y[q0:q0 + cnt], 0.0, 0.01)
        st.tau[:] = np.log(t[q0:q0 + cnt])
        st.tauacc[:] = st.tau
        st.accepts[:] = 1
        t0 = time.perf_counter()
        osys.step(P, st, 1)
        el += time.perf_counter() - t0
        done += cnt
        q0 = (q0 + cnt) % PATHS
        chunk = min(chunk * 2, 8192)
    return done / el, oracle.num_threads(), f"{done} of the {PATHS} paths, one step each, complex128 oracle"


def cpu_baseline_step100(n_paths=4096):
    """The oracle (complex128, all host cores) on the paper's protocol: 100
    consecutive steps in one call on the first n_paths start points of the
    planted-cell workload that bench's step100 tracks on the GPU."""
    import oracle
    import workloads as W
    from oracle import cells
    from paper_2111_14317_gb300 import hpt
    n = N_VARS
    s, pairs = W.paper_shape(n, N_VARS * M_PER_EQ)
    ks = np.zeros((n_paths, n), np.int64)
    ks[:, 0] = np.arange(n_paths)
    x0 = np.ascontiguousarray(hpt.binomial_points(n, s.m, s.exponents, s.coeffs, pairs, ks))
    cell = {"kind": "pairs", "pairs": pairs}
    te = cells.t_exponents(s, cell)
    osys = oracle.System(s, te["e"], te["D"])
    P = oracle.Params(tol_accept=1e-3)
    h = hpt.System.from_laurent(s, cell, hpt.HPT_FP64)   # tau0 = ln(eps0) / s_min, as hpt_paths_init
    tau0 = h.tau0()
    h.close()
    st = oracle.PathState.start(x0, tau0, P.dtau_init)
    t0 = time.perf_counter()
    osys.step(P, st, 100)
    el = time.perf_counter() - t0
    steps = int(st.steps.sum())
    return {"paths": n_paths, "path_steps": steps, "s": el, "value": steps / el, "unit": UNIT,
            "cores": oracle.num_threads(),
            "sample": f"the first {n_paths} of the step100 workload's paths, 100 steps in one call, "
                      "complex128 oracle"}


def cpu_baseline_one_core(seconds=2.0):
    """The same oracle step on one host thread (the paper compares one core
    with eight, Section 8)."""
    import oracle
    k = oracle.num_threads()
    oracle.set_threads(1)
    try:
        v, _, sample = cpu_baseline(seconds)
    finally:
        oracle.set_threads(k)
    return v, sample


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--batch-systems", type=int, default=256, help="0 skips the many-systems batch")
    ap.add_argument("--batch-paths", type=int, default=512)
    ap.add_argument("--batch-reps", type=int, default=3)
    ap.add_argument("--no-autotune", action="store_true", help="batch: keep the default tuning")
    ap.add_argument("--skip-predictors", action="store_true",
                    help="batch: skip the Euler/Hermite comparison at tol 1e-3 (shorter profiling runs)")
    ap.add_argument("--workload", default="all", choices=["all", "step", "batch", "projective", "paper_shapes",
                                                             "start_points", "step100", "adjoint"],
                    help="step: the n=16 hpt_step line only; batch: the many-systems batch only; "
                         "projective: the projective-form step only; adjoint: the track + adjoint "
                         "workload only (the others print their own JSON object, for profiling)")
    args = ap.parse_args()
    ws, rank, _ = _dist()

    if args.impl == "reference":
        if rank != 0:
            return
        ms = []
        for _ in range(args.warmup):
            cpu_baseline(0.5)
        vals = []
        for _ in range(args.steps):
            v, cores, sample = cpu_baseline(max(1.0, args.cpu_seconds / max(args.steps, 1)))
            vals.append(v)
        val = statistics.median(vals)
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": PATHS / val * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": WORKLOAD, "n": N_VARS, "m": M_PER_EQ,
                                                 "paths": PATHS},
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": sample + " per step"},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.workload == "batch":
        import torch
        from paper_2111_14317_gb300 import build as hbuild
        hbuild.build()
        torch.cuda.set_device(0)
        print(json.dumps({"batch": run_batch(args, torch.device("cuda", 0))}))
        return
    if args.workload in ("paper_shapes", "start_points", "step100", "adjoint"):
        import torch
        from paper_2111_14317_gb300 import build as hbuild
        hbuild.build()
        torch.cuda.set_device(0)
        fn = {"paper_shapes": run_paper_shapes, "start_points": run_start_points,
              "step100": run_step100, "adjoint": run_track_adjoint}[args.workload]
        print(json.dumps({args.workload: fn(args, torch.device("cuda", 0))}))
        return
    if args.workload == "projective":
        import torch
        from paper_2111_14317_gb300 import build as hbuild
        hbuild.build()
        torch.cuda.set_device(0)
        print(json.dumps({"projective": run_projective(args, torch.device("cuda", 0))}))
        return
    if args.workload == "step":
        args.batch_systems = 0
    out, ws, rank = run_gpu(args)
    if rank != 0:
        return
    peaks, peak_kind = _peaks()
    mx, fp = out["mixed"], out["fp64"]
    value = whole_job_rate(ws, PATHS, mx["ms_per_step"] * 1e-3)
    fp_value = whole_job_rate(ws, PATHS, fp["ms_per_step"] * 1e-3)
    kinfo, roof, step_roof = step_roofline(mx, peaks, peak_kind, out["sms"])
    cpu_v, cores, sample = cpu_baseline(args.cpu_seconds)
    one_v, one_sample = cpu_baseline_one_core(min(3.0, max(0.5, args.cpu_seconds / 4)))
    s100 = cpu_baseline_step100() if args.workload == "all" else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": mx["steps"],
        "warmup": args.warmup, "ms_per_step": mx["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3-split/f32 (mixed form)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_VARS, "m": M_PER_EQ, "paths": PATHS,
                   "steps_per_call": 1, "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"replicas x{ws} (paths shard, no collective)"},
        "fp64_form": {"value": fp_value, "unit": UNIT, "ms_per_step": fp["ms_per_step"],
                      "steps": fp["steps"], "kernels": {k: {"launches": v[0], "ms": v[1]}
                                                        for k, v in fp["kernels"].items()}},
        "mixed_vs_fp64": value / fp_value,
        "roofline": roof,
        "step_roofline": step_roof,
        "kernels": kinfo,
        "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "one_core": {"value": one_v, "unit": UNIT, "cores": 1, "sample": one_sample},
                         "step100": s100},
        "e2e": {"value": ws * PATHS / mx["e2e_s"], "unit": UNIT, "h2d_bytes_per_step": mx["h2d"],
                "d2h_bytes_per_step": mx["d2h"]},
        "clocks": mx["clocks"],
        "gpu_launches": mx["launches"],
    }
    if "batch" in out:
        line["batch"] = out["batch"]
    if "track_adjoint" in out:
        line["track_adjoint"] = out["track_adjoint"]
    if "projective" in out:
        line["projective"] = out["projective"]
    if "paper_shapes" in out:
        line["paper_shapes"] = out["paper_shapes"]
    if "start_points" in out:
        line["start_points"] = out["start_points"]
    if "step100" in out:
        line["step100"] = out["step100"]
    print(json.dumps(line))


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark of the shifted-CG hot path on the 32^3 x 8 workload.

One step = one complete call of mshift_cg: the 16-pole rational approximation of
x^{-1/2} on [4m^2, 16 + 4m^2] (m = 0.02) applied to a Gaussian source, solved to a
true FP64 residual of 1e-10 for every shift (Section 4, Eq. ratapprx), in the
mixed mode (double-FP32 until |r| <= 1e-3 |b|, then FP32 links and Krylov vectors;
dot products, solution accumulation, reliable updates and final residuals with
FP64-class accuracy as double-FP32 pairs) -- every row of the hot path:
Dslash, A-apply, reductions, shifted updates, reliable updates, refinement and
the rational application.

Printed JSON line (rank 0): value = ms per solve (mixed), plus the FP64 solve,
the 12-real and 16-bit variants, the Dslash roofline (algorithmic bytes per
launch over the CUDA-event time per launch of a CUDA graph of launches that
rotate over eight gauge fields, so that every launch reads from HBM; the same
launches from the host stream and the isolated launch after an L2 flush are
reported beside it), the end-to-end number through the C ABI with host buffers,
and the oracle timed on the host cores (cpu_baseline).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
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
# hardware work queues for the concurrent solve graphs of the batch workload (the CUDA runtime default
# of 8 serialises the streams of more than 8 concurrent solves onto 8 queues); read when the process
# creates its CUDA context, a per-process setting
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "multishift-CG time/solve to 1e-10, mixed vs FP64 at 32^3x8; Dslash % HBM peak"
WORKLOAD = "32^3x8"
DIMS = (32, 32, 32, 8)
MASS = 0.02
NPOLES = 16
TOL = 1e-10
GAUGE_SEED, VEC_SEED = 5, 6
# Dslash algorithmic bytes per output site (8 links + 1 input + 1 output vector, each crossing HBM once)
DSLASH_BYTES_PER_SITE = {"fp32": 8 * 72 + 24 + 24, "fp32_r12": 8 * 48 + 24 + 24, "fp32_r8": 8 * 32 + 24 + 24,
                         "fp32_l16": 8 * 24 + 24 + 24, "fp64": 8 * 144 + 48 + 48}
DSLASH_FLOPS_PER_SITE = 570
# The double-FP32 half Dslash (the checks and the first phase of the mixed solve): per output site 8 hops x
# 9 link entries x 4 real products, each one compensated multiply-add of 12 FP32 operations (product,
# its exact error and the two cross terms: 4; TwoSum into the running sum: 6; the compensation: 2), and
# 6 final renormalisations of 2; bytes, counted as for the FP32 Dslash (each crossing HBM once): 8 link
# pairs (hi, lo: 2 x 72), the input pair (2 x 24, re-read from L2 by the neighbours) and the output pair
DF_OPS_PER_SITE = 8 * 9 * 4 * 12 + 6 * 2
DF_BYTES_PER_SITE = 8 * 144 + 48 + 48


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash(files=("dslash.cu", "common.cuh")):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1710_09178_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload_key, record="dslash_fp32_32c8.json", files=("dslash.cu", "common.cuh")):
    """DRAM bytes per launch of a kernel from its committed ncu record (profiles/<record>: the FP32
    Dslash by default), if it was captured on this kernel source."""
    p = os.path.join(ROOT, "profiles", record)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    if rec.get("source_hash") != kernel_source_hash(files):
        return None
    return float(rec["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


class L2Flusher:
    """Write a 256 MB buffer, then read another one (both > 129 MB of L2): the read pass evicts the
    dirty lines of the write pass, so the next kernel starts from a clean, cold L2."""

    def __init__(self, torch):
        self.w = torch.zeros(64 << 20, dtype=torch.float32, device="cuda")
        self.r = torch.ones(64 << 20, dtype=torch.float32, device="cuda")
        self.sink = torch.zeros(1, dtype=torch.float32, device="cuda")

    def add_(self, _):
        self.w.add_(1.0)
        self.sink.add_(self.r.sum())


def replica_aggregate(total_ms, steps, world, dist, device):
    """N independent replicas (one lattice solve per rank, no data-path collective): the timed
    region is the slowest rank's, and the whole job completes steps x world solves in it.
    Returns (max timed ms, ms per solve of one replica, whole-job ms per solve)."""
    if dist is not None and world > 1:
        import torch

        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, total_ms / steps, total_ms / (steps * world)


def solve_algorithmic_bytes(st, vh, fp64):
    """Minimum traffic of the plain shifted CG's base iterations (every vector and link crossing HBM
    once): per iteration and site the A-apply (two half-Dslash + the own-site read), the r and p
    updates, and per active shift the p_k and x_k read-modify-writes."""
    per_iter = (2 * 1248 + 48 + 144 + 144) if fp64 else (2 * 624 + 24 + 72 + 72)
    per_shift = (96 + 96) if fp64 else (48 + 96)
    return vh * (st["iterations"] * per_iter + st.get("shift_iterations", 0) * per_shift)


def setup_problem(lq, torch):
    from paper_1710_09178_gb300 import inputs

    U = inputs.gauge_field(DIMS, seed=GAUGE_SEED)
    b = inputs.gaussian_vector(DIMS, VEC_SEED)
    lo, hi = 4 * MASS * MASS, 16 + 4 * MASS * MASS
    c0, res, poles, err = lq.rational_coeffs(-0.5, lo, hi, NPOLES)
    return U, b, (c0, res, poles, err)


def time_solves(lq, torch, ctx, bd, xs, y, coeffs, prec, steps, warmup, flush_buf):
    c0, res, poles, _ = coeffs
    st = None
    for _ in range(warmup):
        rc, st = lq.mshift_cg(ctx, poles, res, c0, bd, xs, y, tol=TOL, prec=prec)
    times, stats = [], []
    stream = torch.cuda.current_stream()
    for _ in range(steps):
        flush_buf.add_(1)  # evict the previous solve's data from L2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, st = lq.mshift_cg(ctx, poles, res, c0, bd, xs, y, tol=TOL, prec=prec)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        stats.append(st)
    return times, stats


def time_dslash(lq, torch, ctx, prec_name, prec, reps, flush_buf):
    """Average duration of one Dslash launch (D_oe then D_eo alternately), L2 flushed before each."""
    vin = ctx.new_vector(prec)
    vout = ctx.new_vector(prec)
    vin.view(torch.float32 if prec != lq.FP64 else torch.float64).normal_()
    stream = torch.cuda.current_stream()
    for p in (0, 1, 0, 1):
        lq.dslash_eo(ctx, vout, vin, p, prec)
    evs = []
    for r in range(reps):
        flush_buf.add_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lq.dslash_eo(ctx, vout, vin, r & 1, prec)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    return statistics.mean(ms), statistics.median(ms)


def fp64_peak_tflops(torch, n=4096, reps=5):
    """FP64 matrix-multiply rate (cuBLAS DGEMM, 2 n^3 flops per product), best of reps."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 0.0
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


STREAM_FIELDS = 8  # 8 x 75.5 MB of FP32 links: each field is ~528 MB of traffic old when it is read again


def make_stream_contexts(lq, torch, Ud, n, stream=None):
    """n contexts holding their own copies of the same gauge field (distinct buffers, so distinct
    L2 lines), with one input and one output vector each, launching on `stream` (default: current)."""
    out = []
    for _ in range(n):
        c = lq.Context(DIMS, MASS, stream=None if stream is None else stream.cuda_stream)
        c.set_gauge(Ud)
        vin, vout = c.new_vector(lq.FP32), c.new_vector(lq.FP32)
        vin.view(torch.float32).normal_()
        out.append((c, vin, vout))
    return out


def time_dslash_stream(lq, torch, sctx, prec, reps):
    """Average duration of back-to-back Dslash launches that rotate over the gauge fields of sctx.
    Between two reads of one field the other fields move 7 x 75.5 MB through L2 (129 MB), so every
    launch streams its links and vectors from HBM, as the isolated launches after an L2 flush do.
    Each launch is one call through the C ABI from Python, so the host's per-call time shows up as
    gaps between the kernels."""
    stream = torch.cuda.current_stream()
    n = len(sctx)

    def launch(i):
        c, vin, vout = sctx[i % n]
        lq.dslash_eo(c, vout, vin, (i // n) & 1, prec)

    for i in range(2 * n):
        launch(i)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(reps):
        launch(i)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def time_dslash_graph(lq, torch, Ud, prec, reps, n_fields=STREAM_FIELDS):
    """As time_dslash_stream, with the reps launches captured in one CUDA graph (the way the
    solver runs them): the host launch gaps between the kernels are gone and what is left is the
    kernel's own duration from HBM.  Returns ms per launch (median of 5 replays), or None where
    the capture is refused."""
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    sctx = make_stream_contexts(lq, torch, Ud, n_fields, stream=s)
    n = len(sctx)
    try:
        with torch.cuda.stream(s):
            for i in range(2 * n):
                c, vin, vout = sctx[i % n]
                lq.dslash_eo(c, vout, vin, (i // n) & 1, prec)
            s.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
                for i in range(reps):
                    c, vin, vout = sctx[i % n]
                    lq.dslash_eo(c, vout, vin, (i // n) & 1, prec)
            graph.replay()
            ms = []
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s)
                graph.replay()
                e1.record(s)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1) / reps)
        return statistics.median(ms)
    except (RuntimeError, lq.LqcdError):
        return None
    finally:
        torch.cuda.synchronize()
        for c, _, _ in sctx:
            c.close()


def time_df_dslash_graph(lq, torch, Ud, reps=64):
    """The double-FP32 half Dslash (dslash_eo with LQCD_DF64 vectors) at the bench workload: reps
    launches in one CUDA graph, alternating parities; its 151 MB of hi + lo links exceed L2.  Returns ms
    per launch (median of 5 replays), or None where the capture is refused."""
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    c = lq.Context(DIMS, MASS, stream=s.cuda_stream)
    try:
        c.set_gauge(Ud)
        vin, vout = c.new_vector(lq.DF64), c.new_vector(lq.DF64)
        vin.view(torch.float32).normal_()
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            for i in range(4):
                lq.dslash_eo(c, vout, vin, i & 1, lq.DF64)
            s.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
                for i in range(reps):
                    lq.dslash_eo(c, vout, vin, i & 1, lq.DF64)
            graph.replay()
            ms = []
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s)
                graph.replay()
                e1.record(s)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1) / reps)
        return statistics.median(ms)
    except (RuntimeError, lq.LqcdError):
        return None
    finally:
        torch.cuda.synchronize()
        c.close()


def cpu_oracle_solves(U, b, coeffs):
    """The C++ FP64 oracle's complete shifted-CG solve of the bench workload on the host cores: once
    with OpenMP on every core and once on one core, each to the same 1e-10 stopping rule.  Returns
    the timings (per solve, per iteration, per half-lattice hop) and the OpenMP solve's solutions and
    y = c0 b + sum_k c_k x_k, against which the GPU results are measured."""
    from oracle import cpp_oracle

    c0, res, poles, _ = coeffs
    out = {}
    sol = None
    for kind, threaded in (("all_cores", True), ("one_core", False)):
        orc = cpp_oracle.load(threaded=threaded)
        lat = orc.lattice(DIMS, U, MASS)
        xs, info = lat.multishift_cg(b, poles, tol=TOL)
        out[kind] = {"ms_per_solve": info["seconds"] * 1e3, "threads": orc.threads(),
                     "iterations": info["iterations"], "shift_iterations": int(info["shift_iterations"]),
                     "ms_per_iteration": info["seconds"] * 1e3 / max(1, info["iterations"]),
                     "ms_per_dslash": info["seconds_dslash"] * 1e3 / max(1, info["dslash_calls"])}
        if sol is None:
            tr = lat.true_residuals(b, xs, poles)
            out[kind]["max_true_residual"] = float(tr.max())
            sol = (xs, orc.rational_apply(b, xs, c0, res))
        lat.close()
    return out, sol


def errors_vs_oracle(xs_gpu, y_gpu, sol):
    """Per shift |x_k - x_k^oracle| / |x_k^oracle| and |y - y^oracle| / |y^oracle| (FP64 norms)."""
    xs_o, y_o = sol
    ex = [float(np.linalg.norm(a - o) / np.linalg.norm(o)) for a, o in zip(xs_gpu, xs_o)]
    return {"x_k": ex, "max_x_k": max(ex), "y": float(np.linalg.norm(y_gpu - y_o) / np.linalg.norm(y_o))}


def host_cpu():
    """CPU model and logical core count of this host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    return {"model": model, "nproc": os.cpu_count()}


def run_reference(args, rank, world):
    """--impl reference: the C++ FP64 oracle on all host cores (OpenMP), same metric and unit.

    Every timed step is one complete shifted-CG solve of the bench workload (32^3x8, 16 poles,
    true residual 1e-10); warm-up steps run one iteration each.  Under torchrun only rank 0 runs."""
    if rank != 0:
        return
    from oracle import cpp_oracle, rational
    from paper_1710_09178_gb300 import inputs

    U = inputs.gauge_field(DIMS, seed=GAUGE_SEED)
    b = inputs.gaussian_vector(DIMS, VEC_SEED)
    lo, hi = 4 * MASS * MASS, 16 + 4 * MASS * MASS
    c0, res, poles, err = rational.zolotarev_inv_sqrt(NPOLES, lo, hi)
    orc = cpp_oracle.load(threaded=True)
    lat = orc.lattice(DIMS, U, MASS)
    for _ in range(args.warmup):
        lat.multishift_cg(b, poles, fixed_iters=1)
    per, infos = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xs, info = lat.multishift_cg(b, poles, tol=TOL)
        per.append(info["seconds"] * 1e3)
        infos.append(info)
    wall = time.perf_counter() - t0
    value = statistics.mean(per)
    last = infos[-1]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ms/solve", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": list(DIMS), "mass": MASS, "poles": NPOLES, "tol": TOL,
                   "precision": "fp64 oracle (C++, OpenMP)"},
        "cpu_baseline": {"value": value, "unit": "ms/solve", "cores": orc.threads(), "kind": "oracle",
                         "host": host_cpu(),
                         "sample": f"complete solves: every step is one full shifted-CG solve at 32^3x8 with 16 "
                                   f"shifts to 1e-10 ({last['iterations']} iterations, "
                                   f"{last['seconds'] * 1e3 / max(1, last['iterations']):.1f} ms/iteration, "
                                   f"{last['seconds_dslash'] * 1e3 / max(1, last['dslash_calls']):.2f} ms per "
                                   f"half-lattice hop) on {orc.threads()} OpenMP threads"},
        "e2e": {"value": value, "unit": "ms/solve", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s_timed": wall,
    }
    lat.close()
    print(json.dumps(line), flush=True)


TRAJ_DIMS, TRAJ_MASS, TRAJ_BETA, TRAJ_TAU, TRAJ_STEPS, TRAJ_POLES = (24, 24, 24, 6), 0.025, 5.4, 1.0, 25, 16


def run_trajectories(lq, torch, n_traj, md_tol=1e-7, nsteps=TRAJ_STEPS, n_therm=0):
    """RHMC trajectories on 24^3x6 (beta 5.4, m 0.025, 16-pole x^{-1/2} and x^{1/4}, Omelyan tau 1, 25 steps).

    Momenta, Gaussian sources and Metropolis numbers come from the counter-based generator (seed 9
    and per-trajectory streams).  MD force solves in mixed precision to md_tol; heatbath and
    Hamiltonian solves in mixed precision to a true FP64 residual of 1e-10.  The first n_therm
    trajectories thermalise the synthetic start: they are accepted whatever their dH (Metropolis
    number 0), which leaves the chain's fixed point alone and only shortens the approach to it; the
    remaining n_traj - n_therm use the Metropolis test.  Every trajectory's result carries the
    plaquette action per site after it."""
    from paper_1710_09178_gb300 import inputs

    lo, hi = 4 * TRAJ_MASS ** 2, 16 + 4 * TRAJ_MASS ** 2
    ca, ra, pa, _ = lq.rational_coeffs(-0.5, lo, hi, TRAJ_POLES)
    ch, rh, ph, _ = lq.rational_coeffs(0.25, lo, hi, TRAJ_POLES)
    V = int(np.prod(TRAJ_DIMS))
    ctx = lq.Context(TRAJ_DIMS, TRAJ_MASS)
    U = torch.from_numpy(inputs.gauge_field(TRAJ_DIMS, seed=9)).cuda()
    ctx.set_gauge(U)
    out = []
    for t in range(n_traj):
        mom = inputs.counter_normal_pairs(9000 + t, np.arange(4 * V, dtype=np.uint64), 4).reshape(V, 4, 8)
        xi = inputs.gaussian_vector(TRAJ_DIMS, 9500 + t)
        uni = 0.0 if t < n_therm else float(inputs.counter_uniform(9999, np.array([t], dtype=np.uint64), 0)[0])
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        md = torch.from_numpy(mom).cuda()
        xd = torch.from_numpy(xi).cuda()
        e0.record()
        rc, res = lq.rhmc_trajectory(ctx, U, md, xd, uni, TRAJ_BETA, TRAJ_TAU, nsteps, (ca, ra, pa), (ch, rh, ph),
                                     tol=1e-10, md_tol=md_tol, prec=lq.FP32, prec_action=lq.FP32)
        e1.record()
        e1.synchronize()
        res["event_ms"] = e0.elapsed_time(e1)
        res["therm"] = t < n_therm
        res["plaquette_action_per_site"] = (res["gauge1"] if res["accepted"] else res["gauge0"]) / TRAJ_BETA / (6 * V)
        out.append(res)
    ctx.close()
    return out


def rhmc_summary(tr, nsteps):
    """Acceptance and <exp(-dH)> over the Metropolis trajectories of run_trajectories."""
    meas = [r for r in tr if not r["therm"]]
    dh = np.array([r["dH"] for r in meas])
    ex = np.exp(-dh)
    return {"workload": "24^3x6", "beta": TRAJ_BETA, "mass": TRAJ_MASS, "tau": TRAJ_TAU, "steps": nsteps,
            "poles": TRAJ_POLES, "thermalising_trajectories": len(tr) - len(meas), "measured_trajectories": len(meas),
            "acceptance": float(np.mean([r["accepted"] for r in meas])) if meas else None,
            "mean_exp_minus_dH": float(ex.mean()) if meas else None,
            "stderr_exp_minus_dH": float(ex.std(ddof=1) / np.sqrt(len(ex))) if len(ex) > 1 else None,
            "mean_dH": float(dh.mean()) if meas else None,
            "dH": [r["dH"] for r in tr], "accepted": [r["accepted"] for r in tr],
            "plaquette_action_per_site": [r["plaquette_action_per_site"] for r in tr],
            "ms_per_trajectory": float(np.median([r["event_ms"] for r in tr])),
            "solves_per_trajectory": tr[-1]["solves"], "iterations_per_trajectory": tr[-1]["iterations"]}


C4_VOLUMES = [(8, 8, 8, 8), (12, 12, 12, 4), (16, 16, 16, 4), (16, 16, 16, 8)]
C4_MASSES = [0.02, 0.05, 0.1]


def run_batch(lq, torch, n_lat=64, n_pf=4, npoles=12, nthreads=16, autotune=True):
    """64 independent lattices (sizes and masses drawn uniformly, seed 7), 4 Gaussian pseudofermions
    each, 12-pole x^{-1/2} shifted CG to 1e-10 in FP32 mode: sequential vs mshift_cg_batch."""
    from paper_1710_09178_gb300 import inputs

    owners, problems, picks, tps = [], [], [], []
    for l in range(n_lat):
        vi = int(inputs.counter_uniform(7, np.array([l], dtype=np.uint64), 0)[0] * len(C4_VOLUMES))
        mi = int(inputs.counter_uniform(7, np.array([l], dtype=np.uint64), 1)[0] * len(C4_MASSES))
        dims, mass = C4_VOLUMES[vi], C4_MASSES[mi]
        picks.append((dims, mass))
        owner = lq.Context(dims, mass)
        owner.set_gauge(torch.from_numpy(inputs.gauge_field(dims, seed=7000 + l)).cuda())
        if autotune:
            tps.append(owner.autotune(lq.FP32))
        owners.append(owner)
        c0, res, poles, _ = lq.rational_coeffs(-0.5, 4 * mass * mass, 16 + 4 * mass * mass, npoles)
        for f in range(n_pf):
            ctx = lq.Context(dims, mass)
            ctx.share_gauge(owner)
            if autotune:
                ctx.set_option(lq.OPT_DSLASH_TPS, tps[-1])
            b = torch.from_numpy(inputs.gaussian_vector(dims, 8 + f * 100000 + l)).cuda()
            xs = [torch.empty_like(b) for _ in range(npoles)]
            problems.append(dict(ctx=ctx, shifts=poles, residues=res, c0=c0, b=b, xs=xs, y=torch.empty_like(b),
                                 tol=1e-10, prec=lq.FP32))
    # the same sources as one multi-right-hand-side problem per lattice (mshift_cg_multi on the owner
    # context: the four pseudofermions share the kernel launches and the FP32 Dslash link loads)
    multi = []
    for l, owner in enumerate(owners):
        mine = problems[l * n_pf:(l + 1) * n_pf]
        multi.append(dict(ctx=owner, shifts=mine[0]["shifts"], residues=mine[0]["residues"], c0=mine[0]["c0"],
                          bs=[p["b"] for p in mine], xss=[[torch.empty_like(p["b"]) for _ in p["xs"]] for p in mine],
                          ys=[torch.empty_like(p["b"]) for p in mine], tol=1e-10, prec=lq.FP32))
    # warm-up (workspace allocation, graph capture), then timed runs
    lq.mshift_cg_batch(problems, nthreads=nthreads)
    lq.mshift_cg_batch(multi, nthreads=min(nthreads, len(multi)))
    torch.cuda.synchronize()
    out = {}
    for name, probs, nt in (("sequential", problems, 1), ("batched", problems, nthreads),
                            ("multi_rhs_batched", multi, min(nthreads, len(multi)))):
        t0 = time.perf_counter()
        rc, st, stats = lq.mshift_cg_batch(probs, nthreads=nt)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        flat = [x for s in stats for x in (s if isinstance(s, list) else [s])]
        out[name] = {"ms": dt * 1e3, "problems_per_s": len(problems) / dt, "status_ok": all(x == 0 for x in st),
                     "max_true_residual": max(max(s["true_residual"]) for s in flat), "host_threads": nt,
                     "solve_calls": len(probs)}
    # the multi-RHS solves against the stand-alone ones (bit-identical when the stand-alone solve runs
    # one thread per site; the autotuned contexts may run more, which reorders the Dslash sums)
    out["multi_rhs_vs_single_max_rel_diff"] = max(
        float(torch.linalg.vector_norm(a - c) / torch.linalg.vector_norm(c))
        for l, mp in enumerate(multi) for f in range(n_pf) for a, c in zip(mp["xss"][f], problems[l * n_pf + f]["xs"]))
    sites = sum(int(np.prod(d)) // 2 for d, _ in picks) * n_pf
    out.update({"lattices": n_lat, "pseudofermions": n_pf, "poles": npoles, "problems": len(problems),
                "even_sites_total": sites, "threads": nthreads,
                "speedup": out["sequential"]["ms"] / out["batched"]["ms"],
                "speedup_multi_rhs": out["sequential"]["ms"] / out["multi_rhs_batched"]["ms"],
                "volumes_drawn": {str(v): sum(1 for d, _ in picks if d == v) for v in C4_VOLUMES},
                "autotuned_tps": {str(v): sorted(set(t for (d, _), t in zip(picks, tps) if d == v)) for v in C4_VOLUMES}
                if autotune else None})
    for p in problems:
        p["ctx"].close()
    for o in owners:
        o.close()
    out["dslash_batch"] = run_batch_dslash(lq, torch, picks)
    return out


def batch_summary(b, peak):
    """The batch workload's headline numbers for the default bench line."""
    d = b["dslash_batch"]["persistent_batch"]
    return {"workload": f"{b['lattices']} lattices (8^4, 12^3x4, 16^3x4, 16^3x8 drawn with seed 7) x "
                        f"{b['pseudofermions']} pseudofermions, {b['poles']}-pole x^-1/2 to 1e-10, FP32 mode",
            "problems": b["problems"],
            "ms_sequential": b["sequential"]["ms"], "ms_batched": b["batched"]["ms"],
            "ms_multi_rhs_batched": b["multi_rhs_batched"]["ms"],
            "problems_per_s_multi_rhs": b["multi_rhs_batched"]["problems_per_s"],
            "problems_per_s_batched": b["batched"]["problems_per_s"],
            "multi_rhs_vs_single_max_rel_diff": b["multi_rhs_vs_single_max_rel_diff"],
            "max_true_residual": max(b[k]["max_true_residual"] for k in ("sequential", "batched", "multi_rhs_batched")),
            "dslash_sweep_us": d["us_per_sweep"], "dslash_sweep_GBps": d["algorithmic_GBps"],
            "dslash_sweep_frac_of_hbm": d["algorithmic_GBps"] / peak,
            "dslash_launches_per_sweep": d["launches_per_sweep"]}


def run_batch_dslash(lq, torch, picks, reps=20):
    """The half-Dslash of every lattice of the batch workload (FP32 links, both parities in turn):
    one persistent dslash_eo_batch launch over all lattices vs one dslash_eo launch per lattice
    (each with its autotuned threads per site), each variant captured reps times in a CUDA graph.
    Returns per-sweep times and algorithmic GB/s."""
    from paper_1710_09178_gb300 import inputs

    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    ctxs, ins, outs = [], [], []
    for l, (dims, mass) in enumerate(picks):
        c = lq.Context(dims, mass, stream=s.cuda_stream)
        c.set_gauge(torch.from_numpy(inputs.gauge_field(dims, seed=7000 + l)).cuda())
        c.autotune(lq.FP32)  # the per-lattice launches use their best threads per site
        vin, vout = c.new_vector(lq.FP32), c.new_vector(lq.FP32)
        vin.view(torch.float32).normal_()
        ctxs.append(c)
        ins.append(vin)
        outs.append(vout)
    torch.cuda.synchronize()
    n = len(ctxs)
    bytes_sweep = sum(DSLASH_BYTES_PER_SITE["fp32"] * (int(np.prod(d)) // 2) for d, _ in picks)

    def batched(r):
        lq.dslash_eo_batch(ctxs, outs, ins, [r & 1] * n, lq.FP32)

    def single(r):
        for c, vi, vo in zip(ctxs, ins, outs):
            lq.dslash_eo(c, vo, vi, r & 1, lq.FP32)

    res = {}
    with torch.cuda.stream(s):
        for name, fn in (("persistent_batch", batched), ("one_launch_per_lattice", single)):
            fn(0)
            fn(1)
            s.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s, capture_error_mode="thread_local"):
                for r in range(reps):
                    fn(r)
            graph.replay()
            ms = []
            for _ in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s)
                graph.replay()
                e1.record(s)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1) / reps)
            m = statistics.median(ms)
            res[name] = {"us_per_sweep": m * 1e3, "algorithmic_GBps": bytes_sweep / (m * 1e-3) / 1e9,
                         "launches_per_sweep": 1 if name == "persistent_batch" else n}
    res["speedup"] = res["one_launch_per_lattice"]["us_per_sweep"] / res["persistent_batch"]["us_per_sweep"]
    res["lattices"] = n
    res["bytes_per_sweep"] = bytes_sweep
    res["timing"] = f"{reps} sweeps per CUDA graph, median of 5 replays"
    for c in ctxs:
        c.close()
    return res


def tiled_field(torch, base_dims, reps, seed):
    """The seeded field of base_dims tiled reps[mu] times along each direction (a valid SU(3) field
    of the larger lattice, periodic with the base extents), built on the device."""
    from paper_1710_09178_gb300 import inputs

    U = torch.from_numpy(inputs.gauge_field(base_dims, seed=seed)).cuda()
    nx, ny, nz, nt = base_dims
    U = U.reshape(nt, nz, ny, nx, 4, 3, 3)  # l = x + nx (y + ny (z + nz t))
    U = U.repeat(reps[3], reps[2], reps[1], reps[0], 1, 1, 1)
    dims = tuple(b * r for b, r in zip(base_dims, reps))
    return dims, U.reshape(-1, 4, 3, 3).contiguous()


def run_formats(lq, torch, dims_list=((32, 32, 32, 8), (48, 48, 48, 12)), reps=20):
    """Every link format of the half-Dslash (FP32 18-real, 12-real, 8-real, 16-bit) with 1, 2 and 4
    threads per site, at 32^3x8 (FP32 links 75.5 MB, inside the L2) and 48^3x12 (382 MB, the
    seeded 24^3x6 field tiled 2x2x2x2): CUDA-event time per launch of a graph of launches
    rotating over enough copies of the field that every launch reads its links from HBM, and the
    mixed solve (16 poles, tol 1e-10) in each format."""
    from paper_1710_09178_gb300 import inputs

    fmts = (("fp32", lq.FP32), ("fp32_r12", lq.FP32_R12), ("fp32_r8", lq.FP32_R8), ("fp32_l16", lq.FP32_L16))
    peak, _ = read_peaks()
    out = {}
    flush = L2Flusher(torch)
    for dims in dims_list:
        if dims == (32, 32, 32, 8):
            U = torch.from_numpy(inputs.gauge_field(dims, seed=GAUGE_SEED)).cuda()
            src = "seeded field, seed 5"
        else:
            dims, U = tiled_field(torch, (24, 24, 24, 6), (2, 2, 2, 2), 9)
            src = "the seeded 24^3x6 field (seed 9) tiled 2x2x2x2"
        vh = int(np.prod(dims)) // 2
        n_fields = max(2, int(np.ceil(2 * 160e6 / (72 * 4 * 2 * vh))) + 1)
        res = {"source": src, "fields_rotated": n_fields}
        for name, prec in fmts:
            row = {}
            for tps in (1, 2, 4):
                s_ = torch.cuda.Stream()
                torch.cuda.synchronize()
                sctx = []
                for _ in range(n_fields):
                    c = lq.Context(dims, MASS, stream=s_.cuda_stream)
                    c.set_gauge(U)
                    c.set_option(lq.OPT_DSLASH_TPS, tps)
                    vin, vout = c.new_vector(prec), c.new_vector(prec)
                    vin.view(torch.float32).normal_()
                    sctx.append((c, vin, vout))
                with torch.cuda.stream(s_):
                    for i in range(2 * n_fields):
                        c, vin, vout = sctx[i % n_fields]
                        lq.dslash_eo(c, vout, vin, (i // n_fields) & 1, prec)
                    s_.synchronize()
                    g = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(g, stream=s_, capture_error_mode="thread_local"):
                        for i in range(reps * n_fields):
                            c, vin, vout = sctx[i % n_fields]
                            lq.dslash_eo(c, vout, vin, (i // n_fields) & 1, prec)
                    g.replay()
                    ms = []
                    for _ in range(3):
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(s_)
                        g.replay()
                        e1.record(s_)
                        e1.synchronize()
                        ms.append(e0.elapsed_time(e1) / (reps * n_fields))
                torch.cuda.synchronize()
                for c, _, _ in sctx:
                    c.close()
                m = statistics.median(ms)
                gbs = DSLASH_BYTES_PER_SITE[name] * vh / (m * 1e-3) / 1e9
                row[f"tps{tps}"] = {"us": m * 1e3, "algorithmic_GBps": gbs, "frac_of_hbm": gbs / peak}
            # the mixed solve in this format
            ctx = lq.Context(dims, MASS)
            ctx.set_gauge(U)
            b = torch.from_numpy(inputs.gaussian_vector(dims, VEC_SEED)).cuda()
            c0, rr, poles, _ = lq.rational_coeffs(-0.5, 4 * MASS * MASS, 16 + 4 * MASS * MASS, NPOLES)
            xs = [torch.empty_like(b) for _ in poles]
            tms, sts = time_solves(lq, torch, ctx, b, xs, None, (c0, rr, poles, None), prec, 3, 1, flush)
            row["solve_ms"] = statistics.median(tms)
            row["solve_iterations"] = sts[-1]["iterations"]
            row["solve_refine_iterations"] = sts[-1]["refine_iterations"]
            row["solve_max_true_residual"] = max(sts[-1]["true_residual"])
            ctx.close()
            res[name] = row
        out["x".join(str(d) for d in dims)] = res
    return out


def run_profile_target(kind, prec_name):
    """Small fixed workloads for ncu (no timing): `dslash` = 8 half-Dslash launches at 32^3x8,
    `dslash48` = the same at 48^3x12 (the seeded 24^3x6 field tiled 2x2x2x2, FP32 links 382 MB),
    `dslash_graph` = the roofline's graph of 96 launches over 8 gauge fields (16 warm-up launches,
    then 6 replays of the graph: 592 launches), `df_dslash` = 8 double-FP32 half-Dslash launches,
    `solve` = one shifted-CG solve with CUDA graphs off, so that every kernel is a separate launch,
    `solve_graph` = two solves with CUDA graphs on (the second is the timed configuration),
    `multi` = the same for four sources solved together (mshift_cg_multi)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_1710_09178_gb300 as lq
    from paper_1710_09178_gb300 import inputs

    prec = lq.PRECISIONS[prec_name]
    if kind == "dslash48":
        # the link-format sweep's large lattice: links far beyond L2
        dims48, U48 = tiled_field(torch, (24, 24, 24, 6), (2, 2, 2, 2), 9)
        ctx = lq.Context(dims48, MASS)
        ctx.set_gauge(U48)
        vin = ctx.new_vector(prec)
        vout = ctx.new_vector(prec)
        vin.view(torch.float32 if prec != lq.FP64 else torch.float64).normal_()
        for r in range(8):
            lq.dslash_eo(ctx, vout, vin, r & 1, prec)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "dslash48", "dims": list(dims48), "prec": prec_name}))
        ctx.close()
        return
    ctx = lq.Context(DIMS, MASS)
    ctx.set_gauge(torch.from_numpy(inputs.gauge_field(DIMS, seed=GAUGE_SEED)).cuda())
    if kind == "dslash_graph":
        ms = time_dslash_graph(lq, torch, torch.from_numpy(inputs.gauge_field(DIMS, seed=GAUGE_SEED)).cuda(), prec, 96)
        print(json.dumps({"profile": "dslash_graph", "ms_per_launch": ms}))
    elif kind == "df_dslash":
        vin = ctx.new_vector(lq.DF64)
        vout = ctx.new_vector(lq.DF64)
        vin.view(torch.float32).normal_()
        for r in range(8):
            lq.dslash_eo(ctx, vout, vin, r & 1, lq.DF64)
    elif kind == "dslash":
        vin = ctx.new_vector(prec)
        vout = ctx.new_vector(prec)
        vin.view(torch.float32 if prec != lq.FP64 else torch.float64).normal_()
        for r in range(8):
            lq.dslash_eo(ctx, vout, vin, r & 1, prec)
    elif kind == "solve_graph":
        # two solves with CUDA graphs on (the first captures the graph): the second one's kernel nodes
        # are what the timed solve runs
        b = torch.from_numpy(inputs.gaussian_vector(DIMS, VEC_SEED)).cuda()
        c0, res, poles, _ = lq.rational_coeffs(-0.5, 4 * MASS * MASS, 16 + 4 * MASS * MASS, NPOLES)
        xs = [torch.empty_like(b) for _ in range(NPOLES)]
        y = torch.empty_like(b)
        for _ in range(2):
            rc, st = lq.mshift_cg(ctx, poles, res, c0, b, xs, y, tol=TOL, prec=prec)
        print(json.dumps({"profile": "solve_graph", "rc": rc, "iterations": st["iterations"],
                          "refine_iterations": st["refine_iterations"], "launches_per_solve": st["kernel_launches"]}))
    elif kind == "multi":
        # four sources solved together (mshift_cg_multi), graphs off
        ctx.set_option(lq.OPT_USE_GRAPH, 0)
        bs = [torch.from_numpy(inputs.gaussian_vector(DIMS, VEC_SEED + 100 * s)).cuda() for s in range(4)]
        c0, res, poles, _ = lq.rational_coeffs(-0.5, 4 * MASS * MASS, 16 + 4 * MASS * MASS, NPOLES)
        rc, sts = lq.mshift_cg_multi(ctx, poles, res, c0, bs, None, None, tol=TOL, prec=prec)
        print(json.dumps({"profile": "multi", "rc": rc, "iterations": [s["iterations"] for s in sts],
                          "refine_iterations": [s["refine_iterations"] for s in sts],
                          "launches": ctx.launch_count()}))
    else:
        ctx.set_option(lq.OPT_USE_GRAPH, 0)
        b = torch.from_numpy(inputs.gaussian_vector(DIMS, VEC_SEED)).cuda()
        c0, res, poles, _ = lq.rational_coeffs(-0.5, 4 * MASS * MASS, 16 + 4 * MASS * MASS, NPOLES)
        xs = [torch.empty_like(b) for _ in range(NPOLES)]
        y = torch.empty_like(b)
        rc, st = lq.mshift_cg(ctx, poles, res, c0, b, xs, y, tol=TOL, prec=prec)
        print(json.dumps({"profile": "solve", "rc": rc, "iterations": st["iterations"],
                          "refine_iterations": st["refine_iterations"], "launches": ctx.launch_count()}))
    torch.cuda.synchronize()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="mixed mode only")
    ap.add_argument("--profile", choices=["dslash", "dslash48", "dslash_graph", "df_dslash", "solve", "solve_graph", "multi"],
                    help="run a small fixed workload for ncu and exit")
    ap.add_argument("--prec", default="fp32", choices=["fp64", "fp32", "fp32_r12", "fp16fix", "fp32_r8", "fp32_l16", "df64"])
    ap.add_argument("--rhmc", type=int, default=0, help="run N RHMC trajectories on 24^3x6, print one JSON line")
    ap.add_argument("--traj-steps", type=int, default=TRAJ_STEPS, help="Omelyan steps per trajectory for --rhmc")
    ap.add_argument("--therm", type=int, default=20, help="thermalising trajectories before the --rhmc ones")
    ap.add_argument("--rhmc-meas", type=int, default=12, help="Metropolis trajectories of the default run's RHMC part")
    ap.add_argument("--batch", action="store_true", help="run the 64-lattice batched workload, print one JSON line")
    ap.add_argument("--formats", action="store_true", help="link formats x threads per site at 32^3x8 and 48^3x12")
    args = ap.parse_args()
    if args.formats:
        import torch

        import __graft_entry__

        __graft_entry__.build()
        import paper_1710_09178_gb300 as lq

        print(json.dumps({"formats": run_formats(lq, torch)}), flush=True)
        return
    if args.batch:
        import torch

        import __graft_entry__

        __graft_entry__.build()
        import paper_1710_09178_gb300 as lq

        print(json.dumps({"batch": run_batch(lq, torch)}), flush=True)
        return
    if args.rhmc:
        import torch

        import __graft_entry__

        __graft_entry__.build()
        import paper_1710_09178_gb300 as lq

        tr = run_trajectories(lq, torch, args.rhmc + args.therm, nsteps=args.traj_steps, n_therm=args.therm)
        print(json.dumps({"rhmc": rhmc_summary(tr, args.traj_steps)}), flush=True)
        return
    if args.profile:
        run_profile_target(args.profile, args.prec)
        return
    args.warmup = max(args.warmup, 3)

    rank = env_int("RANK", 0)
    world = env_int("WORLD_SIZE", 1)
    local_rank = env_int("LOCAL_RANK", 0)

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)

    import __graft_entry__

    __graft_entry__.build()
    import paper_1710_09178_gb300 as lq

    U, b, coeffs = setup_problem(lq, torch)
    ctx = lq.Context(DIMS, MASS)
    Ud = torch.from_numpy(U).cuda()
    ctx.set_gauge(Ud)
    bd = torch.from_numpy(b).cuda()
    xs = [torch.empty_like(bd) for _ in range(NPOLES)]
    y = torch.empty_like(bd)
    flush_buf = L2Flusher(torch)
    launches0 = ctx.launch_count()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- headline: mixed-precision solve ------------------------------------------------
    clocks = ClockSampler(local_rank)
    barrier()
    clocks.start()
    t_wall0 = time.perf_counter()
    times, stats = time_solves(lq, torch, ctx, bd, xs, y, coeffs, lq.FP32, args.steps, args.warmup, flush_buf)
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches_timed = sum(s["kernel_launches"] for s in stats)
    total_ms, ms_per_solve, value = replica_aggregate(sum(times), args.steps, world, dist, "cuda")
    results = {"fp32": ([x.cpu().numpy() for x in xs], y.cpu().numpy())}  # per-result errors vs the oracle

    extra = {}
    if not args.quick:
        # FP64 solve (the plain method) and the other storage modes
        for name, prec in (("fp64", lq.FP64), ("df64", lq.DF64), ("fp32_r12", lq.FP32_R12), ("fp16fix", lq.FP16FIX),
                           ("fp32_r8", lq.FP32_R8), ("fp32_l16", lq.FP32_L16)):
            tms, sts = time_solves(lq, torch, ctx, bd, xs, y, coeffs, prec, max(2, args.steps // 2), 1, flush_buf)
            results[name] = ([x.cpu().numpy() for x in xs], y.cpu().numpy())
            extra[name] = {"ms_per_solve": statistics.mean(tms), "iterations": sts[-1]["iterations"],
                           "algorithmic_GBps": solve_algorithmic_bytes(sts[-1], int(np.prod(DIMS)) // 2,
                                                                       prec in (lq.FP64, lq.DF64))
                           / (statistics.mean(tms) * 1e6),
                           "reliable_updates": sts[-1]["reliable_updates"],
                           "refine_iterations": sts[-1]["refine_iterations"],
                           "max_true_residual": max(sts[-1]["true_residual"])}
        # the heatbath's x^{1/4} (residues c_k < 0, c0 > 0) on the same interval, mixed and FP64
        lo, hi = 4 * MASS * MASS, 16 + 4 * MASS * MASS
        q_coeffs = lq.rational_coeffs(0.25, lo, hi, NPOLES)
        for name, prec in (("fp32_x^1/4", lq.FP32), ("fp64_x^1/4", lq.FP64)):
            tms, sts = time_solves(lq, torch, ctx, bd, xs, y, q_coeffs, prec, max(2, args.steps // 2), 1, flush_buf)
            extra[name] = {"ms_per_solve": statistics.mean(tms), "iterations": sts[-1]["iterations"],
                           "reliable_updates": sts[-1]["reliable_updates"],
                           "refine_iterations": sts[-1]["refine_iterations"],
                           "max_true_residual": max(sts[-1]["true_residual"]),
                           "approximation_error": q_coeffs[3]}

    # ---- Dslash roofline (the kernel that dominates the solve) ------------------------------
    peak, peak_kind = read_peaks()
    vh = int(np.prod(DIMS)) // 2
    dsl = {}
    for name, prec in (("fp32", lq.FP32), ("fp32_r12", lq.FP32_R12), ("fp32_r8", lq.FP32_R8),
                       ("fp32_l16", lq.FP32_L16), ("fp64", lq.FP64)):
        if args.quick and name != "fp32":
            continue
        mean_ms, med_ms = time_dslash(lq, torch, ctx, name, prec, 40, flush_buf)
        gbs = DSLASH_BYTES_PER_SITE[name] * vh / (mean_ms * 1e-3) / 1e9
        dsl[name] = {"ms": mean_ms, "median_ms": med_ms, "algorithmic_GBps": gbs, "frac_of_hbm": gbs / peak,
                     "gflops": DSLASH_FLOPS_PER_SITE * vh / (mean_ms * 1e-3) / 1e9}
    if "fp64" in dsl:
        # the FP64 Dslash against GB300's FP64 rate, measured here with cuBLAS DGEMM (the FP64 pipe's
        # ceiling for plain FP64 arithmetic)
        f64 = fp64_peak_tflops(torch)
        dsl["fp64"]["fp64_peak_tflops_dgemm"] = f64
        dsl["fp64"]["frac_of_fp64_peak"] = dsl["fp64"]["gflops"] / 1e3 / f64
    traffic = profiled_traffic(WORKLOAD)
    d32 = dsl["fp32"]
    sctx = make_stream_contexts(lq, torch, Ud, STREAM_FIELDS)
    s_ms = statistics.median(time_dslash_stream(lq, torch, sctx, lq.FP32, 96) for _ in range(5))
    for c, _, _ in sctx:
        c.close()
    del sctx
    g_ms = time_dslash_graph(lq, torch, Ud, lq.FP32, 96)
    bpl = DSLASH_BYTES_PER_SITE["fp32"] * vh
    streamed = {"ms": s_ms, "achieved": bpl / (s_ms * 1e-3) / 1e9, "frac": bpl / (s_ms * 1e-3) / 1e9 / peak,
                "timing": f"96 back-to-back stream launches rotating over {STREAM_FIELDS} gauge fields "
                          f"({STREAM_FIELDS} x 75.5 MB > L2: every launch reads from HBM), median of 5"}
    isolated = {"ms": d32["ms"], "achieved": d32["algorithmic_GBps"], "frac": d32["algorithmic_GBps"] / peak,
                "timing": "one launch after an L2 flush, launch latency included, mean of 40"}
    if g_ms is not None:
        r_ms, r_timing = g_ms, (f"the same 96 launches over {STREAM_FIELDS} gauge fields captured in one CUDA "
                                f"graph (as in the solver), median of 5 replays")
    else:
        r_ms, r_timing = s_ms, streamed["timing"]
    r_gbs = bpl / (r_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": r_gbs, "peak": peak, "unit": "GB/s",
                "frac": r_gbs / peak, "traffic": traffic, "kernel": "dslash_kernel<L32> (FP32)",
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, burst)" if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "bytes_per_launch": bpl, "ms_per_launch": r_ms, "timing": r_timing,
                "stream_launches": streamed, "isolated_launch": isolated}

    # ---- the double-FP32 Dslash: the largest share of the mixed solve's time (its first phase and
    # every true-residual check), bound by FP32 instruction issue; peak = SMs x 128 FP32 lanes x the
    # maximum SM clock (2070 MHz), one operation per lane and cycle (an FMA counts as one) ----------
    roofline_df = None
    if not args.quick:
        df_ms = time_df_dslash_graph(lq, torch, Ud)
        if df_ms is not None:
            n_sm = torch.cuda.get_device_properties(0).multi_processor_count
            alu_peak = n_sm * 128 * 2070e6 / 1e12  # T FP32 operations per second
            ops = DF_OPS_PER_SITE * vh / (df_ms * 1e-3) / 1e12
            df_gbs = DF_BYTES_PER_SITE * vh / (df_ms * 1e-3) / 1e9
            roofline_df = {"bound": "alu", "achieved": ops, "peak": alu_peak, "unit": "T FP32 op/s", "frac": ops / alu_peak,
                           "traffic": profiled_traffic(WORKLOAD, "df_dslash_32c8.json", ("df64.cu", "common.cuh")),
                           "kernel": "df_dslash_kernel<plain> (double-FP32 links and vectors)",
                           "peak_kind": f"derived: {n_sm} SMs x 128 FP32 lanes x 2070 MHz",
                           "ops_per_site": DF_OPS_PER_SITE, "bytes_per_launch": DF_BYTES_PER_SITE * vh,
                           "ms_per_launch": df_ms, "algorithmic_GBps": df_gbs, "frac_of_hbm": df_gbs / peak,
                           "timing": "64 launches (alternating parities) in one CUDA graph, median of 5 replays"}

    # ---- end to end through the C ABI with host buffers ------------------------------------
    c0, res, poles, _ = coeffs
    b_host = torch.from_numpy(b).pin_memory()
    y_host = torch.empty_like(b_host).pin_memory()
    e2e_ms = []
    stream = torch.cuda.current_stream()
    for i in range(args.steps + 1):
        flush_buf.add_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bd.copy_(b_host, non_blocking=True)
        lq.mshift_cg(ctx, poles, res, c0, bd, xs, y, tol=TOL, prec=lq.FP32)
        y_host.copy_(y, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if i > 0:
            e2e_ms.append(e0.elapsed_time(e1))
    assert np.array_equal(y_host.numpy(), y.cpu().numpy())
    nbytes = b.nbytes

    # ---- one RHMC trajectory on 24^3x6 (NEXT rows: force + integrator), after one warm-up ----
    traj = None
    batch = None
    if not args.quick:
        # 20 thermalising trajectories from the synthetic start (accepted whatever their dH), then 12
        # with the Metropolis test: acceptance and <exp(-dH)> of the equilibrated chain
        tr = run_trajectories(lq, torch, args.therm + args.rhmc_meas, n_therm=args.therm)
        traj = rhmc_summary(tr, TRAJ_STEPS)
        traj["start"] = ("the synthetic exp(i 0.5 H) field, thermalised by the first trajectories (accepted whatever "
                         "their dH); the summary statistics cover the Metropolis trajectories after them")
        # the batched workload: 64 lattices x 4 pseudofermions
        batch = batch_summary(run_batch(lq, torch), read_peaks()[0])

    # ---- CPU baseline: the C++ FP64 oracle's complete solve on the host cores; GPU errors against it ----
    cpu = None
    errors = None
    if rank == 0 and not args.no_cpu_baseline:
        oc, sol = cpu_oracle_solves(U, b, coeffs)
        a, o = oc["all_cores"], oc["one_core"]
        cpu = {"value": a["ms_per_solve"], "unit": "ms/solve", "cores": a["threads"], "kind": "oracle",
               "host": host_cpu(),
               "sample": f"one complete solve of the workload (32^3x8, 16 shifts, true residual 1e-10, "
                         f"{a['iterations']} iterations) by the C++ FP64 oracle with OpenMP on {a['threads']} "
                         f"threads; the same solve on one core beside it",
               "all_cores": a, "one_core": o}
        errors = {name: errors_vs_oracle(xr, yr, sol) for name, (xr, yr) in results.items()}
        errors["note"] = ("|x_k - x_k^oracle| / |x_k^oracle| per shift (shift order of the poles) and the same for "
                          "y = c0 b + sum c_k x_k; both sides solved to a true residual of 1e-10, so each x_k "
                          "difference is bounded by about 2 kappa_k 1e-10 (kappa_k = (16 + 4m^2 + d_k) / "
                          "(4m^2 + d_k))")

    last = stats[-1]
    line = {
        "metric": METRIC, "value": value, "unit": "ms/solve", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_solve, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": list(DIMS), "mass": MASS, "poles": NPOLES,
                   "approximation": "x^-1/2 on [4m^2, 16+4m^2], Zolotarev (n,n)", "tol": TOL,
                   "precision": "double-FP32 (FP32 hi/lo) first phase until |r| <= 1e-3 |b|, then FP32 links+Krylov vectors; double-FP32 dots, x_k, reliable updates and true residuals; FP64 per-shift recurrences; 12-real FP32 links in the refinement",
                   "gauge": "exp(i 0.5 H) SU(3), seed 5", "source": "complex Gaussian, seed 6",
                   "l2": "flushed (256 MB written, then another 256 MB read) between timed steps and before every "
                         "isolated Dslash launch; the graph-launched Dslash of the roofline rotates over "
                         "8 gauge fields (604 MB of links > L2)",
                   "parallelism": f"replicas x{world}"},
        "mixed": {"iterations": last["iterations"], "shift_iterations": last["shift_iterations"],
                  "algorithmic_GBps": solve_algorithmic_bytes(last, int(np.prod(DIMS)) // 2, False) / (ms_per_solve * 1e6),
                  "algorithmic_bytes_note": "plain shifted CG base iterations (A-apply, r/p updates, active-shift "
                                            "p_k/x_k updates) / whole solve time incl. checks and refinement",
                  "reliable_updates": last["reliable_updates"],
                  "refine_iterations": last["refine_iterations"], "refined_shifts": last["refined_shifts"],
                  "max_true_residual": max(last["true_residual"]), "ms_per_solve_all": times},
        "fp64_vs_mixed": (extra["fp64"]["ms_per_solve"] / ms_per_solve) if "fp64" in extra else None,
        "fp64_vs_df64": (extra["fp64"]["ms_per_solve"] / extra["df64"]["ms_per_solve"]) if "df64" in extra else None,
        "modes": extra,
        "dslash": dsl,
        "roofline": roofline,
        "roofline_df": roofline_df,
        "e2e": {"value": statistics.mean(e2e_ms), "unit": "ms/solve", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "rhmc_trajectory": traj,
        "batch": batch,
        "gpu_launches": launches_timed,
        "clocks": clk,
        "wall_s_timed": t_wall,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
        line["errors_vs_oracle"] = errors
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

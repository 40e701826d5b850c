#!/usr/bin/env python3
"""Benchmark of the RBF neural-field hot path on one GB300.

Workload (the precision configuration): torus R = 1, r = 0.4 with n = 100,000
jittered spiral-lattice nodes, k = 48 stencils, PHS r^3 + degree-4 polynomials,
Mexican-hat kernel (1, 0.1, 0.5, 0.2), sigmoid beta = 50, theta = 0.2, six bumps as
u0, RK4 with dt = 0.05, one trajectory.  Stencils and quadrature weights are built
on the GPU first (setup, not timed in `value`).

A step is one RK4 step (four stages, each: nonlocal sum of Eq. (2.9) over all
n^2 pairs + fused stage update).  `value` is pair evaluations per second
(4 n^2 per step) of the fastest path; every path is reported under `paths`:
  mf          matrix-free FP32 pair kernel (TMA-staged tiles, SFU exponentials)
  dense_fp32  precomputed W diag(q) in FP32, HBM-streamed GEMV
  bf16x2      precomputed W diag(q)/s_i as bf16 hi + lo planes, FP32 accumulate
Timing: CUDA events on the launching stream around each step, L2 flushed (a
256 MiB write) between timed steps; the dominant kernel is timed live by events
captured around it inside the step graph.  With --gpus N under torchrun every rank
runs an independent replica (the single-trajectory path does not shard without a
per-stage all-gather), value = all ranks' pairs / max time ("weak" scaling).

--impl reference times the FP64 CPU oracle (the reference arm of the measurement) on a
bounded sample of the same workload: a step is one nonlocal stage over a row sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PATHS = {"mf": 0, "dense_fp32": 1, "bf16x2": 2, "dense_sym": 4, "dense_sym_bf16x2": 5}
METRIC = "pair-evals/s & RK4 steps/s at N=1e5, mixed/batched vs plain FP32, same GB300"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--paths", default="mf,dense_fp32,bf16x2,dense_sym,dense_sym_bf16x2")
    ap.add_argument("--n", type=int, default=100000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched tensor-core section")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the differentiation section")
    ap.add_argument("--no-models", action="store_true", help="skip the §5 models section (depression, AB5)")
    ap.add_argument("--no-geometries", action="store_true", help="skip the curved-geometry weights section")
    ap.add_argument("--no-periodic", action="store_true", help="skip the periodic-square section")
    ap.add_argument("--no-configs", action="store_true", help="skip the flat and sphere configurations")
    ap.add_argument("--convergence", action="store_true",
                    help="run the manufactured-solution convergence studies on the periodic square and the torus")
    ap.add_argument("--batched-scale", type=float, default=1.0,
                    help="scale the batched node counts (profiling captures use a smaller case)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while a region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [v.strip() for v in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return out
        sm = [r[0] for r in rows]
        mx = max(r[1] for r in rows)
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        out.update(sm_mhz=float(np.median(loaded)), sm_max_mhz=mx, reasons=reasons, samples=len(rows))
        return out


# ----------------------------------------------------------------------------- helpers
def max_over_ranks(values, world, device=None):
    """Element-wise maximum of per-rank timings (a timing reduction, not a data path)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def whole_job_rate(units_per_rank, world, max_ms):
    """Units processed by all replicas per second, timed by the slowest rank."""
    return world * float(units_per_rank) / (max_ms * 1e-3)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# Lane operations per ordered pair of the symmetric matrix-free kernel in its expanded form
# with s2^2 / s1^2 = 4 (the workload's kernel): per unordered pair 3 FMA (exponent) +
# 2 MUL (e1 = e2^4) + 1 FMA (pair weight e2 + c_i e1) + 1 FMA (row sum) + 1 FMA (column
# sum), plus per column and 8-row pass 3 SUB + 3 FMA (centred column and n_j) and 1 ADD
# (column sums into shared memory): 8.875 per unordered pair, 4.4375 per ordered pair; and
# one SFU exponential per unordered pair.  Diagonal block pairs evaluate their ordered
# pairs one by one, a 1/nb share of the work.  The rates these counts are divided by (FP32 FMA-pipe lane operations and SFU ex2
# per clock per SM) are measured in the same run by nf_probe_pipe; the nominal figures
# (128 FP32 lanes, 16 SFU operations per clock per SM) are kept only as a fallback.
FMA_LANES_PER_CLK_SM_NOMINAL = 128.0
LANE_OPS_PER_PAIR = 8.875 / 2.0
EX2_PER_PAIR = 0.5

# DRAM bytes (read + write) per launch from ncu captures of the current kernels:
# mf_sym_kernel<8, 4> on the n = 100,000 torus (--set full); tc_grouped_kernel<4> (an RK4
# stage-4 launch) on the full batched workload (dram__bytes_read/write.sum, one pass)
MF_TRAFFIC_BYTES = 2.182e6 + 0.140e6
TC_TRAFFIC_BYTES = 11.90e9 + 0.214e9


def run_reference(args, rank, world):
    """FP64 CPU oracle on bounded row samples of the same workload."""
    import oracle
    from nodesets import workloads as W

    if rank != 0:
        return None
    wl = W.precision(args.n)
    x = wl.ns.nodes.astype(np.float32).astype(np.float64)
    q = np.full(wl.n, wl.ns.area / wl.n)
    u = wl.u0.astype(np.float32).astype(np.float64)
    kern = tuple(float(np.float32(v)) for v in wl.kernel)
    rng = np.random.default_rng(0)
    # calibrate a row sample to about (cpu-seconds / steps) per step
    t = time.perf_counter()
    oracle.nonlocal_sum(x, q, u, kern, wl.beta, wl.theta, rows=np.arange(32))
    per_row = (time.perf_counter() - t) / 32
    budget = max(1.0, args.cpu_seconds * 2 / max(1, args.steps + args.warmup))
    rows_per_step = int(min(wl.n, max(16, budget / per_row)))
    for _ in range(args.warmup):
        oracle.nonlocal_sum(x, q, u, kern, wl.beta, wl.theta, rows=rng.choice(wl.n, rows_per_step, replace=False))
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.nonlocal_sum(x, q, u, kern, wl.beta, wl.theta, rows=rng.choice(wl.n, rows_per_step, replace=False))
    dt = time.perf_counter() - t
    value = rows_per_step * wl.n * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"precision torus n={wl.n}", "rows_per_step": rows_per_step, "B": 1},
        "cpu_baseline": {"value": value, "unit": "pair-evals/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{rows_per_step} random rows x {wl.n} columns of one nonlocal stage per step"},
        "e2e": {"value": value, "unit": "pair-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return line


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def cpu_baseline(wl, q32, seconds, gpu_sums):
    """The FP64 oracle's nonlocal sum of the first stage input on the host cores, timed on
    a bounded random row sample; its values on that sample also give each GPU path's
    relative L2 error (gpu_sums: path -> the path's sum of the same input)."""
    import oracle

    x = f32(wl.ns.nodes)
    u = f32(wl.u0)
    kern = tuple(float(np.float32(v)) for v in wl.kernel)
    beta, theta = f32(wl.beta), f32(wl.theta)
    t = time.perf_counter()
    oracle.nonlocal_sum(x, q32, u, kern, beta, theta, rows=np.arange(32))
    per_row = (time.perf_counter() - t) / 32
    rows = int(min(wl.n, max(64, seconds / per_row)))
    sel = np.random.default_rng(1).choice(wl.n, rows, replace=False)
    t = time.perf_counter()
    want = np.asarray(oracle.nonlocal_sum(x, q32, u, kern, beta, theta, rows=sel)).ravel()
    dt = time.perf_counter() - t
    acc = {p: float(np.linalg.norm(got[sel] - want) / np.linalg.norm(want)) for p, got in gpu_sums.items()}
    cores = oracle.num_threads()
    # the same sum on one thread, on a tenth of the sample
    oracle.set_threads(1)
    try:
        sel1 = sel[: max(16, rows // (10 * max(1, cores // 16)))]
        t = time.perf_counter()
        oracle.nonlocal_sum(x, q32, u, kern, beta, theta, rows=sel1)
        dt1 = time.perf_counter() - t
    finally:
        oracle.set_threads(0)
    # setup (stencils + weights) on a sample of elements, all cores
    ns = wl.ns
    esel = np.random.default_rng(2).choice(ns.m, 2000, replace=False)
    t = time.perf_counter()
    st = oracle.knn(ns.nodes, ns.tris, wl.k, elems=esel)
    nbr = oracle.tri_neighbors(ns.tris)
    for e, sten in zip(esel, st):
        oracle.surface_element_weights(ns.nodes, ns.normals, ns.tris, nbr, int(e), sten, wl.deg)
    dts = time.perf_counter() - t
    return {"value": rows * wl.n / dt, "unit": "pair-evals/s", "cores": cores, "kind": "oracle",
            "sample": f"one nonlocal stage on {rows} random rows x {wl.n} columns (FP64, {dt:.1f} s)",
            "single_thread": {"value": len(sel1) * wl.n / dt1, "unit": "pair-evals/s", "cores": 1,
                              "sample": f"{len(sel1)} rows x {wl.n} columns ({dt1:.1f} s)"},
            "setup": {"elements_per_s": len(esel) / dts, "elements": int(ns.m),
                      "extrapolated_full_setup_s": ns.m / (len(esel) / dts),
                      "sample": f"stencils (k = {wl.k}) and surface weights (deg {wl.deg}) of 2000 random "
                                f"elements, one element after another ({dts:.1f} s); the per-element weights "
                                "run serially in this sample"}}, acc


def batched_accuracy(wls, xs, qs, u0, beta, theta, got, rows_per_group=8):
    """Relative L2 error of the batched path's first-stage sums against the FP64 oracle on
    a few sampled rows of every node set (all trajectories); part of the CPU-baseline leg."""
    import oracle

    rng = np.random.default_rng(2)
    err2 = ref2 = 0.0
    off = toff = 0
    for wl, x, q in zip(wls, xs, qs):
        rows = rng.choice(wl.n, rows_per_group, replace=False)
        ub = u0[off:off + wl.B * wl.n].reshape(wl.B, wl.n)
        want = np.asarray(oracle.nonlocal_sum(f32(x), f32(q), f32(ub), tuple(float(np.float32(v)) for v in wl.kernel),
                                              f32(beta[toff:toff + wl.B]), f32(theta[toff:toff + wl.B]), rows=rows))
        g = got[off:off + wl.B * wl.n].reshape(wl.B, wl.n)[:, rows]
        err2 += float(np.sum((g - want) ** 2))
        ref2 += float(np.sum(want ** 2))
        off += wl.B * wl.n
        toff += wl.B
    return (err2 / ref2) ** 0.5


def run_batched(args, dev, steps, pipes=None):
    """Batched workload: 448 trajectories on four node sets.  Tensor-core path (grouped
    tcgen05 GEMM, bf16 x 3) against two plain FP32 comparators on the same node sets and
    the same fused RK4 stage kernel: the dense FP32 operators with the SIMT FP32 GEMM
    (W streamed from HBM, FFMA on the CUDA cores), and the matrix-free FP32 pair kernel."""
    import torch

    import paper_2504_13379_gb300 as nf
    from nodesets import workloads as W

    stream = torch.cuda.current_stream(dev)
    sizes = tuple(int(round(s * args.batched_scale / 2) * 2) for s in (40000, 8000, 15000, 30000))
    wls = W.batched(sizes=sizes)
    qs, xs = [], []
    t0 = time.perf_counter()
    for wl in wls:
        nodes = torch.as_tensor(wl.ns.nodes, device=dev)
        tris = torch.as_tensor(wl.ns.tris, device=dev)
        st = nf.nf_build_stencils(nodes, tris, wl.k)
        q = nf.nf_quad_weights(nodes, tris, st, wl.deg, normals=torch.as_tensor(wl.ns.normals, device=dev))
        qs.append(q.to(torch.float32).contiguous())
        xs.append(torch.as_tensor(wl.ns.nodes.astype(np.float32), device=dev))
    torch.cuda.synchronize(dev)
    setup_ms = 1e3 * (time.perf_counter() - t0)
    pairs_per_stage = float(sum(wl.B * wl.n * wl.n for wl in wls))
    w_bytes = float(sum(4 * wl.n * wl.n for wl in wls))
    flops = float(sum(3 * 2 * wl.B * wl.n * wl.n for wl in wls))
    u0 = torch.cat([torch.as_tensor(wl.u0.astype(np.float32), device=dev).reshape(-1) for wl in wls])
    beta = torch.cat([torch.as_tensor(wl.beta.astype(np.float32), device=dev) for wl in wls])
    theta = torch.cat([torch.as_tensor(wl.theta.astype(np.float32), device=dev) for wl in wls])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {"workload": f"sphere {sizes[0]} x 256 traj + ellipsoids (1:0.8:0.6) {sizes[1]}/{sizes[2]}/{sizes[3]} "
                       f"x 64 traj, k=32 deg=3",
           "setup_ms": setup_ms, "pair_evals_per_stage": pairs_per_stage}

    def timed(step_fn, nsteps, history_fn=None):
        """Mean step time over nsteps back-to-back steps (L2 flushed between them); with
        history_fn, the mean nonlocal-kernel time per launch read after the loop."""
        for _ in range(3):
            step_fn()
        torch.cuda.synchronize(dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            step_fn()
            b.record(stream)
        torch.cuda.synchronize(dev)
        tot = sum(a.elapsed_time(b) for a, b in evs)
        kern = float(sum(sum(st) for st in history_fn(nsteps))) if history_fn else None
        return tot / nsteps, (kern / (4 * nsteps) if history_fn else None)

    # ---- tensor-core path
    t0 = time.perf_counter()
    ops = [nf.Operator(x, q, wl.kernel, nf.DENSE_BF16X2) for x, q, wl in zip(xs, qs, wls)]
    grp = nf.GroupedOperator(ops, [wl.B for wl in wls])
    torch.cuda.synchronize(dev)
    build_ms = 1e3 * (time.perf_counter() - t0)
    grp.profile(True, ring=steps)
    first_sums = nf.nf_nonlocal_apply(grp, u0.view(1, -1), beta, theta).double().cpu().numpy().ravel()
    u = u0.clone()
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    ms, kms = timed(lambda: nf.nf_rk4_advance(grp, u, 0.0, 0.05, 1, beta, theta), steps, grp.kernel_ms_history)
    clocks = sampler.stop()
    grp.check()
    pk = peaks()
    hbm = w_bytes / (kms * 1e-3) / 1e9
    tfl = flops / (kms * 1e-3) / 1e12
    hbm_peak = pk.get("hbm_gbs", 6800.0)
    tc_peak = pk.get("bf16_tflops_sustained", 1700.0)
    out["tc_bf16x3"] = {
        "ms_per_step": ms, "rk4_steps_per_s": 1e3 / ms, "pair_evals_per_s": 4 * pairs_per_stage / (ms * 1e-3),
        "kernel_ms_per_launch": kms, "build_ms": build_ms, "clocks": clocks,
        "roofline": {"bound": "hbm" if hbm / hbm_peak >= tfl / tc_peak else "tensor",
                     "traffic": TC_TRAFFIC_BYTES if args.batched_scale == 1.0 else None,
                     "traffic_unit": "bytes per launch",
                     "hbm": {"achieved": hbm, "peak": hbm_peak, "unit": "GB/s", "frac": hbm / hbm_peak},
                     "tensor": {"achieved": tfl, "peak": tc_peak, "unit": "TFLOP/s", "frac": tfl / tc_peak,
                                "peak_basis": "MEASURED_PEAKS bf16_tflops_sustained (kernel inside a long step)"}},
        "gpu_launches_per_step": 4, "tuning": grp.tuning()}
    if args.accuracy:
        out["tc_bf16x3"]["rel_l2_vs_oracle"] = batched_accuracy(
            wls, [x.cpu().numpy() for x in xs], [q.cpu().numpy() for q in qs], u0.cpu().numpy(),
            beta.cpu().numpy(), theta.cpu().numpy(), first_sums)
        out["tc_bf16x3"]["accuracy_sample"] = "8 random rows of each node set, all trajectories, first stage"
    grp.close()
    for op in ops:
        op.close()
    del grp, ops
    torch.cuda.empty_cache()
    blocks = []
    off, toff = 0, 0
    for wl in wls:
        blocks.append((u0[off:off + wl.B * wl.n].view(wl.B, wl.n).clone(), beta[toff:toff + wl.B].contiguous(),
                       theta[toff:toff + wl.B].contiguous()))
        off += wl.B * wl.n
        toff += wl.B
    # ---- plain FP32 comparator 1: dense FP32 W planes, SIMT FP32 GEMM per node set
    t0 = time.perf_counter()
    dops = [nf.Operator(x, q, wl.kernel, nf.DENSE_FP32) for x, q, wl in zip(xs, qs, wls)]
    torch.cuda.synchronize(dev)
    dbuild_ms = 1e3 * (time.perf_counter() - t0)
    dense_first = torch.cat([nf.nf_nonlocal_apply(op, ub, be, th).reshape(-1)
                             for op, (ub, be, th) in zip(dops, blocks)]).double().cpu().numpy()
    dblocks = [(ub.clone(), be, th) for ub, be, th in blocks]
    for op in dops:
        op.profile(True, ring=steps)

    def dense_step():
        for op, (ub, be, th) in zip(dops, dblocks):
            nf.nf_rk4_advance(op, ub, 0.0, 0.05, 1, be, th)

    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    ms_d, _ = timed(dense_step, steps)
    dclocks = sampler.stop()
    kd = sum(float(sum(sum(st) for st in op.kernel_ms_history(steps))) for op in dops) / (4 * steps)
    for op in dops:
        op.check()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_flops = float(sum(2 * wl.B * wl.n * wl.n for wl in wls))
    lanes = (pipes or {}).get("fma_f32x2", {}).get("per_clk_per_sm") or 128.0
    mhz = dclocks["sm_mhz"] or 1900.0
    fp32_peak = sms * lanes * 2.0 * mhz * 1e6 / 1e12
    fp32_ach = fp32_flops / (kd * 1e-3) / 1e12
    out["simt_fp32_dense"] = {
        "ms_per_step": ms_d, "rk4_steps_per_s": 1e3 / ms_d, "pair_evals_per_s": 4 * pairs_per_stage / (ms_d * 1e-3),
        "kernel_ms_per_stage": kd, "build_ms": dbuild_ms, "clocks": dclocks,
        "roofline": {"bound": "alu", "fp32": {"achieved": fp32_ach, "peak": fp32_peak, "unit": "TFLOP/s",
                                              "frac": fp32_ach / fp32_peak,
                                              "peak_basis": f"{sms} SMs x {lanes:.1f} FP32 FMA lanes/clk/SM "
                                                            f"(measured f32x2 probe) x 2 flop x {mhz:.0f} MHz"}},
        "gpu_launches_per_step": 4 * len(dops)}
    if args.accuracy:
        out["simt_fp32_dense"]["rel_l2_vs_oracle"] = batched_accuracy(
            wls, [x.cpu().numpy() for x in xs], [q.cpu().numpy() for q in qs], u0.cpu().numpy(),
            beta.cpu().numpy(), theta.cpu().numpy(), dense_first)
    out["tc_speedup_vs_simt_fp32_dense"] = ms_d / ms
    for op in dops:
        op.close()
    del dops
    torch.cuda.empty_cache()
    # ---- plain FP32 comparator 2: matrix-free pair kernel, B_g trajectories per node set
    mops = [nf.Operator(x, q, wl.kernel, nf.MATRIX_FREE) for x, q, wl in zip(xs, qs, wls)]

    def mf_step():
        for op, (ub, be, th) in zip(mops, blocks):
            nf.nf_rk4_advance(op, ub, 0.0, 0.05, 1, be, th)

    cmp_steps = max(1, min(steps, 5))
    ms_mf, _ = timed(mf_step, cmp_steps)
    out["mf_fp32"] = {"ms_per_step": ms_mf, "rk4_steps_per_s": 1e3 / ms_mf,
                      "pair_evals_per_s": 4 * pairs_per_stage / (ms_mf * 1e-3), "steps_timed": cmp_steps}
    out["tc_speedup_vs_plain_fp32"] = ms_mf / ms
    for op in mops:
        op.close()
    torch.cuda.empty_cache()
    return out


def run_models(args, dev, wl, x32, q32, u0):
    """§5 models on the precision workload (matrix-free path): the synaptic-depression model
    with the C^4 smooth-step rate, stepped by AB5 (one nonlocal sum per step) and by RK4.
    AB5 steady state: the time of 4 + K steps minus the time of its 4 RK4 start-up steps."""
    import torch

    import paper_2504_13379_gb300 as nf

    op = nf.Operator(x32, q32, wl.kernel, nf.MATRIX_FREE)
    stream = torch.cuda.current_stream(dev)
    K = max(8, min(args.steps, 40))
    model = dict(rate=nf.RATE_SMOOTHSTEP, a=0.06, b=0.54, tau=20.0, beta_d=0.5)

    def timed(nsteps, integrator):
        u = u0.clone().view(1, -1)
        s = torch.ones_like(u)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        nf.nf_field_advance(op, u, wl.dt, nsteps, 20.0, 0.2, s=s, integrator=integrator, **model)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b)

    timed(6, "ab5")  # warm-up
    t_start = timed(4, "ab5")
    t_ab5 = (timed(4 + K, "ab5") - t_start) / K
    t_rk4 = timed(K, "rk4") / K
    op.check()
    op.close()
    n = wl.n
    return {"workload": f"synaptic depression (tau 20, beta_d 0.5) with the C^4 smooth step on [0.06, 0.54], "
                        f"precision torus n={n}, matrix-free, dt={wl.dt}",
            "ab5": {"ms_per_step": t_ab5, "steps_per_s": 1e3 / t_ab5, "pair_evals_per_s": n * n / (t_ab5 * 1e-3),
                    "nonlocal_sums_per_step": 1, "steps_timed": K},
            "rk4": {"ms_per_step": t_rk4, "steps_per_s": 1e3 / t_rk4, "pair_evals_per_s": 4 * n * n / (t_rk4 * 1e-3),
                    "nonlocal_sums_per_step": 4, "steps_timed": K}}


def run_geometries(dev, n=100000):
    """Surface quadrature setup on the paper's deformed sphere (gamma = 0.8) and ring Dupin
    cyclide at n ~ 1e5 nodes (k = 32, degree 3): GPU stencils + weights time, and the
    relative error of sum(q) against the surface area (parameter-space reference)."""
    import torch

    import nodesets
    import paper_2504_13379_gb300 as nf

    out = {}
    for name, ns in (("deformed_sphere_gamma0.8", nodesets.deformed_sphere(n, 0.8)),
                     ("dupin_cyclide_ring", nodesets.cyclide_lattice(n))):
        nodes = torch.as_tensor(ns.nodes, device=dev)
        tris = torch.as_tensor(ns.tris, device=dev)
        normals = torch.as_tensor(ns.normals, device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        st = nf.nf_build_stencils(nodes, tris, 32)
        q = nf.nf_quad_weights(nodes, tris, st, 3, normals=normals)
        torch.cuda.synchronize(dev)
        ms = 1e3 * (time.perf_counter() - t0)
        out[name] = {"n": ns.n, "elements": ns.m, "stencils_plus_weights_ms": ms,
                     "sum_q_minus_area_rel": float((q.sum().item() - ns.area) / ns.area)}
    return out


# ------------------------------------------------------------ convergence studies (§4.3, §4.4)
# Paper parameters: firing rate gain 5, threshold 1/2; w = Gauss(., .; 1/40) under the
# doubly periodic distance of side 2 pi; u* = f^-1[Gauss(x, x0(t); 11/10) + 1/10],
# x0(t) = (cos t, sin t) / 5; t in [0, 1/10]; PHS r^3, stencils of 21 nodes.
MMS_GAIN, MMS_THRESH, MMS_T, MMS_DT = 5.0, 0.5, 0.1, 0.01
MMS_SIGMA_W, MMS_SIGMA, MMS_C, MMS_RADIUS, MMS_K = 1.0 / 40.0, 1.1, 0.1, 0.2, 21
TORUS_R, TORUS_r = 3.0, 1.0


def mms_kernel():
    """Gauss(sigma_w) as (A1, s1, A2, s2, period): A1 = 1 / (2 pi sigma_w^2), s1 = sqrt(2) sigma_w, no second
    Gaussian (s2 = 2 s1 only selects the one-exponential form)."""
    s1 = math.sqrt(2.0) * MMS_SIGMA_W
    return (1.0 / (2.0 * math.pi * MMS_SIGMA_W ** 2), s1, 0.0, 2.0 * s1, 2.0 * math.pi)


def mms_solution(xy, t):
    """u*(t, x) on the periodic square of side 2 pi (the closed form the study measures against)."""
    L = 2.0 * math.pi
    d = xy - MMS_RADIUS * np.array([math.cos(t), math.sin(t)])
    d -= L * np.round(d / L)
    z = np.exp(-(d ** 2).sum(1) / (2 * MMS_SIGMA ** 2)) / (2 * math.pi * MMS_SIGMA ** 2) + MMS_C
    return MMS_THRESH + np.log(z / (1.0 - z)) / MMS_GAIN


def mms_case(geometry, n):
    """Nodes, elements, normals, and the map to the periodic square: flat -- Halton nodes
    with a Delaunay triangulation of [0, 2 pi]^2 (§4.3); torus -- the spiral lattice on
    R = 3, r = 1 (§4.4), square coordinates (phi, theta), weights divided by R + r cos theta."""
    import nodesets

    if geometry == "flat":
        ns = nodesets.square_halton(n)
        xy = ns.coords() * (2.0 * math.pi)
        return {"nodes": xy, "tris": ns.tris, "normals": None, "xy": xy, "qscale": np.ones(ns.n),
                "scale": 1.0, "n": ns.n, "h": 2.0 * math.pi / math.sqrt(ns.n)}
    ns = nodesets.torus_lattice(n, R=TORUS_R, r=TORUS_r, jitter=0.0)
    th = ns.meta["theta"]
    xy = np.mod(np.stack([ns.meta["phi"], th], 1), 2.0 * math.pi)
    return {"nodes": ns.nodes, "tris": ns.tris, "normals": ns.normals, "xy": xy,
            "qscale": 1.0 / (TORUS_R + TORUS_r * np.cos(th)), "scale": TORUS_r, "n": ns.n,
            "h": 1.0 / math.sqrt(ns.n)}


def mms_run(dev, geometry, n, degs, cull=True):
    """One node set: GPU stencils and weights per degree, then RK4 on the matrix-free
    periodic path with the flat manufactured forcing; errors at T against u*.  cull: skip
    the block pairs whose contributions are exactly zero (bit-identical sums)."""
    import torch

    import paper_2504_13379_gb300 as nf

    cs = mms_case(geometry, n)
    nodes = torch.as_tensor(cs["nodes"], device=dev)
    tris = torch.as_tensor(cs["tris"], device=dev)
    normals = torch.as_tensor(cs["normals"], device=dev) if cs["normals"] is not None else None
    st = nf.nf_build_stencils(nodes, tris, MMS_K)
    X = np.concatenate([cs["xy"], np.zeros((cs["n"], 1))], 1).astype(np.float32)
    x32 = torch.as_tensor(X, device=dev)
    u0 = torch.as_tensor(mms_solution(cs["xy"], 0.0).astype(np.float32), device=dev).view(1, -1)
    exact = mms_solution(X[:, :2].astype(np.float64), MMS_T)
    nsteps = int(round(MMS_T / MMS_DT))
    stream = torch.cuda.current_stream(dev)
    rows = []
    for deg in degs:
        try:
            q = nf.nf_quad_weights(nodes, tris, st, deg, normals=normals)
        except nf.NFError as e:  # e.g. a stencil on too few lattice rows for the degree
            rows.append({"deg": deg, "n": cs["n"], "h": cs["h"], "weights": str(e)})
            continue
        qd = q.cpu().numpy() * cs["qscale"]
        op = nf.Operator(x32, torch.as_tensor(qd.astype(np.float32), device=dev), mms_kernel(), nf.MATRIX_FREE)
        live, total = op.mf_cull(cull)
        F = nf.Forcing.flat(MMS_C, MMS_RADIUS, MMS_SIGMA, cs["scale"])
        u = u0.clone()
        nf.nf_rk4_advance(op, u, 0.0, MMS_DT, 1, MMS_GAIN, MMS_THRESH, forcing=F)  # graph capture
        u = u0.clone()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        nf.nf_rk4_advance(op, u, 0.0, MMS_DT, nsteps, MMS_GAIN, MMS_THRESH, forcing=F)
        b.record(stream)
        b.synchronize()
        op.check()
        got = u.double().cpu().numpy().ravel()
        err = got - exact
        w = np.abs(qd)
        rows.append({"deg": deg, "n": cs["n"], "h": cs["h"],
                     "rel_max_err": float(np.abs(err).max() / np.abs(exact).max()),
                     "rel_l2_err": float(math.sqrt((w * err ** 2).sum() / (w * exact ** 2).sum())),
                     "rk4_ms": a.elapsed_time(b), "ms_per_nonlocal_sum": a.elapsed_time(b) / (4 * nsteps),
                     "live_block_pairs": live, "block_pairs": total, "culled": bool(cull)})
        op.close()
    return rows


def observed_orders(rows):
    """Least-squares slope of log(error) against log(h), per degree."""
    out = {}
    for deg in sorted({r["deg"] for r in rows}):
        rs = [r for r in rows if r["deg"] == deg and "rel_l2_err" in r]
        if len(rs) < 2:
            continue
        lh = np.log([r["h"] for r in rs])
        le = np.log([r["rel_l2_err"] for r in rs])
        out[str(deg)] = float(np.polyfit(lh, le, 1)[0])
    return out


def run_periodic(dev):
    """The periodic-square path at one size: §4.3's manufactured problem on 2^17 Halton
    nodes (degree 3), error at T and the time per nonlocal sum, without and with block-pair
    culling (whose sums are bit-identical)."""
    out = {"workload": "§4.3 manufactured solution on the periodic square of side 2 pi, Gauss(1/40) kernel, "
                       "matrix-free periodic path (one-Gaussian form), RK4 dt=0.01 to T=0.1"}
    for key, cull in (("all_pairs", False), ("culled", True)):
        r = mms_run(dev, "flat", 1 << 17, [3], cull=cull)[0]
        n = r["n"]
        r["pair_evals_per_s"] = n * n / (r["ms_per_nonlocal_sum"] * 1e-3)
        out[key] = r
    return out


def run_convergence(dev):
    """§4.3 (square, degrees 2-4) and §4.4 (torus, degrees 1-3: on the regular spiral
    lattice a 21-node stencil can lie on four lattice rows, which no degree-4 system
    resolves) manufactured-solution studies over node counts."""
    out = {}
    for geometry, sizes, degs in (("flat", [1 << 14, 1 << 15, 1 << 16, 1 << 17, 1 << 18, 1 << 19], (2, 3, 4)),
                                  ("torus", [1 << 16, 1 << 17, 1 << 18, 1 << 19, 1 << 20], (1, 2, 3))):
        rows = []
        for n in sizes:
            rows += mms_run(dev, geometry, n, list(degs))
        out[geometry] = {"rows": rows, "observed_order_l2": observed_orders(rows),
                         "h": "2 pi / sqrt(n)" if geometry == "flat" else "n^(-1/2)"}
    return out


def run_configs(dev):
    """The small configurations: the flat square (n = 1,500, 100 RK4 steps, the whole run
    as one call; L2-resident, latency bound) on every single-trajectory path, and the unit
    sphere with the manufactured forcing (n = 20,000, 200 steps) with its error against u*."""
    import torch

    import paper_2504_13379_gb300 as nf
    from nodesets import workloads as W

    stream = torch.cuda.current_stream(dev)

    def whole_run(op, u0, wl, forcing=None):
        u = u0.clone()
        nf.nf_rk4_advance(op, u, 0.0, wl.dt, 1, float(wl.beta[0]), float(wl.theta[0]), forcing=forcing)
        u = u0.clone()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        nf.nf_rk4_advance(op, u, 0.0, wl.dt, wl.nsteps, float(wl.beta[0]), float(wl.theta[0]), forcing=forcing)
        b.record(stream)
        b.synchronize()
        op.check()
        return a.elapsed_time(b), u

    out = {}
    wl = W.flat()
    X2 = torch.as_tensor(wl.ns.coords(), device=dev)
    tris = torch.as_tensor(wl.ns.tris, device=dev)
    q = nf.nf_quad_weights(X2, tris, nf.nf_build_stencils(X2, tris, wl.k), wl.deg).to(torch.float32)
    x32 = torch.as_tensor(wl.ns.nodes.astype(np.float32), device=dev)
    u0 = torch.as_tensor(wl.u0.astype(np.float32), device=dev)
    flat = {"workload": f"flat square n={wl.n} k={wl.k} deg={wl.deg}, {wl.nsteps} RK4 steps dt={wl.dt}, "
                        "one call (graph replay)"}
    for pname, path in PATHS.items():
        op = nf.Operator(x32, q, wl.kernel, path)
        ms, _ = whole_run(op, u0, wl)
        flat[pname] = {"run_ms": ms, "rk4_steps_per_s": wl.nsteps * 1e3 / ms}
        op.close()
    out["flat"] = flat
    wl = W.sphere()
    nodes = torch.as_tensor(wl.ns.nodes, device=dev)
    tris = torch.as_tensor(wl.ns.tris, device=dev)
    st = nf.nf_build_stencils(nodes, tris, wl.k)
    q = nf.nf_quad_weights(nodes, tris, st, wl.deg, normals=torch.as_tensor(wl.ns.normals, device=dev))
    X = wl.ns.nodes
    x32 = torch.as_tensor(X.astype(np.float32), device=dev)
    c, a0 = wl.forcing["c"], wl.forcing["a0"]
    F = nf.Forcing.sphere(c, a0)  # Y1 = z/2, Y2 = x y and the eigenvalues from the operator
    op = nf.Operator(x32, q.to(torch.float32), wl.kernel, nf.MATRIX_FREE)
    u0 = torch.as_tensor(wl.u0.astype(np.float32), device=dev)
    ms, u = whole_run(op, u0, wl, forcing=F)
    op.close()
    T = wl.dt * wl.nsteps
    z = c + a0 * math.cos(T) * (0.5 * X[:, 2] + X[:, 0] * X[:, 1])
    exact = wl.theta[0] + np.log(z / (1.0 - z)) / wl.beta[0]
    err = u.double().cpu().numpy().ravel() - exact
    out["sphere"] = {"workload": f"unit sphere n={wl.n} k={wl.k} deg={wl.deg}, manufactured forcing, "
                                 f"{wl.nsteps} RK4 steps dt={wl.dt}, matrix-free",
                     "run_ms": ms, "rk4_steps_per_s": wl.nsteps * 1e3 / ms,
                     "pair_evals_per_s": 4.0 * wl.n * wl.n * wl.nsteps / (ms * 1e-3),
                     "rel_max_err_vs_u_star": float(np.abs(err).max() / np.abs(exact).max())}
    return out


def run_culling(args, dev, wl, x32, q32, u0):
    """Block-pair culling on the precision workload: RK4 steps with the culled symmetric
    kernel, the live fraction, and a bitwise comparison with the full sum after one step.
    Not part of the headline value (which counts every pair evaluated)."""
    import torch

    import paper_2504_13379_gb300 as nf

    beta, theta = float(wl.beta[0]), float(wl.theta[0])
    full = nf.Operator(x32, q32, wl.kernel, nf.MATRIX_FREE)
    op = nf.Operator(x32, q32, wl.kernel, nf.MATRIX_FREE)
    live, total = op.mf_cull(True)
    ua, ub = u0.clone().view(1, -1), u0.clone().view(1, -1)
    nf.nf_rk4_advance(full, ua, 0.0, wl.dt, 1, beta, theta)
    nf.nf_rk4_advance(op, ub, 0.0, wl.dt, 1, beta, theta)
    identical = bool(torch.equal(ua, ub))
    full.close()
    stream = torch.cuda.current_stream(dev)
    K = max(4, min(args.steps, 40))
    u = u0.clone().view(1, -1)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    nf.nf_rk4_advance(op, u, 0.0, wl.dt, K, beta, theta)
    b.record(stream)
    b.synchronize()
    op.check()
    op.close()
    ms = a.elapsed_time(b) / K
    return {"workload": f"precision torus n={wl.n}, matrix-free symmetric kernel with block-pair culling",
            "ms_per_step": ms, "rk4_steps_per_s": 1e3 / ms, "live_block_pairs": live, "block_pairs": total,
            "bit_identical_to_full_sum": identical, "steps_timed": K}


def run_adjoint(args, dev):
    """Differentiation workload: gradient of L = |u(T) - u_target|^2 w.r.t. the kernel
    parameters and u0 through the discrete RK4 adjoint (checkpoints every C steps)."""
    import torch

    import paper_2504_13379_gb300 as nf
    from nodesets import workloads as W

    wl = W.adjoint()
    n, C, nsteps, dt = wl.n, wl.extra["C"], wl.nsteps, wl.dt
    nodes = torch.as_tensor(wl.ns.nodes, device=dev)
    tris = torch.as_tensor(wl.ns.tris, device=dev)
    st = nf.nf_build_stencils(nodes, tris, wl.k)
    q = nf.nf_quad_weights(nodes, tris, st, wl.deg, normals=torch.as_tensor(wl.ns.normals, device=dev))
    x32 = torch.as_tensor(wl.ns.nodes.astype(np.float32), device=dev)
    q32 = q.to(torch.float32).contiguous()
    beta, theta = float(wl.beta[0]), float(wl.theta[0])
    u0 = torch.as_tensor(wl.u0.astype(np.float32), device=dev)
    target = u0.clone()
    op_t = nf.Operator(x32, q32, wl.extra["target_kernel"], nf.MATRIX_FREE)
    nf.nf_rk4_advance(op_t, target, 0.0, dt, nsteps, beta, theta)
    op_t.close()
    op = nf.Operator(x32, q32, wl.kernel, nf.MATRIX_FREE)
    ck = torch.empty((nsteps // C + 1, 1, n), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def gradient():
        u = u0.clone()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        nf.nf_rk4_advance(op, u, 0.0, dt, nsteps, beta, theta, ckpt=ck, C_every=C)
        b.record(stream)
        gu, gk = nf.nf_adjoint(op, ck, C, 0.0, dt, nsteps, beta, theta, 2.0 * (u - target))
        c.record(stream)
        c.synchronize()
        return a.elapsed_time(b), b.elapsed_time(c), float(((u - target) ** 2).sum()), gk[0].tolist()

    gradient()  # warm-up (graph capture, allocations)
    fwd_ms, adj_ms, loss, gk = gradient()
    op.check()
    op.close()
    pairs = float(n) * n
    return {"workload": f"torus R=1 r=0.4 n={n} k={wl.k} deg={wl.deg}, {nsteps} RK4 steps dt={dt}, checkpoints every {C}",
            "forward_ms": fwd_ms, "adjoint_ms": adj_ms, "gradient_ms": fwd_ms + adj_ms, "loss": loss,
            "grad_kernel": dict(zip(["A1", "s1", "A2", "s2"], gk)),
            "adjoint_pair_evals_per_s": pairs * 4 * nsteps * 2 / (adj_ms * 1e-3),
            "note": "adjoint time includes the forward recomputation of each segment (4 nsteps stages) "
                    "and 4 nsteps adjoint pair passes"}


def probe_pipes(dev):
    """Measured FP32 FMA (scalar and packed f32x2) and SFU ex2 rates per clock per SM."""
    import paper_2504_13379_gb300 as nf

    out = {}
    for name, kind, iters in (("fma_f32", nf.PROBE_FMA, 100000), ("fma_f32x2", nf.PROBE_FMA2, 100000),
                              ("ex2", nf.PROBE_EX2, 20000), ("fma_f32x2_outer", nf.PROBE_FMA2_OUTER, 100000)):
        nf.nf_probe_pipe(kind, 1000)  # warm-up
        rate, mhz, ms = nf.nf_probe_pipe(kind, iters)
        out[name] = {"per_clk_per_sm": rate, "sm_mhz": mhz, "ms": ms}
    out["basis"] = ("one CTA of 1,024 threads per SM, 8 independent chains per thread, cycles from each SM's "
                    "clock64; median over SMs (nf_probe_pipe)")
    return out


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_2504_13379_gb300 as nf
    from nodesets import workloads as W

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    # accuracy vs the FP64 oracle is computed in the CPU-baseline leg (rank 0, one GPU)
    args.accuracy = rank == 0 and world == 1 and not args.no_cpu_baseline
    wl = W.precision(args.n)
    n = wl.n
    # ---- setup on the GPU: stencils and quadrature weights (§3.1-3.3)
    nodes = torch.as_tensor(wl.ns.nodes, device=dev)
    tris = torch.as_tensor(wl.ns.tris, device=dev)
    normals = torch.as_tensor(wl.ns.normals, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    st = nf.nf_build_stencils(nodes, tris, wl.k)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    q = nf.nf_quad_weights(nodes, tris, st, wl.deg, normals=normals)
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    setup = {"stencils_ms": 1e3 * (t1 - t0), "weights_ms": 1e3 * (t2 - t1),
             "sum_q_minus_area_rel": float((q.sum().item() - wl.ns.area) / wl.ns.area)}
    x32 = torch.as_tensor(wl.ns.nodes.astype(np.float32), device=dev)
    q32 = q.to(torch.float32).contiguous()
    u0 = torch.as_tensor(wl.u0.astype(np.float32), device=dev)
    beta, theta = float(wl.beta[0]), float(wl.theta[0])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    results = {}
    first_sums = {}
    clocks_all = []
    launches_total = 0
    for pname in [p for p in args.paths.split(",") if p]:
        path = PATHS[pname]
        torch.cuda.synchronize(dev)
        tb = time.perf_counter()
        op = nf.Operator(x32, q32, wl.kernel, path)
        torch.cuda.synchronize(dev)
        build_ms = 1e3 * (time.perf_counter() - tb)
        first_sums[pname] = nf.nf_nonlocal_apply(op, u0.view(1, -1), beta, theta).double().cpu().numpy().ravel()
        op.profile(True, ring=args.steps)  # every timed step keeps its own kernel timings
        u = u0.clone()
        t_sim = 0.0
        for _ in range(args.warmup):
            nf.nf_rk4_advance(op, u, t_sim, wl.dt, 1, beta, theta)
            t_sim += wl.dt
        op.check()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        sampler = ClockSampler(dev.index if dev.index is not None else 0)
        sampler.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            nf.nf_rk4_advance(op, u, t_sim, wl.dt, 1, beta, theta)
            ev[k][1].record(stream)
            t_sim += wl.dt
        torch.cuda.synchronize(dev)
        clocks = sampler.stop()
        # the nonlocal kernels' durations in every timed step, read after the loop
        kern_ms = float(sum(sum(st) for st in op.kernel_ms_history(args.steps)))
        clocks_all.append(clocks)
        op.check()
        step_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        launches_per_step = 2 + 4 * 2  # prep + clock, then 4 x (nonlocal, stage) for one trajectory
        launches_total += launches_per_step * args.steps
        # ---- end to end through the public API with host buffers
        uh = torch.empty_like(u, device="cpu").pin_memory()
        uh.copy_(u0.cpu())
        uo = torch.empty_like(uh).pin_memory()
        e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            e2e_ev[k][0].record(stream)
            u.copy_(uh, non_blocking=True)
            nf.nf_rk4_advance(op, u, t_sim, wl.dt, 1, beta, theta)
            uo.copy_(u, non_blocking=True)
            e2e_ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        e2e_ms = sum(a.elapsed_time(b) for a, b in e2e_ev) / args.steps
        res = {"ms_per_step": step_ms, "rk4_steps_per_s": 1e3 / step_ms,
               "pair_evals_per_s": 4.0 * n * n / (step_ms * 1e-3),
               "kernel_ms_per_launch": kern_ms / (4 * args.steps), "build_ms": build_ms,
               "e2e_ms_per_step": e2e_ms, "clocks": clocks}
        if path == nf.MATRIX_FREE:
            res["launch_shape"] = op.launch_shape()
        else:  # HBM stream: stored bytes per launch / kernel time
            nb = -(-n // 1024)
            stored = (4.0 * (nb * (nb + 1) // 2) * 1024 * 1024 if path in (nf.DENSE_SYM_FP32, nf.DENSE_SYM_BF16X2)
                      else 4.0 * n * nb * 1024)
            res["hbm_gbs"] = stored / (res["kernel_ms_per_launch"] * 1e-3) / 1e9
            res["stored_bytes"] = stored
        results[pname] = res
        op.close()
        del op
        torch.cuda.empty_cache()
    # ---- FP32 FMA and SFU rates (cycle counts, so independent of when they run; measured
    # after the timed paths so that their full-power launches precede no operator's set-up)
    pipes = probe_pipes(dev)
    # ---- aggregate over ranks (max time)
    best = min(results, key=lambda p: results[p]["ms_per_step"])
    r = results[best]
    step_ms = r["ms_per_step"]
    e2e_ms = r["e2e_ms_per_step"]
    step_ms, e2e_ms = max_over_ranks([step_ms, e2e_ms], world, dev)
    value = whole_job_rate(4.0 * n * n, world, step_ms)
    pk = peaks()
    clocks = r["clocks"]
    kms = r["kernel_ms_per_launch"]
    if best == "mf":
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clocks["sm_mhz"] or pk.get("clocks_under_load", {}).get("sm_mhz_median") or 1432.0
        nb = -(-n // 1024)
        ops = LANE_OPS_PER_PAIR * (1.0 + 1.0 / nb)
        lanes = pipes["fma_f32x2"]["per_clk_per_sm"]
        ex2 = pipes["ex2"]["per_clk_per_sm"]
        fma_peak = sms * lanes * mhz * 1e6 / ops / 1e9                      # Gpair/s on the FP32 FMA pipe
        lanes_gen = pipes["fma_f32x2_outer"]["per_clk_per_sm"]  # packed FMAs with varied operands
        fma_peak_gen = sms * lanes_gen * mhz * 1e6 / ops / 1e9
        sfu_peak = sms * ex2 * mhz * 1e6 / (EX2_PER_PAIR * (1.0 + 1.0 / nb)) / 1e9  # Gpair/s on the SFU
        peak = min(fma_peak, sfu_peak)
        achieved = n * n / (kms * 1e-3) / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s", "frac": achieved / peak,
                "traffic": MF_TRAFFIC_BYTES if n == 100000 else None, "traffic_unit": "bytes per launch",
                "peak_basis": f"measured: {sms} SMs x {lanes:.1f} FP32 FMA-pipe lane operations/clk/SM (f32x2 "
                              f"probe in this run) x {mhz:.0f} MHz (median SM clock in the timed region) / "
                              f"{ops:.3f} lane operations per ordered pair (symmetric kernel, expanded form, m = 4); "
                              f"SFU ceiling {sfu_peak:.0f} Gpair/s from {ex2:.1f} ex2/clk/SM measured and "
                              f"{EX2_PER_PAIR} exponentials per ordered pair",
                "fma_pipe_peak": fma_peak, "sfu_peak": sfu_peak,
                "fma_pipe_peak_varied_operands": fma_peak_gen, "frac_vs_varied_operands": achieved / fma_peak_gen,
                "nominal_peak_128_lanes": sms * FMA_LANES_PER_CLK_SM_NOMINAL * mhz * 1e6 / ops / 1e9}
    else:
        bytes_per = 4.0 * n * n
        achieved = bytes_per / (kms * 1e-3) / 1e9
        peak = pk.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "peak_basis": "MEASURED_PEAKS hbm_gbs" if "hbm_gbs" in pk else "fallback 6.8 TB/s"}
    line = {
        "metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"precision torus R=1 r=0.4 n={n} k={wl.k} deg={wl.deg}, B=1, RK4 dt={wl.dt}",
                   "path": best, "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "rk4_steps_per_s": world * 1e3 / step_ms,
        "paths": results,
        "setup": setup,
        "roofline": roof,
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"]},
        "e2e": {"value": world * 4.0 * n * n / (e2e_ms * 1e-3), "unit": "pair-evals/s",
                "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n},
        "gpu_launches": launches_total,
        "pipe_rates": pipes,
    }
    # the further sections are measured on rank 0 only (they are not part of `value`)
    extra = rank == 0
    if extra and not args.no_batched:
        line["batched"] = run_batched(args, dev, args.steps, pipes)
        line["gpu_launches"] += 4 * args.steps  # tensor-core path: one grouped GEMM per stage
    if extra and not args.no_adjoint:
        line["adjoint"] = run_adjoint(args, dev)
    if extra and not args.no_models:
        line["models"] = run_models(args, dev, wl, x32, q32, u0)
    if extra and not args.no_geometries:
        line["geometries"] = run_geometries(dev)
    if extra and not args.no_periodic:
        line["periodic"] = run_periodic(dev)
        line["culling"] = run_culling(args, dev, wl, x32, q32, u0)
    if extra and not args.no_configs:
        line["configs"] = run_configs(dev)
    if extra and args.convergence:
        line["convergence"] = run_convergence(dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], acc = cpu_baseline(wl, q32.double().cpu().numpy(), args.cpu_seconds, first_sums)
        for p, e in acc.items():
            line["paths"][p]["rel_l2_vs_oracle"] = e
        line["accuracy"] = {"metric": "relative L2 error of the first-stage sum vs the FP64 oracle",
                            "sample": line["cpu_baseline"]["sample"], **acc}
    if "batched" in line:  # a compact copy as the last key, where a truncated log still shows it
        line["batched_summary"] = batched_summary(line["batched"])
    return line if rank == 0 else None


def batched_summary(b):
    """Steps/s of the batched paths on the same box, roofline fractions, error, clocks."""
    out = {"workload": b["workload"]}
    for key in ("tc_bf16x3", "simt_fp32_dense", "mf_fp32"):
        if key not in b:
            continue
        r = b[key]
        e = {"rk4_steps_per_s": r["rk4_steps_per_s"], "ms_per_step": r["ms_per_step"]}
        roof = r.get("roofline", {})
        for part in ("hbm", "tensor", "fp32"):
            if part in roof:
                e[f"{part}_frac"] = roof[part]["frac"]
        if "rel_l2_vs_oracle" in r:
            e["rel_l2_vs_oracle"] = r["rel_l2_vs_oracle"]
        if "clocks" in r:
            e["sm_mhz"] = r["clocks"].get("sm_mhz")
            e["clock_reasons"] = r["clocks"].get("reasons")
        out[key] = e
    for key in ("tc_speedup_vs_simt_fp32_dense", "tc_speedup_vs_plain_fp32"):
        if key in b:
            out[key] = b[key]
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        line = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

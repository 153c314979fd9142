"""Benchmark: cell-collision evaluations per second on the sudden-wall-heating slab.

Workload (one "step" = one Strang step of the whole hot path): 128 uniform
cells on [0, 1], N = 16 velocity points per dimension on [-6, 6]^3, hard
spheres (lambda = 1), Knudsen number eps = 0.1, gas initially a Maxwellian at
rest (rho = 1, T = 1), diffuse wall at x = 0 heated to T_w = 2, specular wall
at x = 1, dt = 0.5 dx / max|v1| (CFL 0.5). A step is T(dt/2) C(dt) T(dt/2):
two transport half steps (second-order upwind/minmod) and one Heun step of the
collision operator over all 128 cells, i.e. 2 x 128 = 256 cell-collision
evaluations (forward DFT, FP32 weighted convolution, inverse DFT, FP64
conservation projection), replayed from one CUDA graph.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun, one rank per GPU) runs independent replicas of the slab
("scaling": "weak"); the only collectives are the barrier and the max-reduction
of the timings. --impl reference times the FP64 CPU oracle on the same step.
"""
import argparse
import hashlib
import json
import math
import os
import signal
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N, L, LAM = 16, 6.0, 1.0
NX, EPS, TW = 128, 0.1, 2.0
DT = 0.5 * (1.0 / NX) / L
EVALS_PER_STEP = 2 * NX
METRIC = "cell-collision evals/s at N=16/32 vs plain FP64 GPU op, at stated rel-L2 error"
UNIT = "cell-collision evals/s"
LEARNED_TOL_OFF = 1 << 30  # learned_tol_ppm upper bound: a threshold of ~1e3 that no indicator reaches
WORKLOAD = ("sudden wall heating: 128 cells x N=16^3 velocities (L=6, hard spheres, Kn=0.1, "
            "Tw=2 diffuse / specular), one Strang step = 2 transport half steps + RK2 over "
            "128 cells = 256 collision evals")
FLUSH_BYTES = 512 << 20  # > 129 MB L2
WORKLOADS = ("wall-heating", "wall-heating-200", "homog-1cell", "sweep-n32", "sweep-n48", "uneven-4096",
             "learned-n16", "sudden-heating-refined", "collision-models")
SMS, FP32_LANES = 152, 128
PROFILES = os.path.join(ROOT, "profiles")


def conv_pairs_per_cell(n):
    """Unordered (zeta, {xi, zeta - xi}) pairs the FP32 kernel evaluates per cell."""
    h = n // 2

    def lo(k):
        return max(0, k - h + 1)

    def hi(k):
        return min(n - 1, k + h)

    row = sum(hi(k) - lo(k) + 1 for k in range(n))
    blocks = 0
    for k1 in range(n):
        for k2 in range(n):
            for m1 in range(lo(k1), hi(k1) + 1):
                n1 = k1 - m1 + h
                if m1 > n1:
                    continue
                for m2 in range(lo(k2), hi(k2) + 1):
                    if m1 == n1 and m2 > k2 - m2 + h:
                        continue
                    blocks += 1
    return blocks * row


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="use the library's default configuration")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON tuning cache: loaded if it exists (no tuning), else written after tuning; "
                         "lets a profiler run the configuration a plain run chose")
    ap.add_argument("--conv-impl", type=int, default=None,
                    help="convolution kernel variant (bte_set_option conv_impl); default: library choice")
    ap.add_argument("--conv-warps", type=int, default=None, help="warps per CTA of the convolution (conv_warps)")
    ap.add_argument("--conv-split", type=int, default=None, choices=[0, 1],
                    help="variant 4: cut the costliest pencil items in two (conv_split)")
    ap.add_argument("--dft-split", type=int, default=None, help="CTAs per cell in the fused transforms (1, 2, 4)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="wall-heating",
                    help="wall-heating (the headline line) or one of the secondary workloads")
    ap.add_argument("--cells", type=int, default=256, help="sweep-n32: number of cells (default 256)")
    ap.add_argument("--train-states", type=int, default=200000, help="learned-n16: training pairs")
    ap.add_argument("--epochs", type=int, default=30, help="learned-n16: training epochs")
    return ap.parse_args()


def source_hash():
    """Hash of the convolution kernel's source (conv32_device.cuh holds the
    kernels and their item loop, conv32.cu their launch configuration)."""
    h = hashlib.sha256()
    for name in ("conv32_device.cuh", "conv32.cu"):
        with open(os.path.join(ROOT, "paper_1211_0540_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic():
    """DRAM bytes per launch of the convolution kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(PROFILES, "conv32_wallheating_n16_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != source_hash():
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").strip()
        ids = [v.strip() for v in vis.split(",") if v.strip()] if vis else []
        self.index = ids[local_rank] if local_rank < len(ids) else str(local_rank)
        self.proc = None
        self.fh = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL, start_new_session=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.fh.flush()
        self.fh.seek(0)
        rows = [r.split(",") for r in self.fh.read().strip().splitlines() if r.strip()]
        os.unlink(self.fh.name)
        mhz, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                mhz.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(mhz)) if mhz else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(mhz)}


def max_over_ranks(value, device):
    """Largest value over the ranks of the default process group: the job's
    time is the slowest rank's. A plain float with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, total_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (total_ms * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_strang_step(f, oracle):
    return oracle.strang_step(N, L, LAM, f, DT, EPS, x0=0.0, x1=1.0, bc_left=oracle.BC_DIFFUSE,
                              bc_right=oracle.BC_SPECULAR, Tw_left=TW, Tw_right=1.0)


def tune(args, ctx, f, stream, inst=None, reps=3):
    """The FP32 configuration of this run: none (--no-autotune), the one stored in
    --tune-cache, or a fresh bte_autotune (saved to --tune-cache if given)."""
    if args.no_autotune:
        return None
    if args.tune_cache and os.path.exists(args.tune_cache):
        if ctx.tune_load(args.tune_cache) > 0:
            with open(args.tune_cache) as fh:
                entries = json.load(fh)["entries"]
            return dict(entries[0], source=args.tune_cache)
    cfg = ctx.autotune(f, inst=inst, reps=reps, stream=stream)
    if args.tune_cache:
        ctx.tune_save(args.tune_cache)
    return cfg


def run_reference(args):
    """The FP64 CPU oracle, as it stands, on the same Strang step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1211_0540_gb300 import inputs
    cores = oracle.get_threads()
    f = inputs.wall_heating_initial(N, L, NX)
    oracle.weights(N, L, LAM)  # table build is set-up, not part of a step
    for _ in range(args.warmup):
        f = oracle_strang_step(f, oracle)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = oracle_strang_step(f, oracle)
    dt = time.perf_counter() - t0
    value = EVALS_PER_STEP * args.steps / dt
    sample = "the full workload: every step is one whole Strang step of the 128-cell slab"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "arm": "FP64 CPU oracle (direct sums)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "wall-heating":
        return run_secondary(args)
    import torch
    import torch.distributed as dist

    from paper_1211_0540_gb300 import bte, inputs

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    ctx = bte.Context(local)
    ctx.init_weights([(N, L, LAM)])
    if args.conv_impl is not None:
        ctx.set_option("conv_impl", args.conv_impl)
    if args.conv_warps is not None:
        ctx.set_option("conv_warps", args.conv_warps)
    if args.conv_split is not None:
        ctx.set_option("conv_split", args.conv_split)
    if args.dft_split is not None:
        ctx.set_option("dft_split", args.dft_split)
    ctx.set_option("profile_mask", 1)  # timed steps: events around the convolution only
    tr = dict(nx=NX, x0=0.0, x1=1.0, bc_left=bte.BC_DIFFUSE, bc_right=bte.BC_SPECULAR, Tw_left=TW,
              Tw_right=1.0)
    f0 = inputs.wall_heating_initial(N, L, NX)
    f = torch.from_numpy(f0).cuda()
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    tuned = None
    if args.conv_impl is None and args.conv_warps is None and args.conv_split is None and args.dft_split is None:
        tuned = tune(args, ctx, f, stream, reps=10)  # untimed: picks the launch configuration
    ctx.profile_enable(True)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            ctx.step(f, DT, EPS, transport=tr, mode=bte.FP32, stream=stream)
    ctx.sync_status(stream)
    ctx.profile_read("*", stream)

    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = ctx.launch_count()
    step_ms, conv_ms, conv_n = [], 0.0, 0
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps' launches
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(i & 0xff)  # L2 flush, outside the timed events
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.step(f, DT, EPS, transport=tr, mode=bte.FP32, stream=stream)
            e1.record(stream)
            n, ms = ctx.profile_read("conv32", stream)
            conv_n += n
            conv_ms += ms
            step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = ctx.launch_count() - n0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ctx.sync_status(stream)
    total_ms = max_over_ranks(float(sum(step_ms)), "cuda")
    value = job_rate(EVALS_PER_STEP * args.steps, world, total_ms)

    # per-stage device times, in a separate pass (events around every stage
    # lengthen the step, so the timed steps above carry them around conv32 only)
    ctx.set_option("profile_mask", 63)
    part_ms = {"conv32": 0.0, "forward": 0.0, "inverse": 0.0, "transport": 0.0}
    with torch.cuda.stream(stream):
        ctx.step(f, DT, EPS, transport=tr, mode=bte.FP32, stream=stream)  # capture
        ctx.profile_read("*", stream)
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            ctx.step(f, DT, EPS, transport=tr, mode=bte.FP32, stream=stream)
            for name in part_ms:
                part_ms[name] += ctx.profile_read(name, stream)[1]
        ctx.profile_read("*", stream)
    ctx.set_option("profile_mask", 1)  # drops the graphs: capture again before the end-to-end timing
    with torch.cuda.stream(stream):
        ctx.step(f, DT, EPS, transport=tr, mode=bte.FP32, stream=stream)
    ctx.profile_read("*", stream)

    # end to end through the public API: pinned host state in and out every step
    # (bte_transfer: the library's copy kernels read and write the pinned buffers)
    fh_in = torch.from_numpy(f.cpu().numpy()).pin_memory()
    fh_out = torch.empty_like(fh_in).pin_memory()
    e2e_ms = []
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.transfer(f, fh_in, stream=stream)
            ctx.step(f, DT, EPS, transport=tr, mode=bte.FP32, stream=stream)
            ctx.transfer(fh_out, f, stream=stream)
            e1.record(stream)
            e1.synchronize()
            e2e_ms.append(e0.elapsed_time(e1))
    ctx.profile_read("*", stream)
    e2e_total = max_over_ranks(float(sum(e2e_ms)), "cuda")
    e2e_value = job_rate(EVALS_PER_STEP * args.steps, world, e2e_total)
    nbytes = f.numel() * 8

    # plain FP64 GPU operator on the same state (the metric's comparator)
    f64 = f.clone()
    with torch.cuda.stream(stream):
        ctx.step(f64, DT, EPS, transport=tr, mode=bte.FP64_PLAIN, stream=stream)  # build + capture
        ctx.sync_status(stream)
        ctx.profile_read("*", stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            ctx.step(f64, DT, EPS, transport=tr, mode=bte.FP64_PLAIN, stream=stream)
        e1.record(stream)
        ctx.profile_read("*", stream)
    fp64_value = EVALS_PER_STEP * reps / (e0.elapsed_time(e1) * 1e-3)

    # stated accuracy of the FP32 operator on the benchmark state
    out = {}
    if rank == 0:
        import oracle
        Qg = ctx.collide(f, mode=bte.FP32, stream=stream)
        Q64 = ctx.collide(f, mode=bte.FP64_PLAIN, stream=stream)
        ctx.sync_status(stream)
        Qg, Q64 = Qg.cpu().numpy().reshape(NX, -1), Q64.cpu().numpy().reshape(NX, -1)
        fs = f.cpu().numpy().reshape(NX, -1)
        pick = [0, 1, 2, NX // 2, NX - 1]
        Qo = oracle.collide(N, L, LAM, fs[pick])
        Qm = oracle.collide(N, L, LAM, fs[pick], part=1, project=False)
        rel = np.linalg.norm(Qg[pick] - Qo, axis=1) / np.linalg.norm(Qm, axis=1)
        rel64 = np.linalg.norm(Q64[pick] - Qo, axis=1) / np.linalg.norm(Qm, axis=1)
        mom = oracle.moments(N, L, Qg)
        out["accuracy"] = {"fp32_rel_l2_vs_oracle_max": float(rel.max()),
                           "fp64_plain_rel_l2_vs_oracle_max": float(rel64.max()),
                           "cells_checked": pick, "norm": "||Q - Q_oracle|| / ||Q_loss_oracle||",
                           "fp32_max_abs_moment": float(np.abs(mom).max())}

    conv_pairs = conv_pairs_per_cell(N)
    flops_per_launch = 10.0 * conv_pairs * NX
    conv_avg_ms = conv_ms / max(conv_n, 1)
    achieved = flops_per_launch / (conv_avg_ms * 1e-3) / 1e12
    peak, clk = _alu_peak(clocks)
    fma = _measured_fma(ctx, stream)
    traffic = load_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": NX, "N": N, "L": L, "lambda": LAM, "eps": EPS,
                   "dt": DT, "l2": "flushed (512 MB write) before every timed step",
                   "arith": "FP32 convolution (TwoSum-compensated), FP32 DFTs, FP64 projection/state",
                   "autotuned": tuned,
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": {"bound": "alu", "kernel": "conv32 (FP32 weighted convolution)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_basis": _peak_basis(clk, fma), "measured_fma": fma,
                     "frac_of_measured_ffma2": achieved / fma["fp32_ffma2_tflops"],
                     "flops_per_launch": flops_per_launch,
                     "flop_unit": "10 flops per evaluated (zeta, {xi, zeta-xi}) pair per cell",
                     "conv_ms_per_launch": conv_avg_ms, "conv_launches_timed": conv_n},
        "stage_ms_per_step": dict({k: v / args.steps for k, v in part_ms.items()},
                                  note="separate pass with events around every stage (each figure includes "
                                       "the graph's launch gap before the stage)"),
        "fp64_plain": {"value": fp64_value, "unit": UNIT, "speedup_fp32_over_fp64": value / fp64_value},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    line.update(out)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        fs = f0.copy()
        t0 = time.perf_counter()
        oracle_strang_step(fs, oracle)
        tcpu = time.perf_counter() - t0
        cores = oracle.get_threads()
        # the same oracle on one core: projected collides of 8 cells of the slab
        oracle.set_threads(1)
        try:
            t0 = time.perf_counter()
            oracle.collide(N, L, LAM, f0[:8])
            t1c = time.perf_counter() - t0
        finally:
            oracle.set_threads(cores)
        line["cpu_baseline"] = {"value": EVALS_PER_STEP / tcpu, "unit": UNIT,
                                "cores": cores, "kind": "oracle",
                                "sample": "one whole Strang step of the 128-cell slab (256 evals)",
                                "one_core": {"value": 8 / t1c, "unit": UNIT,
                                             "sample": "8 projected collides of slab cells, 1 thread"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()
    return 0


# ---------------------------------------------------------------------------
# Secondary workloads (one JSON line each; the headline is wall-heating).

def _timed_steps(torch, fn, steps, stream, flush, tag="timed"):
    """Device time of each call of fn, L2 flushed before each (outside the events);
    the calls sit in an NVTX range named tag (profilers can select them)."""
    ev = []
    torch.cuda.nvtx.range_push(tag)
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(i & 0xff)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            ev.append((e0, e1))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    return [a.elapsed_time(b) for a, b in ev]


def _moment_rel(oracle, n, q):
    """max_i |(C Q)_i| / max(m_0(|Q|), m_4(|Q|)) over the cells of q (2-D)."""
    m = oracle.moments(n, L, q)
    a = oracle.moments(n, L, np.abs(q))
    scale = np.maximum(np.abs(a[:, 0]), np.abs(a[:, 4]))
    return float((np.abs(m).max(axis=1) / scale).max())


def _alu_peak(clocks):
    """FP32 ALU peak from the unit counts and the SM clock sampled during the
    timed region; no clock samples is an error, not a guess."""
    clk = clocks.get("sm_mhz")
    if not clk:
        raise RuntimeError("no SM clock samples during the timed region (nvidia-smi): the ALU peak is unknown")
    return SMS * FP32_LANES * 2 * clk * 1e6 / 1e12, clk


def _measured_fma(ctx, stream):
    """FMA rates measured on this GPU in this run (bte_alu_peak, untimed)."""
    return {"fp32_ffma_tflops": ctx.alu_peak(0, stream), "fp32_ffma2_tflops": ctx.alu_peak(1, stream),
            "fp64_dfma_tflops": ctx.alu_peak(2, stream),
            "how": "bte_alu_peak: 2048 threads per SM of independent FMA chains, 5 launches after a warm-up"}


def _peak_basis(clk, fma):
    return ("152 SMs x 128 FP32 lanes x 2 flop x median SM clock %.0f MHz during the timed region; measured in "
            "this run (bte_alu_peak): FFMA %.1f, FFMA2 %.1f TFLOP/s" % (clk, fma["fp32_ffma_tflops"],
                                                                      fma["fp32_ffma2_tflops"]))


def _line(args, metric, value, unit, ms_per_step, workload, extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "l2": "flushed (512 MB write) before every timed step"}}
    line.update(extra)
    return line


def run_homog1(args, ctx, torch, bte, inputs, oracle, stream, flush, sampler):
    """One space-homogeneous cell, N = 16, hard spheres, 20 Heun steps of dt = 0.01
    (40 evaluations), FP64 plain and FP32 paths, against the oracle's trajectory."""
    n, lam, eps, dt, nsteps = 16, 1.0, 1.0, 0.01, 20
    ctx.init_weights([(n, L, lam)])
    f0 = inputs.homogeneous_cells(n, L, 1, seed=1)
    ref = [f0]
    for _ in range(nsteps):
        ref.append(oracle.rk2_homogeneous(n, L, lam, ref[-1], dt, eps))
    res = {}
    sampler.start()
    n0 = ctx.launch_count()
    for name, mode in (("fp64_plain", bte.FP64_PLAIN), ("fp32", bte.FP32)):
        f = torch.from_numpy(f0.copy()).cuda().reshape(-1)
        with torch.cuda.stream(stream):
            for _ in range(max(args.warmup, 3)):
                ctx.step(f, dt, eps, mode=mode, stream=stream)
        ctx.sync_status(stream)
        f.copy_(torch.from_numpy(f0.reshape(-1)))
        torch.cuda.synchronize()
        states, ev = [], []
        with torch.cuda.stream(stream):
            for i in range(nsteps):
                flush.fill_(i & 0xff)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.step(f, dt, eps, mode=mode, stream=stream)
                e1.record(stream)
                states.append(f.clone())  # after the step's events
                ev.append((e0, e1))
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        ctx.sync_status(stream)
        traj = np.stack([x.cpu().numpy() for x in states])
        err = max(np.linalg.norm(traj[i] - ref[i + 1][0]) / np.linalg.norm(ref[i + 1][0]) for i in range(nsteps))
        m0 = oracle.moments(n, L, f0)[0]
        m1 = oracle.moments(n, L, traj[-1:])[0]
        drift = float(np.abs(m1 - m0).max() / max(abs(m0[0]), abs(m0[4])))
        tot = float(sum(ms))
        res[name] = {"evals_per_s": 2 * nsteps / (tot * 1e-3), "us_per_eval": 1e3 * tot / (2 * nsteps),
                     "rel_l2_vs_oracle_trajectory_max": float(err), "moment_drift_rel": drift,
                     "ms_trajectory": tot}
    launches = ctx.launch_count() - n0
    clocks = sampler.stop()
    wl = ("space-homogeneous 1 cell, N=16, L=6, hard spheres, eps=1, bi-Maxwellian (seed 1), "
          "20 Heun steps dt=0.01 = 40 evals, projection each stage")
    return _line(args, "cell-collision evals/s (1 cell, FP64 plain operator)", res["fp64_plain"]["evals_per_s"],
                 UNIT, res["fp64_plain"]["ms_trajectory"] / nsteps, wl,
                 {"steps": nsteps, "dtype": "f64", "fp64_plain": res["fp64_plain"], "fp32": res["fp32"],
                  "gpu_launches": launches, "clocks": clocks})


def run_sweep32(args, ctx, torch, bte, inputs, oracle, stream, flush, sampler, n=32):
    """256 bi-Maxwellian cells at N = 32 (means ~ U(-1.5, 1.5)^3), FP32 operator;
    oracle on 16 seeded cells; plain FP64 operator timed once. With n = 48 (the
    sweep-n48 workload): 64 cells, the stored FP32 table (10 GB, built on first
    use in a few seconds) with the autotuned variant (--conv-impl 5 builds the
    weights on the fly instead), oracle on 2 cells, no FP64 comparator (its
    table: 41 GB)."""
    lam, nc = 1.0, args.cells if n == 32 else min(args.cells, 64)
    ctx.init_weights([(n, L, lam)])
    if n > 32 and args.conv_impl is not None:
        ctx.set_option("conv_impl", args.conv_impl)
    fn = inputs.precision_sweep_cells(n, L, nc, seed=3)
    f = torch.from_numpy(fn).cuda().reshape(-1)
    Q = torch.empty_like(f)
    explicit = args.conv_impl is not None or args.conv_warps is not None
    tuned = None if explicit else tune(args, ctx, f, stream, reps=2)
    ctx.profile_enable(True)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            ctx.collide(f, Q, mode=bte.FP32, stream=stream)
    ctx.sync_status(stream)
    ctx.profile_read("*", stream)
    conv = [0.0, 0]

    def one():
        ctx.collide(f, Q, mode=bte.FP32, stream=stream)

    sampler.start()
    n0 = ctx.launch_count()
    ms = _timed_steps(torch, one, args.steps, stream, flush)
    launches = ctx.launch_count() - n0
    clocks = sampler.stop()
    k, t = ctx.profile_read("conv32", stream)
    conv = [t, k]
    ctx.sync_status(stream)
    Qg = Q.cpu().numpy().reshape(nc, -1)
    tot = float(sum(ms))
    value = nc * args.steps / (tot * 1e-3)
    # plain FP64 operator (table build and first call outside the timing)
    fp64_value = None
    if n <= 32:
        Q64 = torch.empty_like(f)
        with torch.cuda.stream(stream):
            ctx.collide(f, Q64, mode=bte.FP64_PLAIN, stream=stream)
        ctx.sync_status(stream)
        ms64 = _timed_steps(torch, lambda: ctx.collide(f, Q64, mode=bte.FP64_PLAIN, stream=stream), 1, stream,
                            flush)
        fp64_value = nc / (ms64[0] * 1e-3)
    pick = np.sort(np.random.default_rng(3).choice(nc, 16 if n <= 32 else 2, replace=False))
    Qo = oracle.collide(n, L, lam, fn[pick])
    Qm = oracle.collide(n, L, lam, fn[pick], part=1, project=False)
    rel = np.linalg.norm(Qg[pick] - Qo, axis=1) / np.linalg.norm(Qm, axis=1)
    relp = np.linalg.norm(Qg[pick] - Qo, axis=1) / np.linalg.norm(Qo, axis=1)
    peak, clk = _alu_peak(clocks)
    fma = _measured_fma(ctx, stream)
    pairs = conv_pairs_per_cell(n)
    conv_ms = conv[0] / max(conv[1], 1)
    achieved = 10.0 * pairs * nc / (conv_ms * 1e-3) / 1e12
    wl = ("precision sweep: %d bi-Maxwellian cells (means ~ U(-1.5,1.5)^3, T ~ U(0.5,2), seed 3), "
          "N=%d, L=6, hard spheres; one projected collision evaluation of all cells per step%s"
          % (nc, n, "; weights built on the fly (conv_impl 5)" if args.conv_impl == 5 else
             ("; stored FP32 weight table (10 GB)" if n > 32 else "")))
    return _line(args, "cell-collision evals/s at N=%d (FP32 operator)" % n, value, UNIT, tot / args.steps, wl, {
        "roofline": {"bound": "alu", "kernel": "conv32 (FP32 weighted convolution)", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "peak_basis": _peak_basis(clk, fma), "measured_fma": fma,
                     "flops_per_launch": 10.0 * pairs * nc, "conv_ms_per_launch": conv_ms,
                     "weight_gbs": 4.0 * pairs / (conv_ms * 1e-3) / 1e9},
        "fp64_plain": ({"value": fp64_value, "unit": UNIT, "speedup_fp32_over_fp64": value / fp64_value}
                       if fp64_value else None),
        "conv_impl": ctx.get_option("conv_impl") if tuned is None else tuned.get("conv_impl"),
        "autotuned": tuned,
        "accuracy": {"rel_l2_loss_norm_max": float(rel.max()), "rel_l2_loss_norm_median": float(np.median(rel)),
                     "rel_l2_plain_max": float(relp.max()), "cells_checked": pick.tolist(),
                     "moment_rel_max": _moment_rel(oracle, n, Qg)},
        "gpu_launches": launches, "clocks": clocks})


def run_uneven(args, ctx, torch, bte, inputs, oracle, stream, flush, sampler):
    """4096 homogeneous instances, N in {12,16,24,32} (p = .4/.3/.2/.1), lambda in
    {0,1}; one Heun step of the whole batch per step (one CUDA graph)."""
    Ns, lams = (12, 16, 24, 32), (0.0, 1.0)
    grids = [(n, L, lam) for n in Ns for lam in lams]
    ids = dict(zip([(g[0], g[2]) for g in grids], ctx.init_weights(grids)))
    items = inputs.uneven_batch(4096, seed=4)
    offs, off = [], 0
    for (n, lam, fi) in items:
        offs.append(off)
        off += n ** 3
    buf = np.empty(off)
    for (n, lam, fi), o in zip(items, offs):
        buf[o:o + fi.size] = fi
    inst = [(ids[(n, lam)], o) for (n, lam, _), o in zip(items, offs)]
    dt, eps = 0.01, 1.0
    f = torch.from_numpy(buf).cuda()
    tuned = tune(args, ctx, f, stream, inst=inst, reps=2)
    ctx.profile_enable(True)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            ctx.step(f, dt, eps, inst=inst, mode=bte.FP32, stream=stream)
    ctx.sync_status(stream)
    ctx.profile_read("*", stream)
    sampler.start()
    n0 = ctx.launch_count()
    ms = _timed_steps(torch, lambda: ctx.step(f, dt, eps, inst=inst, mode=bte.FP32, stream=stream),
                      args.steps, stream, flush)
    launches = ctx.launch_count() - n0
    clocks = sampler.stop()
    k, t = ctx.profile_read("conv32", stream)
    ctx.sync_status(stream)
    tot = float(sum(ms))
    evals = 2 * len(items)
    value = evals * args.steps / (tot * 1e-3)
    flops_step = sum(2 * 10.0 * conv_pairs_per_cell(n) for (n, _, _) in items)
    conv_ms = t / max(k, 1)
    peak, clk = _alu_peak(clocks)
    fma = _measured_fma(ctx, stream)
    achieved = flops_step / 2 / (conv_ms * 1e-3) / 1e12
    # accuracy of one collision evaluation of the batch on sampled instances
    fb = torch.from_numpy(buf).cuda()
    Q = ctx.collide(fb, inst=inst, mode=bte.FP32, stream=stream)
    ctx.sync_status(stream)
    Qn = Q.cpu().numpy()
    rng = np.random.default_rng(4)
    errs = {}
    for n in Ns:
        cand = [i for i, it in enumerate(items) if it[0] == n]
        for i in rng.choice(cand, 2 if n < 32 else 1, replace=False):
            n_, lam, fi = items[i]
            qo = oracle.collide(n_, L, lam, fi[None])[0]
            qm = oracle.collide(n_, L, lam, fi[None], part=1, project=False)[0]
            e = float(np.linalg.norm(Qn[offs[i]:offs[i] + n_ ** 3] - qo) / np.linalg.norm(qm))
            errs[n] = max(errs.get(n, 0.0), e)
    mix = {str(n): sum(1 for it in items if it[0] == n) for n in Ns}
    wl = ("uneven batch: 4096 space-homogeneous instances, N in {12,16,24,32} w.p. .4/.3/.2/.1, lambda in "
          "{0,1} w.p. .5/.5 (8 tables), BKW or bi-Maxwellian data (seed 4); one Heun step of the whole batch "
          "(2 evals per instance) replayed from one CUDA graph")
    return _line(args, "cell-collision evals/s, uneven batch (FP32 operator)", value, UNIT, tot / args.steps, wl, {
        "instances_by_N": mix, "evals_per_step": evals, "autotuned": tuned,
        "roofline": {"bound": "alu", "kernel": "conv32 (FP32 weighted convolution, all sizes in one launch)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "conv_ms_per_launch": conv_ms,
                     "peak_basis": _peak_basis(clk, fma), "measured_fma": fma},
        "flop_rate_whole_step_tflops": flops_step / (tot / args.steps * 1e-3) / 1e12,
        "accuracy": {"rel_l2_loss_norm_max_by_N": {str(k_): v for k_, v in errs.items()}},
        "gpu_launches": launches, "clocks": clocks})


def _surrogate_gemm_rates(torch, ctx, rows, info, stream, reps=10):
    """The surrogate's three layer GEMMs at the inference shape (rows = cells in
    the batch), each timed alone on the tensor-core kernel (bf16 in, FP32
    accumulate) with CUDA events: TFLOP/s against the measured bf16 peak."""
    width, ndim = int(info["width"]), int(info["ndim"])
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peak, basis = float(json.load(fh)["bf16_tflops"]), "of measured (cuBLAS bf16 burst)"
    except (OSError, ValueError, KeyError):
        peak, basis = 1900.0, "of fallback"
    g = torch.Generator(device="cuda").manual_seed(0)
    out = []
    for name, (M, N, K) in (("W1", (rows, width, ndim)), ("W2", (rows, width, width)), ("W3", (rows, ndim, width))):
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
        with torch.cuda.stream(stream):
            for _ in range(3):
                ctx.tc_gemm(A, B, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                ctx.tc_gemm(A, B, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
        out.append({"layer": name, "M": M, "N": N, "K": K, "us": ms * 1e3, "tflops": tf, "frac": tf / peak})
    ctx.sync_status(stream)
    return {"peak_tflops": peak, "peak_basis": basis, "layers": out,
            "note": "each GEMM alone, FP32 output (the surrogate fuses bias, GELU and the bf16 store instead)"}


def run_learned(args, ctx, torch, bte, inputs, oracle, stream, flush, sampler):
    """Surrogate trained on seeded pairs (f, Q_FP32(f)) at N = 16, evaluated with the
    fallback indicator on 1024 cells of the wall-heating slab after 200 steps."""
    from paper_1211_0540_gb300 import surrogate
    n, lam, nx = 16, 1.0, 1024
    M = n ** 3
    ctx.init_weights([(n, L, lam)])
    ctx.mlp_init(0, 1024, seed=1)
    t0 = time.perf_counter()
    f_tr, Q_tr = surrogate.make_training_set(ctx, n, L, args.train_states, seed=5)
    t_data = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = surrogate.train(ctx, f_tr, Q_tr, n, L, epochs=args.epochs, batch=1024, lr=1e-3, seed=0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del f_tr, Q_tr
    info = ctx.mlp_info()
    # evaluation states: the wall-heating slab at nx = 1024 after 200 Strang steps
    fw = torch.from_numpy(inputs.wall_heating_initial(n, L, nx)).cuda().reshape(-1)
    tr = dict(nx=nx, x0=0.0, x1=1.0, bc_left=bte.BC_DIFFUSE, bc_right=bte.BC_SPECULAR, Tw_left=TW,
              Tw_right=1.0)
    with torch.cuda.stream(stream):
        for _ in range(200):
            ctx.step(fw, 0.5 * (1.0 / nx) / L, EPS, transport=tr, mode=bte.FP32, stream=stream)
    ctx.sync_status(stream)
    # the FP32 configuration of the 1024-cell batch (its collide, and the
    # indicator's forward transform of the same batch); untimed
    tuned = tune(args, ctx, fw, stream, reps=5)
    Q32 = torch.empty_like(fw)
    Ql = torch.empty_like(fw)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            ctx.collide(fw, Q32, mode=bte.FP32, stream=stream)
            ctx.collide(fw, Ql, mode=bte.LEARNED, stream=stream)
    ctx.sync_status(stream)
    ctx.learned_stats(reset=True)
    sampler.start()
    n0 = ctx.launch_count()
    ms_l = _timed_steps(torch, lambda: ctx.collide(fw, Ql, mode=bte.LEARNED, stream=stream), args.steps,
                        stream, flush, tag="learned")
    launches = ctx.launch_count() - n0
    clocks = sampler.stop()
    st = ctx.learned_stats(reset=True)
    Qs = torch.empty_like(fw)  # the timed variants below must not overwrite Ql
    ms_nn = _timed_steps(torch, lambda: ctx.collide(fw, Qs, mode=bte.LEARNED, fallback=False, stream=stream),
                         args.steps, stream, flush, tag="surrogate")
    tol0 = ctx.get_option("learned_tol_ppm")
    ctx.set_option("learned_tol_ppm", LEARNED_TOL_OFF)  # indicator evaluated, no cell falls back
    try:
        ms_ind = _timed_steps(torch, lambda: ctx.collide(fw, Qs, mode=bte.LEARNED, stream=stream),
                              args.steps, stream, flush, tag="indicator")
    finally:
        ctx.set_option("learned_tol_ppm", tol0)
    ms_f = _timed_steps(torch, lambda: ctx.collide(fw, Q32, mode=bte.FP32, stream=stream), args.steps,
                        stream, flush, tag="fp32")
    Q64 = torch.empty_like(fw)
    with torch.cuda.stream(stream):
        ctx.collide(fw, Q64, mode=bte.FP64_PLAIN, stream=stream)
    ms_64 = _timed_steps(torch, lambda: ctx.collide(fw, Q64, mode=bte.FP64_PLAIN, stream=stream), 1,
                         stream, flush, tag="fp64")
    # whole Strang steps of the slab (two transport half steps and a Heun step
    # whose two stages use the learned collide, fallback included), against
    # the same steps with the FP32 operator; each from a copy of the state
    dt = 0.5 * (1.0 / nx) / L
    steps = {}
    for name, mode in (("learned", bte.LEARNED), ("fp32", bte.FP32)):
        fs = fw.clone()
        with torch.cuda.stream(stream):
            for _ in range(3):
                ctx.step(fs, dt, EPS, transport=tr, mode=mode, stream=stream)
        ctx.sync_status(stream)
        ctx.learned_stats(reset=True)
        ms = _timed_steps(torch, lambda: ctx.step(fs, dt, EPS, transport=tr, mode=mode, stream=stream),
                          args.steps, stream, flush, tag="step-" + name)
        sst = ctx.learned_stats(reset=True)
        steps[name] = {"value": 2 * nx * args.steps / (sum(ms) * 1e-3), "unit": UNIT,
                       "ms_per_step": sum(ms) / args.steps}
        if name == "learned":
            steps[name]["fallback_rate"] = sst["fallbacks"] / max(sst["cells"], 1)
    steps["note"] = ("one Strang step of the 1024-cell slab = 2048 collision evaluations, replayed from a "
                     "captured graph (the learned one builds its fallback list on the device)")
    Qnn = ctx.collide(fw, mode=bte.LEARNED, fallback=False, stream=stream)
    ctx.sync_status(stream)
    a32, al, ann = (x.cpu().numpy().reshape(nx, M) for x in (Q32, Ql, Qnn))
    fwn = fw.cpu().numpy().reshape(nx, M)
    # errors normalised by the loss term (Q itself is near 0 in the equilibrated interior), every cell
    pick = np.arange(nx)
    qm = np.linalg.norm(oracle.collide(n, L, lam, fwn, part=1, project=False), axis=1)
    qo = oracle.collide(n, L, lam, fwn)
    e_l = np.linalg.norm(al[pick] - qo, axis=1) / qm
    e_nn = np.linalg.norm(ann[pick] - qo, axis=1) / qm
    e_32 = np.linalg.norm(a32[pick] - qo, axis=1) / qm
    v_l = nx * args.steps / (sum(ms_l) * 1e-3)
    v_f = nx * args.steps / (sum(ms_f) * 1e-3)
    v_64 = nx / (ms_64[0] * 1e-3)
    gemms = _surrogate_gemm_rates(torch, ctx, nx, info, stream)
    wl = ("learned surrogate (residual MLP, width 1024, BF16 tensor cores) + P_N + fallback indicator "
          "(64 zeta points, tolerance 1e-2) on 1024 cells of the wall-heating slab (N=16, L=6, lambda=1, "
          "Kn=0.1) after 200 FP32 Strang steps; trained on %d seeded pairs, %d epochs" % (args.train_states,
                                                                                        args.epochs))
    return _line(args, "cell-collision evals/s, learned mode with fallback (N=16)", v_l, UNIT,
                 sum(ms_l) / args.steps, wl, {
        "dtype": "bf16",
        "fp32": {"value": v_f, "unit": UNIT}, "fp64_plain": {"value": v_64, "unit": UNIT},
        "surrogate_only": {"value": nx * args.steps / (sum(ms_nn) * 1e-3), "unit": UNIT,
                           "note": "surrogate + projection, no indicator and no fallback"},
        "surrogate_indicator": {"value": nx * args.steps / (sum(ms_ind) * 1e-3), "unit": UNIT,
                                "note": "surrogate + projection + indicator, threshold set so that no cell "
                                        "falls back"},
        "surrogate_gemms": gemms,
        "strang_steps": steps,
        "autotuned": tuned,
        "fallback": {"cells": st["cells"], "fallbacks": st["fallbacks"],
                     "rate": st["fallbacks"] / max(st["cells"], 1), "max_indicator": st["max_indicator"]},
        "accuracy": {"norm": "||Q - Q_oracle|| / ||Q_loss_oracle|| on all %d cells" % len(pick),
                     "learned_with_fallback_max": float(e_l.max()),
                     "learned_with_fallback_median": float(np.median(e_l)),
                     "surrogate_only_max": float(e_nn.max()), "surrogate_only_median": float(np.median(e_nn)),
                     "fp32_max": float(e_32.max()), "cells_checked": int(len(pick))},
        "training": {"states": args.train_states, "epochs": args.epochs, "final_loss": float(loss),
                     "data_s": t_data, "train_s": t_train,
                     "samples_per_s": args.train_states * args.epochs / t_train, "params": info},
        "gpu_launches": launches, "clocks": clocks})


def run_wall200(args, ctx, torch, bte, inputs, oracle, stream, flush, sampler):
    """The wall-heating slab over 200 Strang steps with the FP32 path and with the
    plain FP64 operator: conservation drift of each trajectory, the FP32 state's
    deviation from the FP64 one, and the FP32 operator against the oracle on
    sampled cells of the final state."""
    nsteps = 200
    ctx.init_weights([(N, L, LAM)])
    tr = dict(nx=NX, x0=0.0, x1=1.0, bc_left=bte.BC_DIFFUSE, bc_right=bte.BC_SPECULAR, Tw_left=TW,
              Tw_right=1.0)
    f0 = inputs.wall_heating_initial(N, L, NX)
    tuned = tune(args, ctx, torch.from_numpy(f0).cuda(), stream, reps=5)
    out, ms = {}, {}
    sampler.start()
    for name, mode in (("fp32", bte.FP32), ("fp64_plain", bte.FP64_PLAIN)):
        f = torch.from_numpy(f0.copy()).cuda()
        with torch.cuda.stream(stream):
            ctx.step(f, DT, EPS, transport=tr, mode=mode, stream=stream)  # capture, then restart
        ctx.sync_status(stream)
        f.copy_(torch.from_numpy(f0))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(nsteps):
                ctx.step(f, DT, EPS, transport=tr, mode=mode, stream=stream)
            e1.record(stream)
        ctx.sync_status(stream)
        ms[name] = e0.elapsed_time(e1)
        out[name] = f.cpu().numpy().reshape(NX, -1)
    clocks = sampler.stop()
    m0 = oracle.moments(N, L, f0).sum(axis=0)
    drift = {}
    for name, fs in out.items():
        m = oracle.moments(N, L, fs).sum(axis=0)
        # mass is conserved by the walls; momentum and energy change through the walls
        drift[name] = {"mass_rel": float(abs(m[0] - m0[0]) / m0[0])}
    dev = float(np.abs(out["fp32"] - out["fp64_plain"]).max() / np.abs(out["fp64_plain"]).max())
    pick = [0, 1, 2, 8, 64, NX - 1]
    Qg = ctx.collide(torch.from_numpy(out["fp32"]).cuda().reshape(-1), mode=bte.FP32, stream=stream)
    ctx.sync_status(stream)
    Qg = Qg.cpu().numpy().reshape(NX, -1)
    Qo = oracle.collide(N, L, LAM, out["fp32"][pick])
    Qm = oracle.collide(N, L, LAM, out["fp32"][pick], part=1, project=False)
    rel = np.linalg.norm(Qg[pick] - Qo, axis=1) / np.linalg.norm(Qm, axis=1)
    value = EVALS_PER_STEP * nsteps / (ms["fp32"] * 1e-3)
    wl = ("sudden wall heating, 200 Strang steps (the run of the paper's Sec. 5 set-up at Kn = 0.1): 128 "
          "cells, N = 16, L = 6, hard spheres, Tw = 2 diffuse / specular, CFL 0.5; FP32 path and plain "
          "FP64 operator from the same initial state")
    return _line(args, METRIC, value, UNIT, ms["fp32"] / nsteps, wl, {
        "steps": nsteps, "fp64_plain": {"value": EVALS_PER_STEP * nsteps / (ms["fp64_plain"] * 1e-3), "unit": UNIT},
        "autotuned": tuned, "conservation": drift,
        "accuracy": {"state_max_dev_fp32_vs_fp64_rel": dev,
                     "final_state_Q_rel_l2_loss_norm_max": float(rel.max()), "cells_checked": pick},
        "clocks": clocks})


def run_refined(args, ctx, torch, bte, inputs, oracle, stream, flush, sampler):
    """The paper's own sudden-heating set-up (Sec. 5): Knudsen number 1, eight
    cells per mean free path at the heated wall and two inside (56 cells of
    unequal width on [0, 20]), diffuse wall at T = 2, no flux for incoming
    characteristics at the far end; N = 16, hard spheres; 100 Strang steps at
    CFL 0.5 of the smallest cell, FP32 path and plain FP64 operator."""
    n, lam, eps, nsteps = 16, 1.0, 1.0, 100
    dx = inputs.sudden_heating_grid()
    nx = dx.size
    ctx.init_weights([(n, L, lam)])
    dt = 0.5 * dx.min() / L
    tr = dict(nx=nx, dx=list(dx), bc_left=bte.BC_DIFFUSE, bc_right=bte.BC_NOFLUX, Tw_left=TW, Tw_right=1.0)
    f0 = inputs.wall_heating_initial(n, L, nx)
    tuned = tune(args, ctx, torch.from_numpy(f0).cuda(), stream, reps=5)
    out, ms = {}, {}
    sampler.start()
    n0 = ctx.launch_count()
    for name, mode in (("fp32", bte.FP32), ("fp64_plain", bte.FP64_PLAIN)):
        f = torch.from_numpy(f0.copy()).cuda()
        with torch.cuda.stream(stream):
            ctx.step(f, dt, eps, transport=tr, mode=mode, stream=stream)  # capture, then restart
        ctx.sync_status(stream)
        f.copy_(torch.from_numpy(f0))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(nsteps):
                ctx.step(f, dt, eps, transport=tr, mode=mode, stream=stream)
            e1.record(stream)
        ctx.sync_status(stream)
        ms[name] = e0.elapsed_time(e1)
        out[name] = f.cpu().numpy().reshape(nx, -1)
        if name == "fp32":
            launches = ctx.launch_count() - n0
    clocks = sampler.stop()
    dv3 = (2 * L / n) ** 3
    mass = {k: float((dx[:, None] * v).sum() * dv3) for k, v in out.items()}
    dev = float(np.abs(out["fp32"] - out["fp64_plain"]).max() / np.abs(out["fp64_plain"]).max())
    pick = [0, 1, 8, 16, 30, nx - 1]
    Qg = ctx.collide(torch.from_numpy(out["fp32"]).cuda().reshape(-1), mode=bte.FP32, stream=stream)
    ctx.sync_status(stream)
    Qg = Qg.cpu().numpy().reshape(nx, -1)
    Qo = oracle.collide(n, L, lam, out["fp32"][pick])
    Qm = oracle.collide(n, L, lam, out["fp32"][pick], part=1, project=False)
    rel = np.linalg.norm(Qg[pick] - Qo, axis=1) / np.linalg.norm(Qm, axis=1)
    evals = 2 * nx
    value = evals * nsteps / (ms["fp32"] * 1e-3)
    # bulk velocity profile u1(x) of the final state (the quantity of the paper's Fig. 1)
    v1 = inputs.velocity_nodes(n, L)[0].ravel()
    rho = out["fp32"].sum(axis=1) * dv3
    u1 = (out["fp32"] * v1).sum(axis=1) * dv3 / rho
    wl = ("sudden heating on the paper's refined grid (Sec. 5): Kn = 1, 56 cells of [0, 20] (dx 1/8 at the wall, "
          "~1/2 inside), diffuse wall Tw = 2 / no flux for incoming characteristics, N = 16, L = 6, hard spheres, "
          "100 Strang steps at CFL 0.5 of the smallest cell")
    return _line(args, "cell-collision evals/s, refined-grid sudden heating (FP32 operator)", value, UNIT,
                 ms["fp32"] / nsteps, wl, {
        "steps": nsteps, "fp64_plain": {"value": evals * nsteps / (ms["fp64_plain"] * 1e-3), "unit": UNIT},
        "autotuned": tuned, "dt": dt,
        "mass": {"initial": float((dx[:, None] * f0).sum() * dv3), "final": mass,
                 "note": "the open boundary lets gas leave; the diffuse wall keeps its own balance"},
        "bulk_velocity_u1": {"x_centres": (np.cumsum(dx) - 0.5 * dx).round(4).tolist(), "u1": u1.round(6).tolist()},
        "accuracy": {"state_max_dev_fp32_vs_fp64_rel": dev,
                     "final_state_Q_rel_l2_loss_norm_max": float(rel.max()), "cells_checked": pick},
        "gpu_launches": launches, "clocks": clocks})


def run_models(args, ctx, torch, bte, inputs, oracle, stream, flush, sampler):
    """One projected FP32 collision evaluation of 128 bi-Maxwellian cells at N = 16
    for each collision model the weights encode (Sec. 2.2): hard spheres,
    variable hard potentials (lambda = 0.5, weights by quadrature), Maxwell
    molecules, variable soft potentials (lambda = -1, -2.5; Sec. 2.1), and
    inelastic collisions (beta = 0.8, 0.6; energy row dropped)."""
    n, nc = 16, 128
    models = [(1.0, 1.0), (0.5, 1.0), (0.0, 1.0), (-1.0, 1.0), (-2.5, 1.0), (1.0, 0.8), (0.0, 0.6)]
    ids = ctx.init_weights([(n, L, lam, beta) for lam, beta in models])
    f = inputs.homogeneous_cells(n, L, nc, seed=9)
    M = n ** 3
    buf = np.concatenate([f.reshape(-1)] * len(models))
    fb = torch.from_numpy(buf).cuda()
    rows = []
    sampler.start()
    tuned = None
    for k, (lam, beta) in enumerate(models):
        inst = [(ids[k], (k * nc + c) * M) for c in range(nc)]
        if k == 0:  # one batch shape for all models: one configuration
            tuned = tune(args, ctx, fb, stream, inst=inst, reps=3)
        Q = torch.zeros_like(fb)
        with torch.cuda.stream(stream):
            for _ in range(3):
                ctx.collide(fb, Q, inst=inst, mode=bte.FP32, stream=stream)
        ms = _timed_steps(torch, lambda: ctx.collide(fb, Q, inst=inst, mode=bte.FP32, stream=stream), args.steps,
                          stream, flush, tag="model%d" % k)
        ctx.sync_status(stream)
        Qg = Q.cpu().numpy()[k * nc * M:(k + 1) * nc * M].reshape(nc, M)
        pick = [0, 37, nc - 1]
        Qo = oracle.collide(n, L, lam, f[pick], beta=beta)
        Qm = oracle.collide(n, L, lam, f[pick], part=1, project=False, beta=beta)
        rel = np.linalg.norm(Qg[pick] - Qo, axis=1) / np.linalg.norm(Qm, axis=1)
        mom = oracle.moments(n, L, Qg)
        rows.append({"lambda": lam, "beta": beta, "evals_per_s": nc * args.steps / (sum(ms) * 1e-3),
                     "rel_l2_loss_norm_max": float(rel.max()), "cells_checked": pick,
                     "max_abs_mass_momentum_moment": float(np.abs(mom[:, :4]).max()),
                     "energy_moment_mean": float(mom[:, 4].mean())})
    clocks = sampler.stop()
    wl = ("collision models in the weights (Sec. 2.2): 128 bi-Maxwellian cells at N = 16, L = 6; (lambda, beta) "
          "= (1, 1), (0.5, 1), (0, 1), (-1, 1), (-2.5, 1), (1, 0.8), (0, 0.6); one projected FP32 evaluation per step")
    value = rows[0]["evals_per_s"]
    return _line(args, "cell-collision evals/s per collision model (FP32 operator, N=16)", value, UNIT,
                 nc / value * 1e3, wl, {"models": rows, "autotuned": tuned, "clocks": clocks})


def run_secondary(args):
    import torch

    import oracle
    from paper_1211_0540_gb300 import bte, inputs

    rank, world, local = dist_env()
    if world > 1:
        raise SystemExit("secondary workloads run on one GPU")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    ctx = bte.Context(local)
    if args.conv_impl is not None:
        ctx.set_option("conv_impl", args.conv_impl)
    if args.conv_warps is not None:
        ctx.set_option("conv_warps", args.conv_warps)
    if args.conv_split is not None:
        ctx.set_option("conv_split", args.conv_split)
    if args.dft_split is not None:
        ctx.set_option("dft_split", args.dft_split)
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    sampler = ClockSampler(local)
    fn = {"homog-1cell": run_homog1, "sweep-n32": run_sweep32,
          "sweep-n48": lambda *a: run_sweep32(*a, n=48), "uneven-4096": run_uneven,
          "learned-n16": run_learned, "wall-heating-200": run_wall200, "sudden-heating-refined": run_refined,
          "collision-models": run_models}[args.workload]
    line = fn(args, ctx, torch, bte, inputs, oracle, stream, flush, sampler)
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())

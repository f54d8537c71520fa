#!/usr/bin/env python
"""Benchmark of the CVO hot path on one GB300 (or N replicas).

Workload: one VGA-scale frame pair. A procedural room is ray-cast to 640x480
depth + colour, the high-gradient pixels are kept and subsampled to 20,000
points per frame, and the second frame follows a 3 deg / 3 cm camera motion.
One step is one full solve (cvo_align) from the identity: every iteration's
gradient pass, step pass, FP64 step and exponential-map update, on the device.

Metric: pair evaluations per second (Gpairs/s). A pair evaluation is one kept
(in-cutoff) (i, j) pair in one gradient or step pass. frame_pairs_per_s is
reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cvo|reference]

For N > 1 launch under torch.distributed.run. Every rank solves its own copy
of the workload (the solve does not shard; replicas only), and the value is
all ranks' pairs divided by the slowest rank's time.

--impl reference times the FP64 CPU oracle on this machine's host cores on a
bounded sample of the same workload: each step is one iteration (gradient
pass + step pass) of the solve.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "CVO pair evals/sec (Gpairs/s) and frame-pairs/sec; p50/p99 served latency vs plain"
UNIT = "Gpairs/s"
N_POINTS = 20000
WORKLOAD = ("room VGA pair: 640x480 ray-cast room (6x5x3 m box + 20 cuboids), "
            "80th-percentile gradient pixels subsampled to 20000 points/frame, 3 deg / 3 cm "
            "motion, 5-D features, ell 0.15 x0.9 -> 0.02, kcut 1e-3, <= 200 iterations")

# FP32 roofline of the pair passes (GB300: 152 SMs x 128 FP32 lanes, FMA = 2 flops,
# 2070 MHz maximum SM clock) and the FP32 flops each kept pair needs.
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
PEAK_FP32_TFLOPS = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12


def flops_per_pair(D: int) -> dict:
    """Algorithmic FP32 flops per kept pair (FMA = 2). Gradient pass:
    e (3) + |e|^2 (5) + feature difference and norm (3D - 1) + exponent (2) +
    accumulation of w and w e (7). Step pass: e, |e|^2, features, exponent as
    above, beta (5), gamma/delta/eps (18), g2..g4 (16), accumulation of S0..S4 (9)."""
    return {"grad": 16 + 3 * D, "step": 57 + 3 * D}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cvo", choices=["cvo", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline_sample(d, n_iters: int, prm=None):
    """The oracle as it stands, timed on the host cores: the first n_iters
    iterations of the same solve. Returns (Gpairs/s, cores, seconds, pairs)."""
    import oracle
    prm = prm or oracle.Params(max_iters=n_iters)
    t0 = time.perf_counter()
    r = oracle.align(d["X"], d["FX"], d["Z"], d["FZ"], np.eye(4), prm)
    dt = time.perf_counter() - t0
    return r["pair_evals"] / dt / 1e9, oracle.num_threads(), dt, r["pair_evals"]


def run_reference(args, world, rank):
    """FP64 CPU oracle arm: each step is one iteration of the solve."""
    if rank != 0:
        return
    import oracle
    d = synth.room_pair(N_POINTS, seed=synth.seed_for(2))
    prm = oracle.Params()
    ells = oracle.ell_schedule(prm, 8)
    P = np.eye(4)
    times, pairs = [], 0
    for k in range(args.warmup + args.steps):
        ell = ells[k % len(ells)]
        t0 = time.perf_counter()
        s = oracle.pair_sums(d["X"], d["FX"], d["Z"], d["FZ"], P, ell, prm)
        xi = oracle.gradient(s, prm)
        s2 = oracle.pair_sums(d["X"], d["FX"], d["Z"], d["FZ"], P, ell, prm, xi=xi)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            pairs += s["nnz"] + s2["nnz"]
    total = sum(times)
    value = pairs / total / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "l2": "inputs re-read from host memory"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": "one solve iteration (gradient + step pass, exhaustive "
                                       "all-pairs FP64) per step, ell cycling over the first 8 "
                                       "schedule values, identity pose, full 20000x20000 pair"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_cvo(args, world, rank, local):
    import torch

    import paper_1904_02266_gb300 as cvo
    from paper_1904_02266_gb300 import build as cvo_build

    cvo_build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    d = synth.room_pair(N_POINTS, seed=synth.seed_for(2))
    X, FX, Z, FZ = d["X"], d["FX"], d["Z"], d["FZ"]
    D = FX.shape[1]
    ctx = cvo.Context(device=local)
    ht, hs = ctx.set_cloud(X, FX), ctx.set_cloud(Z, FZ)
    stream = torch.cuda.ExternalStream(ctx.stream, device=torch.device("cuda", local))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=f"cuda:{local}")

    def timed(fn, n):
        tot_ms, outs = 0.0, []
        for _ in range(n):
            with torch.cuda.stream(stream):
                flush.zero_()              # evict the 129 MB L2 between steps
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            out = fn()
            with torch.cuda.stream(stream):
                e1.record(stream)
            e1.synchronize()
            tot_ms += e0.elapsed_time(e1)
            outs.append(out)
        return tot_ms, outs

    for _ in range(max(3, args.warmup)):
        ctx.align(ht, hs)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, outs = timed(lambda: ctx.align(ht, hs), args.steps)
        torch.cuda.synchronize()
    clocks = clk.summary()
    pairs = sum(o[1]["pair_evals"] for o in outs)
    iters = [o[1]["iters"] for o in outs]
    launches = len(iters)   # one solve_kernel launch per step
    P_final = outs[-1][0]

    # end to end through the public API from host buffers: upload both clouds
    # (grids, plan and graph are rebuilt for the new target), solve, read back
    def e2e_step():
        a, b = ctx.set_cloud(X, FX), ctx.set_cloud(Z, FZ)
        P, st = ctx.align(a, b)
        ctx.release(a)
        ctx.release(b)
        return st["pair_evals"]

    for _ in range(2):
        e2e_step()
    e2e_ms, e2e_pairs = timed(e2e_step, args.steps)
    h2d = X.nbytes + FX.nbytes + Z.nbytes + FZ.nbytes + 16 * 8
    import ctypes
    d2h = 16 * 8 + ctypes.sizeof(cvo.cvo_stats)

    # roofline of the solve kernel (the only kernel of a timed step): algorithmic
    # FP32 flops of the kept pairs of one solve over the CUDA-event time per
    # solve; the per-phase split comes from the kernel's own timestamps
    _, pst, recs = ctx.align_profile(ht, hs)
    fpp = flops_per_pair(D)
    grad_pairs = sum(r["grad_pairs"] for r in recs)
    step_pairs = sum(r["step_pairs"] for r in recs)
    cand = sum(r["grad_candidates"] for r in recs)
    flops_per_solve = grad_pairs * fpp["grad"] + step_pairs * fpp["step"]
    achieved = flops_per_solve / (ms / args.steps * 1e-3) / 1e12
    phases = {k: sum(r[k] for r in recs) for k in ("plan_ms", "grad_ms", "step_ms")}
    traffic = recorded_traffic("solve_kernel")

    # max over ranks
    total_ms = ms
    if dist:
        t = torch.tensor([ms, float(pairs), e2e_ms, float(sum(e2e_pairs))], dtype=torch.float64,
                         device=f"cuda:{local}")
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm_ = t.clone()
        dist.all_reduce(sm_, op=dist.ReduceOp.SUM)
        total_ms, pairs, e2e_ms = mx[0].item(), sm_[1].item(), mx[2].item()
        e2e_total_pairs = sm_[3].item()
    else:
        e2e_total_pairs = float(sum(e2e_pairs))
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = pairs / (total_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "points_per_frame": N_POINTS, "feat_dim": D,
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "frame_pairs_per_s": world * args.steps / (total_ms * 1e-3),
        "iters_per_solve": statistics.median(iters),
        "pair_evals_per_solve": pairs / (world * args.steps),
        "candidates_per_kept_pair": cand / max(1, grad_pairs),
        "pose_vs_truth": list(synth_pose_err(P_final, d["P_gt"])),
        "e2e": {"value": e2e_total_pairs / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms / args.steps},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": "solve_kernel", "achieved": achieved,
                     "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s", "frac": achieved / PEAK_FP32_TFLOPS,
                     "traffic": traffic,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz",
                     "flops_per_launch": flops_per_solve,
                     "phase_ms_per_solve": phases},
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and world == 1:
        v, cores, dt, cp = cpu_baseline_sample(d, 6)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"first 6 iterations of the same solve, exhaustive "
                                          f"FP64 all-pairs oracle ({cp} kept pair evals, "
                                          f"{dt:.1f} s)"}
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def recorded_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the
    summary was taken on the current kernel source (else None)."""
    import glob
    import hashlib
    src = os.path.join(ROOT, "paper_1904_02266_gb300", "csrc", "pair_kernels.cu")
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for path in glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_*.md")):
        fields = {}
        for line in open(path):
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip()
        if fields.get("source_sha256_16") == digest and "dram_bytes_per_launch" in fields:
            try:
                return float(fields["dram_bytes_per_launch"])
            except ValueError:
                return None
    return None


def synth_pose_err(P, Pref):
    dR = P[:3, :3] @ Pref[:3, :3].T
    c = np.clip((np.trace(dR) - 1) / 2, -1, 1)
    s = np.linalg.norm([dR[2, 1] - dR[1, 2], dR[0, 2] - dR[2, 0], dR[1, 0] - dR[0, 1]]) / 2
    return float(np.arctan2(s, c)), float(np.linalg.norm(P[:3, 3] - dR @ Pref[:3, 3]))


def main():
    args = parse_args()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_cvo(args, world, rank, local)


if __name__ == "__main__":
    main()

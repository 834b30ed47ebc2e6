#!/usr/bin/env python
"""Benchmark: codewords enumerated per second by the Brouwer-Zimmerman minimum-distance
run of one random binary [192,64] code (three full-rank information sets) on GB300.

One step = one whole Alg. 1 run over the prepared code (every (g, j) unit from g = 1
until L >= U) with d, the witness key and the counters exact.  `value` is timed with
CUDA events on the launching stream (inputs resident on the device); `e2e` is the same
run through the C-ABI from host buffers (prepare = information sets + host-to-device
copy, run, result read back) timed on the host clock.  `--impl reference` times the
CPU oracle on a bounded sample of the same run.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "codewords enumerated/s (XOR+POPC) and codes/s batched vs plain, 1 GB300, d exact"
UNIT = "codewords/s"
WORKLOADS = {
    "192x64": "single random [192,64] code, G=[I_64|R], R iid Bernoulli(1/2) from SplitMix64 "
              "(first seed >= 1 whose greedy information sets have ranks 64,64,64)",
    "150x64": "single random [150,64] code (ranks 64,64,22)",
    "300x50": "single random [300,50] code (six rank-50 sets)",
    "60x30": "single random [60,30] code, seed 1",
}
# POPC retired per SM per clock on compute capability 7.0-10.x (CUDA C++ Programming
# Guide, arithmetic-instruction throughput table: "population count" 16)
POPC_PER_CLK_SM = 16
L2_FLUSH_BYTES = 256 << 20


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.rows = []
        self.proc = None
        self.thread = None
        self.gpu_id = gpu_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        if not self.rows:
            return None
        clk = [float(r[1]) for r in self.rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(clk) if clk else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _gpu_uuid(torch, dev):
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:  # noqa: BLE001
        return None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except OSError:
        return {}


def workload(name):
    import synth.configs as cfg
    from paper_1603_06757_gb300 import api

    return cfg.single_code(name, lambda G, n, k: [int(r) for r in api.partition_host(G, n)["ranks"]])


def oracle_sample(G, n, max_g, nthreads):
    """Alg. 1 units (g, j), g <= max_g, of the oracle, in order; (codewords, seconds)."""
    import oracle

    part = oracle.partition(G, n)
    total = 0
    t0 = time.perf_counter()
    for g in range(1, max_g + 1):
        for j in range(part["m"]):
            r = oracle.enumerate_unit(part["gammas"][j], n, g, nthreads=nthreads, want_hist=False)
            total += r["count"]
    return total, time.perf_counter() - t0


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    import oracle

    n, k, seed, G = workload(args.workload)
    threads = os.cpu_count() or 1
    step_vals = []
    for i in range(args.warmup + args.steps):
        cw, sec = oracle_sample(G, n, args.ref_levels, threads)
        if i >= args.warmup:
            step_vals.append((cw, sec))
    cw = sum(c for c, _ in step_vals)
    sec = sum(s for _, s in step_vals)
    value = cw / sec
    sample = (f"Alg. 1 units (g, j), g <= {args.ref_levels}, of the {args.workload} code "
              f"({step_vals[0][0]} codewords per step)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "n": n, "k": k, "seed": seed, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np  # noqa: F401
    import torch

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__

    __graft_entry__.build()
    from paper_1603_06757_gb300 import api

    n, k, seed, G = workload(args.workload)
    stream = torch.cuda.current_stream()
    code = api.Code(G, n)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def step():
        code.reset()
        code.run()
        return code.result()

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()

    sampler = ClockSampler(_gpu_uuid(torch, local))
    sampler.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kernel_ms = 0.0
    launches = 0
    combos = 0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        res = step()
        ends[i].record(stream)
        kernel_ms += res["kernel_ms"]
        launches += res["launches"]
        combos += res["total_combos"]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms_max = float(t.item())
    value = world * combos / (total_ms_max / 1e3)

    # ---- end to end through the C-ABI from host buffers ----
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_cw = 0
    h2d = d2h = 0
    for _ in range(e2e_steps):
        r = api.min_distance(G, n)
        e2e_cw += r["total_combos"]
        h2d, d2h = r["h2d_bytes"], r["d2h_bytes"]
    torch.cuda.synchronize()
    e2e_sec = time.perf_counter() - t0
    t = torch.tensor([e2e_sec], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_value = world * e2e_cw / float(t.item())

    # ---- roofline of the enumerator kernel (bound: POPC pipe) ----
    info = api.device_info()
    peaks = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz") or info["max_sm_clock_khz"] / 1e3)
    part = api.partition_host(G, n)
    popc_per_cw = max(1, math.ceil((n - k) / 32)) if all(int(r) == k for r in part["ranks"]) else math.ceil(n / 32)
    peak = info["sm_count"] * sm_mhz * 1e6 * POPC_PER_CLK_SM / popc_per_cw
    achieved = combos / (kernel_ms / 1e3)
    try:
        mb = {w: api.microbench(w)["per_clock_per_sm"] for w in ("popc", "lop3", "step4")}
    except Exception:  # noqa: BLE001
        mb = None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        cw, sec = oracle_sample(G, n, args.cpu_levels, threads)
        cpu = {"value": cw / sec, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"Alg. 1 units (g, j), g <= {args.cpu_levels}, of the same code: {cw} codewords "
                         f"in {sec:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n": n, "k": k, "seed": seed, "d": res["d"],
                       "g_final": res["g_final"], "ranks": res["ranks"], "codewords_per_step": res["total_combos"],
                       "launches_per_step": res["launches"], "parallelism": f"replicas x{world}",
                       "l2": "flushed (256 MiB write) before every timed step; inputs ~2 KB"},
            "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gcodewords/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_basis": f"{info['sm_count']} SMs x {sm_mhz:.0f} MHz x {POPC_PER_CLK_SM} POPC/clk/SM "
                                       f"/ {popc_per_cw} POPC per codeword (32-bit words of the stored row)",
                         "kernel_ms_per_step": kernel_ms / args.steps, "microbench_per_clk_sm": mb},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    code.close()
    if dist:
        dist.destroy_process_group()
    return 0


def run_profile_unit(args):
    """One enumerator launch of the dominant level of the workload, at the threshold
    the full run uses there (U = d - 1 once the witness is known), run twice (the
    first is a warm-up).  Small, self-contained command for profiler captures."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1603_06757_gb300 import api

    n, k, seed, G = workload(args.workload)
    g = args.profile_unit
    with api.Code(G, n) as code:
        d = code.min_distance()["d"] if args.profile_d <= 0 else args.profile_d
        out = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            U, key, combos = code.enumerate_level(g, 0, U=d - 1)
            torch.cuda.synchronize()
            out.append(time.perf_counter() - t0)
    print(json.dumps({"workload": args.workload, "g": g, "j": 0, "U": d - 1, "combos": combos[0],
                      "seconds": out, "codewords_per_s": combos[0] / out[-1]}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="192x64")
    ap.add_argument("--cpu-levels", type=int, default=8)
    ap.add_argument("--ref-levels", type=int, default=7)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-unit", type=int, default=0, help="run one unit of this level (profiling)")
    ap.add_argument("--profile-d", type=int, default=0, help="d of the workload if known (skips the full run)")
    args = ap.parse_args()
    if args.profile_unit:
        return run_profile_unit(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Benchmark: codewords enumerated per second by the Brouwer-Zimmerman minimum-distance
run of one random binary [192,64] code (three full-rank information sets) on GB300.

One step = one whole Alg. 1 run over the prepared code (every (g, j) unit from g = 1
until L >= U) with d, the witness key and the counters exact.  `value` is timed with
CUDA events on the launching stream (inputs resident on the device); `e2e` is the same
run through the C-ABI from host buffers (prepare = information sets + host-to-device
copy, run, result read back) timed on the host clock.  `roofline` is the dominant
kernel's (the tcgen05 enumerator's flops against the measured bf16 tensor peak x 2);
`alu_path` is the same run on the ALU enumerator alone (`tensor_cores=1`) against the
integer/POPC roofline.  `--impl reference` times the CPU oracle on a bounded sample of
the same run.

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

import numpy as np

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
    "96x64": "single random [96,64] code, seed 1 (n < 2k: disjoint sets of ranks 64, 32; see --overlap-sets)",
    "112x64": "single random [112,64] code, seed 1 (n < 2k: disjoint sets of ranks 64, 48; see --overlap-sets)",
}
# POPC retired per SM per clock on compute capability 7.0-10.x (CUDA C++ Programming
# Guide, arithmetic-instruction throughput table: "population count" 16)
POPC_PER_CLK_SM = 16
# integer ALU pipe (LOP3 / IADD3 / IMNMX / ISETP): 64 lanes per SM per clock (2 warp
# instructions); the LOP3 probe reaches ~112 because LOP3 also issues to the FMA pipe
ALU_PER_CLK_SM = 64
L2_FLUSH_BYTES = 256 << 20
# dense fp8 / bf16 tensor throughput, nominal (2.25 and 4.5 PFLOP/s per GB300)
FP8_PER_BF16 = 2.0
# DRAM bytes (read + write) per launch of the dominant kernel (the tensor-core
# enumerator), from the one-launch ncu captures of levels 1-11 (set 0) summarised in
# profiles/: a timed step runs each level once per set, 33 launches, so the mean of the
# eleven; None until captured for the current kernel and plan
_TRAFFIC_192x64_MB = (0.23, 0.31, 0.60, 1.43, 3.97, 10.86, 27.51, 74.36, 204.35, 578.59, 1520.36)  # levels 1..11
TRAFFIC_PER_LAUNCH = {"192x64": int(sum(_TRAFFIC_192x64_MB) / len(_TRAFFIC_192x64_MB) * 1e6)}  # gram_kernel<4>


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


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """Largest x over the ranks of the process group (x itself without one)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world: int, units_per_rank: float, max_seconds: float) -> float:
    """Whole-job throughput of N replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / max_seconds


def workload(name, ranks_by="library"):
    """(n, k, seed, G) of a single-code workload.  The seed rule needs information-set
    ranks: the library's host partition on the GPU arm, the oracle's own partition on
    the oracle arm (which then loads nothing of the package).  Both follow the same
    reading and agree set for set (tested)."""
    import synth.configs as cfg

    if ranks_by == "oracle":
        import oracle

        return cfg.single_code(name, lambda G, n, k: [int(r) for r in oracle.partition(G, n)["ranks"]])
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
    n, k, seed, G = workload(args.workload, ranks_by="oracle")
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
    code = api.Code(G, n, tensor_cores=args.tensor_cores, overlap_sets=args.overlap_sets)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    sharded = args.shard and world > 1
    if sharded:
        from paper_1603_06757_gb300 import parallel

        exchange = parallel.TorchExchange(dist, "cuda")

    def step():
        code.reset()
        if sharded:  # this rank's slice of every unit, combined over the ranks by NCCL
            code.run_sharded(rank, world, exchange)
        else:
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
    tc_ms = 0.0
    tc_launches = 0
    tc_combos = 0
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
        tc_ms += res["tc_ms"]
        tc_launches += res["tc_launches"]
        tc_combos += res["tc_combos"]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    total_ms_max = max_over_ranks(total_ms, dist, "cuda")
    # replicas: every rank runs the whole code; sharded: the ranks split one run (each
    # rank's counters are the combined unit counts, so one rank's total is the run's)
    value = (combos / (total_ms_max / 1e3)) if sharded else weak_value(world, combos, total_ms_max / 1e3)

    # ---- end to end through the C-ABI from host buffers ----
    e2e_steps = max(1, min(args.steps, 3))
    # one untimed call first: the caching allocator grows once per process to hold a
    # second handle's tables beside the timed handle's (a warm-up, like the steps')
    api.min_distance(G, n, tensor_cores=args.tensor_cores, overlap_sets=args.overlap_sets)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_cw = 0
    h2d = d2h = 0
    for _ in range(e2e_steps):
        r = api.min_distance(G, n, tensor_cores=args.tensor_cores, overlap_sets=args.overlap_sets)
        e2e_cw += r["total_combos"]
        h2d, d2h = r["h2d_bytes"], r["d2h_bytes"]
    torch.cuda.synchronize()
    e2e_sec = time.perf_counter() - t0
    e2e_value = weak_value(world, e2e_cw, max_over_ranks(e2e_sec, dist, "cuda"))

    # ---- the same runs on the ALU enumerator alone (XOR / POPC, no tensor cores) ----
    alu_steps = 2
    code_alu = api.Code(G, n, tensor_cores=1, overlap_sets=args.overlap_sets)
    code_alu.reset()
    code_alu.run()
    torch.cuda.synchronize()
    alu_path_ms, alu_path_wall, alu_path_cw = 0.0, 0.0, 0
    for _ in range(alu_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        code_alu.reset()
        code_alu.run()
        r_alu = code_alu.result()
        torch.cuda.synchronize()
        alu_path_wall += time.perf_counter() - t0
        alu_path_ms += r_alu["kernel_ms"]  # the library's CUDA events around each wave, on its stream
        alu_path_cw += r_alu["total_combos"]
    code_alu.close()
    assert r_alu["key"] == res["key"] and r_alu["d"] == res["d"]

    # ---- roofline of the dominant kernel ----
    # The tensor-core enumerator contracts n_bits sign columns per codeword: 2 n_bits
    # flops (fp8 operands) per codeword, timed per launch by the library's CUDA events on
    # the launching stream.  Peak: the measured bf16 tensor throughput x the nominal
    # fp8 / bf16 ratio.  The ALU enumerator (the small product blocks and levels) is
    # reported beside it against its own pipe roofline.
    info = api.device_info()
    peaks = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz") or info["max_sm_clock_khz"] / 1e3)
    part = api.partition_host(G, n)
    full = args.overlap_sets > 0 or all(int(r) == k for r in part["ranks"])
    n_bits = (n - k) if full else n
    nwords = max(1, math.ceil(n_bits / 32))
    try:
        mb = {w: api.microbench(w)["per_clock_per_sm"]
              for w in ("popc", "lop3", "step4", "step4_or2", "step4_or4", "mma")}
    except Exception:  # noqa: BLE001
        mb = None
    per_clk = min(POPC_PER_CLK_SM / 1.0, ALU_PER_CLK_SM / nwords)
    alu_peak = info["sm_count"] * sm_mhz * 1e6 * per_clk
    alu_ms = kernel_ms - tc_ms
    if combos > tc_combos:
        alu_achieved = (combos - tc_combos) / (alu_ms / 1e3) if alu_ms > 0 else None
        alu_part = {"bound": "alu", "achieved": alu_achieved / 1e9 if alu_achieved else None, "peak": alu_peak / 1e9,
                    "unit": "Gcodewords/s", "frac": alu_achieved / alu_peak if alu_achieved else None,
                    "ms_per_step": alu_ms / args.steps, "codewords_per_step": (combos - tc_combos) // args.steps,
                    "peak_basis": f"{info['sm_count']} SMs x {sm_mhz:.0f} MHz x min({POPC_PER_CLK_SM} POPC, "
                                  f"{ALU_PER_CLK_SM} ALU / {nwords} words) per clk per SM"}
    else:  # the default plan put every codeword of this code on the tensor cores
        alu_part = {"codewords_per_step": 0, "other_ms_per_step": alu_ms / args.steps,
                    "note": "no codeword on the ALU enumerator in this plan (its own line: alu_path); "
                            "other_ms_per_step = unit event time outside the tensor-core launches"}
    alu_only = alu_path_cw / (alu_path_ms / 1e3)
    alu_path = {"value": alu_only, "unit": UNIT, "ms_per_step": alu_path_ms / alu_steps, "steps": alu_steps,
                "wall_ms_per_step": 1e3 * alu_path_wall / alu_steps,
                "frac_of_alu_popc_roofline": alu_only / alu_peak,
                "frac_of_exact_popc_roofline": alu_only / (info["sm_count"] * sm_mhz * 1e6 * POPC_PER_CLK_SM / nwords),
                "note": "tensor_cores=1: every codeword by XOR / POPC (OR-group lower bounds first), same d, key "
                        "and counts"}
    if tc_launches:
        bf16 = peaks.get("bf16_tflops")
        bf16_s = peaks.get("bf16_tflops_sustained")
        basis = "of measured" if bf16 else "of fallback"
        peak = (bf16 or 1900.0) * FP8_PER_BF16
        achieved = 2.0 * n_bits * tc_combos / (tc_ms / 1e3) / 1e12
        mma_peak = (2.0 * mb["mma"] * info["sm_count"] * sm_mhz * 1e6 / 1e12) if mb else None
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": TRAFFIC_PER_LAUNCH.get(args.workload),
                    "kernel": f"gram_kernel<{nwords}> (tcgen05 kind::f8f6f4, E4M3 sign operands, f32 accumulators, max-reducing TMEM loads)",
                    "peak_basis": f"bf16 {bf16 or 1900.0} TFLOP/s x {FP8_PER_BF16} (nominal fp8/bf16 dense), {basis}",
                    "frac_of_sustained": achieved / (bf16_s * FP8_PER_BF16) if bf16_s else None,
                    "mma_probe_peak": mma_peak, "frac_of_mma_probe": achieved / mma_peak if mma_peak else None,
                    "flops_per_codeword": 2 * n_bits, "launches_per_step": tc_launches / args.steps,
                    "ms_per_launch": tc_ms / tc_launches, "codewords_per_launch": tc_combos / tc_launches,
                    "share_of_kernel_time": tc_ms / kernel_ms if kernel_ms > 0 else None,
                    "alu_kernel": alu_part, "microbench_per_clk_sm": mb}
    else:
        roofline = dict(alu_part, traffic=None, microbench_per_clk_sm=mb)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        cw, sec = oracle_sample(G, n, args.cpu_levels, threads)
        cpu = {"value": cw / sec, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"Alg. 1 units (g, j), g <= {args.cpu_levels}, of the same code: {cw} codewords "
                         f"in {sec:.1f} s"}

    ext = {}
    if rank == 0 and world == 1 and not args.no_extensions:
        # the other half of the metric: batched and served codes/s against plain runs
        # (outside the timed region of `value`)
        code.close()
        ext["batch"] = batch_report(args)
        ext["serve"] = serve_report(args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "fp8+u32",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n": n, "k": k, "seed": seed, "d": res["d"],
                       "g_final": res["g_final"], "ranks": res["ranks"], "codewords_per_step": res["total_combos"],
                       "launches_per_step": res["launches"], "overlap_sets": args.overlap_sets,
                       "parallelism": f"one code split over {world} ranks" if sharded else f"replicas x{world}",
                       "l2": "flushed (256 MiB write) before every timed step; inputs ~2 KB"},
            "roofline": roofline,
            "alu_path": alu_path,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            **ext,
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
    with api.Code(G, n, tensor_cores=args.tensor_cores) as code:
        d = code.min_distance()["d"] if args.profile_d <= 0 else args.profile_d
        if args.profile_tables:  # set 0's levels below g first: its tables built level by level, as in a run
            for g2 in range(1, g):
                code.enumerate_level(g2, 0, U=0)
        out = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            U, key, combos = code.enumerate_level(g, 0, U=d - 1)
            torch.cuda.synchronize()
            out.append(time.perf_counter() - t0)
    print(json.dumps({"workload": args.workload, "g": g, "j": 0, "U": d - 1, "combos": combos[0],
                      "tensor_cores": args.tensor_cores,
                      "seconds": out, "codewords_per_s": combos[0] / out[-1]}), flush=True)
    return 0


def run_profile_batch(args):
    """The batched engine on the first N codes of the batched workload whose work estimate
    is below 10^8 codewords (all in the graph, none routed), run twice (the first is a
    warm-up).  Small, self-contained command for profiler captures of batch_enum."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    codes = batch_codes(args.profile_batch, 2024, 1000, cap=1e8)
    out = []
    for _ in range(2):
        cps, res, info = run_batched(codes)
        out.append({"codes_per_s": cps, "rounds": info["rounds"], "gpu_ms": info["gpu_ms"]})
    print(json.dumps({"codes": len(codes), "codewords": sum(r["total_combos"] for r in res), "runs": out}),
          flush=True)
    return 0


# ----------------------------------------------------------------------------------
# batched codes and the predictor (config: 4096 random codes, k in [24, 56], n in [2k, 3k])
# ----------------------------------------------------------------------------------

def gv_work(n, k, ranks):
    """Codewords up to the level at which the bound reaches the Gilbert-Varshamov
    estimate of d (the library's routing estimate without a hint)."""
    from paper_1603_06757_gb300 import predict

    _, w = predict.gv_estimate(n, k, ranks)
    return sum(len(ranks) * math.comb(k, g) for g in range(1, w + 1))


def batch_codes(count, seed, seed_base, cap=None, k_lo=24, k_hi=56, nmul_hi=3):
    """Codes of the batched workload (all of them, or those whose Gilbert-Varshamov work
    estimate is <= cap): list of (n, k, G, ranks)."""
    import synth
    from paper_1603_06757_gb300 import api, predict

    out = []
    for s in synth.batch_specs(count, k_lo, k_hi, 2, nmul_hi, seed=seed, seed_base=seed_base):
        G = synth.random_systematic(s.n, s.k, s.seed)
        ranks = [int(r) for r in api.partition_host(G, s.n)["ranks"]]
        if cap is None or gv_work(s.n, s.k, ranks) <= cap:
            out.append((s.n, s.k, G, ranks))
    return out


def run_plain(codes, hints=None):
    """One code after the other through mdist_prepare + mdist_min_distance."""
    import torch

    from paper_1603_06757_gb300 import api

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = []
    for i, (n, k, G, _) in enumerate(codes):
        with api.Code(G, n, wstar_hint=hints[i] if hints else 0) as c:
            res.append(c.min_distance())
    torch.cuda.synchronize()
    return len(codes) / (time.perf_counter() - t0), res


def run_batched(codes, hints=None, blocks_per_sm=0, rounds_per_graph=0, tensor_cores=0, route_work_log10=0):
    """All codes in one batched run (rounds captured in one CUDA graph; large codes on
    the single-code tensor-core path unless tensor_cores=1)."""
    import torch

    from paper_1603_06757_gb300 import api

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with api.Batch(blocks_per_sm=blocks_per_sm, tensor_cores=tensor_cores, route_work_log10=route_work_log10) as b:
        for i, (n, k, G, _) in enumerate(codes):
            b.add(G, n, wstar_hint=hints[i] if hints else 0)
        b.run(rounds_per_graph)
        res = [b.result(i) for i in range(len(codes))]
        info = b.info()
    torch.cuda.synchronize()
    return len(codes) / (time.perf_counter() - t0), res, info


def train_predictor(train_codes, steps=3000):
    """MLP on features -> (d / n, w* / k), labels from the batched engine's own runs."""
    from paper_1603_06757_gb300 import predict

    _, res, _ = run_batched(train_codes)
    codes = [(G, n) for (n, k, G, _) in train_codes]
    labels = [(r["d"], r["g_final"], r["ranks"]) for r in res]
    mlp, curve = predict.train_predictor(codes, labels, steps=steps)
    return mlp, curve


def predictor_report(mlp, test_codes, test_res):
    from paper_1603_06757_gb300 import predict

    shapes = [(n, k, ranks) for (n, k, G, ranks) in test_codes]
    feats = np.stack([predict.features(G, n) for (n, k, G, _) in test_codes])
    truth = [(r["g_final"], r["d"]) for r in test_res]
    p_mlp = predict.Predictor(mlp).predict(feats, shapes)
    p_gv = predict.Predictor(None).predict(feats, shapes)
    return p_mlp, p_gv, {"mlp": predict.errors(p_mlp, truth), "gv": predict.errors(p_gv, truth)}


def _same_results(a_list, b_list):
    return all(a["d"] == b["d"] and a["key"] == b["key"] and a["message"] == b["message"] and
               np.array_equal(a["counts"], b["counts"]) for a, b in zip(a_list, b_list))


def batch_report(args, full=False):
    """Batched vs plain codes/s on the 4096-code workload (every code: the light ones in
    the batched graph, the large ones on the single-code tensor-core path), with the
    predictor's hints (MLP, Gilbert-Varshamov, none) deciding the first round's levels and
    the routing.  full: also the launch-shape autotuner and hinted plain runs."""
    from paper_1603_06757_gb300 import predict

    codes = batch_codes(args.batch_codes, 2024, 1000)
    train = batch_codes(args.batch_train, 77, 500000, cap=args.batch_cap)
    t0 = time.perf_counter()
    mlp, curve = train_predictor(train)
    train_s = time.perf_counter() - t0
    shapes = [(n, k, ranks) for (n, k, G, ranks) in codes]
    feats = np.stack([predict.features(G, n) for (n, k, G, _) in codes])
    p_mlp = predict.Predictor(mlp).predict(feats, shapes)
    p_gv = predict.Predictor(None).predict(feats, shapes)
    hints = {"mlp": [w for (w, d) in p_mlp], "gv": [w for (w, d) in p_gv], "none": None}
    run_batched(codes[:64])  # warm-up of both paths
    run_plain(codes[:16])
    cps, res, info = {}, {}, {}
    for name, h in hints.items():
        cps[name], res[name], info[name] = run_batched(codes, h, route_work_log10=args.route_work_log10)
    cps_plain, res_plain = run_plain(codes)
    same = all(_same_results(res[name], res_plain) for name in hints)
    truth = [(r["g_final"], r["d"]) for r in res_plain]
    errs = {"mlp": predict.errors(p_mlp, truth), "gv": predict.errors(p_gv, truth)}
    # the light codes alone (those the default routing keeps in the graph)
    light = [c for c in codes if gv_work(c[0], c[1], c[3]) < 10.0 ** args.route_work_log10]
    cps_light_b, res_lb, _ = run_batched(light, route_work_log10=args.route_work_log10)
    cps_light_p, res_lp = run_plain(light)
    best = max(cps, key=cps.get)
    out = {
        "metric": "codes/s, batched vs plain (one code per prepare/run)", "unit": "codes/s",
        "value": cps[best], "best": f"batched, {best} hints", "higher_is_better": True,
        "config": {"workload": f"{len(codes)} random codes, k ~ U[24,56], n ~ U[2k,3k], R iid Bernoulli(1/2), "
                               "seeds 1000+i (every code)",
                   "codewords": sum(r["total_combos"] for r in res_plain),
                   "large_codes": info["none"]["large_codes"],
                   "route_work_log10": args.route_work_log10,
                   "route_basis": "codes estimated at >= 10^route_work_log10 codewords run on the single-code "
                                  "tensor-core path; 10 = tune.py's choice on a 256-code sample of this workload",
                   "train_codes": len(train)},
        "codes_per_s": {"plain": cps_plain, **{f"batched_{k}_hints": v for k, v in cps.items()}},
        "speedup_vs_plain": cps[best] / cps_plain,
        "light_codes": {"codes": len(light), "batched": cps_light_b, "plain": cps_light_p,
                        "speedup": cps_light_b / cps_light_p, "results_identical": _same_results(res_lb, res_lp)},
        "rounds": {k: v["rounds"] for k, v in info.items()},
        "large_codes": {k: v["large_codes"] for k, v in info.items()},
        "gpu_ms": {k: v["gpu_ms"] + v["large_ms"] for k, v in info.items()},
        "predictor": errs, "predictor_train_s": train_s, "train_loss_last": float(curve[-50:].mean()),
        "results_identical": bool(same),
    }
    if full:
        from paper_1603_06757_gb300 import tune

        best_hints = hints[best] or [0] * len(codes)
        tuned = tune.autotune_batch([(G, n, hh) for (n, k, G, _), hh in zip(codes, best_hints)],
                                    sample=args.tune_sample)
        shape = {"blocks_per_sm": tuned["blocks_per_sm"], "route_work_log10": tuned["route_work_log10"]}
        out["autotune"] = {"chosen": shape, "sample": tuned["sample"], "seconds_best": tuned["seconds_best"],
                           "seconds_worst": tuned["seconds_worst"], "candidates": len(tuned["table"]),
                           "codes_per_s_tuned": run_batched(codes, hints[best], **shape)[0]}
        out["codes_per_s"]["plain_mlp_hints"] = run_plain(codes, hints["mlp"])[0]
        out["codes_per_s"]["plain_gv_hints"] = run_plain(codes, hints["gv"])[0]
        out["codes_per_s"]["batched_no_routing"] = run_batched(codes, hints[best], tensor_cores=1)[0]
    return out


def run_batch_bench(args):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    line = batch_report(args, full=True)
    line.update({"n_gpus": 1, "data": "synthetic"})
    print(json.dumps(line), flush=True)
    return 0


def serve_requests(count, seed, cap):
    """Request stream: k ~ U[20,64], n ~ U[2k,4k]; a draw whose GV work estimate exceeds
    cap is redrawn from the same stream (rejection sampling)."""
    import synth
    from paper_1603_06757_gb300 import api, predict

    rng = synth.SplitMix64(seed)
    out, rejected = [], 0
    while len(out) < count:
        k = rng.uniform_int(20, 64)
        n = rng.uniform_int(2 * k, 4 * k)
        cs = rng.next()
        G = synth.random_systematic(n, k, cs)
        ranks = [int(r) for r in api.partition_host(G, n, max_sets=8)["ranks"]]
        _, w = predict.gv_estimate(n, k, ranks)
        if sum(len(ranks) * math.comb(k, g) for g in range(1, w + 1)) > cap:
            rejected += 1
            continue
        out.append((n, k, G, ranks))
    return out, rejected


def serve_report(args):
    """Served capacity vs plain per-code launches on the same seeded sample of the request
    stream, then the latency of the whole Poisson stream at a fraction of that capacity."""
    import threading as th

    import synth
    from paper_1603_06757_gb300 import api, predict, tune

    reqs, rejected = serve_requests(args.serve_requests, 4242, args.serve_cap)
    train = batch_codes(args.batch_train, 77, 500000, args.batch_cap, k_lo=20, k_hi=64, nmul_hi=4)
    mlp, _ = train_predictor(train)
    shapes = [(n, k, ranks) for (n, k, G, ranks) in reqs]
    feats = np.stack([predict.features(G, n) for (n, k, G, _) in reqs])
    if args.serve_hints == "mlp":
        hints = [w for (w, d) in predict.Predictor(mlp).predict(feats, shapes)]
    elif args.serve_hints == "gv":
        hints = [w for (w, d) in predict.Predictor(None).predict(feats, shapes)]
    else:
        hints = [0] * len(reqs)
    idx = tune.sample_indices(len(reqs), min(len(reqs), args.serve_capacity_sample), 5)
    sample = [reqs[i] for i in idx]
    run_plain(sample[:16])  # warm-up
    cps_plain, res_plain = run_plain(sample)
    with api.Server(max_slots=args.serve_slots, rows_pool_bytes=64 << 20) as srv:
        t0 = time.perf_counter()
        ids = [srv.submit(reqs[i][2], reqs[i][0], wstar_hint=hints[i]) for i in idx]
        got = {}
        while len(got) < len(ids):
            for rid in ids:
                if rid not in got:
                    r = srv.poll(rid, wait_ms=0)
                    if r is not None:
                        got[rid] = r
            time.sleep(0.001)
        cps_served = len(ids) / (time.perf_counter() - t0)
    same = _same_results([got[rid] for rid in ids], res_plain)
    rate = args.serve_rate if args.serve_rate > 0 else args.serve_load * cps_served
    arrivals = synth.poisson_arrivals(len(reqs), rate, seed=99)
    with api.Server(max_slots=args.serve_slots, rows_pool_bytes=64 << 20) as srv:
        ids = [None] * len(reqs)
        t0 = time.perf_counter()

        def feeder():
            for i, (n, k, G, _) in enumerate(reqs):
                dt = arrivals[i] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                ids[i] = srv.submit(G, n, wstar_hint=hints[i])

        f = th.Thread(target=feeder)
        f.start()
        lat = {}
        while len(lat) < len(reqs):
            for i in range(len(reqs)):
                if i not in lat and ids[i] is not None:
                    r = srv.poll(ids[i], wait_ms=0)
                    if r is not None:
                        lat[i] = r["latency_s"]
            time.sleep(0.002)
        f.join()
        wall = time.perf_counter() - t0
        info = srv.info()
    lats = np.array([lat[i] for i in range(len(reqs))])
    return {
        "metric": "served codes/s and latency vs plain per-code launches", "unit": "codes/s",
        "value": cps_served, "higher_is_better": True,
        "config": {"workload": f"Poisson stream of {len(reqs)} requests, k ~ U[20,64], n ~ U[2k,4k], R iid "
                               f"Bernoulli(1/2); draws with GV work estimate > {args.serve_cap:.0e} codewords "
                               f"redrawn ({rejected} redrawn)",
                   "capacity_sample": len(idx), "arrival_rate_per_s": rate,
                   "load": f"{args.serve_load} x served capacity", "slots": args.serve_slots,
                   "hints": args.serve_hints},
        "codes_per_s": {"served": cps_served, "plain": cps_plain, "served_at_load": len(reqs) / wall},
        "speedup_vs_plain": cps_served / cps_plain,
        "latency_s": {"p50": float(np.percentile(lats, 50)), "p99": float(np.percentile(lats, 99)),
                      "mean": float(lats.mean()), "max": float(lats.max())},
        "rounds": info["rounds"], "gpu_ms": info["gpu_ms"],
        "results_identical": bool(same),
    }


def run_serve_bench(args):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    line = serve_report(args)
    line.update({"n_gpus": 1, "data": "synthetic"})
    print(json.dumps(line), flush=True)
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
    ap.add_argument("--overlap-sets", type=int, default=0,
                    help="M > 0: M overlapping information sets (the non-disjoint bound) instead of disjoint ones")
    ap.add_argument("--shard", action="store_true",
                    help="N > 1: split one code's units over the ranks (strong scaling) instead of N replicas")
    ap.add_argument("--no-extensions", action="store_true",
                    help="leave out the batched and served measurements of the default line")
    ap.add_argument("--mode", choices=["single", "batch", "serve"], default="single")
    ap.add_argument("--batch-codes", type=int, default=4096)
    ap.add_argument("--batch-train", type=int, default=1500)
    ap.add_argument("--batch-cap", type=float, default=1e10)
    ap.add_argument("--route-work-log10", type=int, default=10,
                    help="batched engine: routing threshold of the tensor-core path (10^x codewords)")
    ap.add_argument("--tune-sample", type=int, default=256, help="codes the batched launch-shape autotuner times")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--serve-cap", type=float, default=1e11)
    ap.add_argument("--serve-load", type=float, default=0.7)
    ap.add_argument("--serve-slots", type=int, default=1024)
    ap.add_argument("--serve-plain-sample", type=int, default=500)
    ap.add_argument("--serve-capacity-sample", type=int, default=4000)
    ap.add_argument("--serve-hints", choices=["mlp", "gv", "none"], default="mlp")
    ap.add_argument("--serve-rate", type=float, default=0.0, help="arrivals/s (0: load x served capacity)")
    ap.add_argument("--tensor-cores", type=int, choices=[0, 1, 2, 3], default=0,
                    help="0: large product blocks on the tcgen05 enumerator, 1: ALU enumerator only, 2: all blocks, "
                         "3: as 0, every block with a small side split whatever its size")
    ap.add_argument("--profile-unit", type=int, default=0, help="run one unit of this level (profiling)")
    ap.add_argument("--profile-tables", action="store_true",
                    help="with --profile-unit: run set 0's lower levels first (tables built level by level)")
    ap.add_argument("--profile-d", type=int, default=0, help="d of the workload if known (skips the full run)")
    ap.add_argument("--profile-batch", type=int, default=0, help="run the batched engine on this many light codes")
    args = ap.parse_args()
    if args.profile_unit:
        return run_profile_unit(args)
    if args.profile_batch:
        return run_profile_batch(args)
    if args.mode == "batch":
        return run_batch_bench(args)
    if args.mode == "serve":
        return run_serve_bench(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

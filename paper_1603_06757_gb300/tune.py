"""Autotuner of the batched engine's shapes.

Two choices decide how the batched engine (mdist_batch_*) spends the GPU: the CTAs per
SM of the persistent per-bucket ALU enumerator (its grid: 0 = as many as fit) and the
split of the codes between the batched graph and the single-code tensor-core path (a
code whose estimated work reaches 10^route_work_log10 codewords takes the tensor-core
path).  `autotune_batch` times every candidate pair on a seeded sample of the workload
(wall time of a whole batched run of the sample, after one warm-up run) and returns the
fastest.  Results never depend on the choice, only the speed does.
"""

from __future__ import annotations

import time

import numpy as np

DEFAULT_BLOCKS_PER_SM = (0, 1, 2, 3)
DEFAULT_ROUTE_WORK_LOG10 = (7, 8, 9, 10)


def sample_indices(count: int, size: int, seed: int) -> list[int]:
    """`size` distinct indices of range(count), drawn by SplitMix64(seed), sorted."""
    import synth

    if size >= count:
        return list(range(count))
    rng = synth.SplitMix64(seed)
    pool = list(range(count))
    for i in range(size):  # partial Fisher-Yates
        j = i + rng.uniform_int(0, count - i - 1)
        pool[i], pool[j] = pool[j], pool[i]
    return sorted(pool[:size])


def _run_batch(sample, blocks_per_sm: int, route_work_log10: int) -> float:
    from . import api

    t0 = time.perf_counter()
    with api.Batch(blocks_per_sm=blocks_per_sm, route_work_log10=route_work_log10) as b:
        for G, n, hint in sample:
            b.add(G, n, wstar_hint=hint)
        b.run()
    return time.perf_counter() - t0


def autotune_batch(codes, *, sample: int = 256, seed: int = 1, blocks_per_sm=DEFAULT_BLOCKS_PER_SM,
                   route_work_log10=DEFAULT_ROUTE_WORK_LOG10, repeats: int = 1, runner=None) -> dict:
    """Pick (blocks_per_sm, route_work_log10) for a batch of `codes` = [(G, n)] or
    [(G, n, wstar_hint)].  `runner(sample, blocks_per_sm, route_work_log10) -> seconds`
    replaces the timed batched run (tests)."""
    run = runner or _run_batch
    norm = [(c[0], c[1], c[2] if len(c) > 2 else 0) for c in codes]
    if not norm:
        raise ValueError("autotune_batch needs at least one code")
    picked = [norm[i] for i in sample_indices(len(norm), sample, seed)]
    run(picked, blocks_per_sm[0], route_work_log10[0])  # warm-up: builds, first graph
    table = []
    for bps in blocks_per_sm:
        for rw in route_work_log10:
            secs = min(run(picked, bps, rw) for _ in range(max(1, repeats)))
            table.append({"blocks_per_sm": int(bps), "route_work_log10": int(rw), "seconds": float(secs)})
    best = min(table, key=lambda r: r["seconds"])
    secs = np.array([r["seconds"] for r in table])
    return {"blocks_per_sm": best["blocks_per_sm"], "route_work_log10": best["route_work_log10"],
            "sample": len(picked), "seconds_best": best["seconds"], "seconds_worst": float(secs.max()),
            "table": table}


__all__ = ["autotune_batch", "sample_indices", "DEFAULT_BLOCKS_PER_SM", "DEFAULT_ROUTE_WORK_LOG10"]

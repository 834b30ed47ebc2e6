"""Multi-rank paths with gloo ranks on the CPU: bench.py's aggregation of N replicas
(barrier, max over ranks, whole-job value), and one code split over ranks — every unit's
combinations cut into contiguous slices, one per rank, combined by the exchange the
library's sharded run calls (least key, summed count) — giving the oracle's run."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_seconds = 1.0 + rank  # rank 1 is the slow one
    dist.barrier()
    m = bench.max_over_ranks(local_seconds, dist, "cpu")
    v = bench.weak_value(world, 1000.0, m)
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in out:
        assert m == pytest.approx(2.0)          # the slowest rank's time
        assert v == pytest.approx(2 * 1000 / 2.0)  # all ranks' units / that time


def test_single_process_defaults():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.weak_value(1, 10.0, 2.0) == 5.0


# ---- one code split over ranks: the exchange and the combination of unit slices ----

def _slice_unit(gamma_bits, k, g, thr, lo, hi):
    """Least device key (weight << 54 | lexicographic rank) among the weight-<= thr
    codewords of combinations lo..hi-1 (lexicographic order) of unit g, and their count."""
    import itertools

    best, count = (1 << 64) - 1, 0
    for rank, comb in enumerate(itertools.combinations(range(k), g)):
        if rank < lo:
            continue
        if rank >= hi:
            break
        w = int(np.bitwise_xor.reduce(gamma_bits[list(comb)], axis=0).sum())
        count += 1
        if w <= thr:
            best = min(best, (w << 54) | rank)
    return best, count


def _fold(n, k, ranks, gam_bits, exchange, part, nparts):
    """Alg. 1, level check, over units whose slices are combined by `exchange` (a plain
    restatement of the single-code driver's fold for this test)."""
    import math

    m = len(ranks)
    U, L, key = n - k + 1, 1, None
    counts = {}
    g = 1
    while g <= k and L < U:
        for j in range(m):
            thr = key[0] - 1 if key else U
            total = math.comb(k, g)
            lo, hi = total * part // nparts, total * (part + 1) // nparts
            kv, cnt = exchange(*_slice_unit(gam_bits[j], k, g, thr, lo, hi))
            counts[(g, j)] = cnt
            if kv != (1 << 64) - 1:
                w = kv >> 54
                if key is None or w < key[0]:
                    key = (w, g, j, kv & ((1 << 54) - 1))
                U = min(U, w)
        L = sum(max(0, g + 1 - (k - r)) for r in ranks)
        if L >= U:
            break
        g += 1
    return U, key, counts


def _sharded_rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    from paper_1603_06757_gb300 import parallel

    ex = parallel.TorchExchange(dist, "cpu")
    # the exchange itself: least key (no key = 2^64-1 from every rank but one), summed count
    keys = [(1 << 64) - 1, (7 << 54) | 5, (9 << 54) | 1]
    got = ex(keys[rank], 10 + rank)
    out = {"exchange": got}
    results = []
    for n, k, seed in [(30, 10, 1), (36, 12, 2), (28, 14, 3)]:
        G = synth.random_systematic(n, k, seed)
        p = oracle.partition(G, n)
        gam_bits = [synth.unpack_bits(p["gammas"][j], n).astype(np.uint8) for j in range(p["m"])]
        U, key, counts = _fold(n, k, [int(r) for r in p["ranks"]], gam_bits, ex, rank, world)
        results.append((U, key, sorted(counts.items())))
    out["runs"] = results
    q.put((rank, out))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_units_split_over_gloo_ranks(world):
    """world gloo ranks each take a contiguous slice of every unit; combined by
    TorchExchange (min key, summed count), every rank folds the same run, equal to the
    oracle's (d, key, per-unit counts)."""
    import oracle
    import synth

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    outs = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    keys = [(1 << 64) - 1, (7 << 54) | 5, (9 << 54) | 1][:world]
    for r in range(world):
        assert outs[r]["exchange"] == (min(keys), sum(10 + i for i in range(world)))
        assert outs[r]["runs"] == outs[0]["runs"]
    for (n, k, seed), (U, key, counts) in zip([(30, 10, 1), (36, 12, 2), (28, 14, 3)], outs[0]["runs"]):
        want = oracle.min_distance(synth.random_systematic(n, k, seed), n)
        assert U == want["d"] and key == want["key"]
        for (g, j), c in counts:
            assert c == int(want["counts"][g][j])


def test_thread_exchange():
    import threading

    from paper_1603_06757_gb300 import parallel

    ex = parallel.ThreadExchange(3, timeout_s=30)
    got = [None] * 3
    keys = [(5 << 54) | 9, (1 << 64) - 1, (5 << 54) | 2]

    def run(r):
        got[r] = [ex.for_rank(r)(keys[r], r + 1) for _ in range(2)]  # two units in a row

    ts = [threading.Thread(target=run, args=(r,)) for r in range(3)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert all(g == [((5 << 54) | 2, 6)] * 2 for g in got)


def test_thread_exchange_lost_rank_times_out():
    import threading

    from paper_1603_06757_gb300 import parallel

    ex = parallel.ThreadExchange(2, timeout_s=0.5)
    errs = []

    def run():
        try:
            ex.for_rank(0)(1, 1)  # rank 1 never arrives
        except threading.BrokenBarrierError as e:
            errs.append(e)

    t = threading.Thread(target=run)
    t.start()
    t.join(timeout=10)
    assert errs

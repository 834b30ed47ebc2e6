"""One code's Alg. 1 run split over several ranks: every (g, j) unit's work is cut into
`nparts` contiguous slices, rank r enumerates slice r on its own GPU (or its own handle
of one GPU), and the library calls back after each unit to combine the slices — the
least 64-bit device key (weight << 54 | lexicographic rank: the least weight, then the
least rank) and the summed combination count — before folding the unit exactly as the
single-code driver does (mdist_run_sharded; paper §2, Alg. 1).  Every rank ends with the
same result, equal to mdist_min_distance's.

This module only supplies the exchange on the host: `TorchExchange` (torch.distributed:
NCCL between GPUs, gloo on CPUs) or `ThreadExchange` (host threads of one process meeting
at a barrier).  No kernel ever waits for another rank.
"""

from __future__ import annotations

import threading

NO_KEY = (1 << 64) - 1
_INT64_MAX = (1 << 63) - 1


class TorchExchange:
    """exchange(key, count) over an initialised torch.distributed group: one MIN and one
    SUM all-reduce of an int64.  Device keys are below 2^63 (weight <= 512 < 2^9 above 54
    rank bits), so "no key" travels as the largest int64."""

    def __init__(self, dist, device="cpu"):
        import torch

        self.dist, self.torch, self.device = dist, torch, device

    def __call__(self, key: int, count: int):
        t = self.torch.tensor([_INT64_MAX if key == NO_KEY else key, count], dtype=self.torch.int64,
                              device=self.device)
        k = t[:1].clone()
        c = t[1:].clone()
        self.dist.all_reduce(k, op=self.dist.ReduceOp.MIN)
        self.dist.all_reduce(c, op=self.dist.ReduceOp.SUM)
        kv = int(k.item())
        return (NO_KEY if kv == _INT64_MAX else kv), int(c.item())


class ThreadExchange:
    """The exchange of `nranks` host threads of one process: each call deposits this
    rank's (key, count), waits at a barrier (timeout_s: a rank that never arrives breaks
    it, and the run stops with MDIST_ECANCELLED) and returns the combination."""

    def __init__(self, nranks: int, timeout_s: float = 60.0):
        self.n = int(nranks)
        self.timeout = timeout_s
        self.barrier = threading.Barrier(self.n)
        self.slots = [None] * self.n
        self.lock = threading.Lock()

    def for_rank(self, rank: int):
        def exchange(key: int, count: int):
            self.slots[rank] = (key, count)
            self.barrier.wait(self.timeout)          # every rank has deposited
            with self.lock:
                best = min(k for k, _ in self.slots)
                total = sum(c for _, c in self.slots)
            self.barrier.wait(self.timeout)          # every rank has read before the next unit
            return best, total

        return exchange


def sharded_min_distance(G, n: int, part: int, nparts: int, exchange, **code_kw) -> dict:
    """mdist_min_distance of G with this rank running slice `part` of `nparts` of every
    unit (its own GPU, or its own handle); exchange(key, count) combines a unit's slices.
    Every rank gets the whole result."""
    from . import api

    with api.Code(G, n, **code_kw) as code:
        code.run_sharded(part, nparts, exchange)
        return code.result()


def sharded_min_distance_threads(G, n: int, nparts: int, **code_kw) -> list[dict]:
    """The same with `nparts` host threads of this process, each driving its own handle on
    the current GPU (one GPU standing in for several, for tests): the list of the ranks'
    results."""
    ex = ThreadExchange(nparts)
    out = [None] * nparts
    errs = []

    def rank(r):
        try:
            out[r] = sharded_min_distance(G, n, r, nparts, ex.for_rank(r), **code_kw)
        except Exception as e:  # noqa: BLE001
            errs.append(e)
            ex.barrier.abort()

    import torch

    dev = torch.cuda.current_device()

    def start(r):
        torch.cuda.set_device(dev)
        rank(r)

    ths = [threading.Thread(target=start, args=(r,)) for r in range(nparts)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    if errs:
        raise errs[0]
    return out

"""Write the oracle's result for every light code of the batched workload to
``tests/golden/oracle_batch_4096.txt``.

The batched workload is 4096 random codes, k uniform in [24, 56], n uniform in
[2k, 3k], G = [I_k | R] with R drawn from the SplitMix64 stream at each code's seed
(``synth.batch_specs(4096, 24, 56, 2, 3, seed=2024, seed_base=1000)``). A code is light
when its Gilbert-Varshamov work estimate is at most the cap: 10^9 codewords by default
(2914 codes, 71 %, about 2.7·10^11 estimated codewords), 10^10 with ``--cap 1e10``
(3362 codes, 82 %, seven times the work). The estimate is d_GV, the least w with sum_{i<=w} C(n, i) >= 2^(n-k); then
w*, the least level g whose bound L(g) = sum_j max(0, g+1-(k-r_j)) reaches d_GV; then
sum_{g<=w*} m C(k, g). The heavier codes are beyond the oracle's time budget; the GPU
test checks them against the single-code runs.

Only ``oracle/`` computes here (``synth`` draws the specs and matrices and nothing
else). Every stored value comes from the oracle's ``min_distance`` output (Alg. 1,
level check): d, the witness key (weight, g, j, lexicographic rank), message, witness,
last unit and final bound. The codes run in a pool of single-threaded processes.

``--sample N`` writes instead ``oracle_batch_4096_sample.txt``: a seeded sample of N of
the heavier codes, those with an estimate above the cap and at most ten times it.

Usage:  python tests/golden/make_batch_goldens.py [--procs P] [--cap C] [--limit N] [--sample N]
"""

from __future__ import annotations

import argparse
import math
import multiprocessing as mp
import os
import platform
import random
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

COUNT, K_LO, K_HI, NMUL_LO, NMUL_HI, SEED, SEED_BASE = 4096, 24, 56, 2, 3, 2024, 1000
CAP = 10**9


def gv_work(n: int, k: int, ranks) -> int:
    """The Gilbert-Varshamov work estimate of the module docstring."""
    d_gv, acc = 0, 0
    while acc < 2 ** (n - k):
        acc += math.comb(n, d_gv)
        d_gv += 1
    d_gv -= 1  # the least w with sum_{i<=w} C(n, i) >= 2^(n-k)
    g = 0
    while g < k and sum(max(0, g + 1 - (k - r)) for r in ranks) < d_gv:
        g += 1
    return sum(len(ranks) * math.comb(k, h) for h in range(1, g + 1))


def _one(args):
    i, n, k, seed = args
    G = synth.random_systematic(n, k, seed)
    r = oracle.min_distance(G, n, nthreads=1)
    wit = " ".join(format(int(x), "x") for x in r["witness"])
    w, g, j, rank = r["key"]
    return (i, f"{i} {n} {k} {seed} {r['d']} {w} {g} {j} {rank} {r['g_final']} {r['j_final']} "
               f"{r['L_final']} {r['message']:x} {wit}")


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--limit", type=int, default=0, help="only the first N light codes (a trial run)")
    ap.add_argument("--cap", type=float, default=CAP, help="largest Gilbert-Varshamov work estimate kept")
    ap.add_argument("--sample", type=int, default=0, help="a seeded sample of N codes in (cap, 10 cap] instead")
    args = ap.parse_args()
    todo = []
    for i, s in enumerate(synth.batch_specs(COUNT, K_LO, K_HI, NMUL_LO, NMUL_HI, seed=SEED, seed_base=SEED_BASE)):
        ranks = [int(x) for x in oracle.partition(synth.random_systematic(s.n, s.k, s.seed), s.n)["ranks"]]
        w = gv_work(s.n, s.k, ranks)
        if (w <= args.cap) if not args.sample else (args.cap < w <= 10 * args.cap):
            todo.append((i, s.n, s.k, s.seed))
    if args.sample:  # a seeded choice among the heavier codes, in index order
        rng = random.Random(SEED)
        todo = sorted(rng.sample(todo, min(args.sample, len(todo))))
    if args.limit:
        todo = todo[: args.limit]
    t0 = time.time()
    with mp.get_context("spawn").Pool(args.procs) as pool:
        rows = sorted(pool.imap_unordered(_one, todo, chunksize=4))
    secs = time.time() - t0
    name = ("oracle_batch_4096_sample.txt" if args.sample
            else "oracle_batch_4096.txt" if not args.limit else "oracle_batch_trial.txt")
    path = os.path.join(HERE, name)
    head = [
        "# Oracle results (Alg. 1, level check) of " + ("codes" if args.sample else "the light codes")
        + " of the batched workload:",
        f"# synth.batch_specs({COUNT}, {K_LO}, {K_HI}, {NMUL_LO}, {NMUL_HI}, seed={SEED}, seed_base={SEED_BASE}),",
        (f"# a seeded sample of {len(todo)} codes whose Gilbert-Varshamov work estimate is in"
         f" ({args.cap:.0e}, {10 * args.cap:.0e}]." if args.sample else
         f"# the {len(todo)} codes whose Gilbert-Varshamov work estimate is <= {args.cap:.0e}."),
        f"# Written by tests/golden/make_batch_goldens.py in {secs:.0f} s on {args.procs} processes"
        f" ({platform.machine()}).",
        "# columns: index n k seed d weight g j rank g_final j_final L_final message(hex) witness words(hex)",
    ]
    with open(path + ".tmp", "w") as f:
        f.write("\n".join(head + [line for _, line in rows]) + "\n")
    os.replace(path + ".tmp", path)
    print(path, len(rows), f"{secs:.0f} s", flush=True)


if __name__ == "__main__":
    main()

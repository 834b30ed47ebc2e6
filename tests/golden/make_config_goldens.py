"""Write the oracle's whole Alg. 1 run of each full-size single-code workload to
``tests/golden/oracle_run_<name>.txt``.

Only ``oracle/`` computes here (``synth`` draws the seeded matrix and nothing else): the
information sets come from the oracle's greedy partition, and every stored value — d,
the witness key (weight, g, j, lexicographic rank), message, witness, last unit, final
bounds and the number of combinations of every (g, j) unit — is the oracle's
``min_distance`` output (Alg. 1, level check).  The runs take hours of CPU time
([192,64]: 2.8·10^12 codewords, [150,64]: 5.5·10^11, [300,50]: 3.2·10^12), so the files
are committed and the GPU tests only read them.

Usage:  python tests/golden/make_config_goldens.py [--threads T] NAME [NAME ...]
        NAME in 192x64, 150x64, 300x50, 60x30
"""

from __future__ import annotations

import argparse
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth.configs import single_code  # noqa: E402


def oracle_ranks(G, n, k):
    return [int(r) for r in oracle.partition(G, n)["ranks"]]


def write_run(name: str, threads: int) -> str:
    n, k, seed, G = single_code(name, oracle_ranks)
    t0 = time.time()
    r = oracle.min_distance(G, n, nthreads=threads)
    secs = time.time() - t0
    total = int(r["counts"].sum())
    lines = [
        f"# Oracle run (Alg. 1, level check) of the {name} workload: random [n={n},k={k}] code,",
        "# G = [I_k | R], R iid Bernoulli(1/2) from the SplitMix64 stream at the seed below.",
        f"# Written by tests/golden/make_config_goldens.py: {total} codewords in {secs:.0f} s on",
        f"# {threads} threads ({platform.machine()}).",
        f"name {name}",
        f"n {n}",
        f"k {k}",
        f"seed {seed}",
        f"m {r['m']}",
        "ranks " + " ".join(str(x) for x in r["ranks"]),
        f"d {r['d']}",
        "key " + " ".join(str(x) for x in r["key"]),
        f"message {r['message']}",
        "witness " + " ".join(str(int(x)) for x in r["witness"]),
        f"g_final {r['g_final']}",
        f"j_final {r['j_final']}",
        f"L_final {r['L_final']}",
        f"U_final {r['U_final']}",
        f"codewords {total}",
    ]
    counts = r["counts"]
    for g in range(counts.shape[0]):
        if counts[g].any():
            lines.append(f"counts {g} " + " ".join(str(int(x)) for x in counts[g]))
    path = os.path.join(HERE, f"oracle_run_{name}.txt")
    with open(path + ".tmp", "w") as f:
        f.write("\n".join(lines) + "\n")
    os.replace(path + ".tmp", path)
    return path


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=oracle.default_threads())
    ap.add_argument("names", nargs="+")
    args = ap.parse_args()
    for name in args.names:
        print(write_run(name, args.threads), flush=True)


if __name__ == "__main__":
    main()

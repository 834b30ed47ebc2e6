"""The batched workload itself (4096 random codes, k in [24, 56], n in [2k, 3k]) through
one batched run with the default routing: every light code's result equals the
oracle's stored run (`tests/golden/oracle_batch_4096.txt`, written by
`make_batch_goldens.py` from `oracle/` only): d, the witness key, message, witness,
last unit and final bound, with the per-unit combination counts C(k, g) up to that
unit; so does each code of the seeded sample of heavier ones
(`oracle_batch_4096_sample.txt`, when written).  Every code, light or heavy, equals its
single-code run."""

import math
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_batch_4096.txt")
SAMPLE = os.path.join(os.path.dirname(__file__), "golden", "oracle_batch_4096_sample.txt")


@pytest.fixture(scope="module")
def api():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_1603_06757_gb300 import api as a

    return a


def _golden(path):
    rows = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            i, n, k, seed, d, w, g, j, rank, gf, jf, lf = (int(x) for x in p[:12])
            rows[i] = dict(n=n, k=k, seed=seed, d=d, key=(w, g, j, rank), g_final=gf, j_final=jf, L_final=lf,
                           message=int(p[12], 16), witness=[int(x, 16) for x in p[13:]])
    return rows


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="oracle_batch_4096.txt not written yet")
def test_batched_workload_against_oracle_and_single_runs(api):
    gold = _golden(GOLDEN)
    light = len(gold)
    if os.path.exists(SAMPLE):
        gold.update(_golden(SAMPLE))
    specs = synth.batch_specs(4096, 24, 56, 2, 3, seed=2024, seed_base=1000)
    codes = [(s.n, s.k, s.seed, synth.random_systematic(s.n, s.k, s.seed)) for s in specs]
    with api.Batch() as b:
        for n, k, seed, G in codes:
            b.add(G, n)
        b.run()
        got = [b.result(i) for i in range(len(codes))]
    assert light > 2500
    for i, want in gold.items():
        n, k, seed, _ = codes[i]
        assert (n, k, seed) == (want["n"], want["k"], want["seed"])
        r = got[i]
        for key in ("d", "key", "message", "g_final", "j_final", "L_final"):
            assert r[key] == want[key], (i, key)
        assert [int(x) for x in r["witness"]] == want["witness"], i
        counts = r["counts"]
        for g in range(1, counts.shape[0]):  # the level check: every set of every level up to g_final
            for j in range(r["m"]):
                assert counts[g][j] == (math.comb(k, g) if g <= r["g_final"] else 0), (i, g, j)
    # every code (the heavy ones too) equals its single-code run
    rng = np.random.default_rng(7)
    heavy = [i for i in range(len(codes)) if i not in gold]
    for i in list(rng.choice(heavy, size=min(64, len(heavy)), replace=False)) + list(rng.choice(sorted(gold), 64)):
        n, k, seed, G = codes[int(i)]
        one = api.min_distance(G, n)
        for key in ("d", "key", "message", "g_final", "j_final", "m", "L_final"):
            assert got[int(i)][key] == one[key], (int(i), key)
        assert np.array_equal(got[int(i)]["witness"], one["witness"])
        assert np.array_equal(got[int(i)]["counts"], one["counts"])

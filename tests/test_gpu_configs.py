"""The full-size single-code workloads ([192,64], [150,64] with a rank-22 set, [300,50]
with six sets) in the launch configuration the benchmark times (default options):
units the oracle finishes in seconds compared key for key, and properties that hold at
any size for the whole run — the witness re-encodes to a codeword of weight d, every
enumerated unit counts C(k, g) combinations, the bound reached d at the last level — and
the whole run equal to the ALU-only path's."""

import math

import numpy as np
import pytest

import oracle
import synth
from synth.configs import single_code

pytestmark = pytest.mark.gpu

CONFIGS = [("192x64", 6), ("150x64", 6), ("300x50", 6)]


@pytest.fixture(scope="module")
def api():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_1603_06757_gb300 import api as a

    return a


def _bound(g, k, ranks):
    return sum(max(0, g + 1 - (k - r)) for r in ranks)


@pytest.mark.parametrize("name,g_max", CONFIGS)
def test_full_size_config(api, name, g_max):
    n, k, seed, G = single_code(name, lambda G, n, k: [int(r) for r in oracle.partition(G, n)["ranks"]])
    part = oracle.partition(G, n)
    m = part["m"]
    ranks = [int(r) for r in part["ranks"]]
    least = None
    with api.Code(G, n) as c:
        # sampled units against the oracle
        for j in range(m):
            for g in range(1, g_max + 1):
                want = oracle.enumerate_unit(part["gammas"][j], n, g, want_hist=False)
                U, key, combos = c.enumerate_level(g, j, U=n)
                assert combos == [math.comb(k, g)], (g, j)
                assert key == (want["min_w"], g, j, want["min_rank"]), (g, j)
                least = want["min_w"] if least is None else min(least, want["min_w"])
        r = c.min_distance()
    d = r["d"]
    assert r["ranks"] == ranks
    # the witness: message x G, weight d, and the key's weight
    msg = np.array([(r["message"] >> b) & 1 for b in range(k)], dtype=np.int64)
    cw = (msg @ synth.unpack_bits(G, n).astype(np.int64)) % 2
    assert int(cw.sum()) == d == r["key"][0]
    assert np.array_equal(cw.astype(np.uint8), synth.unpack_bits(r["witness"][None, :], n)[0])
    assert d <= least
    # counts: every unit up to the last one enumerated all C(k, g) combinations
    g_final, j_final = r["g_final"], r["j_final"]
    for g in range(1, g_final + 1):
        for j in range(m):
            if (g, j) <= (g_final, j_final):
                assert int(r["counts"][g, j]) == math.comb(k, g), (g, j)
            else:
                assert int(r["counts"][g, j]) == 0, (g, j)
    # termination: the bound reached d after the last level, and not before it when d
    # was already known then
    assert _bound(g_final, k, ranks) >= d
    if r["key"][1] < g_final:
        assert _bound(g_final - 1, k, ranks) < d
    # the same run on the ALU kernel alone
    with api.Code(G, n, tensor_cores=1) as c:
        r1 = c.min_distance()
    for key in ("d", "key", "message", "g_final", "j_final"):
        assert r1[key] == r[key], key
    assert np.array_equal(r1["counts"], r["counts"])

"""The tensor-core (tcgen05 Gram-matrix) enumerator against the oracle: every product
block forced onto it (tensor_cores=2), every block with a small side split into parts
with two large sides (tensor_cores=3), and the default split (large blocks on the
tensor cores, large blocks with a small side split, the rest on the ALU kernel)."""

import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_1603_06757_gb300 import api as a

    return a


# (n, k, seed): 1 to 8 stored words, odd and even k, partial sets
CASES = [(30, 12, 1), (48, 24, 2), (100, 40, 3), (150, 40, 4), (170, 41, 5), (192, 64, 8), (260, 40, 6),
         (96, 24, 5), (129, 64, 8), (290, 40, 7)]


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("n,k,seed", CASES)
def test_unit_keys_all_blocks_on_tensor_cores(api, mode, n, k, seed):
    """Per unit, at four thresholds.  At U = n every pair is a candidate; at U = min
    (the tie) the threshold never moves during the launch, so the pairs the MMA filter
    passes to the exact recheck are exactly the codewords of weight min in the blocks it
    covers: with every block on the tensor cores their count must equal the oracle's
    histogram there, which a wrong accumulator (too low: pairs missed; too high: extra
    pairs) cannot match.  At U = min + 2 the key must still be the oracle's and the pass
    count lies between the weight-min and weight-<=min+2 counts; at U = min - 1 nothing
    passes the recheck."""
    G = synth.random_systematic(n, k, seed)
    part = oracle.partition(G, n)
    checked_tie = 0
    with api.Code(G, n, tensor_cores=mode) as c:
        for j in range(part["m"]):
            for g in range(1, k + 1):
                C = math.comb(k, g)
                if C > 3_000_000:
                    break
                want = oracle.enumerate_unit(part["gammas"][j], n, g, want_hist=True)
                hist = [int(x) for x in want["hist"]]
                mw = want["min_w"]
                U, key, combos = c.enumerate_level(g, j, U=n)
                assert combos == [C]
                assert key == (mw, g, j, want["min_rank"]), (g, j)
                # the tie: exactly the weight-min codewords pass the filter
                U1, key1, _ = c.enumerate_level(g, j, U=mw)
                assert key1 == (mw, g, j, want["min_rank"]) and U1 == mw, (g, j)
                cnt = c.level_counters()
                if cnt["tc_combos"] == C:
                    assert cnt["tc_candidates"] == hist[mw], (g, j, cnt, hist[mw])
                    checked_tie += 1
                else:
                    assert cnt["tc_candidates"] <= hist[mw], (g, j, cnt)
                # two above the least weight: same key, pass count bounded by the histogram
                U3, key3, _ = c.enumerate_level(g, j, U=mw + 2)
                assert key3 == (mw, g, j, want["min_rank"]) and U3 == mw, (g, j)
                cnt = c.level_counters()
                if cnt["tc_combos"] == C:
                    assert hist[mw] <= cnt["tc_candidates"] <= sum(hist[mw:mw + 3]), (g, j, cnt)
                if C >= 4096:
                    assert cnt["tc_candidates"] * 16 < C, (g, j, cnt)  # the filter, not the recheck, decides
                # a threshold just below the least weight: no candidate at all
                U2, key2, _ = c.enumerate_level(g, j, U=mw - 1)
                assert key2 is None and U2 == mw - 1
    if mode == 2:
        assert checked_tie > 0


@pytest.mark.parametrize("mode", [0, 2, 3])
@pytest.mark.parametrize("n,k,seed", [(120, 36, 3), (150, 36, 14), (96, 24, 5), (180, 36, 13), (60, 30, 1),
                                      (260, 30, 9)])
def test_min_distance_tensor_cores(api, mode, n, k, seed):
    G = synth.random_systematic(n, k, seed)
    with api.Code(G, n, tensor_cores=mode) as c:
        got = c.min_distance()
    want = oracle.min_distance(G, n)
    for key in ("d", "key", "message", "g_final", "j_final", "L_final"):
        assert got[key] == want[key], key
    assert np.array_equal(got["witness"], want["witness"])
    assert np.array_equal(got["counts"], want["counts"])


def test_large_level_matches_alu_kernel(api):
    # a large level of the [192,64] code: tensor-core split vs the ALU kernel alone
    G = synth.random_systematic(192, 64, 8)
    with api.Code(G, 192, tensor_cores=1) as c:
        want = c.enumerate_level(7, 1, U=40)
    with api.Code(G, 192, tensor_cores=0) as c:
        got = c.enumerate_level(7, 1, U=40)
    assert got == want


@pytest.mark.parametrize("g,j", [(6, 0), (7, 0), (6, 1)])
def test_split_blocks_default_mode_vs_oracle(api, g, j):
    # [80,64]: blocks X_1 x Y_(g-1) of >= 2^24 codewords are split over the quarters of
    # H2 in the default mode; set 0 stores 1 word per row, set 1 (rank 16) 3 words
    G = synth.random_systematic(80, 64, 3)
    part = oracle.partition(G, 80)
    want = oracle.enumerate_unit(part["gammas"][j], 80, g, want_hist=False)
    with api.Code(G, 80) as c:
        U, key, combos = c.enumerate_level(g, j, U=80)
        assert combos == [math.comb(64, g)]
        assert key == (want["min_w"], g, j, want["min_rank"])
        U2, key2, _ = c.enumerate_level(g, j, U=want["min_w"] - 1)
        assert key2 is None and U2 == want["min_w"] - 1


@pytest.mark.parametrize("n,k,seed,g,all_tc", [(192, 64, 8, 5, True), (260, 30, 9, 6, True), (60, 30, 1, 5, False)])
def test_default_plan_follows_the_code_size(api, n, k, seed, g, all_tc):
    """tensor_cores = 0 puts every block of a level on the tensor cores on a code whose
    Gilbert-Varshamov work estimate reaches 10^7 codewords ([192,64], [260,30]); a
    small code ([60,30]: about 10^5) keeps its small-side blocks on the ALU kernel.
    Either way the unit's key and count equal the ALU-only run's."""
    G = synth.random_systematic(n, k, seed)
    with api.Code(G, n) as c:
        U, key, combos = c.enumerate_level(g, 0, U=n)
        tc = c.level_counters()["tc_combos"]
    with api.Code(G, n, tensor_cores=1) as c1:
        U1, key1, combos1 = c1.enumerate_level(g, 0, U=n)
    assert (U, key, combos[0]) == (U1, key1, combos1[0]) and combos[0] == math.comb(k, g)
    if all_tc:
        assert tc == math.comb(k, g)
    else:
        assert tc < math.comb(k, g)

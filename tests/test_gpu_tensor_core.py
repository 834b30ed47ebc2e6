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


# (n, k, seed): 1 to 7 stored words, odd and even k, partial sets
CASES = [(30, 12, 1), (48, 24, 2), (100, 40, 3), (150, 40, 4), (170, 41, 5), (192, 64, 8), (260, 40, 6),
         (96, 24, 5), (129, 64, 8)]


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("n,k,seed", CASES)
def test_unit_keys_all_blocks_on_tensor_cores(api, mode, n, k, seed):
    G = synth.random_systematic(n, k, seed)
    part = oracle.partition(G, n)
    with api.Code(G, n, tensor_cores=mode) as c:
        for j in range(part["m"]):
            for g in range(1, k + 1):
                if math.comb(k, g) > 3_000_000:
                    break
                U, key, combos = c.enumerate_level(g, j, U=n)
                want = oracle.enumerate_unit(part["gammas"][j], n, g, want_hist=False)
                assert combos == [math.comb(k, g)]
                assert key == (want["min_w"], g, j, want["min_rank"]), (g, j)
                # a threshold just below the least weight: no candidate at all
                U2, key2, _ = c.enumerate_level(g, j, U=want["min_w"] - 1)
                assert key2 is None and U2 == want["min_w"] - 1


@pytest.mark.parametrize("mode", [0, 2, 3])
@pytest.mark.parametrize("n,k,seed", [(120, 36, 3), (150, 36, 14), (96, 24, 5), (180, 36, 13), (60, 30, 1)])
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

"""The overlapping-information-set mode (mdist_options.overlap_sets, the non-disjoint
case of §2) on the GPU against the oracle's restatement of it: the whole Alg. 1 run —
d, witness key, message, witness, last unit, final bounds and every per-unit count —
bit for bit, in both check modes and with the tensor-core enumerator on and off."""

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


def _same(got, want):
    for key in ("d", "key", "message", "g_final", "j_final", "m", "L_final"):
        assert got[key] == want[key], key
    assert got["ranks"] == [int(r) for r in want["ranks"]]
    assert np.array_equal(got["witness"], want["witness"])
    assert np.array_equal(got["counts"], want["counts"])


def _codes():
    out = []
    for seed in range(36):
        rng = synth.SplitMix64(12000 + seed)
        k = rng.uniform_int(8, 40)
        n = rng.uniform_int(k + 2, 2 * k - 1) if seed % 4 else rng.uniform_int(2 * k, 3 * k)
        out.append((n, k, rng.uniform_int(2, 5), seed))
    return out


@pytest.mark.parametrize("n,k,M,seed", _codes())
def test_overlap_run_matches_oracle(api, n, k, M, seed):
    G = synth.random_systematic(n, k, seed)
    want = oracle.min_distance(G, n, overlap_sets=M)
    got = api.min_distance(G, n, overlap_sets=M)
    _same(got, want)
    # the information sets on the device handle are the oracle's
    with api.Code(G, n, overlap_sets=M) as c:
        sets = c.info_sets()
    o = oracle.partition_overlap(G, n, M)
    for key in ("ranks", "pivcols", "gammas", "transforms"):
        assert np.array_equal(sets[key], o[key]), key


@pytest.mark.parametrize("per_matrix", [False, True])
@pytest.mark.parametrize("tc", [0, 1, 2])
def test_overlap_modes(api, per_matrix, tc):
    for n, k, M, seed in [(96, 64, 3, 1), (60, 40, 4, 2), (70, 36, 2, 3)]:
        G = synth.random_systematic(n, k, seed)
        want = oracle.min_distance(G, n, overlap_sets=M, check_per_matrix=per_matrix)
        got = api.min_distance(G, n, overlap_sets=M, check_per_matrix=per_matrix, tensor_cores=tc)
        _same(got, want)


def test_overlap_saves_work_when_n_below_2k(api):
    # [96,64]: disjoint sets of ranks 64 and 32 against three overlapping sets
    G = synth.random_systematic(96, 64, 1)
    plain = api.min_distance(G, 96)
    over = api.min_distance(G, 96, overlap_sets=3)
    assert plain["d"] == over["d"]
    assert over["total_combos"] * 20 < plain["total_combos"]

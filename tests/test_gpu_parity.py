"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Everything is exact integer work, so every comparison is bit-exact: information sets,
per-unit weight histograms and counts, per-unit least (weight, rank), and the whole
Alg. 1 run (d, witness key, message, witness, last unit, counts, final bounds)."""

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


def _gpu_min_distance(api, G, n, per_matrix=False):
    return api.min_distance(G, n, check_per_matrix=per_matrix)


def _assert_same_run(got, want):
    assert got["d"] == want["d"]
    assert got["key"] == want["key"]
    assert got["message"] == want["message"]
    assert np.array_equal(got["witness"], want["witness"])
    assert got["g_final"] == want["g_final"]
    assert got["j_final"] == want["j_final"]
    assert got["m"] == want["m"]
    assert got["ranks"] == list(want["ranks"])
    assert got["L_final"] == want["L_final"]
    assert np.array_equal(got["counts"], want["counts"])


def test_info_sets_on_device_handle(api):
    for n, k, seed in [(60, 30, 1), (150, 64, 3), (300, 50, 2), (97, 33, 4)]:
        G = synth.random_systematic(n, k, seed)
        with api.Code(G, n) as c:
            got = c.info_sets()
        want = oracle.partition(G, n)
        for key in ("ranks", "pivcols", "gammas", "transforms"):
            assert np.array_equal(got[key], want[key]), key


# (n, k, seed): row widths from 1 to 16 32-bit words, full and partial sets, halves of
# odd size, several tiles per product block and ragged tails
HIST_CASES = [
    (30, 12, 1),    # n-k = 18 -> 1 word; partial second set
    (48, 24, 2),    # 1 word, two full sets
    (100, 40, 3),   # 2 words
    (150, 40, 4),   # 4 words, partial fourth set (30 columns)
    (170, 41, 5),   # odd k, 5 words
    (300, 40, 6),   # 9 words
    (512, 40, 7),   # 15 words (full), 16 words (partial set)
    (129, 64, 8),   # k = 64, 3 words, second set of rank 64? (65 columns)
    (200, 64, 9),   # k = 64, partial third set (72 columns)
]


@pytest.mark.parametrize("n,k,seed", HIST_CASES)
def test_unit_histograms_and_counts(api, n, k, seed):
    G = synth.random_systematic(n, k, seed)
    part = oracle.partition(G, n)
    budget = 4_000_000
    with api.Code(G, n) as c:
        for j in range(part["m"]):
            for g in range(1, k + 1):
                if math.comb(k, g) > budget:
                    break
                hist, cnt = c.unit_histogram(g, j)
                want = oracle.enumerate_unit(part["gammas"][j], n, g)
                assert cnt == want["count"] == math.comb(k, g)
                assert np.array_equal(hist, want["hist"]), (g, j)


@pytest.mark.parametrize("n,k,seed", HIST_CASES)
def test_unit_least_key(api, n, k, seed):
    G = synth.random_systematic(n, k, seed)
    part = oracle.partition(G, n)
    budget = 4_000_000
    with api.Code(G, n) as c:
        for j in range(part["m"]):
            for g in range(1, k + 1):
                if math.comb(k, g) > budget:
                    break
                U, key, combos = c.enumerate_level(g, j, U=n)
                want = oracle.enumerate_unit(part["gammas"][j], n, g, want_hist=False)
                assert key == (want["min_w"], g, j, want["min_rank"]), (g, j)
                assert U == want["min_w"]
                assert combos == [math.comb(k, g)]


def test_threshold_semantics(api):
    n, k = 120, 40
    G = synth.random_systematic(n, k, 12)
    part = oracle.partition(G, n)
    want = oracle.enumerate_unit(part["gammas"][1], n, 4, want_hist=False)
    with api.Code(G, n) as c:
        # below the least weight: no candidate, U unchanged
        U, key, _ = c.enumerate_level(4, 1, U=want["min_w"] - 1)
        assert key is None and U == want["min_w"] - 1
        # at the least weight: the tie is a candidate
        U, key, _ = c.enumerate_level(4, 1, U=want["min_w"])
        assert key == (want["min_w"], 4, 1, want["min_rank"])
        # an existing smaller key is kept
        U, key, _ = c.enumerate_level(4, 1, U=n, key=(1, 1, 0, 0))
        assert key == (1, 1, 0, 0)


def test_all_sets_in_one_call(api):
    n, k = 150, 50
    G = synth.random_systematic(n, k, 21)
    part = oracle.partition(G, n)
    best = None
    for j in range(part["m"]):
        u = oracle.enumerate_unit(part["gammas"][j], n, 3, want_hist=False)
        cand = (u["min_w"], 3, j, u["min_rank"])
        best = cand if best is None or cand < best else best
    with api.Code(G, n) as c:
        U, key, combos = c.enumerate_level(3, -1, U=n)
    assert key == best and U == best[0]
    assert combos == [math.comb(k, 3)] * part["m"]


TEXTBOOK = [
    ("hamming", synth.hamming_7_4, 7, 3),
    ("golay", synth.golay_24_12, 24, 8),
    ("rm15", synth.reed_muller_1_5, 32, 16),
    ("rep5", lambda: synth.repetition(5), 5, 5),
    ("even4", lambda: synth.even_weight(4), 4, 2),
    ("rep64", lambda: synth.repetition(64), 64, 64),
]


@pytest.mark.parametrize("name,make,n,d", TEXTBOOK, ids=[t[0] for t in TEXTBOOK])
@pytest.mark.parametrize("per_matrix", [False, True])
def test_textbook_codes(api, name, make, n, d, per_matrix):
    G = make()
    got = _gpu_min_distance(api, G, n, per_matrix)
    assert got["d"] == d
    _assert_same_run(got, oracle.min_distance(G, n, check_per_matrix=per_matrix))


ORACLE_BUDGET = 3e9  # combinations the oracle may need for one run in these tests


@pytest.mark.parametrize("seed", range(60))
def test_min_distance_random_vs_oracle(api, seed):
    rng = synth.SplitMix64(31000 + seed)
    k = rng.uniform_int(1, 40)
    n = rng.uniform_int(k + 1, min(512, 4 * k + 1))
    G = synth.random_systematic(n, k, seed)
    per_matrix = bool(seed % 2)
    got = _gpu_min_distance(api, G, n, per_matrix)
    if got["total_combos"] > ORACLE_BUDGET:  # size check only; parity below is against the oracle
        pytest.skip("oracle too slow for this draw")
    _assert_same_run(got, oracle.min_distance(G, n, check_per_matrix=per_matrix))
    if k <= 24:
        assert got["d"] == oracle.brute_force_distance(G, n)


def test_config_60_30_against_brute_force(api):
    # [60,30]: G = [I_30 | R], R from SplitMix64 seed 1; d checked against all 2^30 codewords
    n, k = 60, 30
    G = synth.random_systematic(n, k, 1)
    got = _gpu_min_distance(api, G, n)
    assert got["d"] == oracle.brute_force_distance(G, n)
    _assert_same_run(got, oracle.min_distance(G, n))
    for per_matrix in (True,):
        _assert_same_run(_gpu_min_distance(api, G, n, per_matrix), oracle.min_distance(G, n, per_matrix))


def test_checkpoint_resume(api):
    n, k = 120, 36
    G = synth.random_systematic(n, k, 5)
    straight = _gpu_min_distance(api, G, n)
    with api.Code(G, n) as c:
        assert not c.run(max_units=5)
        blob = c.state_save()
    with api.Code(G, n) as c2:
        c2.state_load(blob)
        assert c2.run()
        resumed = c2.result()
    _assert_same_run(resumed, straight)
    # a blob does not load into another code
    with api.Code(synth.random_systematic(n, k, 6), n) as c3:
        with pytest.raises(Exception):
            c3.state_load(blob)


def test_errors(api):
    from paper_1603_06757_gb300 import _lib as L

    G = synth.random_systematic(128, 64, 1)
    with api.Code(G, 128) as c:
        with pytest.raises(L.MdistError) as e:
            c.enumerate_level(32, 0, U=128)  # C(64, 32) >= 2^54
        assert e.value.code == L.ERANGE
        with pytest.raises(L.MdistError) as e:
            c.enumerate_level(0, 0)
        assert e.value.code == L.EINVAL
    bad = G.copy()
    bad[0, 1] |= np.uint64(1) << np.uint64(63)  # a bit past column n = 100
    with pytest.raises(L.MdistError) as e:
        api.Code(bad[:, :2], 100)
    assert e.value.code == L.EINVAL
    dup = np.vstack([G[:1], G[:1]])
    with pytest.raises(L.MdistError) as e:
        api.Code(dup, 128)
    assert e.value.code == L.ERANK


def test_side_stream(api):
    import torch

    n, k = 90, 30
    G = synth.random_systematic(n, k, 3)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        got = api.min_distance(G, n)
    _assert_same_run(got, oracle.min_distance(G, n))


# (n, k, seed): 3, 4, 5, 9 and 15 words per stored row, Alg. 1 work small enough for the oracle
VARIANT_CASES = [(120, 36, 3), (150, 36, 14), (180, 36, 13), (300, 30, 2), (500, 25, 6), (96, 24, 5)]


@pytest.mark.parametrize("fg", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n,k,seed", VARIANT_CASES)
def test_filter_variants_identical(api, fg, n, k, seed):
    # every enumerator variant (exact, OR-groups of 2, 3, 4 words, 4 then 2) gives the same run
    G = synth.random_systematic(n, k, seed)
    with api.Code(G, n, filter_group=fg) as c:
        got = c.min_distance()
    assert got["total_combos"] <= ORACLE_BUDGET
    _assert_same_run(got, oracle.min_distance(G, n))


@pytest.mark.parametrize("hint", [2, 4, 7, 30])
@pytest.mark.parametrize("per_matrix", [False, True])
def test_wave_hint_does_not_change_results(api, hint, per_matrix):
    # levels launched ahead as one wave (hint too small, about right, far too large)
    for n, k, seed in [(120, 36, 3), (96, 24, 5), (150, 36, 14)]:
        G = synth.random_systematic(n, k, seed)
        with api.Code(G, n, check_per_matrix=per_matrix, wstar_hint=hint) as c:
            got = c.min_distance()
        _assert_same_run(got, oracle.min_distance(G, n, check_per_matrix=per_matrix))

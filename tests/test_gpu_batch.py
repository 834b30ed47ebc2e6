"""The batched engine gives, code by code, exactly the single-code run's result (and
the oracle's), whatever the mix of shapes, the speculation hints or the check mode."""

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
    assert got["ranks"] == list(want["ranks"])
    assert np.array_equal(got["witness"], want["witness"])
    assert np.array_equal(got["counts"], want["counts"])


def _mix(count, seed, k_lo=6, k_hi=40):
    specs = synth.batch_specs(count, k_lo, k_hi, 2, 3, seed=seed, seed_base=5000 + seed)
    return [(s.n, s.k, synth.random_systematic(s.n, s.k, s.seed)) for s in specs]


@pytest.mark.parametrize("per_matrix", [False, True])
def test_batch_matches_single_runs(api, per_matrix):
    codes = _mix(120, 1)
    with api.Batch(check_per_matrix=per_matrix) as b:
        for n, k, G in codes:
            b.add(G, n)
        b.run()
        info = b.info()
        got = [b.result(i) for i in range(len(codes))]
    # the default run is ONE launch of the loop graph, however many rounds it takes
    assert info["codes"] == len(codes) and info["graph_launches"] == 1 and info["rounds"] >= 2
    for (n, k, G), r in zip(codes, got):
        _same(r, api.min_distance(G, n, check_per_matrix=per_matrix))


def test_batch_matches_oracle(api):
    codes = _mix(40, 2, k_lo=4, k_hi=28)
    with api.Batch() as b:
        for n, k, G in codes:
            b.add(G, n)
        b.run()
        got = [b.result(i) for i in range(len(codes))]
    for (n, k, G), r in zip(codes, got):
        _same(r, oracle.min_distance(G, n))


@pytest.mark.parametrize("hint", [0, 2, 5, 40])
def test_batch_speculation_does_not_change_results(api, hint):
    # levels enumerated ahead (hint too small, about right, far too large) never change a result
    codes = _mix(30, 3, k_lo=8, k_hi=30)
    with api.Batch() as b:
        for n, k, G in codes:
            b.add(G, n, wstar_hint=hint)
        b.run(rounds_per_graph=3)
        got = [b.result(i) for i in range(len(codes))]
    for (n, k, G), r in zip(codes, got):
        _same(r, api.min_distance(G, n))


def test_batch_textbook_and_edges(api):
    items = [(synth.hamming_7_4(), 7), (synth.golay_24_12(), 24), (synth.reed_muller_1_5(), 32),
             (synth.repetition(5), 5), (synth.even_weight(4), 4), (synth.repetition(64), 64),
             (synth.random_systematic(512, 40, 7), 512), (synth.random_systematic(65, 64, 2), 65)]
    with api.Batch() as b:
        for G, n in items:
            b.add(G, n)
        b.run()
        got = [b.result(i) for i in range(len(items))]
    for (G, n), r in zip(items, got):
        _same(r, api.min_distance(G, n))


@pytest.mark.parametrize("tc", [0, 2])
def test_batch_routes_large_codes_to_tensor_core_path(api, tc):
    # a mix with codes of >= 10^9 estimated codewords: those run on the single-code
    # tensor-core path inside mdist_batch_run (tc = 0), or every code does (tc = 2);
    # every result is the single-code run's, and the light codes' the oracle's
    codes = _mix(24, 4, k_lo=10, k_hi=30) + [(n, k, synth.random_systematic(n, k, 900 + i))
                                             for i, (n, k) in enumerate([(112, 48), (116, 48), (120, 48)])]
    with api.Batch(tensor_cores=tc) as b:
        for n, k, G in codes:
            b.add(G, n)
        b.run()
        info = b.info()
        got = [b.result(i) for i in range(len(codes))]
    assert info["large_codes"] == (len(codes) if tc == 2 else 3)
    assert info["large_ms"] > 0
    for (n, k, G), r in zip(codes, got):
        _same(r, api.min_distance(G, n))
        if k <= 30:
            _same(r, oracle.min_distance(G, n))

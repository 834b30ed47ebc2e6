"""Serving loop: requests admitted while others are in flight (continuous batching),
bounded by slots and rows memory; large requests routed to the single-code tensor-core
path between rounds; every result equals the code's run alone and, for the requests
the oracle finishes in well under a second (k <= 36), the oracle's."""

import time

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


def _requests(count, seed, k_lo=10, k_hi=36):
    rng = synth.SplitMix64(seed)
    out = []
    for i in range(count):
        k = rng.uniform_int(k_lo, k_hi)
        n = rng.uniform_int(2 * k, 4 * k)
        out.append((n, k, synth.random_systematic(n, k, 90000 + seed * 1000 + i)))
    return out


def _drain(srv, ids, timeout_s=120):
    res = {}
    t0 = time.time()
    while len(res) < len(ids):
        for rid in ids:
            if rid not in res:
                r = srv.poll(rid, wait_ms=5)
                if r is not None:
                    res[rid] = r
        assert time.time() - t0 < timeout_s
    return res


@pytest.mark.parametrize("per_matrix", [False, True])
def test_results_same_alone_and_in_the_mix(api, per_matrix):
    reqs = _requests(120, 1)
    with api.Server(max_slots=64, rows_pool_bytes=4 << 20, check_per_matrix=per_matrix) as srv:
        ids = []
        for i, (n, k, G) in enumerate(reqs):
            ids.append(srv.submit(G, n))
            if i % 20 == 19:
                time.sleep(0.01)  # later requests arrive while earlier ones are on the GPU
        res = _drain(srv, ids)
        info = srv.info()
    assert info["completed"] == len(reqs) and info["queued"] == 0 and info["in_flight"] == 0
    assert info["rounds"] > 0
    for rid, (n, k, G) in zip(ids, reqs):
        _same(res[rid], api.min_distance(G, n, check_per_matrix=per_matrix, max_sets=8))
        _same(res[rid], oracle.min_distance(G, n, check_per_matrix=per_matrix, max_sets=8))
        assert res[rid]["latency_s"] > 0


def test_admission_bounded_by_memory_and_slots(api):
    reqs = _requests(40, 2, k_lo=16, k_hi=30)
    # a pool a few requests large and 3 slots: requests wait in the queue, all complete
    with api.Server(max_slots=3, rows_pool_bytes=16 << 10) as srv:
        ids = [srv.submit(G, n) for n, k, G in reqs]
        res = _drain(srv, ids)
    for rid, (n, k, G) in zip(ids, reqs):
        _same(res[rid], api.min_distance(G, n, max_sets=8))
        _same(res[rid], oracle.min_distance(G, n, max_sets=8))


def test_oversize_request_rejected(api):
    from paper_1603_06757_gb300 import _lib as L

    G = synth.random_systematic(300, 60, 1)
    with api.Server(max_slots=2, rows_pool_bytes=4096) as srv:
        with pytest.raises(L.MdistError) as e:
            srv.submit(G, 300)
        assert e.value.code == L.ENOMEM


@pytest.mark.parametrize("tc", [0, 2])
def test_large_requests_on_the_tensor_core_path(api, tc):
    # tc=2: every request on the single-code path; tc=0: the large ones only (k up to 56:
    # several exceed 10^9 estimated codewords); both mixed with batched requests
    reqs = _requests(24, 3, k_lo=20, k_hi=56)
    with api.Server(max_slots=16, rows_pool_bytes=4 << 20, tensor_cores=tc) as srv:
        ids = []
        for i, (n, k, G) in enumerate(reqs):
            ids.append(srv.submit(G, n))
            if i % 6 == 5:
                time.sleep(0.01)
        res = _drain(srv, ids, timeout_s=300)
        info = srv.info()
    assert info["completed"] == len(reqs) and info["queued"] == 0 and info["in_flight"] == 0
    for rid, (n, k, G) in zip(ids, reqs):
        _same(res[rid], api.min_distance(G, n, max_sets=8))
        if k <= 36:
            _same(res[rid], oracle.min_distance(G, n, max_sets=8))

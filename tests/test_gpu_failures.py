"""Failure paths, made on the host or by a bounded device wait — no GPU fault:

- an allocator that refuses memory (the library's dev_alloc hook): mdist_prepare
  reports MDIST_ENOMEM; refused subset-sum tables leave their blocks on the ALU
  enumerator with the oracle's result; a refused histogram buffer is MDIST_ENOMEM and the
  handle stays usable;
- the tensor-core enumerator's pipeline waits bounded to one poll (timeout_cycles = 1):
  the call returns MDIST_ETIMEOUT after the launch has drained, and the device keeps
  working;
- a serving request cancelled while queued or in flight polls as MDIST_ECANCELLED; the
  others are unaffected."""

import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_1603_06757_gb300 import _lib as L
    from paper_1603_06757_gb300 import api

    return torch, L, api


def _refusing_allocator(api, torch, refuse):
    """torch's caching allocator behind the hook, except where refuse(nbytes, calls) is true."""

    class Refusing(api._TorchAllocator):
        def __init__(self):
            super().__init__(torch, torch.cuda.current_device())
            self.calls = 0
            self.refused = 0
            self.alloc_cb = api.L.ALLOC_FN(self._maybe)

        def _maybe(self, nbytes, ctx):
            self.calls += 1
            if refuse(int(nbytes), self):
                self.refused += 1
                return None
            return self._alloc(nbytes, ctx)

    return Refusing()


def test_prepare_reports_enomem(env):
    torch, L, api = env
    G = synth.random_systematic(96, 24, 5)
    a = _refusing_allocator(api, torch, lambda nbytes, s: True)
    with pytest.raises(L.MdistError) as e:
        api.Code(G, 96, allocator=a)
    assert e.value.code == L.ENOMEM and a.refused >= 1


def test_refused_tables_stay_on_alu_kernel(env):
    torch, L, api = env
    n, k = 120, 36
    G = synth.random_systematic(n, k, 3)
    want = oracle.min_distance(G, n)
    with api.Code(G, n) as c:
        normal = c.min_distance()
    assert normal["tc_launches"] > 0  # the tables are used when they can be had
    a = _refusing_allocator(api, torch, lambda nbytes, s: nbytes > (8 << 20))
    with api.Code(G, n, allocator=a) as c:
        got = c.min_distance()
    assert a.refused > 0 and got["tc_launches"] == 0
    for key in ("d", "key", "message", "g_final", "j_final", "L_final"):
        assert got[key] == want[key], key
    assert np.array_equal(got["counts"], want["counts"])


def test_refused_histogram_buffer(env):
    torch, L, api = env
    n, k = 96, 24
    G = synth.random_systematic(n, k, 5)
    part = oracle.partition(G, n)
    state = {"closed": False}
    a = _refusing_allocator(api, torch, lambda nbytes, s: state["closed"])
    with api.Code(G, n, allocator=a) as c:
        state["closed"] = True  # everything after mdist_prepare is refused
        with pytest.raises(L.MdistError) as e:
            c.unit_histogram(3, 0)
        assert e.value.code == L.ENOMEM
        U, key, combos = c.enumerate_level(3, 0, U=n)  # the handle still works
        w = oracle.enumerate_unit(part["gammas"][0], n, 3, want_hist=False)
        assert key == (w["min_w"], 3, 0, w["min_rank"]) and combos == [math.comb(k, 3)]


def test_bounded_waits_report_timeout(env):
    torch, L, api = env
    n, k = 192, 64
    G = synth.random_systematic(n, k, 8)
    part = oracle.partition(G, n)
    g = 5  # every block on the tensor cores: thousands of waits per launch
    timeouts = ok = 0
    with api.Code(G, n, tensor_cores=2, timeout_cycles=1) as c:
        for _ in range(4):
            try:
                c.enumerate_level(g, 0, U=n)
                ok += 1
            except L.MdistError as e:
                assert e.code == L.ETIMEOUT
                timeouts += 1
    assert timeouts >= 1
    # the device and a default handle carry on
    want = oracle.enumerate_unit(part["gammas"][0], n, g, want_hist=False)
    with api.Code(G, n, tensor_cores=2) as c:
        U, key, combos = c.enumerate_level(g, 0, U=n)
    assert key == (want["min_w"], g, 0, want["min_rank"]) and combos == [math.comb(k, g)]


def test_server_cancel(env):
    torch, L, api = env
    reqs = [(n, synth.random_systematic(n, k, 300 + i)) for i, (n, k) in
            enumerate([(80, 30), (90, 32), (84, 28), (100, 34), (76, 30), (88, 30)])]
    with api.Server(max_slots=1, rows_pool_bytes=1 << 20, tensor_cores=1) as srv:
        ids = [srv.submit(G, n) for (n, G) in reqs]
        assert srv.cancel(ids[4]) == L.OK  # one slot: the fifth request is still queued
        first = srv.cancel(ids[0])         # in flight, or already done
        assert first in (L.OK, L.EAGAIN)
        assert srv.cancel(10**9) == L.EINVAL
        for i, rid in enumerate(ids):
            cancelled = i == 4 or (i == 0 and first == L.OK)
            if cancelled:
                with pytest.raises(L.MdistError) as e:
                    while srv.poll(rid, wait_ms=200) is None:
                        pass
                assert e.value.code == L.ECANCELLED
                assert srv.cancel(rid) == L.EINVAL  # polled: forgotten
                continue
            r = None
            while r is None:
                r = srv.poll(rid, wait_ms=200)
            n, G = reqs[i]
            want = oracle.min_distance(G, n, max_sets=8)
            assert r["d"] == want["d"] and r["key"] == want["key"]
            assert np.array_equal(r["counts"], want["counts"][:, : r["m"]])

"""One code's run split over ranks (mdist_enumerate_level_part, mdist_run_sharded), with
host threads standing in for the ranks on one GPU (each thread its own handle; the
exchange meets at a host barrier, so no kernel waits on another rank): every rank's
result equals the oracle's whole run, in both check modes and with the tensor-core
enumerator's work units split too; a unit's slices partition its combinations; a rank
that fails its exchange stops the run with MDIST_ECANCELLED."""

import functools
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
    from paper_1603_06757_gb300 import api, parallel

    return L, api, parallel


@functools.lru_cache(maxsize=None)
def _oracle_run(n, k, seed, per_matrix):
    return oracle.min_distance(synth.random_systematic(n, k, seed), n, check_per_matrix=per_matrix)


def _same(got, want):
    for key in ("d", "key", "message", "g_final", "j_final", "m", "L_final"):
        assert got[key] == want[key], key
    assert np.array_equal(got["witness"], want["witness"])
    assert np.array_equal(got["counts"], want["counts"])


@pytest.mark.parametrize("per_matrix", [False, True])
@pytest.mark.parametrize("nparts", [2, 3])
@pytest.mark.parametrize("n,k,seed", [(60, 30, 1), (120, 36, 3), (96, 24, 5), (150, 40, 4), (80, 64, 3)])
def test_sharded_run_matches_oracle(env, per_matrix, nparts, n, k, seed):
    L, api, parallel = env
    G = synth.random_systematic(n, k, seed)
    want = _oracle_run(n, k, seed, per_matrix)
    outs = parallel.sharded_min_distance_threads(G, n, nparts, check_per_matrix=per_matrix)
    for r in outs:
        _same(r, want)


def test_unit_slices_partition_the_unit(env):
    L, api, parallel = env
    G = synth.random_systematic(192, 64, 8)
    with api.Code(G, 192) as c:
        for g in (5, 7):
            U, key, combos = c.enumerate_level(g, 1, U=192)
            tc_whole = c.level_counters()["tc_combos"]
            keys, total = [], 0
            for p in range(4):
                Up, kp, cp = c.enumerate_level_part(g, 1, p, 4, U=192)
                keys.append(kp)
                total += cp[0]
            assert tc_whole > 0  # the tensor-core work units are split too
            assert total == combos[0] == math.comb(64, g)
            assert min(k for k in keys if k is not None) == key


def test_sharded_large_config_equals_single_run(env):
    L, api, parallel = env
    G = synth.random_systematic(150, 64, 1)  # ranks 64, 64, 22
    want = api.min_distance(G, 150)
    outs = parallel.sharded_min_distance_threads(G, 150, 2)
    for r in outs:
        _same(r, want)


def test_failed_exchange_cancels(env):
    L, api, parallel = env
    G = synth.random_systematic(60, 30, 1)

    def broken(key, count):
        raise RuntimeError("rank lost")

    with pytest.raises(L.MdistError) as e:
        parallel.sharded_min_distance(G, 60, 0, 2, broken)
    assert e.value.code == L.ECANCELLED

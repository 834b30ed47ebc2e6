"""Whole Alg. 1 runs of the full-size single-code workloads ([150,64], [192,64],
[300,50]; [60,30] too) in the launch configuration the benchmark times, against the
oracle's runs of the same codes stored by tests/golden/make_config_goldens.py (hours of
CPU time each): d, witness key, message, witness, last unit, final bounds and the
combination count of every (g, j) unit, field by field.  Plus the dominant level's units
of [192,64] (level 8, the tensor-core enumerator's large launches) against the oracle
computed here: key, count, and at the tie threshold the filter's pass count against the
oracle's histogram."""

import math
import os

import numpy as np
import pytest

import oracle
from conftest import golden_path
from synth.configs import single_code

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_1603_06757_gb300 import api as a

    return a


def _read_golden(name):
    out = {"counts": {}}
    with open(golden_path(f"oracle_run_{name}.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            if key == "counts":
                out["counts"][int(vals[0])] = [int(v) for v in vals[1:]]
            elif key == "name":
                out[key] = vals[0]
            else:
                out[key] = [int(v) for v in vals] if len(vals) > 1 or key in ("ranks", "witness", "key") else int(vals[0])
    return out


def _oracle_ranks(G, n, k):
    return [int(r) for r in oracle.partition(G, n)["ranks"]]


@pytest.mark.parametrize("name", ["60x30", "150x64", "192x64", "300x50"])
def test_whole_run_matches_oracle_golden(api, name):
    if not os.path.exists(golden_path(f"oracle_run_{name}.txt")):
        pytest.skip(f"oracle run of {name} not written yet (tests/golden/make_config_goldens.py)")
    want = _read_golden(name)
    n, k, seed, G = single_code(name, _oracle_ranks)
    assert (n, k, seed) == (want["n"], want["k"], want["seed"])
    got = api.min_distance(G, n)  # default options: the benchmark's launch configuration
    assert got["d"] == want["d"]
    assert list(got["key"]) == want["key"]
    assert got["message"] == want["message"]
    assert [int(w) for w in got["witness"]] == want["witness"]
    assert got["ranks"] == want["ranks"] and got["m"] == want["m"]
    assert (got["g_final"], got["j_final"]) == (want["g_final"], want["j_final"])
    assert (got["L_final"], got["U_final"]) == (want["L_final"], want["U_final"])
    counts = got["counts"]
    for g in range(counts.shape[0]):
        row = [int(x) for x in counts[g]]
        assert row == want["counts"].get(g, [0] * want["m"]), g
    assert got["total_combos"] == want["codewords"]
    if name != "60x30":
        assert got["tc_launches"] > 0  # the large levels ran on the tensor cores


def test_192x64_level8_units_vs_oracle(api):
    n, k, seed, G = single_code("192x64", _oracle_ranks)
    part = oracle.partition(G, n)
    g = 8
    with api.Code(G, n) as c:
        for j in range(part["m"]):
            want = oracle.enumerate_unit(part["gammas"][j], n, g, want_hist=True)
            mw, hist = want["min_w"], [int(x) for x in want["hist"]]
            U, key, combos = c.enumerate_level(g, j, U=n)
            assert combos == [math.comb(k, g)] and key == (mw, g, j, want["min_rank"]), j
            U1, key1, _ = c.enumerate_level(g, j, U=mw)  # the tie: the threshold never moves
            assert key1 == (mw, g, j, want["min_rank"]) and U1 == mw
            cnt = c.level_counters()
            assert cnt["tc_combos"] > math.comb(k, g) // 2  # most of the level on the tensor cores
            assert cnt["tc_candidates"] <= hist[mw]

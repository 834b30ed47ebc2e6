"""Pins of the oracle's overlapping-information-set mode (the non-disjoint case of §2),
against facts that do not come from the oracle's own formulas: the greedy set formation
re-derived with an independent GF(2) rank, the lower bound checked against brute-force
minimum supports (never above them; equal in the cases with a closed form), d against
brute force on random codes with n < 2k, and planted wrong bounds that the brute-force
comparison catches."""

import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from test_oracle_pins import _gf2_rank, _random_full_rank


def _family_min_support(sets, need, n):
    """Least |X|, X a subset of range(n), with |X & S_j| >= need[j] for every j (brute force)."""
    for w in range(n + 1):
        for X in itertools.combinations(range(n), w):
            xs = set(X)
            if all(len(xs & S) >= t for S, t in zip(sets, need)):
                return w
    return n + 1


@pytest.mark.parametrize("seed", range(12))
def test_partition_overlap_properties(seed):
    rng = synth.SplitMix64(4000 + seed)
    k = rng.uniform_int(2, 10)
    n = rng.uniform_int(k + 1, 2 * k)
    M = rng.uniform_int(2, 5)
    bits = _random_full_rank(n, k, 90 + seed)
    G = synth.pack_bits(bits)
    p = oracle.partition_overlap(G, n, M)
    cover = [0] * n
    for j in range(M):
        piv = [int(c) for c in p["pivcols"][j]]
        # greedy over the columns ordered by (cover so far, index): a column is taken iff
        # it is independent of those already taken
        order = sorted(range(n), key=lambda c: (cover[c], c))
        chosen = []
        for c in order:
            if _gf2_rank(bits[:, chosen + [c]]) > len(chosen):
                chosen.append(c)
            if len(chosen) == k:
                break
        assert chosen == piv
        assert int(p["ranks"][j]) == sum(1 for c in piv if cover[c] == 0)
        # Gamma_j = T_j G, the identity on the pivots (row i has its 1 on pivot i)
        T = synth.unpack_bits(p["transforms"][j][:, None], 64)[:, :k]
        assert _gf2_rank(T) == k
        gam = synth.unpack_bits(p["gammas"][j], n)
        assert np.array_equal(gam, (T.astype(np.int64) @ bits.astype(np.int64)) % 2)
        assert np.array_equal(gam[:, piv], np.eye(k, dtype=np.uint8))
        for c in piv:
            cover[c] += 1
    assert list(p["cover"]) == cover


def _random_family(rng, n, k, m):
    sets = []
    for _ in range(m):
        cols = list(range(n))
        for i in range(n - 1, 0, -1):  # Fisher-Yates with the seeded stream
            j = rng.uniform_int(0, i)
            cols[i], cols[j] = cols[j], cols[i]
        sets.append(sorted(cols[:k]))
    return sets


def _rel_and_cover(sets, n):
    cover = [0] * n
    rel = []
    for S in sets:
        rel.append(sum(1 for c in S if cover[c] == 0))
        for c in S:
            cover[c] += 1
    return rel, cover


@pytest.mark.parametrize("seed", range(40))
def test_bound_never_exceeds_the_least_support(seed):
    # any codeword not yet seen has >= h_j + 1 ones in every S_j, so the bound must not
    # exceed the least size of such a support (found here by brute force)
    rng = synth.SplitMix64(5000 + seed)
    n = rng.uniform_int(4, 11)
    k = rng.uniform_int(2, n - 1)
    m = rng.uniform_int(2, 4)
    sets = _random_family(rng, n, k, m)
    rel, cover = _rel_and_cover(sets, n)
    for _ in range(4):
        h = [rng.uniform_int(0, k - 1) for _ in range(m)]
        L = oracle.overlap_bound(h, k, rel, cover)
        best = _family_min_support([set(S) for S in sets], [t + 1 for t in h], n)
        assert L <= best, (sets, h, L, best)


@pytest.mark.parametrize("h", range(0, 5))
def test_bound_closed_forms(h):
    # disjoint sets (each position covered once): the least support is sum_j (h + 1)
    k, m = 5, 3
    sets = [list(range(j * k, (j + 1) * k)) for j in range(m)]
    rel, cover = _rel_and_cover(sets, m * k)
    assert oracle.overlap_bound([h] * m, k, rel, cover) == m * (h + 1)
    # three sets A+B, C+A, B+C over blocks of k/2 positions (every position covered
    # twice): the least support is ceil(3 (h + 1) / 2) while the relative ranks give
    # (h + 1) + max(0, h + 1 - k/2)
    k = 8
    A, B, C = list(range(0, 4)), list(range(4, 8)), list(range(8, 12))
    sets = [A + B, C + A, B + C]
    rel, cover = _rel_and_cover(sets, 12)
    want = _family_min_support([set(S) for S in sets], [h + 1] * 3, 12)
    assert want == math.ceil(3 * (h + 1) / 2)
    assert oracle.overlap_bound([h] * 3, k, rel, cover) == want


def _overlap_codes():
    out = []
    for seed in range(240):
        rng = synth.SplitMix64(9100 + seed)
        k = rng.uniform_int(3, 18)
        n = rng.uniform_int(k + 1, 2 * k - 1) if seed % 6 else rng.uniform_int(2 * k, 3 * k)
        M = rng.uniform_int(2, 5)
        out.append((n, k, M, synth.random_systematic(n, k, seed)))
    return out


@pytest.mark.parametrize("per_matrix", [False, True])
def test_overlap_bz_equals_bruteforce(per_matrix):
    saved = 0
    for n, k, M, G in _overlap_codes():
        d = oracle.brute_force_distance(G, n, nthreads=2)
        r = oracle.min_distance(G, n, overlap_sets=M, check_per_matrix=per_matrix, nthreads=2)
        assert r["d"] == d == r["key"][0], (n, k, M)
        msg = np.array([(r["message"] >> b) & 1 for b in range(k)], dtype=np.int64)
        cw = (msg @ synth.unpack_bits(G, n).astype(np.int64)) % 2
        assert np.array_equal(cw.astype(np.uint8), synth.unpack_bits(r["witness"][None, :], n)[0])
        assert r["m"] == M and r["L_final"] >= d or r["g_final"] == k
        g_end = r["g_final"]
        for g in range(1, k + 1):
            for j in range(M):
                done = g < g_end or (g == g_end and (not per_matrix or j <= r["j_final"]))
                assert int(r["counts"][g][j]) == (math.comb(k, g) if done else 0)
        if not per_matrix and n < 2 * k:
            saved += int(oracle.min_distance(G, n, nthreads=2)["counts"].sum()) - int(r["counts"].sum())
    if not per_matrix:
        assert saved > 0  # the mode pays off on codes with n < 2k


def _replay(G, n, k, M, bound):
    """Alg. 1 over the oracle's overlapping sets with a given bound(levels, part)."""
    part = oracle.partition_overlap(G, n, M)
    U, L, g = n - k + 1, 1, 1
    while g <= k and L < U:
        for j in range(M):
            U = min(U, oracle.enumerate_unit(part["gammas"][j], n, g, want_hist=False)["min_w"])
        L = bound([g] * M, part)
        g += 1
    return U


@pytest.mark.parametrize("plant", ["coverage_ignored", "off_by_one"])
def test_planted_bound_mistakes_are_caught(plant):
    def wrong(levels, part):
        if plant == "coverage_ignored":  # the sets counted as if they were disjoint
            return sum(h + 1 for h in levels)
        return oracle.overlap_bound(levels, k, part["ranks"], part["cover"]) + 1

    caught = 0
    for n, k, M, G in _overlap_codes()[:120]:
        if _replay(G, n, k, M, wrong) != oracle.brute_force_distance(G, n, nthreads=2):
            caught += 1
    assert caught > 0

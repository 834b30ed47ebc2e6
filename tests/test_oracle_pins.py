"""Pins of the CPU oracle against facts that do not come from the oracle itself:
textbook weight enumerators, the MacWilliams identity, brute force on tiny inputs,
the paper's printed combination-order examples, closed-form counts and invariants."""

import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import golden_path


def _read_enumerators():
    out = {}
    with open(golden_path("textbook_weight_enumerators.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, tail = line.split("|")
            name, n, k, d = head.split()
            A = {int(a.split(":")[0]): int(a.split(":")[1]) for a in tail.split()}
            out[name] = (int(n), int(k), int(d), A)
    return out


TEXTBOOK = {
    "hamming_7_4": synth.hamming_7_4,
    "golay_24_12": synth.golay_24_12,
    "rm_1_5": synth.reed_muller_1_5,
    "repetition_5": lambda: synth.repetition(5),
    "even_weight_4": lambda: synth.even_weight(4),
}


@pytest.mark.parametrize("name", list(TEXTBOOK))
def test_textbook_weight_enumerator(name):
    n, k, d, A = _read_enumerators()[name]
    G = TEXTBOOK[name]()
    assert G.shape[0] == k
    got = oracle.weight_enumerator(G, n, nthreads=3)
    want = np.zeros(n + 1, dtype=np.uint64)
    for w, c in A.items():
        want[w] = c
    assert np.array_equal(got, want)
    assert oracle.brute_force_distance(G, n) == d


@pytest.mark.parametrize("name", list(TEXTBOOK))
@pytest.mark.parametrize("per_matrix", [False, True])
def test_textbook_bz_distance(name, per_matrix):
    n, k, d, _ = _read_enumerators()[name]
    G = TEXTBOOK[name]()
    r = oracle.min_distance(G, n, check_per_matrix=per_matrix, nthreads=2)
    assert r["d"] == d
    assert r["key"][0] == d
    w = synth.unpack_bits(r["witness"][None, :], n)[0]
    assert int(w.sum()) == d


def test_singleton_edge_witness():
    # [5,1,5]: d = n-k+1, the initial U; the witness must still be set (at unit (1, 0))
    r = oracle.min_distance(synth.repetition(5), 5)
    assert r["d"] == 5 and r["key"] == (5, 1, 0, 0) and r["message"] == 1
    assert r["m"] == 5 and r["ranks"] == [1] * 5


def _krawtchouk(j, i, n):
    return sum((-1) ** s * math.comb(i, s) * math.comb(n - i, j - s) for s in range(0, j + 1))


def _dual_of_systematic(n, k, seed):
    R = synth.random_redundancy(n, k, seed)
    H = np.concatenate([R.T, np.eye(n - k, dtype=np.uint8)], axis=1)
    return synth.pack_bits(H)


@pytest.mark.parametrize("seed", range(8))
def test_macwilliams_identity(seed):
    rng = synth.SplitMix64(100 + seed)
    k = rng.uniform_int(2, 9)
    n = rng.uniform_int(k + 1, min(2 * k + 4, 18))
    G = synth.random_systematic(n, k, seed)
    H = _dual_of_systematic(n, k, seed)
    A = [int(a) for a in oracle.weight_enumerator(G, n, nthreads=2)]
    B = [int(b) for b in oracle.weight_enumerator(H, n, nthreads=2)]
    for j in range(n + 1):
        s = sum(A[i] * _krawtchouk(j, i, n) for i in range(n + 1))
        assert s == B[j] * (1 << k)


def test_bruteforce_thread_independent():
    G = synth.random_systematic(40, 20, 7)
    a1 = oracle.weight_enumerator(G, 40, nthreads=1)
    a7 = oracle.weight_enumerator(G, 40, nthreads=7)
    assert np.array_equal(a1, a7)
    assert int(a1.sum()) == 1 << 20


def _np_weights_of_combos(gamma_bits, combos):
    return [int(np.bitwise_xor.reduce(gamma_bits[list(c)], axis=0).sum()) for c in combos]


@pytest.mark.parametrize("seed", range(6))
def test_unit_vs_itertools(seed):
    rng = synth.SplitMix64(seed)
    k = rng.uniform_int(3, 10)
    n = rng.uniform_int(k + 1, 3 * k)
    gamma = synth.random_systematic(n, k, 50 + seed)
    bits = synth.unpack_bits(gamma, n)
    for g in range(1, k + 1):
        combos = list(itertools.combinations(range(k), g))  # lexicographic order
        ws = _np_weights_of_combos(bits, combos)
        r = oracle.enumerate_unit(gamma, n, g, nthreads=3)
        assert r["count"] == len(combos) == math.comb(k, g)
        assert r["min_w"] == min(ws)
        assert r["min_rank"] == ws.index(min(ws))
        hist = np.bincount(ws, minlength=n + 1)
        assert np.array_equal(r["hist"], hist.astype(np.uint64))
        xa = np.zeros(n, dtype=np.uint8)
        for c in combos:
            xa ^= np.bitwise_xor.reduce(bits[list(c)], axis=0)
        assert np.array_equal(synth.unpack_bits(r["xor_all"][None, :], n)[0], xa)


@pytest.mark.parametrize("k,g", [(20, 5), (24, 7), (30, 4), (17, 8)])
def test_xor_parity_invariant(k, g):
    # every row lies in C(k-1, g-1) of the C(k, g) combinations
    n = 3 * k
    gamma = synth.random_systematic(n, k, k * 31 + g)
    r = oracle.enumerate_unit(gamma, n, g, nthreads=4, want_hist=False)
    par = math.comb(k - 1, g - 1) % 2
    want = np.bitwise_xor.reduce(gamma, axis=0) if par else np.zeros(gamma.shape[1], dtype=np.uint64)
    assert np.array_equal(r["xor_all"], want)
    assert r["count"] == math.comb(k, g)


@pytest.mark.parametrize("seed", range(5))
def test_unit_histograms_sum_to_enumerator(seed):
    # each nonzero codeword is c * Gamma_1 for exactly one nonzero c (Gamma_1 invertible
    # transform of G), so the level histograms of Gamma_1 add up to the weight enumerator
    k, n = 12, 30
    G = synth.random_systematic(n, k, 200 + seed)
    A = oracle.weight_enumerator(G, n)
    part = oracle.partition(G, n)
    tot = np.zeros(n + 1, dtype=np.uint64)
    tot[0] = 1
    for g in range(1, k + 1):
        tot += oracle.enumerate_unit(part["gammas"][0], n, g)["hist"]
    assert np.array_equal(tot, A)


def _gf2_rank(bits):
    m = bits.copy() % 2
    r = 0
    rows, cols = m.shape
    for c in range(cols):
        piv = [i for i in range(r, rows) if m[i, c]]
        if not piv:
            continue
        m[[r, piv[0]]] = m[[piv[0], r]]
        for i in range(rows):
            if i != r and m[i, c]:
                m[i] ^= m[r]
        r += 1
        if r == rows:
            break
    return r


def _random_full_rank(n, k, seed):
    rng = synth.SplitMix64(seed)
    while True:
        bits = np.array([[rng.next() & 1 for _ in range(n)] for _ in range(k)], dtype=np.uint8)
        if _gf2_rank(bits) == k:
            return bits


@pytest.mark.parametrize("seed", range(10))
def test_partition_properties(seed):
    rng = synth.SplitMix64(1000 + seed)
    k = rng.uniform_int(2, 12)
    n = rng.uniform_int(k + 1, 5 * k)
    bits = _random_full_rank(n, k, seed)
    G = synth.pack_bits(bits)
    p = oracle.partition(G, n)
    used = set()
    for j in range(p["m"]):
        r = int(p["ranks"][j])
        piv = [int(c) for c in p["pivcols"][j][:r]]
        assert not (set(piv) & used)
        # greedy: scanning unused columns in ascending order, a column is a pivot iff it
        # is independent of the pivots already chosen for this set
        chosen = []
        for c in range(n):
            if c in used:
                continue
            if _gf2_rank(bits[:, chosen + [c]]) > len(chosen):
                chosen.append(c)
            if len(chosen) == k:
                break
        assert chosen == piv
        T = synth.unpack_bits(p["transforms"][j][:, None], 64)[:, :k]
        assert _gf2_rank(T) == k
        gam = synth.unpack_bits(p["gammas"][j], n)
        assert np.array_equal(gam, (T.astype(np.int64) @ bits.astype(np.int64)) % 2)
        # identity on the pivot columns, zeros below rank
        sub = gam[:, piv]
        want = np.zeros((k, r), dtype=np.uint8)
        want[:r, :r] = np.eye(r, dtype=np.uint8)
        assert np.array_equal(sub, want)
        used |= set(piv)
    # sets stop when no columns are left or the leftover columns have rank 0
    rest = [c for c in range(n) if c not in used]
    assert p["m"] == oracle.MAX_SETS or not rest or _gf2_rank(bits[:, rest]) == 0


def test_partition_systematic_first_set():
    G = synth.random_systematic(90, 30, 3)
    p = oracle.partition(G, 90)
    assert list(p["pivcols"][0]) == list(range(30))


def _bound(g, k, ranks):
    return sum(max(0, g + 1 - (k - r)) for r in ranks)


@pytest.mark.parametrize("seed", range(300))
def test_bz_equals_bruteforce_random(seed):
    rng = synth.SplitMix64(7000 + seed)
    k = rng.uniform_int(1, 16)
    n = rng.uniform_int(k + 1, 4 * k + 1)
    G = synth.random_systematic(n, k, seed)
    d = oracle.brute_force_distance(G, n, nthreads=2)
    for per_matrix in (False, True):
        r = oracle.min_distance(G, n, check_per_matrix=per_matrix, nthreads=2)
        assert r["d"] == d
        assert r["key"][0] == d
        # witness is the codeword of the message, of weight d
        msg_bits = np.array([(r["message"] >> b) & 1 for b in range(k)], dtype=np.int64)
        cw = (msg_bits @ synth.unpack_bits(G, n).astype(np.int64)) % 2
        assert np.array_equal(cw.astype(np.uint8), synth.unpack_bits(r["witness"][None, :], n)[0])
        assert int(cw.sum()) == d
        # termination: bound reached (or every level done), counts are C(k, g) up to the end
        g_end = r["g_final"]
        assert r["L_final"] >= d or g_end == k
        if not per_matrix:
            assert r["L_final"] == _bound(g_end, k, r["ranks"])
        for g in range(1, k + 1):
            for j in range(r["m"]):
                done = g < g_end or (g == g_end and (not per_matrix or j <= r["j_final"]))
                assert int(r["counts"][g][j]) == (math.comb(k, g) if done else 0)


def test_key_is_least_over_units():
    # the key is the least (weight, g, j, rank) over every unit enumerated
    n, k = 40, 14
    G = synth.random_systematic(n, k, 77)
    r = oracle.min_distance(G, n)
    part = oracle.partition(G, n)
    best = None
    for g in range(1, r["g_final"] + 1):
        for j in range(part["m"]):
            u = oracle.enumerate_unit(part["gammas"][j], n, g)
            cand = (u["min_w"], g, j, u["min_rank"])
            best = cand if best is None or cand < best else best
    assert best == r["key"]


def test_golden_combination_order():
    with open(golden_path("paper_combination_order.txt")) as f:
        rows = [ln for ln in f if ln.strip() and not ln.startswith("#")]
    for ln in rows:
        head, tail = ln.split("|")
        k, g, rank = (int(x) for x in head.split())
        elems = [int(x) for x in tail.split()]
        mask = oracle.unrank_lex(k, g, rank)
        assert [b for b in range(k) if (mask >> b) & 1] == elems


def test_unrank_lex_vs_itertools():
    for k in range(1, 11):
        for g in range(1, k + 1):
            for rank, c in enumerate(itertools.combinations(range(k), g)):
                assert oracle.unrank_lex(k, g, rank) == sum(1 << e for e in c)


def test_lexrank_closed_form():
    # rank(c_1<...<c_g) = C(k,g) - 1 - sum_i C(k-1-c_i, g-i+1); written out independently
    for k in range(1, 12):
        for g in range(1, k + 1):
            for rank, c in enumerate(itertools.combinations(range(k), g)):
                f = math.comb(k, g) - 1 - sum(math.comb(k - 1 - ci, g - i) for i, ci in enumerate(c))
                assert f == rank


def test_binomials():
    for a in range(0, 65):
        for b in range(0, a + 1):
            assert oracle.binomial(a, b) == math.comb(a, b)


def test_planted_mistake_is_caught():
    # A wrong lower bound (off by one per set) must make BZ stop early on some code and
    # disagree with brute force: shows the random-code comparison has teeth.
    caught = False
    for seed in range(60):
        rng = synth.SplitMix64(seed)
        k = rng.uniform_int(4, 12)
        n = rng.uniform_int(2 * k, 4 * k)
        G = synth.random_systematic(n, k, seed)
        d = oracle.brute_force_distance(G, n)
        part = oracle.partition(G, n)
        # plant: L(g) computed with g+2 instead of g+1, replayed in Python on the oracle's units
        U, L, g = n - k + 1, 1, 1
        while g <= k and L < U:
            for j in range(part["m"]):
                U = min(U, oracle.enumerate_unit(part["gammas"][j], n, g, want_hist=False)["min_w"])
            L = sum(max(0, g + 2 - (k - r)) for r in part["ranks"])
            g += 1
        if U != d:
            caught = True
            break
    assert caught


def _skip_codes():
    # rate > 1/2: the greedy sets after the first are partial, so some sets are idle at
    # the low levels
    out = []
    for seed in range(1, 241):
        n, k = 30 + seed % 9, 20
        out.append((n, k, synth.random_systematic(n, k, seed)))
    return out


def test_skip_idle_sets_equals_bruteforce():
    # the mode that leaves idle sets out (and lets them catch up) reaches the same d as
    # the plain definition, enumerates each set's levels as a prefix 1..h_j, and its key
    # is a codeword of weight d
    saved = 0
    for n, k, G in _skip_codes():
        d = oracle.brute_force_distance(G, n)
        r = oracle.min_distance(G, n, skip_idle_sets=True)
        full = oracle.min_distance(G, n)
        assert r["d"] == d == full["d"]
        assert r["key"][0] == d
        cw = synth.unpack_bits(r["witness"][None, :], n)[0]
        assert int(cw.sum()) == d
        msg = np.array([(r["message"] >> b) & 1 for b in range(k)], dtype=np.int64)
        assert np.array_equal((msg @ synth.unpack_bits(G, n).astype(np.int64)) % 2, cw.astype(np.int64))
        for j in range(r["m"]):
            col = [int(x) for x in r["counts"][1:, j]]
            h = sum(1 for x in col if x)
            assert all(col[g - 1] == math.comb(k, g) for g in range(1, h + 1)), (j, col)
            assert all(x == 0 for x in col[h:])
        saved += int(full["counts"].sum()) - int(r["counts"].sum())
    assert saved > 0


def test_skip_without_catch_up_is_caught():
    # planted mistake: idle sets left out but never caught up; the comparison with brute
    # force has to catch it on some code of the same family
    caught = 0
    for n, k, G in _skip_codes():
        part = oracle.partition(G, n)
        ranks = [int(x) for x in part["ranks"]]
        U, L, g = n - k + 1, 1, 1
        while g <= k and L < U:
            for j in range(part["m"]):
                if max(0, g + 1 - (k - ranks[j])) > 0:
                    U = min(U, oracle.enumerate_unit(part["gammas"][j], n, g, want_hist=False)["min_w"])
            L = sum(max(0, g + 1 - (k - r)) for r in ranks)
            if L >= U:
                break
            g += 1
        if U != oracle.brute_force_distance(G, n):
            caught += 1
    assert caught > 0

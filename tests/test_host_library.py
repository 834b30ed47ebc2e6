"""CPU tests of libmdist.so without a GPU: it loads, exports every entry point the
header declares, and its host logic (information sets, row layout, the kernels'
combination indexing and level plan) matches independent computations."""

import ctypes
import itertools
import math
import os
import re

import numpy as np
import pytest

import oracle
import synth
from conftest import ROOT
from paper_1603_06757_gb300 import _lib as L

P64 = L.P64


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build_library()
    return L.lib()


def test_header_symbols_exported(lib):
    hdr = open(os.path.join(ROOT, "include", "mdist.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"\b(mdist_[a-z_0-9]+)\s*\(", hdr))
    declared -= {"mdist_alloc_fn", "mdist_free_fn"}
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(lib, name), name
        assert name in L.SIGNATURES, name
    assert set(L.SIGNATURES) == declared


def _partition_lib(lib, G, n):
    k, W = G.shape
    m = ctypes.c_int()
    ranks = np.zeros(64, dtype=np.int32)
    piv = np.zeros(64 * k, dtype=np.int32)
    gam = np.zeros(64 * k * W, dtype=np.uint64)
    tr = np.zeros(64 * k, dtype=np.uint64)
    rc = lib.mdist_partition_host(G.ctypes.data_as(P64), n, k, W, 0, ctypes.byref(m), ranks.ctypes.data_as(L.PI),
                                  piv.ctypes.data_as(L.PI32), gam.ctypes.data_as(P64), tr.ctypes.data_as(P64))
    if rc != 0:
        raise L.MdistError(rc, "partition")
    mm = m.value
    return mm, ranks[:mm], piv.reshape(64, k)[:mm], gam.reshape(64, k, W)[:mm], tr.reshape(64, k)[:mm]


def _random_full_rank(n, k, seed):
    rng = synth.SplitMix64(seed)
    for _ in range(1000):
        bits = np.array([[rng.next() & 1 for _ in range(n)] for _ in range(k)], dtype=np.uint8)
        G = synth.pack_bits(bits)
        try:
            oracle.partition(G, n)
            return G
        except ValueError:
            continue
    raise RuntimeError


CODES = [
    ("hamming", synth.hamming_7_4(), 7),
    ("golay", synth.golay_24_12(), 24),
    ("rm15", synth.reed_muller_1_5(), 32),
    ("rep5", synth.repetition(5), 5),
    ("even4", synth.even_weight(4), 4),
    ("s1", synth.random_systematic(60, 30, 1), 60),
    ("s3a", synth.random_systematic(150, 64, 1), 150),
    ("s3b", synth.random_systematic(300, 50, 1), 300),
    ("n512", synth.random_systematic(512, 64, 5), 512),
]


@pytest.mark.parametrize("name,G,n", CODES, ids=[c[0] for c in CODES])
def test_partition_matches_oracle(lib, name, G, n):
    m, ranks, piv, gam, tr = _partition_lib(lib, G, n)
    o = oracle.partition(G, n)
    assert m == o["m"]
    assert np.array_equal(ranks, o["ranks"])
    assert np.array_equal(piv, o["pivcols"])
    assert np.array_equal(gam, o["gammas"])
    assert np.array_equal(tr, o["transforms"])


@pytest.mark.parametrize("seed", range(40))
def test_partition_matches_oracle_random(lib, seed):
    rng = synth.SplitMix64(500 + seed)
    k = rng.uniform_int(1, 24)
    n = rng.uniform_int(k + 1, min(512, 6 * k + 2))
    G = _random_full_rank(n, k, seed) if seed % 2 else synth.random_systematic(n, k, seed)
    m, ranks, piv, gam, tr = _partition_lib(lib, G, n)
    o = oracle.partition(G, n)
    assert m == o["m"] and np.array_equal(ranks, o["ranks"]) and np.array_equal(piv, o["pivcols"])
    assert np.array_equal(gam, o["gammas"]) and np.array_equal(tr, o["transforms"])


def test_partition_rank_deficient(lib):
    bits = np.zeros((3, 10), dtype=np.uint8)
    bits[0, :5] = 1
    bits[1, :5] = 1  # duplicate row
    bits[2, 5:] = 1
    G = synth.pack_bits(bits)
    with pytest.raises(L.MdistError) as e:
        _partition_lib(lib, G, 10)
    assert e.value.code == L.ERANK


@pytest.mark.parametrize("name,G,n", CODES, ids=[c[0] for c in CODES])
def test_row_layout_preserves_weight(lib, name, G, n):
    k, W = G.shape
    m, ranks, piv, gam, tr = _partition_lib(lib, G, n)
    rng = np.random.default_rng(0)
    for j in range(m):
        full = ctypes.c_int()
        nb = ctypes.c_int()
        nw = ctypes.c_int()
        words = np.zeros(k * 16, dtype=np.uint32)
        rc = lib.mdist_debug_set_rows(G.ctypes.data_as(P64), n, k, W, j, ctypes.byref(full), ctypes.byref(nb),
                                      ctypes.byref(nw), words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
        assert rc == 0
        assert bool(full.value) == (ranks[j] == k)
        assert nb.value == (n - k if full.value else n)
        rows = words[: k * nw.value].reshape(k, nw.value)
        gbits = synth.unpack_bits(gam[j], n)
        for _ in range(40):
            c = rng.integers(0, 2, size=k).astype(bool)
            if not c.any():
                continue
            cw = np.bitwise_xor.reduce(gbits[c], axis=0)
            red = np.bitwise_xor.reduce(rows[c], axis=0)
            rw = sum(bin(int(v)).count("1") for v in red)
            base = int(c.sum()) if full.value else 0
            assert base + rw == int(cw.sum())


def test_unrank_colex_and_successor(lib):
    out = ctypes.c_uint32()
    for kh in range(0, 11):
        for t in range(0, kh + 1):
            masks = sorted(sum(1 << e for e in c) for c in itertools.combinations(range(kh), t))
            for r, mk in enumerate(masks):
                assert lib.mdist_debug_unrank_colex(kh, t, r, ctypes.byref(out)) == 0
                assert out.value == mk
                if t and r + 1 < len(masks):
                    assert lib.mdist_debug_next_colex(mk, ctypes.byref(out)) == 0
                    assert out.value == masks[r + 1]


def _colex_unrank_py(kh, t, r):
    mask = 0
    for i in range(t, 0, -1):
        c = i - 1
        while math.comb(c + 1, i) <= r:
            c += 1
        mask |= 1 << c
        r -= math.comb(c, i)
    return mask


def test_unrank_colex_large_halves(lib):
    out = ctypes.c_uint32()
    rng = synth.SplitMix64(9)
    for _ in range(3000):
        kh = rng.uniform_int(20, 32)
        t = rng.uniform_int(1, kh)
        r = rng.uniform_int(0, math.comb(kh, t) - 1)
        assert lib.mdist_debug_unrank_colex(kh, t, r, ctypes.byref(out)) == 0
        assert out.value == _colex_unrank_py(kh, t, r)
        if r + 1 < math.comb(kh, t):
            nxt = ctypes.c_uint32()
            assert lib.mdist_debug_next_colex(out.value, ctypes.byref(nxt)) == 0
            assert nxt.value == _colex_unrank_py(kh, t, r + 1)


def test_lexrank_vs_itertools(lib):
    out = ctypes.c_uint64()
    for k in range(1, 12):
        for g in range(1, k + 1):
            for rank, c in enumerate(itertools.combinations(range(k), g)):
                assert lib.mdist_debug_lexrank(sum(1 << e for e in c), k, g, ctypes.byref(out)) == 0
                assert out.value == rank


def test_lexrank_k64_vs_oracle_unrank(lib):
    out = ctypes.c_uint64()
    rng = synth.SplitMix64(11)
    for _ in range(2000):
        k = rng.uniform_int(30, 64)
        g = rng.uniform_int(1, 14)
        r = rng.uniform_int(0, min(math.comb(k, g), 1 << 54) - 1)
        mask = oracle.unrank_lex(k, g, r)
        assert lib.mdist_debug_lexrank(mask, k, g, ctypes.byref(out)) == 0
        assert out.value == r


def _plan(lib, k, g, nw):
    nb = ctypes.c_int()
    blocks = np.zeros(34 * 7, dtype=np.uint64)
    tt = ctypes.c_uint64()
    lc = ctypes.c_int()
    wc = ctypes.c_int()
    rc = lib.mdist_debug_level_plan(k, g, nw, ctypes.byref(nb), blocks.ctypes.data_as(P64), ctypes.byref(tt),
                                    ctypes.byref(lc), ctypes.byref(wc))
    return rc, blocks.reshape(34, 7)[: nb.value], tt.value, lc.value, wc.value


@pytest.mark.parametrize("k", [1, 2, 5, 17, 30, 31, 50, 63, 64])
@pytest.mark.parametrize("nw", [1, 4, 5, 8, 16])
def test_level_plan_covers_level(lib, k, nw):
    k1 = (k + 1) // 2
    k2 = k - k1
    for g in range(1, k + 1):
        rc, blocks, tt, lc, wc = _plan(lib, k, g, nw)
        if math.comb(k, g) >= 1 << 54:
            assert rc == L.ERANGE
            continue
        assert rc == 0
        total = 0
        tiles = 0
        seen_i = []
        for b in blocks:
            half, lt, wt, ln, wn, wch, tb = (int(v) for v in b)
            assert lt + wt == g
            i = lt if half == 0 else wt
            seen_i.append(i)
            assert ln == math.comb(k1 if half == 0 else k2, lt)
            assert wn == math.comb(k2 if half == 0 else k1, wt)
            assert ln >= wn
            assert wch == -(-wn // wc)
            assert tb == tiles
            tiles += -(-ln // lc) * wch
            total += ln * wn
        assert seen_i == list(range(max(0, g - k2), min(g, k1) + 1))
        assert total == math.comb(k, g)  # Vandermonde: the blocks partition the level
        assert tt == tiles


def _choice(lib, nw, nb, thr):
    g = ctypes.c_int()
    assert lib.mdist_debug_filter_choice(nw, nb, thr, ctypes.byref(g)) == 0
    return g.value


def test_filter_choice(lib):
    # threshold at or above the row width: every codeword is a candidate -> exact
    assert _choice(lib, 4, 128, 128) == 0
    # one word: nothing to group
    assert _choice(lib, 1, 20, 3) == 0
    # the last levels of [192,64] (reduced weight <= 24 of 128 bits): groups of 4, then 2
    assert _choice(lib, 4, 128, 24) == 5
    assert _choice(lib, 4, 128, 28) == 2
    assert _choice(lib, 4, 128, 12) == 4
    # threshold near the mean of a random codeword: the bound rarely rejects -> exact
    assert _choice(lib, 4, 128, 62) == 0
    # [300,50]-like rows (250 bits, threshold ~67): pairs of words
    assert _choice(lib, 8, 250, 67) in (2, 3)

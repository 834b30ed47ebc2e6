"""The tensor-core enumerator's subset-sum tables (mdist_debug_side_tables, the kernel the
enumerator builds its A and B sides with), entry by entry against their definition:
entry e is the XOR of the rows of the component-0 subset of colex rank e mod C(kc0, t0)
(rows off0 + its elements) and of the component-1 subset of colex rank e div C(kc0, t0).
Colex order (§3.1's enumeration reads subsets in this order inside a half) is generated
here by sorting itertools' subsets on their largest element first, an independent route
to the same order.  Every row width 1..8 words, one- and two-component sides, empty and
full subsets, several sides per launch (sharing and not sharing the low-subset table), sides
whose low-subset sums come from a table of an earlier launch (the way the library
builds later levels), and full-size sides (28 million entries) on sampled entries."""

import itertools
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_1603_06757_gb300 import api

    return api


def colex(kc, t):
    """All t-subsets of range(kc) in colex order, one row each (elements ascending)."""
    if t == 0:
        return np.zeros((1, 0), dtype=np.int64)
    c = np.array(list(itertools.combinations(range(kc), t)), dtype=np.int64)
    order = np.lexsort(tuple(c[:, i] for i in range(t)))  # last key (largest element) first
    return c[order]


def expected(rows, side):
    off0, kc0, t0, off1, kc1, t1 = side
    nw = rows.shape[1]
    c0 = colex(kc0, t0)
    x0 = np.zeros((len(c0), nw), dtype=np.uint32)
    for i in range(t0):
        x0 ^= rows[off0 + c0[:, i]]
    if t1 < 0:
        return x0
    c1 = colex(kc1, t1)
    x1 = np.zeros((len(c1), nw), dtype=np.uint32)
    for i in range(t1):
        x1 ^= rows[off1 + c1[:, i]]
    return (x1[:, None, :] ^ x0[None, :, :]).reshape(-1, nw)  # component 0 fastest


def rows_for(k, nw, seed):
    return np.random.default_rng(seed).integers(0, 2**32, size=(k, nw), dtype=np.uint64).astype(np.uint32)


ONE = [(0, 1, 0), (0, 1, 1), (3, 5, 2), (0, 5, 5), (32, 32, 0), (32, 32, 1), (32, 32, 2), (0, 32, 3),
       (0, 32, 4), (32, 32, 5), (16, 16, 8), (48, 16, 16), (7, 20, 6)]


@pytest.mark.parametrize("nw", [1, 2, 3, 4, 5, 6, 7, 8])
def test_one_component_sides(api, nw):
    rows = rows_for(64, nw, 100 + nw)
    sides = [(o, kc, t, 0, 0, -1) for (o, kc, t) in ONE]
    got = api.side_tables(rows, sides)
    for side, g in zip(sides, got):
        assert np.array_equal(g, expected(rows, side)), side


TWO = [(0, 16, 0, 16, 16, 3), (0, 16, 1, 16, 16, 2), (0, 16, 2, 16, 16, 2), (0, 16, 3, 16, 16, 1),
       (0, 16, 4, 16, 16, 3), (32, 16, 5, 48, 16, 0), (40, 13, 5, 3, 9, 2), (0, 5, 5, 5, 6, 6), (10, 6, 0, 20, 6, 0)]


@pytest.mark.parametrize("nw", [1, 4, 7, 8])
def test_two_component_sides(api, nw):
    rows = rows_for(64, nw, 200 + nw)
    got = api.side_tables(rows, TWO)
    for side, g in zip(TWO, got):
        assert np.array_equal(g, expected(rows, side)), side


def test_many_sides_one_launch(api):
    """A launch of 40 sides in shuffled order: sides with the same low-subset table
    (same component-0 rows, t0 >= 3) share one build, the others rebuild it."""
    rows = rows_for(64, 4, 7)
    rng = np.random.default_rng(3)
    sides = []
    for _ in range(40):
        off0 = int(rng.choice([0, 16, 32]))
        kc0 = int(rng.choice([16, 32]))
        t0 = int(rng.integers(0, 6))
        if rng.random() < 0.4:
            sides.append((off0, kc0, t0, 0, 0, -1))
        else:
            off1 = 48 if off0 + kc0 <= 48 else 0  # rows apart from component 0's
            sides.append((off0, kc0, t0, off1, 16, int(rng.integers(0, 3))))
    got = api.side_tables(rows, sides)
    for side, g in zip(sides, got):
        assert np.array_equal(g, expected(rows, side)), side


def _unrank_colex(kc, t, r):
    out = []
    c = kc - 1
    for i in range(t, 0, -1):
        while math.comb(c, i) > r:
            c -= 1
        out.append(c)
        r -= math.comb(c, i)
        c -= 1
    return out


@pytest.mark.parametrize("nw", [1, 3, 4, 8])
def test_sides_from_earlier_tables(api, nw):
    """The low-subset sums read from the table of a one-component side (off0, kc0, u)
    built by an earlier launch, u from 1 to t0 - 1, for one- and two-component sides."""
    rows = rows_for(64, nw, 300 + nw)
    sides, lows = [], []
    for (off0, kc0, u) in [(0, 32, 4), (32, 32, 5), (16, 16, 4), (0, 20, 6), (0, 16, 1), (32, 32, 3), (48, 16, 2)]:
        sides.append((off0, kc0, u, 0, 0, -1))
        lows.append(None)
        base = len(sides) - 1
        for t0 in range(u + 1, min(kc0, u + 3) + 1):
            if math.comb(kc0, t0) > 1000000:
                continue
            sides.append((off0, kc0, t0, 0, 0, -1))
            lows.append(base)
            if off0 + kc0 <= 48:
                sides.append((off0, kc0, t0, 48, 16, 1))
                lows.append(base)
    got = api.side_tables(rows, sides, lows)
    for side, g in zip(sides, got):
        assert np.array_equal(g, expected(rows, side)), side


@pytest.mark.parametrize("side,low", [((0, 32, 9, 0, 0, -1), None), ((0, 32, 9, 0, 0, -1), 6),
                                      ((32, 32, 8, 0, 0, -1), 5), ((32, 16, 7, 0, 16, 5), None),
                                      ((32, 16, 7, 0, 16, 5), 4)])
def test_full_size_side_sampled(api, side, low):
    """28 million entries of a [192,64] level-11 side (and a two-component side of
    50 million), built in shared memory alone and from an earlier table, checked at
    sampled entries and at both ends."""
    rows = rows_for(64, 4, 11)
    if low is None:
        got = api.side_tables(rows, [side])[0]
    else:
        got = api.side_tables(rows, [(side[0], side[1], low, 0, 0, -1), side], [None, 0])[1]
    off0, kc0, t0, off1, kc1, t1 = side
    cnt0 = math.comb(kc0, t0)
    n = cnt0 * (math.comb(kc1, t1) if t1 >= 0 else 1)
    assert got.shape == (n, 4)
    rng = np.random.default_rng(5)
    for e in [0, 1, n - 1] + [int(v) for v in rng.integers(0, n, 3000)]:
        want = np.zeros(4, dtype=np.uint32)
        for c in _unrank_colex(kc0, t0, e % cnt0):
            want ^= rows[off0 + c]
        if t1 >= 0:
            for c in _unrank_colex(kc1, t1, e // cnt0):
                want ^= rows[off1 + c]
        assert np.array_equal(got[e], want), e

"""The entry point for callers that cannot allocate device memory
(mdist_enumerate_unit_noalloc) gives the same unit results as the allocating entry
points, call after call.

Collected last on purpose (file name), so a run that stops at the first failure has
already run every other test.  It works both alone in a fresh process and after the
other tests: the scratch array's device address is set up by the first call on the
device, and every call clears the scratch it needs."""

import ctypes
import math

import numpy as np
import pytest

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


def _rows_on_device(torch, G, n, j):
    """Gamma_j's enumerator rows, computed by the host-only entry point and placed in a
    caller-owned device tensor (the caller's memory, not the library's)."""
    from paper_1603_06757_gb300 import _lib as L

    k, W = G.shape
    full = ctypes.c_int()
    nb = ctypes.c_int()
    nw = ctypes.c_int()
    words = np.zeros(k * 16, dtype=np.uint32)
    rc = L.lib().mdist_debug_set_rows(G.ctypes.data_as(L.P64), n, k, W, j, ctypes.byref(full), ctypes.byref(nb),
                                      ctypes.byref(nw), words.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    assert rc == 0
    rows = torch.from_numpy(words[: k * nw.value].view(np.int32).copy()).cuda()
    return rows, full.value, nb.value, nw.value


def _call(torch, L, rows, k, nw, nb, full, g, U, want_hist):
    bins = (nb + (g if full else 0) + 1) if want_hist else 0
    out = torch.zeros(3 + bins, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = L.lib().mdist_enumerate_unit_noalloc(ctypes.c_void_p(rows.data_ptr()), k, nw, nb, full, g, U,
                                              1 if want_hist else 0, ctypes.c_void_p(out.data_ptr()),
                                              ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, L.strerror(rc)
    torch.cuda.synchronize()
    o = out.cpu().numpy().view(np.uint64)
    key = int(o[1])
    return int(o[0]), key, int(o[2]), o[3:].copy()


@pytest.mark.parametrize("n,k,seed,j,g", [(150, 40, 4, 0, 4), (150, 40, 4, 3, 3), (192, 64, 8, 1, 3),
                                          (300, 50, 5, 2, 4)])
def test_noalloc_matches_allocating_entry_points(env, n, k, seed, j, g):
    torch, L, api = env
    G = synth.random_systematic(n, k, seed)
    rows, full, nb, nw = _rows_on_device(torch, G, n, j)
    with api.Code(G, n) as code:
        want_U, want_key, want_combos = code.enumerate_level(g, j, U=n)
        want_hist, want_cnt = code.unit_histogram(g, j)
    for _ in range(2):  # two calls in a row share (and must re-clear) the scratch
        U, key, cnt, hist = _call(torch, L, rows, k, nw, nb, full, g, n, True)
        assert cnt == want_cnt == want_combos[0] == math.comb(k, g)
        assert U == want_U
        assert (key >> 54, key & ((1 << 54) - 1)) == (want_key[0], want_key[3])
        assert np.array_equal(hist, want_hist[: hist.size])
        assert not want_hist[hist.size:].any()
    # and without the histogram, at a threshold below the least weight: no candidate
    U, key, cnt, _ = _call(torch, L, rows, k, nw, nb, full, g, want_U - 1, False)
    assert key == (1 << 64) - 1 and U == want_U - 1 and cnt == math.comb(k, g)


@pytest.mark.parametrize("n,k,seed,j,g", [(150, 40, 4, 0, 3), (300, 50, 5, 2, 3)])
def test_noalloc_ignores_padding_bits(env, n, k, seed, j, g):
    """Rows whose padding (bits past n_bits in the last word, and a whole extra word per
    row) holds ones give the same threshold, key and count as the clean rows.  Only the
    histogram-free form is run on dirty rows."""
    torch, L, api = env
    G = synth.random_systematic(n, k, seed)
    rows, full, nb, nw = _rows_on_device(torch, G, n, j)
    clean = _call(torch, L, rows, k, nw, nb, full, g, n, False)
    host = rows.cpu().numpy().view(np.uint32).reshape(k, nw)
    dirty = np.full((k, nw + 1), 0xA5A5A5A5, dtype=np.uint32)
    dirty[:, :nw] = host
    if nb % 32:
        dirty[:, nw - 1] |= np.uint32(~((1 << (nb % 32)) - 1) & 0xFFFFFFFF)
    assert not np.array_equal(dirty[:, :nw], host) or nb % 32 == 0
    drows = torch.from_numpy(dirty.reshape(-1).view(np.int32).copy()).cuda()
    for _ in range(2):
        got = _call(torch, L, drows, k, nw + 1, nb, full, g, n, False)
        assert got[:3] == clean[:3]
    assert clean[2] == math.comb(k, g)


def test_noalloc_histogram_at_the_size_limit(env):
    """n = 512 (the library's limit), a full-rank set of a k = 8 code at g = k: the
    histogram has n_bits + g + 1 = 513 bins, exactly the scratch array's capacity."""
    torch, L, api = env
    n, k = 512, 8
    G = synth.random_systematic(n, k, 3)
    rows, full, nb, nw = _rows_on_device(torch, G, n, 0)
    assert full == 1 and nb == n - k and nb + k + 1 == 513
    with api.Code(G, n) as code:
        want_hist, want_cnt = code.unit_histogram(k, 0)
    U, key, cnt, hist = _call(torch, L, rows, k, nw, nb, full, k, n, True)
    assert hist.size == 513 and cnt == want_cnt == 1
    assert np.array_equal(hist, want_hist)


def test_noalloc_rejects_oversize(env):
    torch, L, api = env
    G = synth.random_systematic(150, 40, 4)
    rows, full, nb, nw = _rows_on_device(torch, G, 150, 0)
    out = torch.zeros(700, dtype=torch.int64, device="cuda")
    # a histogram wider than the scratch holds (n_bits + g + 1 > MDIST_NOALLOC_MAX_HIST_BINS)
    rc = L.lib().mdist_enumerate_unit_noalloc(ctypes.c_void_p(rows.data_ptr()), 64, 16, 512, 1, 40, 100, 1,
                                              ctypes.c_void_p(out.data_ptr()), None)
    assert rc == L.ERANGE

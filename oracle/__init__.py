"""CPU oracle for the minimum distance of binary linear codes (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg
and ``--impl reference``) may import this package.  The product path
(``paper_1603_06757_gb300``) never imports it, and it imports nothing from there.

Every function here is a thin ctypes wrapper over ``oracle.c`` (plain C, compiled with
gcc); see that file's header for which passage of the paper each function follows.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_K = 64
MAX_N = 512
MAX_W = MAX_N // 64
MAX_SETS = 64


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (portable flags: same results on x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", _LIB + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class OrcResult(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int32),
        ("key_w", ctypes.c_int32),
        ("key_g", ctypes.c_int32),
        ("key_j", ctypes.c_int32),
        ("key_rank", ctypes.c_uint64),
        ("g_final", ctypes.c_int32),
        ("j_final", ctypes.c_int32),
        ("m", ctypes.c_int32),
        ("L_final", ctypes.c_int32),
        ("U_final", ctypes.c_int32),
        ("ranks", ctypes.c_int32 * MAX_SETS),
        ("message", ctypes.c_uint64),
        ("witness", ctypes.c_uint64 * MAX_W),
        ("counts", ctypes.c_uint64 * ((MAX_K + 1) * MAX_SETS)),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P64 = ctypes.POINTER(ctypes.c_uint64)
            PI = ctypes.POINTER(ctypes.c_int)
            lib.orc_weight_enumerator.argtypes = [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P64]
            lib.orc_partition.argtypes = [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          PI, PI, PI, P64, P64]
            lib.orc_enumerate_unit.argtypes = [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, PI, P64, P64, P64, P64]
            lib.orc_min_distance.argtypes = [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.POINTER(OrcResult)]
            lib.orc_min_distance_skip.argtypes = [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.POINTER(OrcResult)]
            lib.orc_partition_overlap.argtypes = [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                  PI, PI, P64, P64, PI]
            lib.orc_overlap_bound.argtypes = [ctypes.c_int, PI, ctypes.c_int, PI, ctypes.c_int, PI]
            lib.orc_min_distance_overlap.argtypes = [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_int, ctypes.c_int, ctypes.POINTER(OrcResult)]
            lib.orc_unrank_lex.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64]
            lib.orc_unrank_lex.restype = ctypes.c_uint64
            lib.orc_binomial.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.orc_binomial.restype = ctypes.c_uint64
            _lib = lib
    return _lib


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _pi(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _as_matrix(G, n):
    G = np.ascontiguousarray(np.asarray(G, dtype=np.uint64))
    if G.ndim != 2:
        raise ValueError("G must be (k, W) uint64")
    return G


def weight_enumerator(G, n: int, nthreads: int | None = None) -> np.ndarray:
    """A[w] = number of codewords of weight w over all 2^k messages (k <= 40)."""
    G = _as_matrix(G, n)
    k, W = G.shape
    A = np.zeros(n + 1, dtype=np.uint64)
    rc = _load().orc_weight_enumerator(_p64(G), n, k, W, nthreads or default_threads(), _p64(A))
    if rc != 0:
        raise ValueError(f"orc_weight_enumerator failed ({rc})")
    return A


def brute_force_distance(G, n: int, nthreads: int | None = None) -> int:
    A = weight_enumerator(G, n, nthreads)
    nz = [w for w in range(1, n + 1) if A[w]]
    if A[0] != 1:
        raise ValueError("generator matrix is rank deficient")
    return nz[0]


def partition(G, n: int, max_sets: int = MAX_SETS):
    """Greedy disjoint information sets.  Returns dict with m, ranks[m], pivcols[m,k],
    gammas[m,k,W], transforms[m,k]."""
    G = _as_matrix(G, n)
    k, W = G.shape
    m = np.zeros(1, dtype=np.int32)
    ranks = np.zeros(MAX_SETS, dtype=np.int32)
    piv = np.zeros(MAX_SETS * k, dtype=np.int32)
    gam = np.zeros(MAX_SETS * k * W, dtype=np.uint64)
    tr = np.zeros(MAX_SETS * k, dtype=np.uint64)
    rc = _load().orc_partition(_p64(G), n, k, W, max_sets, _pi(m), _pi(ranks), _pi(piv), _p64(gam), _p64(tr))
    if rc == -2:
        raise ValueError("rank(G) < k")
    if rc != 0:
        raise ValueError(f"orc_partition failed ({rc})")
    mm = int(m[0])
    return {
        "m": mm,
        "ranks": ranks[:mm].copy(),
        "pivcols": piv.reshape(MAX_SETS, k)[:mm].copy(),
        "gammas": gam.reshape(MAX_SETS, k, W)[:mm].copy(),
        "transforms": tr.reshape(MAX_SETS, k)[:mm].copy(),
    }


def enumerate_unit(gamma, n: int, g: int, nthreads: int | None = None, want_hist: bool = True):
    """Every weight-g combination of the rows of one Gamma.  Returns dict with min_w,
    min_rank (lexicographic), count, hist[0..n], xor_all[W]."""
    gamma = np.ascontiguousarray(np.asarray(gamma, dtype=np.uint64))
    k, W = gamma.shape
    mw = np.zeros(1, dtype=np.int32)
    mr = np.zeros(1, dtype=np.uint64)
    cnt = np.zeros(1, dtype=np.uint64)
    hist = np.zeros(n + 1, dtype=np.uint64)
    xa = np.zeros(W, dtype=np.uint64)
    rc = _load().orc_enumerate_unit(_p64(gamma), n, k, W, g, nthreads or default_threads(), _pi(mw), _p64(mr),
                                    _p64(cnt), _p64(hist) if want_hist else None, _p64(xa))
    if rc != 0:
        raise ValueError(f"orc_enumerate_unit failed ({rc})")
    return {"min_w": int(mw[0]), "min_rank": int(mr[0]), "count": int(cnt[0]), "hist": hist, "xor_all": xa}


def partition_overlap(G, n: int, msets: int):
    """M overlapping full information sets (orc_partition_overlap).  Returns dict with m,
    ranks[m] (relative ranks), pivcols[m,k] (scan order), gammas[m,k,W],
    transforms[m,k], cover[n]."""
    G = _as_matrix(G, n)
    k, W = G.shape
    rel = np.zeros(MAX_SETS, dtype=np.int32)
    piv = np.zeros(MAX_SETS * k, dtype=np.int32)
    gam = np.zeros(MAX_SETS * k * W, dtype=np.uint64)
    tr = np.zeros(MAX_SETS * k, dtype=np.uint64)
    cover = np.zeros(n, dtype=np.int32)
    rc = _load().orc_partition_overlap(_p64(G), n, k, W, int(msets), _pi(rel), _pi(piv), _p64(gam), _p64(tr),
                                       _pi(cover))
    if rc == -2:
        raise ValueError("rank(G) < k")
    if rc != 0:
        raise ValueError(f"orc_partition_overlap failed ({rc})")
    m = int(msets)
    return {
        "m": m,
        "ranks": rel[:m].copy(),
        "pivcols": piv.reshape(MAX_SETS, k)[:m].copy(),
        "gammas": gam.reshape(MAX_SETS, k, W)[:m].copy(),
        "transforms": tr.reshape(MAX_SETS, k)[:m].copy(),
        "cover": cover,
    }


def overlap_bound(levels, k: int, rel_ranks, cover) -> int:
    """orc_overlap_bound: the lower bound once set j has all its levels <= levels[j] done."""
    h = np.ascontiguousarray(np.asarray(levels, dtype=np.int32))
    rel = np.ascontiguousarray(np.asarray(rel_ranks, dtype=np.int32))
    cov = np.ascontiguousarray(np.asarray(cover, dtype=np.int32))
    return int(_load().orc_overlap_bound(len(h), _pi(h), int(k), _pi(rel), len(cov), _pi(cov)))


def min_distance(G, n: int, check_per_matrix: bool = False, max_sets: int = MAX_SETS,
                 nthreads: int | None = None, skip_idle_sets: bool = False, overlap_sets: int = 0) -> dict:
    """Alg. 1 (plain Brouwer-Zimmerman).  Returns a dict with d, key (w, g, j, rank),
    message, witness[W], g_final, j_final, m, ranks, counts[g][j], L_final, U_final.
    skip_idle_sets: the sets whose bound term is still 0 are left out until it becomes
    positive, then catch up (orc_min_distance_skip; level check only).
    overlap_sets = M > 0: M overlapping full information sets with the bound of
    orc_overlap_bound (orc_min_distance_overlap; ranks are the relative ranks)."""
    G = _as_matrix(G, n)
    k, W = G.shape
    res = OrcResult()
    if overlap_sets:
        if skip_idle_sets:
            raise ValueError("overlap_sets and skip_idle_sets are exclusive")
        rc = _load().orc_min_distance_overlap(_p64(G), n, k, W, int(overlap_sets), 1 if check_per_matrix else 0,
                                              nthreads or default_threads(), ctypes.byref(res))
    elif skip_idle_sets:
        if check_per_matrix:
            raise ValueError("skip_idle_sets works with the level check only")
        rc = _load().orc_min_distance_skip(_p64(G), n, k, W, max_sets, nthreads or default_threads(),
                                           ctypes.byref(res))
    else:
        rc = _load().orc_min_distance(_p64(G), n, k, W, 1 if check_per_matrix else 0, max_sets,
                                      nthreads or default_threads(), ctypes.byref(res))
    if rc == -2:
        raise ValueError("rank(G) < k")
    if rc != 0:
        raise ValueError(f"orc_min_distance failed ({rc})")
    counts = np.ctypeslib.as_array(res.counts).reshape(MAX_K + 1, MAX_SETS)
    return {
        "d": res.d,
        "key": (res.key_w, res.key_g, res.key_j, int(res.key_rank)),
        "message": int(res.message),
        "witness": np.array(list(res.witness)[:W], dtype=np.uint64),
        "g_final": res.g_final,
        "j_final": res.j_final,
        "m": res.m,
        "ranks": list(res.ranks)[: res.m],
        "counts": counts[:, : res.m].copy(),
        "L_final": res.L_final,
        "U_final": res.U_final,
    }


def unrank_lex(k: int, g: int, rank: int) -> int:
    return int(_load().orc_unrank_lex(k, g, rank))


def binomial(a: int, b: int) -> int:
    return int(_load().orc_binomial(a, b))

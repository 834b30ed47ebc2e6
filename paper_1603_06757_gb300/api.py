"""Python binding of libmdist.so: argument marshalling only.

Every step of the computation (information sets on the host in C++, the level
enumeration on the GPU) runs inside the library.  PyTorch supplies the device memory
(through the library's allocator hooks, so the caching allocator owns it) and the
CUDA stream.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L


def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("mdist needs a CUDA device")
    return torch


class _TorchAllocator:
    """Device allocations for the library, served by torch's caching allocator."""

    def __init__(self, torch, device):
        self.torch = torch
        self.device = device
        self.live = {}
        self.alloc_cb = L.ALLOC_FN(self._alloc)
        self.free_cb = L.FREE_FN(self._free)

    def _alloc(self, nbytes, _ctx):
        try:
            t = self.torch.empty(max(int(nbytes), 1), dtype=self.torch.uint8, device=self.device)
        except Exception:  # noqa: BLE001 - out of memory is reported to C as NULL
            return None
        ptr = t.data_ptr()
        self.live[ptr] = t
        return ptr

    def _free(self, ptr, _ctx):
        self.live.pop(int(ptr or 0), None)


def as_packed(G, n: int) -> np.ndarray:
    """(k, W) uint64, C-contiguous (the library's bit layout)."""
    G = np.ascontiguousarray(np.asarray(G, dtype=np.uint64))
    if G.ndim != 2 or G.shape[1] < (n + 63) // 64:
        raise ValueError("G must be (k, >= ceil(n/64)) uint64")
    return G


def _p64(a):
    return a.ctypes.data_as(L.P64)


class Code:
    """A prepared code: information sets on the host, packed Gamma_j on the device."""

    def __init__(self, G, n: int, *, check_per_matrix: bool = False, max_sets: int = 0, blocks_per_sm: int = 0,
                 filter_group: int = 0, wstar_hint: int = 0, tensor_cores: int = 0, skip_idle_sets: bool = False,
                 timeout_cycles: int = 0, overlap_sets: int = 0, stream=None, torch_alloc: bool = True,
                 allocator=None):
        """allocator: an object with alloc_cb / free_cb (ctypes callbacks of the
        library's allocator hooks) used instead of torch's caching allocator."""
        torch = _torch()
        self.n = int(n)
        self.G = as_packed(G, n)
        self.k, self.W = self.G.shape
        self._lib = L.lib()
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        if allocator is not None:
            self._alloc = allocator
        else:
            self._alloc = _TorchAllocator(torch, self._stream.device) if torch_alloc else None
        opts = L.Options()
        opts.check_per_matrix = 1 if check_per_matrix else 0
        opts.max_sets = int(max_sets)
        opts.blocks_per_sm = int(blocks_per_sm)
        opts.filter_group = int(filter_group)
        opts.wstar_hint = int(wstar_hint)
        opts.tensor_cores = int(tensor_cores)
        opts.skip_idle_sets = 1 if skip_idle_sets else 0
        opts.timeout_cycles = int(timeout_cycles)
        opts.overlap_sets = int(overlap_sets)
        if self._alloc is not None:
            opts.dev_alloc = self._alloc.alloc_cb
            opts.dev_free = self._alloc.free_cb
        self._opts = opts
        h = ctypes.c_void_p()
        with torch.cuda.device(self._stream.device):
            rc = self._lib.mdist_prepare(_p64(self.G), self.n, self.k, self.W, ctypes.byref(opts),
                                         ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(h))
        L.check(rc, "mdist_prepare")
        self._h = h

    # -- lifetime ------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.mdist_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- information sets ----------------------------------------------------------
    def info_sets(self) -> dict:
        m = ctypes.c_int()
        ranks = np.zeros(L.MAX_SETS, dtype=np.int32)
        piv = np.zeros(L.MAX_SETS * self.k, dtype=np.int32)
        gam = np.zeros(L.MAX_SETS * self.k * self.W, dtype=np.uint64)
        tr = np.zeros(L.MAX_SETS * self.k, dtype=np.uint64)
        rc = self._lib.mdist_info_sets(self._h, ctypes.byref(m), ranks.ctypes.data_as(L.PI),
                                       piv.ctypes.data_as(L.PI32), _p64(gam), _p64(tr))
        L.check(rc, "mdist_info_sets")
        mm = m.value
        return {
            "m": mm,
            "ranks": ranks[:mm].copy(),
            "pivcols": piv.reshape(L.MAX_SETS, self.k)[:mm].copy(),
            "gammas": gam.reshape(L.MAX_SETS, self.k, self.W)[:mm].copy(),
            "transforms": tr.reshape(L.MAX_SETS, self.k)[:mm].copy(),
        }

    @property
    def m(self) -> int:
        m = ctypes.c_int()
        L.check(self._lib.mdist_info_sets(self._h, ctypes.byref(m), None, None, None, None), "mdist_info_sets")
        return m.value

    # -- single units ----------------------------------------------------------------
    def enumerate_level(self, g: int, j: int = -1, U: int | None = None, key=None):
        """Units (g, j) (j = -1: every set).  Returns (U, key tuple or None, combos list)."""
        Uc = ctypes.c_int(self.n if U is None else int(U))
        k = L.Key(2**31 - 1, 0, 0, 0, 0) if key is None else L.Key(key[0], key[1], key[2], 0, key[3])
        nunits = self.m if j < 0 else 1
        combos = np.zeros(nunits, dtype=np.uint64)
        rc = self._lib.mdist_enumerate_level(self._h, int(g), int(j), ctypes.byref(Uc), ctypes.byref(k),
                                             _p64(combos))
        L.check(rc, "mdist_enumerate_level")
        kt = k.as_tuple()
        return Uc.value, (None if kt[0] == 2**31 - 1 else kt), [int(c) for c in combos]

    def enumerate_level_part(self, g: int, j: int, part: int, nparts: int, U: int | None = None):
        """Slice `part` of `nparts` of unit (g, j) (j = -1: every set).  Returns (U, key tuple
        or None, combos list) as enumerate_level."""
        Uc = ctypes.c_int(self.n if U is None else int(U))
        k = L.Key(2**31 - 1, 0, 0, 0, 0)
        nunits = self.m if j < 0 else 1
        combos = np.zeros(nunits, dtype=np.uint64)
        rc = self._lib.mdist_enumerate_level_part(self._h, int(g), int(j), int(part), int(nparts), ctypes.byref(Uc),
                                                  ctypes.byref(k), _p64(combos))
        L.check(rc, "mdist_enumerate_level_part")
        kt = k.as_tuple()
        return Uc.value, (None if kt[0] == 2**31 - 1 else kt), [int(c) for c in combos]

    def run_sharded(self, part: int, nparts: int, exchange) -> bool:
        """mdist_run_sharded: this handle runs slice `part` of every unit; exchange(key, count)
        returns the (least key, summed count) over all ranks.  An exception inside it ends
        the run with MDIST_ECANCELLED."""
        def cb(kp, cp, _ctx):
            try:
                kk, cc = exchange(int(kp[0]), int(cp[0]))
                kp[0], cp[0] = int(kk), int(cc)
                return 0
            except Exception:  # noqa: BLE001 - reported to C as a failed exchange
                return 1

        fn = L.EXCHANGE_FN(cb)
        fin = ctypes.c_int()
        L.check(self._lib.mdist_run_sharded(self._h, int(part), int(nparts), fn, None, ctypes.byref(fin)),
                "mdist_run_sharded")
        return bool(fin.value)

    def level_counters(self) -> dict:
        """Tensor-core counters of the last enumerate_level call: combinations covered
        and pairs re-weighed exactly (the filter's pass count)."""
        a = np.zeros(1, dtype=np.uint64)
        b = np.zeros(1, dtype=np.uint64)
        L.check(self._lib.mdist_level_counters(self._h, _p64(a), _p64(b)), "mdist_level_counters")
        return {"tc_combos": int(a[0]), "tc_candidates": int(b[0])}

    def unit_histogram(self, g: int, j: int):
        hist = np.zeros(self.n + 1, dtype=np.uint64)
        cnt = np.zeros(1, dtype=np.uint64)
        rc = self._lib.mdist_unit_histogram(self._h, int(g), int(j), _p64(hist), _p64(cnt))
        L.check(rc, "mdist_unit_histogram")
        return hist, int(cnt[0])

    # -- Alg. 1 ----------------------------------------------------------------------
    def reset(self) -> None:
        L.check(self._lib.mdist_reset(self._h), "mdist_reset")

    def run(self, max_units: int = 0) -> bool:
        fin = ctypes.c_int()
        L.check(self._lib.mdist_run(self._h, int(max_units), ctypes.byref(fin)), "mdist_run")
        return bool(fin.value)

    def result(self) -> dict:
        d = ctypes.c_int()
        wit = np.zeros(self.W, dtype=np.uint64)
        msg = np.zeros(1, dtype=np.uint64)
        key = L.Key()
        st = L.Stats()
        rc = self._lib.mdist_result(self._h, ctypes.byref(d), _p64(wit), _p64(msg), ctypes.byref(key),
                                    ctypes.byref(st))
        L.check(rc, "mdist_result")
        return _result_dict(d.value, wit, msg, key, st)

    def min_distance(self) -> dict:
        d = ctypes.c_int()
        wit = np.zeros(self.W, dtype=np.uint64)
        msg = np.zeros(1, dtype=np.uint64)
        key = L.Key()
        st = L.Stats()
        rc = self._lib.mdist_min_distance(self._h, ctypes.byref(d), _p64(wit), _p64(msg), ctypes.byref(key),
                                          ctypes.byref(st))
        L.check(rc, "mdist_min_distance")
        return _result_dict(d.value, wit, msg, key, st)

    # -- checkpoint ------------------------------------------------------------------
    def state_save(self) -> bytes:
        n = ctypes.c_size_t(0)
        self._lib.mdist_state_save(self._h, None, ctypes.byref(n))
        buf = ctypes.create_string_buffer(n.value)
        L.check(self._lib.mdist_state_save(self._h, buf, ctypes.byref(n)), "mdist_state_save")
        return buf.raw[: n.value]

    def state_load(self, blob: bytes) -> None:
        buf = ctypes.create_string_buffer(blob, len(blob))
        L.check(self._lib.mdist_state_load(self._h, buf, len(blob)), "mdist_state_load")


def _result_dict(d, wit, msg, key, st) -> dict:
    m = st.m
    combos = np.ctypeslib.as_array(st.combos).reshape(L.MAX_K + 1, L.MAX_SETS)[:, :m].copy()
    return {
        "d": int(d),
        "key": key.as_tuple(),
        "message": int(msg[0]),
        "witness": wit,
        "g_final": int(st.g_final),
        "j_final": int(st.j_final),
        "m": int(m),
        "ranks": [int(r) for r in st.ranks[:m]],
        "counts": combos,
        "L_final": int(st.L_final),
        "U_final": int(st.U_final),
        "launches": int(st.launches),
        "total_combos": int(st.total_combos),
        "seconds": float(st.seconds),
        "kernel_ms": float(st.kernel_ms),
        "h2d_bytes": int(st.h2d_bytes),
        "d2h_bytes": int(st.d2h_bytes),
        "tc_ms": float(st.tc_ms),
        "tc_launches": int(st.tc_launches),
        "tc_combos": int(st.tc_combos),
        "tc_candidates": int(st.tc_candidates),
    }


def min_distance(G, n: int, **kw) -> dict:
    """d, witness, key and statistics of the code generated by G (k x W uint64)."""
    with Code(G, n, **kw) as c:
        return c.min_distance()


def device_info() -> dict:
    sm = ctypes.c_int()
    clk = ctypes.c_int()
    ma = ctypes.c_int()
    mi = ctypes.c_int()
    L.check(L.lib().mdist_device_info(ctypes.byref(sm), ctypes.byref(clk), ctypes.byref(ma), ctypes.byref(mi)),
            "mdist_device_info")
    return {"sm_count": sm.value, "max_sm_clock_khz": clk.value, "cc": (ma.value, mi.value)}


class Server:
    """Continuous-batching serving loop (mdist_server_*)."""

    def __init__(self, *, max_slots: int = 1024, rows_pool_bytes: int = 64 << 20, check_per_matrix: bool = False,
                 max_sets: int = 0, blocks_per_sm: int = 0, tensor_cores: int = 0, torch_alloc: bool = True):
        """tensor_cores: 0 = large requests (>= 10^9 codewords estimated) on the single-code
        tensor-core path, 1 = every request batched, 2 = every request on that path."""
        torch = _torch()
        self._lib = L.lib()
        self._alloc = _TorchAllocator(torch, torch.cuda.current_device()) if torch_alloc else None
        opts = L.Options()
        opts.check_per_matrix = 1 if check_per_matrix else 0
        opts.max_sets = int(max_sets)
        opts.blocks_per_sm = int(blocks_per_sm)
        opts.tensor_cores = int(tensor_cores)
        if self._alloc is not None:
            opts.dev_alloc = self._alloc.alloc_cb
            opts.dev_free = self._alloc.free_cb
        self._opts = opts
        h = ctypes.c_void_p()
        L.check(self._lib.mdist_server_create(ctypes.byref(opts), int(max_slots), int(rows_pool_bytes),
                                              ctypes.byref(h)), "mdist_server_create")
        self._h = h
        self._W = {}

    def submit(self, G, n: int, wstar_hint: int = 0) -> int:
        G = as_packed(G, n)
        k, W = G.shape
        rid = ctypes.c_longlong()
        L.check(self._lib.mdist_server_submit(self._h, _p64(G), int(n), k, W, int(wstar_hint), ctypes.byref(rid)),
                "mdist_server_submit")
        self._W[rid.value] = W
        return rid.value

    def poll(self, rid: int, wait_ms: int = 0):
        """Result dict (with 'latency_s') or None if not finished yet."""
        W = self._W[rid]
        d = ctypes.c_int()
        wit = np.zeros(W, dtype=np.uint64)
        msg = np.zeros(1, dtype=np.uint64)
        key = L.Key()
        st = L.Stats()
        lat = ctypes.c_double()
        rc = self._lib.mdist_server_poll(self._h, int(rid), int(wait_ms), ctypes.byref(d), _p64(wit), _p64(msg),
                                         ctypes.byref(key), ctypes.byref(st), ctypes.byref(lat))
        if rc == L.EAGAIN:
            return None
        L.check(rc, "mdist_server_poll")
        self._W.pop(rid, None)
        out = _result_dict(d.value, wit, msg, key, st)
        out["latency_s"] = lat.value
        return out

    def cancel(self, rid: int) -> int:
        """mdist_server_cancel: OK (queued or in flight: its poll raises ECANCELLED),
        EAGAIN (already finished) or EINVAL (unknown id); returns the code."""
        return int(self._lib.mdist_server_cancel(self._h, int(rid)))

    def info(self) -> dict:
        a, c, r = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        q, f = ctypes.c_int(), ctypes.c_int()
        ms = ctypes.c_double()
        rc = self._lib.mdist_server_info(self._h, ctypes.byref(a), ctypes.byref(c), ctypes.byref(r), ctypes.byref(q),
                                         ctypes.byref(f), ctypes.byref(ms))
        L.check(rc, "mdist_server_info")
        return {"admitted": a.value, "completed": c.value, "rounds": r.value, "queued": q.value,
                "in_flight": f.value, "gpu_ms": ms.value}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mdist_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def partition_host(G, n: int, max_sets: int = 0) -> dict:
    """The information sets mdist_prepare would form, computed on the host only."""
    G = as_packed(G, n)
    k, W = G.shape
    m = ctypes.c_int()
    ranks = np.zeros(L.MAX_SETS, dtype=np.int32)
    piv = np.zeros(L.MAX_SETS * k, dtype=np.int32)
    gam = np.zeros(L.MAX_SETS * k * W, dtype=np.uint64)
    tr = np.zeros(L.MAX_SETS * k, dtype=np.uint64)
    rc = L.lib().mdist_partition_host(_p64(G), int(n), k, W, int(max_sets), ctypes.byref(m),
                                      ranks.ctypes.data_as(L.PI), piv.ctypes.data_as(L.PI32), _p64(gam), _p64(tr))
    L.check(rc, "mdist_partition_host")
    mm = m.value
    return {
        "m": mm,
        "ranks": ranks[:mm].copy(),
        "pivcols": piv.reshape(L.MAX_SETS, k)[:mm].copy(),
        "gammas": gam.reshape(L.MAX_SETS, k, W)[:mm].copy(),
        "transforms": tr.reshape(L.MAX_SETS, k)[:mm].copy(),
    }


def partition_overlap_host(G, n: int, msets: int) -> dict:
    """The overlapping information sets of overlap_sets = msets, computed on the host."""
    G = as_packed(G, n)
    k, W = G.shape
    ranks = np.zeros(msets, dtype=np.int32)
    piv = np.zeros(msets * k, dtype=np.int32)
    gam = np.zeros(msets * k * W, dtype=np.uint64)
    tr = np.zeros(msets * k, dtype=np.uint64)
    cover = np.zeros(n, dtype=np.int32)
    rc = L.lib().mdist_partition_overlap_host(_p64(G), int(n), k, W, int(msets), ranks.ctypes.data_as(L.PI),
                                              piv.ctypes.data_as(L.PI32), _p64(gam), _p64(tr),
                                              cover.ctypes.data_as(L.PI32))
    L.check(rc, "mdist_partition_overlap_host")
    return {"m": int(msets), "ranks": ranks, "pivcols": piv.reshape(msets, k), "gammas": gam.reshape(msets, k, W),
            "transforms": tr.reshape(msets, k), "cover": cover}


def overlap_bound_host(G, n: int, msets: int, levels) -> int:
    G = as_packed(G, n)
    k, W = G.shape
    lv = np.ascontiguousarray(np.asarray(levels, dtype=np.int32))
    out = ctypes.c_int()
    L.check(L.lib().mdist_overlap_bound_host(_p64(G), int(n), k, W, int(msets), lv.ctypes.data_as(L.PI),
                                             ctypes.byref(out)), "mdist_overlap_bound_host")
    return out.value


def side_tables(rows, sides, lows=None) -> list:
    """The tensor-core enumerator's subset-sum tables (mdist_debug_side_tables), built on
    the current device: rows (k, nwords) uint32; sides: tuples (off0, kc0, t0, off1, kc1,
    t1), t1 = -1 for one component; lows: per side None or the index of an earlier side of
    the same list, a one-component side (off0, kc0, u), 0 < u < t0, whose table is built
    first (a separate launch) and read as the low-subset sums.  Returns one
    (entries, nwords) uint32 array per side."""
    import math

    torch = _torch()
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.uint32))
    k, nw = rows.shape
    d_rows = torch.from_numpy(rows.view(np.int32).copy()).cuda()
    lows = list(lows) if lows is not None else [None] * len(sides)
    outs = []
    for (off0, kc0, t0, off1, kc1, t1) in sides:
        cnt = math.comb(kc0, t0) * (math.comb(kc1, t1) if t1 >= 0 else 1)
        outs.append((torch.empty(max(cnt * nw, 4), dtype=torch.int32, device=d_rows.device), cnt))
    stream = torch.cuda.current_stream()

    def launch(idx):
        flat = np.ascontiguousarray(np.asarray([sides[i] for i in idx], dtype=np.int32).reshape(-1))
        parr = (ctypes.c_void_p * len(idx))(*[outs[i][0].data_ptr() for i in idx])
        larr = (ctypes.c_void_p * len(idx))(*[outs[lows[i]][0].data_ptr() if lows[i] is not None else None
                                              for i in idx])
        lt = np.asarray([sides[lows[i]][2] if lows[i] is not None else 0 for i in idx], dtype=np.int32)
        L.check(L.lib().mdist_debug_side_tables(ctypes.c_void_p(d_rows.data_ptr()), k, nw, len(idx),
                                                flat.ctypes.data_as(L.PI), parr, larr, lt.ctypes.data_as(L.PI),
                                                ctypes.c_void_p(stream.cuda_stream)), "mdist_debug_side_tables")

    first = [i for i in range(len(sides)) if lows[i] is None]
    second = [i for i in range(len(sides)) if lows[i] is not None]
    for part in (first, second):
        for a in range(0, len(part), 128):
            launch(part[a:a + 128])
    stream.synchronize()
    return [t[: cnt * nw].cpu().numpy().view(np.uint32).reshape(cnt, nw) for t, cnt in outs]


def microbench(which: str, iters: int = 20000) -> dict:
    """Per-SM-per-clock throughput of 'popc', 'lop3', 'step4', 'step4_or2', 'step4_or4' or
    of the fp8 tensor-core MMA ('mma' no swizzle, 'mma_sw128', 'mma_sw32': multiply-adds)
    (see include/mdist.h)."""
    idx = {"popc": 0, "lop3": 1, "step4": 2, "step4_or2": 3, "step4_or4": 4, "mma": 5, "mma_sw128": 6,
           "mma_sw32": 7}[which]
    v = ctypes.c_double()
    s = ctypes.c_double()
    L.check(L.probe_lib().mdist_microbench(idx, int(iters), ctypes.byref(v), ctypes.byref(s)), "mdist_microbench")
    return {"per_clock_per_sm": v.value, "seconds": s.value}


class Batch:
    """Many codes through Alg. 1 together (mdist_batch_*): one graph of rounds."""

    def __init__(self, *, check_per_matrix: bool = False, max_sets: int = 0, blocks_per_sm: int = 0, stream=None,
                 torch_alloc: bool = True, tensor_cores: int = 0, route_work_log10: int = 0):
        """tensor_cores: 0 = codes estimated at >= 10^route_work_log10 (0: 10^9) codewords
        on the single-code tensor-core path, 1 = every code in the graph, 2 = every code on
        that path."""
        torch = _torch()
        self._lib = L.lib()
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        self._alloc = _TorchAllocator(torch, self._stream.device) if torch_alloc else None
        opts = L.Options()
        opts.check_per_matrix = 1 if check_per_matrix else 0
        opts.max_sets = int(max_sets)
        opts.blocks_per_sm = int(blocks_per_sm)
        opts.tensor_cores = int(tensor_cores)
        opts.route_work_log10 = int(route_work_log10)
        if self._alloc is not None:
            opts.dev_alloc = self._alloc.alloc_cb
            opts.dev_free = self._alloc.free_cb
        self._opts = opts
        h = ctypes.c_void_p()
        L.check(self._lib.mdist_batch_create(ctypes.byref(opts), ctypes.c_void_p(self._stream.cuda_stream),
                                             ctypes.byref(h)), "mdist_batch_create")
        self._h = h
        self._shapes = []

    def add(self, G, n: int, wstar_hint: int = 0) -> int:
        G = as_packed(G, n)
        k, W = G.shape
        idx = ctypes.c_int()
        L.check(self._lib.mdist_batch_add(self._h, _p64(G), int(n), k, W, int(wstar_hint), ctypes.byref(idx)),
                "mdist_batch_add")
        self._shapes.append((n, k, W))
        return idx.value

    def run(self, rounds_per_graph: int = 0) -> None:
        L.check(self._lib.mdist_batch_run(self._h, int(rounds_per_graph)), "mdist_batch_run")

    def info(self) -> dict:
        nc, gl, rd, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms, sec, lms = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        L.check(self._lib.mdist_batch_info(self._h, ctypes.byref(nc), ctypes.byref(gl), ctypes.byref(rd),
                                           ctypes.byref(ms), ctypes.byref(sec), ctypes.byref(nl),
                                           ctypes.byref(lms)), "mdist_batch_info")
        return {"codes": nc.value, "graph_launches": gl.value, "rounds": rd.value, "gpu_ms": ms.value,
                "seconds": sec.value, "large_codes": nl.value, "large_ms": lms.value}

    def result(self, index: int) -> dict:
        n, k, W = self._shapes[index]
        d = ctypes.c_int()
        wit = np.zeros(W, dtype=np.uint64)
        msg = np.zeros(1, dtype=np.uint64)
        key = L.Key()
        st = L.Stats()
        rc = self._lib.mdist_batch_result(self._h, int(index), ctypes.byref(d), _p64(wit), _p64(msg),
                                          ctypes.byref(key), ctypes.byref(st))
        L.check(rc, "mdist_batch_result")
        return _result_dict(d.value, wit, msg, key, st)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mdist_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

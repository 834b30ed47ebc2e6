"""ctypes declarations of libmdist.so (mirror of include/mdist.h).

Loading fails loudly when the library has not been built: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmdist.so")

MAX_K = 64
MAX_N = 512
MAX_SETS = 64

OK = 0
EINVAL = -1
ERANK = -2
ENOMEM = -3
ECUDA = -4
ETIMEOUT = -5
ECANCELLED = -6
ERANGE = -7
ESTATE = -8
EAGAIN = -9

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                               ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [
        ("check_per_matrix", ctypes.c_int),
        ("max_sets", ctypes.c_int),
        ("blocks_per_sm", ctypes.c_int),
        ("filter_group", ctypes.c_int),
        ("timeout_cycles", ctypes.c_longlong),
        ("dev_alloc", ALLOC_FN),
        ("dev_free", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
        ("wstar_hint", ctypes.c_int),
        ("tensor_cores", ctypes.c_int),
        ("skip_idle_sets", ctypes.c_int),
        ("overlap_sets", ctypes.c_int),
        ("route_work_log10", ctypes.c_int),
    ]


class Key(ctypes.Structure):
    _fields_ = [
        ("weight", ctypes.c_int32),
        ("g", ctypes.c_int32),
        ("j", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("rank", ctypes.c_uint64),
    ]

    def as_tuple(self):
        return (int(self.weight), int(self.g), int(self.j), int(self.rank))


class Stats(ctypes.Structure):
    _fields_ = [
        ("g_final", ctypes.c_int32),
        ("j_final", ctypes.c_int32),
        ("m", ctypes.c_int32),
        ("L_final", ctypes.c_int32),
        ("U_final", ctypes.c_int32),
        ("launches", ctypes.c_int32),
        ("ranks", ctypes.c_int32 * MAX_SETS),
        ("combos", (ctypes.c_uint64 * MAX_SETS) * (MAX_K + 1)),
        ("total_combos", ctypes.c_uint64),
        ("seconds", ctypes.c_double),
        ("kernel_ms", ctypes.c_double),
        ("h2d_bytes", ctypes.c_uint64),
        ("d2h_bytes", ctypes.c_uint64),
        ("tc_ms", ctypes.c_double),
        ("tc_launches", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("tc_combos", ctypes.c_uint64),
        ("tc_candidates", ctypes.c_uint64),
    ]


class MdistError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


_lock = threading.Lock()
_lib = None

P64 = ctypes.POINTER(ctypes.c_uint64)
PI = ctypes.POINTER(ctypes.c_int)
PI32 = ctypes.POINTER(ctypes.c_int32)
PCODE = ctypes.c_void_p
PF = ctypes.POINTER(ctypes.c_float)

# name -> (restype, argtypes): every entry point of include/mdist.h
SIGNATURES = {
    "mdist_prepare": (ctypes.c_int, [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Options),
                                     ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "mdist_info_sets": (ctypes.c_int, [PCODE, PI, PI, PI32, P64, P64]),
    "mdist_enumerate_level": (ctypes.c_int, [PCODE, ctypes.c_int, ctypes.c_int, PI, ctypes.POINTER(Key), P64]),
    "mdist_unit_histogram": (ctypes.c_int, [PCODE, ctypes.c_int, ctypes.c_int, P64, P64]),
    "mdist_level_counters": (ctypes.c_int, [PCODE, P64, P64]),
    "mdist_run": (ctypes.c_int, [PCODE, ctypes.c_int, PI]),
    "mdist_enumerate_level_part": (ctypes.c_int, [PCODE, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, PI,
                                                  ctypes.POINTER(Key), P64]),
    "mdist_run_sharded": (ctypes.c_int, [PCODE, ctypes.c_int, ctypes.c_int, EXCHANGE_FN, ctypes.c_void_p, PI]),
    "mdist_reset": (ctypes.c_int, [PCODE]),
    "mdist_result": (ctypes.c_int, [PCODE, PI, P64, P64, ctypes.POINTER(Key), ctypes.POINTER(Stats)]),
    "mdist_min_distance": (ctypes.c_int, [PCODE, PI, P64, P64, ctypes.POINTER(Key), ctypes.POINTER(Stats)]),
    "mdist_state_save": (ctypes.c_int, [PCODE, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "mdist_state_load": (ctypes.c_int, [PCODE, ctypes.c_void_p, ctypes.c_size_t]),
    "mdist_set_stream": (ctypes.c_int, [PCODE, ctypes.c_void_p]),
    "mdist_free": (None, [PCODE]),
    "mdist_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "mdist_device_info": (ctypes.c_int, [PI, PI, PI, PI]),
    "mdist_batch_create": (ctypes.c_int, [ctypes.POINTER(Options), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "mdist_batch_add": (ctypes.c_int, [ctypes.c_void_p, P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       PI]),
    "mdist_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "mdist_batch_result": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, PI, P64, P64, ctypes.POINTER(Key),
                                          ctypes.POINTER(Stats)]),
    "mdist_batch_info": (ctypes.c_int, [ctypes.c_void_p, PI, PI, PI, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), PI, ctypes.POINTER(ctypes.c_double)]),
    "mdist_batch_free": (None, [ctypes.c_void_p]),
    "mdist_server_create": (ctypes.c_int, [ctypes.POINTER(Options), ctypes.c_int, ctypes.c_size_t,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "mdist_server_submit": (ctypes.c_int, [ctypes.c_void_p, P64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]),
    "mdist_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, PI, P64, P64,
                                         ctypes.POINTER(Key), ctypes.POINTER(Stats), ctypes.POINTER(ctypes.c_double)]),
    "mdist_server_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), PI, PI,
                                         ctypes.POINTER(ctypes.c_double)]),
    "mdist_server_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong]),
    "mdist_server_free": (None, [ctypes.c_void_p]),
    "mdist_features": (ctypes.c_int, [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, PF]),
    "mdist_gv_estimate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, PI, PI, PI]),
    "mdist_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "mdist_mlp_num_params": (ctypes.c_int, [ctypes.c_void_p, PI]),
    "mdist_mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, PF]),
    "mdist_mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, PF]),
    "mdist_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, PF, ctypes.c_int, PF]),
    "mdist_mlp_loss_grad": (ctypes.c_int, [ctypes.c_void_p, PF, PF, ctypes.c_int, PF, PF]),
    "mdist_mlp_train": (ctypes.c_int, [ctypes.c_void_p, PF, PF, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_float, ctypes.c_uint64, PF]),
    "mdist_mlp_free": (None, [ctypes.c_void_p]),
    "mdist_enumerate_unit_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_void_p, ctypes.c_void_p]),
    "mdist_partition_host": (ctypes.c_int, [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, PI, PI,
                                            PI32, P64, P64]),
    "mdist_partition_overlap_host": (ctypes.c_int, [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, PI,
                                                    PI32, P64, P64, PI32]),
    "mdist_overlap_bound_host": (ctypes.c_int, [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, PI, PI]),
    "mdist_debug_set_rows": (ctypes.c_int, [P64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, PI, PI, PI,
                                            ctypes.POINTER(ctypes.c_uint32)]),
    "mdist_debug_unrank_colex": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_uint32,
                                                ctypes.POINTER(ctypes.c_uint32)]),
    "mdist_debug_next_colex": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]),
    "mdist_debug_lexrank": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, P64]),
    "mdist_debug_filter_choice": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, PI]),
    "mdist_debug_level_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, PI, P64, P64, PI, PI]),
    "mdist_debug_gram_plan": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, PI, PI, P64,
                                             PI]),
    "mdist_debug_side_tables": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, PI,
                                                ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), PI,
                                                ctypes.c_void_p]),
}


# the measurement probes of include/mdist_probe.h, in libmdist_probe.so
PROBE_LIB_PATH = os.path.join(HERE, "libmdist_probe.so")
PROBE_SIGNATURES = {
    "mdist_microbench": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
    "mdist_tc_probe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, PF]),
}
_probe = None


def probe_lib():
    """The loaded libmdist_probe.so (tests and the benchmark only)."""
    global _probe
    with _lock:
        if _probe is None:
            if not os.path.exists(PROBE_LIB_PATH):
                raise ImportError(f"{PROBE_LIB_PATH} is missing: build the CUDA libraries first")
            handle = ctypes.CDLL(PROBE_LIB_PATH)
            for name, (res, args) in PROBE_SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _probe = handle
    return _probe


def lib():
    """The loaded libmdist.so.  Raises ImportError if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            handle = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().mdist_strerror(code).decode()
    except ImportError:
        return "library not loaded"


def check(code: int, what: str) -> None:
    if code != OK:
        raise MdistError(code, what)

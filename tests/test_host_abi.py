"""C-ABI behaviour that needs no GPU: argument and shape checks answer before any CUDA
call, a rank-deficient G is refused on the host, every error code has its message,
and a valid code on a machine without a device is refused with MDIST_ECUDA (the
library has no CPU path to fall back to).  The Python binding refuses to run without
a device or without the built library.  The header is plain C: a C99 program
(`tests/c_abi_example.c`) compiles against it and links with the library."""

import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from conftest import ROOT
from paper_1603_06757_gb300 import _lib as L

P64 = L.P64


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build_library()
    return L.lib()


def _prepare(lib, G, n, k, W, opts=None):
    out = ctypes.c_void_p()
    Gp = None if G is None else np.ascontiguousarray(G, dtype=np.uint64)
    rc = lib.mdist_prepare(None if Gp is None else Gp.ctypes.data_as(P64), n, k, W,
                           ctypes.byref(opts) if opts is not None else None, None, ctypes.byref(out))
    if out.value:
        lib.mdist_free(out)
    return rc


def _no_device():
    import torch

    return not torch.cuda.is_available()


@pytest.mark.parametrize("n,k,W", [
    (64, 64, 1),     # n <= k
    (60, 64, 1),     # n < k
    (300, 65, 5),    # k > 64
    (100, 0, 2),     # k < 1
    (513, 64, 9),    # n > 512
    (130, 64, 2),    # W < ceil(n / 64)
    (130, 64, 65),   # W > 64
])
def test_prepare_rejects_shapes(lib, n, k, W):
    G = np.zeros((max(k, 1), max(W, 1)), dtype=np.uint64)
    assert _prepare(lib, G, n, k, W) == L.EINVAL


def test_prepare_rejects_null_pointers(lib):
    G = synth.random_systematic(128, 64, 1)
    assert _prepare(lib, None, 128, 64, 2) == L.EINVAL
    assert lib.mdist_prepare(G.ctypes.data_as(P64), 128, 64, 2, None, None, None) == L.EINVAL


def test_prepare_rejects_bits_past_n(lib):
    n, k = 100, 40
    G = synth.random_systematic(n, k, 2)
    bad = G.copy()
    bad[k - 1, 1] |= np.uint64(1) << np.uint64(n - 64)  # column n, one past the last
    assert _prepare(lib, bad, n, k, 2) == L.EINVAL
    wide = np.zeros((k, 3), dtype=np.uint64)  # a third word: columns 128..191, all past n
    wide[:, :2] = G
    wide[0, 2] = np.uint64(1)
    assert _prepare(lib, wide, n, k, 3) == L.EINVAL


@pytest.mark.parametrize("field,value", [
    ("filter_group", -1), ("filter_group", 6), ("tensor_cores", -1), ("tensor_cores", 4),
    ("skip_idle_sets", 2), ("skip_idle_sets", -1),
])
def test_prepare_rejects_options(lib, field, value):
    G = synth.random_systematic(128, 64, 1)
    o = L.Options()
    setattr(o, field, value)
    assert _prepare(lib, G, 128, 64, 2, o) == L.EINVAL


def test_prepare_rejects_skip_with_per_matrix_check(lib):
    G = synth.random_systematic(128, 64, 1)
    o = L.Options()
    o.skip_idle_sets = 1
    o.check_per_matrix = 1
    assert _prepare(lib, G, 128, 64, 2, o) == L.EINVAL


def test_prepare_rank_deficient_on_host(lib):
    G = synth.random_systematic(128, 64, 1)
    G[5] = G[3] ^ G[7]
    assert _prepare(lib, G, 128, 64, 2) == L.ERANK


@pytest.mark.skipif(not _no_device(), reason="checks the refusal on a machine without a GPU")
def test_prepare_valid_code_without_device_is_refused(lib):
    for n, k, seed in [(60, 30, 1), (192, 64, 8), (300, 50, 5)]:
        G = synth.random_systematic(n, k, seed)
        assert _prepare(lib, G, n, k, G.shape[1]) == L.ECUDA
    out = ctypes.c_void_p()
    assert lib.mdist_batch_create(None, None, ctypes.byref(out)) == L.ECUDA
    assert not out.value


def test_batch_create_rejects_skip_idle_sets(lib):
    o = L.Options()
    o.skip_idle_sets = 1
    out = ctypes.c_void_p()
    assert lib.mdist_batch_create(ctypes.byref(o), None, ctypes.byref(out)) == L.EINVAL
    assert lib.mdist_batch_create(None, None, None) == L.EINVAL


def test_every_error_code_has_a_message(lib):
    codes = [0, L.EINVAL, L.ERANK, L.ENOMEM, L.ECUDA, L.ETIMEOUT, L.ECANCELLED, L.ERANGE, L.ESTATE, L.EAGAIN]
    msgs = [lib.mdist_strerror(c).decode() for c in codes]
    assert msgs[0] == "ok"
    assert len(set(msgs)) == len(msgs) and "unknown error" not in msgs
    assert lib.mdist_strerror(-100).decode() == "unknown error"
    assert lib.mdist_strerror(1).decode() == "unknown error"


def test_free_null_is_a_no_op(lib):
    lib.mdist_free(None)


@pytest.mark.skipif(not _no_device(), reason="checks the refusal on a machine without a GPU")
def test_python_binding_refuses_without_device(lib):
    from paper_1603_06757_gb300 import api

    G = synth.random_systematic(60, 30, 1)
    with pytest.raises(RuntimeError, match="CUDA device"):
        api.Code(G, 60)


def test_python_binding_refuses_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "libmdist.so"))
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(ImportError, match="build the CUDA library"):
        L.lib()


def _compile_example(tmp_path, compiler, std):
    cc = shutil.which(compiler)
    if cc is None:
        pytest.skip(f"{compiler} not found")
    exe = tmp_path / f"c_abi_example_{compiler.replace('+', 'x')}"
    src = os.path.join(ROOT, "tests", "c_abi_example.c")
    lang = ["-x", "c++"] if compiler.endswith("++") else []
    cmd = [cc, *lang, f"-std={std}", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           src, "-x", "none", "-L", os.path.dirname(L.LIB_PATH), "-lmdist",
           f"-Wl,-rpath,{os.path.dirname(L.LIB_PATH)}", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


@pytest.mark.parametrize("compiler,std", [("gcc", "c99"), ("g++", "c++17")])
def test_header_is_plain_c_and_links(lib, tmp_path, compiler, std):
    """The header compiles as strict C99 (and C++17) and a C program linked against the
    library runs: without a device it is refused with the CUDA error, with one it
    computes d = 3 for the [7,4] Hamming code."""
    exe = _compile_example(tmp_path, compiler, std)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    if _no_device():
        assert r.returncode == 2 and r.stdout.strip() == lib.mdist_strerror(L.ECUDA).decode()
    else:
        assert r.returncode == 0 and r.stdout.startswith("d = 3"), r.stdout

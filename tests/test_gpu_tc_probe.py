"""The tensor-core building block of the Gram-matrix enumerator: one tcgen05 fp8
(E4M3) product with f32 accumulation, against the exact product of the decoded values."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# E4M3 codes of small integers (sign, 4 exponent bits with bias 7, 3 mantissa bits)
E4M3 = {0: 0x00, 1: 0x38, 2: 0x40, 3: 0x44, 4: 0x48, 5: 0x4A, 6: 0x4C, 7: 0x4E, 8: 0x50, 64: 0x68, -2: 0xC0}


def _decode(code):
    s = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 7
    return s * (2.0 ** (e - 7)) * (1 + m / 8) if e else s * (2.0 ** -6) * (m / 8)


def test_e4m3_table():
    for v, c in E4M3.items():
        assert _decode(c) == v


@pytest.mark.parametrize("N,K", [(256, 160), (128, 128), (32, 32), (256, 256)])
def test_tc_product_exact(N, K):
    import __graft_entry__

    __graft_entry__.build()
    from paper_1603_06757_gb300 import _lib as L

    rng = np.random.default_rng(N * 1000 + K)
    vals = np.array(list(E4M3.keys()))
    a_idx = rng.integers(0, len(vals), size=(128, K))
    b_idx = rng.integers(0, len(vals), size=(N, K))
    A = np.vectorize(lambda i: E4M3[vals[i]])(a_idx).astype(np.uint8)
    B = np.vectorize(lambda i: E4M3[vals[i]])(b_idx).astype(np.uint8)
    want = vals[a_idx].astype(np.float64) @ vals[b_idx].astype(np.float64).T
    D = np.zeros((128, N), dtype=np.float32)
    rc = L.probe_lib().mdist_tc_probe(A.ctypes.data_as(ctypes.c_void_p), B.ctypes.data_as(ctypes.c_void_p), N, K,
                                D.ctypes.data_as(L.PF))
    assert rc == 0, L.strerror(rc)
    assert np.array_equal(D.astype(np.float64), want)

"""Host-side predictor inputs (no GPU): features against independent computations,
and the Gilbert-Varshamov fallback against its definition."""

import math

import numpy as np
import pytest

import oracle
import synth
from paper_1603_06757_gb300 import predict


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build_library()


def _gv_py(n, k):
    target = 1 << (n - k)
    s = 0
    for w in range(n + 1):
        s += math.comb(n, w)
        if s >= target:
            return w
    return n


@pytest.mark.parametrize("n,k", [(60, 30), (192, 64), (150, 64), (300, 50), (48, 24), (100, 20), (512, 64)])
def test_gv_estimate(n, k):
    ranks = [int(r) for r in oracle.partition(synth.random_systematic(n, k, 1), n)["ranks"]]
    d, w = predict.gv_estimate(n, k, ranks)
    assert d == _gv_py(n, k)
    L = lambda g: sum(max(0, g + 1 - (k - r)) for r in ranks)  # noqa: E731
    assert L(w) >= d or w == k
    assert w == 1 or L(w - 1) < d


@pytest.mark.parametrize("n,k,seed", [(60, 30, 1), (120, 40, 2), (150, 64, 1), (96, 24, 5), (200, 33, 4)])
def test_features_against_oracle(n, k, seed):
    G = synth.random_systematic(n, k, seed)
    f = predict.features(G, n)
    assert f.shape == (predict.NFEATURES,) and np.all(np.isfinite(f))
    part = oracle.partition(G, n)
    assert f[0] == pytest.approx(n / 512) and f[1] == pytest.approx(k / 64) and f[2] == pytest.approx(k / n)
    assert f[3] == pytest.approx(part["m"] / 16)
    for j in range(min(4, part["m"])):
        assert f[4 + j] == pytest.approx(part["ranks"][j] / k)
    # least weights at level 1 and at levels <= 2, over every set
    w1 = min(oracle.enumerate_unit(part["gammas"][j], n, 1, want_hist=False)["min_w"] for j in range(part["m"]))
    w2 = min(oracle.enumerate_unit(part["gammas"][j], n, 2, want_hist=False)["min_w"] for j in range(part["m"]))
    assert f[10] == pytest.approx(w1 / n)
    assert f[11] == pytest.approx(min(w1, w2) / n)
    # column-weight histogram of the full-rank sets sums to one
    assert float(f[13:21].sum()) == pytest.approx(1.0, abs=1e-5)

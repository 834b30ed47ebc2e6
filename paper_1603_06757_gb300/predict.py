"""Termination-level / distance predictor (sizing and packing only; results never
depend on it).

Features come from mdist_features (host C++), the network is the library's fp32 MLP
(hand-written CUDA forward / backward / Adam), the fallback is the analytic
Gilbert-Varshamov estimate (mdist_gv_estimate).  The network learns corrections to
that estimate: targets (d - d_GV) / 4 and (w* - w*_GV) / 2, so an untrained (zero)
output is the GV estimate itself.
"""

from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _lib as L
from .api import _torch, as_packed, _p64

NFEATURES = 24


def _pf(a):
    return a.ctypes.data_as(L.PF)


def features(G, n: int) -> np.ndarray:
    G = as_packed(G, n)
    k, W = G.shape
    f = np.zeros(NFEATURES, dtype=np.float32)
    L.check(L.lib().mdist_features(_p64(G), int(n), k, W, _pf(f)), "mdist_features")
    return f


def gv_estimate(n: int, k: int, ranks) -> tuple[int, int]:
    r = np.ascontiguousarray(np.asarray(ranks, dtype=np.int32))
    d = ctypes.c_int()
    w = ctypes.c_int()
    L.check(L.lib().mdist_gv_estimate(int(n), int(k), len(r), r.ctypes.data_as(L.PI), ctypes.byref(d),
                                      ctypes.byref(w)), "mdist_gv_estimate")
    return d.value, w.value


def wstar_from_d(k: int, ranks, d: float) -> int:
    """Least g with L(g) = sum_j max(0, g + 1 - (k - r_j)) >= d."""
    for g in range(1, k + 1):
        if sum(max(0, g + 1 - (k - int(r))) for r in ranks) >= d:
            return g
    return k


class MLP:
    """fp32 MLP on the GPU: in -> hidden x layers (ReLU) -> out."""

    def __init__(self, in_features: int = NFEATURES, hidden: int = 64, hidden_layers: int = 3, outputs: int = 2,
                 seed: int = 1, stream=None):
        torch = _torch()
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        L.check(L.lib().mdist_mlp_create(in_features, hidden, hidden_layers, outputs, seed,
                                         ctypes.c_void_p(self._stream.cuda_stream), ctypes.byref(h)),
                "mdist_mlp_create")
        self._h = h
        self.F, self.O = in_features, outputs
        self.hidden, self.hidden_layers = hidden, hidden_layers
        n = ctypes.c_int()
        L.check(L.lib().mdist_mlp_num_params(h, ctypes.byref(n)), "mdist_mlp_num_params")
        self.nparams = n.value

    def close(self):
        if getattr(self, "_h", None):
            L.lib().mdist_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.nparams, dtype=np.float32)
        L.check(L.lib().mdist_mlp_get_params(self._h, _pf(p)), "mdist_mlp_get_params")
        return p

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        assert p.size == self.nparams
        L.check(L.lib().mdist_mlp_set_params(self._h, _pf(p)), "mdist_mlp_set_params")

    def forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
        Y = np.zeros((X.shape[0], self.O), dtype=np.float32)
        L.check(L.lib().mdist_mlp_forward(self._h, _pf(X), X.shape[0], _pf(Y)), "mdist_mlp_forward")
        return Y

    def loss_grad(self, X, T):
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
        T = np.ascontiguousarray(np.asarray(T, dtype=np.float32))
        loss = np.zeros(1, dtype=np.float32)
        g = np.zeros(self.nparams, dtype=np.float32)
        L.check(L.lib().mdist_mlp_loss_grad(self._h, _pf(X), _pf(T), X.shape[0], _pf(loss), _pf(g)),
                "mdist_mlp_loss_grad")
        return float(loss[0]), g

    def train(self, X, T, steps: int = 2000, batch: int = 128, lr: float = 2e-3, seed: int = 7) -> np.ndarray:
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
        T = np.ascontiguousarray(np.asarray(T, dtype=np.float32))
        curve = np.zeros(steps, dtype=np.float32)
        L.check(L.lib().mdist_mlp_train(self._h, _pf(X), _pf(T), X.shape[0], steps, batch, ctypes.c_float(lr), seed,
                                        _pf(curve)), "mdist_mlp_train")
        return curve


class Predictor:
    """w* and d of codes: the trained MLP, or the GV estimate when no model is given."""

    def __init__(self, mlp: MLP | None = None):
        self.mlp = mlp

    D_SCALE = 4.0
    W_SCALE = 2.0

    @staticmethod
    def targets(n: int, k: int, ranks, d: int, wstar: int) -> np.ndarray:
        dg, wg = gv_estimate(n, k, ranks)
        return np.array([(d - dg) / Predictor.D_SCALE, (wstar - wg) / Predictor.W_SCALE], dtype=np.float32)

    def predict(self, feats: np.ndarray, shapes) -> list[tuple[int, int]]:
        """(w*, d) per code; shapes = [(n, k, ranks)]."""
        gv = [gv_estimate(n, k, ranks) for n, k, ranks in shapes]
        if self.mlp is None:
            return [(w, d) for d, w in gv]
        Y = self.mlp.forward(np.asarray(feats, dtype=np.float32).reshape(len(shapes), -1))
        out = []
        for (n, k, ranks), (dg, wg), y in zip(shapes, gv, Y):
            d = max(1, dg + int(round(float(y[0]) * self.D_SCALE)))
            w = max(1, min(k, wg + int(round(float(y[1]) * self.W_SCALE))))
            out.append((w, d))
        return out


def train_predictor(codes, labels, *, hidden=64, hidden_layers=3, steps=3000, batch=128, lr=2e-3, seed=1):
    """codes = [(G, n)], labels = [(d, g_final, ranks)] from the method's own runs."""
    X = np.stack([features(G, n) for G, n in codes])
    T = np.stack([Predictor.targets(n, G.shape[0], r, d, w) for (G, n), (d, w, r) in zip(codes, labels)])
    mlp = MLP(NFEATURES, hidden, hidden_layers, 2, seed=seed)
    curve = mlp.train(X, T, steps=steps, batch=batch, lr=lr, seed=seed + 1)
    return mlp, curve


def errors(pred, truth) -> dict:
    """MAE of d and exact-match rate of w* (pred, truth: lists of (w*, d))."""
    dm = [abs(p[1] - t[1]) for p, t in zip(pred, truth)]
    wm = [p[0] == t[0] for p, t in zip(pred, truth)]
    return {"d_mae": float(np.mean(dm)), "wstar_acc": float(np.mean(wm)), "n": len(truth)}


__all__ = ["features", "gv_estimate", "wstar_from_d", "MLP", "Predictor", "train_predictor", "errors",
           "NFEATURES", "math"]

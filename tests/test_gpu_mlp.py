"""The predictor's MLP kernels against a plain numpy (float64) reference: forward,
backprop gradients, finite differences, and that training lowers the loss."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def predict():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    from paper_1603_06757_gb300 import predict as p

    return p


def _unpack(p, sizes):
    """Layer list [(W (in x out), b)] from the flat parameter vector."""
    out, off = [], 0
    for i, o in sizes:
        W = p[off: off + i * o].reshape(i, o)
        off += i * o
        b = p[off: off + o]
        off += o
        out.append((W, b))
    assert off == p.size
    return out


def _sizes(F, H, layers, O):
    dims = [F] + [H] * layers + [O]
    return list(zip(dims[:-1], dims[1:]))


def np_forward(params, X):
    acts = [X]
    for li, (W, b) in enumerate(params):
        z = acts[-1] @ W + b
        acts.append(np.maximum(z, 0.0) if li + 1 < len(params) else z)
    return acts


def np_loss_grad(params, X, T):
    acts = np_forward(params, X)
    Y = acts[-1]
    n = Y.size
    loss = float(((Y - T) ** 2).sum() / n)
    dY = 2.0 * (Y - T) / n
    grads = []
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        A = acts[li]
        grads.append((A.T @ dY, dY.sum(axis=0)))
        if li > 0:
            dY = (dY @ W.T) * (A > 0)
    grads.reverse()
    return loss, np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def _data(N, F, O, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, size=(N, F)).astype(np.float32)
    T = np.stack([np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2], np.cos(2 * X[:, 3]) - X[:, 4]], axis=1)[:, :O]
    return X, T.astype(np.float32)


@pytest.mark.parametrize("F,H,layers,O", [(24, 64, 3, 2), (7, 16, 1, 3), (5, 8, 0, 1)])
def test_forward_matches_numpy(predict, F, H, layers, O):
    mlp = predict.MLP(F, H, layers, O, seed=3)
    p = mlp.get_params().astype(np.float64)
    X = np.random.default_rng(1).uniform(-1, 1, size=(300, F)).astype(np.float32)
    want = np_forward(_unpack(p, _sizes(F, H, layers, O)), X.astype(np.float64))[-1]
    got = mlp.forward(X)
    assert np.allclose(got, want, rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("F,H,layers,O", [(24, 64, 3, 2), (7, 16, 2, 3)])
def test_gradients_match_backprop_and_finite_differences(predict, F, H, layers, O):
    mlp = predict.MLP(F, H, layers, O, seed=5)
    X, T = _data(200, max(F, 5), 2, seed=2)
    X, T = X[:, :F], np.pad(T, ((0, 0), (0, max(0, O - 2))))[:, :O]
    p = mlp.get_params().astype(np.float64)
    sizes = _sizes(F, H, layers, O)
    loss_np, g_np = np_loss_grad(_unpack(p, sizes), X.astype(np.float64), T.astype(np.float64))
    loss, g = mlp.loss_grad(X, T)
    assert loss == pytest.approx(loss_np, rel=1e-4)
    assert np.allclose(g, g_np, rtol=2e-3, atol=2e-6)
    # central differences of the float64 reference loss at sampled parameters
    rng = np.random.default_rng(9)
    for idx in rng.choice(p.size, size=40, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[idx] += h
        pm[idx] -= h
        lp, _ = np_loss_grad(_unpack(pp, sizes), X.astype(np.float64), T.astype(np.float64))
        lm, _ = np_loss_grad(_unpack(pm, sizes), X.astype(np.float64), T.astype(np.float64))
        fd = (lp - lm) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=5e-3, abs=5e-6)


def test_training_lowers_loss(predict):
    mlp = predict.MLP(8, 32, 2, 2, seed=11)
    X, T = _data(2000, 8, 2, seed=4)
    l0, _ = mlp.loss_grad(X, T)
    curve = mlp.train(X, T, steps=800, batch=128, lr=3e-3, seed=3)
    l1, _ = mlp.loss_grad(X, T)
    assert curve.shape == (800,) and np.all(np.isfinite(curve))
    assert l1 < 0.2 * l0
    # parameters round-trip
    p = mlp.get_params()
    mlp.set_params(p)
    assert np.array_equal(mlp.get_params(), p)

"""Pins for the route-predictor oracle (CPU only): torch autograd in fp64
(a library routine, no code shared) and central finite differences."""
import numpy as np
import pytest

from oracle import mlp


def _batch(B=37, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(B, mlp.IN))
    y = rng.integers(0, 2, size=B)
    t = rng.normal(size=B)
    w = (rng.random(B) < 0.6).astype(np.float64)
    return X, y, t, w


def test_forward_and_gradients_match_torch_autograd():
    torch = pytest.importorskip("torch")
    p = mlp.init_params(3)
    X, y, t, w = _batch()
    act = mlp.forward(p, X)
    g = mlp.backward(p, act, y, t, w)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    tx = torch.tensor(X)
    h1 = torch.relu(tx @ tp["W1"].T + tp["b1"])
    h2 = torch.relu(h1 @ tp["W2"].T + tp["b2"])
    o = h2 @ tp["W3"].T + tp["b3"]
    ce = torch.nn.functional.cross_entropy(o[:, :2], torch.tensor(y), reduction="none")
    L = (ce + mlp.LAMBDA * torch.tensor(w) * (o[:, 2] - torch.tensor(t)) ** 2).mean()
    L.backward()
    assert np.allclose(act["o"], o.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert abs(mlp.loss(act["o"], y, t, w) - L.item()) < 1e-12
    for k in p:
        assert np.allclose(g[k], tp[k].grad.numpy(), rtol=1e-10, atol=1e-12), k


def test_gradients_match_central_differences():
    p = mlp.init_params(5)
    X, y, t, w = _batch(B=9, seed=2)
    g = mlp.backward(p, mlp.forward(p, X), y, t, w)
    rng = np.random.default_rng(0)
    h = 1e-6
    for k in p:
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in p[k].shape)
            old = p[k][idx]
            p[k][idx] = old + h
            lp = mlp.loss(mlp.forward(p, X)["o"], y, t, w)
            p[k][idx] = old - h
            lm = mlp.loss(mlp.forward(p, X)["o"], y, t, w)
            p[k][idx] = old
            num = (lp - lm) / (2 * h)
            assert abs(num - g[k][idx]) < 1e-6 * max(1.0, abs(num)), (k, idx, num, g[k][idx])


def test_adam_decreases_the_loss():
    p = mlp.init_params(7)
    X, y, t, w = _batch(B=64, seed=4)
    st = {}
    l0 = mlp.loss(mlp.forward(p, X)["o"], y, t, w)
    for _ in range(200):
        mlp.adam_step(p, mlp.backward(p, mlp.forward(p, X), y, t, w), st, lr=3e-3)
    assert mlp.loss(mlp.forward(p, X)["o"], y, t, w) < 0.2 * l0


def test_route_features_hand_computed():
    """A star on vertex 16 (degree 10), vertex 0 isolated, pair (32, 33):
    sampled vertices 0, 16, 32 have degrees 0, 10, 1 -> buckets 0, 4, 1; the
    probe from 16 reaches 10 vertices at level 1 and none after."""
    import math

    e = np.array([(16, i) for i in range(1, 11)] + [(32, 33)], dtype=np.int32)
    x = mlp.route_features(e, 40)
    want = np.zeros(69)
    want[[0, 1, 4]] = 1.0 / 3.0
    want[64] = math.log(40) / 20
    want[65] = math.log(12) / 20
    want[66] = math.log(11) / 20
    assert np.allclose(x, want)

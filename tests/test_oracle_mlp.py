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


def _adam(grads, lr=0.1, b1=0.9, b2=0.999, eps=1e-8):
    """Parameter moves of successive Adam steps from zero."""
    p = {"w": np.zeros(len(grads[0]))}
    st, moves = {}, []
    for g in grads:
        before = p["w"].copy()
        mlp.adam_step(p, {"w": np.asarray(g, dtype=np.float64)}, st, lr=lr, b1=b1, b2=b2, eps=eps)
        moves.append(p["w"] - before)
    return moves


def test_adam_first_and_repeated_steps_closed_form():
    """Kingma & Ba, Algorithm 1. From zero moments, the bias-corrected first
    moment after t steps of one constant gradient g is
    (1 - b1) sum_k b1^k g / (1 - b1^t) = g, and the second is g^2 likewise, so
    every step moves a parameter by -lr g / (|g| + eps): -lr sign(g) for
    |g| >> eps, nothing for g = 0, and -lr / 2 for g = eps. Without the bias
    correction the first step would be lr (1 - b1) / sqrt(1 - b2) = 3.16 lr."""
    lr, eps = 0.1, 1e-8
    g = np.array([0.5, -2.0, 0.0, 1e-8])
    want = -lr * g / (np.abs(g) + eps)
    assert np.allclose(want, [-lr, lr, 0.0, -lr / 2], rtol=1e-7)
    for mv in _adam([g, g, g], lr=lr, eps=eps):
        assert np.allclose(mv, want, rtol=1e-9, atol=1e-15), mv


def test_adam_reversed_gradient_closed_form():
    """Gradient g, then -g: m_2 = b1 (1 - b1) g - (1 - b1) g = -(1 - b1)^2 g,
    so m_2 / (1 - b1^2) = -(1 - b1) / (1 + b1) g, while v_2 / (1 - b2^2) = g^2
    still. The second step moves +lr (1 - b1) / (1 + b1) sign(g): 0.1 / 1.9
    of lr for b1 = 0.9. A second moment that tracked g instead of g^2 would
    give a different magnitude, and one without the square root a different
    scale."""
    lr = 0.1
    g = np.array([0.5, -2.0, 3.0])
    m1, m2 = _adam([g, -g], lr=lr)
    assert np.allclose(m1, -lr * g / (np.abs(g) + 1e-8), rtol=1e-9)
    assert np.allclose(m2, lr * (0.1 / 1.9) * g / (np.abs(g) + 1e-8), rtol=1e-9)


def test_adam_is_invariant_to_gradient_scale():
    """Dividing the first moment by the root of the second makes the update
    independent of the gradient's scale (for |g| >> eps), over any sequence."""
    rng = np.random.default_rng(5)
    seq = [rng.normal(size=6) for _ in range(5)]
    a = _adam(seq)
    b = _adam([1000.0 * s for s in seq])
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-6)


def _feature_graph():
    """40 blocks of 256 pairs on n = 4096. Blocks 0, 16 and 32 are the
    sampled ones ((k // 256) % 16 == 0). Filler pairs (1, 2) fill every slot
    not listed; vertices 1 and 2 are not multiples of 16 and are never
    reached from the hub. Slots within a block (in brackets) are spread over
    the block.
      block 0 [253-255]: (32, 100), (32, 101), (32, 102)   level 1 from 32: 3
      block 16 [100, 170, 240]: (100, 200), (101, 201),
                (201, 202)                             level 2: {200, 201}
      block 32 [255, 17]: (200, 203), (203, 700)       level 3: {202, 203};
                                                       700 is level 4, not a feature
      block 1:  (100, 600), block 17: (200, 601)       in unsampled blocks next to
                                                       sampled ones
      block 8:  (101, 801)                             sampled by a rule of 1 in 8
      block 5:  (102, 500); blocks 2-4: (32, 400 + j), j < 20, and (48, 1000 + j), j < 8
      block 6:  a self-loop (64, 64) and the pair (80, 81) twice
    """
    pairs = [(1, 2)] * (40 * 256)
    put = lambda blk, i, pr: pairs.__setitem__(blk * 256 + i, pr)
    for i, v in enumerate((100, 101, 102)):
        put(0, 253 + i, (32, v))
    for i, pr in enumerate([(100, 200), (101, 201), (201, 202)]):
        put(16, 100 + 70 * i, pr)
    put(32, 255, (200, 203))
    put(32, 17, (203, 700))
    put(1, 0, (100, 600))
    put(17, 0, (200, 601))
    put(8, 5, (101, 801))
    put(5, 0, (102, 500))
    for j in range(20):
        put(2 + j // 10, j % 10, (32, 400 + j))
    for j in range(8):
        put(4, j, (48, 1000 + j))
    put(6, 0, (64, 64))
    put(6, 1, (80, 81))
    put(6, 2, (80, 81))
    return np.array(pairs, dtype=np.int64)


def test_route_features_sampled_blocks_and_three_levels():
    """Sampled vertices (ids 0, 16, ..., 4080: 256 of them): 32 has degree
    3 + 20 = 23 (bucket 5) and is the hub; 48 has 8 (bucket 4); 64 (self-loop,
    counted twice) and 80 (a duplicated pair) have 2 (bucket 2); 400 and 416
    have 1 (bucket 1); the other 250 have 0. The probe over the sampled
    blocks reaches 3, 2 and 2 new vertices at levels 1, 2 and 3."""
    import math

    e = _feature_graph()
    x = mlp.route_features(e, 4096)
    want = np.zeros(69)
    want[0] = 250 / 256
    want[1] = 2 / 256
    want[2] = 2 / 256
    want[4] = 1 / 256
    want[5] = 1 / 256
    want[64] = math.log(4096) / 20
    want[65] = math.log(40 * 256 + 1) / 20
    want[66] = math.log(1 + 3) / 20
    want[67] = math.log(1 + 2) / 20
    want[68] = math.log(1 + 2) / 20
    assert np.allclose(x, want, rtol=0, atol=1e-15), np.nonzero(~np.isclose(x, want))

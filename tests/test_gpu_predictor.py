"""Learned route predictor on the GPU: the project's training kernels against
the fp64 oracle, the sampled features against their plain definition, and
the learned route end to end (labels exact whatever it predicts).

Tolerances: the kernels compute in fp32 with sums of up to B * 128 terms, so
relative errors of a few 1e-6 per term and ~1e-4 on the largest entries of a
gradient are expected; the tests use 2e-3 of each array's max magnitude.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import mlp
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"]])


def _unflat(f):
    sizes = [("W1", (128, 69)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (3, 128)), ("b3", (3,))]
    out, o = {}, 0
    for k, shp in sizes:
        c = int(np.prod(shp))
        out[k] = f[o:o + c].reshape(shp)
        o += c
    return out


def _close(a, b, rel=2e-3):
    scale = max(np.abs(b).max(), 1e-6)
    return np.abs(a - b).max() <= rel * scale


def test_forward_backward_adam_match_oracle():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    rng = np.random.default_rng(0)
    p = mlp.init_params(1)
    p["b1"] = rng.normal(scale=0.1, size=128)
    p["b2"] = rng.normal(scale=0.1, size=128)
    p["b3"] = rng.normal(scale=0.1, size=3)
    B = 301
    X = rng.normal(size=(B, mlp.IN))
    y = rng.integers(0, 2, size=B)
    t = rng.normal(size=B)
    w = (rng.random(B) < 0.5).astype(np.float64)
    dev = "cuda"
    P = torch.tensor(_flat(p), dtype=torch.float32, device=dev)
    Xd = torch.tensor(X, dtype=torch.float32, device=dev)
    act = torch.empty(B * (2 * 128 + 3), dtype=torch.float32, device=dev)
    cc.mlp_forward(P, Xd, act)
    ref = mlp.forward(p, X)
    a = act.cpu().numpy()
    assert _close(a[:B * 128].reshape(B, 128), ref["h1"])
    assert _close(a[B * 128:2 * B * 128].reshape(B, 128), ref["h2"])
    assert _close(a[2 * B * 128:].reshape(B, 3), ref["o"])
    grad = torch.zeros(cc.MLP_PARAMS, dtype=torch.float32, device=dev)
    scratch = torch.empty(B * (3 + 2 * 128), dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    cc.mlp_backward(P, Xd, torch.tensor(y, dtype=torch.int32, device=dev), torch.tensor(t, dtype=torch.float32, device=dev),
                    torch.tensor(w, dtype=torch.float32, device=dev), mlp.LAMBDA, act, grad, scratch, loss)
    g_ref = mlp.backward(p, ref, y, t, w)
    g = _unflat(grad.cpu().numpy().astype(np.float64))
    for k in g_ref:
        assert _close(g[k], g_ref[k]), k
    assert abs(loss.item() - mlp.loss(ref["o"], y, t, w)) < 1e-4 * max(1.0, abs(mlp.loss(ref["o"], y, t, w)))
    # one Adam step from the oracle's gradients
    gd = torch.tensor(_flat(g_ref), dtype=torch.float32, device=dev)
    mm = torch.zeros_like(P)
    vv = torch.zeros_like(P)
    cc.mlp_adam(P, gd, mm, vv, 1e-3, 1)
    st = {}
    mlp.adam_step(p, g_ref, st, lr=1e-3)
    assert np.allclose(P.cpu().numpy(), _flat(p), atol=2e-6)


@pytest.mark.parametrize("maker", [
    lambda: gg.rmat(seed=2, scale=15, edge_factor=8),
    lambda: gg.chung_lu(seed=3, n=40000, avg_degree=6),
    lambda: gg.grid_chains(seed=4, W=150, nchains=3000, id_bytes=8),
])
def test_route_features_match_definition(maker):
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    g = maker()
    eng = cc.Engine(id_bytes=g.id_bytes)
    x = eng.route_features(torch.from_numpy(g.edges).cuda(), g.n).cpu().numpy()
    eng.close()
    assert np.allclose(x, mlp.route_features(g.edges, g.n), atol=1e-6)


def test_route_features_on_the_hand_built_graph():
    """The graph whose features the oracle test checks by hand: sampled and
    unsampled blocks of pairs, three BFS levels and a fourth that must not
    count, a self-loop and a duplicated pair."""
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc
    from tests.test_oracle_mlp import _feature_graph

    e = _feature_graph().astype(np.int32)
    eng = cc.Engine(id_bytes=4)
    x = eng.route_features(torch.from_numpy(e).cuda(), 4096).cpu().numpy()
    eng.close()
    assert np.allclose(x, mlp.route_features(e, 4096), atol=1e-6)


def test_learned_route_labels_exact_and_fallback():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    rng = np.random.default_rng(1)
    params = _flat(mlp.init_params(2)).astype(np.float32)
    for g in (gg.rmat(seed=5, scale=16, edge_factor=8), gg.chung_lu(seed=6, n=1 << 15, avg_degree=8),
              gg.planted(seed=7, n=30000, ncomp=200)):
        want = oracle.cc_labels(g.edges, g.n)
        e = torch.from_numpy(g.edges).cuda()
        for conf in (0.0, 1.0):  # 0: always trust the network; 1: always fall back to K-S
            for bias in (-5.0, 5.0):  # push the route logits towards SV / BFS
                p = params.copy()
                p[-3] = -bias
                p[-2] = bias
                eng = cc.Engine(id_bytes=g.id_bytes, route="learned")
                eng.set_predictor(p, min_confidence=conf)
                lab = eng.labels(e, g.n).cpu().numpy().astype(np.int64)
                st = eng.stats()
                eng.close()
                assert np.array_equal(lab, want)
                if conf == 0.0:
                    assert st["route_source"] == 1 and st["route"] == st["pred_route"]
                else:
                    assert st["route_source"] == 0
    del rng


def test_trained_predictor_gains_over_the_heuristic():
    """The committed network (trained on 20,000 seeded graphs) against the
    K-S heuristic on graphs it was not trained on (another seed): labels
    equal to the oracle's on every graph, and less total time. The learned route reads a
    1/16 vertex sample instead of the exact degree pass and K-S fit."""
    torch_cuda()
    from paper_1607_06156_gb300.train_predictor import default_weights_path, evaluate, load_params

    params, n_train = load_params(default_weights_path())
    assert n_train >= 20000
    check = lambda e, n, lab: np.array_equal(oracle.labels_uf(e, n), lab.astype(np.int64))
    summ = evaluate(params, count=30, seed=777, big=0, log=lambda *a, **k: None, check=check)
    assert summ["labels_equal"] and all(r["checked"] for r in summ["rows"])
    assert summ["gain_learned_over_heuristic"] > 1.1, summ["gain_learned_over_heuristic"]

"""Route-predictor network in fp64 numpy (oracle for the CUDA training kernels).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The learned route predictor replaces the paper's K-S threshold (Section 3.2,
Table 2) only in choosing between BFS-then-SV and SV only, and the BFS
cutoff; labels never depend on it. Network (the plain definition):

    h1 = relu(W1 x + b1)           W1: [128, 69]
    h2 = relu(W2 h1 + b2)          W2: [128, 128]
    o  = W3 h2 + b3                W3: [3, 128]
    o[0:2] route logits (0 = SV only, 1 = BFS first), o[2] = log BFS cutoff

Loss of a batch (mean over its B samples):

    L = 1/B sum_b [ -log softmax(o_b[0:2])[y_b] + lam * w_b * (o_b[2] - t_b)^2 ]

with y_b the fastest route, t_b the log of the best cutoff and w_b = 1 when
the BFS route won (the cutoff only matters then), else 0.
"""
from __future__ import annotations

import numpy as np

IN, HID, OUT = 69, 128, 3
LAMBDA = 0.1


def init_params(seed: int = 0, dtype=np.float64) -> dict:
    """He-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)

    def he(fan_out, fan_in):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=(fan_out, fan_in)).astype(dtype)

    return {"W1": he(HID, IN), "b1": np.zeros(HID, dtype), "W2": he(HID, HID), "b2": np.zeros(HID, dtype),
            "W3": he(OUT, HID), "b3": np.zeros(OUT, dtype)}


def forward(p: dict, X: np.ndarray) -> dict:
    """Activations of every layer for inputs X [B, 69]."""
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    o = h2 @ p["W3"].T + p["b3"]
    return {"X": X, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "o": o}


def loss(o: np.ndarray, y: np.ndarray, t: np.ndarray, w: np.ndarray, lam: float = LAMBDA) -> float:
    logits = o[:, :2]
    mx = logits.max(axis=1, keepdims=True)
    lse = mx[:, 0] + np.log(np.exp(logits - mx).sum(axis=1))
    ce = lse - logits[np.arange(len(y)), y]
    return float(np.mean(ce + lam * w * (o[:, 2] - t) ** 2))


def backward(p: dict, act: dict, y: np.ndarray, t: np.ndarray, w: np.ndarray, lam: float = LAMBDA) -> dict:
    """Gradients of the batch-mean loss with respect to every parameter."""
    o = act["o"]
    B = o.shape[0]
    logits = o[:, :2]
    e = np.exp(logits - logits.max(axis=1, keepdims=True))
    sm = e / e.sum(axis=1, keepdims=True)
    do = np.zeros_like(o)
    do[:, :2] = sm
    do[np.arange(B), y] -= 1.0
    do[:, 2] = 2.0 * lam * w * (o[:, 2] - t)
    do /= B
    g = {"W3": do.T @ act["h2"], "b3": do.sum(axis=0)}
    dz2 = (do @ p["W3"]) * (act["z2"] > 0)
    g["W2"] = dz2.T @ act["h1"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (act["z1"] > 0)
    g["W1"] = dz1.T @ act["X"]
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(p: dict, g: dict, state: dict, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update (Kingma & Ba 2015) with bias correction, in place."""
    state["t"] = state.get("t", 0) + 1
    tt = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** tt)
        vh = v / (1 - b2 ** tt)
        p[k] -= lr * mh / (np.sqrt(vh) + eps)


def route_features(edges: np.ndarray, n: int) -> np.ndarray:
    """The predictor's 69 input features, by their plain definition.

    [0, 64)  log2-degree histogram (bucket 0: degree 0, bucket b: degrees in
             [2^(b-1), 2^b)) of the vertices whose id is a multiple of 16, as
             fractions of those vertices (degrees count both pair ends)
    64, 65   ln(n)/20, ln(m+1)/20
    66..68   ln(1 + new vertices)/20 at BFS levels 1..3 from the sampled
             vertex of highest degree (ties: smallest id), over the pairs in
             every 16th block of 256 pairs (pair k is used iff (k // 256) % 16 == 0)
    """
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    m = e.shape[0]
    deg = np.bincount(e.ravel(), minlength=n)[:n] if m else np.zeros(n, dtype=np.int64)
    sampled = np.arange(0, n, 16)
    sd = deg[sampled]
    x = np.zeros(IN, dtype=np.float64)
    buckets = np.where(sd == 0, 0, np.floor(np.log2(np.maximum(sd, 1))).astype(np.int64) + 1)
    buckets = np.minimum(buckets, 63)
    x[:64] = np.bincount(buckets, minlength=64)[:64] / sampled.size
    x[64] = np.log(n) / 20.0
    x[65] = np.log(m + 1.0) / 20.0
    seed = int(sampled[int(np.argmax(sd))]) if sampled.size else 0
    k = np.arange(m)
    sp = e[(k // 256) % 16 == 0]
    adj = {}
    for u, v in sp.tolist():
        adj.setdefault(u, []).append(v)
        adj.setdefault(v, []).append(u)
    visited = {seed}
    front = {seed}
    for level in range(3):
        nxt = set()
        for u in front:
            for v in adj.get(u, ()):
                if v not in visited:
                    visited.add(v)
                    nxt.add(v)
        x[66 + level] = np.log1p(len(nxt)) / 20.0
        front = nxt
    return x

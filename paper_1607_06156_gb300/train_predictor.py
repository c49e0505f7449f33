"""Trains and evaluates the learned route predictor of the engine.

The predictor replaces the K-S threshold of Section 3.2 (Table 2) only in
choosing BFS first vs SV only and the BFS cutoff; the K-S heuristic stays as
fallback when the network is unsure. Labels never depend on the route.

  collect   seeded graphs from five families (R-MAT, Chung-Lu power law,
            percolated grid + chains, planted small components, chain
            forests); for each: the device features (cc_route_features) and
            the measured time of SV only and of BFS first with cutoffs
            2, 4, 8, 16 and none (median of timed runs after a warm-up)
  train     the fp32 network on the GPU with the library's own kernels
            (cc_mlp_forward / cc_mlp_backward / cc_mlp_adam), with a
            checkpoint every few epochs (params, Adam moments, step) that
            --resume picks up
  evaluate  on held-out graphs: the heuristic route vs the learned route
            (median time of each, labels compared), aggregate pairs/s

Weights file: magic b"CCRP", uint32 version, uint32 parameter count, uint32
training graphs, float32 parameters, uint32 CRC-32 of everything before it.

Usage (on a GPU host):
  python -m paper_1607_06156_gb300.train_predictor --train 1200 --heldout 200 \
      --out paper_1607_06156_gb300/route_predictor.bin --summary summary.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import struct
import sys
import time
import zlib

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MAGIC, VERSION = b"CCRP", 1
CUTOFFS = (2, 4, 8, 16, 0)  # 0 = BFS to completion
NO_CUTOFF_LEVELS = 64.0     # the log-cutoff target standing for "no cutoff"
LAMBDA = 0.1


# ---------------------------------------------------------------------------
def save_params(path: str, params: np.ndarray, n_train: int) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    body = MAGIC + struct.pack("<III", VERSION, p.size, n_train) + p.tobytes()
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(body + struct.pack("<I", zlib.crc32(body) & 0xffffffff))
    os.replace(tmp, path)


def load_params(path: str) -> tuple[np.ndarray, int]:
    data = open(path, "rb").read()
    body, crc = data[:-4], struct.unpack("<I", data[-4:])[0]
    if body[:4] != MAGIC or (zlib.crc32(body) & 0xffffffff) != crc:
        raise ValueError(f"{path}: not a route-predictor file or corrupted")
    version, count, n_train = struct.unpack("<III", body[4:16])
    if version != VERSION:
        raise ValueError(f"{path}: version {version}, expected {VERSION}")
    return np.frombuffer(body[16:], dtype=np.float32, count=count).copy(), n_train


def default_weights_path() -> str:
    return os.path.join(HERE, "route_predictor.bin")


# ---------------------------------------------------------------------------
def make_graph(rng: np.random.Generator, family: str, big: bool = False):
    import graphgen as gg

    seed = int(rng.integers(1, 2 ** 40))
    if family == "rmat":
        scale = int(rng.integers(12, 23 if big else 20))
        ef = int(rng.choice([4, 8, 16]))
        a, b, c = [(0.57, 0.19, 0.19), (0.45, 0.25, 0.15), (0.5, 0.2, 0.2), (0.6, 0.15, 0.15)][int(rng.integers(4))]
        return gg.rmat(seed=seed, scale=scale, edge_factor=ef, a=a, b=b, c=c)
    if family == "chung_lu":
        n = int(2 ** rng.uniform(12, 21 if big else 20))
        return gg.chung_lu(seed=seed, n=n, avg_degree=float(rng.choice([2, 4, 8, 16])), alpha=float(rng.uniform(2.0, 3.2)))
    if family == "grid_chains":
        W = int(2 ** rng.uniform(6, 12 if big else 10.5))
        return gg.grid_chains(seed=seed, W=W, p=float(rng.uniform(0.4, 0.7)),
                              nchains=int(rng.choice([0, 1000, 10000, 100000])), id_bytes=4)
    if family == "planted":
        n = int(2 ** rng.uniform(12, 20))
        return gg.planted(seed=seed, n=n, ncomp=int(min(n // 8, 2 ** rng.uniform(3, 13))),
                          extra_per_vertex=float(rng.uniform(0.3, 3.0)))
    if family == "chains":
        return gg.grid_chains(seed=seed, W=1, nchains=int(2 ** rng.uniform(8, 17)), id_bytes=4)
    raise ValueError(family)


FAMILIES = ("rmat", "chung_lu", "grid_chains", "planted", "chains")


def constant_params(route: int, cutoff: int) -> np.ndarray:
    """A network whose output ignores its input: route logits and log cutoff fixed."""
    p = np.zeros(128 * 69 + 128 + 128 * 128 + 128 + 3 * 128 + 3, dtype=np.float32)
    p[-3], p[-2] = (10.0, -10.0) if route == 0 else (-10.0, 10.0)
    p[-1] = math.log(cutoff if cutoff > 0 else NO_CUTOFF_LEVELS)
    return p


class Timer:
    """Median device time of one cc_labels call per route configuration.

    The candidate routes are timed exactly as the learned policy runs them
    (sampled features, network, then the chosen route without the exact
    degree pass): learned engines whose network is a constant."""

    def __init__(self, torch, cc, id_bytes: int = 4):
        self.torch, self.cc = torch, cc
        self.eng = {"auto": cc.Engine(id_bytes=id_bytes, route="auto")}
        sv = cc.Engine(id_bytes=id_bytes, route="learned")
        sv.set_predictor(constant_params(0, 0), min_confidence=0.0)
        self.eng["sv"] = sv
        for L in CUTOFFS:
            e = cc.Engine(id_bytes=id_bytes, route="learned")
            e.set_predictor(constant_params(1, L), min_confidence=0.0)
            self.eng[f"bfs{L}"] = e
        self.feat = cc.Engine(id_bytes=id_bytes)

    def time(self, key_or_engine, edges, n: int, out, reps: int = 3) -> float:
        torch = self.torch
        eng = self.eng[key_or_engine] if isinstance(key_or_engine, str) else key_or_engine
        eng.labels(edges, n, out=out)  # warm-up (workspace growth happens here)
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            eng.labels(edges, n, out=out)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    def close(self):
        for e in self.eng.values():
            e.close()
        self.feat.close()


def collect(count: int, seed: int, big: bool = False, log=print) -> dict:
    import torch

    import paper_1607_06156_gb300 as cc

    rng = np.random.default_rng(seed)
    timer = Timer(torch, cc)
    X, T, meta = [], [], []
    t0 = time.time()
    for i in range(count):
        fam = FAMILIES[i % len(FAMILIES)]
        g = make_graph(rng, fam, big=big)
        e = torch.from_numpy(g.edges).cuda()
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        x = timer.feat.route_features(e, g.n).cpu().numpy()
        times = [timer.time("sv", e, g.n, out)] + [timer.time(f"bfs{L}", e, g.n, out) for L in CUTOFFS]
        X.append(x)
        T.append(times)
        meta.append({"family": fam, "name": g.name, "n": g.n, "m": g.m})
        del e, out
        if (i + 1) % 50 == 0:
            log(f"collected {i + 1}/{count} graphs in {time.time() - t0:.0f} s")
    timer.close()
    return {"X": np.array(X, dtype=np.float32), "T": np.array(T, dtype=np.float64), "meta": meta}


def targets(T: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """y = fastest route (0 SV, 1 BFS), t = ln(best cutoff), w = 1 where BFS won."""
    best_bfs = T[:, 1:].argmin(axis=1)
    y = (T[np.arange(len(T)), 1 + best_bfs] < T[:, 0]).astype(np.int32)
    L = np.array([CUTOFFS[k] if CUTOFFS[k] > 0 else NO_CUTOFF_LEVELS for k in best_bfs], dtype=np.float64)
    return y, np.log(L).astype(np.float32), y.astype(np.float32)


def train(X: np.ndarray, y: np.ndarray, t: np.ndarray, w: np.ndarray, epochs: int = 400, batch: int = 256,
          lr: float = 2e-3, seed: int = 0, ckpt: str | None = None, resume: bool = False, log=print) -> np.ndarray:
    """Adam on the GPU with the library's kernels; returns fp32 parameters."""
    import torch

    import paper_1607_06156_gb300 as cc

    dev = "cuda"
    P = torch.tensor(init_params(seed), dtype=torch.float32, device=dev)
    M, V = torch.zeros_like(P), torch.zeros_like(P)
    step, start = 0, 0
    if resume and ckpt and os.path.exists(ckpt):
        d = np.load(ckpt)
        P.copy_(torch.from_numpy(d["P"]))
        M.copy_(torch.from_numpy(d["M"]))
        V.copy_(torch.from_numpy(d["V"]))
        step, start = int(d["step"]), int(d["epoch"])
        log(f"resumed from {ckpt} at epoch {start}")
    Xd = torch.tensor(X, dtype=torch.float32, device=dev)
    yd = torch.tensor(y, dtype=torch.int32, device=dev)
    td = torch.tensor(t, dtype=torch.float32, device=dev)
    wd = torch.tensor(w, dtype=torch.float32, device=dev)
    N = X.shape[0]
    grad = torch.zeros_like(P)
    act = torch.empty(batch * (2 * cc.MLP_HIDDEN + cc.MLP_OUT), dtype=torch.float32, device=dev)
    scratch = torch.empty(batch * (3 + 2 * cc.MLP_HIDDEN), dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    rng = np.random.default_rng(seed + start)
    for ep in range(start, epochs):
        order = torch.from_numpy(rng.permutation(N)).to(dev)
        loss.zero_()
        for b0 in range(0, N, batch):
            idx = order[b0:b0 + batch]
            B = idx.numel()
            xb, yb, tb, wb = Xd[idx].contiguous(), yd[idx].contiguous(), td[idx].contiguous(), wd[idx].contiguous()
            cc.mlp_forward(P, xb, act[:B * (2 * cc.MLP_HIDDEN + cc.MLP_OUT)])
            cc.mlp_backward(P, xb, yb, tb, wb, LAMBDA, act, grad, scratch, loss)
            step += 1
            cc.mlp_adam(P, grad, M, V, lr, step)
        if ckpt and ((ep + 1) % 50 == 0 or ep + 1 == epochs):
            np.savez(ckpt, P=P.cpu().numpy(), M=M.cpu().numpy(), V=V.cpu().numpy(), step=step, epoch=ep + 1)
        if (ep + 1) % 50 == 0:
            log(f"epoch {ep + 1}: mean batch loss {loss.item() / math.ceil(N / batch):.4f}")
    return P.cpu().numpy()


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights, zero biases, in the flat parameter layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((128, 69), (128, 128), (3, 128)):
        lim = math.sqrt(6.0 / fan_in)
        parts += [rng.uniform(-lim, lim, size=fan_out * fan_in), np.zeros(fan_out)]
    return np.concatenate(parts).astype(np.float32)


def predict_routes(params: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Route chosen by the network (argmax of the two logits) with the library's forward kernel."""
    import torch

    import paper_1607_06156_gb300 as cc

    P = torch.tensor(params, dtype=torch.float32, device="cuda")
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    act = torch.empty(X.shape[0] * (2 * cc.MLP_HIDDEN + cc.MLP_OUT), dtype=torch.float32, device="cuda")
    cc.mlp_forward(P, Xd, act)
    O = act[2 * X.shape[0] * cc.MLP_HIDDEN:].view(-1, 3).cpu().numpy()
    return (O[:, 1] > O[:, 0]).astype(np.int32)


def evaluate(params: np.ndarray, count: int, seed: int, big: int = 0, min_conf: float = 0.75, log=print,
             check=None) -> dict:
    """Heuristic vs learned route on held-out graphs (labels must agree).

    `check(edges, n, labels)`, when given, is called with every graph's
    learned-route labels (host int32) and must return True: the caller's
    independent reference for the labels (the tests pass the CPU oracle)."""
    import torch

    import paper_1607_06156_gb300 as cc

    rng = np.random.default_rng(seed)
    timer = Timer(torch, cc)
    learned = cc.Engine(id_bytes=4, route="learned")
    learned.set_predictor(params, min_confidence=min_conf)
    rows = []
    graphs = [(FAMILIES[i % len(FAMILIES)], False) for i in range(count)]
    graphs += [("rmat", True), ("grid_chains", True)] * big
    for i, (fam, is_big) in enumerate(graphs):
        if is_big and fam == "rmat":
            import graphgen as gg
            g = gg.rmat(seed=int(rng.integers(1, 2 ** 40)), scale=22, edge_factor=16)
        elif is_big:
            import graphgen as gg
            g = gg.grid_chains(seed=int(rng.integers(1, 2 ** 40)), W=4096, p=0.55, nchains=0, id_bytes=4)
        else:
            g = make_graph(rng, fam)
        e = torch.from_numpy(g.edges).cuda()
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        t_auto = timer.time("auto", e, g.n, out)
        lab_auto = out.clone()
        t_learn = timer.time(learned, e, g.n, out)
        st = learned.stats()
        same = bool(torch.equal(lab_auto, out))
        if check is not None:
            same = same and bool(check(g.edges, g.n, out.cpu().numpy()))
        t_sv = timer.time("sv", e, g.n, out)
        t_bfs = timer.time("bfs0", e, g.n, out)
        rows.append({"family": fam, "big": is_big, "n": g.n, "m": g.m, "t_heuristic": t_auto, "t_learned": t_learn,
                     "t_sv": t_sv, "t_bfs": t_bfs, "checked": check is not None, "learned_route": st["route"], "route_source": st["route_source"],
                     "confidence": st["pred_confidence"], "labels_equal": same})
        if not same:
            raise SystemExit(f"learned route labels differ from the heuristic route or the reference on {g.name}")
        del e, out
    learned.close()
    timer.close()
    m = np.array([r["m"] for r in rows], dtype=np.float64)
    th = np.array([r["t_heuristic"] for r in rows])
    tl = np.array([r["t_learned"] for r in rows])
    tb = np.minimum([r["t_sv"] for r in rows], [r["t_bfs"] for r in rows])
    summ = {"graphs": len(rows), "pairs_per_s_heuristic": m.sum() / (th.sum() / 1e3),
            "pairs_per_s_learned": m.sum() / (tl.sum() / 1e3), "pairs_per_s_best_forced": m.sum() / (tb.sum() / 1e3),
            "gain_learned_over_heuristic": th.sum() / tl.sum(), "labels_equal": all(r["labels_equal"] for r in rows),
            "per_family": {}}
    for fam in sorted(set(r["family"] + ("_big" if r["big"] else "") for r in rows)):
        sel = [r for r in rows if r["family"] + ("_big" if r["big"] else "") == fam]
        summ["per_family"][fam] = {"graphs": len(sel), "t_heuristic_ms": sum(r["t_heuristic"] for r in sel),
                                   "t_learned_ms": sum(r["t_learned"] for r in sel),
                                   "learned_routes_bfs": sum(r["learned_route"] for r in sel),
                                   "fallbacks": sum(r["route_source"] == 0 for r in sel)}
    summ["rows"] = rows
    return summ


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=1200)
    ap.add_argument("--heldout", type=int, default=200)
    ap.add_argument("--big", type=int, default=1, help="pairs of large held-out graphs (R-MAT 22, 4096^2 grid)")
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--out", default=default_weights_path())
    ap.add_argument("--data", default=None, help="save / reuse the collected training set (.npz)")
    ap.add_argument("--ckpt", default=None)
    ap.add_argument("--resume", action="store_true")
    ap.add_argument("--summary", default=None)
    args = ap.parse_args()
    if args.data and os.path.exists(args.data):
        d = np.load(args.data)
        X, T = d["X"], d["T"]
    else:
        ds = collect(args.train, args.seed)
        X, T = ds["X"], ds["T"]
        if args.data:
            np.savez(args.data, X=X, T=T)
    y, t, w = targets(T)
    print(f"training set: {len(y)} graphs, BFS fastest on {int(y.sum())}", flush=True)
    params = train(X, y, t, w, epochs=args.epochs, seed=args.seed, ckpt=args.ckpt, resume=args.resume)
    save_params(args.out, params, len(y))
    r = predict_routes(params, X)
    summ = evaluate(params, args.heldout, args.seed + 1, big=args.big)
    summ["train_accuracy"] = float((r == y).mean())
    summ["train_graphs"] = int(len(y))
    summ["train_bfs_fastest"] = int(y.sum())
    print(json.dumps({k: v for k, v in summ.items() if k != "rows"}, indent=1), flush=True)
    if args.summary:
        json.dump(summ, open(args.summary, "w"), indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())

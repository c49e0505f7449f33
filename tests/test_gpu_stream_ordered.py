"""cc_labels is stream-ordered: the route decision, the BFS levels and the SV
iterations are all taken on the device (conditional nodes of one CUDA
graph), so the call returns once its work is enqueued, and it can be
captured into the caller's CUDA graph and replayed on new inputs of the same
shape (Algorithm 2 with no host round trip).

Graphs of the same (n, m) that take different routes: a power-law graph
(Chung-Lu, BFS first under the K-S heuristic) and uniform random pairs over
the same vertices (SV only)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _pair_of_graphs(id_bytes=4):
    g = gg.chung_lu(seed=3, n=1 << 16, avg_degree=8, alpha=2.3)
    rng = np.random.default_rng(9)
    dt = np.int32 if id_bytes == 4 else np.int64
    uni = rng.integers(0, g.n, size=(g.m, 2)).astype(dt)
    return g.n, g.edges.astype(dt), uni


def _check(lab, edges, n):
    assert np.array_equal(lab.cpu().numpy().astype(np.int64), oracle.cc_labels(edges, n))


def test_call_returns_before_the_labels_are_ready():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    n, e_bfs, _ = _pair_of_graphs()
    eng = cc.Engine()
    e = torch.from_numpy(e_bfs).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    eng.labels(e, n, out=out)  # sizes the workspace and captures the route once
    eng.check()
    side = torch.cuda.Stream()
    done = torch.cuda.Event()
    out.fill_(-1)
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        torch.cuda._sleep(200_000_000)  # keeps the stream busy well past the host call
        eng.labels(e, n, out=out, stream=side)
        done.record(side)
    assert not done.query(), "cc_labels waited for its stream"
    done.synchronize()
    eng.check()
    _check(out, e_bfs, n)
    st = eng.stats()
    assert st["route"] == 1 and st["status"] == 0
    eng.close()


@pytest.mark.parametrize("route,extra", [("auto", {}), ("auto", {"bfs_mode": 1}), ("sv", {}), ("bfs", {})])
def test_captured_into_a_cuda_graph_and_replayed_on_new_inputs(route, extra):
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    n, e_bfs, e_uni = _pair_of_graphs()
    eng = cc.Engine(route=route, **extra)
    edges = torch.from_numpy(e_bfs).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    # warm-up outside the capture: the workspace is sized for this shape
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        eng.labels(edges, n, out=out)
    torch.cuda.current_stream().wait_stream(s)
    eng.check()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        eng.labels(edges, n, out=out)
    routes = []
    for src in (e_bfs, e_uni, e_bfs):
        edges.copy_(torch.from_numpy(src))
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        _check(out, src, n)
        st = eng.stats()
        assert st["status"] == 0
        routes.append(st["route"])
    if route == "auto":
        assert routes == [1, 0, 1]  # the device took a different branch per input
    else:
        assert len(set(routes)) == 1
    del g
    eng.close()


def test_learned_route_captured():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc
    from paper_1607_06156_gb300.train_predictor import default_weights_path, load_params

    trained, _ = load_params(default_weights_path())
    unsure = np.zeros_like(trained)  # equal route logits: probability 0.5, below the 0.75 threshold
    n, e_bfs, e_uni = _pair_of_graphs()
    for params, conf in ((trained, 0.0), (unsure, 0.75)):  # trust the network / fall back to the K-S heuristic
        eng = cc.Engine(route="learned")
        eng.set_predictor(params, min_confidence=conf)
        edges = torch.from_numpy(e_uni).cuda()
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        eng.labels(edges, n, out=out)
        eng.check()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            eng.labels(edges, n, out=out)
        for src in (e_uni, e_bfs):
            edges.copy_(torch.from_numpy(src))
            g.replay()
            torch.cuda.synchronize()
            _check(out, src, n)
            st = eng.stats()
            assert st["route_source"] == (1 if conf == 0.0 else 0)
        del g
        eng.close()


def test_capture_needs_a_sized_workspace():
    """Inside a capture nothing may allocate: a first call at a new size is refused."""
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    n, e_bfs, _ = _pair_of_graphs()
    eng = cc.Engine()
    edges = torch.from_numpy(e_bfs).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    g = torch.cuda.CUDAGraph()
    with pytest.raises(cc.CCError) as ei:
        with torch.cuda.graph(g):
            eng.labels(edges, n, out=out)
    assert ei.value.status == 7  # CC_ERR_UNSUPPORTED
    del g
    # after a call outside the capture the same shape captures
    eng.labels(edges, n, out=out)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        eng.labels(edges, n, out=out)
    g.replay()
    torch.cuda.synchronize()
    _check(out, e_bfs, n)
    eng.close()


# ---------------------------------------------------------------------------
# The batched form: the offsets stay on the device, the per-graph routes, the
# overflow fallback of the fits and the BFS step of the routed graphs are
# decided on the device.

def _batch_pair():
    """Two batches of the same shape (G, pairs and vertices per graph) with
    different graphs: power-law graphs (BFS under the K-S heuristic) in the
    first, uniform random pairs over the same vertices in the second."""
    sizes = [3000, 1 << 14, 500, 1 << 15, 7000]
    first = [gg.chung_lu(seed=20 + i, n=s, avg_degree=8, alpha=2.3).edges for i, s in enumerate(sizes)]
    rng = np.random.default_rng(21)
    second = [rng.integers(0, s, size=e.shape).astype(np.int32) for s, e in zip(sizes, first)]
    eo = np.concatenate([[0], np.cumsum([e.shape[0] for e in first])]).astype(np.int64)
    vo = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return sizes, np.concatenate(first).astype(np.int32), np.concatenate(second), eo, vo


def _check_batch(out, edges, eo, vo, sizes):
    got = out.cpu().numpy().astype(np.int64)
    for g, n in enumerate(sizes):
        want = oracle.cc_labels(np.ascontiguousarray(edges[eo[g]:eo[g + 1]]), n)
        assert np.array_equal(got[vo[g]:vo[g + 1]], want), g


@pytest.mark.parametrize("route", ["auto", "sv", "bfs"])
def test_batched_captured_and_replayed(route):
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    sizes, e1, e2, eo, vo = _batch_pair()
    eng = cc.Engine(route=route)
    edges = torch.from_numpy(e1).cuda()
    eo_d, vo_d = torch.from_numpy(eo).cuda(), torch.from_numpy(vo).cuda()
    m, n = int(eo[-1]), int(vo[-1])
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    eng.labels_batched_dev(edges, eo_d, vo_d, m, n, out)
    eng.check()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        eng.labels_batched_dev(edges, eo_d, vo_d, m, n, out)
    routed = []
    for src in (e1, e2, e1):
        edges.copy_(torch.from_numpy(src))
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        _check_batch(out, src, eo, vo, sizes)
        st = eng.stats()
        assert st["status"] == 0
        routed.append(st["route"])
    if route == "auto":
        assert routed[0] > 0 and routed[1] == 0 and routed[2] == routed[0]
    elif route == "bfs":
        assert routed == [len(sizes)] * 3
    else:
        assert routed == [0, 0, 0]
    del g
    eng.close()


def test_batched_returns_before_the_labels_are_ready():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    sizes, e1, _, eo, vo = _batch_pair()
    eng = cc.Engine()
    edges = torch.from_numpy(e1).cuda()
    eo_d, vo_d = torch.from_numpy(eo).cuda(), torch.from_numpy(vo).cuda()
    m, n = int(eo[-1]), int(vo[-1])
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    eng.labels_batched_dev(edges, eo_d, vo_d, m, n, out)
    eng.check()
    side, done = torch.cuda.Stream(), torch.cuda.Event()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        torch.cuda._sleep(200_000_000)
        eng.labels_batched_dev(edges, eo_d, vo_d, m, n, out, stream=side)
        done.record(side)
    assert not done.query(), "cc_labels_batched waited for its stream"
    done.synchronize()
    eng.check()
    _check_batch(out, e1, eo, vo, sizes)
    eng.close()


@pytest.mark.parametrize("bad", ["decreasing", "wrong_total", "first_not_zero"])
def test_batched_offsets_checked_on_the_device(bad):
    """Offsets that are not non-decreasing from 0 to the totals give
    CC_ERR_INVALID_ARG from the device status; no kernel indexes with them,
    and the context stays usable."""
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    sizes, e1, _, eo, vo = _batch_pair()
    eo_bad, vo_bad = eo.copy(), vo.copy()
    if bad == "decreasing":
        eo_bad[2] = eo_bad[3] + 5
    elif bad == "wrong_total":
        vo_bad[-1] += 1000
    else:
        eo_bad[0] = 7
    eng = cc.Engine()
    edges = torch.from_numpy(e1).cuda()
    m, n = int(eo[-1]), int(vo[-1])
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    eng.labels_batched_dev(edges, torch.from_numpy(eo_bad).cuda(), torch.from_numpy(vo_bad).cuda(), m, n, out)
    with pytest.raises(cc.CCError) as ei:
        eng.check()
    assert ei.value.status == 1
    eng.labels_batched_dev(edges, torch.from_numpy(eo).cuda(), torch.from_numpy(vo).cuda(), m, n, out)
    eng.check()
    _check_batch(out, e1, eo, vo, sizes)
    eng.close()

"""Helpers shared by the GPU tests: run the engine on numpy edges, compare with the oracle."""
import numpy as np

import oracle


def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        import pytest

        pytest.skip("no CUDA device")
    return torch


def run_engine(edges: np.ndarray, n: int, route: str = "auto", **opts):
    """Labels from the CUDA engine (as int64 numpy) and the engine's stats."""
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    id_bytes = edges.dtype.itemsize
    eng = cc.Engine(id_bytes=id_bytes, route=route, **opts)
    try:
        e = torch.from_numpy(np.ascontiguousarray(edges)).cuda()
        lab = eng.labels(e, n)
        torch.cuda.synchronize()
        assert lab.dtype.itemsize == id_bytes
        return lab.cpu().numpy().astype(np.int64), eng.stats()
    finally:
        eng.close()


def assert_labels_match(edges: np.ndarray, n: int, want=None, routes=("auto", "sv", "bfs"), **opts):
    if want is None:
        want = oracle.cc_labels(edges, n)
    out = {}
    for r in routes:
        got, st = run_engine(edges, n, route=r, **opts)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, f"route={r}: {bad.size} labels differ, first at v={bad[:5]} got={got[bad[:5]]} want={want[bad[:5]]} stats={st}"
        out[r] = st
    return out

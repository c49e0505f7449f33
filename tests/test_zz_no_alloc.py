"""cc_labels_static: labels computed with the library's built-in scratch.

This entry point is for callers that may not allocate device memory
themselves (a plugin whose host application's pool owns the device, or a
loop where cudaMalloc's device synchronisation is not allowed). Its labels
must equal the oracle's and those of cc_labels, the entry point that manages
its own workspace. The tests call the C ABI directly through ctypes, twice in
a row on different graphs (the shared scratch keeps the previous call's
contents, so the second call checks that everything that must start at zero
is cleared), check that warmed-up calls leave the device's free memory
unchanged, and that oversized inputs are refused before any work.
The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
from tests.gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _static_labels(torch, lib, edges_d, n):
    out = torch.full((n,), -1, dtype=edges_d.dtype, device=edges_d.device)
    m = edges_d.shape[0]
    rc = lib.cc_labels_static(ctypes.c_void_p(edges_d.data_ptr() if m else None), edges_d.element_size(),
                              ctypes.c_int64(n), ctypes.c_int64(m), ctypes.c_void_p(out.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, out


def _workspace_labels(torch, edges_d, n):
    import paper_1607_06156_gb300 as cc

    eng = cc.Engine(id_bytes=edges_d.element_size(), route="auto")
    out = eng.labels(edges_d, n)
    torch.cuda.synchronize()
    eng.close()
    return out


def test_static_entry_point_matches_oracle_and_cc_labels_twice_in_a_row():
    import oracle

    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    lib = cc.lib()
    graphs = [gg.rmat(seed=3, scale=18, edge_factor=4),            # n = 262,144, m = 1,048,576
              gg.planted(seed=2, n=60001, ncomp=333, id_bytes=8)]  # int64 ids, odd n
    for g in graphs:
        e = torch.from_numpy(g.edges).cuda()
        rc, got = _static_labels(torch, lib, e, g.n)
        assert rc == 0, cc.strerror(rc)
        assert np.array_equal(got.cpu().numpy().astype(np.int64), oracle.cc_labels(g.edges, g.n)), g.name
        want = _workspace_labels(torch, e, g.n)
        assert torch.equal(got, want), g.name


def test_static_entry_point_allocates_no_device_memory():
    """After a first call of each id width (which loads the library's kernels
    and its scratch array), further calls leave the device's free memory
    unchanged: the outputs are allocated before the measurement and the
    calls go straight to the C ABI."""
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    lib = cc.lib()
    g4 = gg.rmat(seed=5, scale=16, edge_factor=8)
    g8 = gg.planted(seed=7, n=30000, ncomp=100, id_bytes=8)
    runs = []
    for g in (g4, g8):
        e = torch.from_numpy(g.edges).cuda()
        out = torch.empty(g.n, dtype=e.dtype, device="cuda")
        runs.append((e, out, g.n))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(e, out, n):
        rc = lib.cc_labels_static(ctypes.c_void_p(e.data_ptr()), e.element_size(), ctypes.c_int64(n),
                                  ctypes.c_int64(e.shape[0]), ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, cc.strerror(rc)

    for r in runs:
        call(*r)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        for r in runs:
            call(*r)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_entry_point_limits():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    lib = cc.lib()
    e = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    out = torch.empty(8, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    too_many_vertices = lib.cc_labels_static(ctypes.c_void_p(e.data_ptr()), 4, ctypes.c_int64(cc.STATIC_MAX_VERTICES + 1),
                                             ctypes.c_int64(4), ctypes.c_void_p(out.data_ptr()), stream)
    too_many_pairs = lib.cc_labels_static(ctypes.c_void_p(e.data_ptr()), 4, ctypes.c_int64(8),
                                          ctypes.c_int64(cc.STATIC_MAX_PAIRS + 1), ctypes.c_void_p(out.data_ptr()),
                                          stream)
    assert too_many_vertices == 7 and too_many_pairs == 7  # CC_ERR_UNSUPPORTED
    # at the limits exactly: a path over all 2^20 vertices
    n = cc.STATIC_MAX_VERTICES
    path = torch.stack([torch.arange(n - 1), torch.arange(1, n)], dim=1).to(torch.int32).cuda()
    rc, got = _static_labels(torch, lib, path, n)
    assert rc == 0 and bool((got == 0).all())

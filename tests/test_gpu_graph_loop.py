"""The SV route as one CUDA graph with a device-driven WHILE loop (the default
when per-kernel profiling is off) against the host-driven loop (profile=1):
identical labels, iteration caps, fault injection and graph re-capture when
the arguments change."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.gpu_util import run_engine, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("maker", [
    lambda: gg.rmat(seed=5, scale=17, edge_factor=16),
    lambda: gg.planted(seed=2),
    lambda: gg.grid_chains(seed=5, W=300, nchains=20000, id_bytes=8),
])
def test_graph_loop_matches_host_loop(maker):
    g = maker()
    want = oracle.cc_labels(g.edges, g.n)
    a, sa = run_engine(g.edges, g.n, route="sv", profile=0)
    b, sb = run_engine(g.edges, g.n, route="sv", profile=1)
    assert np.array_equal(a, want) and np.array_equal(b, want)
    for st in (sa, sb):
        assert st["m_active"][0] == g.m and st["m_active"][1] == g.m
        assert st["sv_iters"] >= 2
        assert st["m_active"][st["sv_iters"] - 1] > 0 or st["sv_iters"] == 2
    # the device loop stops on the same rule: the last iteration kept nothing
    assert sa["launches"] >= 7


def test_graph_cache_recaptures_on_new_arguments():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    graphs = [gg.rmat(seed=s, scale=sc, edge_factor=8) for s, sc in ((1, 12), (2, 14), (3, 12))]
    eng = cc.Engine(route="sv")
    for rep in range(2):
        for g in graphs:
            e = torch.from_numpy(g.edges).cuda()
            out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
            eng.labels(e, g.n, out=out)
            assert np.array_equal(out.cpu().numpy().astype(np.int64), oracle.cc_labels(g.edges, g.n))
    eng.close()


@pytest.mark.parametrize("profile", [0, 1])
def test_iteration_cap_reports_no_convergence(profile):
    """A path of 2^16 vertices with reversed ids needs many SV iterations; a
    cap of 2 stops the loop with CC_ERR_NO_CONVERGENCE and the context stays
    usable."""
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    n = 1 << 16
    perm = np.random.default_rng(4).permutation(n)
    e = perm[np.stack([np.arange(n - 1), np.arange(1, n)], axis=1)].astype(np.int32)
    eng = cc.Engine(route="sv", max_iters=2, profile=profile, debug_checks=1)
    with pytest.raises(cc.CCError) as ei:
        eng.labels(torch.from_numpy(e).cuda(), n)
    assert ei.value.status == 4
    eng.set_options(max_iters=0)
    lab = eng.labels(torch.from_numpy(e).cuda(), n)
    assert (lab.cpu().numpy() == 0).all()
    eng.close()


def test_fault_injection_host_side():
    """CC_FAULT_ITER_CAP forces the cap to 1 and CC_FAULT_ALLOC fails the next
    workspace allocation; both are host-side, and the context recovers."""
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    g = gg.rmat(seed=7, scale=12, edge_factor=8)
    e = torch.from_numpy(g.edges).cuda()
    eng = cc.Engine(route="sv", fault_inject=cc.FAULT_ITER_CAP, debug_checks=1)
    with pytest.raises(cc.CCError) as ei:
        eng.labels(e, g.n)
    assert ei.value.status == 4
    eng.set_options(fault_inject=0)
    assert np.array_equal(eng.labels(e, g.n).cpu().numpy().astype(np.int64), oracle.cc_labels(g.edges, g.n))
    eng.close()
    eng = cc.Engine(route="sv", fault_inject=cc.FAULT_ALLOC)
    with pytest.raises(cc.CCError) as ei:
        eng.labels(e, g.n)
    assert ei.value.status == 3
    eng.set_options(fault_inject=0)
    assert np.array_equal(eng.labels(e, g.n).cpu().numpy().astype(np.int64), oracle.cc_labels(g.edges, g.n))
    eng.close()

"""GPU parity: CUDA labels are bit-identical to the oracle's on every route.

Labels are the minimum vertex id of each component (Section 3.1.1); the
route (K-S heuristic, forced BFS, forced SV; Algorithm 2) never changes
them. Sizes here span several tiles of every kernel plus ragged tails.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.gpu_util import assert_labels_match, run_engine, torch_cuda

pytestmark = pytest.mark.gpu


def test_planted_config_small():
    g = gg.planted(seed=1)  # n = 65,536, 512 components, ~163K pairs
    st = assert_labels_match(g.edges, g.n)
    assert st["auto"]["route"] == 0  # no power-law tail: SV only
    assert st["bfs"]["route"] == 1 and st["bfs"]["bfs_visited"] > 0


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_planted_seeds_int64(seed):
    g = gg.planted(seed=seed, n=50000, ncomp=700, id_bytes=8)
    assert_labels_match(g.edges, g.n)


@pytest.mark.parametrize("scale,ef", [(12, 4), (16, 16), (18, 8)])
def test_rmat(scale, ef):
    g = gg.rmat(seed=scale, scale=scale, edge_factor=ef)
    assert_labels_match(g.edges, g.n)


def test_chung_lu_takes_bfs_route():
    g = gg.chung_lu(seed=5, n=1 << 17, avg_degree=12, alpha=2.3)
    st = assert_labels_match(g.edges, g.n, routes=("auto",))["auto"]
    assert st["route"] == 1, st
    assert st["ks_d"] < 0.05
    assert st["bfs_visited"] > g.n // 4
    assert st["seed_vertex"] == int(np.argmax(np.bincount(g.edges.ravel(), minlength=g.n)))


def test_grid_chains_int64():
    g = gg.grid_chains(seed=3, W=300, p=0.55, nchains=20000, id_bytes=8)
    st = assert_labels_match(g.edges, g.n)
    assert st["auto"]["route"] == 0


def test_grid_chains_int32():
    g = gg.grid_chains(seed=4, W=257, p=0.5, nchains=5000, id_bytes=4)
    assert_labels_match(g.edges, g.n)


@pytest.mark.parametrize("cutoff", [1, 2, 3, 5])
def test_bfs_cutoff_keeps_labels_exact(cutoff):
    g = gg.chung_lu(seed=7, n=1 << 15, avg_degree=6, alpha=2.5)
    st = assert_labels_match(g.edges, g.n, routes=("bfs",), bfs_cutoff_levels=cutoff)["bfs"]
    assert st["bfs_levels"] <= cutoff


def _arr(pairs, dt=np.int32):
    return np.array(pairs, dtype=dt).reshape(-1, 2)


def test_empty_and_tiny():
    for n in (1, 2, 3, 7, 100, 1001):
        assert_labels_match(np.zeros((0, 2), np.int32), n)
    assert_labels_match(_arr([(0, 1)]), 2)
    assert_labels_match(_arr([(1, 0)]), 5)
    assert_labels_match(_arr([(2, 2)]), 3)
    assert_labels_match(_arr([(4, 3), (1, 2), (3, 0)]), 6)  # odd m: ragged vector tail


def test_self_loops_and_duplicates():
    n = 5000
    loops = np.repeat(np.arange(n, dtype=np.int32)[:, None], 2, axis=1)
    assert_labels_match(loops, n)
    rng = np.random.default_rng(0)
    base = rng.integers(0, n, size=(3000, 2)).astype(np.int32)
    dup = np.concatenate([base, base, base[::-1], loops[:777]])
    assert_labels_match(dup, n)


def test_long_paths_sorted_and_reversed_ids():
    """Diameter n-1: the worst case for BFS levels and for hook chains."""
    n = 200_001
    fwd = np.stack([np.arange(n - 1), np.arange(1, n)], axis=1).astype(np.int32)
    want = np.zeros(n, dtype=np.int64)
    assert_labels_match(fwd, n, want=want, routes=("sv", "auto"))
    assert_labels_match(fwd[::-1, ::-1].copy(), n, want=want, routes=("sv",))
    perm = np.random.default_rng(1).permutation(n).astype(np.int32)
    assert_labels_match(perm[fwd], n, want=want, routes=("sv",))


def test_long_path_bfs_route():
    n = 3000
    perm = np.random.default_rng(2).permutation(n).astype(np.int32)
    e = perm[np.stack([np.arange(n - 1), np.arange(1, n)], axis=1)]
    assert_labels_match(e, n, want=np.zeros(n, np.int64), routes=("bfs",))


def test_star_and_isolated():
    n = 100_000
    hub = n - 1
    star = np.stack([np.full(n // 2, hub), np.arange(0, n // 2) * 2 % (n - 1)], axis=1).astype(np.int32)
    assert_labels_match(star, n)


def test_large_ids_int64():
    """ids near and above 2^31 with int64 edges (n = 2^31 + 4096)."""
    torch = torch_cuda()
    n = (1 << 31) + 4096
    rng = np.random.default_rng(3)
    ids = np.unique(np.concatenate([rng.integers(n - 100000, n, 3000), [n - 1, (1 << 31) - 1, 1 << 31]]))
    e_local = rng.integers(0, ids.size, size=(2500, 2))
    e = ids[e_local].astype(np.int64)
    got, _ = run_engine(e, n, route="sv")
    want_local = oracle.cc_labels(e_local, ids.size)
    want = np.arange(n, dtype=np.int64)
    want[ids] = ids[want_local]
    assert np.array_equal(got[ids], want[ids])
    sample = rng.integers(0, n, 100000)
    assert np.array_equal(got[sample], want[sample])
    del torch


@pytest.mark.parametrize("route", ["auto", "sv", "bfs"])
def test_invalid_ids_rejected(route):
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    for bad, dt in ((_arr([(0, 1), (2, 10)]), np.int32), (_arr([(0, 1), (-1, 2)]), np.int32),
                    (_arr([(0, 1), (3, 1 << 40)], np.int64), np.int64)):
        # debug_checks: the call itself waits and returns the device status
        eng = cc.Engine(id_bytes=np.dtype(dt).itemsize, route=route, debug_checks=1)
        with pytest.raises(cc.CCError) as ei:
            eng.labels(torch.from_numpy(bad).cuda(), 10)
        assert ei.value.status == 2
        # the context stays usable
        ok = eng.labels(torch.from_numpy(_arr([(0, 1)], dt)).cuda(), 3)
        assert ok.cpu().tolist() == [0, 0, 2]
        eng.close()
        # stream-ordered (the default): the error is the stream's, read by check()
        eng = cc.Engine(id_bytes=np.dtype(dt).itemsize, route=route)
        eng.labels(torch.from_numpy(bad).cuda(), 10)
        with pytest.raises(cc.CCError) as ei:
            eng.check()
        assert ei.value.status == 2
        ok = eng.labels(torch.from_numpy(_arr([(0, 1)], dt)).cuda(), 3)
        eng.check()
        assert ok.cpu().tolist() == [0, 0, 2]
        eng.close()


def test_repeated_runs_are_identical():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    g = gg.rmat(seed=9, scale=15, edge_factor=8)
    want = oracle.cc_labels(g.edges, g.n)
    e = torch.from_numpy(g.edges).cuda()
    for route in ("sv", "bfs"):
        eng = cc.Engine(route=route)
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for _ in range(25):
            eng.labels(e, g.n, out=out)
            assert np.array_equal(out.cpu().numpy().astype(np.int64), want)
        eng.close()


def test_degree_distribution_parity():
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    for g in (gg.rmat(seed=2, scale=16, edge_factor=16), gg.grid_chains(seed=2, W=100, nchains=3000, id_bytes=8),
              gg.planted(seed=2)):
        deg_o = oracle.degrees(g.edges, g.n)
        hist_o = oracle.histogram(deg_o)
        eng = cc.Engine(id_bytes=g.id_bytes)
        deg, hist = eng.degree_distribution(torch.from_numpy(g.edges).cuda(), g.n, hist_len=hist_o.size + 3)
        assert np.array_equal(deg.cpu().numpy().astype(np.int64), deg_o)
        h = hist.cpu().numpy()
        assert np.array_equal(h[:hist_o.size], hist_o) and (h[hist_o.size:] == 0).all()
        eng.close()


def test_degree_overflow_bins():
    """A vertex of degree >= 2^20 goes through the overflow list."""
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    n = 3 << 20
    hubs = np.array([5, 77, 1 << 21], dtype=np.int64)
    parts = [np.stack([np.full(k, h), np.arange(k) + (1 << 20) * i], axis=1) for i, (h, k) in
             enumerate(zip(hubs, [(1 << 20) + 3, (1 << 20) + 3, 1 << 20]))]
    e = np.concatenate(parts).astype(np.int32)
    e[:, 1] %= n
    deg_o = oracle.degrees(e, n)
    eng = cc.Engine()
    deg, hist = eng.degree_distribution(torch.from_numpy(e).cuda(), n, hist_len=int(deg_o.max()) + 1)
    assert np.array_equal(deg.cpu().numpy().astype(np.int64), deg_o)
    assert np.array_equal(hist.cpu().numpy(), oracle.histogram(deg_o))
    got, st = run_engine(e, n, route="auto")
    assert np.array_equal(got, oracle.cc_labels(e, n))
    assert st["max_degree"] == int(deg_o.max())
    eng.close()


def _ks_dev(hist):
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    eng = cc.Engine()
    r = eng.ks_statistic(torch.from_numpy(np.ascontiguousarray(hist, dtype=np.int64)).cuda())
    eng.close()
    return r


@pytest.mark.parametrize("maker", [
    lambda: gg.rmat(seed=1, scale=18, edge_factor=16),
    lambda: gg.chung_lu(seed=3, n=1 << 18, avg_degree=16, alpha=2.5),
    lambda: gg.chung_lu(seed=4, n=1 << 16, avg_degree=4, alpha=3.2),
    lambda: gg.planted(seed=1),
    lambda: gg.grid_chains(seed=1, W=256, nchains=50000),
])
def test_ks_statistic_parity(maker):
    """Device D / alpha agree with the fp64 oracle to 1e-9; xmin and counts exactly."""
    g = maker()
    hist = oracle.histogram(oracle.degrees(g.edges, g.n))
    want = oracle.ks_fit(hist)
    got = _ks_dev(hist)
    assert got["ncand"] == want["ncand"]
    assert abs(got["D"] - want["D"]) < 1e-9, (got, want)
    assert got["xmin"] == want["xmin"] and got["ntail"] == want["ntail"]
    assert abs(got["alpha"] - want["alpha"]) < 1e-9 * max(1.0, want["alpha"])
    _, st = run_engine(g.edges, g.n, route="auto")
    assert abs(st["ks_d"] - want["D"]) < 1e-9
    assert st["route"] == int(oracle.route_is_bfs(want["D"]))


def test_ks_statistic_synthetic_histograms():
    rng = np.random.default_rng(11)
    for trial in range(20):
        L = int(rng.integers(10, 5000))
        hist = np.zeros(L, dtype=np.int64)
        k = int(rng.integers(3, min(L, 400)))
        xs = rng.choice(np.arange(1, L), size=k, replace=False)
        hist[xs] = rng.integers(1, 10 ** int(rng.integers(1, 7)), size=k)
        hist[0] = int(rng.integers(0, 1000))
        want = oracle.ks_fit(hist)
        got = _ks_dev(hist)
        assert got["ncand"] == want["ncand"] and got["xmin"] == want["xmin"], (got, want)
        assert abs(got["D"] - want["D"]) < 1e-9, (got, want)


@pytest.mark.parametrize("id_bytes", [4, 8])
def test_partitioned_degree_and_csr_paths(id_bytes):
    """m >= 2^20 takes the vertex-block partitioned degree pass and CSR build;
    an odd m exercises the ragged last pair, a hub the merged smem atomics."""
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    g = gg.rmat(seed=21, scale=16, edge_factor=16, m=(1 << 20) + 7, id_bytes=id_bytes)
    hub = np.stack([np.full(70000, 12345), np.arange(70000) * 3 % g.n], axis=1).astype(g.edges.dtype)
    e = np.concatenate([g.edges, hub])
    deg_o = oracle.degrees(e, g.n)
    eng = cc.Engine(id_bytes=id_bytes)
    deg, hist = eng.degree_distribution(torch.from_numpy(e).cuda(), g.n, hist_len=int(deg_o.max()) + 2)
    assert np.array_equal(deg.cpu().numpy().astype(np.int64), deg_o)
    assert np.array_equal(hist.cpu().numpy()[:-1], oracle.histogram(deg_o))
    eng.close()
    st = assert_labels_match(e, g.n, routes=("auto", "bfs"))["bfs"]
    _check_bfs_reach(e, g.n, st)


def _check_bfs_reach(e, n, st):
    """The CSR BFS from the max-degree vertex reached exactly that vertex's
    component: a missing or a wrong adjacency entry changes the count."""
    from oracle import multi_bfs

    starts, reached = multi_bfs.multi_bfs_reached(e, n, 1)
    assert st["route"] == 1 and st["bfs_visited"] == int(reached.sum()), (st["bfs_visited"], int(reached.sum()))


def test_csr_placement_of_a_vertex_block_with_a_hub():
    """One vertex of degree 2^21 makes its vertex block hold far more entries
    than the average: the placement merges the lanes that hit it. The BFS
    from it must reach exactly its component."""
    rng = np.random.default_rng(11)
    n = 1 << 20
    leaves = rng.choice(n, size=1 << 21)
    star = np.stack([np.full(leaves.size, 777), leaves], axis=1)
    noise = rng.integers(0, n, size=(1 << 19, 2))
    e = np.concatenate([star, noise]).astype(np.int32)
    e = e[rng.permutation(len(e))]
    st = assert_labels_match(e, n, routes=("bfs",))["bfs"]
    _check_bfs_reach(e, n, st)


def test_partitioned_paths_many_vertex_blocks():
    """n close to the partition limit (1024 blocks of 2^15 vertices)."""
    n = (1 << 25) - 5
    rng = np.random.default_rng(8)
    e = rng.integers(0, n, size=((1 << 21) + 1, 2)).astype(np.int32)
    st = assert_labels_match(e, n, routes=("bfs",))["bfs"]
    _check_bfs_reach(e, n, st)


@pytest.mark.parametrize("seed", list(range(12)))
def test_stress_many_chains_sv(seed):
    """Many short chains plus a percolated grid, forced SV: deep hook chains in
    one iteration make concurrent shortcuts race; labels must stay exact."""
    g = gg.grid_chains(seed=100 + seed, W=700, p=0.55, nchains=150_000, id_bytes=4)
    assert_labels_match(g.edges, g.n, routes=("sv",))


@pytest.mark.parametrize("cutoff", [0, 1, 3])
def test_edge_list_bfs_mode(cutoff):
    """bfs_mode 1: BFS as streaming passes over the active pairs (no CSR)."""
    for g in (gg.chung_lu(seed=9, n=1 << 16, avg_degree=8), gg.rmat(seed=10, scale=17, edge_factor=16),
              gg.grid_chains(seed=11, W=200, nchains=5000, id_bytes=8), gg.planted(seed=12, n=40000, ncomp=100)):
        st = assert_labels_match(g.edges, g.n, routes=("bfs",), bfs_mode=1, bfs_cutoff_levels=cutoff)["bfs"]
        assert st["route"] == 1 and st["bfs_visited"] >= 1
        if cutoff:
            assert st["bfs_levels"] <= cutoff


def test_edge_list_bfs_matches_csr_bfs_visited_set():
    g = gg.chung_lu(seed=13, n=1 << 17, avg_degree=10)
    a = assert_labels_match(g.edges, g.n, routes=("bfs",), bfs_mode=1)["bfs"]
    b = assert_labels_match(g.edges, g.n, routes=("bfs",), bfs_mode=0)["bfs"]
    assert a["bfs_visited"] == b["bfs_visited"] and a["comp_min"] == b["comp_min"]


def _degree_check(e, n, id_bytes):
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    deg_o = oracle.degrees(e, n)
    eng = cc.Engine(id_bytes=id_bytes)
    deg, hist = eng.degree_distribution(torch.from_numpy(e).cuda(), n, hist_len=int(deg_o.max()) + 1)
    assert np.array_equal(deg.cpu().numpy().astype(np.int64), deg_o)
    assert np.array_equal(hist.cpu().numpy(), oracle.histogram(deg_o))
    st = eng.stats()
    eng.close()
    return st


@pytest.mark.parametrize("id_bytes,m,n", [
    (4, (1 << 20) + 1, (1 << 25) + 1),        # 5 windows; a last chunk of one int32 pair (a bulk copy of 0 bytes)
    (4, 1 << 21, 1 << 26),                    # a whole number of 8,192-pair chunks
    (4, (1 << 21) + 3, (1 << 28) + 7),        # 33 windows of 2^23 vertices, the last one short
    (8, (1 << 20) + 4097, (1 << 25) + 100003),  # int64: 4,096-pair chunks and a ragged last one
])
def test_partitioned_degree_pass_chunks_and_windows(id_bytes, m, n):
    """The degree pass of graphs with n > 2^25 (endpoints partitioned into
    windows of 2^23 vertices, then counted window by window): chunk and
    window boundaries, counts exact."""
    rng = np.random.default_rng(m % 1000 + n % 1000)
    e = rng.integers(0, n, size=(m, 2)).astype(np.int32 if id_bytes == 4 else np.int64)
    e[::97, 1] = e[::97, 0]  # self-loops
    assert _degree_check(e, n, id_bytes)["degree_form"] == 3


@pytest.mark.parametrize("id_bytes,m,n", [
    (4, (1 << 20) + 1, (1 << 25) + 1),
    (8, (1 << 20) + 4097, (1 << 25) + 100003),
])
@pytest.mark.parametrize("profile", [0, 1])
def test_first_hooks_inside_the_windowed_degree_pass(id_bytes, m, n, profile):
    """With n > 2^25 and no SV front end the window pass also applies the first
    hook pass (atomicMin on the parent of each pair's larger end) while the
    window's parents are in L2: labels exact on the heuristic route (the hooks
    fused) and on the forced routes (not fused), with chains so that the
    hooks build deep trees, self-loops and duplicated pairs."""
    rng = np.random.default_rng(7 + id_bytes)
    dt = np.int32 if id_bytes == 4 else np.int64
    e = rng.integers(0, n, size=(m, 2))
    perm = rng.permutation(n)
    k = m // 4  # a few long paths through random vertices
    e[:k, 0] = perm[:k]
    e[:k, 1] = perm[1:k + 1]
    e[k:k + 1000] = e[:1000]  # duplicates
    e[::101, 1] = e[::101, 0]  # self-loops
    e = np.ascontiguousarray(e[rng.permutation(m)].astype(dt))
    want = oracle.cc_labels(e, n, cross_check=False)
    out = assert_labels_match(e, n, want=want, routes=("auto", "sv", "bfs"), profile=profile)
    assert out["auto"]["route"] == 0 and out["auto"]["sv_sample_stride"] == 1


def test_partitioned_degree_pass_window_overflow():
    """One vertex is an endpoint of every pair: its window holds more than
    twice the average entries, and the entries past its capacity are counted
    with global atomics."""
    n, m = (1 << 25) + 1, (1 << 21) + 9
    rng = np.random.default_rng(43)
    e = np.stack([np.full(m, 12345), rng.integers(0, n, size=m)], axis=1).astype(np.int32)
    _degree_check(e, n, 4)
    assert_labels_match(e, n, routes=("auto",))


@pytest.mark.parametrize("id_bytes,extra", [(4, 0), (4, 3), (8, 1)])
def test_hub_aware_degree_pass(id_bytes, extra):
    """m >= 2^24 with n < 2^20 (or 2^24 < n <= 2^25) takes the hub-aware
    degree pass (prefix counts pick the hubs, the rest is counted with hubs in
    shared memory); counts stay exact."""
    g = gg.rmat(seed=31, scale=19, edge_factor=32, m=(1 << 24) + extra, id_bytes=id_bytes)
    # hubs whose pairs mostly come after the prefix
    hub = np.stack([np.full(300000, 77), np.arange(300000) * 7 % g.n], axis=1).astype(g.edges.dtype)
    e = np.concatenate([g.edges, hub])
    assert _degree_check(e, g.n, id_bytes)["degree_form"] == 2
    got, st = run_engine(e, g.n, route="auto")
    assert np.array_equal(got, oracle.cc_labels(e, g.n, cross_check=False))
    assert st["max_degree"] == int(oracle.degrees(e, g.n).max())
    assert st["degree_form"] == 2


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["uniform", "star"])
def test_hub_aware_degree_pass_extremes(kind):
    """No vertex clears the hub threshold (uniform pairs: every prefix count
    is small), or one vertex is an endpoint of every pair (its per-block
    shared-memory count runs into the hundreds of thousands)."""
    torch = torch_cuda()
    import paper_1607_06156_gb300 as cc

    m = (1 << 24) + 5
    rng = np.random.default_rng(41)
    if kind == "uniform":
        n = (1 << 24) + 12345
        e = rng.integers(0, n, size=(m, 2), dtype=np.int64).astype(np.int32)
    else:
        n = (1 << 20) - 1
        e = np.stack([np.full(m, 12345), rng.integers(0, n, size=m)], axis=1).astype(np.int32)
    deg_o = oracle.degrees(e, n)
    eng = cc.Engine(id_bytes=4)
    deg, hist = eng.degree_distribution(torch.from_numpy(e).cuda(), n, hist_len=int(deg_o.max()) + 1)
    assert np.array_equal(deg.cpu().numpy().astype(np.int64), deg_o)
    assert np.array_equal(hist.cpu().numpy(), oracle.histogram(deg_o))
    assert eng.stats()["degree_form"] == 2
    eng.close()


@pytest.mark.gpu
@pytest.mark.parametrize("id_bytes,m,n", [
    (4, (1 << 22) + 7, 1 << 24),          # 512 windows of 2^15 vertices, a ragged last chunk
    (8, (1 << 22) + 4097, 3_000_001),     # int64; 367 windows of 2^13, the last one short
    (4, (1 << 22) + 1, 1 << 20),          # 512 windows of 2^11 (the smallest)
])
def test_shared_window_degree_pass(id_bytes, m, n):
    """2^20 <= n <= 2^24 with m >= 2^22: the endpoints are partitioned into at
    most 512 windows of at most 2^15 vertices (16-bit entries) and each window
    is counted in shared memory, its sampled hub in registers. Counts exact
    with a hub that holds about 30% of its window (within the window's
    capacity), a second heavy vertex in the same window, a star vertex whose
    window runs far past its capacity (the rest counted in global memory), and
    self-loops; labels exact on the heuristic route through that pass."""
    rng = np.random.default_rng(n % 997 + m % 991)
    dt = np.int32 if id_bytes == 4 else np.int64
    e = rng.integers(0, n, size=(m, 2))
    wb = 11
    while (n + (1 << wb) - 1) >> wb > 512:
        wb += 1
    avg = 2 * m // ((n + (1 << wb) - 1) >> wb)
    h1 = (n // 2) | 5
    h2 = h1 ^ 3  # the same window
    star = 7
    rows = rng.permutation(m)
    k1, k2, k3 = int(0.45 * avg), avg // 10, m // 8  # h1 and h2 stay within 1.5x the average
    e[rows[:k1], 0] = h1
    e[rows[k1:k1 + k2], 1] = h2
    e[rows[k1 + k2:k1 + k2 + k3], 0] = star
    e[::97, 1] = e[::97, 0]
    e = np.ascontiguousarray(e.astype(dt))
    assert _degree_check(e, n, id_bytes)["degree_form"] == 4
    want = oracle.cc_labels(e, n, cross_check=False)
    # graphs of at most 2^20 vertices and 2m < 4096 * 4097 take the one-block
    # fit, whose degree pass is one atomic per endpoint
    form = 1 if n <= (1 << 20) and 2 * m < 4096 * 4097 else 4
    for profile in (0, 1):
        out = assert_labels_match(e, n, want=want, routes=("auto",), profile=profile)
        assert out["auto"]["degree_form"] == form


@pytest.mark.parametrize("maker", [
    lambda: gg.chung_lu(seed=8, n=1 << 20, avg_degree=6, alpha=2.4),   # n = 2^20: the one-block fit
    lambda: gg.chung_lu(seed=8, n=(1 << 20) + 1, avg_degree=6, alpha=2.4),  # one more vertex: the grid-wide fit
    lambda: gg.planted(seed=4),
])
def test_small_and_grid_fits_agree_with_oracle(maker):
    """Graphs of at most 2^20 vertices (and fewer than 4,097 vertices of degree
    >= 4,096 possible) take the one-block fit inside cc_labels, larger ones the
    grid-wide kernels; both match the oracle's fit of the same histogram."""
    g = maker()
    deg = oracle.degrees(g.edges, g.n)
    want = oracle.ks_fit(oracle.histogram(deg))
    got, st = run_engine(g.edges, g.n, route="auto")
    assert abs(st["ks_d"] - want["D"]) < 1e-9
    assert st["ks_xmin"] == want["xmin"] and st["ks_ncand"] == want["ncand"]
    assert st["route"] == int(oracle.route_is_bfs(want["D"]))
    assert st["max_degree"] == int(deg.max()) and st["seed_vertex"] == int(np.argmax(deg))
    assert np.array_equal(got, oracle.cc_labels(g.edges, g.n, cross_check=False))


@pytest.mark.gpu
@pytest.mark.parametrize("stride", [0, 1, 2, 8, 1024])
@pytest.mark.parametrize("route", ["auto", "sv"])
def test_sv_sample_front_end(stride, route):
    """The SV front end hooks over one tile of pairs in `stride` before the
    first pass over all pairs (default 8 from 2^22 pairs, 1 = none). Labels
    are the oracle's for every stride, on the graph-driven and the
    host-driven (profiled) loop, with an odd number of pairs."""
    g = gg.rmat(seed=44, scale=18, edge_factor=16, m=(1 << 22) + 3)
    want = oracle.cc_labels(g.edges, g.n, cross_check=False)
    for profile in (0, 1):
        got, st = run_engine(g.edges, g.n, route=route, sv_sample_stride=stride, profile=profile)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, f"stride={stride} profile={profile}: {bad.size} labels differ, first at {bad[:5]}"
        # 2m / n = 32: the default samples one block in 32
        assert st["sv_sample_stride"] == (32 if stride == 0 else stride)


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["sorted", "chains64", "planted"])
def test_sv_sample_front_end_inputs(kind):
    """Pairs sorted by their first id (a strided sample still covers every
    vertex range), int64 chain forests (long paths the sample cuts into
    pieces), and a graph below the default threshold with a forced stride."""
    if kind == "sorted":
        g = gg.chung_lu(seed=5, n=1 << 20, avg_degree=10, alpha=2.3)
        e = g.edges[np.lexsort((g.edges[:, 1], g.edges[:, 0]))]
        n, strides = g.n, (0, 4)
    elif kind == "chains64":  # 2m / n ~ 2: no front end by default
        g = gg.grid_chains(seed=6, W=600, nchains=300_000, id_bytes=8)
        e, n, strides = g.edges, g.n, (0, 3, 16)
        _, st = run_engine(e, n, route="sv")
        assert st["sv_sample_stride"] == 1
    else:
        g = gg.planted(seed=7)
        e, n, strides = g.edges, g.n, (0, 2, 5)
    want = oracle.cc_labels(e, n, cross_check=False)
    for k in strides:
        assert_labels_match(e, n, want=want, routes=("auto", "sv"), sv_sample_stride=k)


@pytest.mark.gpu
def test_sv_sample_stride_validated():
    torch_cuda()
    import paper_1607_06156_gb300 as cc

    for bad in (-1, 1025):
        with pytest.raises(cc.CCError):
            cc.Engine(sv_sample_stride=bad)


@pytest.mark.gpu
@pytest.mark.parametrize("id_bytes", [4, 8])
def test_sparse_graph_over_2_25_vertices(id_bytes):
    """n > 2^25 vertices (a parent array larger than L2): mostly isolated
    vertices (their own roots), random pairs and a long chain (deep trees
    before the last shortcut), n not a multiple of 4."""
    n = (1 << 25) + 13
    rng = np.random.default_rng(71)
    rand = rng.integers(0, n, size=(1 << 21, 2))
    chain = rng.permutation(n)[:600_000]
    e = np.concatenate([rand, np.stack([chain[:-1], chain[1:]], axis=1), [[n - 1, n - 2], [n - 13, 3]]])
    e = e.astype(np.int32 if id_bytes == 4 else np.int64)
    assert_labels_match(e, n)

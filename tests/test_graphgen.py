"""Input generators: determinism, sizes and planted structure (CPU only)."""
import numpy as np

import graphgen as gg


def test_permutation_is_a_bijection():
    for n in (1, 2, 3, 17, 1000, 4096, 12345):
        x = np.arange(n, dtype=np.uint64)
        y = gg.permute(n, 99, 7, x)
        assert np.array_equal(np.sort(y), x)


def test_deterministic_and_seed_sensitive():
    a = gg.rmat(seed=3, scale=12, edge_factor=4)
    b = gg.rmat(seed=3, scale=12, edge_factor=4)
    c = gg.rmat(seed=4, scale=12, edge_factor=4)
    assert np.array_equal(a.edges, b.edges)
    assert not np.array_equal(a.edges, c.edges)
    assert a.edges.min() >= 0 and a.edges.max() < a.n


def test_planted_sizes_and_counts():
    g = gg.planted(seed=1)
    s = g.meta["sizes"]
    assert s.sum() == g.n == 65536 and s.size == 512 and s.min() >= 1
    assert np.array_equal(np.bincount(g.meta["comp"], minlength=512), s)
    # each component: spanning tree (s-1) + round(1.5 s) extra pairs (halves round up)
    assert g.m == int(np.sum(s - 1 + np.floor(1.5 * s + 0.5)))  # round half away from zero
    # pairs never cross components
    comp = g.meta["comp"]
    assert (comp[g.edges[:, 0]] == comp[g.edges[:, 1]]).all()


def test_grid_chains_shape():
    W, nch = 64, 500
    g = gg.grid_chains(seed=2, W=W, p=0.55, nchains=nch, id_bytes=8)
    off = g.meta["chain_off"]
    assert g.n == W * W + off[-1]
    assert g.edges.dtype == np.int64 and g.edges.min() >= 0 and g.edges.max() < g.n
    bonds = 2 * W * (W - 1)
    chain_edges = off[-1] - nch
    extra = g.m - chain_edges
    assert 0.45 * bonds < extra < 0.65 * bonds + 0.05 * off[-1]


def test_batch_offsets_and_local_ids():
    b = gg.batch(seed=1, G=12, nmin=1000, nmax=20000)
    assert b.edge_offsets[0] == 0 and b.edge_offsets[-1] == b.edges.shape[0]
    for g in range(b.G):
        gr = b.graph(g)
        assert 1000 <= gr.n <= 20000
        if gr.m:
            assert gr.edges.min() >= 0 and gr.edges.max() < gr.n
        if g % 3 == 0:
            assert gr.m == 8 * gr.n



def test_batch4096_sizes_follow_the_workload():
    """The 4,096-graph batch: vertex counts log-uniform in [1K, 1M] (each
    decade holds about a third of the graphs), R-MAT every third graph with
    8 pairs per vertex, and the same sizes whichever graphs are kept."""
    ng, mg = gg.batch_sizes(seed=1, G=4096)
    assert ng.size == mg.size == 4096
    assert ng.min() >= 1000 and ng.max() <= 1_000_000
    dec = np.bincount(np.minimum((np.log10(ng) - 3).astype(int), 2), minlength=3) / 4096
    assert np.all(np.abs(dec - 1 / 3) < 0.04)
    assert np.array_equal(mg[0::3], 8 * ng[0::3])
    assert (mg > 0).all()
    sub = gg.batch(seed=1, G=30, nmin=1000, nmax=5000, graphs=[29, 3, 17])
    n30, m30 = gg.batch_sizes(seed=1, G=30, nmin=1000, nmax=5000)
    assert np.diff(sub.vertex_offsets).tolist() == n30[[29, 3, 17]].tolist()
    assert np.diff(sub.edge_offsets).tolist() == m30[[29, 3, 17]].tolist()


def test_union_keeps_each_part_a_separate_set_of_components():
    """The union relabels by one permutation: each part's pairs stay within
    that part's vertices, and the parts' vertex sets partition [0, n)."""
    parts = [gg.chung_lu(seed=3 + i, n=500 + 100 * i, avg_degree=6) for i in range(4)]
    u = gg.union(parts, seed=9)
    assert u.n == sum(p.n for p in parts) and u.m == sum(p.m for p in parts)
    part = u.meta["comp_of_part"]
    assert np.array_equal(np.bincount(part), [p.n for p in parts])
    assert np.array_equal(part[u.edges[:, 0]], part[u.edges[:, 1]])
    # the degree sequence of each part survives the relabelling
    deg = np.bincount(u.edges.ravel(), minlength=u.n)
    for i, p in enumerate(parts):
        want = np.sort(np.bincount(p.edges.ravel(), minlength=p.n))
        assert np.array_equal(np.sort(deg[part == i]), want)
    assert np.array_equal(gg.union(parts, seed=9).edges, u.edges)

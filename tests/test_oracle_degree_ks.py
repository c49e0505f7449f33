"""Pins for the oracle's degree distribution, Hurwitz zeta and K-S fit (CPU only).

Section 3.2 / Algorithm 2: degree distribution, discrete power-law fit
(Clauset et al.), one-sample K-S statistic, BFS iff D < tau = 0.05 (Table 2).
"""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle


def test_degrees_match_bincount_with_loops_and_duplicates():
    rng = np.random.default_rng(1)
    e = rng.integers(0, 100, size=(5000, 2)).astype(np.int32)
    e[:50, 1] = e[:50, 0]  # self-loops count twice
    deg = oracle.degrees(e, 100)
    assert np.array_equal(deg, np.bincount(e.ravel(), minlength=100))
    assert oracle.degrees(np.array([[3, 3]], np.int32), 5).tolist() == [0, 0, 0, 2, 0]
    hist = oracle.histogram(deg)
    assert np.array_equal(hist, np.bincount(deg))
    assert hist.sum() == 100


def test_log2_buckets():
    hist = np.zeros(20, dtype=np.int64)
    hist[[0, 1, 2, 3, 4, 7, 8, 19]] = [5, 1, 2, 3, 4, 5, 6, 7]
    b = oracle.log2_buckets(hist)
    assert b[0] == 5 and b[1] == 1 and b[2] == 2 + 3 and b[3] == 4 + 5 and b[4] == 6 and b[5] == 7
    assert b.sum() == hist.sum()


@pytest.mark.parametrize("s,q,want", [
    (2.0, 1.0, math.pi ** 2 / 6),
    (4.0, 1.0, math.pi ** 4 / 90),
    (6.0, 1.0, math.pi ** 6 / 945),
    (2.0, 0.5, math.pi ** 2 / 2),          # zeta(s, 1/2) = (2^s - 1) zeta(s)
    (3.0, 2.0, 1.2020569031595942 - 1.0),  # zeta(3) - 1 (Apery's constant)
])
def test_hurwitz_zeta_closed_forms(s, q, want):
    assert oracle.hurwitz_zeta(s, q) == pytest.approx(want, rel=1e-13)


def test_hurwitz_zeta_vs_scipy_and_recurrence():
    sc = pytest.importorskip("scipy.special")
    for s in (1.05, 1.5, 2.0, 2.37, 3.1, 5.0):
        for q in (1.0, 2.0, 3.0, 17.0, 123.0, 1e4, 7.5e5):
            z = oracle.hurwitz_zeta(s, q)
            assert z == pytest.approx(float(sc.zeta(s, q)), rel=1e-12)
            assert z - oracle.hurwitz_zeta(s, q + 1) == pytest.approx(q ** -s, rel=1e-9)


def _ks_brute(hist, xmin, alpha):
    """sup_x |S(x) - P(x)| over EVERY integer x in [xmin, xmax + 2000], with
    P(x) = sum_{k=xmin..x} k^-alpha / zeta(alpha, xmin) summed term by term in
    50-digit arithmetic (mpmath's Hurwitz zeta for the normaliser)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    hist = np.asarray(hist, dtype=np.int64)
    xmax = hist.size - 1
    N = int(hist[xmin:].sum())
    a = mp.mpf(alpha)
    Z = mp.zeta(a, xmin)
    D, S, P = mp.mpf(0), mp.mpf(0), mp.mpf(0)
    for x in range(xmin, xmax + 2001):
        if x <= xmax:
            S += mp.mpf(int(hist[x])) / N
        P += mp.power(x, -a) / Z
        D = max(D, abs(S - P))
    return float(D)


def test_ks_matches_brute_force_sup_at_every_integer():
    """The oracle's D at its chosen xmin equals the sup over every integer."""
    rng = np.random.default_rng(5)
    for trial in range(12):
        xmax = int(rng.integers(8, 200))
        hist = np.zeros(xmax + 1, dtype=np.int64)
        xs = rng.integers(1, xmax + 1, size=int(rng.integers(3, 40)))
        hist[xs] += rng.integers(1, 60, size=xs.size)
        hist[0] = 17  # degree-0 vertices never enter the fit
        r = oracle.ks_fit(hist, min_tail=1, min_distinct=1, min_span=0.0)
        if r["ncand"] == 0:
            continue
        assert r["D"] == pytest.approx(_ks_brute(hist, r["xmin"], r["alpha"]), abs=1e-12)
        # the chosen xmin minimises D: every other candidate has D >= it
        for xmin in np.nonzero(hist[1:])[0][:6] + 1:
            tail = hist[xmin:]
            N = tail.sum()
            alpha = 1 + N / np.sum(tail * np.log(np.arange(xmin, hist.size) / (xmin - 0.5)))
            assert _ks_brute(hist, int(xmin), alpha) >= r["D"] - 1e-12


def test_ks_alpha_estimator_on_exact_power_law():
    """An exact discrete power law: eq. 3.7 of Clauset et al. recovers alpha
    (within its known ~1% bias at xmin >= 6) and D is tiny."""
    sc = pytest.importorskip("scipy.special")
    alpha, xmin, N = 2.5, 6, 10 ** 9
    xs = np.arange(xmin, 200000)
    pmf = xs ** -alpha / float(sc.zeta(alpha, xmin))
    hist = np.zeros(xs[-1] + 1, dtype=np.int64)
    hist[xs] = np.round(pmf * N).astype(np.int64)
    r = oracle.ks_fit(hist)
    assert r["xmin"] >= xmin
    assert abs(r["alpha"] - alpha) < 0.03
    assert r["D"] < 0.01


def test_ks_candidate_rules():
    """Tail-size, distinct-value and decade-span rules each remove candidates."""
    hist = np.zeros(401, dtype=np.int64)
    hist[[4, 5, 6, 7, 8, 9]] = [4000, 2000, 900, 400, 150, 60]  # a steep short tail ...
    hist[[40, 400]] = [1, 1]  # ... with two stragglers reaching a decade and beyond
    every = oracle.ks_fit(hist, min_tail=1, min_distinct=1, min_span=0.0)
    assert every["ncand"] == 8
    assert oracle.ks_fit(hist, min_tail=1, min_distinct=3, min_span=0.0)["ncand"] == 6
    assert oracle.ks_fit(hist, min_tail=100, min_distinct=1, min_span=0.0)["ncand"] == 5
    spanned = oracle.ks_fit(hist, min_tail=1, min_distinct=1, min_span=10.0)
    assert spanned["ncand"] == 7  # xmin = 40 reaches 400 = 10 * 40; xmin = 400 does not
    assert spanned["D"] >= every["D"]


def test_ks_no_candidate_and_regular_degrees():
    hist = np.zeros(5, dtype=np.int64)
    hist[4] = 1000  # a 4-regular graph: one distinct degree, no candidate tail
    r = oracle.ks_fit(hist)
    assert r["ncand"] == 0 and r["D"] == 1.0
    assert not oracle.route_is_bfs(r["D"])


def test_ks_table2_split_scale_free_vs_mesh():
    """Table 2's qualitative split: a graph with a power-law degree tail fits
    (D < 0.05, BFS runs); mesh-like, chain and planted small-component graphs
    do not (no candidate tail spans a decade, or D well above 0.05). R-MAT
    sits in between under this fit (its degree histogram is a staircase of
    binomial humps): D ~ 0.09 at scale 18, below the others but above tau."""
    g = gg.chung_lu(seed=1, n=1 << 18, avg_degree=16, alpha=2.5)
    r = oracle.ks_fit(oracle.histogram(oracle.degrees(g.edges, g.n)))
    assert r["D"] < oracle.KS_TAU, r
    assert oracle.route_is_bfs(r["D"])
    assert abs(r["alpha"] - 2.5) < 0.1
    h = gg.grid_chains(seed=1, W=512, p=0.55, nchains=100000)
    r2 = oracle.ks_fit(oracle.histogram(oracle.degrees(h.edges, h.n)))
    assert r2["D"] > 0.15, r2
    p = gg.planted(seed=1)
    r3 = oracle.ks_fit(oracle.histogram(oracle.degrees(p.edges, p.n)))
    assert r3["D"] > 0.15, r3
    k = gg.rmat(seed=1, scale=18, edge_factor=16)
    r4 = oracle.ks_fit(oracle.histogram(oracle.degrees(k.edges, k.n)))
    assert r["D"] < r4["D"] < min(r2["D"], r3["D"]), (r4, r2, r3)

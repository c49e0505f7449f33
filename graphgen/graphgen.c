/*
 * Seeded synthetic graph generators.
 *
 * These produce the undirected edge lists (interleaved (u,v) pairs) that both
 * the CPU oracle and the CUDA path consume. They hold none of the
 * connected-components arithmetic: only random graph construction.
 *
 * Randomness is counter based, so every draw is a pure function of
 * (seed, stream, counter) and the output does not depend on thread count or
 * machine:
 *   - mix64 is the SplitMix64 output function (Steele, Lea & Flood,
 *     "Fast splittable pseudorandom number generators", OOPSLA 2014; the
 *     constants are Stafford's "Mix13" variant used by SplitMix64).
 *   - rnd(seed, stream, ctr) = mix64(mix64(seed ^ mix64(stream)) + ctr * gamma)
 * Vertex ids are permuted by a 4-round balanced Feistel network with cycle
 * walking (Black & Rogaway, "Ciphers with arbitrary finite domains", 2002),
 * a bijection on [0, n) that needs no table.
 *
 * Graph families (sizes and parameters are passed in):
 *   planted   : K components of log-uniform size, each a random spanning
 *               tree (random attachment) plus uniform extra intra-component
 *               pairs; ids permuted, pairs randomly oriented and shuffled.
 *   rmat      : recursive-matrix generator (Chakrabarti, Zhan & Faloutsos,
 *               SDM 2004) with quadrant probabilities a, b, c, d = 1-a-b-c,
 *               duplicates and self-loops kept, ids permuted.
 *   grid+chains: W x W lattice with each bond kept with probability p,
 *               unioned with disjoint chains of geometric length whose
 *               vertices get, with probability q, one extra edge to a
 *               uniform vertex of the same chain; ids permuted.
 *   batch     : G independent graphs of log-uniform size cycling through
 *               R-MAT, percolated grid and chain forest; local ids.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GAMMA 0x9e3779b97f4a7c15ULL

static inline uint64_t mix64(uint64_t z) {
    z += GAMMA;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline uint64_t rnd(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return mix64(mix64(seed ^ mix64(stream)) + ctr * GAMMA);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, k) (k < 2^32 here; the bias of a 64-bit multiply-shift is < 2^-32) */
static inline uint64_t below(uint64_t x, uint64_t k) {
    return (uint64_t)(((unsigned __int128)x * k) >> 64);
}

/* ---------------- Feistel permutation on [0, n) ---------------- */
typedef struct {
    uint64_t n;
    int h;           /* half width in bits */
    uint64_t mask;   /* (1 << h) - 1 */
    uint64_t key[4];
} perm_t;

static void perm_init(perm_t *p, uint64_t n, uint64_t seed, uint64_t stream) {
    int bits = 0;
    while (bits < 64 && (1ULL << bits) < n) bits++;
    if (bits < 2) bits = 2;
    p->n = n;
    p->h = (bits + 1) / 2;
    p->mask = (1ULL << p->h) - 1;
    for (int r = 0; r < 4; r++) p->key[r] = rnd(seed, stream, (uint64_t)r);
}

static inline uint64_t feistel(const perm_t *p, uint64_t x) {
    uint64_t L = x >> p->h, R = x & p->mask;
    for (int r = 0; r < 4; r++) {
        uint64_t F = mix64(R ^ p->key[r]) & p->mask;
        uint64_t nl = R;
        R = L ^ F;
        L = nl;
    }
    return (L << p->h) | R;
}

static inline uint64_t perm_apply(const perm_t *p, uint64_t x) {
    uint64_t y = feistel(p, x);
    while (y >= p->n) y = feistel(p, y);
    return y;
}

static inline void put_edge(void *out, int id_bytes, uint64_t k, uint64_t u, uint64_t v) {
    if (id_bytes == 4) {
        int32_t *e = (int32_t *)out;
        e[2 * k] = (int32_t)u;
        e[2 * k + 1] = (int32_t)v;
    } else {
        int64_t *e = (int64_t *)out;
        e[2 * k] = (int64_t)u;
        e[2 * k + 1] = (int64_t)v;
    }
}

/* public: apply the id permutation to values (used by tests to check bijectivity) */
void gg_permute(uint64_t n, uint64_t seed, uint64_t stream, const uint64_t *in, uint64_t *out, int64_t count) {
    perm_t p;
    perm_init(&p, n, seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; i++) out[i] = perm_apply(&p, in[i]);
}

/* ---------------- planted components ---------------- */
/*
 * Component sizes: s_i = exp(U(ln lo, ln hi)), rescaled by largest remainder
 * so that they sum to exactly n (each >= 1). Extra pairs per component:
 * round(extra_per_vertex * s_i). Writes sizes_out[ncomp]; returns m.
 */
int64_t gg_planted_sizes(uint64_t seed, int64_t n, int64_t ncomp, double lo, double hi,
                         double extra_per_vertex, int64_t *sizes_out) {
    double *raw = (double *)malloc(sizeof(double) * ncomp);
    double *frac = (double *)malloc(sizeof(double) * ncomp);
    double tot = 0.0;
    for (int64_t i = 0; i < ncomp; i++) {
        raw[i] = exp(log(lo) + u01(rnd(seed, 1, (uint64_t)i)) * (log(hi) - log(lo)));
        tot += raw[i];
    }
    int64_t assigned = 0;
    for (int64_t i = 0; i < ncomp; i++) {
        double t = raw[i] * (double)n / tot;
        int64_t f = (int64_t)floor(t);
        if (f < 1) f = 1;
        sizes_out[i] = f;
        frac[i] = t - floor(t);
        assigned += f;
    }
    /* largest remainder: hand out (or take back) one vertex at a time */
    while (assigned < n) {
        int64_t best = 0;
        for (int64_t i = 1; i < ncomp; i++) if (frac[i] > frac[best]) best = i;
        sizes_out[best]++;
        frac[best] = -1.0;
        assigned++;
    }
    while (assigned > n) {
        int64_t best = -1;
        for (int64_t i = 0; i < ncomp; i++)
            if (sizes_out[i] > 1 && (best < 0 || frac[i] < frac[best])) best = i;
        sizes_out[best]--;
        frac[best] = 2.0;
        assigned--;
    }
    int64_t m = 0;
    for (int64_t i = 0; i < ncomp; i++) m += (sizes_out[i] - 1) + (int64_t)llround(extra_per_vertex * (double)sizes_out[i]);
    free(raw);
    free(frac);
    return m;
}

/*
 * Fill the planted graph. comp_out[v] = component index of (permuted) vertex v.
 */
void gg_planted_fill(uint64_t seed, int64_t n, int64_t ncomp, const int64_t *sizes, double extra_per_vertex,
                     int id_bytes, void *edges_out, int64_t m, int32_t *comp_out) {
    int64_t *voff = (int64_t *)malloc(sizeof(int64_t) * (ncomp + 1));
    int64_t *eoff = (int64_t *)malloc(sizeof(int64_t) * (ncomp + 1));
    voff[0] = 0;
    eoff[0] = 0;
    for (int64_t i = 0; i < ncomp; i++) {
        voff[i + 1] = voff[i] + sizes[i];
        eoff[i + 1] = eoff[i] + (sizes[i] - 1) + (int64_t)llround(extra_per_vertex * (double)sizes[i]);
    }
    perm_t pv, pe;
    perm_init(&pv, (uint64_t)n, seed, 2);
    perm_init(&pe, (uint64_t)(m > 1 ? m : 2), seed, 3);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < ncomp; i++) {
        int64_t s = sizes[i], base = voff[i], k = eoff[i];
        for (int64_t j = 0; j < s; j++) comp_out[perm_apply(&pv, (uint64_t)(base + j))] = (int32_t)i;
        for (int64_t j = 1; j < s; j++, k++) {
            uint64_t r = rnd(seed, 4, (uint64_t)k);
            uint64_t a = (uint64_t)(base + j), b = (uint64_t)base + below(r, (uint64_t)j);
            uint64_t pa = perm_apply(&pv, a), pb = perm_apply(&pv, b);
            uint64_t slot = (m > 1) ? perm_apply(&pe, (uint64_t)k) : (uint64_t)k;
            if (rnd(seed, 5, (uint64_t)k) & 1) put_edge(edges_out, id_bytes, slot, pa, pb);
            else put_edge(edges_out, id_bytes, slot, pb, pa);
        }
        int64_t extra = (int64_t)llround(extra_per_vertex * (double)s);
        for (int64_t j = 0; j < extra; j++, k++) {
            uint64_t a = (uint64_t)base + below(rnd(seed, 6, (uint64_t)k), (uint64_t)s);
            uint64_t b = (uint64_t)base + below(rnd(seed, 7, (uint64_t)k), (uint64_t)s);
            uint64_t slot = (m > 1) ? perm_apply(&pe, (uint64_t)k) : (uint64_t)k;
            put_edge(edges_out, id_bytes, slot, perm_apply(&pv, a), perm_apply(&pv, b));
        }
    }
    free(voff);
    free(eoff);
}

/* ---------------- R-MAT ---------------- */
/*
 * m pairs on 2^scale vertices. Each level draws one uniform and picks a
 * quadrant: [0,a) -> (0,0), [a,a+b) -> (0,1), [a+b,a+b+c) -> (1,0), else (1,1).
 * Ids are then permuted on [0, 2^scale); if n_mod > 0 they are reduced mod n_mod.
 * The first pair written is out[k0].
 */
void gg_rmat_fill(uint64_t seed, int scale, int64_t m, double a, double b, double c, uint64_t n_mod,
                  int id_bytes, void *edges_out, int64_t k0) {
    perm_t pv;
    perm_init(&pv, 1ULL << scale, seed, 11);
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; k++) {
        uint64_t u = 0, v = 0;
        for (int l = 0; l < scale; l++) {
            double r = u01(rnd(seed, 12, (uint64_t)k * 64u + (uint64_t)l));
            int bu, bv;
            if (r < a) { bu = 0; bv = 0; }
            else if (r < ab) { bu = 0; bv = 1; }
            else if (r < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | (uint64_t)bu;
            v = (v << 1) | (uint64_t)bv;
        }
        u = perm_apply(&pv, u);
        v = perm_apply(&pv, v);
        if (n_mod) { u %= n_mod; v %= n_mod; }
        put_edge(edges_out, id_bytes, (uint64_t)(k0 + k), u, v);
    }
}

/* ---------------- percolated grid + chains ---------------- */
/*
 * Bonds of a W x W lattice: index e in [0, W(W-1)) is horizontal (r, c)-(r, c+1)
 * with r = e / (W-1), c = e % (W-1); index W(W-1) + e is vertical (c, r)-(c+1, r)
 * (transposed the same way). A bond is kept iff U(seed, 21, e) < p.
 * Chains: length L_j = 1 + floor(ln(1-U)/ln(1-1/mean)) (geometric on {1,2,..}).
 * Each chain vertex gets, with probability q, one branch edge to a uniform
 * vertex of its own chain. Pre-permutation ids: grid vertex (r,c) = r*W + c,
 * chain j vertex i = W*W + off_j + i.
 *
 * gg_gridchain_count returns m and writes n, the chain offsets (nchains+1) and
 * per-block kept-bond counts used by the fill step.
 */
#define GC_BLOCK 65536
static inline int bond_kept(uint64_t seed, uint64_t e, double p) { return u01(rnd(seed, 21, e)) < p; }

int64_t gg_gridchain_count(uint64_t seed, int64_t W, double p, int64_t nchains, double mean_len, double q,
                           int64_t *n_out, int64_t *chain_off /* nchains+1 */) {
    const int64_t nb = (W > 1) ? 2 * W * (W - 1) : 0;
    int64_t kept = 0;
#pragma omp parallel for schedule(static) reduction(+ : kept)
    for (int64_t e = 0; e < nb; e++) kept += bond_kept(seed, (uint64_t)e, p);
    const double lq = log(1.0 - 1.0 / mean_len);
    chain_off[0] = 0;
    for (int64_t j = 0; j < nchains; j++) {
        double u = u01(rnd(seed, 22, (uint64_t)j));
        int64_t L = 1 + (int64_t)floor(log(1.0 - u) / lq);
        chain_off[j + 1] = chain_off[j] + L;
    }
    const int64_t nc = chain_off[nchains];
    int64_t branches = 0;
#pragma omp parallel for schedule(static) reduction(+ : branches)
    for (int64_t i = 0; i < nc; i++) branches += u01(rnd(seed, 23, (uint64_t)i)) < q;
    *n_out = W * W + nc;
    return kept + (nc - nchains) + branches;
}

static int64_t find_chain(const int64_t *off, int64_t nchains, int64_t i) {
    int64_t lo = 0, hi = nchains; /* off[lo] <= i < off[hi] */
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (off[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

void gg_gridchain_fill(uint64_t seed, int64_t W, double p, int64_t nchains, double q, const int64_t *chain_off,
                       int64_t n, int id_bytes, void *edges_out, int64_t m) {
    (void)m;
    perm_t pv;
    perm_init(&pv, (uint64_t)n, seed, 24);
    const int64_t nb = (W > 1) ? 2 * W * (W - 1) : 0;
    const int64_t nblk = (nb + GC_BLOCK - 1) / GC_BLOCK;
    int64_t *bc = (int64_t *)calloc((size_t)nblk + 1, sizeof(int64_t));
#pragma omp parallel for schedule(static)
    for (int64_t bk = 0; bk < nblk; bk++) {
        int64_t e1 = (bk + 1) * GC_BLOCK < nb ? (bk + 1) * GC_BLOCK : nb, cnt = 0;
        for (int64_t e = bk * GC_BLOCK; e < e1; e++) cnt += bond_kept(seed, (uint64_t)e, p);
        bc[bk + 1] = cnt;
    }
    for (int64_t bk = 0; bk < nblk; bk++) bc[bk + 1] += bc[bk];
    const int64_t hb = W * (W - 1);
#pragma omp parallel for schedule(static)
    for (int64_t bk = 0; bk < nblk; bk++) {
        int64_t e1 = (bk + 1) * GC_BLOCK < nb ? (bk + 1) * GC_BLOCK : nb, k = bc[bk];
        for (int64_t e = bk * GC_BLOCK; e < e1; e++) {
            if (!bond_kept(seed, (uint64_t)e, p)) continue;
            int64_t t = e < hb ? e : e - hb;
            int64_t r = t / (W - 1), c = t % (W - 1);
            uint64_t a, b;
            if (e < hb) { a = (uint64_t)(r * W + c); b = a + 1; }
            else { a = (uint64_t)(c * W + r); b = a + (uint64_t)W; }
            put_edge(edges_out, id_bytes, (uint64_t)k++, perm_apply(&pv, a), perm_apply(&pv, b));
        }
    }
    const int64_t kept = bc[nblk];
    free(bc);
    /* chain edges: chain j contributes L_j - 1 edges starting at kept + off_j - j */
    const int64_t base = W * W;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t j = 0; j < nchains; j++) {
        int64_t o = chain_off[j], L = chain_off[j + 1] - o, k = kept + o - j;
        for (int64_t i = 0; i + 1 < L; i++)
            put_edge(edges_out, id_bytes, (uint64_t)(k + i), perm_apply(&pv, (uint64_t)(base + o + i)),
                     perm_apply(&pv, (uint64_t)(base + o + i + 1)));
    }
    const int64_t nc = chain_off[nchains];
    int64_t k = kept + nc - nchains;
    /* branch edges, in chain-vertex order (block counts make this parallel) */
    const int64_t nbb = (nc + GC_BLOCK - 1) / GC_BLOCK;
    int64_t *bb = (int64_t *)calloc((size_t)nbb + 1, sizeof(int64_t));
#pragma omp parallel for schedule(static)
    for (int64_t bk = 0; bk < nbb; bk++) {
        int64_t i1 = (bk + 1) * GC_BLOCK < nc ? (bk + 1) * GC_BLOCK : nc, cnt = 0;
        for (int64_t i = bk * GC_BLOCK; i < i1; i++) cnt += u01(rnd(seed, 23, (uint64_t)i)) < q;
        bb[bk + 1] = cnt;
    }
    for (int64_t bk = 0; bk < nbb; bk++) bb[bk + 1] += bb[bk];
#pragma omp parallel for schedule(static)
    for (int64_t bk = 0; bk < nbb; bk++) {
        int64_t i1 = (bk + 1) * GC_BLOCK < nc ? (bk + 1) * GC_BLOCK : nc, kk = k + bb[bk];
        for (int64_t i = bk * GC_BLOCK; i < i1; i++) {
            if (!(u01(rnd(seed, 23, (uint64_t)i)) < q)) continue;
            int64_t j = find_chain(chain_off, nchains, i);
            int64_t o = chain_off[j], L = chain_off[j + 1] - o;
            uint64_t tgt = (uint64_t)(base + o) + below(rnd(seed, 25, (uint64_t)i), (uint64_t)L);
            put_edge(edges_out, id_bytes, (uint64_t)kk++, perm_apply(&pv, (uint64_t)(base + i)), perm_apply(&pv, tgt));
        }
    }
    free(bb);
}

/* ---------------- batch of independent graphs ---------------- */
/*
 * Graph g: n_g = round(exp(U(ln nmin, ln nmax))), type = g mod 3:
 *   0: R-MAT, edge factor ef, scale ceil(log2 n_g), ids permuted then mod n_g
 *   1: grid of side floor(sqrt(n_g)) with bond probability p (leftover ids isolated)
 *   2: chain forest: chains of geometric length (mean) until n_g vertices are
 *      used (the last chain is cut), branch probability q
 * Each graph uses its own sub-seed rnd(seed, 31, g). Writes n_g and m_g.
 */
static int ceil_log2(int64_t x) { int s = 0; while ((1LL << s) < x) s++; return s; }

static int64_t chain_forest_lengths(uint64_t s, int64_t ng, double mean_len, int64_t *off /* may be NULL */) {
    const double lq = log(1.0 - 1.0 / mean_len);
    int64_t used = 0, j = 0;
    if (off) off[0] = 0;
    while (used < ng) {
        double u = u01(rnd(s, 22, (uint64_t)j));
        int64_t L = 1 + (int64_t)floor(log(1.0 - u) / lq);
        if (L > ng - used) L = ng - used;
        used += L;
        j++;
        if (off) off[j] = used;
    }
    return j;
}

void gg_batch_sizes(uint64_t seed, int64_t G, int64_t nmin, int64_t nmax, int ef, double p, double mean_len,
                    double q, int64_t *n_out, int64_t *m_out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t g = 0; g < G; g++) {
        uint64_t s = rnd(seed, 31, (uint64_t)g);
        int64_t ng = (int64_t)llround(exp(log((double)nmin) + u01(rnd(seed, 32, (uint64_t)g)) * (log((double)nmax) - log((double)nmin))));
        if (ng < 1) ng = 1;
        n_out[g] = ng;
        int t = (int)(g % 3);
        if (t == 0) {
            m_out[g] = (int64_t)ef * ng;
        } else if (t == 1) {
            int64_t W = (int64_t)floor(sqrt((double)ng));
            while ((W + 1) * (W + 1) <= ng) W++;
            while (W * W > ng) W--;
            int64_t nb = (W > 1) ? 2 * W * (W - 1) : 0, kept = 0;
            for (int64_t e = 0; e < nb; e++) kept += bond_kept(s, (uint64_t)e, p);
            m_out[g] = kept;
        } else {
            int64_t nch = chain_forest_lengths(s, ng, mean_len, NULL);
            int64_t br = 0;
            for (int64_t i = 0; i < ng; i++) br += u01(rnd(s, 23, (uint64_t)i)) < q;
            m_out[g] = (ng - nch) + br;
        }
    }
}

/* Graph number gid of a batch (its type is gid % 3, its draws are keyed by
 * gid) with ng vertices, written from pair k on. */
static void batch_fill_one(uint64_t seed, int64_t gid, int64_t ng, int64_t k, double p, double mean_len, double q,
                           int32_t *edges_out) {
    int t = (int)(gid % 3);
    uint64_t s = rnd(seed, 31, (uint64_t)gid);
    perm_t pv;
    perm_init(&pv, (uint64_t)ng, s, 24);
    if (t == 1) {
        int64_t W = (int64_t)floor(sqrt((double)ng));
        while ((W + 1) * (W + 1) <= ng) W++;
        while (W * W > ng) W--;
        int64_t nb = (W > 1) ? 2 * W * (W - 1) : 0, hb = W * (W - 1);
        for (int64_t e = 0; e < nb; e++) {
            if (!bond_kept(s, (uint64_t)e, p)) continue;
            int64_t tt = e < hb ? e : e - hb;
            int64_t r = tt / (W - 1), cc = tt % (W - 1);
            uint64_t x, y;
            if (e < hb) { x = (uint64_t)(r * W + cc); y = x + 1; }
            else { x = (uint64_t)(cc * W + r); y = x + (uint64_t)W; }
            put_edge(edges_out, 4, (uint64_t)k++, perm_apply(&pv, x), perm_apply(&pv, y));
        }
    } else {
        int64_t nch = chain_forest_lengths(s, ng, mean_len, NULL);
        int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (nch + 1));
        chain_forest_lengths(s, ng, mean_len, off);
        for (int64_t j = 0; j < nch; j++)
            for (int64_t i = off[j]; i + 1 < off[j + 1]; i++)
                put_edge(edges_out, 4, (uint64_t)k++, perm_apply(&pv, (uint64_t)i), perm_apply(&pv, (uint64_t)(i + 1)));
        int64_t j = 0;
        for (int64_t i = 0; i < ng; i++) {
            while (off[j + 1] <= i) j++;
            if (!(u01(rnd(s, 23, (uint64_t)i)) < q)) continue;
            int64_t L = off[j + 1] - off[j];
            uint64_t tgt = (uint64_t)off[j] + below(rnd(s, 25, (uint64_t)i), (uint64_t)L);
            put_edge(edges_out, 4, (uint64_t)k++, perm_apply(&pv, (uint64_t)i), perm_apply(&pv, tgt));
        }
        free(off);
    }
}

/* The graphs gids[0..count) of a batch, graph gids[i] with n_g[i] vertices
 * written from pair edge_off[i] on: the same pairs as in the whole batch. */
void gg_batch_fill_ids(uint64_t seed, int64_t count, const int64_t *gids, const int64_t *n_g, const int64_t *edge_off,
                       double a, double b, double c, double p, double mean_len, double q, int32_t *edges_out) {
    /* R-MAT graphs are filled with the (internally parallel) R-MAT routine */
    for (int64_t i = 0; i < count; i++) {
        if (gids[i] % 3 != 0) continue;
        uint64_t s = rnd(seed, 31, (uint64_t)gids[i]);
        gg_rmat_fill(s, ceil_log2(n_g[i] > 1 ? n_g[i] : 2), edge_off[i + 1] - edge_off[i], a, b, c, (uint64_t)n_g[i],
                     4, edges_out, edge_off[i]);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < count; i++) {
        if (gids[i] % 3 == 0) continue;
        batch_fill_one(seed, gids[i], n_g[i], edge_off[i], p, mean_len, q, edges_out);
    }
}

void gg_batch_fill(uint64_t seed, int64_t G, const int64_t *n_g, const int64_t *edge_off, int ef, double a, double b,
                   double c, double p, double mean_len, double q, int32_t *edges_out) {
    (void)ef;
    int64_t *gids = (int64_t *)malloc(sizeof(int64_t) * (G > 0 ? G : 1));
    for (int64_t g = 0; g < G; g++) gids[g] = g;
    gg_batch_fill_ids(seed, G, gids, n_g, edge_off, a, b, c, p, mean_len, q, edges_out);
    free(gids);
}

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------- Chung-Lu power-law graph ---------------- */
/*
 * n vertices with weights w_i = (i + i0)^(-1/(alpha-1)) (a Zipf sequence,
 * i0 = 1), m pairs whose endpoints are drawn independently with probability
 * proportional to w (inverse CDF over the cumulative weights); ids permuted.
 * The expected degree of vertex i is 2 m w_i / sum(w), a power law of
 * exponent alpha in the tail (Chung & Lu, "Connected components in random
 * graphs with given expected degree sequences", 2002).
 */
static int64_t cdf_find(const double *cdf, int64_t n, double r) {
    int64_t lo = 0, hi = n - 1; /* smallest i with cdf[i] > r */
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (cdf[mid] > r) hi = mid; else lo = mid + 1;
    }
    return lo;
}

void gg_chung_lu_fill(uint64_t seed, int64_t n, int64_t m, double alpha, int id_bytes, void *edges_out) {
    double *cdf = (double *)malloc(sizeof(double) * (size_t)n);
    double acc = 0.0;
    for (int64_t i = 0; i < n; i++) {
        acc += pow((double)(i + 1), -1.0 / (alpha - 1.0));
        cdf[i] = acc;
    }
    for (int64_t i = 0; i < n; i++) cdf[i] /= acc;
    perm_t pv;
    perm_init(&pv, (uint64_t)n, seed, 41);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; k++) {
        int64_t u = cdf_find(cdf, n, u01(rnd(seed, 42, (uint64_t)k)));
        int64_t v = cdf_find(cdf, n, u01(rnd(seed, 43, (uint64_t)k)));
        put_edge(edges_out, id_bytes, (uint64_t)k, perm_apply(&pv, (uint64_t)u), perm_apply(&pv, (uint64_t)v));
    }
    free(cdf);
}

/*
 * CPU oracle for the hybrid connected-components path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or
 * call this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it. It shares no code with the CUDA path.
 *
 * Everything here is the plain definition of what the hybrid route
 * computes, written for obviousness, single threaded, in 64-bit integers and
 * fp64:
 *
 *  - Component labels (Section 1, problem statement; Section 3.1.1 and the
 *    Figure 1 caption: at termination every vertex carries the numerically
 *    smallest id of its component, "min(u, v1, v2)" in the worked example;
 *    Section 3.1.2: the final label of u is the partition p of any tuple
 *    <p,_,u>, which is the component minimum):
 *        label[v] = min { u : u reachable from v }.
 *    Computed three independent ways:
 *      oracle_uf_labels      union-find (Section 1 names union-find as one of
 *                            the two linear-time sequential methods), union
 *                            by smaller root id, path halving; with min-root
 *                            union every root is its set's minimum.
 *      oracle_bfs_labels     one BFS per component (Section 1, the other
 *                            sequential method), scanning seeds in
 *                            increasing id so the seed is the minimum.
 *      oracle_closure_labels boolean transitive closure (Warshall) for tiny
 *                            n, the definition of reachability itself.
 *
 *  - Degree distribution (Section 3.2, Algorithm 2 "Degree_Distribution"):
 *    each undirected pair is stored in both directions, so deg[v] counts the
 *    pair endpoints equal to v; a self-loop (v,v) adds 2 and duplicates
 *    count. hist[d] = #{v : deg[v] = d}.
 *
 *  - Power-law fit and one-sample Kolmogorov-Smirnov statistic
 *    (Section 3.2 and Table 2, following Clauset, Shalizi & Newman 2009):
 *      tail(xmin) = vertices with degree >= xmin (degree 0 never enters),
 *      alpha(xmin) = 1 + N / sum_{tail} ln(d / (xmin - 1/2))   (discrete
 *                    approximation, Clauset et al. eq. 3.7),
 *      model CDF   P(x) = 1 - zeta(alpha, x+1) / zeta(alpha, xmin),
 *      empirical   S(x) = #{tail d <= x} / N,
 *      D(xmin)     = sup_{x >= xmin} |S(x) - P(x)|,
 *    and the statistic is min D over the candidate xmin: every distinct
 *    degree d >= 1 whose tail holds at least min_tail vertices and at least
 *    min_distinct distinct degree values, and whose range reaches
 *    max degree >= min_span * xmin (a power law is a statement about a
 *    range of scales; without this a short steep tail of a Poisson-like
 *    distribution passes for one). The sup is taken exactly: S is a
 *    step function of the integers and P is increasing, so on every run of
 *    integers [a, b-1] between consecutive observed degrees a < b the
 *    extremes of |S - P| sit at x = a and x = b - 1; both are evaluated
 *    (beyond the largest degree S = 1 and |S - P| only shrinks).
 *    zeta(s, q) is the Hurwitz zeta function, evaluated by Euler-Maclaurin
 *    summation: 16 explicit terms, the integral tail, and 8 Bernoulli
 *    correction terms; the ratio is formed from xmin^alpha * zeta so that
 *    neither factor underflows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline int64_t edge_at(const void *edges, int id_bytes, int64_t i) {
    if (id_bytes == 4) return (int64_t)((const int32_t *)edges)[i];
    return ((const int64_t *)edges)[i];
}

/* returns 0 if every id lies in [0, n), else 1 */
int oracle_check_ids(const void *edges, int id_bytes, int64_t n, int64_t m) {
    for (int64_t i = 0; i < 2 * m; i++) {
        int64_t x = edge_at(edges, id_bytes, i);
        if (x < 0 || x >= n) return 1;
    }
    return 0;
}

/* ---------------- union-find ---------------- */
static int64_t uf_find(int64_t *parent, int64_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]]; /* path halving */
        x = parent[x];
    }
    return x;
}

int oracle_uf_labels(const void *edges, int id_bytes, int64_t n, int64_t m, int64_t *labels) {
    if (oracle_check_ids(edges, id_bytes, n, m)) return 1;
    int64_t *parent = labels; /* the label array doubles as the parent array */
    for (int64_t v = 0; v < n; v++) parent[v] = v;
    for (int64_t i = 0; i < m; i++) {
        int64_t ru = uf_find(parent, edge_at(edges, id_bytes, 2 * i));
        int64_t rv = uf_find(parent, edge_at(edges, id_bytes, 2 * i + 1));
        if (ru == rv) continue;
        if (ru < rv) parent[rv] = ru; /* link the larger root under the smaller */
        else parent[ru] = rv;
    }
    for (int64_t v = 0; v < n; v++) labels[v] = uf_find(parent, v);
    return 0;
}

/* ---------------- BFS labeller ---------------- */
int oracle_bfs_labels(const void *edges, int id_bytes, int64_t n, int64_t m, int64_t *labels) {
    if (oracle_check_ids(edges, id_bytes, n, m)) return 1;
    int64_t *start = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *adj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!start || !adj || !fill || !queue) {
        free(start); free(adj); free(fill); free(queue);
        return 2;
    }
    for (int64_t i = 0; i < m; i++) {
        start[edge_at(edges, id_bytes, 2 * i) + 1]++;
        start[edge_at(edges, id_bytes, 2 * i + 1) + 1]++;
    }
    for (int64_t v = 0; v < n; v++) start[v + 1] += start[v];
    memcpy(fill, start, sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < m; i++) {
        int64_t u = edge_at(edges, id_bytes, 2 * i), v = edge_at(edges, id_bytes, 2 * i + 1);
        adj[fill[u]++] = v;
        adj[fill[v]++] = u;
    }
    for (int64_t v = 0; v < n; v++) labels[v] = -1;
    for (int64_t s = 0; s < n; s++) {
        if (labels[s] >= 0) continue;
        int64_t head = 0, tail = 0;
        labels[s] = s;
        queue[tail++] = s;
        while (head < tail) {
            int64_t x = queue[head++];
            for (int64_t k = start[x]; k < start[x + 1]; k++) {
                int64_t y = adj[k];
                if (labels[y] < 0) {
                    labels[y] = s;
                    queue[tail++] = y;
                }
            }
        }
    }
    free(start); free(adj); free(fill); free(queue);
    return 0;
}

/* ---------------- multi-source BFS distances ---------------- */
/*
 * The BFS step of Section 3.2 from several starts at once: dist[v] = the
 * least number of pairs on a path from any start to v, -1 if no start
 * reaches v. A queue holds the vertices in increasing distance; with
 * cutoff > 0 vertices at distance cutoff are not expanded (the traversal
 * stops after `cutoff` levels). Returns 0, 1 for an id outside [0, n), 2
 * when memory runs out.
 */
int oracle_multi_bfs(const void *edges, int id_bytes, int64_t n, int64_t m, const int64_t *starts, int64_t nstarts,
                     int64_t cutoff, int64_t *dist) {
    if (oracle_check_ids(edges, id_bytes, n, m)) return 1;
    for (int64_t i = 0; i < nstarts; i++)
        if (starts[i] < 0 || starts[i] >= n) return 1;
    int64_t *start = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *adj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!start || !adj || !fill || !queue) {
        free(start); free(adj); free(fill); free(queue);
        return 2;
    }
    for (int64_t i = 0; i < m; i++) {
        start[edge_at(edges, id_bytes, 2 * i) + 1]++;
        start[edge_at(edges, id_bytes, 2 * i + 1) + 1]++;
    }
    for (int64_t v = 0; v < n; v++) start[v + 1] += start[v];
    memcpy(fill, start, sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < m; i++) {
        int64_t u = edge_at(edges, id_bytes, 2 * i), v = edge_at(edges, id_bytes, 2 * i + 1);
        adj[fill[u]++] = v;
        adj[fill[v]++] = u;
    }
    for (int64_t v = 0; v < n; v++) dist[v] = -1;
    int64_t head = 0, tail = 0;
    for (int64_t i = 0; i < nstarts; i++)
        if (dist[starts[i]] < 0) {
            dist[starts[i]] = 0;
            queue[tail++] = starts[i];
        }
    while (head < tail) {
        int64_t x = queue[head++];
        if (cutoff > 0 && dist[x] >= cutoff) continue;
        for (int64_t k = start[x]; k < start[x + 1]; k++) {
            int64_t y = adj[k];
            if (dist[y] < 0) {
                dist[y] = dist[x] + 1;
                queue[tail++] = y;
            }
        }
    }
    free(start); free(adj); free(fill); free(queue);
    return 0;
}

/* ---------------- transitive closure (tiny n) ---------------- */
int oracle_closure_labels(const void *edges, int id_bytes, int64_t n, int64_t m, int64_t *labels) {
    if (n > 256) return 3;
    if (oracle_check_ids(edges, id_bytes, n, m)) return 1;
    unsigned char *R = (unsigned char *)calloc((size_t)(n * n + 1), 1);
    for (int64_t v = 0; v < n; v++) R[v * n + v] = 1;
    for (int64_t i = 0; i < m; i++) {
        int64_t u = edge_at(edges, id_bytes, 2 * i), v = edge_at(edges, id_bytes, 2 * i + 1);
        R[u * n + v] = 1;
        R[v * n + u] = 1;
    }
    for (int64_t k = 0; k < n; k++)
        for (int64_t i = 0; i < n; i++)
            if (R[i * n + k])
                for (int64_t j = 0; j < n; j++)
                    if (R[k * n + j]) R[i * n + j] = 1;
    for (int64_t v = 0; v < n; v++) {
        int64_t u = 0;
        while (!R[v * n + u]) u++;
        labels[v] = u;
    }
    free(R);
    return 0;
}

/* ---------------- degree distribution ---------------- */
int oracle_degrees(const void *edges, int id_bytes, int64_t n, int64_t m, int64_t *deg) {
    if (oracle_check_ids(edges, id_bytes, n, m)) return 1;
    for (int64_t v = 0; v < n; v++) deg[v] = 0;
    for (int64_t i = 0; i < 2 * m; i++) deg[edge_at(edges, id_bytes, i)]++;
    return 0;
}

/* hist must hold maxdeg+1 entries; returns maxdeg */
int64_t oracle_max_degree(const int64_t *deg, int64_t n) {
    int64_t mx = 0;
    for (int64_t v = 0; v < n; v++) if (deg[v] > mx) mx = deg[v];
    return mx;
}

void oracle_histogram(const int64_t *deg, int64_t n, int64_t *hist, int64_t len) {
    for (int64_t d = 0; d < len; d++) hist[d] = 0;
    for (int64_t v = 0; v < n; v++) hist[deg[v]]++;
}

/* ---------------- Hurwitz zeta ---------------- */
/*
 * Scaled Hurwitz zeta c^s * zeta(s, q) = sum_{k>=0} ((q+k)/c)^-s for s > 1,
 * q > 0, c > 0, by Euler-Maclaurin summation with N explicit terms:
 *   sum_{k<N} ((q+k)/c)^-s + A (q+N)/(s-1) + A/2
 *   + sum_{j=1..8} B_{2j}/(2j)! * s(s+1)...(s+2j-2) * A (q+N)^{-(2j-1)},
 * with A = ((q+N)/c)^-s. Scaling by c = xmin keeps every term of the K-S
 * ratio zeta(alpha, x) / zeta(alpha, xmin) in range when alpha * ln(xmin) is
 * large (tight tails at high degree); c = 1 gives zeta itself.
 */
double oracle_hurwitz_zeta_scaled(double s, double q, double c) {
    static const double B2j[9] = {0.0, 1.0 / 6.0, -1.0 / 30.0, 1.0 / 42.0, -1.0 / 30.0, 5.0 / 66.0,
                                  -691.0 / 2730.0, 7.0 / 6.0, -3617.0 / 510.0};
    const int N = 16;
    double sum = 0.0;
    for (int k = 0; k < N; k++) sum += pow((q + k) / c, -s);
    double a = q + N;
    double A = pow(a / c, -s);
    sum += A * a / (s - 1.0);
    sum += 0.5 * A;
    double rising = s;      /* s(s+1)...(s+2j-2) */
    double fact = 2.0;      /* (2j)! */
    double apow = A / a;    /* A * a^-(2j-1) */
    for (int j = 1; j <= 8; j++) {
        sum += B2j[j] / fact * rising * apow;
        rising *= (s + 2 * j - 1) * (s + 2 * j);
        fact *= (double)(2 * j + 1) * (double)(2 * j + 2);
        apow /= a * a;
    }
    return sum;
}

double oracle_hurwitz_zeta(double s, double q) { return oracle_hurwitz_zeta_scaled(s, q, 1.0); }

/* ---------------- power-law fit + K-S statistic ---------------- */
/*
 * hist[d], d in [0, len). Candidate rules as in the header. out[0] = min D, out[1] = alpha at the argmin,
 * out[2] = xmin at the argmin, out[3] = tail size there, out[4] = number of
 * candidates. If no candidate qualifies, D = 1, alpha = 0, xmin = 0.
 * Ties in D keep the smaller xmin.
 */
void oracle_ks_fit(const int64_t *hist, int64_t len, int64_t min_tail, int64_t min_distinct, double min_span,
                   double *out) {
    /* distinct degrees >= 1 in increasing order */
    int64_t nd = 0;
    for (int64_t d = 1; d < len; d++) if (hist[d] > 0) nd++;
    int64_t *xs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nd + 1));
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nd + 1));
    int64_t k = 0;
    for (int64_t d = 1; d < len; d++) if (hist[d] > 0) { xs[k] = d; cnt[k] = hist[d]; k++; }
    double best = 1.0, best_alpha = 0.0;
    int64_t best_xmin = 0, best_n = 0, ncand = 0;
    for (int64_t i = 0; i < nd; i++) {
        int64_t xmin = xs[i];
        int64_t N = 0;
        for (int64_t j = i; j < nd; j++) N += cnt[j];
        if (N < min_tail || nd - i < min_distinct) continue;
        if ((double)xs[nd - 1] < min_span * (double)xmin) continue;
        ncand++;
        double lsum = 0.0;
        for (int64_t j = i; j < nd; j++) lsum += (double)cnt[j] * log((double)xs[j] / ((double)xmin - 0.5));
        double alpha = 1.0 + (double)N / lsum;
        double Z = oracle_hurwitz_zeta_scaled(alpha, (double)xmin, (double)xmin);
        double D = 0.0, cum = 0.0;
        for (int64_t j = i; j < nd; j++) {
            double x = (double)xs[j];
            if (j > i) {
                /* x - 1, the last integer before this degree: S still holds the previous value */
                double P = 1.0 - oracle_hurwitz_zeta_scaled(alpha, x, (double)xmin) / Z;
                double dd = fabs(cum / (double)N - P);
                if (dd > D) D = dd;
            }
            cum += (double)cnt[j];
            double P = 1.0 - oracle_hurwitz_zeta_scaled(alpha, x + 1.0, (double)xmin) / Z;
            double dd = fabs(cum / (double)N - P);
            if (dd > D) D = dd;
        }
        if (D < best) {
            best = D;
            best_alpha = alpha;
            best_xmin = xmin;
            best_n = N;
        }
    }
    out[0] = best;
    out[1] = best_alpha;
    out[2] = (double)best_xmin;
    out[3] = (double)best_n;
    out[4] = (double)ncand;
    free(xs);
    free(cnt);
}

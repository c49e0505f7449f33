// Route prediction of the batched form (Algorithm 2 lines 1-3, Section 3.2,
// for each of G graphs): the degrees of every graph in one pass over the
// union, then one block per graph for its degree histogram, the power-law
// fit with the K-S statistic, the route and the max-degree seed. The
// arithmetic is the single-graph fit's (ks_math.cuh): fp32 screen of every
// (candidate, degree) term, fp64 refinement of the terms within the screen
// slack, minimum D over candidates with ties to the smaller xmin.
//
//  k_degree_batch   deg[vo[g] + x] = number of pair endpoints equal to local
//                   id x of graph g (local ids checked against n_g)
//  k_ks_batch       per graph: the distinct degrees (dense shared-memory bins
//                   below kBB, a sorted shared-memory list above), candidate
//                   setup, terms, selection; graphs with more than kBOvf
//                   vertices of degree >= kBB are flagged for the
//                   single-graph fit instead
//  k_merge_visited  after a graph's BFS: every visited vertex takes the
//                   visited minimum as parent (atomicMin keeps the forest)
#include "cc_common.cuh"
#include "cc_kernels.h"
#include "ks_math.cuh"

namespace ccg {

constexpr int kBB = 4096;          // dense degree bins per graph (degrees 1..kBB-1)
constexpr int kBOvf = 4096;        // degrees >= kBB held per graph
constexpr int kBThreads = 256;
constexpr int kZTab = 128;         // zeta table entries per warp (the refinement of step 6)
constexpr int kSmallHistKeyAt = 2 * kBB + 2;  // word of the argmax key in k_small_hist's output (8-byte aligned)

// ---------------------------------------------------------------------------
// Blocks take tiles of kBlock * kDegVec vectors (two pairs each) from `next`
// (a zeroed counter). The pairs are cut into R contiguous regions worked on
// side by side: fetch f takes tile f / R of region f % R. Within a region
// the tiles go in increasing order, so the tiles in flight stay within a
// window of a few graphs per region and their counters stay in L2 (with a
// fixed stride, blocks drift apart and the counters of many graphs compete
// for it). With R = 1 every SM works on the same graph at once, and the
// increments of that graph's hubs queue on a few L2 lines: on 512 graphs
// (R-MAT, grids, chains) the pass ran at 50% of the L2 atomic rate, its
// blocks stalled on their loads and their barrier whatever their vectors
// per thread (2, 4 or 8 measured 4.25-4.31 ms); with R = 8 it took 2.91 ms.
// Thread 0 fetches the next tile's number and first and last graph while
// the block's loads of the current tile are in flight (two slots in shared
// memory, one barrier per tile). A tile inside one graph - nearly every
// tile, since the graphs hold thousands to millions of pairs - reads that
// graph's base and size once; a tile across graphs finds each pair's graph
// by stepping from its first graph.
//
// With `hook` (the parent array, every vertex its own root) the pass also
// applies the first SV hook pass of Section 3.1 to every pair:
// atomicMin(parent[max], min) in union ids, while the graphs in flight have
// their parents in L2 beside their counts.
constexpr int kDegVec = 2;
__device__ __forceinline__ void batch_hook(vid_t *hook, long long a, long long b) {
    if (a == b) return;
    const vid_t hi = (vid_t)(a > b ? a : b), lo = (vid_t)(a > b ? b : a);
    atomicMin(&hook[hi], lo);
}

__global__ void __launch_bounds__(kBlock, 6) k_degree_batch(const int32_t *__restrict__ in, long long m,
                                                            const int64_t *__restrict__ eo,
                                                            const int64_t *__restrict__ vo, int G, uint32_t *deg,
                                                            DevState *st, unsigned long long *next, int regions,
                                                            vid_t *hook) {
    constexpr int V = kDegVec;
    __shared__ long long s_t[2];
    __shared__ int s_g0[2], s_g1[2];
    constexpr long long kTile = (long long)kBlock * V;
    const long long nvec = m >> 1;
    const long long ntiles = (nvec + kTile - 1) / kTile;
    const long long per = (ntiles + regions - 1) / regions;  // tiles per region
    const long long nfetch = per * regions;
    const int4 *ev = reinterpret_cast<const int4 *>(in);
    auto fetch = [&](int b) {  // thread 0; s_t: the tile, ntiles to skip a fetch past the last tile, -1 when done
        const long long f = (long long)atomicAdd(next, 1ull);
        long long t = f >= nfetch ? -1 : (f % regions) * per + f / regions;
        if (t >= ntiles) t = ntiles;
        s_t[b] = t;
        if (t >= 0 && t < ntiles) {
            const long long last = ((t + 1) * kTile < nvec ? (t + 1) * kTile : nvec) * 2 - 1;
            s_g0[b] = graph_search(eo, G, t * kTile * 2);
            s_g1[b] = graph_search(eo, G, last);
        }
    };
    if (threadIdx.x == 0) fetch(0);
    __syncthreads();
    bool bad = false;
    for (int b = 0;; b ^= 1) {
        const long long t = s_t[b];
        if (t < 0) break;
        if (t >= ntiles) {  // a fetch past the end of the last region: nothing to count
            if (threadIdx.x == 0) fetch(b ^ 1);
            __syncthreads();
            continue;
        }
        const int g0 = s_g0[b], g1 = s_g1[b];
        int4 q[V];
#pragma unroll
        for (int r = 0; r < V; r++) {
            const long long i = t * kTile + (long long)r * kBlock + threadIdx.x;
            q[r] = i < nvec ? ld_stream(ev + i) : make_int4(0, 0, 0, 0);
        }
        if (threadIdx.x == 0) fetch(b ^ 1);
        if (g0 == g1) {
            const long long base = vo[g0];
            const unsigned long long ng = (unsigned long long)(vo[g0 + 1] - base);
#pragma unroll
            for (int r = 0; r < V; r++) {
                const long long i = t * kTile + (long long)r * kBlock + threadIdx.x;
                if (i >= nvec) break;
                const int4 x = q[r];
                const bool ok0 = (unsigned long long)(long long)x.x < ng && (unsigned long long)(long long)x.y < ng;
                const bool ok1 = (unsigned long long)(long long)x.z < ng && (unsigned long long)(long long)x.w < ng;
                if (ok0) {
                    atomicAdd(&deg[base + x.x], 1u);
                    atomicAdd(&deg[base + x.y], 1u);
                    if (hook) batch_hook(hook, base + x.x, base + x.y);
                }
                if (ok1) {
                    atomicAdd(&deg[base + x.z], 1u);
                    atomicAdd(&deg[base + x.w], 1u);
                    if (hook) batch_hook(hook, base + x.z, base + x.w);
                }
                bad |= !(ok0 && ok1);
            }
        } else {
#pragma unroll
            for (int r = 0; r < V; r++) {
                const long long i = t * kTile + (long long)r * kBlock + threadIdx.x;
                if (i >= nvec) break;
                const int4 x = q[r];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const long long u = h ? x.z : x.x, v = h ? x.w : x.y;
                    const int g = graph_advance(eo, G, 2 * i + h, g0);
                    const long long base = vo[g];
                    const unsigned long long ng = (unsigned long long)(vo[g + 1] - base);
                    if ((unsigned long long)u >= ng || (unsigned long long)v >= ng) {
                        bad = true;
                        continue;
                    }
                    atomicAdd(&deg[base + u], 1u);
                    atomicAdd(&deg[base + v], 1u);
                    if (hook) batch_hook(hook, base + u, base + v);
                }
            }
        }
        __syncthreads();  // the slot read above is rewritten by the fetch after next
    }
    if ((m & 1) && blockIdx.x == 0 && threadIdx.x == 0) {  // the odd last pair
        const long long u = in[2 * (m - 1)], v = in[2 * (m - 1) + 1];
        const int g = graph_search(eo, G, m - 1);
        const long long base = vo[g];
        const unsigned long long ng = (unsigned long long)(vo[g + 1] - base);
        if ((unsigned long long)u >= ng || (unsigned long long)v >= ng) bad = true;
        else {
            atomicAdd(&deg[base + u], 1u);
            atomicAdd(&deg[base + v], 1u);
            if (hook) batch_hook(hook, base + u, base + v);
        }
    }
    if (bad) set_err(st, kErrInvalidEdge);
}

// ---------------------------------------------------------------------------
// Per-graph fit. Scratch per block (global): the distinct degrees xs, their
// counts, the exclusive prefix cum (cum[nd] = vertices of degree >= 1),
// ln x, and per candidate D, alpha, Z; kBB + kBOvf entries each.
// Graphs go to blocks largest first through a shared counter (`order`: the
// graphs by decreasing vertex count, `next`: zeroed), so the few largest
// fits start first and the small ones fill the gaps; without `next` block b
// takes graphs b, b + grid, ...
__global__ void __launch_bounds__(kBThreads, 3) k_ks_batch(const uint32_t *__restrict__ deg,
                                                        const int64_t *__restrict__ vo, int G, KsBatchScratch sc,
                                                        KsBatchOut out, long long min_tail, long long min_distinct,
                                                        double min_span, double tau, const int *__restrict__ order,
                                                        int *next, const uint32_t *__restrict__ pre) {
    __shared__ uint32_t hist[kBB];
    __shared__ uint32_t ovf[kBOvf];
    __shared__ unsigned long long s64[33];
    __shared__ int s_novf;
    __shared__ unsigned long long s_key;
    __shared__ double sel_D[kBThreads];
    __shared__ long long sel_I[kBThreads];
    __shared__ double sdbl[33];
    __shared__ long long s64l[33];
    __shared__ int s_gi;
    __shared__ double ztab[kBThreads / 32][kZTab];  // per warp: the zeta table of its contender
    constexpr int kCap = kBB + kBOvf;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kBThreads / 32;
    uint32_t *xs = sc.xs + (size_t)blockIdx.x * kCap;
    unsigned long long *cnt = sc.cnt + (size_t)blockIdx.x * kCap;
    unsigned long long *cum = sc.cum + (size_t)blockIdx.x * (kCap + 1);
    double *lnx = sc.lnx + (size_t)blockIdx.x * kCap;
    double *Dc = sc.Dc + (size_t)blockIdx.x * kCap;
    double *Ac = sc.Ac + (size_t)blockIdx.x * kCap;
    double *Zc = sc.Zc + (size_t)blockIdx.x * kCap;
    for (int gi = blockIdx.x;; gi += gridDim.x) {
        if (next) {
            if (tid == 0) s_gi = atomicAdd(next, 1);
            __syncthreads();
            gi = s_gi;
            __syncthreads();
        }
        if (gi >= G) break;
        const int g = order ? order[gi] : gi;
        const long long v0 = vo[g], ng = vo[g + 1] - v0;
        if (pre) {  // one graph, histogram built by k_small_hist over the whole grid
            for (int i = tid; i < kBB; i += kBThreads) hist[i] = pre[i];
            const unsigned cnt = pre[2 * kBB];
            for (int i = tid; i < kBOvf && i < (int)cnt; i += kBThreads) ovf[i] = pre[kBB + i];
            if (tid == 0) {
                s_novf = (int)(cnt < 0x7fffffffu ? cnt : 0x7fffffffu);
                s_key = *reinterpret_cast<const unsigned long long *>(pre + kSmallHistKeyAt);
            }
            __syncthreads();
        } else {
            // 1. histogram and argmax key (deg << 32) | ~local id
            for (int i = tid; i < kBB; i += kBThreads) hist[i] = 0;
            if (tid == 0) {
                s_novf = 0;
                s_key = 0;
            }
            __syncthreads();
            unsigned long long best = 0;
            // kHistLoads independent loads in flight per thread (one block walks the
            // whole graph, so the loop is bound by load latency, not bandwidth); lanes
            // holding the same degree add to its bin once (degrees of many graphs
            // are concentrated on a few values, whose bins would serialise the atomics).
            // The loop runs warp-uniformly so that every lane joins the match.
            constexpr int kHistLoads = 8;
            for (long long vb = (long long)(tid & ~31); vb < ng; vb += (long long)kBThreads * kHistLoads) {
                uint32_t dv[kHistLoads];
    #pragma unroll
                for (int q = 0; q < kHistLoads; q++) {
                    const long long w = vb + lane + (long long)q * kBThreads;
                    dv[q] = w < ng ? deg[v0 + w] : 0u;
                }
    #pragma unroll
                for (int q = 0; q < kHistLoads; q++) {
                    const long long w = vb + lane + (long long)q * kBThreads;
                    const uint32_t d = dv[q];
                    if (w < ng) {
                        const unsigned long long key =
                            ((unsigned long long)d << 32) | (0xffffffffull - (unsigned long long)w);
                        best = key > best ? key : best;
                    }
                    const uint32_t bin = (w < ng && d != 0 && d < (uint32_t)kBB) ? d : 0xffffffffu;
                    const unsigned peers = __match_any_sync(0xffffffffu, bin);
                    if (bin != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned)__popc(peers));
                    if (w < ng && d >= (uint32_t)kBB) {
                        const int k = atomicAdd(&s_novf, 1);
                        if (k < kBOvf) ovf[k] = d;
                    }
                }
            }
    #pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long b = __shfl_xor_sync(0xffffffffu, best, o);
                best = b > best ? b : best;
            }
            if (lane == 0 && best) atomicMax(&s_key, best);
            __syncthreads();
        }
        const int novf = s_novf;
        if (tid == 0) {
            out.seedkey[g] = s_key;
            out.overflow[g] = novf > kBOvf ? 1 : 0;
        }
        if (novf > kBOvf) {  // left to the single-graph fit (block-uniform)
            __syncthreads();
            continue;
        }
        // 2a. distinct dense degrees, increasing: thread t owns bins [16t, 16t + 16)
        constexpr int B = kBB / kBThreads;
        unsigned long long mynz = 0, mymass = 0;
#pragma unroll
        for (int k = 0; k < B; k++) {
            const int d = tid * B + k;
            const uint32_t h = d > 0 ? hist[d] : 0u;
            mynz += h ? 1 : 0;
            mymass += h;
        }
        unsigned long long tnz, tmass;
        unsigned long long o = block_exclusive_scan<unsigned long long>(mynz, s64, tnz);
        unsigned long long om = block_exclusive_scan<unsigned long long>(mymass, s64, tmass);
        for (int k = 0; k < B; k++) {
            const int d = tid * B + k;
            const uint32_t h = d > 0 ? hist[d] : 0u;
            if (h) {
                xs[o] = (uint32_t)d;
                cnt[o] = h;
                cum[o] = om;
                o++;
                om += h;
            }
        }
        // 2b. degrees >= kBB: bitonic sort in shared memory, then one entry per run
        int P = 1;
        while (P < novf) P <<= 1;
        for (int i = tid; i < P; i += kBThreads)
            if (i >= novf) ovf[i] = 0xffffffffu;
        __syncthreads();
        for (int size = 2; size <= P; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = tid; i < P; i += kBThreads) {
                    const int j = i ^ stride;
                    if (j > i) {
                        const bool up = (i & size) == 0;
                        const uint32_t a = ovf[i], b = ovf[j];
                        if ((a > b) == up) {
                            ovf[i] = b;
                            ovf[j] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        unsigned long long outn = 0;
        for (int r = 0; r < P; r += kBThreads) {
            const int i = r + tid;
            const bool head = i < novf && (i == 0 || ovf[i] != ovf[i - 1]);
            unsigned long long tot;
            const unsigned long long rank = block_exclusive_scan<unsigned long long>(head ? 1ull : 0ull, s64, tot);
            if (head) {
                int e = i + 1;
                while (e < novf && ovf[e] == ovf[i]) e++;
                const unsigned long long q = tnz + outn + rank;
                xs[q] = ovf[i];
                cnt[q] = (unsigned long long)(e - i);
                cum[q] = tmass + (unsigned long long)i;
            }
            outn += tot;
        }
        const long long nd = (long long)(tnz + outn);
        if (tid == 0) cum[nd] = tmass + (unsigned long long)novf;
        __syncthreads();
        // ln x of every distinct degree, one per thread (an owner of many
        // occupied bins would otherwise run its fp64 logs one after another)
        for (long long i = tid; i < nd; i += kBThreads) lnx[i] = log((double)xs[i]);
        __syncthreads();
        // 3. suffix sums SL[i] = sum_{j >= i} cnt[j] ln x[j] (fp64, one reverse
        //    pass in chunks of the block), kept in Zc: they make every
        //    candidate's exponent O(1) instead of a sum over its tail
        const unsigned long long total = nd > 0 ? cum[nd] : 0;
        const double xmax = nd > 0 ? (double)xs[nd - 1] : 0.0;
        {
            double carry = 0.0;  // sum over the entries above the current chunk
            for (long long c0 = ((nd - 1) / kBThreads) * kBThreads; c0 >= 0; c0 -= kBThreads) {
                const long long i = c0 + (kBThreads - 1 - tid);  // thread t takes the t-th from the top
                const double v = i < nd ? (double)cnt[i] * lnx[i] : 0.0;
                double tot;
                const double ex = block_exclusive_scan<double>(v, sdbl, tot);
                if (i < nd) Zc[i] = carry + ex + v;
                carry += tot;
            }
        }
        __syncthreads();
        // 4. candidates (one thread each): the tail rules; alpha by Clauset et
        //    al. eq. 3.7 from the suffix sum: sum_j cnt_j (ln x_j - ln(xmin - 1/2))
        //    = SL[i] - N ln(xmin - 1/2); marked with Dc = 0 (candidate) or 2
        long long nc = 0;
        for (long long i = tid; i < nd; i += kBThreads) {
            const double xmin = (double)xs[i];
            const unsigned long long Nt = total - cum[i];
            if ((long long)Nt < min_tail || nd - i < min_distinct || xmax < min_span * xmin) {
                Dc[i] = 2.0;
                continue;
            }
            Ac[i] = 1.0 + (double)Nt / (Zc[i] - (double)Nt * log(xmin - 0.5));
            Dc[i] = 0.0;
            nc++;
        }
        const long long ncand = block_reduce_sum<long long>(nc, s64l);
        // 5. screen (one warp per candidate): every term in fp32, with the
        //    normaliser zeta(alpha, xmin) in fp32 too; Dc[i] = the fp32 sup
        float fmin_t = 2.0f;
        for (long long i = warp; i < nd; i += nw) {
            if (Dc[i] > 1.0) continue;  // not a candidate (warp-uniform)
            const float alpha_f = (float)Ac[i], lnc_f = (float)lnx[i];
            const float Z_f = zeta_scaled_f(alpha_f, (float)xs[i], lnc_f);
            const unsigned long long ci = cum[i];
            const float invN_f = 1.0f / (float)(total - ci);
            float fm = 0.0f;
            for (long long j = i + lane; j < nd; j += 32) {
                // the empirical CDF fractions in fp32 too (an fp64 divide per term
                // kept the fp64 pipe busy); within ~1e-7 of the fp64 values
                const float before = (float)(cum[j] - ci) * invN_f, at = (float)(cum[j + 1] - ci) * invN_f;
                fm = fmaxf(fm, ks_term_f(alpha_f, Z_f, lnc_f, (float)xs[j], (float)lnx[j], before, at, j == i));
            }
#pragma unroll
            for (int o2 = 16; o2 > 0; o2 >>= 1) fm = fmaxf(fm, __shfl_xor_sync(0xffffffffu, fm, o2));
            if (lane == 0) Dc[i] = (double)fm;
            fmin_t = fminf(fmin_t, fm);
        }
        const double fmin = block_reduce_min((double)fmin_t, sdbl);
        // 6. refinement (one warp per contender): only a candidate whose fp32 sup
        //    is within two screen slacks of the smallest can hold the fp64
        //    minimum (the fp32 terms are within ~5e-6 of the fp64 ones); its
        //    normaliser and the terms within one slack of its fp32 sup are
        //    evaluated in fp64. The others are marked 1.5 (never selected).
        for (long long i = warp; i < nd; i += nw) {
            const double df = Dc[i];
            if (df > 1.0) continue;
            if (df > fmin + 2.0 * (double)kScreenSlack) {
                if (lane == 0) Dc[i] = 1.5;
                continue;
            }
            const double alpha = Ac[i], lnc = lnx[i];
            const long long xmin = (long long)xs[i];
            // the zeta terms below the remainder threshold once for this
            // exponent (one fp64 power per lane) instead of a loop of them per term
            double tail = 0.0;
            double *tab = ztab[warp];
            const long long T = zeta_table_warp(alpha, xmin, lnc, tab, kZTab, tail);
            const double Z = (T >= 0 && xmin < T) ? tab[0] + tail : zeta_scaled(alpha, (double)xmin, lnc);
            const float alpha_f = (float)alpha, lnc_f = (float)lnc;
            const float Z_f = zeta_scaled_f(alpha_f, (float)xs[i], lnc_f);
            const unsigned long long ci = cum[i];
            const double N = (double)(total - ci);
            const float invN_f = 1.0f / (float)(total - ci);
            const float cut = (float)df - kScreenSlack;
            double dm = 0.0;
            for (long long j = i + lane; j < nd; j += 32) {
                const double x = (double)xs[j];
                // the screen's fp32 term (the same arithmetic as in step 5)
                const float d32 = ks_term_f(alpha_f, Z_f, lnc_f, (float)x, (float)lnx[j], (float)(cum[j] - ci) * invN_f,
                                            (float)(cum[j + 1] - ci) * invN_f, j == i);
                if (d32 >= cut) {
                    const double before = (double)(cum[j] - ci) / N, at = (double)(cum[j + 1] - ci) / N;
                    double zb, za;
                    const long long xi = (long long)xs[j];
                    if (T >= 0 && xi < T) {
                        zb = tab[xi - xmin] + tail;
                        za = (xi + 1 < T ? tab[xi + 1 - xmin] : 0.0) + tail;
                    } else {
                        zeta_pair(alpha, x, lnx[j], lnc, zb, za);
                    }
                    double d = fabs(at - (1.0 - za / Z));
                    if (j > i) d = fmax(d, fabs(before - (1.0 - zb / Z)));
                    dm = fmax(dm, d);
                }
            }
#pragma unroll
            for (int o2 = 16; o2 > 0; o2 >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o2));
            if (lane == 0) Dc[i] = dm;
            __syncwarp();  // the table is rewritten for the warp's next contender
        }
        __syncthreads();
        // 5. selection: minimum D, ties to the smaller xmin (per-thread scan, then a block reduction)
        double bd = 2.0;
        long long bi = -1;
        for (long long i = tid; i < nd; i += kBThreads) {
            const double d = Dc[i];
            if (d <= 1.0 && d < bd) {  // i increases per thread, so ties keep the smaller i
                bd = d;
                bi = i;
            }
        }
        sel_D[tid] = bd;
        sel_I[tid] = bi;
        __syncthreads();
        for (int o2 = kBThreads / 2; o2 > 0; o2 >>= 1) {
            if (tid < o2) {
                const double d2 = sel_D[tid + o2];
                const long long i2 = sel_I[tid + o2];
                if (i2 >= 0 && (d2 < sel_D[tid] || (d2 == sel_D[tid] && (sel_I[tid] < 0 || i2 < sel_I[tid])))) {
                    sel_D[tid] = d2;
                    sel_I[tid] = i2;
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            const long long bi0 = sel_I[0];
            const double D = bi0 < 0 ? 1.0 : sel_D[0];
            out.D[g] = D;
            out.alpha[g] = bi0 < 0 ? 0.0 : Ac[bi0];
            out.xmin[g] = bi0 < 0 ? 0 : (long long)xs[bi0];
            out.ntail[g] = bi0 < 0 ? 0 : (long long)(total - cum[bi0]);
            out.ncand[g] = ncand;
            out.route[g] = D < tau ? 1 : 0;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// vis: the BFS's visited bitmap over local ids of graph g; cmin_local: its minimum.
__global__ void __launch_bounds__(kBlock) k_merge_visited(const uint32_t *__restrict__ vis, long long ng,
                                                          long long base, const DevState *st, vid_t *parent) {
    const vid_t c = st->cmin;
    if ((long long)c >= ng) return;
    for (long long v = gtid(); v < ng; v += gstride())
        if ((vis[v >> 5] >> (v & 31)) & 1u) atomicMin(&parent[base + v], (vid_t)(base + c));
}

// ---------------------------------------------------------------------------
// One graph through the per-graph fit: the offsets {0, n}, and the result
// copied into the fields the single-graph route reads (as k_ks_select and
// k_hist leave them).
__global__ void k_fit_one_offsets(int64_t *vo, long long n) {
    vo[0] = 0;
    vo[1] = n;
}
__global__ void k_fit_one_to_state(KsBatchOut out, DevState *st, double tau) {
    st->ks_out[0] = out.D[0];
    st->ks_out[1] = out.alpha[0];
    st->ks_out[2] = (double)out.xmin[0];
    st->ks_out[3] = (double)out.ntail[0];
    st->ks_out[4] = (double)out.ncand[0];
    st->ncand = (unsigned long long)out.ncand[0];
    st->route = out.D[0] < tau ? 1 : 0;
    st->maxkey = out.seedkey[0];
}

// The one-block fit's histogram over the whole grid (one block walking all
// n degrees was most of the fit on small graphs): h[d] for degrees 1..kBB-1
// (privatised per block), the degrees >= kBB listed from h[kBB] on (their
// count at h[2 kBB]; at most kBOvf kept), the argmax key at kSmallHistKeyAt.
__global__ void __launch_bounds__(kBlock) k_small_hist(const uint32_t *__restrict__ deg, long long n, uint32_t *h) {
    __shared__ uint32_t sh[kBB];
    for (int i = threadIdx.x; i < kBB; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    unsigned long long best = 0;
    for (long long v = gtid(); v < n; v += gstride()) {
        const uint32_t d = deg[v];
        const unsigned long long key = ((unsigned long long)d << 32) | (0xffffffffull - (unsigned long long)v);
        best = key > best ? key : best;
        if (d == 0) continue;
        if (d < (uint32_t)kBB) {
            atomicAdd(&sh[d], 1u);
        } else {
            const unsigned k = atomicAdd(&h[2 * kBB], 1u);
            if (k < (unsigned)kBOvf) h[kBB + k] = d;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, best, o);
        best = b > best ? b : best;
    }
    if ((threadIdx.x & 31) == 0 && best)
        atomicMax(reinterpret_cast<unsigned long long *>(h + kSmallHistKeyAt), best);
    __syncthreads();
    for (int i = threadIdx.x; i < kBB; i += blockDim.x)
        if (sh[i]) atomicAdd(&h[i], sh[i]);
}

size_t small_hist_words() { return (size_t)kSmallHistKeyAt + 2; }

void launch_fit_one(const uint32_t *deg, long long n, int64_t *vo, KsBatchScratch sc, KsBatchOut out, DevState *st,
                    long long min_tail, long long min_distinct, double min_span, double tau, uint32_t *hist_scratch,
                    int grid, cudaStream_t s) {
    k_fit_one_offsets<<<1, 1, 0, s>>>(vo, n);
    if (hist_scratch) {
        cudaMemsetAsync(hist_scratch, 0, small_hist_words() * 4, s);
        k_small_hist<<<fit_grid((const void *)k_small_hist, grid, kBlock), kBlock, 0, s>>>(deg, n, hist_scratch);
    }
    k_ks_batch<<<1, kBThreads, 0, s>>>(deg, vo, 1, sc, out, min_tail, min_distinct, min_span, tau, nullptr, nullptr,
                                       hist_scratch);
    k_fit_one_to_state<<<1, 1, 0, s>>>(out, st, tau);
}

// ---------------------------------------------------------------------------
void launch_degree_batch(const int32_t *in, long long m, const int64_t *eo, const int64_t *vo, int G, uint32_t *deg,
                         DevState *st, int grid, unsigned long long *next, int regions, cudaStream_t s, vid_t *hook) {
    if (m <= 0) return;
    cudaMemsetAsync(next, 0, sizeof(unsigned long long), s);
    k_degree_batch<<<fit_grid((const void *)k_degree_batch, grid, kBlock), kBlock, 0, s>>>(
        in, m, eo, vo, G, deg, st, next, regions > 0 ? regions : 1, hook);
}

__global__ void __launch_bounds__(kBlock) k_tile_graphs(const int64_t *__restrict__ off, int G, long long ntiles,
                                                        uint32_t *out) {
    for (long long k = gtid(); k < ntiles; k += gstride()) out[k] = (uint32_t)graph_search(off, G, k << kTileShift);
}

void launch_tile_graphs(const int64_t *off, int G, long long count, uint32_t *out, int grid, cudaStream_t s) {
    const long long ntiles = (count >> kTileShift) + 1;
    k_tile_graphs<<<grid, kBlock, 0, s>>>(off, G, ntiles, out);
}

size_t ks_batch_entries() { return (size_t)(kBB + kBOvf); }

void launch_ks_batch(const uint32_t *deg, const int64_t *vo, int G, KsBatchScratch sc, KsBatchOut out,
                     long long min_tail, long long min_distinct, double min_span, double tau, int blocks,
                     const int *order, int *next, cudaStream_t s) {
    if (G <= 0) return;
    if (next) cudaMemsetAsync(next, 0, sizeof(int), s);
    k_ks_batch<<<blocks < G ? blocks : G, kBThreads, 0, s>>>(deg, vo, G, sc, out, min_tail, min_distinct, min_span,
                                                             tau, order, next, nullptr);
}

void launch_merge_visited(const uint32_t *vis, long long ng, long long base, const DevState *st, vid_t *parent,
                          int grid, cudaStream_t s) {
    if (ng > 0) k_merge_visited<<<grid, kBlock, 0, s>>>(vis, ng, base, st, parent);
}

}  // namespace ccg

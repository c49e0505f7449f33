// Degree pass of the batched form (Algorithm 2 line 1 for each of G graphs)
// with the counts in shared memory, and with the first SV hook pass of
// Section 3.1 (atomicMin(parent[max], min), every vertex its own root)
// applied in the same pass. The L2 form (k_degree_batch) makes three
// scattered L2 atomics per pair; here every one of them happens in shared
// memory:
//
//  k_bwin_plan        one block: each graph g of at most 2^20 vertices gets
//                     nw_g = ceil(n_g / 2^12) windows of 4,096 vertices and
//                     a region of nw_g * cap_g entries, cap_g = 3 m_g / nw_g
//                     + 64 (1.5 times the average of a window), by two
//                     exclusive scans over the graphs
//  k_bwin_graphs      the graph of every window; clears the windows' fill
//                     counters and flags
//  k_degree_split_batch  two CTAs of 512 threads per SM stream 24 KB chunks of
//                     pairs into shared memory (bulk copies, two in flight).
//                     Each endpoint x of graph g (local ids) becomes the
//                     32-bit entry (x mod 4096) | partner << 12 of window
//                     wo[g] + x / 4096; the chunk's entries are counting-
//                     sorted by window in shared memory (staged as window <<
//                     32 | entry, one 8-byte access each way), one reservation
//                     per window and chunk, and written out run by run
//  k_degree_window_batch  one CTA per window counts its entries and hooks its
//                     vertices in shared memory (the window's sampled hub in
//                     registers), then writes deg and parent once
//
// Entries that do not fit this scheme are counted and hooked with global
// atomics directly, so the result is exact for any batch: the pairs of a
// graph of more than 2^20 vertices (its partner ids need more than 20 bits),
// the entries of a window past its capacity, and every pair of a chunk whose
// graphs span more than 512 windows (graphs of a few pairs each); a window
// that received such entries adds its counts and takes the minimum of its
// parents instead of storing them.
//
// The graph of a chunk's first pair comes from the tile table of the batch
// (the graph of every 2^kTileShift-th pair): the chunks are multiples of that
// tile, so no search is needed.
#include "cc_common.cuh"
#include "cc_kernels.h"

namespace ccg {

constexpr int kBWinBits = 12;                      // vertices per window
constexpr int kBWinSize = 1 << kBWinBits;
constexpr long long kBMaxN = 1LL << (32 - kBWinBits);  // graphs with more vertices go direct
constexpr int kBSplitThreads = 512;
constexpr int kBSplitChunk = 24576;                // bytes of int32 pairs per chunk (3,072 pairs)
constexpr int kBSplitVecs = kBSplitChunk / 16;
constexpr int kBSplitSlots = kBSplitVecs / kBSplitThreads;
constexpr int kBSplitPairs = kBSplitChunk / 8;
constexpr int kBSplitMaxEnd = 2 * kBSplitPairs;
constexpr int kBMaxWin = 512;                      // windows of one chunk
constexpr int kBWinThreads = 256;
constexpr int kBSampleVecs = 512;                  // 2,048 entries sampled for the window's hub
constexpr unsigned long long kBWaitNs = 1000000000ull;  // bounded mbarrier waits: 1 s
static_assert(kBSplitPairs % (1 << kTileShift) == 0, "chunks are whole tiles of the tile table");
static_assert(kBSplitVecs % kBSplitThreads == 0, "whole vectors per thread");

// Scratch layout (bytes): the counters and tables first, the regions after.
struct BWinLayout {
    size_t wo, rog, capg, wg, fill, dirty, tot, part, bytes;
    long long wmax;
};

static BWinLayout bwin_layout(long long m, long long n, int G) {
    BWinLayout L{};
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    L.wmax = (n >> kBWinBits) + G + 1;  // >= sum of ceil(n_g / 4096)
    size_t o = 0;
    L.tot = o;
    o = up(o + 16);
    L.wo = o;
    o = up(o + ((size_t)G + 1) * 4);
    L.rog = o;
    o = up(o + ((size_t)G + 1) * 8);
    L.capg = o;
    o = up(o + ((size_t)G + 1) * 4);
    L.wg = o;
    o = up(o + (size_t)L.wmax * 4);
    L.fill = o;
    o = up(o + (size_t)L.wmax * 4);
    L.dirty = o;
    o = up(o + (size_t)L.wmax * 4);
    L.part = o;
    // sum of nw_g * cap_g <= 3m + 68 * (number of windows)
    o = up(o + ((size_t)3 * (size_t)m + 68 * (size_t)L.wmax + 4) * 4);
    L.bytes = o;
    return L;
}

size_t batch_win_scratch_bytes(long long m, long long n, int G) { return bwin_layout(m, n, G).bytes; }

// One block: windows and regions of every graph (two exclusive scans over
// the graphs in rounds of the block's size); tot[0] = windows, tot[1..2] =
// region entries (64-bit).
__global__ void __launch_bounds__(1024) k_bwin_plan(const int64_t *__restrict__ eo, const int64_t *__restrict__ vo,
                                                    int G, uint32_t *wo, unsigned long long *rog, uint32_t *capg,
                                                    uint32_t *tot) {
    __shared__ uint32_t s_w[32];
    __shared__ unsigned long long s_r[32];
    __shared__ uint32_t c_w;
    __shared__ unsigned long long c_r;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) {
        c_w = 0u;
        c_r = 0ull;
    }
    __syncthreads();
    for (int g0 = 0; g0 < G; g0 += blockDim.x) {
        const int g = g0 + t;
        uint32_t nw = 0u, cap = 0u;
        if (g < G) {
            const long long ng = vo[g + 1] - vo[g], mg = eo[g + 1] - eo[g];
            if (ng > 0 && ng <= kBMaxN) {
                nw = (uint32_t)((ng + kBWinSize - 1) >> kBWinBits);
                cap = (uint32_t)(((3 * mg + nw - 1) / nw + 64 + 3) & ~3LL);
            }
        }
        unsigned long long r = (unsigned long long)nw * cap;
        uint32_t iw = nw;
        unsigned long long ir = r;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t yw = __shfl_up_sync(0xffffffffu, iw, o);
            const unsigned long long yr = __shfl_up_sync(0xffffffffu, ir, o);
            if (lane >= o) {
                iw += yw;
                ir += yr;
            }
        }
        if (lane == 31) {
            s_w[warp] = iw;
            s_r[warp] = ir;
        }
        __syncthreads();
        if (warp == 0) {
            const int nwp = blockDim.x >> 5;
            uint32_t w = lane < nwp ? s_w[lane] : 0u, wi = w;
            unsigned long long rr = lane < nwp ? s_r[lane] : 0ull, ri = rr;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t yw = __shfl_up_sync(0xffffffffu, wi, o);
                const unsigned long long yr = __shfl_up_sync(0xffffffffu, ri, o);
                if (lane >= o) {
                    wi += yw;
                    ri += yr;
                }
            }
            if (lane < nwp) {
                s_w[lane] = wi - w;
                s_r[lane] = ri - rr;
            }
        }
        __syncthreads();
        if (g < G) {
            wo[g] = c_w + s_w[warp] + iw - nw;
            rog[g] = c_r + s_r[warp] + ir - r;
            capg[g] = cap;
        }
        __syncthreads();
        if (t == blockDim.x - 1) {
            c_w += s_w[warp] + iw;
            c_r += s_r[warp] + ir;
        }
        __syncthreads();
    }
    if (t == 0) {
        wo[G] = c_w;
        rog[G] = c_r;
        capg[G] = 0u;
        tot[0] = c_w;
        *reinterpret_cast<unsigned long long *>(tot + 2) = c_r;
    }
}

// The graph of every window (the last g with wo[g] <= w); fill and dirty cleared.
__global__ void __launch_bounds__(kBlock) k_bwin_graphs(const uint32_t *__restrict__ wo, int G, long long wmax,
                                                        const uint32_t *__restrict__ tot, uint32_t *wg, uint32_t *fill,
                                                        uint32_t *dirty) {
    const uint32_t W = tot[0];
    for (long long w = gtid(); w < wmax; w += gstride()) {
        fill[w] = 0u;
        dirty[w] = 0u;
        if (w < W) {
            int lo = 0, hi = G - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((long long)wo[mid] <= w) lo = mid;
                else hi = mid - 1;
            }
            wg[w] = (uint32_t)lo;
        }
    }
}

struct __align__(128) BSplitShared {
    int4 buf[2][kBSplitVecs];        // two chunks of pairs (bulk-copy destinations)
    unsigned long long se[kBSplitMaxEnd];  // window within the chunk's range << 32 | entry, in window order
    uint32_t hist[kBMaxWin];
    unsigned long long goff[kBMaxWin];  // the window's region + its reservation - its first stage slot
    uint32_t loff[kBMaxWin];         // the window's first stage slot
    uint32_t gend[kBMaxWin];         // the end of its stage slots that fit in the region
    uint32_t vx0[kBMaxWin];          // the union id of the window's first vertex
    uint32_t vg[kBMaxWin];           // the union id of its graph's first vertex
    unsigned long long mbar[2];
    int g0[2], g1[2];                // first and last graph of the chunk in each buffer
    uint32_t wsum[kBSplitThreads / 32];
};

__device__ __forceinline__ uint32_t bs_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bs_try(unsigned long long *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bs_smem(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool bs_wait(unsigned long long *b, uint32_t parity) {
    if (bs_try(b, parity)) return true;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (bs_try(b, parity)) return true;
        unsigned long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        if (t1 - t0 > kBWaitNs) return false;
    }
}

// Count and hook one pair of graph g (union base vb) with global atomics.
__device__ __forceinline__ void bwin_direct(long long u, long long v, long long vb, uint32_t *deg, vid_t *hook) {
    atomicAdd(&deg[vb + u], 1u);
    atomicAdd(&deg[vb + v], 1u);
    if (hook && u != v) {
        const vid_t hi = (vid_t)(vb + (u > v ? u : v)), lo = (vid_t)(vb + (u > v ? v : u));
        atomicMin(&hook[hi], lo);
    }
}

__global__ void __launch_bounds__(kBSplitThreads, 2)
    k_degree_split_batch(const int32_t *__restrict__ edges, long long m, const int64_t *__restrict__ eo,
                         const int64_t *__restrict__ vo, int G, const uint32_t *__restrict__ tile_pairs,
                         const uint32_t *__restrict__ wo, const unsigned long long *__restrict__ rog,
                         const uint32_t *__restrict__ capg, const uint32_t *__restrict__ wg, uint32_t *fill,
                         uint32_t *dirty, uint32_t *__restrict__ part, uint32_t *deg, vid_t *hook, DevState *st) {
    extern __shared__ __align__(128) unsigned char bsplit_smem[];
    BSplitShared &S = *reinterpret_cast<BSplitShared *>(bsplit_smem);
    constexpr long long CP = kBSplitPairs;
    constexpr int NE = kBSplitSlots * 2;  // pairs per thread and chunk
    constexpr int NW = kBSplitThreads / 32;
    constexpr int WPT = kBMaxWin / kBSplitThreads;
    static_assert(kBMaxWin % kBSplitThreads == 0, "whole windows per thread in the scan");
    const long long nch = (m + CP - 1) / CP;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long G2 = gridDim.x;
    constexpr uint32_t kLow = kBWinSize - 1u;
    auto chunk_len = [&](long long c) { return m - c * CP < CP ? m - c * CP : CP; };
    bool inflight[2] = {false, false};
    auto issue = [&](long long c, int slot) {  // thread 0
        const long long np = chunk_len(c);
        const int ga = (int)tile_pairs[(c * CP) >> kTileShift];
        S.g0[slot] = ga;
        S.g1[slot] = graph_advance(eo, G, c * CP + np - 1, (int)tile_pairs[(c * CP + np - 1) >> kTileShift]);
        const uint32_t bytes = (uint32_t)(((unsigned long long)np * 8ull) & ~15ull);
        if (bytes) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bs_smem(&S.mbar[slot])),
                         "r"(bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    bs_smem(S.buf[slot])),
                "l"((unsigned long long)__cvta_generic_to_global(edges + 2 * c * CP)), "r"(bytes),
                "r"(bs_smem(&S.mbar[slot]))
                : "memory");
        } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bs_smem(&S.mbar[slot])) : "memory");
        }
        inflight[slot] = true;
    };
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bs_smem(&S.mbar[0])), "r"(1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bs_smem(&S.mbar[1])), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = t; i < kBMaxWin; i += kBSplitThreads) S.hist[i] = 0u;
    __syncthreads();
    if (t == 0) {
        if (blockIdx.x < nch) issue(blockIdx.x, 0);
        if (blockIdx.x + G2 < nch) issue(blockIdx.x + G2, 1);
    }
    uint32_t phase[2] = {0u, 0u};
    bool bad = false, timed_out = false;
    int slot = 0;
    for (long long c = blockIdx.x; c < nch; c += G2, slot ^= 1) {
        const bool ok = bs_wait(&S.mbar[slot], phase[slot]);
        if (ok) phase[slot] ^= 1u;
        const int np = (int)chunk_len(c);
        const int full_vecs = (np * 8) >> 4;
        const int g0 = S.g0[slot], g1 = S.g1[slot];
        const uint32_t wlo = wo[g0], nbw = wo[g1 + 1] - wlo;
        const bool direct = nbw > (uint32_t)kBMaxWin;  // block-uniform
        // the chunk's first graph (most chunks lie in one graph: their windows
        // start at wlo, so a window is x / 4096 and no offset is read per pair)
        const bool one = g0 == g1;
        const long long vb0 = vo[g0];
        const long long ng0 = vo[g0 + 1] - vb0;
        uint32_t pe[2 * NE], rk[NE];
        uint16_t pb[2 * NE];
#pragma unroll
        for (int k = 0; k < kBSplitSlots; k++) {
            const int sv = t + k * kBSplitThreads;
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const int p = sv * 2 + j;
                uint32_t r = 0xffffffffu;
                if (ok && p < np) {
                    long long u, v;
                    if (sv < full_vecs) vec_pair<int32_t>(S.buf[slot][sv], j, u, v);
                    else scalar_pair<int32_t>(edges, c * CP + p, u, v);  // the odd last pair
                    int g = g0;
                    long long vb = vb0, ng = ng0;
                    uint32_t wg0 = 0u;  // the graph's first window - wlo
                    if (!one) {
                        g = graph_advance(eo, G, c * CP + p, g0);
                        vb = vo[g];
                        ng = vo[g + 1] - vb;
                        wg0 = wo[g] - wlo;
                    }
                    if ((unsigned long long)u >= (unsigned long long)ng ||
                        (unsigned long long)v >= (unsigned long long)ng) {
                        bad = true;
                    } else if (direct || ng > kBMaxN) {
                        bwin_direct(u, v, vb, deg, hook);
                        if (ng <= kBMaxN) {  // the windows of both ends add instead of storing
                            atomicOr(&dirty[wo[g] + ((uint32_t)u >> kBWinBits)], 1u);
                            atomicOr(&dirty[wo[g] + ((uint32_t)v >> kBWinBits)], 1u);
                        }
                    } else {
                        const uint32_t bu = wg0 + ((uint32_t)u >> kBWinBits), bv = wg0 + ((uint32_t)v >> kBWinBits);
                        pe[2 * (k * 2 + j)] = ((uint32_t)u & kLow) | ((uint32_t)v << kBWinBits);
                        pe[2 * (k * 2 + j) + 1] = ((uint32_t)v & kLow) | ((uint32_t)u << kBWinBits);
                        pb[2 * (k * 2 + j)] = (uint16_t)bu;
                        pb[2 * (k * 2 + j) + 1] = (uint16_t)bv;
                        r = atomicAdd(&S.hist[bu], 1u) | (atomicAdd(&S.hist[bv], 1u) << 16);
                    }
                }
                rk[k * 2 + j] = r;
            }
        }
        // barrier 1: the counts are complete and the buffer is read
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        if (t == 0) {
            inflight[slot] = false;
            if (c + 2 * G2 < nch) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(c + 2 * G2, slot);
            }
        }
        if (direct) continue;  // uniform: nothing was counted in shared memory
        // exclusive scan of the window counts, one reservation per window and chunk
        uint32_t h[WPT], bt[WPT], hs = 0u;
#pragma unroll
        for (int q = 0; q < WPT; q++) {
            const int b = t * WPT + q;
            h[q] = 0u;
            bt[q] = 0u;
            if (b < (int)nbw) {
                h[q] = S.hist[b];
                S.hist[b] = 0u;
                if (h[q]) bt[q] = atomicAdd(&fill[wlo + b], h[q]);
            }
            hs += h[q];
        }
        uint32_t incl = hs;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) S.wsum[warp] = incl;
        __syncthreads();  // barrier 2
        uint32_t w = lane < NW ? S.wsum[lane] : 0u, wi = w;
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, wi, NW - 1);
        uint32_t lo = __shfl_sync(0xffffffffu, wi - w, warp) + incl - hs;
        bool short_fit = false;
#pragma unroll
        for (int q = 0; q < WPT; q++) {
            const int b = t * WPT + q;
            S.loff[b] = lo;
            if (h[q]) {
                const uint32_t wgl = wlo + (uint32_t)b;
                const int gw = (int)wg[wgl];
                const uint32_t cap = capg[gw];
                const uint32_t k = wgl - wo[gw];
                const uint32_t fit = bt[q] >= cap ? 0u : (cap - bt[q] < h[q] ? cap - bt[q] : h[q]);
                S.gend[b] = lo + fit;
                S.goff[b] = rog[gw] + (unsigned long long)k * cap + bt[q] - lo;
                S.vg[b] = (uint32_t)vo[gw];
                S.vx0[b] = (uint32_t)vo[gw] + (k << kBWinBits);
                short_fit |= fit < h[q];
            }
            lo += h[q];
        }
        // barrier 3; `over`: a window of this chunk runs past its capacity
        const int over = __syncthreads_or(short_fit);
#pragma unroll
        for (int k = 0; k < NE; k++) {
            const uint32_t r = rk[k];
            if (r == 0xffffffffu) continue;
            const uint32_t bu = pb[2 * k], bv = pb[2 * k + 1];
            S.se[S.loff[bu] + (r & 0xffffu)] = ((unsigned long long)bu << 32) | pe[2 * k];
            S.se[S.loff[bv] + (r >> 16)] = ((unsigned long long)bv << 32) | pe[2 * k + 1];
        }
        __syncthreads();  // barrier 4
        if (!over) {
            for (uint32_t i = t; i < tot; i += kBSplitThreads) {
                const unsigned long long x = S.se[i];
                part[S.goff[x >> 32] + i] = (uint32_t)x;
            }
        } else {
            for (uint32_t i = t; i < tot; i += kBSplitThreads) {
                const unsigned long long x = S.se[i];
                const uint32_t b = (uint32_t)(x >> 32), e = (uint32_t)x;
                if (i < S.gend[b]) {
                    part[S.goff[b] + i] = e;
                } else {  // past the region: counted and hooked here
                    const uint32_t x = S.vx0[b] + (e & kLow), y = S.vg[b] + (e >> kBWinBits);
                    atomicAdd(&deg[x], 1u);
                    if (hook && y < x) atomicMin(&hook[x], y);
                }
            }
        }
        // the next chunk's counts go to S.hist (cleared before barrier 2);
        // its scan rewrites loff / gend / goff / vx0 / vg only after its barrier 1
    }
    if (bad) set_err(st, kErrInvalidEdge);
    if (timed_out && t == 0) {
        set_err(st, kErrTimeout);
        for (int k = 0; k < 2; k++)  // leave no copy writing into shared memory after the block exits
            if (inflight[k]) bs_wait(&S.mbar[k], phase[k]);
    }
}

__device__ __forceinline__ void bwin_one(uint32_t e, uint32_t x0, uint32_t hub, uint32_t *cnt, uint32_t *spar,
                                         uint32_t &hc, uint32_t &hmin, bool hooks) {
    const uint32_t xl = e & (kBWinSize - 1u), y = e >> kBWinBits;
    if (xl == hub) {
        hc++;
        if (y < x0 + xl && y < hmin) hmin = y;
    } else {
        atomicAdd(&cnt[xl], 1u);
        if (hooks && y < x0 + xl) atomicMin(&spar[xl], y);
    }
}

__global__ void __launch_bounds__(kBWinThreads) k_degree_window_batch(
    const uint32_t *__restrict__ part, const int64_t *__restrict__ vo, const uint32_t *__restrict__ wo,
    const unsigned long long *__restrict__ rog, const uint32_t *__restrict__ capg, const uint32_t *__restrict__ wg,
    const uint32_t *__restrict__ fill, const uint32_t *__restrict__ dirty, const uint32_t *__restrict__ tot,
    uint32_t *deg, vid_t *hook) {
    __shared__ uint32_t cnt[kBWinSize];
    __shared__ uint32_t spar[kBWinSize];  // the smallest neighbour below each vertex (local ids)
    __shared__ uint32_t red[kBWinThreads / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t w = blockIdx.x;
    if (w >= tot[0]) return;
    const int g = (int)wg[w];
    const uint32_t k = w - wo[g];
    const uint32_t x0 = k << kBWinBits;  // local id of the window's first vertex
    const long long vb = vo[g];
    const uint32_t ng = (uint32_t)(vo[g + 1] - vb);
    const uint32_t lim = ng - x0 < (uint32_t)kBWinSize ? ng - x0 : (uint32_t)kBWinSize;
    const uint32_t cap = capg[g];
    const uint32_t f = fill[w], len = f < cap ? f : cap;
    const bool add = f > cap || dirty[w] != 0u;
    const bool hooks = hook != nullptr;
    for (int i = t; i < kBWinSize; i += kBWinThreads) {
        cnt[i] = 0u;
        spar[i] = x0 + (uint32_t)i;
    }
    __syncthreads();
    const uint32_t *p = part + rog[g] + (unsigned long long)k * cap;  // 16-byte aligned: cap is a multiple of 4
    const uint4 *p4 = reinterpret_cast<const uint4 *>(p);
    const uint32_t nv = len >> 2;
    const uint32_t ns = nv < (uint32_t)kBSampleVecs ? nv : (uint32_t)kBSampleVecs;
    uint32_t hc = 0u, hmin = 0xffffffffu;
    for (uint32_t i = t; i < ns; i += kBWinThreads) {  // the sample, counted plainly
        const uint4 q = __ldcs(p4 + i);
        const uint32_t e4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; j++) bwin_one(e4[j], x0, 0xffffffffu, cnt, spar, hc, hmin, hooks);
    }
    __syncthreads();
    // the hub: the largest sample count (count << 16 | id; counts <= 2,048)
    uint32_t key = 0u;
    for (int i = t; i < kBWinSize; i += kBWinThreads) {
        const uint32_t c = cnt[i];
        if (c && ((c << 16) | (uint32_t)i) > key) key = (c << 16) | (uint32_t)i;
    }
    key = __reduce_max_sync(0xffffffffu, key);
    if (lane == 0) red[warp] = key;
    __syncthreads();
    key = 0u;
#pragma unroll
    for (int i = 0; i < kBWinThreads / 32; i++) key = red[i] > key ? red[i] : key;
    const uint32_t hub = key ? (key & 0xffffu) : 0xffffffffu;
    constexpr int U = 4;
    for (uint32_t i = ns + t; i < nv; i += U * kBWinThreads) {
        uint4 q[U];
#pragma unroll
        for (int j = 0; j < U; j++)
            if (i + j * kBWinThreads < nv) q[j] = __ldcs(p4 + i + j * kBWinThreads);
#pragma unroll
        for (int j = 0; j < U; j++) {
            if (i + j * kBWinThreads >= nv) break;
            bwin_one(q[j].x, x0, hub, cnt, spar, hc, hmin, hooks);
            bwin_one(q[j].y, x0, hub, cnt, spar, hc, hmin, hooks);
            bwin_one(q[j].z, x0, hub, cnt, spar, hc, hmin, hooks);
            bwin_one(q[j].w, x0, hub, cnt, spar, hc, hmin, hooks);
        }
    }
    if ((nv << 2) + t < len) bwin_one(p[(nv << 2) + t], x0, hub, cnt, spar, hc, hmin, hooks);  // len % 4 < 256
    hc = __reduce_add_sync(0xffffffffu, hc);
    hmin = __reduce_min_sync(0xffffffffu, hmin);
    if (lane == 0 && hc) {
        atomicAdd(&cnt[hub], hc);
        if (hooks && hmin != 0xffffffffu) atomicMin(&spar[hub], hmin);
    }
    __syncthreads();
    uint32_t *d = deg + vb + x0;
    vid_t *pa = hooks ? hook + vb + x0 : nullptr;
    const uint32_t base = (uint32_t)vb;
    if (add) {
        for (uint32_t i = t; i < lim; i += kBWinThreads) {
            d[i] += cnt[i];
            if (hooks) atomicMin(&pa[i], base + spar[i]);
        }
    } else {
        for (uint32_t i = t; i < lim; i += kBWinThreads) {
            d[i] = cnt[i];
            if (hooks) pa[i] = base + spar[i];
        }
    }
}

bool degree_batch_win_ok(long long m, long long n) { return m >= (1LL << 20) && n < (1LL << 31); }

void launch_degree_batch_win(const int32_t *in, long long m, const int64_t *eo, const int64_t *vo, int G, long long n,
                             const uint32_t *tile_pairs, uint32_t *deg, DevState *st, void *scratch, int num_sms,
                             cudaStream_t s, vid_t *hook) {
    if (m <= 0 || G <= 0) return;
    const BWinLayout L = bwin_layout(m, n, G);
    char *b = static_cast<char *>(scratch);
    uint32_t *tot = reinterpret_cast<uint32_t *>(b + L.tot), *wo = reinterpret_cast<uint32_t *>(b + L.wo);
    unsigned long long *rog = reinterpret_cast<unsigned long long *>(b + L.rog);
    uint32_t *capg = reinterpret_cast<uint32_t *>(b + L.capg), *wg = reinterpret_cast<uint32_t *>(b + L.wg);
    uint32_t *fill = reinterpret_cast<uint32_t *>(b + L.fill), *dirty = reinterpret_cast<uint32_t *>(b + L.dirty);
    uint32_t *part = reinterpret_cast<uint32_t *>(b + L.part);
    k_bwin_plan<<<1, 1024, 0, s>>>(eo, vo, G, wo, rog, capg, tot);
    const long long wblocks = (L.wmax + kBlock - 1) / kBlock;
    k_bwin_graphs<<<(unsigned)(wblocks < 4LL * num_sms * 8 ? wblocks : 4LL * num_sms * 8), kBlock, 0, s>>>(
        wo, G, L.wmax, tot, wg, fill, dirty);
    const long long nch = (m + kBSplitPairs - 1) / kBSplitPairs;
    const int pgrid = (int)(nch < 2LL * num_sms ? nch : 2LL * num_sms);
    k_degree_split_batch<<<pgrid, kBSplitThreads, sizeof(BSplitShared), s>>>(in, m, eo, vo, G, tile_pairs, wo, rog,
                                                                            capg, wg, fill, dirty, part, deg, hook,
                                                                            st);
    k_degree_window_batch<<<(unsigned)L.wmax, kBWinThreads, 0, s>>>(part, vo, wo, rog, capg, wg, fill, dirty, tot, deg,
                                                                   hook);
}

cudaError_t batch_win_setup() {
    return cudaFuncSetAttribute((const void *)k_degree_split_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(BSplitShared));
}

}  // namespace ccg

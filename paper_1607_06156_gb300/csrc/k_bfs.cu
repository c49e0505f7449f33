// BFS step of the hybrid route (Section 3.2, Algorithm 2 lines 5-9).
//
//  scan      exclusive prefix sum (tile reduce, tile-offset scan, tile scan)
//  CSR       row_ptr = exclusive scan of the degrees; every pair is stored in
//            both directions (Section 3.2 stores each undirected edge as two
//            directed edges) by an atomic cursor per vertex.
//  BFS       level-synchronous, direction optimizing (Beamer et al., cited in
//            Section 1): top-down levels expand the frontier queue edge-parallel
//            (a scan of the frontier degrees splits the work evenly, so a hub
//            of any degree is spread over the whole grid); bottom-up levels give
//            each warp one 32-vertex word of the visited bitmap, every
//            unvisited lane scans its adjacency until it meets a frontier
//            vertex, and the warp's ballot is the word of the next frontier.
//  cmin      smallest visited id: the label the BFS component ends with.
#include "cc_common.cuh"
#include "cc_kernels.h"

namespace ccg {

// ---------------------------------------------------------------------------
// Exclusive scan of uint32 values into uint32 prefix sums (the total must fit).
constexpr int kScanItems = 8;
constexpr int kScanTile = kBlock * kScanItems;

__device__ __forceinline__ unsigned long long block_scan_excl_u64(unsigned long long x, unsigned long long &total) {
    __shared__ unsigned long long sw[33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sw[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < nw ? sw[lane] : 0ull, wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) sw[lane] = wi - w;
        if (lane == nw - 1) sw[32] = wi;
    }
    __syncthreads();
    const unsigned long long r = sw[warp] + incl - x;
    total = sw[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kBlock) k_scan_up(const uint32_t *__restrict__ in, long long len,
                                                    unsigned long long *tsum) {
    const long long t0 = (long long)blockIdx.x * kScanTile;
    unsigned long long s = 0;
    for (int k = 0; k < kScanItems; k++) {
        const long long i = t0 + (long long)threadIdx.x * kScanItems + k;
        if (i < len) s += in[i];
    }
    unsigned long long tot;
    block_scan_excl_u64(s, tot);
    if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kBlock) k_scan_mid(unsigned long long *tsum, long long ntiles,
                                                     unsigned long long *total_out, uint32_t *total_u32) {
    unsigned long long carry = 0;
    for (long long r = 0; r < ntiles; r += blockDim.x) {
        const long long i = r + threadIdx.x;
        const unsigned long long x = i < ntiles ? tsum[i] : 0ull;
        unsigned long long tot;
        const unsigned long long e = block_scan_excl_u64(x, tot);
        if (i < ntiles) tsum[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
    if (threadIdx.x == 0 && total_u32) *total_u32 = (uint32_t)carry;
}

__global__ void __launch_bounds__(kBlock) k_scan_down(const uint32_t *__restrict__ in, long long len,
                                                      const unsigned long long *__restrict__ tsum, uint32_t *out,
                                                      uint32_t *out_copy) {
    const long long t0 = (long long)blockIdx.x * kScanTile;
    uint32_t v[kScanItems];
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const long long i = t0 + (long long)threadIdx.x * kScanItems + k;
        v[k] = i < len ? in[i] : 0u;
        s += v[k];
    }
    unsigned long long tot;
    unsigned long long run = tsum[blockIdx.x] + block_scan_excl_u64(s, tot);
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const long long i = t0 + (long long)threadIdx.x * kScanItems + k;
        if (i < len) {
            out[i] = (uint32_t)run;
            if (out_copy) out_copy[i] = (uint32_t)run;
        }
        run += v[k];
    }
}

void launch_scan_u32(const uint32_t *in, long long len, uint32_t *out, uint32_t *out_copy, unsigned long long *tsum,
                     unsigned long long *total_dev, uint32_t *total_u32, cudaStream_t s) {
    if (len <= 0) return;
    const long long ntiles = (len + kScanTile - 1) / kScanTile;
    k_scan_up<<<(unsigned)ntiles, kBlock, 0, s>>>(in, len, tsum);
    k_scan_mid<<<1, kBlock, 0, s>>>(tsum, ntiles, total_dev, total_u32);
    k_scan_down<<<(unsigned)ntiles, kBlock, 0, s>>>(in, len, tsum, out, out_copy);
}

long long scan_num_tiles(long long len) { return (len + kScanTile - 1) / kScanTile; }

// ---------------------------------------------------------------------------
// CSR scatter: both directions of every valid pair.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_csr_scatter(const T *__restrict__ edges, long long m, vid_t n,
                                                        uint32_t *cursor, vid_t *col) {
    constexpr int P = PairVec<T>::kPairs;
    const long long nvec = m / P;
    const int4 *ev = reinterpret_cast<const int4 *>(edges);
    for (long long i = gtid(); i < nvec; i += gstride()) {
        const int4 q = ld_stream(ev + i);
#pragma unroll
        for (int j = 0; j < P; j++) {
            long long u, v;
            vec_pair<T>(q, j, u, v);
            if ((unsigned long long)u >= n || (unsigned long long)v >= n) continue;
            col[atomicAdd(&cursor[u], 1u)] = (vid_t)v;
            col[atomicAdd(&cursor[v], 1u)] = (vid_t)u;
        }
    }
    if (P == 2 && (m & 1) && gtid() == 0) {
        long long u, v;
        scalar_pair<T>(edges, m - 1, u, v);
        if ((unsigned long long)u < n && (unsigned long long)v < n) {
            col[atomicAdd(&cursor[u], 1u)] = (vid_t)v;
            col[atomicAdd(&cursor[v], 1u)] = (vid_t)u;
        }
    }
}

template <typename T>
void launch_csr_scatter(const void *edges, long long m, vid_t n, uint32_t *cursor, vid_t *col, int grid,
                        cudaStream_t s) {
    if (m <= 0) return;
    k_csr_scatter<T><<<grid, kBlock, 0, s>>>((const T *)edges, m, n, cursor, col);
}
template void launch_csr_scatter<int32_t>(const void *, long long, vid_t, uint32_t *, vid_t *, int, cudaStream_t);
template void launch_csr_scatter<int64_t>(const void *, long long, vid_t, uint32_t *, vid_t *, int, cudaStream_t);

// ---------------------------------------------------------------------------
// BFS

__global__ void k_bfs_init(const uint32_t *__restrict__ row_ptr, vid_t n, uint32_t *vis, vid_t *queue,
                           DevState *st) {
    vid_t s = 0xffffffffu - (vid_t)(st->maxkey & 0xffffffffull);
    if (s >= n) s = 0;
    vis[s >> 5] |= 1u << (s & 31);
    queue[0] = s;
    st->front[0] = 1;
    st->front_edges[0] = row_ptr[s + 1] - row_ptr[s];
    st->cmin = 0xffffffffu;
}

// dq[i] = degree of the i-th frontier vertex
__global__ void __launch_bounds__(kBlock) k_front_degrees(const vid_t *__restrict__ queue, long long f,
                                                          const uint32_t *__restrict__ row_ptr, uint32_t *dq) {
    for (long long i = gtid(); i < f; i += gstride()) {
        const vid_t v = queue[i];
        dq[i] = row_ptr[v + 1] - row_ptr[v];
    }
}

// Top-down: edge slot e of the frontier belongs to frontier vertex k with
// off[k] <= e < off[k] + dq[k]; found by binary search over off.
__global__ void __launch_bounds__(kBlock) k_bfs_topdown(const vid_t *__restrict__ queue, long long f,
                                                        const uint32_t *__restrict__ off, long long total,
                                                        const uint32_t *__restrict__ row_ptr,
                                                        const vid_t *__restrict__ col, uint32_t *vis, vid_t *next,
                                                        DevState *st, int level) {
    const long long stride = gstride();
    const long long rounds = (total + stride - 1) / stride;
    unsigned long long new_edges = 0;
    for (long long r = 0; r < rounds; r++) {
        const long long e = gtid() + r * stride;
        bool fresh = false;
        vid_t w = 0;
        if (e < total) {
            long long lo = 0, hi = f - 1;  // largest k with off[k] <= e
            while (lo < hi) {
                const long long mid = (lo + hi + 1) >> 1;
                if ((long long)off[mid] <= e) lo = mid;
                else hi = mid - 1;
            }
            const vid_t v = queue[lo];
            const uint32_t k = (uint32_t)(e - (long long)off[lo]), b0 = row_ptr[v];
            if (k < row_ptr[v + 1] - b0) {  // always true when total matches the frontier's degree sum
                w = col[b0 + k];
                const uint32_t bit = 1u << (w & 31);
                if (!(__ldcg(&vis[w >> 5]) & bit)) {
                    const uint32_t old = atomicOr(&vis[w >> 5], bit);
                    fresh = !(old & bit);
                }
            }
        }
        const unsigned long long k = warp_append(&st->front[level + 1], fresh);
        if (fresh) {
            next[k] = w;
            new_edges += row_ptr[w + 1] - row_ptr[w];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) new_edges += __shfl_xor_sync(0xffffffffu, new_edges, o);
    if ((threadIdx.x & 31) == 0 && new_edges) atomicAdd(&st->front_edges[level + 1], new_edges);
    if (gtid() == 0) atomicAdd(&st->bfs_inspected, (unsigned long long)total);
}

// Bottom-up: warp w owns vertex word w. Lanes of unvisited vertices with
// neighbours scan their adjacency for a frontier member (bitmap fb).
__global__ void __launch_bounds__(kBlock) k_bfs_bottomup(vid_t n, const uint32_t *__restrict__ row_ptr,
                                                         const vid_t *__restrict__ col,
                                                         const uint32_t *__restrict__ fb, uint32_t *vis, uint32_t *nb,
                                                         DevState *st, int level) {
    const long long nwords = ((long long)n + 31) / 32;
    const int lane = threadIdx.x & 31;
    const long long warp0 = gtid() >> 5, nwarps = gstride() >> 5;
    unsigned long long inspected = 0, new_edges = 0, found_total = 0;
    for (long long w = warp0; w < nwords; w += nwarps) {
        const uint32_t vword = vis[w];
        const long long v = w * 32 + lane;
        bool found = false;
        uint32_t d = 0;
        if (v < (long long)n && !((vword >> lane) & 1u)) {
            const uint32_t b = row_ptr[v], e = row_ptr[v + 1];
            d = e - b;
            for (uint32_t k = b; k < e; k++) {
                const vid_t x = col[k];
                inspected++;
                if ((fb[x >> 5] >> (x & 31)) & 1u) {
                    found = true;
                    break;
                }
            }
        }
        const uint32_t fmask = __ballot_sync(0xffffffffu, found);
        if (found) new_edges += d;
        if (lane == 0) {
            nb[w] = fmask;
            if (fmask) vis[w] = vword | fmask;
            found_total += __popc(fmask);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        inspected += __shfl_xor_sync(0xffffffffu, inspected, o);
        new_edges += __shfl_xor_sync(0xffffffffu, new_edges, o);
    }
    if (lane == 0) {
        if (found_total) atomicAdd(&st->front[level + 1], found_total);
        if (new_edges) atomicAdd(&st->front_edges[level + 1], new_edges);
        if (inspected) atomicAdd(&st->bfs_inspected, inspected);
    }
}

// queue -> bitmap (bitmap cleared beforehand)
__global__ void __launch_bounds__(kBlock) k_queue_to_bitmap(const vid_t *__restrict__ queue, long long f,
                                                            uint32_t *bm) {
    for (long long i = gtid(); i < f; i += gstride()) {
        const vid_t v = queue[i];
        atomicOr(&bm[v >> 5], 1u << (v & 31));
    }
}

// bitmap -> queue (order of appearance is irrelevant to the BFS)
__global__ void __launch_bounds__(kBlock) k_bitmap_to_queue(const uint32_t *__restrict__ bm, long long nwords,
                                                            vid_t *queue, unsigned long long *count) {
    const long long stride = gstride();
    const long long rounds = (nwords + stride - 1) / stride;
    for (long long r = 0; r < rounds; r++) {
        const long long w = gtid() + r * stride;
        uint32_t bits = w < nwords ? bm[w] : 0u;
        const int c = __popc(bits);
        // warp-aggregated reservation of c slots per lane
        unsigned long long incl = (unsigned long long)c;
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned long long wtot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0;
        if (lane == 31 && wtot) base = atomicAdd(count, wtot);
        base = __shfl_sync(0xffffffffu, base, 31) + incl - (unsigned long long)c;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            queue[base++] = (vid_t)(w * 32 + b);
        }
    }
}

// ---------------------------------------------------------------------------
// Edge-list BFS (bfs_mode 1): one level is one streaming pass over the
// active pairs, no CSR. A pair with one end in the frontier bitmap claims
// the other end if it is unvisited (atomicOr on the visited bitmap decides
// the single winner, which also enters the next frontier). A pair whose ends
// are both visited after the level can never claim again (and the SV step
// drops it anyway), so it leaves the active list; with WRITE the surviving
// pairs are compacted into `out`. front[level + 1] counts the claimed
// vertices, front_edges[level + 1] the surviving pairs.
template <typename T> struct EdgeUnroll { static constexpr int U = 2; };
template <> struct EdgeUnroll<int64_t> { static constexpr int U = 4; };

__device__ __forceinline__ bool bit_test(const uint32_t *b, long long v) { return (b[v >> 5] >> (v & 31)) & 1u; }

__device__ __forceinline__ bool claim(uint32_t *vis, uint32_t *next, long long v) {
    const uint32_t bit = 1u << (v & 31);
    if (__ldcg(&vis[v >> 5]) & bit) return false;
    if (atomicOr(&vis[v >> 5], bit) & bit) return false;
    atomicOr(&next[v >> 5], bit);
    return true;
}

template <typename T, bool WRITE>
__global__ void __launch_bounds__(kBlock) k_bfs_edges(const T *__restrict__ in, long long m, vid_t n, uint32_t *vis,
                                                      const uint32_t *__restrict__ cur, uint32_t *next,
                                                      uint2 *__restrict__ out, DevState *st, int level) {
    constexpr int P = PairVec<T>::kPairs;
    constexpr int U = EdgeUnroll<T>::U;
    constexpr int K = P * U;
    __shared__ int sw[32];
    __shared__ unsigned long long sbase;
    const long long nvec = m / P;
    const int4 *ev = reinterpret_cast<const int4 *>(in);
    const long long tile = (long long)kBlock * U;
    const long long ntiles = (nvec + tile - 1) / tile;
    unsigned long long claimed = 0, kept_total = 0;
    for (long long t = blockIdx.x; t < ntiles + (P == 2 && (m & 1) ? 1 : 0); t += gridDim.x) {
        long long u[K], v[K];
        bool valid[K];
        if (t < ntiles) {
            int4 q[U];
#pragma unroll
            for (int k = 0; k < U; k++) {
                const long long i = t * tile + (long long)k * kBlock + threadIdx.x;
                q[k] = i < nvec ? ld_stream(ev + i) : make_int4(0, 0, 0, 0);
            }
#pragma unroll
            for (int k = 0; k < U; k++) {
                const long long i = t * tile + (long long)k * kBlock + threadIdx.x;
#pragma unroll
                for (int j = 0; j < P; j++) {
                    vec_pair<T>(q[k], j, u[k * P + j], v[k * P + j]);
                    valid[k * P + j] = i < nvec;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; k++) {
                u[k] = v[k] = 0;
                valid[k] = false;
            }
            if (threadIdx.x == 0) {
                scalar_pair<T>(in, m - 1, u[0], v[0]);
                valid[0] = true;
            }
        }
        bool keep[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            keep[k] = false;
            if (!valid[k] || (unsigned long long)u[k] >= n || (unsigned long long)v[k] >= n) continue;
            const bool fu = bit_test(cur, u[k]), fv = bit_test(cur, v[k]);
            const bool vu0 = fu || bit_test(vis, u[k]), vv0 = fv || bit_test(vis, v[k]);
            if (fu && !vv0 && claim(vis, next, v[k])) claimed++;
            if (fv && !vu0 && claim(vis, next, u[k])) claimed++;
            // after this pair's claims: u is visited if it was, or if v is in the frontier
            keep[k] = !((vu0 || fv) && (vv0 || fu));
        }
        int c = 0;
#pragma unroll
        for (int k = 0; k < K; k++) c += keep[k];
        kept_total += (unsigned long long)c;
        if (WRITE) {
            unsigned long long o = block_reserve(&st->front_edges[level + 1], c, sw, &sbase);
#pragma unroll
            for (int k = 0; k < K; k++)
                if (keep[k]) out[o++] = make_uint2((vid_t)u[k], (vid_t)v[k]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        claimed += __shfl_xor_sync(0xffffffffu, claimed, o);
        kept_total += __shfl_xor_sync(0xffffffffu, kept_total, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (claimed) atomicAdd(&st->front[level + 1], claimed);
        if (!WRITE && kept_total) atomicAdd(&st->front_edges[level + 1], kept_total);
    }
}

__global__ void k_edge_bfs_seed(uint32_t *vis, uint32_t *cur, vid_t n, const unsigned long long *key, DevState *st) {
    vid_t s = 0xffffffffu - (vid_t)(*key & 0xffffffffull);
    if (s >= n) s = 0;
    vis[s >> 5] |= 1u << (s & 31);
    cur[s >> 5] |= 1u << (s & 31);
    st->front[0] = 1;
    st->cmin = 0xffffffffu;
}

template <typename T>
void launch_bfs_edges(bool write, const void *in, long long m, vid_t n, uint32_t *vis, const uint32_t *cur,
                      uint32_t *next, uint2 *out, DevState *st, int level, int grid, cudaStream_t s) {
    if (m <= 0) return;
    auto kf = write ? k_bfs_edges<T, true> : k_bfs_edges<T, false>;
    kf<<<fit_grid((const void *)kf, grid, kBlock), kBlock, 0, s>>>((const T *)in, m, n, vis, cur, next, out, st, level);
}
template void launch_bfs_edges<int32_t>(bool, const void *, long long, vid_t, uint32_t *, const uint32_t *, uint32_t *,
                                        uint2 *, DevState *, int, int, cudaStream_t);
template void launch_bfs_edges<int64_t>(bool, const void *, long long, vid_t, uint32_t *, const uint32_t *, uint32_t *,
                                        uint2 *, DevState *, int, int, cudaStream_t);
template void launch_bfs_edges<uint32_t>(bool, const void *, long long, vid_t, uint32_t *, const uint32_t *,
                                         uint32_t *, uint2 *, DevState *, int, int, cudaStream_t);

void launch_edge_bfs_seed(uint32_t *vis, uint32_t *cur, vid_t n, const unsigned long long *key, DevState *st,
                          cudaStream_t s) {
    k_edge_bfs_seed<<<1, 1, 0, s>>>(vis, cur, n, key, st);
}

// smallest set bit of the visited bitmap
__global__ void __launch_bounds__(kBlock) k_first_visited(const uint32_t *__restrict__ vis, long long nwords,
                                                          DevState *st) {
    for (long long w = gtid(); w < nwords; w += gstride()) {
        const uint32_t b = vis[w];
        if (b) {
            atomicMin(&st->cmin, (uint32_t)(w * 32 + __ffs(b) - 1));
            return;  // later words of this thread hold larger ids
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_popcount(const uint32_t *__restrict__ bm, long long nwords,
                                                     unsigned long long *out) {
    unsigned long long c = 0;
    for (long long w = gtid(); w < nwords; w += gstride()) c += __popc(bm[w]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

void launch_bfs_init(const uint32_t *row_ptr, vid_t n, uint32_t *vis, vid_t *queue, DevState *st, cudaStream_t s) {
    k_bfs_init<<<1, 1, 0, s>>>(row_ptr, n, vis, queue, st);
}
void launch_front_degrees(const vid_t *queue, long long f, const uint32_t *row_ptr, uint32_t *dq, int grid,
                          cudaStream_t s) {
    if (f > 0) k_front_degrees<<<grid, kBlock, 0, s>>>(queue, f, row_ptr, dq);
}
void launch_bfs_topdown(const vid_t *queue, long long f, const uint32_t *off, long long total, const uint32_t *row_ptr,
                        const vid_t *col, uint32_t *vis, vid_t *next, DevState *st, int level, int grid,
                        cudaStream_t s) {
    if (f > 0 && total > 0)
        k_bfs_topdown<<<grid, kBlock, 0, s>>>(queue, f, off, total, row_ptr, col, vis, next, st, level);
}
void launch_bfs_bottomup(vid_t n, const uint32_t *row_ptr, const vid_t *col, const uint32_t *fb, uint32_t *vis,
                         uint32_t *nb, DevState *st, int level, int grid, cudaStream_t s) {
    k_bfs_bottomup<<<grid, kBlock, 0, s>>>(n, row_ptr, col, fb, vis, nb, st, level);
}
void launch_queue_to_bitmap(const vid_t *queue, long long f, uint32_t *bm, int grid, cudaStream_t s) {
    if (f > 0) k_queue_to_bitmap<<<grid, kBlock, 0, s>>>(queue, f, bm);
}
void launch_bitmap_to_queue(const uint32_t *bm, long long nwords, vid_t *queue, unsigned long long *count, int grid,
                            cudaStream_t s) {
    k_bitmap_to_queue<<<grid, kBlock, 0, s>>>(bm, nwords, queue, count);
}
void launch_first_visited(const uint32_t *vis, long long nwords, DevState *st, int grid, cudaStream_t s) {
    k_first_visited<<<grid, kBlock, 0, s>>>(vis, nwords, st);
}
void launch_popcount(const uint32_t *bm, long long nwords, unsigned long long *out, int grid, cudaStream_t s) {
    k_popcount<<<grid, kBlock, 0, s>>>(bm, nwords, out);
}

// ---------------------------------------------------------------------------
// Device-driven BFS for the stream-ordered cc_labels: the level loop is the
// body of a CUDA graph WHILE node. Each level's frontier size, direction
// and buffers are read from DevState, so no level needs the host. The
// decisions are those of the host loop: Beamer's switching rule (go
// bottom-up when the frontier's edges exceed 1/14 of the unexplored edges,
// come back when the frontier holds fewer than n/24 vertices and shrinks),
// and the same frontier bookkeeping (front[l], front_edges[l]).
// Frontier buffers come in pairs: queue / bitmap number bfs_par is current.

constexpr double kBeamerAlpha = 14.0, kBeamerBeta = 24.0;

__device__ __forceinline__ bool bfs_continue(const DevState *st, int l, unsigned long long f) {
    return f > 0 && l < kMaxLevels - 1 && (st->bfs_cutoff <= 0 || l < st->bfs_cutoff);
}

__global__ void k_bfsg_init(const uint32_t *__restrict__ row_ptr, vid_t n, uint32_t *vis, vid_t *q0, DevState *st,
                            cudaGraphConditionalHandle h) {
    vid_t s = 0xffffffffu - (vid_t)(st->maxkey & 0xffffffffull);
    if (s >= n) s = 0;
    vis[s >> 5] |= 1u << (s & 31);
    q0[0] = s;
    st->front[0] = 1;
    st->front_edges[0] = row_ptr[s + 1] - row_ptr[s];
    st->cmin = 0xffffffffu;
    st->bfs_level = 0;
    st->bfs_par = 0;
    st->bfs_bu = 0;
    st->bfs_queue = 1;
    st->bfs_list = -1;
    st->bfs_explored = 0;
    st->bfs_prev_f = 0;
    cudaGraphSetConditional(h, bfs_continue(st, 0, 1ull) ? 1u : 0u);
}

// direction of this level and the frontier conversion it needs
__global__ void k_bfsg_plan(DevState *st, vid_t n, unsigned long long total_edges) {
    const int l = st->bfs_level;
    const unsigned long long f = st->front[l], fe = st->front_edges[l];
    int bu = st->bfs_bu;
    const unsigned long long unexplored = total_edges > st->bfs_explored ? total_edges - st->bfs_explored : 0;
    if (!bu && (double)fe > (double)unexplored / kBeamerAlpha) bu = 1;
    else if (bu && (double)f < (double)n / kBeamerBeta && f < st->bfs_prev_f) bu = 0;
    st->bfs_bu = bu;
    const int conv = bu && st->bfs_queue ? 1 : (!bu && !st->bfs_queue ? 2 : 0);
    st->bfs_conv = conv;
    if (conv == 2) st->bfs_qcount = 0;
}

// queue -> bitmap, first step: clear the current bitmap
__global__ void __launch_bounds__(kBlock) k_bfsg_q2b_clear(uint32_t *b0, uint32_t *b1, long long nwords,
                                                           const DevState *st) {
    if (st->bfs_conv != 1) return;
    uint32_t *b = st->bfs_par ? b1 : b0;
    for (long long w = gtid(); w < nwords; w += gstride()) b[w] = 0u;
}

__global__ void __launch_bounds__(kBlock) k_bfsg_q2b(const vid_t *q0, const vid_t *q1, uint32_t *b0, uint32_t *b1,
                                                     const DevState *st) {
    if (st->bfs_conv != 1) return;
    const int par = st->bfs_par;
    const vid_t *q = par ? q1 : q0;
    uint32_t *b = par ? b1 : b0;
    const long long f = (long long)st->front[st->bfs_level];
    for (long long i = gtid(); i < f; i += gstride()) atomicOr(&b[q[i] >> 5], 1u << (q[i] & 31));
}

__global__ void __launch_bounds__(kBlock) k_bfsg_b2q(const uint32_t *b0, const uint32_t *b1, long long nwords,
                                                     vid_t *q0, vid_t *q1, DevState *st) {
    if (st->bfs_conv != 2) return;
    const int par = st->bfs_par;
    const uint32_t *bm = par ? b1 : b0;
    vid_t *queue = par ? q1 : q0;
    const long long stride = gstride();
    const long long rounds = (nwords + stride - 1) / stride;
    const int lane = threadIdx.x & 31;
    for (long long r = 0; r < rounds; r++) {
        const long long w = gtid() + r * stride;
        uint32_t bits = w < nwords ? bm[w] : 0u;
        const int c = __popc(bits);
        unsigned long long incl = (unsigned long long)c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned long long wtot = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0;
        if (lane == 31 && wtot) base = atomicAdd(&st->bfs_qcount, wtot);
        base = __shfl_sync(0xffffffffu, base, 31) + incl - (unsigned long long)c;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            queue[base++] = (vid_t)(w * 32 + b);
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_bfsg_front_degrees(const vid_t *q0, const vid_t *q1,
                                                               const uint32_t *__restrict__ row_ptr, uint32_t *dq,
                                                               const DevState *st) {
    if (st->bfs_bu) return;
    const vid_t *q = st->bfs_par ? q1 : q0;
    const long long f = (long long)st->front[st->bfs_level];
    for (long long i = gtid(); i < f; i += gstride()) dq[i] = row_ptr[q[i] + 1] - row_ptr[q[i]];
}

// Exclusive scan of dq over the frontier (top-down levels only), tiles
// taken grid-stride by a fixed grid.
__global__ void __launch_bounds__(kBlock) k_bfsg_scan_up(const uint32_t *__restrict__ in, unsigned long long *tsum,
                                                         const DevState *st) {
    if (st->bfs_bu) return;
    const long long len = (long long)st->front[st->bfs_level];
    const long long ntiles = (len + kScanTile - 1) / kScanTile;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        unsigned long long s = 0;
        for (int k = 0; k < kScanItems; k++) {
            const long long i = t * kScanTile + (long long)threadIdx.x * kScanItems + k;
            if (i < len) s += in[i];
        }
        unsigned long long tot;
        block_scan_excl_u64(s, tot);
        if (threadIdx.x == 0) tsum[t] = tot;
    }
}

__global__ void __launch_bounds__(kBlock) k_bfsg_scan_mid(unsigned long long *tsum, const DevState *st) {
    if (st->bfs_bu) return;
    const long long len = (long long)st->front[st->bfs_level];
    const long long ntiles = (len + kScanTile - 1) / kScanTile;
    unsigned long long carry = 0;
    for (long long r = 0; r < ntiles; r += blockDim.x) {
        const long long i = r + threadIdx.x;
        const unsigned long long x = i < ntiles ? tsum[i] : 0ull;
        unsigned long long tot;
        const unsigned long long e = block_scan_excl_u64(x, tot);
        if (i < ntiles) tsum[i] = carry + e;
        carry += tot;
    }
}

__global__ void __launch_bounds__(kBlock) k_bfsg_scan_down(const uint32_t *__restrict__ in,
                                                           const unsigned long long *__restrict__ tsum, uint32_t *out,
                                                           const DevState *st) {
    if (st->bfs_bu) return;
    const long long len = (long long)st->front[st->bfs_level];
    const long long ntiles = (len + kScanTile - 1) / kScanTile;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint32_t v[kScanItems];
        unsigned long long s = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const long long i = t * kScanTile + (long long)threadIdx.x * kScanItems + k;
            v[k] = i < len ? in[i] : 0u;
            s += v[k];
        }
        unsigned long long tot;
        unsigned long long run = tsum[t] + block_scan_excl_u64(s, tot);
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            const long long i = t * kScanTile + (long long)threadIdx.x * kScanItems + k;
            if (i < len) out[i] = (uint32_t)run;
            run += v[k];
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_bfsg_topdown(const vid_t *q0, const vid_t *q1,
                                                         const uint32_t *__restrict__ off,
                                                         const uint32_t *__restrict__ row_ptr,
                                                         const vid_t *__restrict__ col, uint32_t *vis, vid_t *nq0,
                                                         vid_t *nq1, DevState *st) {
    if (st->bfs_bu) return;
    const int level = st->bfs_level, par = st->bfs_par;
    const vid_t *queue = par ? q1 : q0;
    vid_t *next = par ? nq0 : nq1;
    const long long f = (long long)st->front[level], total = (long long)st->front_edges[level];
    const long long stride = gstride();
    const long long rounds = (total + stride - 1) / stride;
    unsigned long long new_edges = 0;
    for (long long r = 0; r < rounds; r++) {
        const long long e = gtid() + r * stride;
        bool fresh = false;
        vid_t w = 0;
        if (e < total) {
            long long lo = 0, hi = f - 1;  // largest k with off[k] <= e
            while (lo < hi) {
                const long long mid = (lo + hi + 1) >> 1;
                if ((long long)off[mid] <= e) lo = mid;
                else hi = mid - 1;
            }
            const vid_t v = queue[lo];
            const uint32_t k = (uint32_t)(e - (long long)off[lo]), b0 = row_ptr[v];
            if (k < row_ptr[v + 1] - b0) {
                w = col[b0 + k];
                const uint32_t bit = 1u << (w & 31);
                if (!(__ldcg(&vis[w >> 5]) & bit)) {
                    const uint32_t old = atomicOr(&vis[w >> 5], bit);
                    fresh = !(old & bit);
                }
            }
        }
        const unsigned long long k = warp_append(&st->front[level + 1], fresh);
        if (fresh) {
            next[k] = w;
            new_edges += row_ptr[w + 1] - row_ptr[w];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) new_edges += __shfl_xor_sync(0xffffffffu, new_edges, o);
    if ((threadIdx.x & 31) == 0 && new_edges) atomicAdd(&st->front_edges[level + 1], new_edges);
    if (gtid() == 0) atomicAdd(&st->bfs_inspected, (unsigned long long)total);
}

__global__ void __launch_bounds__(kBlock) k_bfsg_bottomup(vid_t n, const uint32_t *__restrict__ row_ptr,
                                                          const vid_t *__restrict__ col, uint32_t *b0, uint32_t *b1,
                                                          uint32_t *vis, DevState *st) {
    if (!st->bfs_bu) return;
    const int level = st->bfs_level, par = st->bfs_par;
    const uint32_t *fb = par ? b1 : b0;
    uint32_t *nb = par ? b0 : b1;
    const long long nwords = ((long long)n + 31) / 32;
    const int lane = threadIdx.x & 31;
    const long long warp0 = gtid() >> 5, nwarps = gstride() >> 5;
    unsigned long long inspected = 0, new_edges = 0, found_total = 0;
    for (long long w = warp0; w < nwords; w += nwarps) {
        const uint32_t vword = vis[w];
        const long long v = w * 32 + lane;
        bool found = false;
        uint32_t d = 0;
        if (v < (long long)n && !((vword >> lane) & 1u)) {
            const uint32_t b = row_ptr[v], e = row_ptr[v + 1];
            d = e - b;
            for (uint32_t k = b; k < e; k++) {
                const vid_t x = col[k];
                inspected++;
                if ((fb[x >> 5] >> (x & 31)) & 1u) {
                    found = true;
                    break;
                }
            }
        }
        const uint32_t fmask = __ballot_sync(0xffffffffu, found);
        if (found) new_edges += d;
        if (lane == 0) {
            nb[w] = fmask;
            if (fmask) vis[w] = vword | fmask;
            found_total += __popc(fmask);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        inspected += __shfl_xor_sync(0xffffffffu, inspected, o);
        new_edges += __shfl_xor_sync(0xffffffffu, new_edges, o);
    }
    if (lane == 0) {
        if (found_total) atomicAdd(&st->front[level + 1], found_total);
        if (new_edges) atomicAdd(&st->front_edges[level + 1], new_edges);
        if (inspected) atomicAdd(&st->bfs_inspected, inspected);
    }
}

__global__ void k_bfsg_step(DevState *st, cudaGraphConditionalHandle h) {
    int l = st->bfs_level;
    st->bfs_explored += st->front_edges[l];
    st->bfs_prev_f = st->front[l];
    st->bfs_queue = st->bfs_bu ? 0 : 1;
    st->bfs_par ^= 1;
    l++;
    st->bfs_level = l;
    cudaGraphSetConditional(h, bfs_continue(st, l, st->front[l]) ? 1u : 0u);
}

void launch_bfsg_init(const uint32_t *row_ptr, vid_t n, uint32_t *vis, vid_t *q0, DevState *st,
                      cudaGraphConditionalHandle h, cudaStream_t s) {
    k_bfsg_init<<<1, 1, 0, s>>>(row_ptr, n, vis, q0, st, h);
}

int launch_bfsg_level(vid_t n, unsigned long long total_edges, const uint32_t *row_ptr, const vid_t *col, uint32_t *vis,
                      vid_t *q0, vid_t *q1, uint32_t *b0, uint32_t *b1, uint32_t *dq, uint32_t *off,
                      unsigned long long *tsum, DevState *st, cudaGraphConditionalHandle h, int grid, cudaStream_t s) {
    const long long nwords = ((long long)n + 31) / 32;
    k_bfsg_plan<<<1, 1, 0, s>>>(st, n, total_edges);
    k_bfsg_q2b_clear<<<grid, kBlock, 0, s>>>(b0, b1, nwords, st);
    k_bfsg_q2b<<<grid, kBlock, 0, s>>>(q0, q1, b0, b1, st);
    k_bfsg_b2q<<<grid, kBlock, 0, s>>>(b0, b1, nwords, q0, q1, st);
    k_bfsg_front_degrees<<<grid, kBlock, 0, s>>>(q0, q1, row_ptr, dq, st);
    k_bfsg_scan_up<<<grid, kBlock, 0, s>>>(dq, tsum, st);
    k_bfsg_scan_mid<<<1, kBlock, 0, s>>>(tsum, st);
    k_bfsg_scan_down<<<grid, kBlock, 0, s>>>(dq, tsum, off, st);
    k_bfsg_topdown<<<grid, kBlock, 0, s>>>(q0, q1, off, row_ptr, col, vis, q0, q1, st);
    k_bfsg_bottomup<<<grid, kBlock, 0, s>>>(n, row_ptr, col, b0, b1, vis, st);
    k_bfsg_step<<<1, 1, 0, s>>>(st, h);
    return 11;
}

// Device-driven edge-list BFS (one WHILE iteration per level). The active
// pairs are the caller's list (bfs_list < 0, read by the T instantiation)
// or ebuf[bfs_list] (the uint32 instantiation); a level compacts them into
// the other buffer once they fall to 70% of the list, as the host loop does.
// Seed: the sampled hub of the learned predictor when it decided the route,
// else the exact max-degree vertex.
__global__ void k_ebfsg_init(uint32_t *vis, uint32_t *b0, vid_t n, long long m, DevState *st,
                             cudaGraphConditionalHandle h) {
    const unsigned long long key = st->route_source == 1 ? st->pred_seedkey : st->maxkey;
    vid_t s = 0xffffffffu - (vid_t)(key & 0xffffffffull);
    if (s >= n) s = 0;
    vis[s >> 5] |= 1u << (s & 31);
    b0[s >> 5] |= 1u << (s & 31);
    st->front[0] = 1;
    st->cmin = 0xffffffffu;
    st->bfs_level = 0;
    st->bfs_par = 0;
    st->bfs_list = -1;
    st->bfs_len = (unsigned long long)m;
    st->bfs_kept_prev = (unsigned long long)m;
    cudaGraphSetConditional(h, 1u);  // level 0 always runs (a cutoff is at least one level)
}

// this level: compact or not; the next frontier bitmap cleared
__global__ void __launch_bounds__(kBlock) k_ebfsg_plan(uint32_t *b0, uint32_t *b1, long long nwords, DevState *st) {
    const int l = st->bfs_level;
    if (gtid() == 0) st->bfs_write = l >= 1 && (double)st->bfs_kept_prev <= 0.7 * (double)st->bfs_len;
    uint32_t *next = st->bfs_par ? b0 : b1;
    for (long long w = gtid(); w < nwords; w += gstride()) next[w] = 0u;
}

// OWN: the multi-start form. own[v] is the tree (start number) that claimed
// v, kNoOwner before; a vertex claimed from u takes own[u]. A pair leaves
// the active list only when its ends are known to be in one tree: the pair
// that claimed one end from the other, or ends whose owners are both
// written and equal. Owners are written once, so a value read is final and
// an end claimed by another pair in this level is at worst read as
// kNoOwner, which keeps the pair for a later level or for SV (where equal
// roots drop it).
template <typename T, bool OWN>
__global__ void __launch_bounds__(kBlock) k_ebfsg_level(const T *__restrict__ caller, long long m, const uint2 *eb0,
                                                        const uint2 *eb1, vid_t n, uint32_t *vis, uint32_t *b0,
                                                        uint32_t *b1, DevState *st, uint32_t *own) {
    constexpr bool kList = sizeof(T) == 4 && T(-1) > T(0);  // uint32_t: the compacted list
    const int list = st->bfs_list;
    if (kList != (list >= 0)) return;
    const T *in = kList ? reinterpret_cast<const T *>(list ? eb1 : eb0) : caller;
    const long long len = kList ? (long long)st->bfs_len : m;
    uint2 *out = const_cast<uint2 *>(list == 0 ? eb1 : eb0);
    const int level = st->bfs_level, par = st->bfs_par;
    const bool write = st->bfs_write != 0;
    const uint32_t *cur = par ? b1 : b0;
    uint32_t *next = par ? b0 : b1;
    constexpr int P = PairVec<T>::kPairs;
    constexpr int U = EdgeUnroll<T>::U;
    constexpr int K = P * U;
    __shared__ int sw[32];
    __shared__ unsigned long long sbase;
    const long long nvec = len / P;
    const int4 *ev = reinterpret_cast<const int4 *>(in);
    const long long tile = (long long)kBlock * U;
    const long long ntiles = (nvec + tile - 1) / tile;
    unsigned long long claimed = 0, kept_total = 0;
    for (long long t = blockIdx.x; t < ntiles + (P == 2 && (len & 1) ? 1 : 0); t += gridDim.x) {
        long long u[K], v[K];
        bool valid[K];
        if (t < ntiles) {
            int4 q[U];
#pragma unroll
            for (int k = 0; k < U; k++) {
                const long long i = t * tile + (long long)k * kBlock + threadIdx.x;
                q[k] = i < nvec ? ld_stream(ev + i) : make_int4(0, 0, 0, 0);
            }
#pragma unroll
            for (int k = 0; k < U; k++) {
                const long long i = t * tile + (long long)k * kBlock + threadIdx.x;
#pragma unroll
                for (int j = 0; j < P; j++) {
                    vec_pair<T>(q[k], j, u[k * P + j], v[k * P + j]);
                    valid[k * P + j] = i < nvec;
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; k++) {
                u[k] = v[k] = 0;
                valid[k] = false;
            }
            if (threadIdx.x == 0) {
                scalar_pair<T>(in, len - 1, u[0], v[0]);
                valid[0] = true;
            }
        }
        bool keep[K];
#pragma unroll
        for (int k = 0; k < K; k++) {
            keep[k] = false;
            if (!valid[k] || (unsigned long long)u[k] >= n || (unsigned long long)v[k] >= n) continue;
            const bool fu = bit_test(cur, u[k]), fv = bit_test(cur, v[k]);
            const bool vu0 = fu || bit_test(vis, u[k]), vv0 = fv || bit_test(vis, v[k]);
            if (OWN) {
                bool joined = false;
                if (fu && !vv0 && claim(vis, next, v[k])) {
                    own[v[k]] = __ldcg(&own[u[k]]);
                    claimed++;
                    joined = true;
                }
                if (fv && !vu0 && claim(vis, next, u[k])) {
                    own[u[k]] = __ldcg(&own[v[k]]);
                    claimed++;
                    joined = true;
                }
                if (joined) keep[k] = false;
                else if (vu0 && vv0) {
                    const uint32_t ou = __ldcg(&own[u[k]]), ov = __ldcg(&own[v[k]]);
                    keep[k] = !(ou != kNoOwner && ou == ov);
                } else
                    keep[k] = true;
            } else {
                if (fu && !vv0 && claim(vis, next, v[k])) claimed++;
                if (fv && !vu0 && claim(vis, next, u[k])) claimed++;
                keep[k] = !((vu0 || fv) && (vv0 || fu));
            }
        }
        int c = 0;
#pragma unroll
        for (int k = 0; k < K; k++) c += keep[k];
        kept_total += (unsigned long long)c;
        if (write) {  // uniform over the grid
            unsigned long long o = block_reserve(&st->front_edges[level + 1], c, sw, &sbase);
#pragma unroll
            for (int k = 0; k < K; k++)
                if (keep[k]) out[o++] = make_uint2((vid_t)u[k], (vid_t)v[k]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        claimed += __shfl_xor_sync(0xffffffffu, claimed, o);
        kept_total += __shfl_xor_sync(0xffffffffu, kept_total, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (claimed) atomicAdd(&st->front[level + 1], claimed);
        if (!write && kept_total) atomicAdd(&st->front_edges[level + 1], kept_total);
    }
}

__global__ void k_ebfsg_step(DevState *st, cudaGraphConditionalHandle h, int has_h) {
    int l = st->bfs_level;
    st->bfs_inspected += 2ull * st->bfs_len;  // the level read both ends of every active pair
    const unsigned long long claimed = st->front[l + 1], kept = st->front_edges[l + 1];
    if (st->bfs_write) {
        st->bfs_list = st->bfs_list == 0 ? 1 : 0;
        st->bfs_len = kept;
    }
    st->bfs_kept_prev = kept;
    st->bfs_par ^= 1;
    l++;
    st->bfs_level = l;
    const bool go = claimed > 0 && l < kMaxLevels - 1 && (st->bfs_cutoff <= 0 || l < st->bfs_cutoff);
    if (has_h) cudaGraphSetConditional(h, go ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Multi-start BFS (the BFS step of Section 3.2 run as several traversals at
// once): the id range [0, n) is cut into k ranges [j n / k, (j + 1) n / k),
// and the vertex of largest degree of range j (ties to the smallest id)
// starts tree j unless that degree is 0. One block per range.
__global__ void __launch_bounds__(kBlock) k_mbfs_starts(const uint32_t *__restrict__ deg, vid_t n, int k,
                                                        uint32_t *vis, uint32_t *b0, uint32_t *own, DevState *st) {
    __shared__ unsigned long long sbest[kBlock / 32];
    const int j = blockIdx.x;
    const long long lo = (long long)n * j / k, hi = (long long)n * (j + 1) / k;
    unsigned long long best = 0;  // (degree << 32) | (0xffffffff - v): the larger key wins
    for (long long v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        const unsigned long long key = ((unsigned long long)deg[v] << 32) | (0xffffffffull - (unsigned long long)v);
        best = key > best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, best, o);
        best = x > best ? x : best;
    }
    if ((threadIdx.x & 31) == 0) sbest[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kBlock / 32; w++) best = sbest[w] > best ? sbest[w] : best;
        if ((best >> 32) > 0) {
            const vid_t v = (vid_t)(0xffffffffull - (best & 0xffffffffull));
            atomicOr(&vis[v >> 5], 1u << (v & 31));
            atomicOr(&b0[v >> 5], 1u << (v & 31));
            own[v] = (uint32_t)j;
            atomicAdd(&st->front[0], 1ull);
            atomicAdd(&st->bfs_starts, 1);
        }
    }
}

// the BFS state once the starts are seeded; level 0 runs if there is a start
__global__ void k_mbfsg_init(long long m, DevState *st, cudaGraphConditionalHandle h, int has_h) {
    st->cmin = 0xffffffffu;
    st->bfs_level = 0;
    st->bfs_par = 0;
    st->bfs_list = -1;
    st->bfs_len = (unsigned long long)m;
    st->bfs_kept_prev = (unsigned long long)m;
    if (has_h) cudaGraphSetConditional(h, st->front[0] > 0 ? 1u : 0u);
}

// tmin[j] = the smallest vertex of tree j: the lanes of a warp with the same
// owner reduce their ids first, so a large tree costs one atomic per warp
__global__ void __launch_bounds__(kBlock) k_mbfs_tree_min(const uint32_t *__restrict__ own, vid_t n,
                                                          uint32_t *tmin) {
    const int lane = threadIdx.x & 31;
    for (long long base = gtid() - lane; base < (long long)n; base += gstride()) {
        const long long v = base + lane;
        const uint32_t o = v < (long long)n ? own[v] : kNoOwner;
        const unsigned act = __ballot_sync(0xffffffffu, o != kNoOwner);
        if (o != kNoOwner) {
            const unsigned grp = __match_any_sync(act, o);
            const unsigned mn = __reduce_min_sync(grp, (unsigned)v);
            if (lane == __ffs(grp) - 1) atomicMin(&tmin[o], mn);
        }
    }
}

// every vertex a tree reached takes the tree's smallest vertex as parent (a
// root: it is in the tree, so its own parent is itself); the rest are roots
__global__ void __launch_bounds__(kBlock) k_mbfs_parents(const uint32_t *__restrict__ own,
                                                         const uint32_t *__restrict__ tmin, vid_t n, vid_t *parent) {
    for (long long v = gtid(); v < (long long)n; v += gstride()) {
        const uint32_t o = own[v];
        parent[v] = o == kNoOwner ? (vid_t)v : tmin[o];
    }
}

void launch_mbfs_start(const uint32_t *deg, vid_t n, long long m, int k, uint32_t *vis, uint32_t *b0, uint32_t *own,
                       uint32_t *tmin, DevState *st, const cudaGraphConditionalHandle *h, cudaStream_t s) {
    const long long nwords = ((long long)n + 31) / 32;
    cudaMemsetAsync(vis, 0, (size_t)nwords * 4, s);
    cudaMemsetAsync(b0, 0, (size_t)nwords * 4, s);
    cudaMemsetAsync(own, 0xff, (size_t)n * 4, s);
    cudaMemsetAsync(tmin, 0xff, (size_t)k * 4, s);
    cudaMemsetAsync(&st->front[0], 0, sizeof(st->front) + sizeof(st->front_edges), s);
    cudaMemsetAsync(&st->bfs_starts, 0, sizeof(st->bfs_starts), s);
    k_mbfs_starts<<<k, kBlock, 0, s>>>(deg, n, k, vis, b0, own, st);
    k_mbfsg_init<<<1, 1, 0, s>>>(m, st, h ? *h : cudaGraphConditionalHandle(), h ? 1 : 0);
}

void launch_mbfs_finish(const uint32_t *own, uint32_t *tmin, vid_t n, vid_t *parent, int grid, cudaStream_t s) {
    k_mbfs_tree_min<<<grid, kBlock, 0, s>>>(own, n, tmin);
    k_mbfs_parents<<<grid, kBlock, 0, s>>>(own, tmin, n, parent);
}

void launch_ebfsg_init(uint32_t *vis, uint32_t *b0, vid_t n, long long m, DevState *st, cudaGraphConditionalHandle h,
                       cudaStream_t s) {
    k_ebfsg_init<<<1, 1, 0, s>>>(vis, b0, n, m, st, h);
}

template <typename T, bool OWN>
void launch_ebfsg_level_k(const void *caller, long long m, const uint2 *eb0, const uint2 *eb1, vid_t n, uint32_t *vis,
                          uint32_t *b0, uint32_t *b1, DevState *st, int grid, cudaStream_t s, uint32_t *own) {
    auto kc = k_ebfsg_level<T, OWN>;
    auto kl = k_ebfsg_level<uint32_t, OWN>;
    kc<<<fit_grid((const void *)kc, grid, kBlock), kBlock, 0, s>>>((const T *)caller, m, eb0, eb1, n, vis, b0, b1, st,
                                                                     own);
    kl<<<fit_grid((const void *)kl, grid, kBlock), kBlock, 0, s>>>(nullptr, 0, eb0, eb1, n, vis, b0, b1, st, own);
}

template <typename T>
int launch_ebfsg_level(const void *caller, long long m, const uint2 *eb0, const uint2 *eb1, vid_t n, uint32_t *vis,
                       uint32_t *b0, uint32_t *b1, DevState *st, cudaGraphConditionalHandle h, int grid,
                       cudaStream_t s, uint32_t *own, bool has_h) {
    const long long nwords = ((long long)n + 31) / 32;
    k_ebfsg_plan<<<grid, kBlock, 0, s>>>(b0, b1, nwords, st);
    if (own) launch_ebfsg_level_k<T, true>(caller, m, eb0, eb1, n, vis, b0, b1, st, grid, s, own);
    else launch_ebfsg_level_k<T, false>(caller, m, eb0, eb1, n, vis, b0, b1, st, grid, s, nullptr);
    k_ebfsg_step<<<1, 1, 0, s>>>(st, h, has_h ? 1 : 0);
    return 4;
}
template int launch_ebfsg_level<int32_t>(const void *, long long, const uint2 *, const uint2 *, vid_t, uint32_t *,
                                         uint32_t *, uint32_t *, DevState *, cudaGraphConditionalHandle, int,
                                         cudaStream_t, uint32_t *, bool);
template int launch_ebfsg_level<int64_t>(const void *, long long, const uint2 *, const uint2 *, vid_t, uint32_t *,
                                         uint32_t *, uint32_t *, DevState *, cudaGraphConditionalHandle, int,
                                         cudaStream_t, uint32_t *, bool);

}  // namespace ccg

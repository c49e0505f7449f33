// Vertex-block partitioned CSR build for the BFS step (every pair stored in
// both directions, Section 3.2).
//
// Placing 2m entries at random per-vertex cursors with global atomics
// scatters 4-byte writes over the whole column array. Instead the directed
// entries x -> y are first partitioned by x's vertex block (2^kBucketBits
// vertices), straight into that block's own CSR range, and then placed in
// the order of that array: blocks take tiles of it in increasing order, so
// the entries in flight span one or two vertex blocks, and their cursors
// (the per-vertex fill positions, 128 KB per vertex block) and the column
// range they write (a few MB) stay in L2 until every sector is written.
// Lanes of a warp that hit the same vertex take their slots with one atomic
// (__match_any_sync), which keeps hubs off a single L2 address.
//
//  k_csr_partition  per tile of pairs: both directed entries of every pair
//                   counted per vertex block in shared memory, staged in
//                   block order, one reservation per vertex block in that
//                   block's CSR range (row_ptr of its first vertex plus a
//                   fill counter), and written as contiguous runs; the order
//                   within a vertex block is whatever the reservations give
//  k_csr_place      in tile order: col[cursor[x]++] = y
#include "cc_common.cuh"
#include "cc_kernels.h"

namespace ccg {

constexpr int kBucketBits = 15;  // 32768 vertices per block: 128 KB of uint32 counters
constexpr int kBucketSize = 1 << kBucketBits;
constexpr int kMaxBuckets = 1024;  // n <= 2^25 takes this path
constexpr int kPartThreads = 512;
constexpr int kPartPairs = 8;  // pairs per thread per tile (two blocks per SM: Chung-Lu 2^24 CSR 4.71 ms, 4.82 with 16 and one)
constexpr int kPartTile = kPartThreads * kPartPairs * 2;  // directed entries per tile (8,192)

struct CsrPartShared {
    unsigned long long stage[kPartTile];  // the tile's entries in vertex-block order (64 KB)
    uint16_t key[kPartTile];              // the vertex block of each staged entry
    uint32_t hist[kMaxBuckets];
    uint32_t loff[kMaxBuckets + 1];
    unsigned long long base[kMaxBuckets];
    uint32_t wsum[kPartThreads / 32];
};
constexpr int kPartWpt = kMaxBuckets / kPartThreads;  // vertex blocks per thread in the scan
constexpr size_t kCsrPartSmem = sizeof(CsrPartShared);

template <typename T>
__global__ void __launch_bounds__(kPartThreads, 2) k_csr_partition(const T *__restrict__ edges, long long m, vid_t n,
                                                                   int nb, const uint32_t *__restrict__ row_ptr,
                                                                   unsigned long long *fill,
                                                                   unsigned long long *out, DevState *st) {
    extern __shared__ uint4 csr_part_smem[];
    CsrPartShared &S = *reinterpret_cast<CsrPartShared *>(csr_part_smem);
    constexpr int P = PairVec<T>::kPairs;
    constexpr int V = kPartPairs / P;  // 16-byte vectors per thread per tile
    const long long nvec = m / P;
    const long long tvec = (long long)kPartThreads * V;
    const long long ntiles = (nvec + tvec - 1) / tvec;
    const int4 *ev = reinterpret_cast<const int4 *>(edges);
    bool bad = false;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (int i = threadIdx.x; i < nb; i += kPartThreads) S.hist[i] = 0;
        __syncthreads();
        // the thread's pairs (ids below n <= 2^25; an invalid pair is marked by pu = ~0)
        // and the ranks of both directed entries within their vertex blocks (16 bits each)
        uint32_t pu[kPartPairs], pv[kPartPairs], rank[kPartPairs];
#pragma unroll
        for (int k = 0; k < V; k++) {
            const long long i = t * tvec + (long long)k * kPartThreads + threadIdx.x;
            const int4 q = i < nvec ? ld_stream(ev + i) : make_int4(0, 0, 0, 0);
#pragma unroll
            for (int j = 0; j < P; j++) {
                const int e = k * P + j;
                long long u, v;
                vec_pair<T>(q, j, u, v);
                const bool ok = i < nvec && (unsigned long long)u < n && (unsigned long long)v < n;
                bad |= i < nvec && !ok;
                pu[e] = ok ? (uint32_t)u : ~0u;
                pv[e] = (uint32_t)v;
            }
        }
#pragma unroll
        for (int e = 0; e < kPartPairs; e++)
            rank[e] = pu[e] != ~0u ? atomicAdd(&S.hist[pu[e] >> kBucketBits], 1u) |
                                         (atomicAdd(&S.hist[pv[e] >> kBucketBits], 1u) << 16)
                                   : 0u;
        __syncthreads();
        {  // block-wide exclusive scan of the nb counts (thread t: blocks t * kPartWpt and on),
           // one reservation per vertex block
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            constexpr int NW = kPartThreads / 32;
            uint32_t h[kPartWpt], hs = 0u;
#pragma unroll
            for (int q = 0; q < kPartWpt; q++) {
                const int b = threadIdx.x * kPartWpt + q;
                h[q] = b < nb ? S.hist[b] : 0u;
                hs += h[q];
                if (h[q])
                    S.base[b] = (unsigned long long)row_ptr[(long long)b << kBucketBits] +
                                atomicAdd(&fill[b], (unsigned long long)h[q]);
            }
            uint32_t incl = hs;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t w = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += w;
            }
            if (lane == 31) S.wsum[warp] = incl;
            __syncthreads();
            const uint32_t w = lane < NW ? S.wsum[lane] : 0u;
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < NW; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            uint32_t lo = __shfl_sync(0xffffffffu, wi - w, warp) + incl - hs;
#pragma unroll
            for (int q = 0; q < kPartWpt; q++) {
                const int b = threadIdx.x * kPartWpt + q;
                if (b < nb) S.loff[b] = lo;
                lo += h[q];
            }
            const uint32_t tot = __shfl_sync(0xffffffffu, wi, NW - 1);
            if (threadIdx.x == 0) S.loff[nb] = tot;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < kPartPairs; e++)
            if (pu[e] != ~0u) {
                const uint32_t bu = pu[e] >> kBucketBits, bv = pv[e] >> kBucketBits;
                const uint32_t iu = S.loff[bu] + (rank[e] & 0xffffu), iv = S.loff[bv] + (rank[e] >> 16);
                S.stage[iu] = ((unsigned long long)pu[e] << 32) | pv[e];
                S.key[iu] = (uint16_t)bu;
                S.stage[iv] = ((unsigned long long)pv[e] << 32) | pu[e];
                S.key[iv] = (uint16_t)bv;
            }
        __syncthreads();
        const uint32_t total = S.loff[nb];
        for (uint32_t i = threadIdx.x; i < total; i += kPartThreads) {
            const uint32_t b = S.key[i];
            out[S.base[b] + (i - S.loff[b])] = S.stage[i];
        }
        __syncthreads();
    }
    if (P == 2 && (m & 1) && blockIdx.x == 0 && threadIdx.x == 0) {  // the odd last pair
        long long u, v;
        scalar_pair<T>(edges, m - 1, u, v);
        if ((unsigned long long)u < n && (unsigned long long)v < n) {
            const unsigned long long xs[2] = {(unsigned long long)u, (unsigned long long)v};
            for (int d = 0; d < 2; d++) {
                const uint32_t b = (uint32_t)(xs[d] >> kBucketBits);
                const unsigned long long at = (unsigned long long)row_ptr[(long long)b << kBucketBits] +
                                              atomicAdd(&fill[b], 1ull);
                out[at] = (xs[d] << 32) | xs[1 - d];
            }
        } else {
            bad = true;
        }
    }
    if (bad) set_err(st, kErrInvalidEdge);
}

// col[cursor[x]++] = y for every entry, in the order of the partitioned
// array: tiles of kPlaceTile entries taken from `next` (a zeroed counter) in
// increasing order, the next tile fetched while the current one is placed.
// The entries of a tile that fall in the vertex block of its first entry
// (all but the few tiles that straddle two blocks) are counted per vertex in
// shared memory (a dense array over the block's 2^15 vertices): each entry
// gets its rank among the tile's entries of its vertex, the first entry of
// each vertex appends the vertex to a list, and one global atomic per
// listed vertex reserves its slots. Measured on R-MAT scale 22, a tile of
// 8,192 entries holds 0.31 distinct vertices per entry (a warp of 32: 0.94),
// Chung-Lu 0.7 (0.98). The other entries take their slots with one atomic
// per vertex and warp (__match_any_sync).
constexpr int kPlaceThreads = 1024;
constexpr int kPlaceVec = 8;  // entries per thread per tile
constexpr long long kPlaceTile = (long long)kPlaceThreads * kPlaceVec;
// per vertex of the tile's block: the count, then the reserved base; the list of the tile's vertices
constexpr size_t kPlaceSmem = (size_t)kBucketSize * sizeof(uint32_t) + (size_t)kPlaceTile * sizeof(uint32_t);

__global__ void __launch_bounds__(kPlaceThreads, 1) k_csr_place(const unsigned long long *__restrict__ entries,
                                                                unsigned long long total, uint32_t *cursor,
                                                                vid_t *col, unsigned long long *next) {
    extern __shared__ uint32_t place_smem[];
    uint32_t *cnt = place_smem, *touched = place_smem + kBucketSize;
    __shared__ unsigned long long s_t[2];
    __shared__ uint32_t s_blk[2];
    __shared__ uint32_t s_nt;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned long long ntiles = (total + kPlaceTile - 1) / kPlaceTile;
    for (int i = threadIdx.x; i < kBucketSize; i += kPlaceThreads) cnt[i] = 0u;
    if (threadIdx.x == 0) s_nt = 0u;
    auto fetch = [&](int b) {  // thread 0: the tile and its first entry's vertex block
        const unsigned long long t = atomicAdd(next, 1ull);
        s_t[b] = t;
        if (t < ntiles) s_blk[b] = (uint32_t)(entries[t * kPlaceTile] >> 32) >> kBucketBits;
    };
    if (threadIdx.x == 0) fetch(0);
    __syncthreads();
    for (int b = 0;; b ^= 1) {
        const unsigned long long t = s_t[b];
        if (t >= ntiles) break;
        const uint32_t blk = s_blk[b], v0 = blk << kBucketBits;
        unsigned long long ent[kPlaceVec];
        uint32_t rank[kPlaceVec];
#pragma unroll
        for (int r = 0; r < kPlaceVec; r++) {
            const unsigned long long i = t * kPlaceTile + (unsigned long long)r * kPlaceThreads + threadIdx.x;
            ent[r] = i < total ? __ldcs(entries + i) : ~0ull;
        }
        if (threadIdx.x == 0) fetch(b ^ 1);
        // entries of the tile's block: ranks among the tile's entries of their vertex; the
        // first entry of each vertex lists it (one list append per warp)
#pragma unroll
        for (int r = 0; r < kPlaceVec; r++) {
            const uint32_t x = (uint32_t)(ent[r] >> 32);
            const bool mine = ent[r] != ~0ull && (x >> kBucketBits) == blk;
            rank[r] = mine ? atomicAdd(&cnt[x - v0], 1u) : 1u;
            const unsigned first = __ballot_sync(0xffffffffu, rank[r] == 0u);
            if (first) {
                uint32_t at = 0;
                if (lane == 0) at = atomicAdd(&s_nt, (uint32_t)__popc(first));
                at = __shfl_sync(0xffffffffu, at, 0);
                if (rank[r] == 0u) touched[at + __popc(first & lt)] = x - v0;
            }
        }
        // the other entries (a tile that straddles two blocks): one atomic per vertex and warp
#pragma unroll
        for (int r = 0; r < kPlaceVec; r++) {
            const uint32_t x = (uint32_t)(ent[r] >> 32);
            const bool other = ent[r] != ~0ull && (x >> kBucketBits) != blk;
            if (!__any_sync(0xffffffffu, other)) continue;
            const unsigned peers = __match_any_sync(0xffffffffu, other ? x : 0xffffffffu);
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (other && lane == leader) base = atomicAdd(&cursor[x], (uint32_t)__popc(peers));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (other) col[base + __popc(peers & lt)] = (vid_t)(ent[r] & 0xffffffffull);
        }
        __syncthreads();
        // one reservation per listed vertex; its count becomes its base
        const uint32_t nt = s_nt;
        for (uint32_t i = threadIdx.x; i < nt; i += kPlaceThreads) {
            const uint32_t lx = touched[i];
            cnt[lx] = atomicAdd(&cursor[v0 + lx], cnt[lx]);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kPlaceVec; r++) {
            const uint32_t x = (uint32_t)(ent[r] >> 32);
            if (ent[r] != ~0ull && (x >> kBucketBits) == blk)
                col[cnt[x - v0] + rank[r]] = (vid_t)(ent[r] & 0xffffffffull);
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < nt; i += kPlaceThreads) cnt[touched[i]] = 0u;
        if (threadIdx.x == 0) s_nt = 0u;
        __syncthreads();  // the reset before the next tile's counts
    }
}

// ---------------------------------------------------------------------------
int bucket_count_for(vid_t n) { return (int)(((long long)n + kBucketSize - 1) >> kBucketBits); }
int bucket_max() { return kMaxBuckets; }

template <typename T>
void launch_csr_bucketed(const void *edges, long long m, vid_t n, const uint32_t *row_ptr, uint32_t *cursor,
                         vid_t *col, BucketScratch bs, unsigned long long *entries, DevState *st, int grid,
                         cudaStream_t s) {
    const int nb = bucket_count_for(n);
    cudaMemsetAsync(bs.fill, 0, (size_t)nb * sizeof(unsigned long long), s);
    cudaMemsetAsync(bs.queue, 0, sizeof(unsigned long long), s);
    auto kp = k_csr_partition<T>;
    kp<<<fit_grid((const void *)kp, grid, kPartThreads, kCsrPartSmem), kPartThreads, kCsrPartSmem, s>>>(
        (const T *)edges, m, n, nb, row_ptr, bs.fill, entries, st);
    k_csr_place<<<fit_grid((const void *)k_csr_place, grid, kPlaceThreads, kPlaceSmem), kPlaceThreads, kPlaceSmem,
                  s>>>(entries, 2ull * (unsigned long long)m, cursor, col, bs.queue);
}
template void launch_csr_bucketed<int32_t>(const void *, long long, vid_t, const uint32_t *, uint32_t *, vid_t *,
                                           BucketScratch, unsigned long long *, DevState *, int, cudaStream_t);
template void launch_csr_bucketed<int64_t>(const void *, long long, vid_t, const uint32_t *, uint32_t *, vid_t *,
                                           BucketScratch, unsigned long long *, DevState *, int, cudaStream_t);

cudaError_t csr_kernels_setup() {
    cudaError_t e = cudaFuncSetAttribute(k_csr_partition<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kCsrPartSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_csr_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPlaceSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_csr_partition<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kCsrPartSmem);
}

}  // namespace ccg

// Vertex-block partitioned CSR build for the BFS step (every pair stored in
// both directions, Section 3.2).
//
// Placing 2m entries at random per-vertex cursors with global atomics
// saturates the L2 (and piles up on the slices that hold hub vertices) and
// scatters 4-byte writes over the whole column array. Instead the directed
// entries x -> y are first partitioned by x's vertex block (2^kBucketBits
// vertices), straight into that block's own CSR range, and then one CTA per
// vertex block places its entries with shared-memory cursors, its writes
// confined to a few MB that stay in L2. Lanes of a warp that hit the same
// vertex are merged with __match_any_sync in oversized blocks (hubs).
//
//  k_bucket_count   counts[k][b]: entries of grid block k falling in vertex block b
//  k_bucket_offsets private write offsets per (grid block, vertex block)
//  k_bucket_scatter (local id of x) << 32 | y into the vertex block's CSR range
//  k_csr_place      one CTA per vertex block: col[cursor[x]++] = y
#include "cc_common.cuh"
#include "cc_kernels.h"

namespace ccg {

constexpr int kBucketBits = 15;  // 32768 vertices per block: 128 KB of uint32 counters
constexpr int kBucketSize = 1 << kBucketBits;
constexpr int kMaxBuckets = 1024;  // n <= 2^25 takes this path

// Both partition kernels walk the pairs in chunks of kBlock * 4 pairs; block
// k of the grid owns the contiguous chunks [k * cpb, (k+1) * cpb), the same
// in the counting and in the scattering kernel, so a count matrix
// counts[k][b] (endpoints of block k's chunks that fall in vertex block b)
// gives every block exact, private write offsets and the scatter needs no
// global atomics.
constexpr int kChunkPairsPerThread = 4;

template <typename T>
__device__ __forceinline__ long long chunk_vectors() {
    return (long long)kBlock * (kChunkPairsPerThread / PairVec<T>::kPairs);
}

// Decodes the chunk's pairs owned by this thread: up to 8 endpoints (both
// ends of 4 pairs). ok[e] marks valid ids; the odd last pair of an int32
// list is taken by thread 0 of the chunk after the last full chunk.
template <typename T>
__device__ __forceinline__ void chunk_endpoints(const T *edges, long long m, vid_t n, long long c, long long (&x)[8],
                                                long long (&y)[8], bool (&ok)[8], bool &bad) {
    constexpr int P = PairVec<T>::kPairs;
    constexpr int V = kChunkPairsPerThread / P;
    const long long nvec = m / P, cv = chunk_vectors<T>();
    const int4 *ev = reinterpret_cast<const int4 *>(edges);
#pragma unroll
    for (int e = 0; e < 8; e++) ok[e] = false;
    if (c * cv < nvec) {
#pragma unroll
        for (int k = 0; k < V; k++) {
            const long long i = c * cv + (long long)k * kBlock + threadIdx.x;
            if (i >= nvec) continue;
            const int4 q = ld_stream(ev + i);
#pragma unroll
            for (int j = 0; j < P; j++) {
                long long u, v;
                vec_pair<T>(q, j, u, v);
                const int e = (k * P + j) * 2;
                if ((unsigned long long)u < n && (unsigned long long)v < n) {
                    x[e] = u;
                    y[e] = v;
                    x[e + 1] = v;
                    y[e + 1] = u;
                    ok[e] = ok[e + 1] = true;
                } else {
                    bad = true;
                }
            }
        }
    } else if (P == 2 && (m & 1) && threadIdx.x == 0) {
        long long u, v;
        scalar_pair<T>(edges, m - 1, u, v);
        if ((unsigned long long)u < n && (unsigned long long)v < n) {
            x[0] = u;
            y[0] = v;
            x[1] = v;
            y[1] = u;
            ok[0] = ok[1] = true;
        } else {
            bad = true;
        }
    }
}

template <typename T>
__host__ __device__ __forceinline__ long long num_chunks(long long m) {
    constexpr int P = PairVec<T>::kPairs;
    const long long nvec = m / P, cv = (long long)kBlock * (kChunkPairsPerThread / P);
    return (nvec + cv - 1) / cv + (P == 2 && (m & 1) ? 1 : 0);
}

// counts[k][b] for block k's chunks (also validates the ids)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_bucket_count(const T *__restrict__ edges, long long m, vid_t n, int nb,
                                                         long long cpb, uint32_t *counts, DevState *st) {
    __shared__ uint32_t h[kMaxBuckets];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const long long nch = num_chunks<T>(m);
    bool bad = false;
    for (long long c = blockIdx.x * cpb; c < (blockIdx.x + 1) * cpb && c < nch; c++) {
        long long x[8], y[8];
        bool ok[8];
        chunk_endpoints<T>(edges, m, n, c, x, y, ok, bad);
#pragma unroll
        for (int e = 0; e < 8; e++)
            if (ok[e]) atomicAdd(&h[x[e] >> kBucketBits], 1u);
    }
    if (bad) set_err(st, kErrInvalidEdge);
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) counts[(long long)blockIdx.x * nb + i] = h[i];
}

// off[k][b] = base[b] + sum_{k' < k} counts[k'][b], one thread per vertex
// block. base = exclusive scan of the block totals (degree partition, also
// written to boff[0..nb]) or row_ptr[b << kBucketBits] (CSR partition).
__global__ void __launch_bounds__(kMaxBuckets) k_bucket_offsets(const uint32_t *counts, int grid, int nb,
                                                                const uint32_t *row_ptr, vid_t n,
                                                                unsigned long long *boff, uint32_t *off) {
    __shared__ unsigned long long tot[kMaxBuckets + 1];
    const int b = threadIdx.x;
    unsigned long long t = 0;
    if (b < nb)
        for (int k = 0; k < grid; k++) t += counts[(long long)k * nb + b];
    tot[b] = t;
    __syncthreads();
    if (b == 0) {
        unsigned long long run = 0;
        for (int i = 0; i < nb; i++) {
            const unsigned long long c = tot[i];
            tot[i] = run;
            run += c;
        }
        tot[nb] = run;
    }
    __syncthreads();
    if (b < nb) {
        unsigned long long run;
        if (row_ptr) {
            const long long v0 = (long long)b << kBucketBits;
            run = row_ptr[v0 < (long long)n ? v0 : (long long)n];
        } else {
            run = tot[b];
        }
        for (int k = 0; k < grid; k++) {
            off[(long long)k * nb + b] = (uint32_t)run;
            run += counts[(long long)k * nb + b];
        }
    }
    if (boff)
        for (int i = b; i <= nb; i += blockDim.x) boff[i] = tot[i];
}

// Shared-memory counting sort of each chunk's entries by vertex block, then
// contiguous runs at the block's private offsets. VAL = uint16_t (degree:
// the endpoint's id within its vertex block) or unsigned long long (CSR:
// (local id of x) << 32 | y).
template <typename T, typename VAL>
__global__ void __launch_bounds__(kBlock) k_bucket_scatter(const T *__restrict__ edges, long long m, vid_t n, int nb,
                                                           long long cpb, const uint32_t *off, VAL *out) {
    __shared__ uint32_t hist[kMaxBuckets], loff[kMaxBuckets + 1], cur[kMaxBuckets];
    __shared__ VAL stage[kBlock * 8];
    __shared__ uint16_t stage_key[kBlock * 8];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) cur[i] = off[(long long)blockIdx.x * nb + i];
    const long long nch = num_chunks<T>(m);
    bool bad = false;
    for (long long c = blockIdx.x * cpb; c < (blockIdx.x + 1) * cpb && c < nch; c++) {
        long long x[8], y[8];
        bool ok[8];
        chunk_endpoints<T>(edges, m, n, c, x, y, ok, bad);
        for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        uint32_t rank[8];
#pragma unroll
        for (int e = 0; e < 8; e++) rank[e] = ok[e] ? atomicAdd(&hist[x[e] >> kBucketBits], 1u) : 0u;
        __syncthreads();
        if (threadIdx.x < 32) {  // warp-parallel exclusive scan of the nb counts
            uint32_t carry = 0;
            for (int b0 = 0; b0 < nb; b0 += 32) {
                const int b = b0 + threadIdx.x;
                const uint32_t v = b < nb ? hist[b] : 0u;
                uint32_t incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t w = __shfl_up_sync(0xffffffffu, incl, o);
                    if ((int)threadIdx.x >= o) incl += w;
                }
                if (b < nb) loff[b] = carry + incl - v;
                carry += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (threadIdx.x == 0) loff[nb] = carry;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < 8; e++)
            if (ok[e]) {
                const uint32_t b = (uint32_t)(x[e] >> kBucketBits), pos = loff[b] + rank[e];
                const unsigned long long lid = (unsigned long long)(x[e] & (kBucketSize - 1));
                if (sizeof(VAL) == 2) stage[pos] = (VAL)lid;
                else stage[pos] = (VAL)((lid << 32) | (unsigned long long)y[e]);
                stage_key[pos] = (uint16_t)b;
            }
        __syncthreads();
        const uint32_t total = loff[nb];
        for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
            const uint32_t b = stage_key[i];
            out[(unsigned long long)cur[b] + (i - loff[b])] = stage[i];
        }
        __syncthreads();
        for (int b = threadIdx.x; b < nb; b += blockDim.x) cur[b] += hist[b];
        __syncthreads();
    }
}

// One CTA per vertex block: col[cursor[x]++] = y for the block's entries.
__global__ void __launch_bounds__(1024) k_csr_place(const unsigned long long *__restrict__ entries,
                                                    const uint32_t *__restrict__ row_ptr, vid_t n, int nb, vid_t *col) {
    extern __shared__ uint32_t cur[];  // kBucketSize cursors
    const int b = blockIdx.x;
    const long long v0 = (long long)b << kBucketBits;
    const long long v1 = v0 + kBucketSize < (long long)n ? v0 + kBucketSize : (long long)n;
    for (long long i = threadIdx.x; i < kBucketSize; i += blockDim.x) cur[i] = v0 + i < v1 ? row_ptr[v0 + i] : 0u;
    __syncthreads();
    const unsigned long long e0 = row_ptr[v0], e1 = row_ptr[v1];
    const bool hot = (e1 - e0) > 2 * ((unsigned long long)row_ptr[n] / (unsigned long long)nb) + 4096;
    const unsigned long long rounds = (e1 - e0 + blockDim.x - 1) / blockDim.x;
    for (unsigned long long r = 0; r < rounds; r++) {
        const unsigned long long i = e0 + r * blockDim.x + threadIdx.x;
        const bool ok = i < e1;
        const unsigned long long ent = ok ? entries[i] : ~0ull;
        const uint32_t x = (uint32_t)(ent >> 32);
        if (hot) {
            const unsigned peers = __match_any_sync(0xffffffffu, x);
            const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (ok && lane == leader) base = atomicAdd(&cur[x], (uint32_t)__popc(peers));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (ok) col[base + __popc(peers & ((1u << lane) - 1u))] = (vid_t)(ent & 0xffffffffu);
        } else if (ok) {
            col[atomicAdd(&cur[x], 1u)] = (vid_t)(ent & 0xffffffffu);
        }
    }
}

// ---------------------------------------------------------------------------
int bucket_count_for(vid_t n) { return (int)(((long long)n + kBucketSize - 1) >> kBucketBits); }
int bucket_max() { return kMaxBuckets; }

template <typename T>
static long long chunks_per_block(long long m, int grid) {
    return (num_chunks<T>(m) + grid - 1) / grid;
}

template <typename T>
void launch_csr_bucketed(const void *edges, long long m, vid_t n, const uint32_t *row_ptr, vid_t *col,
                         BucketScratch bs, unsigned long long *entries, DevState *st, int grid, cudaStream_t s) {
    const int nb = bucket_count_for(n);
    const long long cpb = chunks_per_block<T>(m, grid);
    k_bucket_count<T><<<grid, kBlock, 0, s>>>((const T *)edges, m, n, nb, cpb, bs.counts, st);
    k_bucket_offsets<<<1, kMaxBuckets, 0, s>>>(bs.counts, grid, nb, row_ptr, n, nullptr, bs.off);
    k_bucket_scatter<T, unsigned long long><<<grid, kBlock, 0, s>>>((const T *)edges, m, n, nb, cpb, bs.off, entries);
    k_csr_place<<<nb, 1024, kBucketSize * sizeof(uint32_t), s>>>(entries, row_ptr, n, nb, col);
}
template void launch_csr_bucketed<int32_t>(const void *, long long, vid_t, const uint32_t *, vid_t *, BucketScratch,
                                           unsigned long long *, DevState *, int, cudaStream_t);
template void launch_csr_bucketed<int64_t>(const void *, long long, vid_t, const uint32_t *, vid_t *, BucketScratch,
                                           unsigned long long *, DevState *, int, cudaStream_t);

cudaError_t bucket_kernels_setup() {
    return cudaFuncSetAttribute(k_csr_place, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kBucketSize * (int)sizeof(uint32_t));
}

}  // namespace ccg

// Degree pass (Section 3.2, Algorithm 2 line 1) with the endpoints moved
// into vertex windows first, in two forms: windows of 2^23 vertices counted
// with L2 atomics, for graphs whose count array does not fit in L2 (n > 2^25:
// 128 MB of counts and more); and windows of at most 2^15 vertices counted in
// shared memory, for 2^20 <= n <= 2^24 (the second half of this file).
//
// deg[v] = number of pair endpoints equal to v. With one atomic per
// endpoint, a count array out of L2 turns every endpoint into a DRAM
// read-modify-write of a 32-byte sector at a random address (measured on
// GB300: 35 G increments/s). Here the endpoints are first moved into windows
// of 2^23 vertices, so that each window's counts (32 MB) stay in L2 while
// they are incremented:
//
//  k_degree_partition  one CTA per SM streams 64 KB chunks of pairs into
//                      shared memory with 1-D bulk copies (cp.async.bulk,
//                      completion on an mbarrier, two buffers in flight).
//                      Each chunk's endpoints are counting-sorted by window
//                      in shared memory; one global atomic per window and
//                      chunk reserves the window's run, and each warp writes
//                      whole runs of the ids within the window (32-bit). A
//                      window holds at most `cap` entries; endpoints past it
//                      are counted with global atomics directly, so the
//                      counts stay exact for any input.
//  k_degree_window     one launch per window, one L2 atomic (RED) per
//                      entry: the whole grid works on one window's counts at
//                      a time. (A single grid-stride sweep over all windows
//                      in order measured 9.9 ms on the grid + chains graph
//                      with windows of 2^24: warps drift across window
//                      boundaries, and two live windows fill the L2.)
//
// HBM traffic per call: the pairs once (2wm bytes), the entries written and
// read back (2 x 8m bytes), deg zeroed and written back (8n).
//
// With `hook` (the parent array, every vertex its own root) each entry also
// carries the endpoint's partner (64-bit entries, partner << 32 | id within
// the window), and the window pass applies the first SV hook of Section 3.1
// as well: for the entry of the larger end, atomicMin(parent[hi], lo) - the
// first hook pass over all pairs, done while the window's parents are in L2.
// Out of L2 that pass costs a DRAM read-modify-write per pair (grid + chains:
// 8.1 ms for 268M int64 pairs). The entries double in size (16m bytes more
// written and read back).
#include "cc_common.cuh"
#include "cc_kernels.h"

namespace ccg {

constexpr int kPartThreads = 1024;
constexpr int kPartBits = 23;                                   // vertices per window: 2^23 (32 MB of counts)
constexpr int kPartMaxBuckets = 512;                            // n < 2^32
constexpr unsigned long long kWaitNs = 1000000000ull;           // bounded mbarrier waits: 1 s

// E: the entry type (uint32_t: the id within the window; unsigned long long:
// partner << 32 | id within the window). Chunks of 64 KB of pairs, 32 KB
// with the wider entries, so that both fit in shared memory.
template <typename E> struct PartCfg {
    static constexpr int kChunkBytes = sizeof(E) == 4 ? (1 << 16) : (1 << 15);
    static constexpr int kSlots = kChunkBytes / 16 / kPartThreads;  // 16-byte vectors per thread and chunk
    static constexpr int kMaxEnd = kChunkBytes / 8 * 2;            // endpoints of a chunk of int32 pairs
};

template <typename E>
struct __align__(128) PartShared {
    int4 buf[2][PartCfg<E>::kChunkBytes / 16];  // two chunks of pairs (bulk-copy destinations)
    E stage[PartCfg<E>::kMaxEnd];               // entries sorted by window
    uint32_t hist[kPartMaxBuckets];
    uint32_t loff[kPartMaxBuckets + 1];
    unsigned long long base[kPartMaxBuckets];
    unsigned long long mbar[2];
    uint32_t wsum[32];
    int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_tx(unsigned long long *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// 1-D bulk copy global -> shared; `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, unsigned long long *b) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_u32(b))
        : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of the barrier to complete; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, uint32_t parity) {
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try(b, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}

template <typename T, typename E>
__host__ __device__ constexpr long long part_chunk_pairs() {
    return PartCfg<E>::kChunkBytes / (2 * (long long)sizeof(T));
}

// Pair p of chunk c: from the chunk's shared-memory copy, or (the odd last
// pair of an int32 chunk, which the 16-byte bulk copy leaves out) from global memory.
template <typename T, typename E>
__device__ __forceinline__ void chunk_pair(const PartShared<E> &S, int slot, const T *edges, long long c, int sv,
                                           int j, bool in_smem, long long &u, long long &v) {
    if (in_smem) vec_pair<T>(S.buf[slot][sv], j, u, v);
    else scalar_pair<T>(edges, c * part_chunk_pairs<T, E>() + (long long)sv * PairVec<T>::kPairs + j, u, v);
}

// The entry of endpoint x with partner y; windows of 2^wb vertices.
template <typename E>
__device__ __forceinline__ E part_entry(long long x, long long y, int wb);
template <>
__device__ __forceinline__ uint32_t part_entry<uint32_t>(long long x, long long, int wb) {
    return (uint32_t)x & ((1u << wb) - 1u);
}
template <>
__device__ __forceinline__ unsigned long long part_entry<unsigned long long>(long long x, long long y, int wb) {
    return ((unsigned long long)y << 32) | ((unsigned long long)x & ((1ull << wb) - 1ull));
}

// Count (and with a partner, hook) one entry of window b directly in global memory.
template <typename E>
__device__ __forceinline__ void part_direct(E e, int b, int wb, uint32_t *deg, vid_t *parent) {
    const uint32_t x = ((uint32_t)b << wb) | ((uint32_t)e & ((1u << wb) - 1u));
    atomicAdd(&deg[x], 1u);
    if (sizeof(E) == 8) {
        const uint32_t y = (uint32_t)((unsigned long long)e >> 32);
        if (y < x) atomicMin(&parent[x], y);
    }
}

template <typename T, typename E>
__global__ void __launch_bounds__(kPartThreads, 1)
    k_degree_partition(const T *__restrict__ edges, long long m, vid_t n, int nb, int wb, unsigned long long cap,
                       unsigned long long *__restrict__ fill, E *__restrict__ part, uint32_t *deg, vid_t *parent,
                       DevState *st) {
    extern __shared__ __align__(128) unsigned char part_smem[];
    PartShared<E> &S = *reinterpret_cast<PartShared<E> *>(part_smem);
    constexpr int P = PairVec<T>::kPairs;
    constexpr int kPartSlots = PartCfg<E>::kSlots;
    constexpr long long CP = part_chunk_pairs<T, E>();
    const long long nch = (m + CP - 1) / CP;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long G = gridDim.x;
    auto chunk_len = [&](long long c) { return m - c * CP < CP ? m - c * CP : CP; };
    bool inflight[2] = {false, false};  // thread 0's view of the bulk copies it issued
    auto issue = [&](long long c, int slot) {
        const uint32_t bytes = (uint32_t)(((unsigned long long)chunk_len(c) * 2 * sizeof(T)) & ~15ull);
        if (bytes) {
            mbar_arrive_tx(&S.mbar[slot], bytes);
            bulk_load(S.buf[slot], edges + 2 * c * CP, bytes, &S.mbar[slot]);
        } else {
            mbar_arrive(&S.mbar[slot]);
        }
        inflight[slot] = true;
    };
    if (t == 0) {
        mbar_init(&S.mbar[0], 1);
        mbar_init(&S.mbar[1], 1);
        mbar_fence_init();
        S.abort = 0;
    }
    for (int i = t; i < nb; i += kPartThreads) S.hist[i] = 0;
    __syncthreads();
    if (t == 0) {
        if (blockIdx.x < nch) issue(blockIdx.x, 0);
        if (blockIdx.x + G < nch) issue(blockIdx.x + G, 1);
    }
    uint32_t phase[2] = {0u, 0u};
    bool bad = false;
    int slot = 0;
    for (long long c = blockIdx.x; c < nch; c += G, slot ^= 1) {
        if (mbar_wait(&S.mbar[slot], phase[slot])) {
            phase[slot] ^= 1u;
            if (t == 0) inflight[slot] = false;
        } else {
            S.abort = 1;
        }
        __syncthreads();
        if (S.abort) break;
        const long long np = chunk_len(c);
        const int full_vecs = (int)(((unsigned long long)np * 2 * sizeof(T)) >> 4);  // vectors the copy filled
        // ranks of this thread's endpoints within their windows (packed u | v << 16)
        uint32_t rk[kPartSlots * P];
#pragma unroll
        for (int k = 0; k < kPartSlots; k++) {
            const int sv = t + k * kPartThreads;
#pragma unroll
            for (int j = 0; j < P; j++) {
                const long long p = (long long)sv * P + j;
                uint32_t r = 0xffffffffu;
                if (p < np) {
                    long long u, v;
                    chunk_pair<T, E>(S, slot, edges, c, sv, j, sv < full_vecs, u, v);
                    if ((unsigned long long)u >= n || (unsigned long long)v >= n) {
                        bad = true;
                    } else {
                        const uint32_t ru = atomicAdd(&S.hist[u >> wb], 1u);
                        const uint32_t rv = atomicAdd(&S.hist[v >> wb], 1u);
                        r = ru | (rv << 16);
                    }
                }
                rk[k * P + j] = r;
            }
        }
        __syncthreads();
        // exclusive scan of the window counts (nb <= 512: the first 16 warps),
        // one reservation per window, counts cleared
        if (warp < kPartMaxBuckets / 32) {
            const uint32_t h = t < nb ? S.hist[t] : 0u;
            uint32_t incl = h;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) S.wsum[warp] = incl;
            S.loff[t] = incl - h;  // within the warp; the warp offsets follow
            if (t < nb) {
                S.base[t] = h ? atomicAdd(&fill[t], (unsigned long long)h) : 0ull;
                S.hist[t] = 0u;
            }
        }
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = lane < kPartMaxBuckets / 32 ? S.wsum[lane] : 0u;
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            if (lane < kPartMaxBuckets / 32) S.wsum[lane] = wi - w;
            if (lane == kPartMaxBuckets / 32 - 1) S.loff[kPartMaxBuckets] = wi;
        }
        __syncthreads();
        if (t < kPartMaxBuckets) S.loff[t] += S.wsum[warp];
        __syncthreads();
        // stage the ids within the window in window order
#pragma unroll
        for (int k = 0; k < kPartSlots; k++) {
            const int sv = t + k * kPartThreads;
#pragma unroll
            for (int j = 0; j < P; j++) {
                const uint32_t r = rk[k * P + j];
                if (r == 0xffffffffu) continue;
                long long u, v;
                chunk_pair<T, E>(S, slot, edges, c, sv, j, sv < full_vecs, u, v);
                S.stage[S.loff[u >> wb] + (r & 0xffffu)] = part_entry<E>(u, v, wb);
                S.stage[S.loff[v >> wb] + (r >> 16)] = part_entry<E>(v, u, wb);
            }
        }
        __syncthreads();
        // this buffer is read: fetch the chunk after next into it
        if (t == 0 && c + 2 * G < nch) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(c + 2 * G, slot);
        }
        // each warp writes whole runs: windows warp, warp + 32, ...
        for (int b = warp; b < nb; b += kPartThreads / 32) {
            const uint32_t r0 = S.loff[b], r1 = S.loff[b + 1];
            const unsigned long long o0 = S.base[b];
            for (uint32_t i = r0 + lane; i < r1; i += 32) {
                const unsigned long long o = o0 + (i - r0);
                const E e = S.stage[i];
                if (o < cap) part[(unsigned long long)b * cap + o] = e;
                else part_direct<E>(e, b, wb, deg, parent);
            }
        }
        __syncthreads();
    }
    if (bad) set_err(st, kErrInvalidEdge);
    if (S.abort && t == 0) {
        set_err(st, kErrTimeout);
        // leave no copy writing into shared memory after the block exits
        for (int k = 0; k < 2; k++)
            if (inflight[k]) mbar_wait(&S.mbar[k], phase[k]);
    }
}

// One RED per entry of window b (its counts stay in L2 during the launch).
__global__ void __launch_bounds__(kBlock) k_degree_window(const uint32_t *__restrict__ part, unsigned long long cap,
                                                          const unsigned long long *__restrict__ fill, int b,
                                                          uint32_t *deg) {
    const unsigned long long f = fill[b], len = f < cap ? f : cap;
    const uint4 *p4 = reinterpret_cast<const uint4 *>(part + (unsigned long long)b * cap);
    uint32_t *d = deg + ((unsigned long long)b << kPartBits);
    const unsigned long long nv = len / 4;
    for (unsigned long long k = gtid(); k < nv; k += gstride()) {
        const uint4 q = ld_stream(p4 + k);
        atomicAdd(&d[q.x], 1u);
        atomicAdd(&d[q.y], 1u);
        atomicAdd(&d[q.z], 1u);
        atomicAdd(&d[q.w], 1u);
    }
    const unsigned long long i = nv * 4 + gtid();
    if (i < len) atomicAdd(&d[part[(unsigned long long)b * cap + i]], 1u);
}

// The same with partners: one RED per entry on the counts, and for the entry
// of the larger end of a pair, a RED atomicMin on its parent (both windows
// of 32 MB stay in L2 during the launch).
__global__ void __launch_bounds__(kBlock) k_degree_window_hook(const unsigned long long *__restrict__ part,
                                                               unsigned long long cap,
                                                               const unsigned long long *__restrict__ fill, int b,
                                                               uint32_t *deg, vid_t *parent) {
    const unsigned long long f = fill[b], len = f < cap ? f : cap;
    const ulonglong2 *p2 = reinterpret_cast<const ulonglong2 *>(part + (unsigned long long)b * cap);
    uint32_t *d = deg + ((unsigned long long)b << kPartBits);
    vid_t *pa = parent + ((unsigned long long)b << kPartBits);
    const uint32_t x0 = (uint32_t)b << kPartBits;
    auto one = [&](unsigned long long e) {
        const uint32_t lx = (uint32_t)e & ((1u << kPartBits) - 1u), y = (uint32_t)(e >> 32);
        atomicAdd(&d[lx], 1u);
        if (y < x0 + lx) atomicMin(&pa[lx], y);
    };
    const unsigned long long nv = len / 2;
    for (unsigned long long k = gtid(); k < nv; k += gstride()) {
        const ulonglong2 q = __ldcs(p2 + k);
        one(q.x);
        one(q.y);
    }
    const unsigned long long i = nv * 2 + gtid();
    if (i < len) one(part[(unsigned long long)b * cap + i]);
}

// Shared-memory windows (n <= 2^24). Two launches:
//
//  k_degree_split      two CTAs of 512 threads per SM stream 32 KB chunks of
//                      pairs into shared memory (bulk copies, two in flight).
//                      Each thread keeps its chunk's endpoints in registers,
//                      takes their ranks within their windows with shared
//                      atomics, and after one scan of the window counts and
//                      one reservation per window and chunk stages the ids
//                      within the windows, with their window numbers, in
//                      window order; the block then writes the staged ids out
//                      in that order, so each window's run is one coalesced
//                      store. Four barriers per chunk, and the next copy into
//                      the buffer is issued as soon as the pairs are in
//                      registers; two CTAs per SM overlap one's reservation
//                      round trip with the other's work.
//  k_degree_window_smem one CTA per window of 2^wb vertices counts the
//                      window's ids in shared memory. A vertex that holds a
//                      large share of its window's entries (an R-MAT hub: up
//                      to 41% of one window at scale 24) would serialise the
//                      warps' shared atomics on one address, so the CTA first
//                      counts a sample of the window (its first
//                      kSmemSampleVecs * 8 entries), takes the vertex with the
//                      largest sample count as the window's hub, and then
//                      counts the hub's entries in registers (one shared
//                      atomic per warp at the end) and every other entry with
//                      a shared atomic. The counts are written to deg once,
//                      coalesced; entries of a window past its capacity were
//                      counted in deg directly by the split, so such a window
//                      adds.
//
// HBM traffic per call: the pairs once (2wm), the ids written and read back
// (2 x 4m), deg zeroed and written (8n).
constexpr int kSplitThreads = 512;
constexpr int kSplitChunk = 1 << 15;                  // bytes of pairs per chunk
constexpr int kSplitVecs = kSplitChunk / 16;          // 16-byte vectors per chunk
constexpr int kSplitSlots = kSplitVecs / kSplitThreads;
constexpr int kSplitMaxEnd = kSplitChunk / 8 * 2;     // endpoints of a chunk of int32 pairs
constexpr int kSmemThreads = 1024;
constexpr int kSmemSampleVecs = 2048;                 // 16,384 entries
constexpr int kSmemMaxBits = 15;                      // 128 KB of counts per CTA
constexpr int kSmemMinBits = 11;

constexpr int kSplitWpt = kPartMaxBuckets / kSplitThreads;  // windows per thread in the scan

// I: the type of a window's offset into the regions (uint32_t when all the
// regions hold fewer than 2^32 entries).
template <typename I>
struct __align__(128) SplitShared {
    int4 buf[2][kSplitVecs];        // two chunks of pairs (bulk-copy destinations)
    uint32_t stage[kSplitMaxEnd + kPartMaxBuckets];  // window << 16 | id within the window, in window order
                                                     // (each window's run padded to even length)
    uint32_t hist[kPartMaxBuckets];
    I goff[kPartMaxBuckets];        // the window's region + its reservation - its first stage slot
    uint32_t loff[kPartMaxBuckets]; // the window's first stage slot
    uint32_t gend[kPartMaxBuckets]; // the end of its stage slots that fit in the region
    unsigned long long mbar[2];
    uint32_t wsum[kSplitThreads / 32];
};

template <typename T, typename I>
__global__ void __launch_bounds__(kSplitThreads, 2)
    k_degree_split(const T *__restrict__ edges, long long m, vid_t n, int nb, int wb, uint32_t cap,
                   uint32_t *__restrict__ fill, uint16_t *__restrict__ part, uint32_t *deg, DevState *st) {
    extern __shared__ __align__(128) unsigned char split_smem[];
    SplitShared<I> &S = *reinterpret_cast<SplitShared<I> *>(split_smem);
    constexpr int P = PairVec<T>::kPairs;
    constexpr long long CP = kSplitChunk / (2 * (long long)sizeof(T));
    constexpr int NE = kSplitSlots * P;  // pairs per thread and chunk
    constexpr int NW = kSplitThreads / 32;
    const long long nch = (m + CP - 1) / CP;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long G = gridDim.x;
    const uint32_t low = (1u << wb) - 1u;
    auto chunk_len = [&](long long c) { return m - c * CP < CP ? m - c * CP : CP; };
    bool inflight[2] = {false, false};  // thread 0's view of the bulk copies it issued
    auto issue = [&](long long c, int slot) {
        const uint32_t bytes = (uint32_t)(((unsigned long long)chunk_len(c) * 2 * sizeof(T)) & ~15ull);
        if (bytes) {
            mbar_arrive_tx(&S.mbar[slot], bytes);
            bulk_load(S.buf[slot], edges + 2 * c * CP, bytes, &S.mbar[slot]);
        } else {
            mbar_arrive(&S.mbar[slot]);
        }
        inflight[slot] = true;
    };
    if (t == 0) {
        mbar_init(&S.mbar[0], 1);
        mbar_init(&S.mbar[1], 1);
        mbar_fence_init();
    }
    for (int i = t; i < kPartMaxBuckets; i += kSplitThreads) S.hist[i] = 0;
    __syncthreads();
    if (t == 0) {
        if (blockIdx.x < nch) issue(blockIdx.x, 0);
        if (blockIdx.x + G < nch) issue(blockIdx.x + G, 1);
    }
    uint32_t phase[2] = {0u, 0u};
    bool bad = false, timed_out = false;
    int slot = 0;
    for (long long c = blockIdx.x; c < nch; c += G, slot ^= 1) {
        const bool ok = mbar_wait(&S.mbar[slot], phase[slot]);
        if (ok) phase[slot] ^= 1u;
        const int np = (int)chunk_len(c);  // <= CP
        const int full_vecs = (int)(((unsigned)np * 2 * sizeof(T)) >> 4);  // vectors the copy filled
        uint32_t pu[NE], pv[NE], rk[NE];
#pragma unroll
        for (int k = 0; k < kSplitSlots; k++) {
            const int sv = t + k * kSplitThreads;
#pragma unroll
            for (int j = 0; j < P; j++) {
                const int p = sv * P + j;
                uint32_t r = 0xffffffffu;
                if (ok && p < np) {
                    long long u, v;
                    if (sv < full_vecs) vec_pair<T>(S.buf[slot][sv], j, u, v);
                    else scalar_pair<T>(edges, c * CP + p, u, v);  // the odd last int32 pair
                    // ids of int32 pairs compared as 32-bit: a negative id is above n
                    const bool out = sizeof(T) == 4 ? ((uint32_t)u >= n || (uint32_t)v >= n)
                                                    : ((unsigned long long)u >= n || (unsigned long long)v >= n);
                    if (out) {
                        bad = true;
                    } else {
                        pu[k * P + j] = (uint32_t)u;
                        pv[k * P + j] = (uint32_t)v;
                        r = atomicAdd(&S.hist[(uint32_t)u >> wb], 1u) | (atomicAdd(&S.hist[(uint32_t)v >> wb], 1u) << 16);
                    }
                }
                rk[k * P + j] = r;
            }
        }
        // barrier 1: the counts are complete and the buffer is read
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        if (t == 0) {
            inflight[slot] = false;
            if (c + 2 * G < nch) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(c + 2 * G, slot);
            }
        }
        // exclusive scan of the window counts (thread t: windows t * kSplitWpt
        // and on), one reservation per window, counts cleared
        // A window's run is padded to an even length with the id 2^wb (a
        // count slot past the window's counts), so that every run starts on
        // an even stage slot and an even region offset: the runs are written
        // two ids per 32-bit store.
        uint32_t h[kSplitWpt], bt[kSplitWpt], hs = 0u;
#pragma unroll
        for (int q = 0; q < kSplitWpt; q++) {
            const int b = t * kSplitWpt + q;
            h[q] = 0u;
            bt[q] = 0u;
            if (b < nb) {
                h[q] = S.hist[b];
                S.hist[b] = 0u;
                if (h[q]) bt[q] = atomicAdd(&fill[b], (h[q] + 1u) & ~1u);
            }
            hs += (h[q] + 1u) & ~1u;
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
        for (int q = 0; q < kSplitWpt; q++) {
            const int b = t * kSplitWpt + q;
            const uint32_t hp = (h[q] + 1u) & ~1u;
            const uint32_t fit = bt[q] >= cap ? 0u : (cap - bt[q] < hp ? cap - bt[q] : hp);  // even: cap, bt even
            S.loff[b] = lo;
            S.gend[b] = lo + fit;
            S.goff[b] = (I)((unsigned long long)b * cap + bt[q] - lo);  // mod 2^bits; read only where h > 0
            if (h[q] & 1u) S.stage[lo + h[q]] = ((uint32_t)b << 16) | (1u << wb);  // the pad
            short_fit |= fit < hp;
            lo += hp;
        }
        // barrier 3; `over`: a window of this chunk runs past its capacity
        const int over = __syncthreads_or(short_fit);
#pragma unroll
        for (int k = 0; k < NE; k++) {
            const uint32_t r = rk[k];
            if (r == 0xffffffffu) continue;
            const uint32_t bu = pu[k] >> wb, bv = pv[k] >> wb;
            S.stage[S.loff[bu] + (r & 0xffffu)] = (bu << 16) | (pu[k] & low);
            S.stage[S.loff[bv] + (r >> 16)] = (bv << 16) | (pv[k] & low);
        }
        __syncthreads();  // barrier 4
        // stage slots 2i and 2i + 1 hold ids of one window (tot is even)
        if (!over) {
            for (uint32_t i = 2 * t; i < tot; i += 2 * kSplitThreads) {
                const uint2 x = *reinterpret_cast<const uint2 *>(&S.stage[i]);
                *reinterpret_cast<uint32_t *>(&part[S.goff[x.x >> 16] + (I)i]) = (x.x & 0xffffu) | (x.y << 16);
            }
        } else {
            for (uint32_t i = 2 * t; i < tot; i += 2 * kSplitThreads) {
                const uint2 x = *reinterpret_cast<const uint2 *>(&S.stage[i]);
                const uint32_t b = x.x >> 16;
                if (i < S.gend[b]) {
                    *reinterpret_cast<uint32_t *>(&part[S.goff[b] + (I)i]) = (x.x & 0xffffu) | (x.y << 16);
                } else {  // past the region: counted here (a pad counts nothing)
                    atomicAdd(&deg[(b << wb) | (x.x & 0xffffu)], 1u);
                    if ((x.y & 0xffffu) >> wb == 0u) atomicAdd(&deg[(b << wb) | (x.y & 0xffffu)], 1u);
                }
            }
        }
        // the next chunk's counts go to S.hist (cleared before barrier 2);
        // its scan rewrites loff / gend / goff only after its barrier 1
    }
    if (bad) set_err(st, kErrInvalidEdge);
    if (timed_out && t == 0) {
        set_err(st, kErrTimeout);
        // leave no copy writing into shared memory after the block exits
        for (int k = 0; k < 2; k++)
            if (inflight[k]) mbar_wait(&S.mbar[k], phase[k]);
    }
}

__device__ __forceinline__ void smem_count8(uint32_t *cnt, uint4 q) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
        atomicAdd(&cnt[w[i] & 0xffffu], 1u);
        atomicAdd(&cnt[w[i] >> 16], 1u);
    }
}

__device__ __forceinline__ void smem_count8_hub(uint32_t *cnt, uint4 q, uint32_t hub, uint32_t &hc) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint32_t a = w[i] & 0xffffu, b = w[i] >> 16;
        if (a == hub) hc++;
        else atomicAdd(&cnt[a], 1u);
        if (b == hub) hc++;
        else atomicAdd(&cnt[b], 1u);
    }
}

__global__ void __launch_bounds__(kSmemThreads, 1)
    k_degree_window_smem(const uint16_t *__restrict__ part, uint32_t cap, const uint32_t *__restrict__ fill, int wb,
                         vid_t n, uint32_t *deg) {
    extern __shared__ __align__(16) uint32_t cnt[];  // 2^wb counts, the pads' slot, then 32 words of reduction
    uint32_t *red = cnt + (1u << wb) + 32;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int b = blockIdx.x;
    const uint32_t W = 1u << wb;
    for (uint32_t i = t; i <= W; i += kSmemThreads) cnt[i] = 0u;
    __syncthreads();
    const unsigned long long f = fill[b], len = f < cap ? f : cap;
    const uint16_t *p = part + (unsigned long long)b * cap;  // 16-byte aligned: cap is a multiple of 8
    const uint4 *p4 = reinterpret_cast<const uint4 *>(p);
    const unsigned long long nv = len >> 3;
    const unsigned long long ns = nv < (unsigned long long)kSmemSampleVecs ? nv : (unsigned long long)kSmemSampleVecs;
    for (unsigned long long k = t; k < ns; k += kSmemThreads) smem_count8(cnt, __ldcs(p4 + k));
    __syncthreads();
    // the hub: the largest sample count (< 2^15 + 1), as count << 16 | id
    uint32_t key = 0u;
    for (uint32_t i = t; i < W; i += kSmemThreads) {
        const uint32_t c = cnt[i];
        const uint32_t k2 = (c << 16) | i;
        if (c && k2 > key) key = k2;
    }
    key = __reduce_max_sync(0xffffffffu, key);
    if (lane == 0) red[warp] = key;
    __syncthreads();
    if (warp == 0) {
        key = __reduce_max_sync(0xffffffffu, red[lane]);
        if (lane == 0) red[0] = key;
    }
    __syncthreads();
    key = red[0];
    const uint32_t hub = key ? (key & 0xffffu) : 0x10000u;  // no entry equals 0x10000
    uint32_t hc = 0u;
    constexpr int U = 8;
    for (unsigned long long k = ns + t; k < nv; k += (unsigned long long)U * kSmemThreads) {
        uint4 q[U];
#pragma unroll
        for (int j = 0; j < U; j++) {
            const unsigned long long kk = k + (unsigned long long)j * kSmemThreads;
            if (kk < nv) q[j] = __ldcs(p4 + kk);
        }
#pragma unroll
        for (int j = 0; j < U; j++)
            if (k + (unsigned long long)j * kSmemThreads < nv) smem_count8_hub(cnt, q[j], hub, hc);
    }
    {
        const unsigned long long i = nv * 8 + t;  // the last len % 8 entries
        if (i < len) {
            const uint32_t e = p[i];
            if (e == hub) hc++;
            else atomicAdd(&cnt[e], 1u);
        }
    }
    hc = __reduce_add_sync(0xffffffffu, hc);
    if (lane == 0 && hc) atomicAdd(&cnt[hub], hc);
    __syncthreads();
    const unsigned long long x0 = (unsigned long long)b << wb;
    const uint32_t lim = (unsigned long long)n - x0 < W ? (uint32_t)((unsigned long long)n - x0) : W;
    uint32_t *d = deg + x0;
    if (f > cap) {
        for (uint32_t i = t; i < lim; i += kSmemThreads) d[i] += cnt[i];
    } else {
        for (uint32_t i = t; i < lim; i += kSmemThreads) d[i] = cnt[i];
    }
}

// ---------------------------------------------------------------------------
int degree_part_buckets(vid_t n) { return (int)(((long long)n + (1LL << kPartBits) - 1) >> kPartBits); }

bool degree_part_ok(vid_t n, long long m) { return n > (1u << 25) && m >= (1LL << 20); }

// A window holds up to 1.5 times the average entries (a multiple of 4, so
// every window's region starts on a 16-byte boundary); the ids are permuted
// in every workload here, so windows hold the average to within a fraction
// of a percent, and entries past the cap are counted directly (exact either way).
static unsigned long long part_cap(vid_t n, long long m) {
    const int nb = degree_part_buckets(n);
    const unsigned long long avg = (2ull * (unsigned long long)m + nb - 1) / nb;
    return (avg + avg / 2 + 4096 + 3) & ~3ull;
}

// scratch layout: fill[nb] (64-bit reservation counters) at 0, the window
// regions (nb x cap entries of 8 bytes with partners, else 4) from part_offset(nb)
static size_t part_offset(int nb) { return 256 + (((size_t)nb * 8 + 255) & ~(size_t)255); }

size_t degree_part_scratch_bytes(vid_t n, long long m, bool hook) {
    const int nb = degree_part_buckets(n);
    return part_offset(nb) + (size_t)nb * part_cap(n, m) * (hook ? 8 : 4);
}

template <typename T>
void launch_degree_partitioned(const void *edges, long long m, vid_t n, uint32_t *deg, vid_t *hook, void *scratch,
                               DevState *st, int num_sms, int grid, cudaStream_t s) {
    const int nb = degree_part_buckets(n);
    const unsigned long long cap = part_cap(n, m);
    unsigned long long *fill = reinterpret_cast<unsigned long long *>(scratch);
    void *part = static_cast<char *>(scratch) + part_offset(nb);
    cudaMemsetAsync(fill, 0, (size_t)nb * 8, s);
    cudaMemsetAsync(deg, 0, (size_t)n * 4, s);
    if (hook) {
        using E = unsigned long long;
        const long long nch = (m + part_chunk_pairs<T, E>() - 1) / part_chunk_pairs<T, E>();
        const int pgrid = (int)(nch < num_sms ? nch : num_sms);
        if (pgrid > 0)
            k_degree_partition<T, E><<<pgrid, kPartThreads, sizeof(PartShared<E>), s>>>(
                (const T *)edges, m, n, nb, kPartBits, cap, fill, (E *)part, deg, hook, st);
        for (int b = 0; b < nb; b++) k_degree_window_hook<<<grid, kBlock, 0, s>>>((E *)part, cap, fill, b, deg, hook);
    } else {
        using E = uint32_t;
        const long long nch = (m + part_chunk_pairs<T, E>() - 1) / part_chunk_pairs<T, E>();
        const int pgrid = (int)(nch < num_sms ? nch : num_sms);
        if (pgrid > 0)
            k_degree_partition<T, E><<<pgrid, kPartThreads, sizeof(PartShared<E>), s>>>(
                (const T *)edges, m, n, nb, kPartBits, cap, fill, (E *)part, deg, nullptr, st);
        for (int b = 0; b < nb; b++) k_degree_window<<<grid, kBlock, 0, s>>>((E *)part, cap, fill, b, deg);
    }
}
template void launch_degree_partitioned<int32_t>(const void *, long long, vid_t, uint32_t *, vid_t *, void *,
                                                 DevState *, int, int, cudaStream_t);
template void launch_degree_partitioned<int64_t>(const void *, long long, vid_t, uint32_t *, vid_t *, void *,
                                                 DevState *, int, int, cudaStream_t);

// Shared-memory windows: the smallest window of at least 2^11 vertices that
// gives at most kPartMaxBuckets windows (n <= 2^24: 2^15 vertices at most).
bool degree_smem_ok(vid_t n, long long m) {
    return n >= (1u << 20) && n <= (1u << 24) && m >= (1LL << 22);
}

static int smem_window_bits(vid_t n) {
    int wb = kSmemMinBits;
    while (wb < kSmemMaxBits && (((long long)n + (1LL << wb) - 1) >> wb) > kPartMaxBuckets) wb++;
    return wb;
}

static int smem_buckets(vid_t n) {
    const int wb = smem_window_bits(n);
    return (int)(((long long)n + (1LL << wb) - 1) >> wb);
}

// As part_cap, a multiple of 8 (16 bytes of 16-bit entries).
static unsigned long long smem_cap(vid_t n, long long m) {
    const int nb = smem_buckets(n);
    const unsigned long long avg = (2ull * (unsigned long long)m + nb - 1) / nb;
    return (avg + avg / 2 + 4096 + 7) & ~7ull;
}

size_t degree_smem_scratch_bytes(vid_t n, long long m) {
    const int nb = smem_buckets(n);
    return part_offset(nb) + (size_t)nb * smem_cap(n, m) * 2;
}

template <typename T>
void launch_degree_smem(const void *edges, long long m, vid_t n, uint32_t *deg, void *scratch, DevState *st,
                        int num_sms, cudaStream_t s) {
    const int wb = smem_window_bits(n), nb = smem_buckets(n);
    const uint32_t cap = (uint32_t)smem_cap(n, m);
    uint32_t *fill = reinterpret_cast<uint32_t *>(scratch);
    uint16_t *part = reinterpret_cast<uint16_t *>(static_cast<char *>(scratch) + part_offset(nb));
    cudaMemsetAsync(fill, 0, (size_t)nb * 4, s);
    cudaMemsetAsync(deg, 0, (size_t)n * 4, s);
    constexpr long long CP = kSplitChunk / (2 * (long long)sizeof(T));
    const long long nch = (m + CP - 1) / CP;
    const int pgrid = (int)(nch < 2LL * num_sms ? nch : 2LL * num_sms);
    if (pgrid > 0) {
        if ((unsigned long long)nb * cap < (1ull << 32))
            k_degree_split<T, uint32_t><<<pgrid, kSplitThreads, sizeof(SplitShared<uint32_t>), s>>>(
                (const T *)edges, m, n, nb, wb, cap, fill, part, deg, st);
        else
            k_degree_split<T, unsigned long long><<<pgrid, kSplitThreads, sizeof(SplitShared<unsigned long long>), s>>>(
                (const T *)edges, m, n, nb, wb, cap, fill, part, deg, st);
    }
    k_degree_window_smem<<<nb, kSmemThreads, (4u << wb) + 256, s>>>(part, cap, fill, wb, n, deg);
}
template void launch_degree_smem<int32_t>(const void *, long long, vid_t, uint32_t *, void *, DevState *, int,
                                          cudaStream_t);
template void launch_degree_smem<int64_t>(const void *, long long, vid_t, uint32_t *, void *, DevState *, int,
                                          cudaStream_t);

cudaError_t degree_part_setup() {
    const void *ks[] = {(const void *)k_degree_partition<int32_t, uint32_t>,
                        (const void *)k_degree_partition<int64_t, uint32_t>,
                        (const void *)k_degree_partition<int32_t, unsigned long long>,
                        (const void *)k_degree_partition<int64_t, unsigned long long>,
                        (const void *)k_degree_split<int32_t, uint32_t>,
                        (const void *)k_degree_split<int64_t, uint32_t>,
                        (const void *)k_degree_split<int32_t, unsigned long long>,
                        (const void *)k_degree_split<int64_t, unsigned long long>,
                        (const void *)k_degree_window_smem};
    const int sm[] = {(int)sizeof(PartShared<uint32_t>),           (int)sizeof(PartShared<uint32_t>),
                      (int)sizeof(PartShared<unsigned long long>), (int)sizeof(PartShared<unsigned long long>),
                      (int)sizeof(SplitShared<uint32_t>),          (int)sizeof(SplitShared<uint32_t>),
                      (int)sizeof(SplitShared<unsigned long long>), (int)sizeof(SplitShared<unsigned long long>),
                      (4 << kSmemMaxBits) + 256};
    for (int i = 0; i < 9; i++) {
        const cudaError_t e = cudaFuncSetAttribute(ks[i], cudaFuncAttributeMaxDynamicSharedMemorySize, sm[i]);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ccg

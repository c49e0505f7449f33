// Shared device-side definitions of the GB300 connected-components engine.
//
// Internal vertex ids are 32-bit (n < 2^32 - 1). Inputs may be int32 or int64
// pairs; every kernel that touches the caller's edge list is templated on the
// id type and reads it with 128-bit loads (two int32 pairs or one int64 pair
// per load). Internal edge lists are uint2 pairs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ccg {

typedef uint32_t vid_t;

constexpr int kBlock = 256;            // threads per block for the streaming kernels
constexpr int kMaxIters = 256;         // SV iteration slots recorded on the device
constexpr int kMaxLevels = 4096;       // BFS level slots recorded on the device
constexpr uint32_t kNoOwner = 0xffffffffu;  // multi-start BFS: a vertex no tree reached
constexpr int kMaxBfsStarts = 4096;    // multi-start BFS: most ranges (options.bfs_starts)
constexpr uint32_t kHistDense = 1u << 20;   // degrees below this get a dense histogram bin
constexpr uint32_t kHistSmem = 4096;        // bins privatised in shared memory

// Device error bits (collected in DevState::err).
enum : uint32_t {
    kErrInvalidEdge = 1u,
    kErrOverflow = 2u,     // an internal capacity was exceeded (a bug guard, never expected)
    kErrNoConvergence = 4u,
    kErrTimeout = 8u,      // a bounded device wait (an mbarrier of a bulk copy) ran out
    kErrBadOffsets = 16u,  // batched form: offsets not non-decreasing from 0 to the totals
};

// Device-resident bookkeeping for one cc_labels call. Zeroed at the start of
// each call (cudaMemsetAsync); slots indexed by iteration avoid resets.
struct DevState {
    uint32_t err;
    uint32_t cmin;                          // min id among BFS-visited vertices
    unsigned long long maxkey;              // (deg << 32) | (0xffffffff - v): argmax degree, ties to min id
    unsigned long long n_ovf;               // overflow degrees (>= kHistDense) recorded
    unsigned long long nd;                  // distinct degrees >= 1
    unsigned long long ncand;               // K-S candidates
    unsigned long long bfs_visited;
    unsigned long long bfs_inspected;       // adjacency entries read by the BFS
    double ks_out[5];                       // D, alpha, xmin, ntail, ncand
    int route;                              // 1 = BFS first
    int bfs_starts;                         // multi-start BFS: trees started (ranges with a vertex of degree > 0)
    // learned route predictor
    unsigned long long pred_seedkey;        // (sampled degree << 32) | (0xffffffff - v): probe seed
    unsigned long long pred_probe[3];       // new vertices at probe levels 1..3
    int pred_route;                         // 0 SV only, 1 BFS first
    float pred_conf;                        // probability of the predicted route
    int pred_cutoff;                        // BFS levels (0 = run to completion)
    int pad2;
    // device-driven SV loop (CUDA graph WHILE node)
    int loop_it;                            // iteration being run
    int loop_cur;                           // active pairs of iteration loop_it are in ebuf[loop_cur]
    int loop_cap;                           // iteration cap
    int loop_done;                          // iterations run when the loop stopped (0 = not stopped)
    // graph-driven route (stream-ordered cc_labels): every decision on the device
    int route_taken;                        // 1 = the BFS branch ran
    int route_source;                       // 0 = K-S heuristic, 1 = learned predictor, 2 = forced
    int loop_start_it;                      // the SV loop continues after this iteration,
    int loop_start_cur;                     // whose active pairs are in ebuf[loop_start_cur]
    int bfs_level;                          // BFS levels run so far (the level being run)
    int bfs_par;                            // current frontier: queue / bitmap number bfs_par
    int bfs_bu;                             // this level runs bottom-up
    int bfs_queue;                          // the current frontier is held as a queue (else a bitmap)
    int bfs_conv;                           // this level converts: 1 queue -> bitmap, 2 bitmap -> queue
    int bfs_list;                           // edge-list BFS: active pairs in the caller's list (-1) or ebuf[bfs_list]
    int bfs_write;                          // edge-list BFS: this level compacts its active pairs
    int bfs_cutoff;                         // stop the BFS after this many levels (0 = run to completion)
    unsigned long long bfs_len;             // edge-list BFS: pairs in the active list
    unsigned long long bfs_kept_prev;       // edge-list BFS: pairs that stayed active in the previous level
    unsigned long long bfs_explored;        // CSR BFS: adjacency entries of the levels expanded so far
    unsigned long long bfs_prev_f;          // CSR BFS: frontier size of the previous level
    unsigned long long bfs_qcount;          // CSR BFS: bitmap -> queue counter
    // graph-driven batched form
    int batch_g;                            // graph of the current single-graph fit (G: none left)
    int batch_pad;
    long long batch_base, batch_ng;         // its first union id and vertex count
    unsigned long long kept[kMaxIters];     // active pairs written by SV iteration i
    unsigned long long hooked[kMaxIters];   // roots hooked in SV iteration i
    unsigned long long hook_base[kMaxIters + 1];  // start of iteration i's slice of the hooked list
    unsigned long long kept_base[kMaxIters + 1];  // host-input chunks: start of chunk i's surviving pairs
    unsigned long long front[kMaxLevels];   // BFS frontier size entering level l
    unsigned long long front_edges[kMaxLevels];  // sum of degrees of that frontier
};

// ---------------------------------------------------------------------------
// Loads of the caller's edge list.

// Streaming 128-bit load that does not allocate in L1 (edges are read once per pass).
__device__ __forceinline__ int4 ld_stream(const int4 *p) { return __ldcs(p); }
__device__ __forceinline__ uint4 ld_stream(const uint4 *p) { return __ldcs(p); }

// Number of 128-bit vectors holding whole pairs, and pairs per vector, for id type T.
template <typename T> struct PairVec;
template <> struct PairVec<int32_t> { static constexpr int kPairs = 2; };
template <> struct PairVec<int64_t> { static constexpr int kPairs = 1; };
template <> struct PairVec<uint32_t> { static constexpr int kPairs = 2; };

// Decodes pair `j` (0..kPairs-1) of a 128-bit vector as unsigned 64-bit ids.
template <typename T>
__device__ __forceinline__ void vec_pair(const int4 &q, int j, long long &u, long long &v);
template <>
__device__ __forceinline__ void vec_pair<int32_t>(const int4 &q, int j, long long &u, long long &v) {
    u = j == 0 ? (long long)q.x : (long long)q.z;
    v = j == 0 ? (long long)q.y : (long long)q.w;
}
template <>
__device__ __forceinline__ void vec_pair<int64_t>(const int4 &q, int, long long &u, long long &v) {
    u = (long long)(((unsigned long long)(unsigned)q.y << 32) | (unsigned)q.x);
    v = (long long)(((unsigned long long)(unsigned)q.w << 32) | (unsigned)q.z);
}

template <>
__device__ __forceinline__ void vec_pair<uint32_t>(const int4 &q, int j, long long &u, long long &v) {
    u = j == 0 ? (long long)(unsigned)q.x : (long long)(unsigned)q.z;
    v = j == 0 ? (long long)(unsigned)q.y : (long long)(unsigned)q.w;
}

template <typename T>
__device__ __forceinline__ void scalar_pair(const T *e, long long k, long long &u, long long &v) {
    u = (long long)e[2 * k];
    v = (long long)e[2 * k + 1];
}

// ---------------------------------------------------------------------------
// Warp-aggregated append: every lane with `want` gets a distinct slot of a
// global counter; one atomic per warp.
__device__ __forceinline__ unsigned long long warp_append(unsigned long long *counter, bool want) {
    const unsigned mask = __activemask();
    const unsigned ballot = __ballot_sync(mask, want);
    if (!ballot) return 0;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(ballot) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(ballot));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(ballot & ((1u << lane) - 1u));
}

__device__ __forceinline__ void set_err(DevState *st, uint32_t bit) { atomicOr(&st->err, bit); }

// Block-wide exclusive scan of small per-thread counts; thread 0 reserves
// the block's total from `counter` with one atomic. Returns this thread's
// first slot. Called by every thread of the block.
__device__ __forceinline__ unsigned long long block_reserve(unsigned long long *counter, int c, int *sw,
                                                            unsigned long long *sbase) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sw[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int w = lane < nw ? sw[lane] : 0, wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) sw[lane] = wi - w;
        if (lane == nw - 1) *sbase = wi ? atomicAdd(counter, (unsigned long long)wi) : 0ull;
    }
    __syncthreads();
    const unsigned long long r = *sbase + (unsigned long long)(sw[warp] + incl - c);
    __syncthreads();
    return r;
}


// Batched form: graph g owns pairs [eo[g], eo[g+1]) and vertices [vo[g], vo[g+1]).
// The graph of every 2^kTileShift-th pair (and vertex) is precomputed
// (k_tile_graphs), so a tile starts its forward scan without a search.
constexpr int kTileShift = 9;


// A thread's position in the batch while it walks increasing pair indices:
// the graph, where its pairs end, its first union id and its vertex count.
// Offsets are read only when the walk crosses into the next graph.
struct GraphCursor {
    int g;
    long long kend, base, ng;
    __device__ __forceinline__ void start(const int64_t *eo, const int64_t *vo, int g0) {
        g = g0;
        kend = eo[g + 1];
        base = vo[g];
        ng = vo[g + 1] - base;
    }
    __device__ __forceinline__ void seek(const int64_t *eo, const int64_t *vo, int G, long long k) {
        while (k >= kend && g + 1 < G) {
            g++;
            kend = eo[g + 1];
            base = vo[g];
            ng = vo[g + 1] - base;
        }
    }
};
// largest g in [0, G) with off[g] <= k (skips empty graphs)
__device__ __forceinline__ int graph_search(const int64_t *off, int G, long long k) {
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int graph_advance(const int64_t *off, int G, long long k, int g) {
    while (g + 1 < G && off[g + 1] <= k) g++;
    return g;
}

// block_reserve for two counters at once: a = (count for counter A), b =
// (count for counter B), each below 2^16 per thread and 2^16 per block; one
// block-wide scan of a << 16 | b, one atomic per counter. Returns this
// thread's first slot in each. sbase: two words.
__device__ __forceinline__ void block_reserve2(unsigned long long *ca, unsigned long long *cb, int a, int b, int *sw,
                                               unsigned long long *sbase, unsigned long long &oa,
                                               unsigned long long &ob) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = (a << 16) | b;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sw[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int w = lane < nw ? sw[lane] : 0, wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) sw[lane] = wi - w;
        if (lane == nw - 1) {
            const int ta = wi >> 16, tb = wi & 0xffff;
            sbase[0] = ta ? atomicAdd(ca, (unsigned long long)ta) : 0ull;
            sbase[1] = tb ? atomicAdd(cb, (unsigned long long)tb) : 0ull;
        }
    }
    __syncthreads();
    const int ex = sw[warp] + incl - c;
    oa = sbase[0] + (unsigned long long)(ex >> 16);
    ob = sbase[1] + (unsigned long long)(ex & 0xffff);
    __syncthreads();
}

// Grid-stride helpers
__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

}  // namespace ccg

// Shiloach-Vishkin iterations (Section 3.1) on a parent array.
//
// The paper's Algorithm 1 joins every partition p to its minimum neighbouring
// partition p_min (the first two sorts), revises p_min by pointer doubling
// (the temporary tuples and the last two sorts), and excludes partitions that
// have no neighbour left (Section 3.1.4). Here a partition is a tree of the
// parent array identified by its root, and one iteration is:
//
//  hook     for every active pair (a, b): ra = parent[a], rb = parent[b]
//           (roots at the start of the iteration); if ra != rb the larger
//           root takes atomicMin(parent[max], min), so after the pass every
//           root p that has a smaller neighbouring root points at the
//           smallest of them - the paper's "p joins p_min". The pair is
//           written to the next active list as (ra, rb): completion is
//           detected one iteration late, exactly as in Section 3.1.4, and
//           the list only ever names current roots (edge contraction).
//           Every root hooked in this iteration is recorded once (the
//           atomicMin that sees the old value equal to the root itself).
//  shortcut pointer jumping with path halving over the roots hooked in this
//           iteration, so each of them points at the root at the end of the
//           iteration (the paper's pointer doubling).
//
// Parents only ever decrease and always point at a smaller id, so the
// structure stays a forest; trees only merge, so a dropped pair (equal
// roots) stays resolved. The loop ends when no pair is active. The final
// label of v is its root, the minimum id of its component (Section 3.1.1).
//
// Pass variants: MODE 0 is the first pass over the caller's pairs while
// parent is the identity (no gathers, nothing written); MODE 1 is the first
// pass after the BFS step (Algorithm 2, lines 8-9: pairs with both ends
// visited are dropped, a visited end stands for the BFS component's root);
// MODE 2 gathers parents.
#include "cc_common.cuh"
#include "cc_kernels.h"

namespace ccg {

template <> struct PairVec<uint32_t> { static constexpr int kPairs = 2; };
template <>
__device__ __forceinline__ void vec_pair<uint32_t>(const int4 &q, int j, long long &u, long long &v) {
    u = j == 0 ? (long long)(unsigned)q.x : (long long)(unsigned)q.z;
    v = j == 0 ? (long long)(unsigned)q.y : (long long)(unsigned)q.w;
}
template <>
__device__ __forceinline__ void scalar_pair<uint32_t>(const uint32_t *e, long long k, long long &u, long long &v) {
    u = (long long)e[2 * k];
    v = (long long)e[2 * k + 1];
}

__device__ __forceinline__ bool vis_test(const uint32_t *vis, long long v) {
    return (vis[v >> 5] >> (v & 31)) & 1u;
}

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

// One pair of an SV pass. Returns true if the pair stays active; `hooked`
// is set when this pair's atomicMin turned a root into a non-root (only
// tracked when RECORD). The plain read before the atomic skips hooks that
// cannot lower parent[hi] (parents only decrease, so a stale read is an
// upper bound of the current value).
template <int MODE, bool RECORD>
__device__ __forceinline__ bool sv_pair(long long u, long long v, vid_t n, vid_t *parent, const uint32_t *vis,
                                        vid_t cmin, vid_t &ru, vid_t &rv, bool &hooked, bool &bad) {
    hooked = false;
    if ((unsigned long long)u >= n || (unsigned long long)v >= n) {
        bad = true;
        return false;
    }
    if (MODE == 0) {
        ru = (vid_t)u;
        rv = (vid_t)v;
    } else if (MODE == 1) {
        const bool ok = cmin < n;
        const bool a = ok && vis_test(vis, u), b = ok && vis_test(vis, v);
        ru = a ? cmin : (vid_t)u;
        rv = b ? cmin : (vid_t)v;
    } else {
        ru = parent[u];
        rv = parent[v];
    }
    if (ru == rv) return false;
    const vid_t hi = ru > rv ? ru : rv, lo = ru > rv ? rv : ru;
    if (parent[hi] > lo) {
        if (RECORD) hooked = atomicMin(&parent[hi], lo) == hi;
        else atomicMin(&parent[hi], lo);
    }
    return true;
}

template <typename T> struct PassUnroll { static constexpr int U = 2; };
template <> struct PassUnroll<int64_t> { static constexpr int U = 4; };

template <typename T, int MODE, bool WRITE, bool RECORD>
__global__ void __launch_bounds__(kBlock) k_sv_pass(const T *__restrict__ in, long long m, vid_t n, vid_t *parent,
                                                    const uint32_t *__restrict__ vis, vid_t cmin, vid_t *hooked_list,
                                                    uint2 *__restrict__ out, DevState *st, int it) {
    constexpr int P = PairVec<T>::kPairs;
    constexpr int U = PassUnroll<T>::U;
    constexpr int K = P * U;  // pairs per thread per round
    __shared__ int sw[32];
    __shared__ unsigned long long sbase;
    const long long nvec = m / P;
    const int4 *ev = reinterpret_cast<const int4 *>(in);
    const unsigned long long hbase = RECORD ? st->hook_base[it] : 0ull;
    bool bad = false;
    // block-contiguous tiles of kBlock * U vectors, so the block's rounds are uniform
    const long long tile = (long long)kBlock * U;
    const long long ntiles = (nvec + tile - 1) / tile;
    for (long long t = blockIdx.x; t < ntiles + (P == 2 && (m & 1) ? 1 : 0); t += gridDim.x) {
        vid_t ru[K], rv[K];
        bool keep[K], hk[K];
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
                    long long u, v;
                    vec_pair<T>(q[k], j, u, v);
                    keep[k * P + j] = i < nvec && sv_pair<MODE, RECORD>(u, v, n, parent, vis, cmin, ru[k * P + j],
                                                                        rv[k * P + j], hk[k * P + j], bad);
                    if (i >= nvec) hk[k * P + j] = false;
                }
            }
        } else {  // the odd last pair of an int32 / internal list
#pragma unroll
            for (int k = 0; k < K; k++) keep[k] = hk[k] = false;
            if (threadIdx.x == 0) {
                long long u, v;
                scalar_pair<T>(in, m - 1, u, v);
                keep[0] = sv_pair<MODE, RECORD>(u, v, n, parent, vis, cmin, ru[0], rv[0], hk[0], bad);
            }
        }
        if (WRITE) {
            int c = 0;
#pragma unroll
            for (int k = 0; k < K; k++) c += keep[k];
            unsigned long long o = block_reserve(&st->kept[it], c, sw, &sbase);
#pragma unroll
            for (int k = 0; k < K; k++)
                if (keep[k]) out[o++] = make_uint2(ru[k], rv[k]);
        }
        if (RECORD) {
            int c = 0;
#pragma unroll
            for (int k = 0; k < K; k++) c += hk[k];
            unsigned long long o = block_reserve(&st->hooked[it], c, sw, &sbase);
#pragma unroll
            for (int k = 0; k < K; k++)
                if (hk[k]) hooked_list[hbase + o++] = ru[k] > rv[k] ? ru[k] : rv[k];
        }
    }
    if (bad) set_err(st, kErrInvalidEdge);
}

// Pointer jumping with path halving for every vertex (used after a pass that
// did not record its hooks). Only shortcuts happen while it runs.
__global__ void __launch_bounds__(kBlock) k_shortcut_all(vid_t *parent, vid_t n, DevState *st, int it) {
    for (long long v = gtid(); v < (long long)n; v += gstride()) {
        vid_t y = parent[v];
        if (y == (vid_t)v) continue;
        while (true) {
            const vid_t p = parent[y];
            if (p == y) break;
            const vid_t g = parent[p];
            if (g == p) {
                y = p;
                break;
            }
            parent[y] = g;
            y = g;
        }
        parent[v] = y;
    }
    if (gtid() == 0) st->hook_base[it + 1] = st->hook_base[it] + st->hooked[it];
}

// Path-halving shortcut of the roots hooked in iteration `it`. Only
// shortcuts happen while it runs (no hooks), so every write replaces a
// parent by one of its ancestors and concurrent chases stay consistent.
__global__ void __launch_bounds__(kBlock) k_sv_shortcut(vid_t *parent, const vid_t *__restrict__ hooked_list,
                                                        DevState *st, int it) {
    const unsigned long long base = st->hook_base[it], cnt = st->hooked[it];
    for (long long i = gtid(); i < (long long)cnt; i += gstride()) {
        const vid_t x = hooked_list[base + i];
        vid_t y = x;
        while (true) {
            const vid_t p = parent[y];
            if (p == y) break;
            const vid_t g = parent[p];
            if (g == p) {
                y = p;
                break;
            }
            parent[y] = g;
            y = g;
        }
        parent[x] = y;
    }
    if (gtid() == 0) st->hook_base[it + 1] = base + cnt;
}

// parent[v] = v, or the BFS component's minimum for visited vertices.
__global__ void __launch_bounds__(kBlock) k_parent_init(vid_t *parent, vid_t n, const uint32_t *__restrict__ vis,
                                                        vid_t cmin) {
    for (long long v = gtid(); v < (long long)n; v += gstride()) {
        vid_t p = (vid_t)v;
        if (vis && cmin < n && vis_test(vis, v)) p = cmin;
        parent[v] = p;
    }
}

__device__ __forceinline__ vid_t find_root(vid_t *parent, vid_t v) {
    vid_t p = parent[v];
    vid_t q = parent[p];
    if (q == p) return p;
    while (true) {
        const vid_t r = parent[q];
        if (r == q) break;
        q = r;
    }
    parent[v] = q;  // compress: later chases through v stop here
    return q;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_finalize(vid_t *parent, vid_t n, T *__restrict__ labels) {
    const long long n4 = (long long)n / 4;
    for (long long i = gtid(); i < n4; i += gstride()) {
        const long long v = i * 4;
        const T a = (T)find_root(parent, (vid_t)v), b = (T)find_root(parent, (vid_t)(v + 1));
        const T c = (T)find_root(parent, (vid_t)(v + 2)), d = (T)find_root(parent, (vid_t)(v + 3));
        if (sizeof(T) == 4) {
            reinterpret_cast<int4 *>(labels)[i] = make_int4((int)a, (int)b, (int)c, (int)d);
        } else {
            reinterpret_cast<longlong2 *>(labels)[2 * i] = make_longlong2((long long)a, (long long)b);
            reinterpret_cast<longlong2 *>(labels)[2 * i + 1] = make_longlong2((long long)c, (long long)d);
        }
    }
    for (long long v = n4 * 4 + gtid(); v < (long long)n; v += gstride()) labels[v] = (T)find_root(parent, (vid_t)v);
}

// ---------------------------------------------------------------------------
// Host launchers

template <typename T>
void launch_sv_pass(int mode, bool write, bool record, const void *in, long long m, vid_t n, vid_t *parent,
                    const uint32_t *vis, vid_t cmin, vid_t *hooked_list, uint2 *out, DevState *st, int it, int grid,
                    cudaStream_t s) {
    const T *e = (const T *)in;
#define SVP(M, W, R) k_sv_pass<T, M, W, R><<<grid, kBlock, 0, s>>>(e, m, n, parent, vis, cmin, hooked_list, out, st, it)
    if (mode == 0) {
        if (write) SVP(0, true, false);
        else SVP(0, false, false);
    } else if (mode == 1) {
        SVP(1, true, true);
    } else {
        if (record) SVP(2, true, true);
        else SVP(2, true, false);
    }
#undef SVP
}
template void launch_sv_pass<int32_t>(int, bool, bool, const void *, long long, vid_t, vid_t *, const uint32_t *,
                                      vid_t, vid_t *, uint2 *, DevState *, int, int, cudaStream_t);
template void launch_sv_pass<int64_t>(int, bool, bool, const void *, long long, vid_t, vid_t *, const uint32_t *,
                                      vid_t, vid_t *, uint2 *, DevState *, int, int, cudaStream_t);
template void launch_sv_pass<uint32_t>(int, bool, bool, const void *, long long, vid_t, vid_t *, const uint32_t *,
                                       vid_t, vid_t *, uint2 *, DevState *, int, int, cudaStream_t);

void launch_shortcut_all(vid_t *parent, vid_t n, DevState *st, int it, int grid, cudaStream_t s) {
    k_shortcut_all<<<grid, kBlock, 0, s>>>(parent, n, st, it);
}

void launch_sv_shortcut(vid_t *parent, const vid_t *hooked_list, DevState *st, int it, int grid, cudaStream_t s) {
    k_sv_shortcut<<<grid, kBlock, 0, s>>>(parent, hooked_list, st, it);
}

void launch_parent_init(vid_t *parent, vid_t n, const uint32_t *vis, vid_t cmin, int grid, cudaStream_t s) {
    if (n == 0) return;
    k_parent_init<<<grid, kBlock, 0, s>>>(parent, n, vis, cmin);
}

template <typename T>
void launch_finalize(vid_t *parent, vid_t n, void *labels, int grid, cudaStream_t s) {
    if (n == 0) return;
    k_finalize<T><<<grid, kBlock, 0, s>>>(parent, n, (T *)labels);
}
template void launch_finalize<int32_t>(vid_t *, vid_t, void *, int, cudaStream_t);
template void launch_finalize<int64_t>(vid_t *, vid_t, void *, int, cudaStream_t);

}  // namespace ccg

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

template <int MODE, bool WRITE>
__device__ __forceinline__ void sv_pair(long long u, long long v, bool valid, vid_t n, vid_t *parent,
                                        const uint32_t *vis, vid_t cmin, vid_t *hooked_list, unsigned long long hbase,
                                        uint2 *out, DevState *st, int it, bool &bad) {
    bool keep = false, first = false;
    vid_t ru = 0, rv = 0, hi = 0;
    if (valid) {
        if ((unsigned long long)u >= n || (unsigned long long)v >= n) {
            bad = true;
        } else {
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
            if (ru != rv) {
                hi = ru > rv ? ru : rv;
                const vid_t lo = ru > rv ? rv : ru;
                const vid_t old = atomicMin(&parent[hi], lo);
                first = old == hi;
                keep = true;
            }
        }
    }
    const unsigned long long h = warp_append(&st->hooked[it], first);
    if (first) hooked_list[hbase + h] = hi;
    if (WRITE) {
        const unsigned long long k = warp_append(&st->kept[it], keep);
        if (keep) out[k] = make_uint2(ru, rv);
    }
}

template <typename T, int MODE, bool WRITE>
__global__ void __launch_bounds__(kBlock) k_sv_pass(const T *__restrict__ in, long long m, vid_t n, vid_t *parent,
                                                    const uint32_t *__restrict__ vis, vid_t cmin, vid_t *hooked_list,
                                                    uint2 *__restrict__ out, DevState *st, int it) {
    constexpr int P = PairVec<T>::kPairs;
    constexpr int U = 2;
    const long long nvec = m / P;
    const int4 *ev = reinterpret_cast<const int4 *>(in);
    const unsigned long long hbase = st->hook_base[it];
    bool bad = false;
    const long long stride = gstride();
    // every lane runs the same number of rounds so the warp-aggregated appends stay converged
    const long long rounds = (nvec + stride * U - 1) / (stride * U);
    for (long long r = 0; r < rounds; r++) {
        const long long base = gtid() + r * stride * U;
        int4 q[U];
#pragma unroll
        for (int k = 0; k < U; k++) {
            const long long i = base + (long long)k * stride;
            q[k] = i < nvec ? ld_stream(ev + i) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int k = 0; k < U; k++) {
            const long long i = base + (long long)k * stride;
#pragma unroll
            for (int j = 0; j < P; j++) {
                long long u, v;
                vec_pair<T>(q[k], j, u, v);
                sv_pair<MODE, WRITE>(u, v, i < nvec, n, parent, vis, cmin, hooked_list, hbase, out, st, it, bad);
            }
        }
    }
    if (P == 2 && (m & 1) && blockIdx.x == 0 && threadIdx.x < 32) {
        long long u = 0, v = 0;
        if (threadIdx.x == 0) scalar_pair<T>(in, m - 1, u, v);
        sv_pair<MODE, WRITE>(u, v, threadIdx.x == 0, n, parent, vis, cmin, hooked_list, hbase, out, st, it, bad);
    }
    if (bad) set_err(st, kErrInvalidEdge);
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
void launch_sv_pass(int mode, bool write, const void *in, long long m, vid_t n, vid_t *parent, const uint32_t *vis,
                    vid_t cmin, vid_t *hooked_list, uint2 *out, DevState *st, int it, int grid, cudaStream_t s) {
    const T *e = (const T *)in;
    if (mode == 0) {
        if (write) k_sv_pass<T, 0, true><<<grid, kBlock, 0, s>>>(e, m, n, parent, vis, cmin, hooked_list, out, st, it);
        else k_sv_pass<T, 0, false><<<grid, kBlock, 0, s>>>(e, m, n, parent, vis, cmin, hooked_list, out, st, it);
    } else if (mode == 1) {
        k_sv_pass<T, 1, true><<<grid, kBlock, 0, s>>>(e, m, n, parent, vis, cmin, hooked_list, out, st, it);
    } else {
        k_sv_pass<T, 2, true><<<grid, kBlock, 0, s>>>(e, m, n, parent, vis, cmin, hooked_list, out, st, it);
    }
}
template void launch_sv_pass<int32_t>(int, bool, const void *, long long, vid_t, vid_t *, const uint32_t *, vid_t,
                                      vid_t *, uint2 *, DevState *, int, int, cudaStream_t);
template void launch_sv_pass<int64_t>(int, bool, const void *, long long, vid_t, vid_t *, const uint32_t *, vid_t,
                                      vid_t *, uint2 *, DevState *, int, int, cudaStream_t);
template void launch_sv_pass<uint32_t>(int, bool, const void *, long long, vid_t, vid_t *, const uint32_t *, vid_t,
                                       vid_t *, uint2 *, DevState *, int, int, cudaStream_t);

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

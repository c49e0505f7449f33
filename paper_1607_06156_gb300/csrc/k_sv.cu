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
//           iteration (the paper's pointer doubling); parent writes are
//           atomicMin so concurrent chases cannot leave a vertex one level
//           short of its root.
//
// Parents only ever decrease and always point at a smaller id, so the
// structure stays a forest; trees only merge, so a dropped pair (equal
// roots) stays resolved. The loop ends when no pair is active. The final
// label of v is its root, the minimum id of its component (Section 3.1.1).
//
// Pass variants: MODE 0 is the first pass over the caller's pairs while
// parent is the identity (no gathers, nothing written; MODE 4 is the same
// without the read of parent[max] before the atomicMin); MODE 1 is the first
// pass after the BFS step (Algorithm 2, lines 8-9: pairs with both ends
// visited are dropped, a visited end stands for the BFS component's root);
// MODE 2 gathers parents (one hop: every vertex the pass reads points at a
// root after the previous shortcut); MODE 3 chases each end to its current
// root, for pairs read while parents may be one or more hops from their
// roots (the chunks of the host-input path).
#include "cc_common.cuh"
#include "cc_kernels.h"

namespace ccg {


__device__ __forceinline__ bool vis_test(const uint32_t *vis, long long v) {
    return (vis[v >> 5] >> (v & 31)) & 1u;
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
    if (MODE == 0 || MODE == 4) {
        ru = (vid_t)u;
        rv = (vid_t)v;
        if (MODE == 4) {  // no pre-check: a fire-and-forget atomicMin
            if (ru == rv) return false;
            const vid_t hi = ru > rv ? ru : rv, lo = ru > rv ? rv : ru;
            atomicMin(&parent[hi], lo);
            return true;
        }
    } else if (MODE == 1) {
        const bool ok = cmin < n;
        const bool a = ok && vis_test(vis, u), b = ok && vis_test(vis, v);
        ru = a ? cmin : (vid_t)u;
        rv = b ? cmin : (vid_t)v;
    } else if (MODE == 2) {
        ru = parent[u];
        rv = parent[v];
    } else {  // MODE 3: chase to the roots at read time (parents point at smaller ids, so this ends)
        ru = (vid_t)u;
        for (vid_t p = parent[ru]; p != ru; p = parent[ru]) ru = p;
        rv = (vid_t)v;
        for (vid_t p = parent[rv]; p != rv; p = parent[rv]) rv = p;
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

// MODE 3 (the chunks of the host-input path) appends its surviving pairs
// after those of the earlier chunks: at out + kept_base[it].
//
// SAMPLED passes read one tile in `tstride` (tiles of kBlock * U vectors,
// whole tiles so the reads stay coalesced) and skip the odd last pair: the
// sample front end of the SV route.
template <typename T, int MODE, bool WRITE, bool RECORD, bool SAMPLED = false>
__device__ __forceinline__ void sv_pass_body(const T *__restrict__ in, long long m, vid_t n, vid_t *parent,
                                             const uint32_t *__restrict__ vis, vid_t cmin, vid_t *hooked_list,
                                             uint2 *__restrict__ out, DevState *st, int it, int tstride = 1) {
    if (MODE == 3 && WRITE) out += st->kept_base[it];
    constexpr int P = PairVec<T>::kPairs;
    constexpr int U = PassUnroll<T>::U;
    constexpr int K = P * U;  // pairs per thread per round
    __shared__ int sw[32];
    __shared__ unsigned long long sbase;
    __shared__ unsigned long long sbase2[2];
    const long long nvec = m / P;
    const int4 *ev = reinterpret_cast<const int4 *>(in);
    const unsigned long long hbase = RECORD ? st->hook_base[it] : 0ull;
    bool bad = false;
    // block-contiguous tiles of kBlock * U vectors, so the block's rounds are uniform
    const long long tile = (long long)kBlock * U;
    const long long ntiles = (nvec + tile - 1) / tile;
    const long long nt = SAMPLED ? (ntiles + tstride - 1) / tstride : ntiles + (P == 2 && (m & 1) ? 1 : 0);
    for (long long tt = blockIdx.x; tt < nt; tt += gridDim.x) {
        const long long t = SAMPLED ? tt * tstride : tt;
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
        if (WRITE && RECORD) {  // both lists with one block-wide scan
            int ck = 0, ch = 0;
#pragma unroll
            for (int k = 0; k < K; k++) {
                ck += keep[k];
                ch += hk[k];
            }
            unsigned long long ok, oh;
            block_reserve2(&st->kept[it], &st->hooked[it], ck, ch, sw, sbase2, ok, oh);
#pragma unroll
            for (int k = 0; k < K; k++) {
                if (keep[k]) out[ok++] = make_uint2(ru[k], rv[k]);
                if (hk[k]) hooked_list[hbase + oh++] = ru[k] > rv[k] ? ru[k] : rv[k];
            }
        } else if (WRITE) {
            int c = 0;
#pragma unroll
            for (int k = 0; k < K; k++) c += keep[k];
            unsigned long long o = block_reserve(&st->kept[it], c, sw, &sbase);
#pragma unroll
            for (int k = 0; k < K; k++)
                if (keep[k]) out[o++] = make_uint2(ru[k], rv[k]);
        } else if (RECORD) {
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

// int32 pairs: 8 resident blocks per SM (the grid-stride grid is 8 blocks
// per SM), so at most 32 registers; the int64 forms need more and run fewer
template <typename T> struct PassMinBlocks { static constexpr int v = 8; };
template <> struct PassMinBlocks<int64_t> { static constexpr int v = 1; };

template <typename T, int MODE, bool WRITE, bool RECORD>
__global__ void __launch_bounds__(kBlock, PassMinBlocks<T>::v) k_sv_pass(const T *__restrict__ in, long long m, vid_t n, vid_t *parent,
                                                    const uint32_t *__restrict__ vis, vid_t cmin, vid_t *hooked_list,
                                                    uint2 *__restrict__ out, DevState *st, int it) {
    sv_pass_body<T, MODE, WRITE, RECORD>(in, m, n, parent, vis, cmin, hooked_list, out, st, it);
}

// The sample passes of the SV front end: MODE 0 (identity parents) or
// MODE 2 (one-hop gathers), hooks only (no list is written, no hook recorded).
template <typename T, int MODE>
__global__ void __launch_bounds__(kBlock, PassMinBlocks<T>::v) k_sv_sample(const T *__restrict__ in, long long m, vid_t n,
                                                                           vid_t *parent, DevState *st, int tstride) {
    sv_pass_body<T, MODE, false, false, true>(in, m, n, parent, nullptr, 0, nullptr, nullptr, st, 0, tstride);
}

// ---------------------------------------------------------------------------
// Device-driven SV loop (the body of a CUDA graph WHILE node). The iteration
// number, the ping-pong buffer and the active-pair count live in DevState,
// so the loop runs with no host round trip per iteration:
//   k_sv_loop_init   after iteration it0 (whose pairs are in eb[cur0]): stop
//                    if nothing stayed active, else start iteration it0 + 1
//   k_sv_pass_loop   hook pass over the active list of iteration loop_it
//   k_sv_shortcut_loop
//   k_sv_loop_step   continue while pairs stayed active; past the iteration
//                    cap the loop stops with kErrNoConvergence
// The host loop it replaces ends identically (same iterations, same lists).

__device__ __forceinline__ void sv_loop_decide(DevState *st, int it, cudaGraphConditionalHandle h) {
    // `it` is the iteration just completed
    if (st->kept[it] == 0) {
        st->loop_done = it + 1;
        cudaGraphSetConditional(h, 0u);
    } else if (it + 1 >= st->loop_cap) {
        set_err(st, kErrNoConvergence);
        st->loop_done = it + 1;
        cudaGraphSetConditional(h, 0u);
    } else {
        st->loop_it = it + 1;
        cudaGraphSetConditional(h, 1u);
    }
}

__global__ void k_sv_loop_init(DevState *st, int it0, int cur0, int cap, cudaGraphConditionalHandle h) {
    st->loop_cap = cap < kMaxIters ? cap : kMaxIters;
    st->loop_cur = cur0;
    sv_loop_decide(st, it0, h);
}

__global__ void __launch_bounds__(kBlock, 8) k_sv_pass_loop(const uint2 *eb0, const uint2 *eb1, vid_t n, vid_t *parent,
                                                         vid_t *hooked_list, DevState *st) {
    const int it = st->loop_it, cur = st->loop_cur;
    const long long m = (long long)st->kept[it - 1];
    const uint2 *in = cur ? eb1 : eb0;
    uint2 *out = const_cast<uint2 *>(cur ? eb0 : eb1);
    sv_pass_body<uint32_t, 2, true, true>(reinterpret_cast<const uint32_t *>(in), m, n, parent, nullptr, 0,
                                          hooked_list, out, st, it);
}

__global__ void k_sv_loop_step(DevState *st, cudaGraphConditionalHandle h) {
    const int it = st->loop_it;
    st->loop_cur ^= 1;
    sv_loop_decide(st, it, h);
}

// Chase from x to its root with path halving. No hook runs while a shortcut
// kernel runs, so every value written is an ancestor of the vertex it is
// written to; the writes are atomicMin, so a stale halving write of one
// thread (a grandparent read before another thread pointed the vertex at
// its root) can never undo a later, smaller value: the root is the smallest
// ancestor, and a vertex set to its root stays there. After the kernel every
// vertex it processed points at its root, which the next hook pass relies on
// (its one-jump parent reads are then roots).
__device__ __forceinline__ void shortcut_to_root(vid_t *parent, vid_t x) {
    vid_t y = x;
    while (true) {
        const vid_t p = parent[y];
        if (p == y) break;
        const vid_t g = parent[p];
        if (g == p) {
            y = p;
            break;
        }
        atomicMin(&parent[y], g);
        y = g;
    }
    if (y != x) atomicMin(&parent[x], y);
}

// Shortcut of every vertex (used after a pass that did not record its hooks).
__global__ void __launch_bounds__(kBlock) k_shortcut_all(vid_t *parent, vid_t n, DevState *st, int it) {
    for (long long v = gtid(); v < (long long)n; v += gstride())
        if (parent[v] != (vid_t)v) shortcut_to_root(parent, (vid_t)v);
    if (gtid() == 0) st->hook_base[it + 1] = st->hook_base[it] + st->hooked[it];
}

// Shortcut of the roots hooked in iteration `it` (it < 0: DevState::loop_it).
__global__ void __launch_bounds__(kBlock) k_sv_shortcut(vid_t *parent, const vid_t *__restrict__ hooked_list,
                                                        DevState *st, int it) {
    if (it < 0) it = st->loop_it;
    const unsigned long long base = st->hook_base[it], cnt = st->hooked[it];
    for (long long i = gtid(); i < (long long)cnt; i += gstride()) shortcut_to_root(parent, hooked_list[base + i]);
    if (gtid() == 0) {
        st->hook_base[it + 1] = base + cnt;
        st->kept_base[it + 1] = st->kept_base[it] + st->kept[it];
    }
}

// After the host-input chunks 1..it: kept[it] becomes the length of the one
// list they appended to, which the next iteration reads.
__global__ void k_stream_finish(DevState *st, int it) { st->kept[it] = st->kept_base[it] + st->kept[it]; }

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
// Batched form: G independent graphs as one disjoint union. Graph g owns
// pairs [eo[g], eo[g+1]) with ids local to it and vertices [vo[g], vo[g+1])
// of the union; the union's components are exactly the graphs' components,
// and a component's minimum union id is vo[g] plus its minimum local id.


// The SV front end per graph: a graph with 2 m_g / n_g >= 4 has its tiles
// sampled one in k_g, k_g the largest power of two <= 2 m_g / n_g and at
// most 64 (the single-graph rule: the sample's mean degree is about 1 or
// more, so it holds a giant component); other graphs are not sampled (0).
__device__ __forceinline__ int batch_sample_stride(long long mg, long long ng) {
    if (ng <= 0 || 2 * mg < 4 * ng) return 0;
    int k = 4;
    while (k < 64 && 2 * mg >= 2LL * k * ng) k *= 2;
    return k;
}

// Which tiles a pass takes (FILTER), by the sample stride k of the graph
// holding the tile's first pair: 0 every tile; 1 the front end's first
// pass: every tile of a graph that is not sampled and one tile in k of a
// sampled graph; 2 the front end's second pass: the sampled tiles only.
template <int FILTER>
__device__ __forceinline__ bool batch_take_tile(long long t, long long k0, const int64_t *eo, const int64_t *vo,
                                                int G, int g0) {
    if (FILTER == 0) return true;
    const int g = graph_advance(eo, G, k0, g0);
    const int k = batch_sample_stride(eo[g + 1] - eo[g], vo[g + 1] - vo[g]);
    if (k == 0) return FILTER == 1;
    return (t & (k - 1)) == 0;
}

// U: 16-byte vectors (two pairs each) per thread per tile, and the tile
// order: a grid stride (regions = 0), or tiles from `next` (a zeroed counter)
// over `regions` contiguous regions of the pairs worked on side by side
// (fetch f takes tile f / regions of region f % regions) - the schedule the
// batched form's tuner picks.
template <int MODE, bool WRITE, bool RECORD, int U, int FILTER = 0>
__global__ void __launch_bounds__(kBlock) k_sv_pass_batch(const int32_t *__restrict__ in, long long m,
                                                          const int64_t *__restrict__ eo,
                                                          const int64_t *__restrict__ vo, int G, vid_t ntot,
                                                          vid_t *parent, vid_t *hooked_list, uint2 *__restrict__ out,
                                                          DevState *st, int it, const uint32_t *__restrict__ tg,
                                                          int regions, unsigned long long *next) {
    constexpr int K = 2 * U;
    __shared__ int sw[32];
    __shared__ unsigned long long sbase;
    __shared__ unsigned long long sbase2[2];
    const long long nvec = m / 2;
    const int4 *ev = reinterpret_cast<const int4 *>(in);
    const unsigned long long hbase = RECORD ? st->hook_base[it] : 0ull;
    bool bad = false;
    const long long tile = (long long)kBlock * U;
    const long long ntiles = (nvec + tile - 1) / tile;
    const long long nt_all = ntiles + ((m & 1) ? 1 : 0);  // the odd last pair is a tile of its own
    const long long per = regions > 0 ? (nt_all + regions - 1) / regions : 0;
    const long long nfetch = per * regions;
    __shared__ long long s_f;
    long long slot = blockIdx.x;
    for (;;) {
        long long t;
        if (regions > 0) {
            __syncthreads();  // every thread has read the previous fetch
            if (threadIdx.x == 0) s_f = (long long)atomicAdd(next, 1ull);
            __syncthreads();
            const long long f = s_f;
            if (f >= nfetch) break;
            t = (f % regions) * per + f / regions;
            if (t >= nt_all) continue;  // past the end of the last region
        } else {
            t = slot;
            slot += gridDim.x;
            if (t >= nt_all) break;
        }
        const long long k0 = t < ntiles ? t * tile * 2 : m - 1;  // first pair of the tile
        const int g0 = (int)tg[k0 >> kTileShift];  // a graph at or before the tile's first pair
        if (!batch_take_tile<FILTER>(t, k0, eo, vo, G, g0)) continue;  // the same for the whole block
        long long u[K], v[K], k[K];
        bool valid[K];
        if (t < ntiles) {
#pragma unroll
            for (int r = 0; r < U; r++) {
                const long long i = t * tile + (long long)r * kBlock + threadIdx.x;
                const int4 q = i < nvec ? ld_stream(ev + i) : make_int4(0, 0, 0, 0);
                u[2 * r] = q.x; v[2 * r] = q.y; k[2 * r] = 2 * i;
                u[2 * r + 1] = q.z; v[2 * r + 1] = q.w; k[2 * r + 1] = 2 * i + 1;
                valid[2 * r] = valid[2 * r + 1] = i < nvec;
            }
        } else {
#pragma unroll
            for (int r = 0; r < K; r++) {
                u[r] = v[r] = 0;
                k[r] = m - 1;
                valid[r] = false;
            }
            if (threadIdx.x == 0) {
                u[0] = in[2 * (m - 1)];
                v[0] = in[2 * (m - 1) + 1];
                valid[0] = true;
            }
        }
        vid_t ru[K], rv[K];
        bool keep[K], hk[K];
        GraphCursor gc;
        gc.start(eo, vo, g0);
#pragma unroll
        for (int r = 0; r < K; r++) {
            keep[r] = hk[r] = false;
            if (!valid[r]) continue;
            gc.seek(eo, vo, G, k[r]);
            const long long base = gc.base, ng = gc.ng;
            if (u[r] < 0 || v[r] < 0 || u[r] >= ng || v[r] >= ng) {
                bad = true;
                continue;
            }
            keep[r] = sv_pair<MODE, RECORD>(base + u[r], base + v[r], ntot, parent, nullptr, 0, ru[r], rv[r], hk[r],
                                            bad);
        }
        if (WRITE && RECORD) {  // both lists with one block-wide scan
            int ck = 0, ch = 0;
#pragma unroll
            for (int r = 0; r < K; r++) {
                ck += keep[r];
                ch += hk[r];
            }
            unsigned long long ok, oh;
            block_reserve2(&st->kept[it], &st->hooked[it], ck, ch, sw, sbase2, ok, oh);
#pragma unroll
            for (int r = 0; r < K; r++) {
                if (keep[r]) out[ok++] = make_uint2(ru[r], rv[r]);
                if (hk[r]) hooked_list[hbase + oh++] = ru[r] > rv[r] ? ru[r] : rv[r];
            }
        } else if (WRITE) {
            int c = 0;
#pragma unroll
            for (int r = 0; r < K; r++) c += keep[r];
            unsigned long long o = block_reserve(&st->kept[it], c, sw, &sbase);
#pragma unroll
            for (int r = 0; r < K; r++)
                if (keep[r]) out[o++] = make_uint2(ru[r], rv[r]);
        }
    }
    if (bad) set_err(st, kErrInvalidEdge);
}

// labels[v] = root(v) - vo[g(v)]: the minimum local id of v's component
__global__ void __launch_bounds__(kBlock) k_finalize_batch(vid_t *parent, vid_t ntot, const int64_t *__restrict__ vo,
                                                           int G, int32_t *__restrict__ labels,
                                                           const uint32_t *__restrict__ vg) {
    for (long long v = gtid(); v < (long long)ntot; v += gstride()) {
        const int g = graph_advance(vo, G, v, (int)vg[v >> kTileShift]);
        labels[v] = (int32_t)((long long)find_root(parent, (vid_t)v) - vo[g]);
    }
}

template <int U>
void launch_sv_pass_batch_u(int mode, const int32_t *in, long long m, const int64_t *eo, const int64_t *vo, int G,
                            vid_t ntot, vid_t *parent, vid_t *hooked_list, uint2 *out, DevState *st, int it, int grid,
                            cudaStream_t s, int grid_mult, const uint32_t *sch_tg, int regions,
                            unsigned long long *next) {
    auto kf = mode == 0   ? k_sv_pass_batch<0, false, false, U>
              : mode == 5 ? k_sv_pass_batch<0, false, false, U, 1>   // front end, first pass
              : mode == 6 ? k_sv_pass_batch<2, false, false, U, 2>   // front end, second pass
                          : k_sv_pass_batch<2, true, true, U>;
    const bool ordered = regions > 0 && next;
    const long long g = fit_grid((const void *)kf, grid, kBlock) * (!ordered && grid_mult > 0 ? grid_mult : 1);
    if (ordered) cudaMemsetAsync(next, 0, sizeof(unsigned long long), s);
    kf<<<(unsigned)g, kBlock, 0, s>>>(in, m, eo, vo, G, ntot, parent, hooked_list, out, st, it, sch_tg,
                                      ordered ? regions : 0, next);
}

void launch_sv_pass_batch(int mode, const int32_t *in, long long m, const int64_t *eo, const int64_t *vo, int G,
                          vid_t ntot, vid_t *parent, vid_t *hooked_list, uint2 *out, DevState *st, int it, int grid,
                          cudaStream_t s, BatchSchedule sch) {
    if (m <= 0) return;
    const uint32_t *sch_tg = sch.pair_tiles;
    if (sch.unroll == 1)
        launch_sv_pass_batch_u<1>(mode, in, m, eo, vo, G, ntot, parent, hooked_list, out, st, it, grid, s,
                                  sch.grid_mult, sch_tg, sch.sv_regions, sch.queue);
    else if (sch.unroll == 4)
        launch_sv_pass_batch_u<4>(mode, in, m, eo, vo, G, ntot, parent, hooked_list, out, st, it, grid, s,
                                  sch.grid_mult, sch_tg, sch.sv_regions, sch.queue);
    else
        launch_sv_pass_batch_u<2>(mode, in, m, eo, vo, G, ntot, parent, hooked_list, out, st, it, grid, s,
                                  sch.grid_mult, sch_tg, sch.sv_regions, sch.queue);
}

void launch_finalize_batch(vid_t *parent, vid_t ntot, const int64_t *vo, int G, int32_t *labels, int grid,
                           cudaStream_t s, const uint32_t *vertex_tiles) {
    if (ntot == 0) return;
    k_finalize_batch<<<fit_grid((const void *)k_finalize_batch, grid, kBlock), kBlock, 0, s>>>(parent, ntot, vo, G,
                                                                                                labels, vertex_tiles);
}

// ---------------------------------------------------------------------------
// Stream-ordered route (graph-mode cc_labels): the kernels that take the
// host's decisions on the device.

// parent[v] = v, or the BFS component's minimum (DevState::cmin) for visited v
__global__ void __launch_bounds__(kBlock) k_parent_init_st(vid_t *parent, vid_t n, const uint32_t *__restrict__ vis,
                                                           const DevState *st) {
    const vid_t cmin = st->cmin;
    for (long long v = gtid(); v < (long long)n; v += gstride()) {
        vid_t p = (vid_t)v;
        if (cmin < n && vis_test(vis, v)) p = cmin;
        parent[v] = p;
    }
}

// The first SV pass after the BFS over the pairs the BFS left active: the
// caller's list (bfs_list < 0; the T instantiation runs) or ebuf[bfs_list]
// (the uint32 instantiation runs). MODE 1 after one tree (a pair with both
// ends visited is dropped, a visited end stands for cmin); MODE 2 after the
// multi-start BFS, whose trees already point at their minima (one-hop
// gathers). The surviving pairs go to the other buffer, and the SV loop
// continues after this iteration 0.
template <typename T, int MODE>
__global__ void __launch_bounds__(kBlock) k_sv_after_bfs(const T *__restrict__ caller, long long m, const uint2 *eb0,
                                                         const uint2 *eb1, vid_t n, vid_t *parent,
                                                         const uint32_t *__restrict__ vis, vid_t *hooked_list,
                                                         DevState *st) {
    constexpr bool kList = sizeof(T) == 4 && T(-1) > T(0);
    const int list = st->bfs_list;
    if (kList != (list >= 0)) return;
    const T *in = kList ? reinterpret_cast<const T *>(list ? eb1 : eb0) : caller;
    const long long len = kList ? (long long)st->bfs_len : m;
    const int cur0 = list == 0 ? 1 : 0;
    uint2 *out = const_cast<uint2 *>(cur0 ? eb1 : eb0);
    sv_pass_body<T, MODE, true, true>(in, len, n, parent, vis, st->cmin, hooked_list, out, st, 0);
    if (gtid() == 0) {
        st->loop_start_it = 0;
        st->loop_start_cur = cur0;
    }
}

__global__ void k_sv_loop_init_st(DevState *st, int cap, cudaGraphConditionalHandle h) {
    st->loop_cap = cap < kMaxIters ? cap : kMaxIters;
    st->loop_cur = st->loop_start_cur;
    sv_loop_decide(st, st->loop_start_it, h);
}

// Route of Algorithm 2 (policies as CC_ROUTE_*: 0 K-S heuristic, 1 learned,
// 2 forced BFS, 3 forced SV); sets the IF node's condition (when there is a
// BFS branch: has_if). The SV route continues after SV iteration 1, which
// ran speculatively on ebuf0.
__global__ void k_route_decide(DevState *st, cudaGraphConditionalHandle h, int has_if, int policy, int bfs_ok,
                               int opt_cutoff, float min_conf, int have_pred) {
    int route, src;
    if (policy == 3) {
        route = 0;
        src = 2;
    } else if (policy == 2) {
        route = 1;
        src = 2;
    } else if (policy == 1 && have_pred && st->pred_conf >= min_conf) {
        route = st->pred_route;
        src = 1;
    } else {
        route = st->route;
        src = 0;
    }
    if (!bfs_ok) route = 0;
    st->route_taken = route;
    st->route_source = src;
    st->bfs_cutoff = opt_cutoff > 0 ? opt_cutoff : (src == 1 && route == 1 ? st->pred_cutoff : 0);
    st->loop_start_it = 1;
    st->loop_start_cur = 0;
    if (has_if) cudaGraphSetConditional(h, route ? 1u : 0u);
}

// IF condition: the learned prediction is unsure, the exact degree pass and
// the K-S fit run
__global__ void k_pred_unsure(const DevState *st, cudaGraphConditionalHandle h, float min_conf) {
    cudaGraphSetConditional(h, st->pred_conf < min_conf ? 1u : 0u);
}

void launch_parent_init_st(vid_t *parent, vid_t n, const uint32_t *vis, const DevState *st, int grid, cudaStream_t s) {
    if (n == 0) return;
    k_parent_init_st<<<grid, kBlock, 0, s>>>(parent, n, vis, st);
}

template <typename T, int MODE>
void launch_sv_after_bfs_m(const void *caller, long long m, const uint2 *eb0, const uint2 *eb1, vid_t n,
                           vid_t *parent, const uint32_t *vis, vid_t *hooked_list, DevState *st, int grid,
                           cudaStream_t s) {
    auto kc = k_sv_after_bfs<T, MODE>;
    auto kl = k_sv_after_bfs<uint32_t, MODE>;
    kc<<<fit_grid((const void *)kc, grid, kBlock), kBlock, 0, s>>>((const T *)caller, m, eb0, eb1, n, parent, vis,
                                                                     hooked_list, st);
    kl<<<fit_grid((const void *)kl, grid, kBlock), kBlock, 0, s>>>(nullptr, 0, eb0, eb1, n, parent, vis, hooked_list,
                                                                     st);
}

template <typename T>
int launch_sv_after_bfs(const void *caller, long long m, const uint2 *eb0, const uint2 *eb1, vid_t n, vid_t *parent,
                        const uint32_t *vis, vid_t *hooked_list, DevState *st, int grid, cudaStream_t s, bool trees) {
    if (trees) launch_sv_after_bfs_m<T, 2>(caller, m, eb0, eb1, n, parent, vis, hooked_list, st, grid, s);
    else launch_sv_after_bfs_m<T, 1>(caller, m, eb0, eb1, n, parent, vis, hooked_list, st, grid, s);
    return 2;
}
template int launch_sv_after_bfs<int32_t>(const void *, long long, const uint2 *, const uint2 *, vid_t, vid_t *,
                                          const uint32_t *, vid_t *, DevState *, int, cudaStream_t, bool);
template int launch_sv_after_bfs<int64_t>(const void *, long long, const uint2 *, const uint2 *, vid_t, vid_t *,
                                          const uint32_t *, vid_t *, DevState *, int, cudaStream_t, bool);

void launch_sv_loop_init_st(DevState *st, int cap, cudaGraphConditionalHandle h, cudaStream_t s) {
    k_sv_loop_init_st<<<1, 1, 0, s>>>(st, cap, h);
}

void launch_route_decide(DevState *st, const cudaGraphConditionalHandle *h, int policy, int bfs_ok, int opt_cutoff,
                         float min_conf, int have_pred, cudaStream_t s) {
    k_route_decide<<<1, 1, 0, s>>>(st, h ? *h : cudaGraphConditionalHandle(), h ? 1 : 0, policy, bfs_ok, opt_cutoff,
                                   min_conf, have_pred);
}

void launch_pred_unsure(const DevState *st, cudaGraphConditionalHandle h, float min_conf, cudaStream_t s) {
    k_pred_unsure<<<1, 1, 0, s>>>(st, h, min_conf);
}

// ---------------------------------------------------------------------------
// Host launchers

template <typename T>
void launch_sv_pass(int mode, bool write, bool record, const void *in, long long m, vid_t n, vid_t *parent,
                    const uint32_t *vis, vid_t cmin, vid_t *hooked_list, uint2 *out, DevState *st, int it, int grid,
                    cudaStream_t s) {
    const T *e = (const T *)in;
#define SVP(M, W, R)                                                                                  \
    do {                                                                                              \
        auto kf = k_sv_pass<T, M, W, R>;                                                              \
        kf<<<fit_grid((const void *)kf, grid, kBlock), kBlock, 0, s>>>(e, m, n, parent, vis, cmin,    \
                                                                       hooked_list, out, st, it);     \
    } while (0)
    if (mode == 0) {
        if (write) SVP(0, true, false);
        else SVP(0, false, false);
    } else if (mode == 4) {
        SVP(4, false, false);
    } else if (mode == 1) {
        SVP(1, true, true);
    } else if (mode == 2) {
        if (record) SVP(2, true, true);
        else SVP(2, true, false);
    } else {
        SVP(3, true, true);
    }
#undef SVP
}
template void launch_sv_pass<int32_t>(int, bool, bool, const void *, long long, vid_t, vid_t *, const uint32_t *,
                                      vid_t, vid_t *, uint2 *, DevState *, int, int, cudaStream_t);
template void launch_sv_pass<int64_t>(int, bool, bool, const void *, long long, vid_t, vid_t *, const uint32_t *,
                                      vid_t, vid_t *, uint2 *, DevState *, int, int, cudaStream_t);
template void launch_sv_pass<uint32_t>(int, bool, bool, const void *, long long, vid_t, vid_t *, const uint32_t *,
                                       vid_t, vid_t *, uint2 *, DevState *, int, int, cudaStream_t);

// A hook pass of the SV front end over one tile in tstride of the pairs:
// mode 0 with identity parents, mode 2 with every vertex pointing at a root.
template <typename T>
void launch_sv_sample(int mode, const void *in, long long m, vid_t n, vid_t *parent, DevState *st, int tstride,
                      int grid, cudaStream_t s) {
    if (m <= 0) return;
    auto kf = mode == 0 ? k_sv_sample<T, 0> : k_sv_sample<T, 2>;
    kf<<<fit_grid((const void *)kf, grid, kBlock), kBlock, 0, s>>>((const T *)in, m, n, parent, st, tstride);
}
template void launch_sv_sample<int32_t>(int, const void *, long long, vid_t, vid_t *, DevState *, int, int,
                                        cudaStream_t);
template void launch_sv_sample<int64_t>(int, const void *, long long, vid_t, vid_t *, DevState *, int, int,
                                        cudaStream_t);

// The MODE 2 pass with one tile per block (instead of a resident grid that
// strides over the tiles): blocks retire all through the pass, so kernels of
// a higher-priority stream get SMs within a tile's time rather than after
// the whole pass.
template <typename T>
void launch_sv_gather_tiles(const void *in, long long m, vid_t n, vid_t *parent, vid_t *hooked_list, uint2 *out,
                            DevState *st, int it, cudaStream_t s) {
    if (m <= 0) return;
    constexpr int P = PairVec<T>::kPairs;
    const long long tile = (long long)kBlock * PassUnroll<T>::U;
    const long long nvec = m / P;
    long long blocks = (nvec + tile - 1) / tile + (P == 2 && (m & 1) ? 1 : 0);
    if (blocks > 0x7fffffffLL) blocks = 0x7fffffffLL;
    k_sv_pass<T, 2, true, true><<<(unsigned)blocks, kBlock, 0, s>>>((const T *)in, m, n, parent, nullptr, 0, hooked_list,
                                                                    out, st, it);
}
template void launch_sv_gather_tiles<int32_t>(const void *, long long, vid_t, vid_t *, vid_t *, uint2 *, DevState *,
                                              int, cudaStream_t);
template void launch_sv_gather_tiles<int64_t>(const void *, long long, vid_t, vid_t *, vid_t *, uint2 *, DevState *,
                                              int, cudaStream_t);

void launch_shortcut_all(vid_t *parent, vid_t n, DevState *st, int it, int grid, cudaStream_t s) {
    k_shortcut_all<<<fit_grid((const void *)k_shortcut_all, grid, kBlock), kBlock, 0, s>>>(parent, n, st, it);
}

void launch_sv_shortcut(vid_t *parent, const vid_t *hooked_list, DevState *st, int it, int grid, cudaStream_t s) {
    k_sv_shortcut<<<fit_grid((const void *)k_sv_shortcut, grid, kBlock), kBlock, 0, s>>>(parent, hooked_list, st, it);
}

void launch_sv_loop_init(DevState *st, int it0, int cur0, int cap, cudaGraphConditionalHandle h, cudaStream_t s) {
    k_sv_loop_init<<<1, 1, 0, s>>>(st, it0, cur0, cap, h);
}

void launch_sv_loop_body(const uint2 *eb0, const uint2 *eb1, vid_t n, vid_t *parent, vid_t *hooked_list,
                         DevState *st, cudaGraphConditionalHandle h, int grid, cudaStream_t s) {
    k_sv_pass_loop<<<fit_grid((const void *)k_sv_pass_loop, grid, kBlock), kBlock, 0, s>>>(eb0, eb1, n, parent,
                                                                                            hooked_list, st);
    k_sv_shortcut<<<fit_grid((const void *)k_sv_shortcut, grid, kBlock), kBlock, 0, s>>>(parent, hooked_list, st, -1);
    k_sv_loop_step<<<1, 1, 0, s>>>(st, h);
}

void launch_stream_finish(DevState *st, int it, cudaStream_t s) { k_stream_finish<<<1, 1, 0, s>>>(st, it); }

void launch_parent_init(vid_t *parent, vid_t n, const uint32_t *vis, vid_t cmin, int grid, cudaStream_t s) {
    if (n == 0) return;
    k_parent_init<<<grid, kBlock, 0, s>>>(parent, n, vis, cmin);
}

template <typename T>
void launch_finalize(vid_t *parent, vid_t n, void *labels, int grid, cudaStream_t s) {
    if (n == 0) return;
    k_finalize<T><<<fit_grid((const void *)k_finalize<T>, grid, kBlock), kBlock, 0, s>>>(parent, n, (T *)labels);
}
template void launch_finalize<int32_t>(vid_t *, vid_t, void *, int, cudaStream_t);
template void launch_finalize<int64_t>(vid_t *, vid_t, void *, int, cudaStream_t);

}  // namespace ccg

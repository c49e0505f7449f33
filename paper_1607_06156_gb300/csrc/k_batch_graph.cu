// Batched form, stream-ordered (cc_labels_batched): the per-graph route
// prediction and the BFS step of Algorithm 2 for all G graphs, with every
// decision taken on the device.
//
//  k_batch_offsets     checked copies of the caller's offsets: non-decreasing
//                      from 0 to the totals, else the error bit and offsets
//                      that make one graph of everything (no kernel ever
//                      indexes with unchecked offsets)
//  k_batch_sizes       sort keys: the graphs largest first for the fits
//  k_ovf_seek          the next graph whose large degrees overflow the
//                      per-graph fit (a WHILE node runs the single-graph fit
//                      on each, one per iteration)
//  k_ovf_store         that fit's result into the per-graph outputs
//  k_batch_bfs_*       the BFS step of the graphs routed to it: their pairs
//                      compacted as union ids, one edge-list BFS from all
//                      their seeds at once (the graphs are disjoint, so each
//                      search stays in its graph), then every visited vertex
//                      takes its graph's visited minimum as parent
#include "cc_common.cuh"
#include "cc_kernels.h"

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

namespace ccg {

__global__ void __launch_bounds__(1024) k_batch_offsets(const int64_t *__restrict__ eo, const int64_t *__restrict__ vo,
                                                        int G, long long m, long long n, int64_t *eo_v, int64_t *vo_v,
                                                        DevState *st) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = eo[0] != 0 || vo[0] != 0 || eo[G] != m || vo[G] != n;
    __syncthreads();
    for (int g = threadIdx.x; g < G; g += blockDim.x)
        if (eo[g + 1] < eo[g] || vo[g + 1] < vo[g]) bad = 1;
    __syncthreads();
    const int b = bad;
    for (int g = threadIdx.x; g <= G; g += blockDim.x) {
        eo_v[g] = b ? (g == 0 ? 0 : m) : eo[g];
        vo_v[g] = b ? (g == 0 ? 0 : n) : vo[g];
    }
    if (b && threadIdx.x == 0) set_err(st, kErrBadOffsets);
}

__global__ void __launch_bounds__(kBlock) k_batch_sizes(const int64_t *__restrict__ vo, int G, uint32_t *keys,
                                                        int *idx) {
    for (long long g = gtid(); g < G; g += gstride()) {
        keys[g] = (uint32_t)(vo[g + 1] - vo[g]);
        idx[g] = (int)g;
    }
}

// From graph `from` on (first: from 0), the first graph flagged by the
// per-graph fit; the single-graph fit's fields are cleared for it.
__global__ void __launch_bounds__(1024) k_ovf_seek(const int *__restrict__ flag, int G, const int64_t *__restrict__ vo,
                                                   DevState *st, cudaGraphConditionalHandle h, int first) {
    __shared__ int best;
    const int from = first ? 0 : st->batch_g + 1;
    if (threadIdx.x == 0) best = G;
    __syncthreads();
    for (int g = from + threadIdx.x; g < G; g += blockDim.x)
        if (flag[g]) {
            atomicMin(&best, g);
            break;
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int g = best;
        st->batch_g = g;
        st->batch_base = g < G ? vo[g] : 0;
        st->batch_ng = g < G ? vo[g + 1] - vo[g] : 0;
        st->n_ovf = 0;
        st->nd = 0;
        st->ncand = 0;
        st->maxkey = 0;
        st->route = 0;
        for (int i = 0; i < 5; i++) st->ks_out[i] = 0.0;
        cudaGraphSetConditional(h, g < G ? 1u : 0u);
    }
}

__global__ void k_ovf_store(KsBatchOut out, const DevState *st) {
    const int g = st->batch_g;
    out.D[g] = st->ks_out[0];
    out.alpha[g] = st->ks_out[1];
    out.xmin[g] = (long long)st->ks_out[2];
    out.ntail[g] = (long long)st->ks_out[3];
    out.ncand[g] = (long long)st->ks_out[4];
    out.route[g] = st->route;
    out.seedkey[g] = st->maxkey;
}

// pairs of each graph that takes the BFS step (force_all: every graph)
__global__ void __launch_bounds__(kBlock) k_batch_bfs_counts(const int *__restrict__ route,
                                                             const int64_t *__restrict__ eo,
                                                             const int64_t *__restrict__ vo, int G, int force_all,
                                                             unsigned long long *cnt) {
    for (long long g = gtid(); g < G; g += gstride()) {
        const long long mg = eo[g + 1] - eo[g], ng = vo[g + 1] - vo[g];
        cnt[g] = (force_all || route[g]) && mg > 0 && ng > 0 ? (unsigned long long)mg : 0ull;
    }
}

// the BFS step's state; the IF node runs it when any graph takes it
__global__ void k_batch_bfs_plan(const unsigned long long *cnt, const unsigned long long *off, int G, DevState *st,
                                 cudaGraphConditionalHandle h) {
    const unsigned long long total = G > 0 ? off[G - 1] + cnt[G - 1] : 0ull;
    st->bfs_list = 0;
    st->bfs_len = total;
    st->bfs_kept_prev = total;
    st->bfs_level = 0;
    st->bfs_par = 0;
    st->route_taken = 0;
    cudaGraphSetConditional(h, total > 0 ? 1u : 0u);
}

// the pairs of the BFS graphs, as union ids, into out (graph g's at off[g])
__global__ void __launch_bounds__(kBlock) k_batch_bfs_compact(const int32_t *__restrict__ in, long long m,
                                                              const int64_t *__restrict__ eo,
                                                              const int64_t *__restrict__ vo, int G,
                                                              const uint32_t *__restrict__ tg,
                                                              const unsigned long long *__restrict__ cnt,
                                                              const unsigned long long *__restrict__ off, uint2 *out) {
    for (long long k = gtid(); k < m; k += gstride()) {
        const int g = graph_advance(eo, G, k, (int)tg[k >> kTileShift]);
        if (!cnt[g]) continue;
        const long long base = vo[g], ng = vo[g + 1] - base;
        long long u = in[2 * k], v = in[2 * k + 1];
        if (u < 0 || v < 0 || u >= ng || v >= ng) u = v = 0;  // flagged by the degree pass
        out[off[g] + (unsigned long long)(k - eo[g])] = make_uint2((vid_t)(base + u), (vid_t)(base + v));
    }
}

// every BFS graph's seed (its max-degree vertex) into the visited set and the first frontier
__global__ void __launch_bounds__(kBlock) k_batch_bfs_seeds(const unsigned long long *__restrict__ cnt,
                                                            const int64_t *__restrict__ vo,
                                                            const unsigned long long *__restrict__ seedkey, int G,
                                                            uint32_t *vis, uint32_t *cur, DevState *st) {
    unsigned long long seeds = 0;
    for (long long g = gtid(); g < G; g += gstride()) {
        if (!cnt[g]) continue;
        const long long ng = vo[g + 1] - vo[g];
        long long x = (long long)(0xffffffffull - (seedkey[g] & 0xffffffffull));
        if (x >= ng || seedkey[g] == 0) x = 0;
        const unsigned long long v = (unsigned long long)(vo[g] + x);
        atomicOr(&vis[v >> 5], 1u << (v & 31));
        atomicOr(&cur[v >> 5], 1u << (v & 31));
        seeds++;
    }
    if (seeds) {
        atomicAdd(&st->front[0], seeds);
        atomicAdd(reinterpret_cast<unsigned int *>(&st->route_taken), (unsigned int)seeds);
    }
}

// cmin[g] = smallest visited union id of graph g
__global__ void __launch_bounds__(kBlock) k_batch_cmin(const uint32_t *__restrict__ vis, long long n,
                                                       const int64_t *__restrict__ vo, int G,
                                                       const uint32_t *__restrict__ vtg, uint32_t *cmin) {
    const long long nwords = (n + 31) / 32;
    for (long long w = gtid(); w < nwords; w += gstride()) {
        uint32_t b = vis[w];
        while (b) {
            const long long v = w * 32 + __ffs(b) - 1;
            b &= b - 1;
            const int g = graph_advance(vo, G, v, (int)vtg[v >> kTileShift]);
            atomicMin(&cmin[g], (uint32_t)v);
        }
    }
}

// every visited vertex takes its graph's visited minimum as parent (atomicMin keeps the forest)
__global__ void __launch_bounds__(kBlock) k_batch_merge(const uint32_t *__restrict__ vis, long long n,
                                                        const int64_t *__restrict__ vo, int G,
                                                        const uint32_t *__restrict__ vtg,
                                                        const uint32_t *__restrict__ cmin, vid_t *parent) {
    const long long nwords = (n + 31) / 32;
    for (long long w = gtid(); w < nwords; w += gstride()) {
        uint32_t b = vis[w];
        while (b) {
            const long long v = w * 32 + __ffs(b) - 1;
            b &= b - 1;
            const int g = graph_advance(vo, G, v, (int)vtg[v >> kTileShift]);
            atomicMin(&parent[v], cmin[g]);
        }
    }
}

__global__ void k_set_cond(cudaGraphConditionalHandle h, unsigned v) { cudaGraphSetConditional(h, v); }

// ---------------------------------------------------------------------------
void launch_set_cond(cudaGraphConditionalHandle h, unsigned v, cudaStream_t s) { k_set_cond<<<1, 1, 0, s>>>(h, v); }

size_t batch_cub_bytes(int G) {
    size_t a = 0, b = 0;
    cub::DeviceRadixSort::SortPairsDescending(nullptr, a, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                              (const int *)nullptr, (int *)nullptr, G);
    cub::DeviceScan::ExclusiveSum(nullptr, b, (const unsigned long long *)nullptr, (unsigned long long *)nullptr, G);
    return (a > b ? a : b) + 256;
}

void launch_batch_offsets(const int64_t *eo, const int64_t *vo, int G, long long m, long long n, int64_t *eo_v,
                          int64_t *vo_v, DevState *st, cudaStream_t s) {
    k_batch_offsets<<<1, 1024, 0, s>>>(eo, vo, G, m, n, eo_v, vo_v, st);
}

cudaError_t launch_batch_order(const int64_t *vo, int G, uint32_t *keys, uint32_t *keys_sorted, int *idx, int *order,
                               void *tmp, size_t tmp_bytes, int grid, cudaStream_t s) {
    k_batch_sizes<<<grid, kBlock, 0, s>>>(vo, G, keys, idx);
    return cub::DeviceRadixSort::SortPairsDescending(tmp, tmp_bytes, keys, keys_sorted, idx, order, G, 0, 32, s);
}

void launch_ovf_seek(const int *flag, int G, const int64_t *vo, DevState *st, cudaGraphConditionalHandle h, int first,
                     cudaStream_t s) {
    k_ovf_seek<<<1, 1024, 0, s>>>(flag, G, vo, st, h, first);
}

void launch_ovf_store(KsBatchOut out, const DevState *st, cudaStream_t s) { k_ovf_store<<<1, 1, 0, s>>>(out, st); }

cudaError_t launch_batch_bfs_plan(const int *route, const int64_t *eo, const int64_t *vo, int G, int force_all,
                                  unsigned long long *cnt, unsigned long long *off, void *tmp, size_t tmp_bytes,
                                  DevState *st, cudaGraphConditionalHandle h, int grid, cudaStream_t s) {
    k_batch_bfs_counts<<<grid, kBlock, 0, s>>>(route, eo, vo, G, force_all, cnt);
    const cudaError_t e = cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, cnt, off, G, s);
    k_batch_bfs_plan<<<1, 1, 0, s>>>(cnt, off, G, st, h);
    return e;
}

void launch_batch_bfs_start(const int32_t *in, long long m, const int64_t *eo, const int64_t *vo, int G,
                            const uint32_t *tg, const unsigned long long *cnt, const unsigned long long *off,
                            const unsigned long long *seedkey, uint2 *list, uint32_t *vis, uint32_t *cur, DevState *st,
                            int grid, cudaStream_t s) {
    k_batch_bfs_compact<<<grid, kBlock, 0, s>>>(in, m, eo, vo, G, tg, cnt, off, list);
    k_batch_bfs_seeds<<<grid, kBlock, 0, s>>>(cnt, vo, seedkey, G, vis, cur, st);
}

void launch_batch_bfs_finish(const uint32_t *vis, long long n, const int64_t *vo, int G, const uint32_t *vtg,
                             uint32_t *cmin, vid_t *parent, int grid, cudaStream_t s) {
    cudaMemsetAsync(cmin, 0xff, (size_t)G * 4, s);
    k_batch_cmin<<<grid, kBlock, 0, s>>>(vis, n, vo, G, vtg, cmin);
    k_batch_merge<<<grid, kBlock, 0, s>>>(vis, n, vo, G, vtg, cmin, parent);
}

}  // namespace ccg

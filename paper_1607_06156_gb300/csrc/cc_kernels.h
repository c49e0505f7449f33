// Host-side launchers of the engine's kernels (one definition per .cu file).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cc_common.cuh"

namespace ccg {

// Schedule of the batched hook passes: 16-byte vectors per thread per tile
// and blocks per launch as a multiple of the resident count.
struct BatchSchedule {
    int unroll = 2;
    int grid_mult = 1;
    int deg_regions = 1;  // regions of the pairs the degree pass works on side by side
    int sv_regions = 0;   // the hook passes: 0 = grid stride, else regions of the pairs side by side
    unsigned long long *queue = nullptr;  // the hook passes' tile counter (with sv_regions > 0)
    bool front = false;  // SV front end: per-graph sampled hook passes before the first gather pass
    const uint32_t *pair_tiles = nullptr;  // graph of every 2^kTileShift-th pair (launch_tile_graphs), required
};


// launch_cfg.cu: min(grid, blocks of `kernel` resident on the current device at once)
int fit_grid(const void *kernel, int grid, int block, size_t smem = 0);


// Scratch of the K-S fit (device arrays, sized for the distinct degrees).
struct KsScratch {
    uint32_t *xs;                  // distinct degrees >= 1, increasing
    unsigned long long *cnt;       // vertices per distinct degree
    unsigned long long *cum;       // exclusive prefix of cnt (one extra entry: total)
    double *lnx;                   // ln(xs)
    double *Dc, *Ac, *Zc;          // D, alpha and scaled zeta(alpha, xmin) per candidate xmin
    float *Df;                     // fp32 screen maximum per candidate
    unsigned long long *chunk_nz;  // per-chunk distinct counts, then offsets
    unsigned long long *chunk_mass;
    unsigned long long cap;        // entries of xs/cnt/lnx/Dc/Ac (cum holds cap + 1)
};

// Scratch of the vertex-block partitioned CSR build (k_bucket.cu).
struct BucketScratch {
    unsigned long long *fill;     // [vertex blocks] entries reserved so far in each block's CSR range
    unsigned long long *queue;    // the placement's tile counter
};

// k_bucket.cu
int bucket_count_for(vid_t n);
int bucket_max();
template <typename T>
void launch_csr_bucketed(const void *edges, long long m, vid_t n, const uint32_t *row_ptr, uint32_t *cursor,
                         vid_t *col, BucketScratch bs, unsigned long long *entries, DevState *st, int grid,
                         cudaStream_t s);
cudaError_t csr_kernels_setup();

// Scratch of the sampled route features (k_mlp.cu).
struct FeatScratch {
    uint32_t *sdeg;     // [n/16 + 1] degrees of the sampled vertices
    unsigned *counts;   // [64] log2-bucket counts
    uint32_t *vis, *f0, *f1;  // [n/32 + 1] probe bitmaps
};

// k_mlp.cu
int mlp_num_params();
void mlp_forward(const float *P, const float *X, int B, float *act, cudaStream_t s);
void mlp_backward(const float *P, const float *X, const int *y, const float *t, const float *w, int B, float lam,
                  const float *act, float *G, float *scratch, float *loss, cudaStream_t s);
void mlp_adam(float *P, const float *G, float *M, float *V, int count, float lr, float b1, float b2, float eps, int t,
              cudaStream_t s);
template <typename T>
void launch_route_features(const void *edges, long long m, vid_t n, FeatScratch fs, DevState *st, float *x, int grid,
                           cudaStream_t s);

// k_degree.cu
template <typename T>
void launch_degree(const void *edges, long long m, vid_t n, uint32_t *deg, DevState *st, int grid, cudaStream_t s);
bool degree_uses_hubs(long long m);
template <typename T>
void launch_degree_hubs(const void *edges, long long m, vid_t n, uint32_t *deg, unsigned *scratch, DevState *st,
                        int grid, int num_sms, cudaStream_t s);
size_t degree_hubs_scratch_bytes();
// the hub-aware pass in two parts, for pairs that arrive in chunks: the hub
// table from the first degree_hub_prefix() pairs, then any number of counts
long long degree_hub_prefix();
template <typename T>
void launch_degree_hub_prefix(const void *edges, vid_t n, uint32_t *deg, unsigned *scratch, DevState *st, int grid,
                              cudaStream_t s);
template <typename T>
void launch_degree_hub_count(const void *edges, long long m, vid_t n, uint32_t *deg, const unsigned *scratch,
                             DevState *st, int num_sms, cudaStream_t s);
void launch_hist(const uint32_t *deg, vid_t n, uint32_t *hist, uint32_t *ovf, unsigned long long ovf_cap,
                 DevState *st, int grid, cudaStream_t s);
void launch_ks(const uint32_t *hist, const uint32_t *ovf, unsigned long long ovf_cap, KsScratch ks, DevState *st,
               long long min_tail, long long min_distinct, double min_span, double tau, long long nd_bound, int grid,
               cudaStream_t s);
int ks_num_chunks();
void launch_hist_widen(const uint32_t *hist, const uint32_t *ovf, unsigned long long ovf_cap, const DevState *st,
                       uint64_t *out, long long len, int grid, cudaStream_t s);
void launch_hist_narrow(const uint64_t *in, long long len, uint32_t *hist, DevState *st, int grid, cudaStream_t s);

// Stream-ordered route (graph-mode cc_labels): decisions taken on the device.
// launch_*_level return the kernels they launched (one WHILE iteration).
void launch_bfsg_init(const uint32_t *row_ptr, vid_t n, uint32_t *vis, vid_t *q0, DevState *st,
                      cudaGraphConditionalHandle h, cudaStream_t s);
int launch_bfsg_level(vid_t n, unsigned long long total_edges, const uint32_t *row_ptr, const vid_t *col, uint32_t *vis,
                      vid_t *q0, vid_t *q1, uint32_t *b0, uint32_t *b1, uint32_t *dq, uint32_t *off,
                      unsigned long long *tsum, DevState *st, cudaGraphConditionalHandle h, int grid, cudaStream_t s);
void launch_ebfsg_init(uint32_t *vis, uint32_t *b0, vid_t n, long long m, DevState *st, cudaGraphConditionalHandle h,
                       cudaStream_t s);
// own: the multi-start form's owner array (null: one tree); has_h = false
// runs the level without a WHILE node (the host-driven loop)
template <typename T>
int launch_ebfsg_level(const void *caller, long long m, const uint2 *eb0, const uint2 *eb1, vid_t n, uint32_t *vis,
                       uint32_t *b0, uint32_t *b1, DevState *st, cudaGraphConditionalHandle h, int grid,
                       cudaStream_t s, uint32_t *own = nullptr, bool has_h = true);
// Multi-start BFS: the bitmaps, owners (kNoOwner), tree minima and level
// counters cleared, the starts of k ranges seeded from deg (one block per
// range) and the BFS state set; h (or null) gets "level 0 runs". Then
// launch_ebfsg_level with own, and launch_mbfs_finish: the tree minima and
// parent[v] = the minimum of v's tree (v if no tree reached it).
void launch_mbfs_start(const uint32_t *deg, vid_t n, long long m, int k, uint32_t *vis, uint32_t *b0, uint32_t *own,
                       uint32_t *tmin, DevState *st, const cudaGraphConditionalHandle *h, cudaStream_t s);
void launch_mbfs_finish(const uint32_t *own, uint32_t *tmin, vid_t n, vid_t *parent, int grid, cudaStream_t s);
void launch_parent_init_st(vid_t *parent, vid_t n, const uint32_t *vis, const DevState *st, int grid, cudaStream_t s);
template <typename T>
// trees: after the multi-start BFS (parents already point at the tree minima)
int launch_sv_after_bfs(const void *caller, long long m, const uint2 *eb0, const uint2 *eb1, vid_t n, vid_t *parent,
                        const uint32_t *vis, vid_t *hooked_list, DevState *st, int grid, cudaStream_t s,
                        bool trees = false);
void launch_sv_loop_init_st(DevState *st, int cap, cudaGraphConditionalHandle h, cudaStream_t s);
// h: the IF node's handle, or null when there is no BFS branch
void launch_route_decide(DevState *st, const cudaGraphConditionalHandle *h, int policy, int bfs_ok, int opt_cutoff,
                         float min_conf, int have_pred, cudaStream_t s);
void launch_pred_unsure(const DevState *st, cudaGraphConditionalHandle h, float min_conf, cudaStream_t s);

// k_degree_part.cu: degree pass for n > 2^25 (counts out of L2): the
// endpoints partitioned into windows of 2^23 vertices (bulk copies into
// shared memory), then counted window by window with L2 atomics (one launch
// per window: degree_part_buckets(n) + 1 launches).
// scratch: degree_part_scratch_bytes; grid: blocks of the window count pass.
// hook: the parent array with every vertex its own root, or null; with it the
// window pass also hooks every pair (atomicMin(parent[max], min), the first
// SV hook pass) while the window's parents are in L2.
int degree_part_buckets(vid_t n);
bool degree_part_ok(vid_t n, long long m);
size_t degree_part_scratch_bytes(vid_t n, long long m, bool hook);
template <typename T>
void launch_degree_partitioned(const void *edges, long long m, vid_t n, uint32_t *deg, vid_t *hook, void *scratch,
                               DevState *st, int num_sms, int grid, cudaStream_t s);
// The same for 2^20 <= n <= 2^24 with windows of at most 2^15 vertices whose
// counts stay in shared memory (16-bit entries; two launches). Scratch:
// degree_smem_scratch_bytes.
bool degree_smem_ok(vid_t n, long long m);
size_t degree_smem_scratch_bytes(vid_t n, long long m);
template <typename T>
void launch_degree_smem(const void *edges, long long m, vid_t n, uint32_t *deg, void *scratch, DevState *st,
                        int num_sms, cudaStream_t s);
// k_batch_degree.cu: the batched degree pass (with the first hook pass when
// `hook`) counted in shared-memory windows of 4,096 vertices per graph; four
// launches. Scratch: batch_win_scratch_bytes(m, n, G) bytes; tile_pairs: the
// graph of every 2^kTileShift-th pair of the batch (launch_tile_graphs).
bool degree_batch_win_ok(long long m, long long n);
size_t batch_win_scratch_bytes(long long m, long long n, int G);
void launch_degree_batch_win(const int32_t *in, long long m, const int64_t *eo, const int64_t *vo, int G, long long n,
                             const uint32_t *tile_pairs, uint32_t *deg, DevState *st, void *scratch, int num_sms,
                             cudaStream_t s, vid_t *hook);
cudaError_t batch_win_setup();
cudaError_t degree_part_setup();
cudaError_t degree_hubs_setup();  // dynamic shared memory of the hub-aware degree pass

// k_tuple_sv.cu: the paper's sort-based SV (Section 3.1) as an ablation, with
// the exclusion of completed partitions (Section 3.1.4).
// Tuple buffers hold cap >= n + 2m + n entries (the tuples and the extras).
struct TupleSvBufs {
    uint32_t *t32[4];              // tuple words: two hold the tuples (r, p | extra bit), two are scratch
    unsigned long long *v0, *v1;   // partition-grouped values (double buffer), then the packed tuples
    uint32_t *val, *val2;          // reduce-by-key values
    uint32_t *uniq, *agg;          // reduce-by-key outputs
    uint32_t *dense;               // [n] reduced value by key
    uint32_t *pc;                  // [n] vertex: all its tuples share one partition
    uint32_t *done;                // [n] partition: completed
    unsigned long long *counters;  // [4]: runs, moved, tuples kept
    void *temp;
    size_t temp_bytes;
    long long cap;
    int num_sms;
};
size_t tuple_sv_temp_bytes(long long cap, vid_t n);
// 0: labels written; 1: CUDA error or capacity; 2: no convergence within max_iters
// active_out[i - 1] (i <= active_cap): tuples in the working set entering iteration i
// sort_ms (optional): the summed time of the radix sorts, *sorts their number
template <typename T>
int tuple_sv_run(const void *edges, long long m, vid_t n, void *labels, TupleSvBufs b, DevState *st, int max_iters,
                 int *iters_out, long long *active_out, int active_cap, float *sort_ms, int *sorts, cudaStream_t s);

// k_sv.cu
template <typename T>
void launch_sv_pass(int mode, bool write, bool record, const void *in, long long m, vid_t n, vid_t *parent,
                    const uint32_t *vis, vid_t cmin, vid_t *hooked_list, uint2 *out, DevState *st, int it, int grid,
                    cudaStream_t s);
// hook pass (mode 0 or 2, nothing recorded) over one tile in tstride of the pairs
template <typename T>
void launch_sv_sample(int mode, const void *in, long long m, vid_t n, vid_t *parent, DevState *st, int tstride,
                      int grid, cudaStream_t s);
// MODE 2 with record and write, one tile of pairs per block
template <typename T>
void launch_sv_gather_tiles(const void *in, long long m, vid_t n, vid_t *parent, vid_t *hooked_list, uint2 *out,
                            DevState *st, int it, cudaStream_t s);
void launch_shortcut_all(vid_t *parent, vid_t n, DevState *st, int it, int grid, cudaStream_t s);
// mode 0: first hook pass (identity parents); 2: gather pass with the next
// list and the hooked roots; 5 / 6: the SV front end's first (mode 0 over
// every tile of the graphs that are not sampled and the sampled tiles of the
// others) and second (one-hop gathers over the sampled tiles) hook passes
void launch_sv_pass_batch(int mode, const int32_t *in, long long m, const int64_t *eo, const int64_t *vo, int G,
                          vid_t ntot, vid_t *parent, vid_t *hooked_list, uint2 *out, DevState *st, int it, int grid,
                          cudaStream_t s, BatchSchedule sch = BatchSchedule());
void launch_finalize_batch(vid_t *parent, vid_t ntot, const int64_t *vo, int G, int32_t *labels, int grid,
                           cudaStream_t s,
                           const uint32_t *vertex_tiles);

void launch_sv_shortcut(vid_t *parent, const vid_t *hooked_list, DevState *st, int it, int grid, cudaStream_t s);
void launch_stream_finish(DevState *st, int it, cudaStream_t s);
// device-driven loop: init before a WHILE node on handle h, body inside it
void launch_sv_loop_init(DevState *st, int it0, int cur0, int cap, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_sv_loop_body(const uint2 *eb0, const uint2 *eb1, vid_t n, vid_t *parent, vid_t *hooked_list,
                         DevState *st, cudaGraphConditionalHandle h, int grid, cudaStream_t s);
void launch_parent_init(vid_t *parent, vid_t n, const uint32_t *vis, vid_t cmin, int grid, cudaStream_t s);
template <typename T>
void launch_finalize(vid_t *parent, vid_t n, void *labels, int grid, cudaStream_t s);

// k_bfs.cu
void launch_scan_u32(const uint32_t *in, long long len, uint32_t *out, uint32_t *out_copy, unsigned long long *tsum,
                     unsigned long long *total_dev, uint32_t *total_u32, cudaStream_t s);
long long scan_num_tiles(long long len);
template <typename T>
void launch_csr_scatter(const void *edges, long long m, vid_t n, uint32_t *cursor, vid_t *col, int grid,
                        cudaStream_t s);
void launch_bfs_init(const uint32_t *row_ptr, vid_t n, uint32_t *vis, vid_t *queue, DevState *st, cudaStream_t s);
void launch_front_degrees(const vid_t *queue, long long f, const uint32_t *row_ptr, uint32_t *dq, int grid,
                          cudaStream_t s);
void launch_bfs_topdown(const vid_t *queue, long long f, const uint32_t *off, long long total, const uint32_t *row_ptr,
                        const vid_t *col, uint32_t *vis, vid_t *next, DevState *st, int level, int grid,
                        cudaStream_t s);
void launch_bfs_bottomup(vid_t n, const uint32_t *row_ptr, const vid_t *col, const uint32_t *fb, uint32_t *vis,
                         uint32_t *nb, DevState *st, int level, int grid, cudaStream_t s);
void launch_queue_to_bitmap(const vid_t *queue, long long f, uint32_t *bm, int grid, cudaStream_t s);
void launch_bitmap_to_queue(const uint32_t *bm, long long nwords, vid_t *queue, unsigned long long *count, int grid,
                            cudaStream_t s);
void launch_first_visited(const uint32_t *vis, long long nwords, DevState *st, int grid, cudaStream_t s);
void launch_popcount(const uint32_t *bm, long long nwords, unsigned long long *out, int grid, cudaStream_t s);
template <typename T>
void launch_bfs_edges(bool write, const void *in, long long m, vid_t n, uint32_t *vis, const uint32_t *cur,
                      uint32_t *next, uint2 *out, DevState *st, int level, int grid, cudaStream_t s);
void launch_edge_bfs_seed(uint32_t *vis, uint32_t *cur, vid_t n, const unsigned long long *key, DevState *st,
                          cudaStream_t s);

}  // namespace ccg

#include <cuda_bf16.h>
namespace ccg {
void mlp_prepare_inference(const float *P, __nv_bfloat16 *Wb, float *bias, cudaStream_t s);
void mlp_infer(const __nv_bfloat16 *Wb, const float *bias, const float *x, DevState *st, cudaStream_t s);
// k_probe.cu
void launch_l2_probe(int kind, uint32_t *table, uint32_t mask, long long ops, uint32_t *sink, int grid,
                     cudaStream_t s);

// k_batch_route.cu: per-graph route prediction of the batched form
struct KsBatchScratch {  // per block: ks_batch_entries() of each (cum: one more)
    uint32_t *xs;
    unsigned long long *cnt, *cum;
    double *lnx, *Dc, *Ac, *Zc;
};
struct KsBatchOut {  // per graph
    double *D, *alpha;
    long long *xmin, *ntail, *ncand;
    int *route, *overflow;
    unsigned long long *seedkey;  // (degree << 32) | (0xffffffff - local id) of the max-degree vertex
};
size_t ks_batch_entries();
// next: a device counter the blocks take tiles from (zeroed here); regions:
// contiguous regions of the pairs worked on side by side, each in order;
// hook: the parent array with every vertex its own root, to apply the first
// SV hook pass (atomicMin(parent[max], min)) in the same pass, or null
void launch_degree_batch(const int32_t *in, long long m, const int64_t *eo, const int64_t *vo, int G, uint32_t *deg,
                         DevState *st, int grid, unsigned long long *next, int regions, cudaStream_t s,
                         vid_t *hook = nullptr);
// out[k] = the graph holding item k << kTileShift of the offsets `off` (G + 1 entries), k < (count >> kTileShift) + 1
void launch_tile_graphs(const int64_t *off, int G, long long count, uint32_t *out, int grid, cudaStream_t s);
// order (device, G graph numbers, largest first) and next (device counter) may
// both be null: then block b takes graphs b, b + blocks, ...
void launch_ks_batch(const uint32_t *deg, const int64_t *vo, int G, KsBatchScratch sc, KsBatchOut out,
                     long long min_tail, long long min_distinct, double min_span, double tau, int blocks,
                     const int *order, int *next, cudaStream_t s);
// one graph (n vertices, degrees in deg) through the per-graph fit; results into DevState
// (ks_out, ncand, route, maxkey); vo: 2 int64 of device scratch; hist_scratch: small_hist_words()
// words (8-byte aligned) for a grid-wide histogram, or null (the fit block builds it)
size_t small_hist_words();
void launch_fit_one(const uint32_t *deg, long long n, int64_t *vo, KsBatchScratch sc, KsBatchOut out, DevState *st,
                    long long min_tail, long long min_distinct, double min_span, double tau, uint32_t *hist_scratch,
                    int grid, cudaStream_t s);
void launch_merge_visited(const uint32_t *vis, long long ng, long long base, const DevState *st, vid_t *parent,
                          int grid, cudaStream_t s);

// k_batch_graph.cu: the batched form's prediction and BFS step on the device.
void launch_hist_slice(const uint32_t *deg, uint32_t *hist, uint32_t *ovf, unsigned long long ovf_cap, DevState *st,
                       int grid, cudaStream_t s);
size_t batch_cub_bytes(int G);
void launch_set_cond(cudaGraphConditionalHandle h, unsigned v, cudaStream_t s);
void launch_batch_offsets(const int64_t *eo, const int64_t *vo, int G, long long m, long long n, int64_t *eo_v,
                          int64_t *vo_v, DevState *st, cudaStream_t s);
cudaError_t launch_batch_order(const int64_t *vo, int G, uint32_t *keys, uint32_t *keys_sorted, int *idx, int *order,
                               void *tmp, size_t tmp_bytes, int grid, cudaStream_t s);
void launch_ovf_seek(const int *flag, int G, const int64_t *vo, DevState *st, cudaGraphConditionalHandle h, int first,
                     cudaStream_t s);
void launch_ovf_store(KsBatchOut out, const DevState *st, cudaStream_t s);
cudaError_t launch_batch_bfs_plan(const int *route, const int64_t *eo, const int64_t *vo, int G, int force_all,
                                  unsigned long long *cnt, unsigned long long *off, void *tmp, size_t tmp_bytes,
                                  DevState *st, cudaGraphConditionalHandle h, int grid, cudaStream_t s);
void launch_batch_bfs_start(const int32_t *in, long long m, const int64_t *eo, const int64_t *vo, int G,
                            const uint32_t *tg, const unsigned long long *cnt, const unsigned long long *off,
                            const unsigned long long *seedkey, uint2 *list, uint32_t *vis, uint32_t *cur, DevState *st,
                            int grid, cudaStream_t s);
void launch_batch_bfs_finish(const uint32_t *vis, long long n, const int64_t *vo, int G, const uint32_t *vtg,
                             uint32_t *cmin, vid_t *parent, int grid, cudaStream_t s);

}  // namespace ccg

// C ABI and host orchestration of the hybrid connected-components route
// (Algorithm 2, Section 3.2): degree distribution -> K-S prediction ->
// optional BFS from the max-degree vertex with the visited pairs filtered ->
// Shiloach-Vishkin iterations -> labels. Declared in include/cc_gb300.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/cc_gb300.h"
#include "cc_common.cuh"
#include "cc_kernels.h"

using namespace ccg;

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

enum Ev { EV_START, EV_DEGREE, EV_PREDICT, EV_CSR, EV_BFS, EV_SV, EV_END, EV_COUNT };

// Byte offsets in the context's small counters buffer.
constexpr size_t kCtrBfs = 0;           // BFS visited counts (two 64-bit words)
constexpr size_t kCtrSmallFitVo = 256;  // vertex offsets {0, n} of the one-graph fit (two int64)
constexpr size_t kCtrKsQueue = 1024;    // next graph of the batched fits (int)
constexpr size_t kCtrTileQueue = 1088;  // next tile of the batched degree pass (64-bit)
constexpr size_t kCtrCsrQueue = 1096;   // next tile of the CSR placement (64-bit)
constexpr size_t kCtrSvQueue = 1104;    // next tile of a batched hook pass in region order (64-bit)
constexpr size_t kCountersBytes = 4096;
template <typename P> P *counter_at(Buf &b, size_t off) { return reinterpret_cast<P *>(static_cast<char *>(b.p) + off); }

}  // namespace

struct cc_ctx {
    int device = 0;
    cc_options opt{};
    int num_sms = 0;
    int grid = 0;  // blocks for grid-stride kernels
    // SV / degree workspace
    size_t n_cap = 0, m_cap = 0;
    // workspace of cc_labels_tuple_sv (the sort-based SV of Algorithm 1)
    Buf tsv_t32[4], tsv_v0, tsv_v1, tsv_val, tsv_val2, tsv_uniq, tsv_agg, tsv_dense, tsv_pc, tsv_done, tsv_temp,
        tsv_cnt;
    long long tsv_cap = 0;
    Buf deg, parent, hooked, ebuf0, ebuf1, hist, ovf, ks_xs, ks_cnt, ks_cum, ks_lnx, ks_Dc, ks_Ac, ks_Zc, ks_Df, chunk_nz,
        chunk_mass, st, bk_off;
    Buf dpart;  // endpoints partitioned into vertex windows (degree pass of graphs with n > 2^25)
    Buf bwin;   // the batched degree pass's window tables and regions
    Buf bfs_own, bfs_tmin;  // multi-start BFS: the tree of every vertex, the minimum of every tree
    unsigned long long ovf_cap = 0, ks_cap = 0;
    // BFS workspace
    size_t bn_cap = 0, bm_cap = 0;
    Buf row_ptr, col, vis, fb, nb, q0, q1, dq, off, tsum, counters, csr_entries;
    // learned route predictor
    size_t f_cap = 0;
    Buf f_sdeg, f_counts, f_vis, f_f0, f_f1, f_x, pred_wb, pred_bias, pred_tmp;
    bool have_pred = false;
    double pred_min_conf = 0.75;
    // host side
    DevState *h_st = nullptr;  // pinned mirror of the device state
    cudaEvent_t ev[EV_COUNT] = {};
    bool ev_used[EV_COUNT] = {};
    cudaStream_t last_stream = nullptr;
    cc_stats stats{};
    cc_status last_status = CC_OK;
    int alloc_fail_pending = 0;
    // per-kernel-class event timing (options.profile)
    struct ProfRec {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> evpool;
    size_t evpool_used = 0;
    std::vector<ProfRec> prof;
    // captured SV graphs (device-driven loop), one per entry point, keyed by their arguments
    struct GraphKey {
        long long n, m, G;
        const void *edges, *eo, *vo, *labels, *parent, *hooked, *eb0, *eb1, *st;
        int kind, cap, grid, pad;
    };
    struct LoopGraph {
        cudaGraphExec_t exec = nullptr;
        GraphKey key{};
    };
    LoopGraph g_single, g_batch;
    cudaStream_t cap_s = nullptr, cap_s2 = nullptr, cap_s3 = nullptr;  // private capture streams
    // stream-ordered cc_labels: the whole route as one cached graph, keyed by
    // its arguments, workspace and options, with the host-side facts that
    // turn the device state into statistics
    struct RouteGraph {
        cudaGraphExec_t exec = nullptr;
        std::vector<unsigned char> key;
        long long static_launches = 0;  // kernels outside the conditional bodies
        long long bfs_launches = 0;     // kernels of the BFS branch outside its level loop
        long long unsure_launches = 0;  // kernels of the learned policy's exact-prediction branch
        int level_launches = 0;         // kernels per BFS level
        int sample_stride = 1;          // SV front end stride
        bool edge_bfs = false;          // the BFS branch is the edge-list BFS
        bool batched = false;           // the batched form (route = graphs that took the BFS step)
        int batch_unroll = 0, batch_grid_mult = 0, batch_deg_regions = 0, batch_sv_regions = 0;  // its schedule
        int degree_form = 0;            // the exact degree pass captured (cc_stats.degree_form)
    } g_route;
    RouteGraph g_capture;               // the same facts for a call captured into the caller's graph
    const RouteGraph *rg_last = nullptr; // the facts of the last graph-mode call
    cudaEvent_t ev_done = nullptr;      // after the device status word of the last graph-mode call
    bool async_outstanding = false;     // that call's status word has not been reported yet
    bool graph_last = false;            // the last labelling call ran the graph path
    bool capturing = false;             // enqueueing into the caller's capture: no allocation
    // side stream of the speculative first SV pass, with its fork and join events
    cudaStream_t side_s = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // highest-priority stream of the K-S fit while the speculative pass runs, with its join event
    cudaStream_t fit_s = nullptr;
    cudaEvent_t ev_fit = nullptr;
    // host-input entry point: device copies of the pairs and labels, the copy
    // stream and one event per copied chunk
    Buf hedges, hlabels;
    cudaStream_t copy_s = nullptr;
    std::vector<cudaEvent_t> ev_chunk;
    // per-graph route prediction of the batched form: block scratch, per-graph outputs
    Buf kb_xs, kb_cnt, kb_cum, kb_lnx, kb_Dc, kb_Ac, kb_Zc, kb_D, kb_alpha, kb_xmin, kb_ntail, kb_ncand, kb_route,
        kb_ovf, kb_seed, kb_order;
    int kb_blocks = 0;
    // tuned schedules of the batched hook passes, per shape (log2 pairs << 8 | log2 graphs)
    std::vector<std::pair<int, BatchSchedule>> batch_tuned;
    // graph of every 2^kTileShift-th pair and vertex of the current batch
    Buf tile_pairs, tile_verts;
    // stream-ordered batched form: checked offsets, the fit order, the BFS step's
    // per-graph pair counts / offsets / visited minima, CUB scratch
    Buf bo_e, bo_v, kb_keys, kb_keys2, kb_idx, kb_rcnt, kb_roff, kb_cmin, kb_cub;
    RouteGraph g_batch_route;
};

namespace {

cc_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CC_OK;
    if (e == cudaErrorMemoryAllocation) return CC_ERR_OOM;
    return CC_ERR_CUDA;
}

#define CC_TRY(expr)                             \
    do {                                         \
        cc_status _s = (expr);                   \
        if (_s != CC_OK) return _s;              \
    } while (0)
#define CU_TRY(expr) CC_TRY(cuda_status(expr))

cc_status buf_reserve(cc_ctx *ctx, Buf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return CC_OK;
    // inside the caller's stream capture the workspace must already be large enough
    if (ctx->capturing) return CC_ERR_UNSUPPORTED;
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    if (ctx->alloc_fail_pending) {
        ctx->alloc_fail_pending = 0;
        return CC_ERR_OOM;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return CC_ERR_OOM;
    }
    b.bytes = bytes;
    return CC_OK;
}

void buf_free(Buf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

size_t round4(size_t x) { return (x + 3) & ~(size_t)3; }

// The vertex-block partitioned CSR build handles up to 1024 blocks of 2^15
// vertices; small inputs keep the direct scatter.
bool bucketed_ok(size_t n, size_t m) {
    return n > 0 && bucket_count_for((vid_t)(n < 0xffffffffULL ? n : 0xfffffffeULL)) <= bucket_max() &&
           m >= ((size_t)1 << 20);
}

cc_status ensure_sv(cc_ctx *ctx, size_t n, size_t m) {
    if (n <= ctx->n_cap && m <= ctx->m_cap && ctx->st.p) return CC_OK;
    const size_t N = n > ctx->n_cap ? n : ctx->n_cap, M = m > ctx->m_cap ? m : ctx->m_cap;
    CC_TRY(buf_reserve(ctx, ctx->deg, round4(N + 4) * 4));
    CC_TRY(buf_reserve(ctx, ctx->parent, round4(N + 4) * 4));
    CC_TRY(buf_reserve(ctx, ctx->hooked, round4(N + 4) * 4));
    CC_TRY(buf_reserve(ctx, ctx->ebuf0, (M + 4) * 8));
    CC_TRY(buf_reserve(ctx, ctx->ebuf1, (M + 4) * 8));
    CC_TRY(buf_reserve(ctx, ctx->hist, (size_t)kHistDense * 4));
    ctx->ovf_cap = 2 * (unsigned long long)M / kHistDense + 2;
    CC_TRY(buf_reserve(ctx, ctx->ovf, ctx->ovf_cap * 4));
    const size_t nd = (N < (size_t)kHistDense + 4096 ? N : (size_t)kHistDense + 4096) + 2;
    ctx->ks_cap = nd - 1;
    CC_TRY(buf_reserve(ctx, ctx->ks_xs, nd * 4));
    CC_TRY(buf_reserve(ctx, ctx->ks_cnt, nd * 8));
    CC_TRY(buf_reserve(ctx, ctx->ks_cum, nd * 8));
    CC_TRY(buf_reserve(ctx, ctx->ks_lnx, nd * 8));
    CC_TRY(buf_reserve(ctx, ctx->ks_Dc, nd * 8));
    CC_TRY(buf_reserve(ctx, ctx->ks_Ac, nd * 8));
    CC_TRY(buf_reserve(ctx, ctx->ks_Zc, nd * 8));
    CC_TRY(buf_reserve(ctx, ctx->ks_Df, nd * 4));
    CC_TRY(buf_reserve(ctx, ctx->chunk_nz, (size_t)(ks_num_chunks() + 1) * 8));
    CC_TRY(buf_reserve(ctx, ctx->chunk_mass, (size_t)(ks_num_chunks() + 1) * 8));
    CC_TRY(buf_reserve(ctx, ctx->st, sizeof(DevState)));
    // small device counters (byte offsets kCtr*)
    CC_TRY(buf_reserve(ctx, ctx->counters, kCountersBytes));
    CC_TRY(buf_reserve(ctx, ctx->bk_off, (size_t)(bucket_max() + 2) * 8));
    if (degree_part_ok((vid_t)(N < 0xffffffffULL ? N : 0xfffffffeULL), (long long)M))
        CC_TRY(buf_reserve(ctx, ctx->dpart, degree_part_scratch_bytes((vid_t)N, (long long)M, true)));
    ctx->n_cap = N;
    ctx->m_cap = M;
    return CC_OK;
}

cc_status ensure_bfs(cc_ctx *ctx, size_t n, size_t m) {
    if (n <= ctx->bn_cap && m <= ctx->bm_cap && ctx->row_ptr.p) return CC_OK;
    const size_t N = n > ctx->bn_cap ? n : ctx->bn_cap, M = m > ctx->bm_cap ? m : ctx->bm_cap;
    const size_t words = (N + 31) / 32 + 4;
    CC_TRY(buf_reserve(ctx, ctx->row_ptr, round4(N + 8) * 4));
    CC_TRY(buf_reserve(ctx, ctx->col, (2 * M + 4) * 4));
    CC_TRY(buf_reserve(ctx, ctx->vis, words * 4));
    CC_TRY(buf_reserve(ctx, ctx->fb, words * 4));
    CC_TRY(buf_reserve(ctx, ctx->nb, words * 4));
    CC_TRY(buf_reserve(ctx, ctx->q0, (N + 4) * 4));
    CC_TRY(buf_reserve(ctx, ctx->q1, (N + 4) * 4));
    CC_TRY(buf_reserve(ctx, ctx->dq, (N + 4) * 4));
    CC_TRY(buf_reserve(ctx, ctx->off, (N + 8) * 4));
    CC_TRY(buf_reserve(ctx, ctx->tsum, (size_t)(scan_num_tiles((long long)N + 2) + 4) * 8));
    if (bucketed_ok(N, M)) CC_TRY(buf_reserve(ctx, ctx->csr_entries, (2 * M + 4) * 8));
    ctx->bn_cap = N;
    ctx->bm_cap = M;
    return CC_OK;
}

template <typename P>
P *as(const Buf &b) {
    return reinterpret_cast<P *>(b.p);
}

cc_status ensure_feat(cc_ctx *ctx, size_t n) {
    if (n <= ctx->f_cap && ctx->f_x.p) return CC_OK;
    const size_t N = n > ctx->f_cap ? n : ctx->f_cap;
    const size_t words = (N + 31) / 32 + 4;
    CC_TRY(buf_reserve(ctx, ctx->f_sdeg, ((N + 15) / 16 + 4) * 4));
    CC_TRY(buf_reserve(ctx, ctx->f_counts, 64 * 4));
    CC_TRY(buf_reserve(ctx, ctx->f_vis, words * 4));
    CC_TRY(buf_reserve(ctx, ctx->f_f0, words * 4));
    CC_TRY(buf_reserve(ctx, ctx->f_f1, words * 4));
    CC_TRY(buf_reserve(ctx, ctx->f_x, 128 * 4));
    ctx->f_cap = N;
    return CC_OK;
}

// The multi-start BFS runs on the K-S heuristic and forced routes, which
// count the exact degrees its starts are chosen from (the learned route
// keeps its single sampled hub).
bool multi_start(const cc_ctx *ctx) {
    return ctx->opt.bfs_starts > 1 && !(ctx->opt.route_policy == CC_ROUTE_LEARNED && ctx->have_pred);
}

cc_status ensure_mbfs(cc_ctx *ctx, size_t n) {
    CC_TRY(ensure_feat(ctx, n));
    CC_TRY(buf_reserve(ctx, ctx->bfs_own, (n + 4) * 4));
    CC_TRY(buf_reserve(ctx, ctx->bfs_tmin, (size_t)kMaxBfsStarts * 4));
    return CC_OK;
}

FeatScratch feat_scratch(cc_ctx *ctx) {
    return FeatScratch{as<uint32_t>(ctx->f_sdeg), as<unsigned>(ctx->f_counts), as<uint32_t>(ctx->f_vis),
                       as<uint32_t>(ctx->f_f0), as<uint32_t>(ctx->f_f1)};
}

cc_status check_options(const cc_options *o) {
    if (o->id_bytes != 4 && o->id_bytes != 8) return CC_ERR_INVALID_ARG;
    if (o->route_policy < CC_ROUTE_AUTO || o->route_policy > CC_ROUTE_FORCE_SV) return CC_ERR_INVALID_ARG;
    if (!(o->ks_tau >= 0.0 && o->ks_tau <= 2.0)) return CC_ERR_INVALID_ARG;
    if (o->ks_min_tail < 1 || o->ks_min_distinct < 1 || o->max_iters < 0 || o->bfs_cutoff_levels < 0 ||
        !(o->ks_min_span >= 0.0))
        return CC_ERR_INVALID_ARG;
    if (o->max_iters > kMaxIters - 1) return CC_ERR_INVALID_ARG;
    if (o->bfs_mode < 0 || o->bfs_mode > 1) return CC_ERR_INVALID_ARG;
    if (o->sv_sample_stride < 0 || o->sv_sample_stride > 1024) return CC_ERR_INVALID_ARG;
    if (o->bfs_starts < 0 || o->bfs_starts > kMaxBfsStarts) return CC_ERR_INVALID_ARG;
    if (o->batch_hook_regions < -1 || o->batch_hook_regions > 1024) return CC_ERR_INVALID_ARG;
    return CC_OK;
}

cudaEvent_t pool_event(cc_ctx *ctx) {
    if (ctx->evpool_used < ctx->evpool.size()) return ctx->evpool[ctx->evpool_used++];
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    ctx->evpool.push_back(e);
    ctx->evpool_used++;
    return e;
}

// Counts the launches of one kernel class and, with options.profile, brackets
// them with a pair of events on the launching stream.
struct Scope {
    cc_ctx *ctx;
    int cls;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    Scope(cc_ctx *c, int k, cudaStream_t st, int nlaunch) : ctx(c), cls(k), s(st) {
        ctx->stats.launches += nlaunch;
        if (ctx->opt.profile && ctx->prof.size() < 100000) {
            a = pool_event(ctx);
            if (a) cudaEventRecord(a, s);
        }
    }
    ~Scope() {
        if (!a) return;
        cudaEvent_t b = pool_event(ctx);
        if (!b) return;
        cudaEventRecord(b, s);
        ctx->prof.push_back({cls, a, b});
    }
};

void prof_reset(cc_ctx *ctx) {
    ctx->prof.clear();
    ctx->evpool_used = 0;
}

// Resolves the recorded event pairs (the stream has been synchronised).
void prof_collect(cc_ctx *ctx) {
    for (const auto &r : ctx->prof) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            ctx->stats.kernel_ms[r.cls] += ms;
            ctx->stats.kernel_launches[r.cls] += 1;
        } else {
            cudaGetLastError();
        }
    }
    ctx->prof.clear();
}

void rec(cc_ctx *ctx, Ev e, cudaStream_t s) {
    cudaEventRecord(ctx->ev[e], s);
    ctx->ev_used[e] = true;
}

// Copies `bytes` of the device state at `dev_ptr` (a member of ctx->st) into
// the same offset of the pinned mirror and waits for it.
cc_status read_back(cc_ctx *ctx, const void *dev_ptr, size_t bytes, cudaStream_t s) {
    const size_t off = (size_t)(reinterpret_cast<const char *>(dev_ptr) - reinterpret_cast<const char *>(ctx->st.p));
    CU_TRY(cudaMemcpyAsync(reinterpret_cast<char *>(ctx->h_st) + off, dev_ptr, bytes, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    return CC_OK;
}

cc_status device_error(uint32_t err) {
    if (err & kErrInvalidEdge) return CC_ERR_INVALID_EDGE;
    if (err & kErrNoConvergence) return CC_ERR_NO_CONVERGENCE;
    if (err & kErrTimeout) return CC_ERR_TIMEOUT;
    if (err & kErrBadOffsets) return CC_ERR_INVALID_ARG;
    if (err & kErrOverflow) return CC_ERR_CUDA;
    return CC_OK;
}

int default_max_iters(long long n) {
    int lg = 0;
    while (lg < 62 && (1LL << lg) < n) lg++;
    int c = 64 + 4 * lg;
    return c < kMaxIters - 1 ? c : kMaxIters - 1;
}

// ---------------------------------------------------------------------------
// SV as one CUDA graph: the fixed prefix (`pre`: parent init, the first two
// passes and their shortcuts), a WHILE node whose body is one SV iteration
// over the compacted list (k_sv_pass_loop, k_sv_shortcut, k_sv_loop_step:
// the device decides whether another iteration runs), and the fixed suffix
// (`post`: the labels). One graph launch replaces a host round trip per
// iteration. Graphs are captured on private streams (the caller's stream
// may be the legacy default stream, which cannot be captured) and cached
// per entry point while their arguments stay the same.

cc_ctx::GraphKey graph_key(cc_ctx *ctx, int kind, long long n, long long m, long long G, const void *edges,
                           const void *eo, const void *vo, const void *labels, int cap) {
    cc_ctx::GraphKey k;
    memset(&k, 0, sizeof(k));
    k.n = n;
    k.m = m;
    k.G = G;
    k.edges = edges;
    k.eo = eo;
    k.vo = vo;
    k.labels = labels;
    k.parent = ctx->parent.p;
    k.hooked = ctx->hooked.p;
    k.eb0 = ctx->ebuf0.p;
    k.eb1 = ctx->ebuf1.p;
    k.st = ctx->st.p;
    k.kind = kind;
    k.cap = cap;
    k.grid = ctx->grid;
    return k;
}

void graph_drop(cc_ctx::LoopGraph &lg) {
    if (lg.exec) cudaGraphExecDestroy(lg.exec);
    lg.exec = nullptr;
}

template <typename Pre, typename Post>
cc_status capture_sv_graph(cc_ctx *ctx, vid_t n, int it0, int cur0, int cap, Pre pre, Post post,
                           cudaGraphExec_t *out) {
    if (!ctx->cap_s) CU_TRY(cudaStreamCreateWithFlags(&ctx->cap_s, cudaStreamNonBlocking));
    if (!ctx->cap_s2) CU_TRY(cudaStreamCreateWithFlags(&ctx->cap_s2, cudaStreamNonBlocking));
    cudaStream_t cs = ctx->cap_s, cs2 = ctx->cap_s2;
    DevState *st = as<DevState>(ctx->st);
    CU_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    auto abort = [&](cudaError_t e) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(cs, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        const cc_status r = cuda_status(e);
        return r == CC_OK ? CC_ERR_CUDA : r;
    };
    pre(cs);
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph, &deps, &edata, &ndeps);
    if (e != cudaSuccess || cst != cudaStreamCaptureStatusActive) return abort(e);
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        return abort(e);
    launch_sv_loop_init(st, it0, cur0, cap, h, cs);
    if ((e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &graph, &deps, &edata, &ndeps)) != cudaSuccess)
        return abort(e);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    if ((e = cudaGraphAddNode(&cnode, graph, deps, edata, ndeps, &cp)) != cudaSuccess) return abort(e);
    if ((e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return abort(e);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
        cudaSuccess)
        return abort(e);
    launch_sv_loop_body(as<uint2>(ctx->ebuf0), as<uint2>(ctx->ebuf1), n, as<vid_t>(ctx->parent),
                        as<vid_t>(ctx->hooked), st, h, ctx->grid, cs2);
    cudaGraph_t body_out = nullptr;
    if ((e = cudaStreamEndCapture(cs2, &body_out)) != cudaSuccess) return abort(e);
    post(cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return CC_ERR_CUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return CC_ERR_CUDA;
    }
    return CC_OK;
}

// Launches the cached graph for `key` (capturing it first if the key changed).
template <typename Pre, typename Post>
cc_status launch_sv_graph(cc_ctx *ctx, cc_ctx::LoopGraph &lg, const cc_ctx::GraphKey &key, vid_t n, int it0,
                          int cur0, int cap, Pre pre, Post post, cudaStream_t s) {
    if (!lg.exec || memcmp(&lg.key, &key, sizeof(key)) != 0) {
        graph_drop(lg);
        CC_TRY(capture_sv_graph(ctx, n, it0, cur0, cap, pre, post, &lg.exec));
        lg.key = key;
    }
    CU_TRY(cudaGraphLaunch(lg.exec, s));
    return CC_OK;
}

// After a graph launch: waits, fills the iteration statistics (iteration it0
// and those before it are the prefix's) and returns the device status.
cc_status sv_graph_finish(cc_ctx *ctx, int it0, int prefix_launches, cudaStream_t s) {
    DevState *st = as<DevState>(ctx->st);
    cc_stats &S = ctx->stats;
    CU_TRY(cudaMemcpyAsync(ctx->h_st, st, offsetof(DevState, hook_base), cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    CU_TRY(cudaGetLastError());
    const DevState *h = ctx->h_st;
    const int done = h->loop_done > it0 ? h->loop_done : it0 + 1;
    for (int i = it0 + 1; i < done && i < CC_MAX_SV_ITERS_RECORDED; i++) S.m_active[i] = (int64_t)h->kept[i - 1];
    for (int i = 0; i < CC_MAX_SV_ITERS_RECORDED && i < done; i++) S.sv_hooks[i] = (int64_t)h->hooked[i];
    S.sv_iters = done;
    // prefix + loop init + 3 per loop iteration + the labels kernel
    S.launches += prefix_launches + 1 + 3 * (done - 1 - it0) + 1;
    return device_error(h->err);
}

BucketScratch bucket_scratch(cc_ctx *ctx) {
    return BucketScratch{as<unsigned long long>(ctx->bk_off), counter_at<unsigned long long>(ctx->counters, kCtrCsrQueue)};
}

float ev_ms(cc_ctx *ctx, Ev a, Ev b) {
    if (!ctx->ev_used[a] || !ctx->ev_used[b]) return 0.0f;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ctx->ev[a], ctx->ev[b]) != cudaSuccess) {
        cudaGetLastError();
        return 0.0f;
    }
    return ms;
}

// Degree pass + histogram (Algorithm 2 line 1).
template <typename T>
// hook: the parent array, every vertex its own root, when the windowed pass
// is to apply the first SV hook pass too (fused_hooks); null otherwise.
void enqueue_degree(cc_ctx *ctx, const void *edges, vid_t n, long long m, cudaStream_t s, bool counted = false,
                    vid_t *hook = nullptr) {
    if (counted) {  // the pairs were counted as they arrived (cc_labels_host): histogram only
        ctx->stats.degree_form = 1;
        Scope sc(ctx, CC_K_HIST, s, 1);
        launch_hist(as<uint32_t>(ctx->deg), n, as<uint32_t>(ctx->hist), as<uint32_t>(ctx->ovf), ctx->ovf_cap,
                    as<DevState>(ctx->st), ctx->grid, s);
        return;
    }
    cudaMemsetAsync(ctx->hist.p, 0, (size_t)kHistDense * 4, s);
    if (degree_part_ok(n, m) && ctx->dpart.bytes >= degree_part_scratch_bytes(n, m, hook != nullptr)) {
        ctx->stats.degree_form = 3;
        Scope sc(ctx, CC_K_DEGREE, s, 1 + degree_part_buckets(n));
        launch_degree_partitioned<T>(edges, m, n, as<uint32_t>(ctx->deg), hook, ctx->dpart.p, as<DevState>(ctx->st),
                                     ctx->num_sms, ctx->grid, s);
    } else if (degree_smem_ok(n, m) && ctx->ebuf1.bytes >= degree_smem_scratch_bytes(n, m)) {
        // ebuf1 (8m bytes) is idle until the second SV iteration; the 16-bit
        // entries take about 6m
        ctx->stats.degree_form = 4;
        Scope sc(ctx, CC_K_DEGREE, s, 2);
        launch_degree_smem<T>(edges, m, n, as<uint32_t>(ctx->deg), ctx->ebuf1.p, as<DevState>(ctx->st), ctx->num_sms,
                              s);
    } else if (degree_uses_hubs(m) && ctx->ebuf1.bytes >= degree_hubs_scratch_bytes()) {
        ctx->stats.degree_form = 2;
        cudaMemsetAsync(ctx->deg.p, 0, (size_t)n * 4, s);
        Scope sc(ctx, CC_K_DEGREE, s, 5);
        // ebuf1 is idle until the second SV iteration over the compacted list; m >= 2^24 makes it far larger
        // than the scratch
        launch_degree_hubs<T>(edges, m, n, as<uint32_t>(ctx->deg), as<unsigned>(ctx->ebuf1), as<DevState>(ctx->st),
                              ctx->grid, ctx->num_sms, s);
    } else {
        ctx->stats.degree_form = 1;
        cudaMemsetAsync(ctx->deg.p, 0, (size_t)n * 4, s);
        Scope sc(ctx, CC_K_DEGREE, s, m > 0);
        launch_degree<T>(edges, m, n, as<uint32_t>(ctx->deg), as<DevState>(ctx->st), ctx->grid, s);
    }
    {
        Scope sc(ctx, CC_K_HIST, s, 1);
        launch_hist(as<uint32_t>(ctx->deg), n, as<uint32_t>(ctx->hist), as<uint32_t>(ctx->ovf), ctx->ovf_cap,
                    as<DevState>(ctx->st), ctx->grid, s);
    }
}

// k distinct positive degrees sum to at least k(k+1)/2 <= 2m, so k <= sqrt(4m);
// and k <= n. (`m` < 0: unknown, take the scratch capacity.)
long long distinct_degree_bound(cc_ctx *ctx, long long n, long long m) {
    long long b = (long long)ctx->ks_cap;
    if (n > 0 && n < b) b = n;
    if (m >= 0) {
        const long long r = (long long)sqrt(4.0 * (double)m) + 2;
        if (r < b) b = r;
    }
    return b;
}

void enqueue_ks(cc_ctx *ctx, cudaStream_t s, long long nd_bound) {
    KsScratch ks{as<uint32_t>(ctx->ks_xs), as<unsigned long long>(ctx->ks_cnt), as<unsigned long long>(ctx->ks_cum),
                 as<double>(ctx->ks_lnx), as<double>(ctx->ks_Dc), as<double>(ctx->ks_Ac), as<double>(ctx->ks_Zc),
                 as<float>(ctx->ks_Df),
                 as<unsigned long long>(ctx->chunk_nz), as<unsigned long long>(ctx->chunk_mass), ctx->ks_cap};
    Scope sc(ctx, CC_K_KS, s, 7);
    launch_ks(as<uint32_t>(ctx->hist), as<uint32_t>(ctx->ovf), ctx->ovf_cap, ks, as<DevState>(ctx->st),
              ctx->opt.ks_min_tail, ctx->opt.ks_min_distinct, ctx->opt.ks_min_span, ctx->opt.ks_tau, nd_bound,
              ctx->grid, s);
}

// CSR + direction-optimizing BFS from the max-degree vertex. Returns the
// number of levels run; leaves the visited bitmap in ctx->vis and cmin in DevState.
template <typename T>
cc_status run_bfs(cc_ctx *ctx, const void *edges, vid_t n, long long m, cudaStream_t s, int cutoff, int *levels_out) {
    DevState *st = as<DevState>(ctx->st);
    uint32_t *row_ptr = as<uint32_t>(ctx->row_ptr), *deg = as<uint32_t>(ctx->deg);
    vid_t *col = as<vid_t>(ctx->col);
    const long long nwords = ((long long)n + 31) / 32;
    // row_ptr = exclusive scan of deg
    const bool bucketed = bucketed_ok(n, (size_t)m) && ctx->csr_entries.p;
    {
        Scope sc(ctx, CC_K_SCAN, s, 3);
        // both CSR builds use a copy of row_ptr in deg as their cursors
        launch_scan_u32(deg, n, row_ptr, deg, as<unsigned long long>(ctx->tsum), nullptr, row_ptr + n, s);
    }
    if (bucketed) {
        Scope sc(ctx, CC_K_CSR, s, 2);
        launch_csr_bucketed<T>(edges, m, n, row_ptr, deg, col, bucket_scratch(ctx),
                               as<unsigned long long>(ctx->csr_entries), st, ctx->grid, s);
    } else {
        Scope sc(ctx, CC_K_CSR, s, 1);
        launch_csr_scatter<T>(edges, m, n, deg, col, ctx->grid, s);
    }
    rec(ctx, EV_CSR, s);
    cudaMemsetAsync(ctx->vis.p, 0, (size_t)nwords * 4, s);
    vid_t *qcur = as<vid_t>(ctx->q0), *qnext = as<vid_t>(ctx->q1);
    uint32_t *fb = as<uint32_t>(ctx->fb), *nb = as<uint32_t>(ctx->nb), *vis = as<uint32_t>(ctx->vis);
    {
        Scope sc(ctx, CC_K_BFS_AUX, s, 1);
        launch_bfs_init(row_ptr, n, vis, qcur, st, s);
    }
    // Beamer's switching rule: go bottom-up when the frontier's edges exceed
    // 1/alpha of the unexplored edges; come back when the frontier holds fewer
    // than n/beta vertices and is shrinking.
    const double alpha = 14.0, beta = 24.0;
    bool bottom_up = false, have_queue = true;
    unsigned long long f = 1, fe = 0, explored = 0, prev_f = 0;
    const unsigned long long total_edges = 2ull * (unsigned long long)m;
    CC_TRY(read_back(ctx, &st->front_edges[0], 8, s));
    fe = ctx->h_st->front_edges[0];
    int level = 0;
    unsigned long long *cnt = counter_at<unsigned long long>(ctx->counters, kCtrBfs);
    while (f > 0 && level < kMaxLevels - 1) {
        if (cutoff > 0 && level >= cutoff) break;
        const unsigned long long unexplored = total_edges > explored ? total_edges - explored : 0;
        if (!bottom_up && (double)fe > (double)unexplored / alpha) bottom_up = true;
        else if (bottom_up && (double)f < (double)n / beta && f < prev_f) bottom_up = false;
        if (bottom_up) {
            if (have_queue) {
                cudaMemsetAsync(fb, 0, (size_t)nwords * 4, s);
                Scope sc(ctx, CC_K_BFS_AUX, s, 1);
                launch_queue_to_bitmap(qcur, (long long)f, fb, ctx->grid, s);
                have_queue = false;
            }
            {
                Scope sc(ctx, CC_K_BFS_BOTTOMUP, s, 1);
                launch_bfs_bottomup(n, row_ptr, col, fb, vis, nb, st, level, ctx->grid, s);
            }
            uint32_t *t = fb;
            fb = nb;
            nb = t;
        } else {
            if (!have_queue) {
                cudaMemsetAsync(cnt, 0, 8, s);
                Scope sc(ctx, CC_K_BFS_AUX, s, 1);
                launch_bitmap_to_queue(fb, nwords, qcur, cnt, ctx->grid, s);
                have_queue = true;
            }
            uint32_t *dq = as<uint32_t>(ctx->dq), *off = as<uint32_t>(ctx->off);
            {
                Scope sc(ctx, CC_K_BFS_AUX, s, 1);
                launch_front_degrees(qcur, (long long)f, row_ptr, dq, ctx->grid, s);
            }
            {
                Scope sc(ctx, CC_K_SCAN, s, 3);
                launch_scan_u32(dq, (long long)f, off, nullptr, as<unsigned long long>(ctx->tsum), nullptr, nullptr,
                                s);
            }
            {
                Scope sc(ctx, CC_K_BFS_TOPDOWN, s, 1);
                launch_bfs_topdown(qcur, (long long)f, off, (long long)fe, row_ptr, col, vis, qnext, st, level,
                                   ctx->grid, s);
            }
            vid_t *t = qcur;
            qcur = qnext;
            qnext = t;
        }
        explored += fe;
        CU_TRY(cudaMemcpyAsync(&ctx->h_st->front[level + 1], &st->front[level + 1], 8, cudaMemcpyDeviceToHost, s));
        CC_TRY(read_back(ctx, &st->front_edges[level + 1], 8, s));
        prev_f = f;
        f = ctx->h_st->front[level + 1];
        fe = ctx->h_st->front_edges[level + 1];
        level++;
    }
    *levels_out = level;
    // visited count and the smallest visited id (the BFS component's label)
    cudaMemsetAsync(cnt + 1, 0, 8, s);
    Scope sc(ctx, CC_K_BFS_AUX, s, 2);
    launch_popcount(vis, nwords, cnt + 1, ctx->grid, s);
    launch_first_visited(vis, nwords, st, ctx->grid, s);
    return CC_OK;
}

// SV iterations over the compacted active list until no pair is active
// (Section 3.1.4: completed partitions leave the working set). `src` holds
// m_cur pairs in ebuf[cur]; `it` is the last iteration run so far.
cc_status sv_list_loop(cc_ctx *ctx, vid_t n, const void *src, unsigned long long m_cur, int it, int cap,
                       cudaStream_t s, int cur = 0) {
    DevState *st = as<DevState>(ctx->st);
    cc_stats &S = ctx->stats;
    vid_t *parent = as<vid_t>(ctx->parent), *hooked = as<vid_t>(ctx->hooked);
    uint2 *eb[2] = {as<uint2>(ctx->ebuf0), as<uint2>(ctx->ebuf1)};
    while (m_cur > 0) {
        it++;
        if (it >= cap) {
            S.sv_iters = it;
            return CC_ERR_NO_CONVERGENCE;
        }
        if (it < CC_MAX_SV_ITERS_RECORDED) S.m_active[it] = (int64_t)m_cur;
        {
            Scope sc(ctx, CC_K_SV_GATHER_LIST, s, 1);
            launch_sv_pass<uint32_t>(2, true, true, src, (long long)m_cur, n, parent, nullptr, 0, hooked, eb[1 - cur],
                                     st, it, ctx->grid, s);
        }
        {
            Scope sc(ctx, CC_K_SV_SHORTCUT, s, 1);
            launch_sv_shortcut(parent, hooked, st, it, ctx->grid, s);
        }
        cur = 1 - cur;
        src = eb[cur];
        CU_TRY(cudaMemcpyAsync(&ctx->h_st->kept[it], &st->kept[it], 8, cudaMemcpyDeviceToHost, s));
        CU_TRY(cudaStreamSynchronize(s));
        m_cur = ctx->h_st->kept[it];
    }
    S.sv_iters = it + 1;
    return CC_OK;
}

// Edge-list BFS from the vertex named by *key (Algorithm 2 lines 6-9 without
// a CSR). On return the visited set is in ctx->f_vis, cmin in DevState, and
// the pairs still active (those without both ends visited) are either the
// caller's pairs (*list_buf < 0) or the compacted list in ebuf[*list_buf]
// with *list_len pairs.
template <typename T>
cc_status run_bfs_edges(cc_ctx *ctx, const void *edges, vid_t n, long long m, cudaStream_t s, int cutoff,
                        const unsigned long long *key, int *levels_out, int *list_buf, unsigned long long *list_len) {
    DevState *st = as<DevState>(ctx->st);
    CC_TRY(ensure_feat(ctx, n));
    if (!ctx->counters.p || !ctx->f_vis.p || !ctx->ebuf0.p || !ctx->ebuf1.p) return CC_ERR_CUDA;
    const long long nwords = ((long long)n + 31) / 32;
    uint32_t *vis = as<uint32_t>(ctx->f_vis), *cur = as<uint32_t>(ctx->f_f0), *next = as<uint32_t>(ctx->f_f1);
    uint2 *eb[2] = {as<uint2>(ctx->ebuf0), as<uint2>(ctx->ebuf1)};
    cudaMemsetAsync(vis, 0, (size_t)nwords * 4, s);
    cudaMemsetAsync(cur, 0, (size_t)nwords * 4, s);
    // per-level counters start at zero (the batched form runs one BFS per routed graph in one call)
    CU_TRY(cudaMemsetAsync(&st->front[0], 0, sizeof(st->front) + sizeof(st->front_edges), s));
    {
        Scope sc(ctx, CC_K_BFS_AUX, s, 1);
        launch_edge_bfs_seed(vis, cur, n, key, st, s);
    }
    const void *src = edges;
    unsigned long long len = (unsigned long long)m, kept_prev = (unsigned long long)m;
    int buf = -1, level = 0;
    while (level < kMaxLevels - 1 && (cutoff <= 0 || level < cutoff)) {
        cudaMemsetAsync(next, 0, (size_t)nwords * 4, s);
        // compact once the surviving pairs fall to 70% of the active list
        const bool write = level >= 1 && (double)kept_prev <= 0.7 * (double)len;
        const int ob = buf == 0 ? 1 : 0;
        {
            Scope sc(ctx, CC_K_BFS_BOTTOMUP, s, 1);
            if (buf < 0) launch_bfs_edges<T>(write, src, (long long)len, n, vis, cur, next, eb[ob], st, level, ctx->grid, s);
            else
                launch_bfs_edges<uint32_t>(write, src, (long long)len, n, vis, cur, next, eb[ob], st, level, ctx->grid,
                                           s);
        }
        CU_TRY(cudaMemcpyAsync(&ctx->h_st->front[level + 1], &st->front[level + 1], 8, cudaMemcpyDeviceToHost, s));
        CC_TRY(read_back(ctx, &st->front_edges[level + 1], 8, s));
        const unsigned long long claimed = ctx->h_st->front[level + 1], kept = ctx->h_st->front_edges[level + 1];
        if (write) {
            src = eb[ob];
            len = kept;
            buf = ob;
        }
        kept_prev = kept;
        uint32_t *t = cur;
        cur = next;
        next = t;
        level++;
        if (claimed == 0) break;
    }
    *levels_out = level;
    *list_buf = buf;
    *list_len = len;
    unsigned long long *cnt = counter_at<unsigned long long>(ctx->counters, kCtrBfs);
    cudaMemsetAsync(cnt + 1, 0, 8, s);
    Scope sc(ctx, CC_K_BFS_AUX, s, 2);
    launch_popcount(vis, nwords, cnt + 1, ctx->grid, s);
    launch_first_visited(vis, nwords, st, ctx->grid, s);
    return CC_OK;
}

// The multi-start BFS with the host driving the levels (options.profile):
// the graph route's kernels, each level timed. Leaves the active pairs'
// buffer and length as run_bfs_edges does, the visited count in the BFS
// counter, and the parents of the trees' vertices set to the tree minima.
template <typename T>
cc_status run_mbfs_edges(cc_ctx *ctx, const void *edges, vid_t n, long long m, cudaStream_t s, int cutoff,
                         int *levels_out, int *list_buf, unsigned long long *list_len) {
    DevState *st = as<DevState>(ctx->st);
    CC_TRY(ensure_mbfs(ctx, n));
    const long long nwords = ((long long)n + 31) / 32;
    uint32_t *vis = as<uint32_t>(ctx->f_vis), *b0 = as<uint32_t>(ctx->f_f0), *b1 = as<uint32_t>(ctx->f_f1);
    uint32_t *own = as<uint32_t>(ctx->bfs_own), *tmin = as<uint32_t>(ctx->bfs_tmin);
    uint2 *eb0 = as<uint2>(ctx->ebuf0), *eb1 = as<uint2>(ctx->ebuf1);
    {
        Scope sc(ctx, CC_K_BFS_AUX, s, 2);
        launch_mbfs_start(as<uint32_t>(ctx->deg), n, m, ctx->opt.bfs_starts, vis, b0, own, tmin, st, nullptr, s);
    }
    int level = 0;
    while (level < kMaxLevels - 1 && (cutoff <= 0 || level < cutoff)) {
        {
            Scope sc(ctx, CC_K_BFS_BOTTOMUP, s, 4);
            launch_ebfsg_level<T>(edges, m, eb0, eb1, n, vis, b0, b1, st, cudaGraphConditionalHandle(), ctx->grid, s,
                                  own, false);
        }
        CC_TRY(read_back(ctx, &st->front[level + 1], 8, s));
        level++;
        if (ctx->h_st->front[level] == 0) break;
    }
    CU_TRY(cudaMemcpyAsync(&ctx->h_st->bfs_starts, &st->bfs_starts, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaMemcpyAsync(&ctx->h_st->bfs_len, &st->bfs_len, 8, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaMemcpyAsync(&ctx->h_st->bfs_inspected, &st->bfs_inspected, 8, cudaMemcpyDeviceToHost, s));
    CC_TRY(read_back(ctx, &st->bfs_list, sizeof(int), s));
    *levels_out = level;
    *list_buf = ctx->h_st->bfs_list;
    *list_len = *list_buf < 0 ? (unsigned long long)m : ctx->h_st->bfs_len;
    unsigned long long *cnt = counter_at<unsigned long long>(ctx->counters, kCtrBfs);
    cudaMemsetAsync(cnt + 1, 0, 8, s);
    Scope sc(ctx, CC_K_BFS_AUX, s, 4);
    launch_popcount(vis, nwords, cnt + 1, ctx->grid, s);
    launch_first_visited(vis, nwords, st, ctx->grid, s);
    launch_mbfs_finish(own, tmin, n, as<vid_t>(ctx->parent), ctx->grid, s);
    return CC_OK;
}

cc_status ensure_side(cc_ctx *ctx) {
    // lowest priority: the prediction on the caller's stream (the K-S fit, a
    // few small grids) gets the SMs first and the speculative pass fills the rest
    if (!ctx->side_s) {
        int least = 0, greatest = 0;
        CU_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CU_TRY(cudaStreamCreateWithPriority(&ctx->side_s, cudaStreamNonBlocking, least));
    }
    if (!ctx->ev_fork) CU_TRY(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    if (!ctx->ev_join) CU_TRY(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    return CC_OK;
}

cc_status ensure_fit_stream(cc_ctx *ctx) {
    if (!ctx->fit_s) {
        int least = 0, greatest = 0;
        CU_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CU_TRY(cudaStreamCreateWithPriority(&ctx->fit_s, cudaStreamNonBlocking, greatest));
    }
    if (!ctx->ev_fit) CU_TRY(cudaEventCreateWithFlags(&ctx->ev_fit, cudaEventDisableTiming));
    if (!ctx->ev_fork) CU_TRY(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    return CC_OK;
}

// Orders all later work on `s` after the side stream's speculative pass, on
// every exit path (the next call must not reset state the side stream uses).
struct JoinGuard {
    cc_ctx *ctx;
    cudaStream_t s;
    bool armed = false;
    void join() {
        if (armed) cudaStreamWaitEvent(s, ctx->ev_join, 0);
        armed = false;
    }
    ~JoinGuard() { join(); }
};

cc_status ensure_batch_route(cc_ctx *ctx, int G, int blocks = 0);

// The route of a small graph by the one-block fit (the degrees are in ctx->deg).
cc_status enqueue_small_fit(cc_ctx *ctx, vid_t n, cudaStream_t s) {
    KsBatchScratch sc{as<uint32_t>(ctx->kb_xs), as<unsigned long long>(ctx->kb_cnt), as<unsigned long long>(ctx->kb_cum),
                      as<double>(ctx->kb_lnx), as<double>(ctx->kb_Dc), as<double>(ctx->kb_Ac), as<double>(ctx->kb_Zc)};
    KsBatchOut out{as<double>(ctx->kb_D),     as<double>(ctx->kb_alpha), as<long long>(ctx->kb_xmin),
                   as<long long>(ctx->kb_ntail), as<long long>(ctx->kb_ncand), as<int>(ctx->kb_route),
                   as<int>(ctx->kb_ovf),      as<unsigned long long>(ctx->kb_seed)};
    int64_t *vo = counter_at<int64_t>(ctx->counters, kCtrSmallFitVo);
    Scope sc2(ctx, CC_K_KS, s, 4);
    // the idle degree-histogram buffer (kHistDense words) holds the grid-wide histogram of the small graph
    launch_fit_one(as<uint32_t>(ctx->deg), n, vo, sc, out, as<DevState>(ctx->st), ctx->opt.ks_min_tail,
                   ctx->opt.ks_min_distinct, ctx->opt.ks_min_span, ctx->opt.ks_tau, as<uint32_t>(ctx->hist), ctx->grid,
                   s);
    return CC_OK;
}

// SV front end: hook passes over one tile of pairs in k (a strided sample,
// so that sorted inputs are sampled everywhere) join most of every large
// component before the first pass over all pairs. That pass then drops most
// pairs at once (equal roots) instead of hooking, keeping and re-reading
// them, and the plain hook pass over all pairs disappears. The sample holds
// a giant component only when its mean degree 2m / (n k) is about 1 or more,
// so by default k is the largest power of two <= 2m / n (a sample mean
// degree in [1, 2)), at most kSampleStrideMax, and there is no front end
// when that k is below 4 or m below kSampleMinPairs. Measured (ms, labels
// identical): R-MAT 24 (2m/n = 32): none 7.88, k = 16 5.62, k = 32 5.47;
// R-MAT 24 with 4 pairs per vertex: none 2.63, k = 4 2.21, k = 8 2.12; the
// chain forest plus grid (2m/n ~ 2) with k = 8: 59.3 against 49.6 with none.
// The batched form keeps the plain first pass: a per-graph front end there
// (4,096 graphs) took 116 ms against 109, its extra full shortcut over all
// graphs' vertices costing more than the shorter lists saved.
constexpr long long kSampleMinPairs = 1LL << 22;

// The plain first pass (every vertex its own root) reads parent[max] before
// its atomicMin, which skips hooks that cannot lower it. On graphs with hubs
// many pairs share a larger end and the read saves most atomics; on sparse
// graphs (mean degree 2m/n < 4) nearly every hook lowers its target, and a
// fire-and-forget atomicMin without the read (MODE 4) is faster. Measured:
// grid + chains 8.40 -> 6.81 ms for the pass without the read; R-MAT 24
// without the front end 0.99 -> 2.60 ms.
int first_pass_mode(vid_t n, long long m) { return 2 * m < 4 * (long long)n ? 4 : 0; }
constexpr int kSampleStrideMax = 64;

int sample_stride(const cc_ctx *ctx, vid_t n, long long m) {
    const int k = ctx->opt.sv_sample_stride;
    if (k != 0) return k;
    if (m < kSampleMinPairs || n == 0) return 1;
    const long long r = 2 * m / (long long)n;
    int p = 1;
    while (p * 2 <= r && p * 2 <= kSampleStrideMax) p *= 2;
    return p >= 4 ? p : 1;
}

// The batched form's front end (per-graph strides on the device): on when
// options.sv_sample_stride > 1. Off by default: on the 4,096-graph batch
// (79% of the pairs in R-MAT graphs with 2m/n = 16) it cut the pairs left
// after the first gather pass from 1.71G to 637M, but its passes and the
// extra full shortcut over the union took 24.5 ms against 15.2 ms for one
// hook pass over all pairs, and the gather pass only fell from 23.9 to 22.4
// ms (it is bound by the parent gathers, not by the survivors it writes):
// 94.2 ms a call against 86.8.
bool batch_front(const cc_ctx *ctx, long long m) { return ctx->opt.sv_sample_stride > 1 && m > 0; }

// The first hook pass over all pairs rides on the windowed degree pass (its
// window pass applies atomicMin(parent[max], min) while the window's parents
// are in L2) when that pass runs (n > 2^25) and the SV front end does not
// (the sample passes come before any pass over all pairs).
bool fused_hooks(const cc_ctx *ctx, vid_t n, long long m) {
    return degree_part_ok(n, m) && sample_stride(ctx, n, m) == 1 &&
           ctx->dpart.bytes >= degree_part_scratch_bytes(n, m, true);
}

// The first SV pass on stream s while every vertex is its own root; after it
// every vertex points at its root. With a sample stride k > 1: the front end
// (a hook pass with identity parents and a one-hop hook pass over the sample,
// each followed by a full shortcut); else one hook pass over all pairs and a
// full shortcut. Returns the kernel launches; `scoped` times them (off inside
// a graph capture).
template <typename T>
int enqueue_first_pass(cc_ctx *ctx, const void *edges, vid_t n, long long m, cudaStream_t s, bool scoped) {
    vid_t *parent = as<vid_t>(ctx->parent), *hooked = as<vid_t>(ctx->hooked);
    DevState *st = as<DevState>(ctx->st);
    const int k = sample_stride(ctx, n, m);
    ctx->stats.sv_sample_stride = k;
    auto timed = [&](int cls, auto &&fn) {
        if (scoped) {
            Scope sc(ctx, cls, s, 1);
            fn();
        } else {
            fn();
        }
    };
    auto shortcut = [&] { launch_shortcut_all(parent, n, st, 0, ctx->grid, s); };
    if (k > 1) {
        timed(CC_K_SV_FIRST, [&] { launch_sv_sample<T>(0, edges, m, n, parent, st, k, ctx->grid, s); });
        timed(CC_K_SV_SHORTCUT, shortcut);
        timed(CC_K_SV_FIRST, [&] { launch_sv_sample<T>(2, edges, m, n, parent, st, k, ctx->grid, s); });
        timed(CC_K_SV_SHORTCUT, shortcut);
        return 4;
    }
    const int mode = first_pass_mode(n, m);
    timed(CC_K_SV_FIRST, [&] {
        launch_sv_pass<T>(mode, false, false, edges, m, n, parent, nullptr, 0, hooked, nullptr, st, 0, ctx->grid, s);
    });
    timed(CC_K_SV_SHORTCUT, shortcut);
    return 2;
}

// Speculation of the single-graph route: the side stream runs parent init,
// the first pass and SV iteration 1 (the gather pass over the pairs), forked
// after the degree pass, while the K-S fit runs on a highest-priority stream
// and the gather pass launches one block per tile (so the fit's blocks get
// SMs as gather blocks retire). Measured on R-MAT 24 before the SV front
// end: the first pass alone speculated 7.82 ms, with the gather pass 7.61
// ms, both forked before the degree pass 8.64 ms (the degree pass and the
// hook passes then contend for the L2 atomics). With the front end, R-MAT
// 24 / 22: fit first and the speculative passes after it 5.44 / 1.75 ms,
// fit beside them 5.26 / 1.56 ms; forking the front end alone before the
// degree pass as well 5.29 / 1.53 ms.

// Work cc_labels_host has already enqueued while the pairs were copied: the
// device state zeroed and EV_START recorded, the degrees counted (AUTO), and
// the first SV pass (parent init, unrecorded hook pass, full shortcut) on the
// side stream, ending in ev_join.
struct Staged {
    bool degree_counted = false;
    bool first_pass_done = false;  // parent init, MODE 0 pass and full shortcut
    bool streamed = false;         // or: SV iterations 1..it0 ran chunk by chunk (MODE 3), every
                                   // vertex points at its root, the pairs that crossed are in ebuf0
    int it0 = 0;                   // with kept[it0] of them
    int launches = 0;
};

template <typename T>
cc_status labels_impl(cc_ctx *ctx, const void *edges, vid_t n, long long m, void *labels_out, cudaStream_t s,
                      const Staged *pre = nullptr) {
    DevState *st = as<DevState>(ctx->st);
    cc_stats &S = ctx->stats;
    memset(&S, 0, sizeof(S));
    prof_reset(ctx);
    S.n = n;
    S.m = m;
    for (int e = 0; e < EV_COUNT; e++) ctx->ev_used[e] = false;
    if (pre) {
        S.launches = pre->launches;
        ctx->ev_used[EV_START] = true;
    } else {
        CU_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), s));
        rec(ctx, EV_START, s);
    }
    const int policy = ctx->opt.route_policy;
    int route = 0;
    S.route_source = policy == CC_ROUTE_AUTO || policy == CC_ROUTE_LEARNED ? 0 : 2;
    vid_t *parent = as<vid_t>(ctx->parent), *hooked = as<vid_t>(ctx->hooked);
    // Speculative first SV pass. On the SV route the first pass needs nothing
    // the prediction computes (every vertex starts as its own root), so the
    // parent init, the unrecorded hook pass and the full shortcut run on a
    // side stream while the route prediction runs on `s`. It is forked after
    // the degree pass (both are bound by scattered L2 operations, so running
    // them together gains nothing) to overlap the K-S fit, or at the start
    // of the learned route's sampled features. The BFS route re-initialises
    // the parent array after its BFS, so the speculative work is then unused.
    JoinGuard spec{ctx, s};
    if (pre && (pre->first_pass_done || pre->streamed)) spec.armed = true;
    const bool streamed = pre && pre->streamed;
    const int cap = ctx->opt.fault_inject & CC_FAULT_ITER_CAP ? 1
                    : ctx->opt.max_iters > 0                  ? ctx->opt.max_iters
                                                              : default_max_iters(n);
    bool deep_done = false;  // the side stream also ran SV iteration 1
    // the first hook pass inside the windowed degree pass (parent init first), as on the graph route
    const bool fused = !pre && policy != CC_ROUTE_FORCE_SV && policy != CC_ROUTE_FORCE_BFS &&
                       !(policy == CC_ROUTE_LEARNED && ctx->have_pred) && m > 0 && fused_hooks(ctx, n, m);
    auto speculate = [&]() -> cc_status {
        if (spec.armed || m <= 0) return CC_OK;
        CC_TRY(ensure_side(ctx));
        cudaStream_t side = ctx->side_s;
        CU_TRY(cudaEventRecord(ctx->ev_fork, s));
        CU_TRY(cudaStreamWaitEvent(side, ctx->ev_fork, 0));
        if (fused) {  // parents initialised and hooked by the degree pass: the full shortcut remains
            Scope sc(ctx, CC_K_SV_SHORTCUT, side, 1);
            launch_shortcut_all(parent, n, st, 0, ctx->grid, side);
            ctx->stats.sv_sample_stride = 1;
        } else {
            {
                Scope sc(ctx, CC_K_PARENT_INIT, side, 1);
                launch_parent_init(parent, n, nullptr, 0, ctx->grid, side);
            }
            enqueue_first_pass<T>(ctx, edges, n, m, side, true);
        }
        if (cap >= 2) {
            // SV iteration 1 as well: the gather pass over the pairs, the crossing
            // pairs into ebuf0 (the degree pass keeps its hub table in ebuf1)
            {
                Scope sc(ctx, CC_K_SV_GATHER_INPUT, side, 1);
                launch_sv_gather_tiles<T>(edges, m, n, parent, hooked, as<uint2>(ctx->ebuf0), st, 1, side);
            }
            {
                Scope sc(ctx, CC_K_SV_SHORTCUT, side, 1);
                launch_sv_shortcut(parent, hooked, st, 1, ctx->grid, side);
            }
            deep_done = true;
        }
        CU_TRY(cudaEventRecord(ctx->ev_join, side));
        spec.armed = true;
        return CC_OK;
    };
    int cutoff = ctx->opt.bfs_cutoff_levels;
    // Learned route: sampled features + network; a confident prediction skips
    // the exact degree pass and the K-S fit (its BFS is the edge-list BFS,
    // seeded at the sampled hub).
    bool learned = false;
    S.pred_route = -1;
    if (policy == CC_ROUTE_LEARNED && ctx->have_pred && m > 0) {
        CC_TRY(ensure_feat(ctx, n));
        CC_TRY(speculate());
        {
            Scope sc(ctx, CC_K_PREDICT, s, 12);
            launch_route_features<T>(edges, m, n, feat_scratch(ctx), st, as<float>(ctx->f_x), ctx->grid, s);
            mlp_infer(as<__nv_bfloat16>(ctx->pred_wb), as<float>(ctx->pred_bias), as<float>(ctx->f_x), st, s);
        }
        rec(ctx, EV_DEGREE, s);
        CU_TRY(cudaMemcpyAsync(ctx->h_st, st, offsetof(DevState, kept), cudaMemcpyDeviceToHost, s));
        CU_TRY(cudaStreamSynchronize(s));
        if (ctx->h_st->err) return device_error(ctx->h_st->err);
        S.pred_route = ctx->h_st->pred_route;
        S.pred_confidence = ctx->h_st->pred_conf;
        S.pred_cutoff = ctx->h_st->pred_cutoff;
        S.ms_features = ev_ms(ctx, EV_START, EV_DEGREE);
        if (ctx->h_st->pred_conf >= ctx->pred_min_conf) {
            learned = true;
            route = ctx->h_st->pred_route;
            if (route == 1 && cutoff == 0) cutoff = ctx->h_st->pred_cutoff;
            S.route_source = 1;
        }
    }
    if (!learned && policy != CC_ROUTE_FORCE_SV && m > 0) {
        // Small graphs (n <= 2^20, fewer than 4,097 vertices of degree >= 4,096
        // possible) take the one-block fit of the batched form: the histogram,
        // the fit and the seed in one launch instead of the grid-wide kernels
        // sized for 2^20 histogram bins.
        const bool small = !pre && n <= (1u << 20) && 2 * m < 4096LL * 4097LL && policy != CC_ROUTE_FORCE_BFS;
        if (small) {
            CC_TRY(ensure_batch_route(ctx, 1, 1));
            CU_TRY(cudaMemsetAsync(ctx->deg.p, 0, (size_t)n * 4, s));
            ctx->stats.degree_form = 1;
            {
                Scope sc(ctx, CC_K_DEGREE, s, m > 0);
                launch_degree<T>(edges, m, n, as<uint32_t>(ctx->deg), st, ctx->grid, s);
            }
            rec(ctx, EV_DEGREE, s);
            // the fit is queued ahead of the speculative passes so that its few
            // blocks are not left waiting behind them
            CC_TRY(enqueue_small_fit(ctx, n, s));
            CC_TRY(speculate());
        } else {
            if (fused) {
                Scope sc(ctx, CC_K_PARENT_INIT, s, 1);
                launch_parent_init(parent, n, nullptr, 0, ctx->grid, s);
            }
            enqueue_degree<T>(ctx, edges, n, m, s, pre && pre->degree_counted, fused ? parent : nullptr);
            rec(ctx, EV_DEGREE, s);
            if (policy != CC_ROUTE_FORCE_BFS) {
                // the fit on a highest-priority stream: the speculative gather
                // launches one block per tile, so the fit's blocks are
                // scheduled as soon as gather blocks retire
                CC_TRY(speculate());
                CC_TRY(ensure_fit_stream(ctx));
                CU_TRY(cudaEventRecord(ctx->ev_fork, s));
                CU_TRY(cudaStreamWaitEvent(ctx->fit_s, ctx->ev_fork, 0));
                enqueue_ks(ctx, ctx->fit_s, distinct_degree_bound(ctx, n, m));
                CU_TRY(cudaEventRecord(ctx->ev_fit, ctx->fit_s));
                CU_TRY(cudaStreamWaitEvent(s, ctx->ev_fit, 0));
            }
        }
        rec(ctx, EV_PREDICT, s);
        CU_TRY(cudaMemcpyAsync(ctx->h_st, st, offsetof(DevState, kept), cudaMemcpyDeviceToHost, s));
        CU_TRY(cudaStreamSynchronize(s));
        if (ctx->h_st->err) return device_error(ctx->h_st->err);
        route = policy == CC_ROUTE_FORCE_BFS ? 1 : ctx->h_st->route;
        S.ks_d = ctx->h_st->ks_out[0];
        S.ks_alpha = ctx->h_st->ks_out[1];
        S.ks_xmin = (int64_t)ctx->h_st->ks_out[2];
        S.ks_ntail = (int64_t)ctx->h_st->ks_out[3];
        S.ks_ncand = (int64_t)ctx->h_st->ks_out[4];
        S.max_degree = (int64_t)(ctx->h_st->maxkey >> 32);
        S.seed_vertex = (int64_t)(0xffffffffu - (uint32_t)(ctx->h_st->maxkey & 0xffffffffu));
        if (policy == CC_ROUTE_FORCE_BFS) S.ks_d = 0.0;
    }
    const bool speculated = spec.armed;
    spec.join();  // later work on `s` sees the speculative pass complete
    // the learned route always takes the edge-list BFS (it needs no exact
    // degrees); the CSR uses 32-bit offsets, so the CSR BFS needs 2m < 2^32
    const bool multi = multi_start(ctx);
    const bool edge_bfs = learned || multi || ctx->opt.bfs_mode == 1;
    if (route == 1 && !edge_bfs && 2ull * (unsigned long long)m >= 0xffffffffull) route = 0;
    S.route = route;
    uint2 *eb[2] = {as<uint2>(ctx->ebuf0), as<uint2>(ctx->ebuf1)};
    int it = 0, cur0 = 0;
    unsigned long long m_cur = 0;
    const void *src = nullptr;
    if (route == 1 && (streamed || deep_done)) {
        // the BFS route replaces the iterations the host-input path streamed:
        // clear their per-iteration counters (the side stream is joined)
        CU_TRY(cudaMemsetAsync(&st->kept[0], 0, offsetof(DevState, front) - offsetof(DevState, kept), s));
    }
    if (route == 1) {
        int levels = 0, list_buf = -1;
        unsigned long long list_len = (unsigned long long)m;
        const uint32_t *vis = nullptr;
        if (multi) {
            CC_TRY(run_mbfs_edges<T>(ctx, edges, n, m, s, cutoff, &levels, &list_buf, &list_len));
            vis = as<uint32_t>(ctx->f_vis);
        } else if (edge_bfs) {
            // seed: the exact max-degree vertex when the degree pass ran, else the sampled hub
            const unsigned long long *key = learned ? &st->pred_seedkey : &st->maxkey;
            CC_TRY(run_bfs_edges<T>(ctx, edges, n, m, s, cutoff, key, &levels, &list_buf, &list_len));
            vis = as<uint32_t>(ctx->f_vis);
        } else {
            CC_TRY(ensure_bfs(ctx, n, (size_t)m));
            CC_TRY(run_bfs<T>(ctx, edges, n, m, s, cutoff, &levels));
            vis = as<uint32_t>(ctx->vis);
        }
        rec(ctx, EV_BFS, s);
        CU_TRY(cudaMemcpyAsync(&ctx->h_st->cmin, &st->cmin, 4, cudaMemcpyDeviceToHost, s));
        unsigned long long visited = 0;
        CU_TRY(cudaMemcpyAsync(&visited, counter_at<unsigned long long>(ctx->counters, kCtrBfs) + 1, 8,
                               cudaMemcpyDeviceToHost, s));
        CU_TRY(cudaStreamSynchronize(s));
        const vid_t cmin = ctx->h_st->cmin;
        S.bfs_levels = levels;
        S.bfs_visited = (int64_t)visited;
        S.comp_min = cmin;
        S.bfs_starts = multi ? ctx->h_st->bfs_starts : 1;
        if (multi) S.bfs_edges_inspected = (int64_t)ctx->h_st->bfs_inspected;
        if (!multi) {  // the multi-start BFS set the trees' parents itself
            Scope sc(ctx, CC_K_PARENT_INIT, s, 1);
            launch_parent_init(parent, n, vis, cmin, ctx->grid, s);
        }
        // first SV pass over the pairs the BFS left active (Algorithm 2 lines 8-9): MODE 1
        // after one tree, MODE 2 (one-hop gathers) after several
        const int mode = multi ? 2 : 1;
        cur0 = list_buf == 0 ? 1 : 0;
        {
            Scope sc(ctx, CC_K_SV_FIRST, s, 1);
            if (list_buf < 0)
                launch_sv_pass<T>(mode, true, true, edges, m, n, parent, vis, cmin, hooked, eb[cur0], st, 0,
                                  ctx->grid, s);
            else
                launch_sv_pass<uint32_t>(mode, true, true, eb[list_buf], (long long)list_len, n, parent, vis, cmin,
                                         hooked, eb[cur0], st, 0, ctx->grid, s);
        }
        {
            Scope sc(ctx, CC_K_SV_SHORTCUT, s, 1);
            launch_sv_shortcut(parent, hooked, st, 0, ctx->grid, s);
        }
        S.m_active[0] = (int64_t)list_len;
        CC_TRY(read_back(ctx, &st->kept[0], 8, s));
        m_cur = ctx->h_st->kept[0];
        src = eb[cur0];
    } else if (streamed || deep_done) {
        // SV iterations 1..it0 already ran: per copied chunk (host-input path) or
        // on the side stream during the prediction; the crossing pairs are in ebuf0
        const int it0 = streamed ? pre->it0 : 1;
        S.m_active[0] = m;
        if (deep_done) S.m_active[1] = m;
        if (!ctx->opt.profile) {
            auto pre_none = [&](cudaStream_t) {};
            auto post = [&](cudaStream_t cs) { launch_finalize<T>(parent, n, labels_out, ctx->grid, cs); };
            const cc_ctx::GraphKey key = graph_key(ctx, (sizeof(T) == 4 ? 0 : 1) | 8 | (it0 << 4), n, m, 0, edges,
                                                   nullptr, nullptr, labels_out, cap);
            CC_TRY(launch_sv_graph(ctx, ctx->g_single, key, n, it0, 0, cap, pre_none, post, s));
            rec(ctx, EV_SV, s);
            rec(ctx, EV_END, s);
            return sv_graph_finish(ctx, it0, 0, s);
        }
        it = it0;
        CC_TRY(read_back(ctx, &st->kept[it], 8, s));
        m_cur = ctx->h_st->kept[it];
        src = eb[0];
    } else {
        if (m > 0 && cap >= 2 && !ctx->opt.profile) {
            // the whole SV route as one cached graph with a device-driven loop
            auto pre = [&](cudaStream_t cs) {
                if (!speculated) {
                    launch_parent_init(parent, n, nullptr, 0, ctx->grid, cs);
                    enqueue_first_pass<T>(ctx, edges, n, m, cs, false);
                }
                launch_sv_pass<T>(2, true, true, edges, m, n, parent, nullptr, 0, hooked, eb[0], st, 1, ctx->grid, cs);
                launch_sv_shortcut(parent, hooked, st, 1, ctx->grid, cs);
            };
            auto post = [&](cudaStream_t cs) { launch_finalize<T>(parent, n, labels_out, ctx->grid, cs); };
            const int k = sample_stride(ctx, n, m);
            if (!speculated) S.sv_sample_stride = k;
            const cc_ctx::GraphKey key =
                graph_key(ctx, (sizeof(T) == 4 ? 0 : 1) | (speculated ? 4 : 0) | (speculated ? 0 : k << 16), n, m, 0,
                          edges, nullptr, nullptr, labels_out, cap);
            CC_TRY(launch_sv_graph(ctx, ctx->g_single, key, n, 1, 0, cap, pre, post, s));
            rec(ctx, EV_SV, s);
            rec(ctx, EV_END, s);
            S.m_active[0] = m;
            S.m_active[1] = m;
            // the graph holds parent init and the first pass unless they were speculated
            const int first_launches = speculated ? 0 : 1 + (k > 1 ? 4 : 2);
            return sv_graph_finish(ctx, 1, 2 + first_launches, s);
        }
        if (!speculated) {
            Scope sc(ctx, CC_K_PARENT_INIT, s, 1);
            launch_parent_init(parent, n, nullptr, 0, ctx->grid, s);
        }
        if (m > 0) {
            // every vertex is a root here: hook without recording, then shortcut all vertices
            if (!speculated) enqueue_first_pass<T>(ctx, edges, n, m, s, true);
            S.m_active[0] = m;
            it = 1;
            if (it >= cap) {
                CC_TRY(read_back(ctx, &st->err, 4, s));
                return ctx->h_st->err ? device_error(ctx->h_st->err) : CC_ERR_NO_CONVERGENCE;
            }
            {
                Scope sc(ctx, CC_K_SV_GATHER_INPUT, s, 1);
                launch_sv_pass<T>(2, true, true, edges, m, n, parent, nullptr, 0, hooked, eb[0], st, 1, ctx->grid, s);
            }
            {
                Scope sc(ctx, CC_K_SV_SHORTCUT, s, 1);
                launch_sv_shortcut(parent, hooked, st, 1, ctx->grid, s);
            }
            S.m_active[1] = m;
            CC_TRY(read_back(ctx, &st->kept[1], 8, s));
            m_cur = ctx->h_st->kept[1];
            src = eb[0];
        }
    }
    CC_TRY(sv_list_loop(ctx, n, src, m_cur, it, cap, s, cur0));
    rec(ctx, EV_SV, s);
    {
        Scope sc(ctx, CC_K_FINALIZE, s, 1);
        launch_finalize<T>(parent, n, labels_out, ctx->grid, s);
    }
    rec(ctx, EV_END, s);
    CU_TRY(cudaMemcpyAsync(&ctx->h_st->err, &st->err, 4, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaMemcpyAsync(ctx->h_st->hooked, st->hooked, sizeof(ctx->h_st->hooked), cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    CU_TRY(cudaGetLastError());
    for (int i = 0; i < CC_MAX_SV_ITERS_RECORDED && i <= it; i++) S.sv_hooks[i] = (int64_t)ctx->h_st->hooked[i];
    prof_collect(ctx);
    return device_error(ctx->h_st->err);
}


// ---------------------------------------------------------------------------
// Stream-ordered cc_labels (options.profile == 0). The whole route of
// Algorithm 2 is one CUDA graph in which the device takes every decision the
// host loop takes in the profiled path:
//   * the SV passes that need no route (parent init, the first pass or the
//     sampling front end, SV iteration 1 over the pairs) run speculatively
//     on a side stream while the degree pass and the K-S fit run (the fit on
//     a highest-priority stream); the learned policy runs its sampled
//     features first, and an IF node runs the exact degree pass and the fit
//     only when the network is unsure;
//   * k_route_decide sets an IF node: the BFS branch (the CSR build and the
//     direction-optimizing BFS, or the edge-list BFS, each level one
//     iteration of a WHILE node; then the visited minimum, the parent
//     array and the first SV pass over the pairs the BFS left active);
//   * the SV iterations over the compacted list are a WHILE node that starts
//     after whichever iteration the route left in DevState;
//   * the labels, then a copy of the device state (status word, route,
//     counts) into pinned host memory.
// No host thread waits. The graph is captured once per key (arguments,
// workspace, options) on private streams and launched on the caller's
// stream; if the caller's stream is being captured, the same work is
// captured straight into the caller's graph.

cc_status ensure_streams(cc_ctx *ctx) {
    int least = 0, greatest = 0;
    CU_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    if (!ctx->side_s) CU_TRY(cudaStreamCreateWithPriority(&ctx->side_s, cudaStreamNonBlocking, least));
    if (!ctx->fit_s) CU_TRY(cudaStreamCreateWithPriority(&ctx->fit_s, cudaStreamNonBlocking, greatest));
    if (!ctx->cap_s) CU_TRY(cudaStreamCreateWithFlags(&ctx->cap_s, cudaStreamNonBlocking));
    if (!ctx->cap_s2) CU_TRY(cudaStreamCreateWithFlags(&ctx->cap_s2, cudaStreamNonBlocking));
    if (!ctx->cap_s3) CU_TRY(cudaStreamCreateWithFlags(&ctx->cap_s3, cudaStreamNonBlocking));
    cudaEvent_t *evs[] = {&ctx->ev_fork, &ctx->ev_join, &ctx->ev_fit, &ctx->ev_done};
    for (cudaEvent_t *e : evs)
        if (!*e) CU_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return CC_OK;
}

// A conditional handle in the graph `cs` is capturing into.
cc_status cond_handle(cudaStream_t cs, cudaGraphConditionalHandle *h) {
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    CU_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, &ed, &nd));
    if (cst != cudaStreamCaptureStatusActive) return CC_ERR_CUDA;
    CU_TRY(cudaGraphConditionalHandleCreate(h, g, 0, cudaGraphCondAssignDefault));
    return CC_OK;
}

// Appends a conditional node (IF or WHILE on handle h) to the work captured
// on `cs` so far and captures its body on `bs` with body(bs); `cs` then
// continues after the node.
template <typename Body>
cc_status cond_node(cudaStream_t cs, cudaStream_t bs, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                    Body body) {
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    CU_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, &ed, &nd));
    if (cst != cudaStreamCaptureStatusActive) return CC_ERR_CUDA;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CU_TRY(cudaGraphAddNode(&node, g, deps, ed, nd, &cp));
    CU_TRY(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    CU_TRY(cudaStreamBeginCaptureToGraph(bs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed));
    const cc_status r = body(bs);
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(bs, &out);
    if (r != CC_OK) return r;
    CU_TRY(e);
    return CC_OK;
}

// Whether the small-graph fit (one block) serves a graph (the profiled path's rule).
bool small_fit(vid_t n, long long m, int policy) {
    return n <= (1u << 20) && 2 * m < 4096LL * 4097LL && policy != CC_ROUTE_FORCE_BFS;
}

// Everything the graph depends on besides the device state it reads.
std::vector<unsigned char> route_key(cc_ctx *ctx, int tbytes, long long n, long long m, const void *edges,
                                     void *labels, int cap) {
    struct {
        long long n, m;
        const void *edges, *labels;
        const void *bufs[27];
        cc_options opt;
        double min_conf;
        int tbytes, cap, grid, have_pred;
    } k;
    memset(&k, 0, sizeof(k));
    k.n = n;
    k.m = m;
    k.edges = edges;
    k.labels = labels;
    const Buf *b[] = {&ctx->deg,  &ctx->parent,  &ctx->hooked, &ctx->ebuf0,   &ctx->ebuf1, &ctx->hist,
                      &ctx->ovf,  &ctx->st,      &ctx->dpart,  &ctx->row_ptr, &ctx->col,   &ctx->vis,
                      &ctx->fb,   &ctx->nb,      &ctx->q0,     &ctx->q1,      &ctx->dq,    &ctx->off,
                      &ctx->tsum, &ctx->f_vis,   &ctx->f_f0,   &ctx->f_f1,    &ctx->kb_D,  &ctx->csr_entries,
                      &ctx->bfs_own, &ctx->bfs_tmin, &ctx->bwin};
    for (int i = 0; i < 27; i++) k.bufs[i] = b[i]->p;
    k.opt = ctx->opt;
    k.min_conf = ctx->pred_min_conf;
    k.tbytes = tbytes;
    k.cap = cap;
    k.grid = ctx->grid;
    k.have_pred = ctx->have_pred;
    const unsigned char *p = reinterpret_cast<const unsigned char *>(&k);
    return std::vector<unsigned char>(p, p + sizeof(k));
}

// Captures the route onto `cs` (capturing). Fills the host-side facts in `rg`.
template <typename T>
cc_status enqueue_route(cc_ctx *ctx, const void *edges, vid_t n, long long m, void *labels, int cap, cudaStream_t cs,
                        cc_ctx::RouteGraph &rg) {
    DevState *st = as<DevState>(ctx->st);
    vid_t *parent = as<vid_t>(ctx->parent), *hooked = as<vid_t>(ctx->hooked);
    uint2 *eb0 = as<uint2>(ctx->ebuf0), *eb1 = as<uint2>(ctx->ebuf1);
    const int policy = ctx->opt.route_policy;
    const bool learned = policy == CC_ROUTE_LEARNED && ctx->have_pred;
    const bool multi = multi_start(ctx);
    const bool edge_bfs = learned || multi || ctx->opt.bfs_mode == 1;
    const bool bfs_ok = policy != CC_ROUTE_FORCE_SV && (edge_bfs || 2ull * (unsigned long long)m < 0xffffffffull);
    const bool predict = policy != CC_ROUTE_FORCE_SV;
    const bool speculate = !(policy == CC_ROUTE_FORCE_BFS && bfs_ok);
    const bool small = !learned && small_fit(n, m, policy);
    // the first hook pass inside the windowed degree pass (parent init first)
    const bool fused = predict && !learned && !small && speculate && fused_hooks(ctx, n, m);
    const float min_conf = (float)ctx->pred_min_conf;
    const long long before = ctx->stats.launches;
    long long direct = 0;
    rg.edge_bfs = edge_bfs;
    rg.batched = false;
    rg.level_launches = edge_bfs ? 4 : 11;
    rg.bfs_launches = 0;
    rg.unsure_launches = 0;
    rg.sample_stride = 1;
    ctx->stats.degree_form = 0;
    CU_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), cs));
    if (learned) {
        launch_route_features<T>(edges, m, n, feat_scratch(ctx), st, as<float>(ctx->f_x), ctx->grid, cs);
        mlp_infer(as<__nv_bfloat16>(ctx->pred_wb), as<float>(ctx->pred_bias), as<float>(ctx->f_x), st, cs);
        direct += 12;
    }
    auto speculative = [&](cudaStream_t ss) {
        if (fused) {  // parents initialised and hooked by the degree pass: the full shortcut remains
            launch_shortcut_all(parent, n, st, 0, ctx->grid, ss);
            ctx->stats.sv_sample_stride = 1;
            direct += 1;
        } else {
            launch_parent_init(parent, n, nullptr, 0, ctx->grid, ss);
            direct += 1 + enqueue_first_pass<T>(ctx, edges, n, m, ss, false);
        }
        rg.sample_stride = ctx->stats.sv_sample_stride;
        launch_sv_gather_tiles<T>(edges, m, n, parent, hooked, eb0, st, 1, ss);
        launch_sv_shortcut(parent, hooked, st, 1, ctx->grid, ss);
        direct += 2;
    };
    // the speculative passes fork after the degree pass (both are bound by
    // scattered L2 operations, so running them together gains nothing) and
    // run beside the fit; the learned policy forks them before its features
    auto fork_speculation = [&]() -> cc_status {
        CU_TRY(cudaEventRecord(ctx->ev_fork, cs));
        CU_TRY(cudaStreamWaitEvent(ctx->side_s, ctx->ev_fork, 0));
        speculative(ctx->side_s);
        CU_TRY(cudaEventRecord(ctx->ev_join, ctx->side_s));
        return CC_OK;
    };
    if (!predict && speculate) speculative(cs);  // forced SV: the same passes, nothing to overlap
    if (learned && speculate) CC_TRY(fork_speculation());
    if (learned) {
        cudaGraphConditionalHandle hu;
        CC_TRY(cond_handle(cs, &hu));
        launch_pred_unsure(st, hu, min_conf, cs);
        direct += 1;
        const long long b0 = ctx->stats.launches;
        CC_TRY(cond_node(cs, ctx->cap_s2, hu, cudaGraphCondTypeIf, [&](cudaStream_t bs) -> cc_status {
            enqueue_degree<T>(ctx, edges, n, m, bs);
            enqueue_ks(ctx, bs, distinct_degree_bound(ctx, n, m));
            return CC_OK;
        }));
        rg.unsure_launches = ctx->stats.launches - b0;
        ctx->stats.launches = b0;
    } else if (predict && small) {
        ctx->stats.degree_form = 1;
        CU_TRY(cudaMemsetAsync(ctx->deg.p, 0, (size_t)n * 4, cs));
        launch_degree<T>(edges, m, n, as<uint32_t>(ctx->deg), st, ctx->grid, cs);
        direct += 1;
        // the fit's few blocks are queued ahead of the speculative passes
        CC_TRY(enqueue_small_fit(ctx, n, cs));
        if (speculate) CC_TRY(fork_speculation());
    } else if (predict) {
        if (fused) {
            launch_parent_init(parent, n, nullptr, 0, ctx->grid, cs);
            direct += 1;
        }
        enqueue_degree<T>(ctx, edges, n, m, cs, false, fused ? parent : nullptr);
        if (speculate) CC_TRY(fork_speculation());
        if (policy == CC_ROUTE_AUTO) {
            CU_TRY(cudaEventRecord(ctx->ev_fork, cs));
            CU_TRY(cudaStreamWaitEvent(ctx->fit_s, ctx->ev_fork, 0));
            enqueue_ks(ctx, ctx->fit_s, distinct_degree_bound(ctx, n, m));
            CU_TRY(cudaEventRecord(ctx->ev_fit, ctx->fit_s));
            CU_TRY(cudaStreamWaitEvent(cs, ctx->ev_fit, 0));
        }
    }
    if (speculate && predict) CU_TRY(cudaStreamWaitEvent(cs, ctx->ev_join, 0));
    cudaGraphConditionalHandle hr = cudaGraphConditionalHandle();
    if (bfs_ok) CC_TRY(cond_handle(cs, &hr));  // a handle only where an IF node will use it
    launch_route_decide(st, bfs_ok ? &hr : nullptr, policy, bfs_ok ? 1 : 0, ctx->opt.bfs_cutoff_levels, min_conf,
                        learned ? 1 : 0, cs);
    direct += 1;
    if (bfs_ok) {
        CC_TRY(cond_node(cs, ctx->cap_s2, hr, cudaGraphCondTypeIf, [&](cudaStream_t bs) -> cc_status {
            const long long nwords = ((long long)n + 31) / 32;
            // the speculative SV iterations' counters start over
            CU_TRY(cudaMemsetAsync(&st->kept[0], 0, offsetof(DevState, front) - offsetof(DevState, kept), bs));
            const uint32_t *vis;
            uint32_t *own = multi ? as<uint32_t>(ctx->bfs_own) : nullptr;
            if (edge_bfs) {
                uint32_t *fv = as<uint32_t>(ctx->f_vis), *f0 = as<uint32_t>(ctx->f_f0), *f1 = as<uint32_t>(ctx->f_f1);
                cudaGraphConditionalHandle hb;
                CC_TRY(cond_handle(bs, &hb));
                if (multi) {
                    launch_mbfs_start(as<uint32_t>(ctx->deg), n, m, ctx->opt.bfs_starts, fv, f0, own,
                                      as<uint32_t>(ctx->bfs_tmin), st, &hb, bs);
                    rg.bfs_launches += 2;
                } else {
                    CU_TRY(cudaMemsetAsync(fv, 0, (size_t)nwords * 4, bs));
                    CU_TRY(cudaMemsetAsync(f0, 0, (size_t)nwords * 4, bs));
                    launch_ebfsg_init(fv, f0, n, m, st, hb, bs);
                    rg.bfs_launches += 1;
                }
                CC_TRY(cond_node(bs, ctx->cap_s3, hb, cudaGraphCondTypeWhile, [&](cudaStream_t ls) -> cc_status {
                    launch_ebfsg_level<T>(edges, m, eb0, eb1, n, fv, f0, f1, st, hb, ctx->grid, ls, own);
                    return CC_OK;
                }));
                vis = fv;
            } else {
                uint32_t *row_ptr = as<uint32_t>(ctx->row_ptr), *deg = as<uint32_t>(ctx->deg);
                vid_t *col = as<vid_t>(ctx->col);
                const bool bucketed = bucketed_ok(n, (size_t)m) && ctx->csr_entries.p;
                launch_scan_u32(deg, n, row_ptr, deg, as<unsigned long long>(ctx->tsum), nullptr, row_ptr + n, bs);
                if (bucketed)
                    launch_csr_bucketed<T>(edges, m, n, row_ptr, deg, col, bucket_scratch(ctx),
                                           as<unsigned long long>(ctx->csr_entries), st, ctx->grid, bs);
                else
                    launch_csr_scatter<T>(edges, m, n, deg, col, ctx->grid, bs);
                rg.bfs_launches += 3 + (bucketed ? 2 : 1) + 1;  // the scan, the CSR, the BFS state
                uint32_t *vm = as<uint32_t>(ctx->vis);
                CU_TRY(cudaMemsetAsync(vm, 0, (size_t)nwords * 4, bs));
                cudaGraphConditionalHandle hb;
                CC_TRY(cond_handle(bs, &hb));
                launch_bfsg_init(row_ptr, n, vm, as<vid_t>(ctx->q0), st, hb, bs);
                CC_TRY(cond_node(bs, ctx->cap_s3, hb, cudaGraphCondTypeWhile, [&](cudaStream_t ls) -> cc_status {
                    launch_bfsg_level(n, 2ull * (unsigned long long)m, row_ptr, col, vm, as<vid_t>(ctx->q0),
                                      as<vid_t>(ctx->q1), as<uint32_t>(ctx->fb), as<uint32_t>(ctx->nb),
                                      as<uint32_t>(ctx->dq), as<uint32_t>(ctx->off), as<unsigned long long>(ctx->tsum),
                                      st, hb, ctx->grid, ls);
                    return CC_OK;
                }));
                vis = vm;
            }
            launch_popcount(vis, nwords, &st->bfs_visited, ctx->grid, bs);
            launch_first_visited(vis, nwords, st, ctx->grid, bs);
            if (multi) launch_mbfs_finish(own, as<uint32_t>(ctx->bfs_tmin), n, parent, ctx->grid, bs);
            else launch_parent_init_st(parent, n, vis, st, ctx->grid, bs);
            rg.bfs_launches += 2 + (multi ? 2 : 1) +
                               launch_sv_after_bfs<T>(edges, m, eb0, eb1, n, parent, vis, hooked, st, ctx->grid, bs,
                                                      multi);
            launch_sv_shortcut(parent, hooked, st, 0, ctx->grid, bs);
            rg.bfs_launches += 1;
            return CC_OK;
        }));
    }
    cudaGraphConditionalHandle hs;
    CC_TRY(cond_handle(cs, &hs));
    launch_sv_loop_init_st(st, cap, hs, cs);
    CC_TRY(cond_node(cs, ctx->cap_s2, hs, cudaGraphCondTypeWhile, [&](cudaStream_t bs) -> cc_status {
        launch_sv_loop_body(eb0, eb1, n, parent, hooked, st, hs, ctx->grid, bs);
        return CC_OK;
    }));
    launch_finalize<T>(parent, n, labels, ctx->grid, cs);
    direct += 2;
    CU_TRY(cudaMemcpyAsync(ctx->h_st, st, offsetof(DevState, hook_base), cudaMemcpyDeviceToHost, cs));
    rg.degree_form = ctx->stats.degree_form;
    rg.static_launches = ctx->stats.launches - before + direct;
    return CC_OK;
}

// Workspace of the route for every branch it may take (allocated before any capture).
cc_status ensure_route(cc_ctx *ctx, vid_t n, long long m) {
    const int policy = ctx->opt.route_policy;
    const bool learned = policy == CC_ROUTE_LEARNED && ctx->have_pred;
    if (multi_start(ctx) && policy != CC_ROUTE_FORCE_SV) CC_TRY(ensure_mbfs(ctx, n));
    else if (learned || ctx->opt.bfs_mode == 1) CC_TRY(ensure_feat(ctx, n));
    else if (policy != CC_ROUTE_FORCE_SV && 2ull * (unsigned long long)m < 0xffffffffull)
        CC_TRY(ensure_bfs(ctx, n, (size_t)m));
    if (!learned && small_fit(n, m, policy) && policy != CC_ROUTE_FORCE_SV) CC_TRY(ensure_batch_route(ctx, 1, 1));
    return CC_OK;
}

// Statistics of a graph-mode call from the device state copied to h_st.
void stats_from_device(cc_ctx *ctx) {
    const DevState *h = ctx->h_st;
    const cc_ctx::RouteGraph &rg = ctx->rg_last ? *ctx->rg_last : ctx->g_route;
    cc_stats &S = ctx->stats;
    S.route = h->route_taken;
    S.route_source = h->route_source;
    S.ks_d = h->ks_out[0];
    S.ks_alpha = h->ks_out[1];
    S.ks_xmin = (int64_t)h->ks_out[2];
    S.ks_ntail = (int64_t)h->ks_out[3];
    S.ks_ncand = (int64_t)h->ks_out[4];
    S.max_degree = (int64_t)(h->maxkey >> 32);
    S.seed_vertex = h->maxkey ? (int64_t)(0xffffffffu - (uint32_t)(h->maxkey & 0xffffffffu)) : 0;
    if (h->route_source == 2 && h->route_taken) S.ks_d = 0.0;
    S.pred_route = ctx->opt.route_policy == CC_ROUTE_LEARNED && ctx->have_pred ? h->pred_route : -1;
    S.pred_confidence = h->pred_conf;
    S.pred_cutoff = h->pred_cutoff;
    S.sv_iters = h->loop_done;
    // the SV loop continues after iteration 0 (BFS route) or 1 (SV route; always in the batched form)
    const int it0 = h->route_taken && !rg.batched ? 0 : 1;
    if (rg.batched) {
        S.batch_unroll = rg.batch_unroll;
        S.batch_grid_mult = rg.batch_grid_mult;
        S.batch_deg_regions = rg.batch_deg_regions;
        S.batch_sv_regions = rg.batch_sv_regions;
        S.route_source = ctx->opt.route_policy == CC_ROUTE_AUTO || ctx->opt.route_policy == CC_ROUTE_LEARNED ? 0 : 2;
        S.bfs_levels = h->route_taken ? h->bfs_level : 0;
        S.m_active[0] = S.m;
        S.m_active[1] = S.m;
        S.ks_d = 0.0;
        S.pred_route = -1;
    } else if (h->route_taken) {
        S.bfs_levels = h->bfs_level;
        S.bfs_starts = h->bfs_starts > 0 ? h->bfs_starts : 1;
        S.bfs_visited = (int64_t)h->bfs_visited;
        S.comp_min = h->cmin;
        S.bfs_edges_inspected = (int64_t)h->bfs_inspected;
        S.m_active[0] = rg.edge_bfs && h->bfs_list >= 0 ? (int64_t)h->bfs_len : S.m;
    } else {
        S.m_active[0] = S.m;
        S.m_active[1] = S.m;
    }
    for (int i = it0 + 1; i < h->loop_done && i < CC_MAX_SV_ITERS_RECORDED; i++) S.m_active[i] = (int64_t)h->kept[i - 1];
    for (int i = 0; i < h->loop_done && i < CC_MAX_SV_ITERS_RECORDED; i++) S.sv_hooks[i] = (int64_t)h->hooked[i];
    S.sv_sample_stride = rg.sample_stride;
    S.degree_form = rg.batched || h->route_source == 1 ? 0 : rg.degree_form;
    const long long loops = h->loop_done > it0 + 1 ? h->loop_done - it0 - 1 : 0;
    const bool unsure = h->route_source != 1;  // the learned policy ran the exact prediction
    S.launches = rg.static_launches + (unsure ? rg.unsure_launches : 0) +
                 (h->route_taken ? (long long)h->bfs_level * rg.level_launches + rg.bfs_launches : 0) + 3 * loops;
    S.status = device_error(h->err);
}

template <typename T>
cc_status labels_graph(cc_ctx *ctx, const void *edges, vid_t n, long long m, void *labels, cudaStream_t s) {
    cc_stats &S = ctx->stats;
    const int cap = ctx->opt.fault_inject & CC_FAULT_ITER_CAP ? 1
                    : ctx->opt.max_iters > 0                  ? ctx->opt.max_iters
                                                              : default_max_iters(n);
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    CU_TRY(cudaStreamIsCapturing(s, &cst));
    const bool user_capture = cst == cudaStreamCaptureStatusActive;
    cc_status prior = CC_OK;
    if (!user_capture && ctx->async_outstanding && cudaEventQuery(ctx->ev_done) == cudaSuccess) {
        prior = device_error(ctx->h_st->err);  // an earlier call's device error, reported once
        ctx->async_outstanding = false;
    }
    cudaGetLastError();
    memset(&S, 0, sizeof(S));
    prof_reset(ctx);
    for (int e = 0; e < EV_COUNT; e++) ctx->ev_used[e] = false;
    S.n = n;
    S.m = m;
    ctx->graph_last = true;
    if (user_capture) {
        // captured into the caller's graph: nothing may allocate or wait
        ctx->capturing = true;
        cc_status r = ensure_route(ctx, n, m);
        if (r == CC_OK) r = enqueue_route<T>(ctx, edges, n, m, labels, cap, s, ctx->g_capture);
        ctx->capturing = false;
        ctx->rg_last = &ctx->g_capture;
        return r;
    }
    CC_TRY(ensure_route(ctx, n, m));
    std::vector<unsigned char> key = route_key(ctx, (int)sizeof(T), n, m, edges, labels, cap);
    cc_ctx::RouteGraph &rg = ctx->g_route;
    if (!rg.exec || rg.key != key) {
        if (rg.exec) cudaGraphExecDestroy(rg.exec);
        rg.exec = nullptr;
        CU_TRY(cudaStreamBeginCapture(ctx->cap_s, cudaStreamCaptureModeRelaxed));
        const cc_status r = enqueue_route<T>(ctx, edges, n, m, labels, cap, ctx->cap_s, rg);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ctx->cap_s, &g);
        if (r != CC_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return r != CC_OK ? r : CC_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&rg.exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            cudaGetLastError();
            rg.exec = nullptr;
            return CC_ERR_CUDA;
        }
        rg.key.swap(key);
    }
    ctx->rg_last = &rg;
    rec(ctx, EV_START, s);
    CU_TRY(cudaGraphLaunch(rg.exec, s));
    rec(ctx, EV_END, s);
    CU_TRY(cudaEventRecord(ctx->ev_done, s));
    ctx->async_outstanding = true;
    if (ctx->opt.debug_checks) {
        CU_TRY(cudaStreamSynchronize(s));
        ctx->async_outstanding = false;
        return device_error(ctx->h_st->err);
    }
    return prior;
}

// Host-input form. The pairs are copied in chunks on a copy stream; the
// host link (about 210 GB/s on GB300) is the bound, so the passes that need
// only the pairs seen so far run under the copy, each chunk as it lands:
//   on `s`:    the degree count (K-S route), chunk by chunk;
//   side:      one SV iteration per chunk over that chunk's pairs, with the
//              ends chased to their current roots (MODE 3), the crossing
//              pairs appended to one list and the hooked roots shortcut;
//              after the last chunk a full shortcut.
// After the copy the route is predicted from the complete histogram; the SV
// route continues with the appended list (every pair that crossed roots
// when read is in it, so no connection is lost), the BFS route starts from
// the device copy and re-initialises the parent array.
// The per-chunk iterations reorder the hooks of Section 3.1's iterations
// (a chunk's pairs see the forest the earlier chunks built); the labels are
// the same.
constexpr long long kPipeChunkPairs = 1LL << 23;  // 64 MB of int32 pairs; even, and >= the hub prefix
constexpr long long kPipeMinPairs = 1LL << 24;
constexpr int kPipeMaxChunks = 32;

cc_status ensure_copy(cc_ctx *ctx, int chunks) {
    if (!ctx->copy_s) CU_TRY(cudaStreamCreateWithFlags(&ctx->copy_s, cudaStreamNonBlocking));
    while ((int)ctx->ev_chunk.size() < chunks) {
        cudaEvent_t e = nullptr;
        CU_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->ev_chunk.push_back(e);
    }
    return CC_OK;
}

template <typename T>
cc_status labels_host_impl(cc_ctx *ctx, const void *edges_host, vid_t n, long long m, void *labels_host,
                           cudaStream_t s) {
    char *dev = static_cast<char *>(ctx->hedges.p);
    const char *host = static_cast<const char *>(edges_host);
    const size_t pb = 2 * sizeof(T);
    const int policy = ctx->opt.route_policy;
    const bool pipelined = m >= kPipeMinPairs && (policy == CC_ROUTE_AUTO || policy == CC_ROUTE_FORCE_SV) &&
                           ctx->opt.max_iters == 0 && ctx->opt.fault_inject == 0;
    cc_status rc;
    if (!pipelined) {
        if (m > 0) CU_TRY(cudaMemcpyAsync(dev, host, (size_t)m * pb, cudaMemcpyHostToDevice, s));
        rc = labels_impl<T>(ctx, dev, n, m, ctx->hlabels.p, s);
    } else {
        // chunks of C pairs (even, so each chunk starts on a 16-byte boundary), at most kPipeMaxChunks
        long long C = (m + kPipeMaxChunks - 1) / kPipeMaxChunks;
        C = C < kPipeChunkPairs ? kPipeChunkPairs : (C + 1) & ~1LL;
        const int chunks = (int)((m + C - 1) / C);
        CC_TRY(ensure_side(ctx));
        CC_TRY(ensure_copy(ctx, chunks));
        DevState *st = as<DevState>(ctx->st);
        vid_t *parent = as<vid_t>(ctx->parent), *hooked = as<vid_t>(ctx->hooked);
        uint2 *list = as<uint2>(ctx->ebuf0);
        uint32_t *deg = as<uint32_t>(ctx->deg);
        cudaStream_t cp = ctx->copy_s, side = ctx->side_s;
        Staged pre;
        CU_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), s));
        rec(ctx, EV_START, s);
        const bool count = policy == CC_ROUTE_AUTO;
        if (count) {
            CU_TRY(cudaMemsetAsync(ctx->hist.p, 0, (size_t)kHistDense * 4, s));
            CU_TRY(cudaMemsetAsync(deg, 0, (size_t)n * 4, s));
        }
        CU_TRY(cudaEventRecord(ctx->ev_fork, s));
        CU_TRY(cudaStreamWaitEvent(cp, ctx->ev_fork, 0));
        CU_TRY(cudaStreamWaitEvent(side, ctx->ev_fork, 0));
        for (int i = 0; i < chunks; i++) {
            const long long off = (long long)i * C;
            const long long len = m - off < C ? m - off : C;
            CU_TRY(cudaMemcpyAsync(dev + off * pb, host + off * pb, (size_t)len * pb, cudaMemcpyHostToDevice, cp));
            CU_TRY(cudaEventRecord(ctx->ev_chunk[i], cp));
        }
        launch_parent_init(parent, n, nullptr, 0, ctx->grid, side);
        pre.launches++;
        // Whole SV iterations per chunk pay off while the parent array stays in
        // L2 (their root chases are then L2 hits); above 2^25 vertices each
        // chunk only takes the first pass, which needs no chase.
        const bool stream_sv = n <= (1u << 25);
        // the hub table lives in ebuf1: ebuf0 receives the crossing pairs
        const bool hubs = degree_uses_hubs(m) && ctx->ebuf1.bytes >= degree_hubs_scratch_bytes();
        unsigned *scratch = as<unsigned>(ctx->ebuf1);
        for (int i = 0; i < chunks; i++) {
            const long long off = (long long)i * C;
            const long long len = m - off < C ? m - off : C;
            const char *chunk = dev + off * pb;
            if (count) {
                CU_TRY(cudaStreamWaitEvent(s, ctx->ev_chunk[i], 0));
                if (!hubs) {
                    launch_degree<T>(chunk, len, n, deg, st, ctx->grid, s);
                    pre.launches++;
                } else if (i == 0) {
                    const long long p0 = degree_hub_prefix();
                    launch_degree_hub_prefix<T>(chunk, n, deg, scratch, st, ctx->grid, s);
                    launch_degree_hub_count<T>(chunk + p0 * pb, len - p0, n, deg, scratch, st, ctx->num_sms, s);
                    pre.launches += 5;
                } else {
                    launch_degree_hub_count<T>(chunk, len, n, deg, scratch, st, ctx->num_sms, s);
                    pre.launches++;
                }
            }
            CU_TRY(cudaStreamWaitEvent(side, ctx->ev_chunk[i], 0));
            if (stream_sv) {
                // SV iteration i + 1 over this chunk, appended after the earlier chunks' surviving pairs
                launch_sv_pass<T>(3, true, true, chunk, len, n, parent, nullptr, 0, hooked, list, st, i + 1,
                                  ctx->grid, side);
                launch_sv_shortcut(parent, hooked, st, i + 1, ctx->grid, side);
                pre.launches += 2;
            } else {
                // the first SV pass (every vertex its own root) over this chunk
                launch_sv_pass<T>(first_pass_mode(n, m), false, false, chunk, len, n, parent, nullptr, 0, hooked,
                                  nullptr, st, 0, ctx->grid, side);
                pre.launches++;
            }
        }
        if (stream_sv) {
            launch_shortcut_all(parent, n, st, chunks, ctx->grid, side);
            launch_stream_finish(st, chunks, side);
        } else {
            launch_shortcut_all(parent, n, st, 0, ctx->grid, side);
        }
        pre.launches += stream_sv ? 2 : 1;
        CU_TRY(cudaEventRecord(ctx->ev_join, side));
        // `s` continues after every chunk has landed (the later passes read all pairs)
        CU_TRY(cudaStreamWaitEvent(s, ctx->ev_chunk[chunks - 1], 0));
        pre.degree_counted = count;
        pre.streamed = stream_sv;
        pre.first_pass_done = !stream_sv;
        pre.it0 = stream_sv ? chunks : 0;
        rc = labels_impl<T>(ctx, dev, n, m, ctx->hlabels.p, s, &pre);
    }
    if (rc != CC_OK) return rc;
    CU_TRY(cudaMemcpyAsync(labels_host, ctx->hlabels.p, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    return CC_OK;
}

// ---------------------------------------------------------------------------
// The batched degree pass takes its tiles in order from a device counter;
// null keeps the grid stride. Measured on 4,096 graphs: degree pass 38.8 ms
// with the stride, 33.2 ms in order. The batched hook passes keep the
// stride: with the counter (two more barriers per tile) the gather pass went
// from 23.9 to 26.7 ms.
unsigned long long *tile_queue(cc_ctx *ctx) {
    return counter_at<unsigned long long>(ctx->counters, kCtrTileQueue);
}

// The degree pass of a batch in shared-memory windows when its scratch is
// reserved (ensure_batch_win, before any capture), else one L2 atomic per
// endpoint (k_degree_batch, `regions` of the pairs side by side). With `hook`
// either applies the first hook pass as well. Returns true for the windows.
bool batch_win(const cc_ctx *ctx, long long m, long long n, int G) {
    return degree_batch_win_ok(m, n) && ctx->bwin.bytes >= batch_win_scratch_bytes(m, n, G);
}

cc_status ensure_batch_win(cc_ctx *ctx, long long m, long long n, int G) {
    if (!degree_batch_win_ok(m, n)) return CC_OK;
    return buf_reserve(ctx, ctx->bwin, batch_win_scratch_bytes(m, n, G));
}

bool enqueue_batch_degree(cc_ctx *ctx, const int32_t *edges, long long m, const int64_t *eo, const int64_t *vo, int G,
                          long long n, int regions, cudaStream_t s, vid_t *hook) {
    DevState *st = as<DevState>(ctx->st);
    if (batch_win(ctx, m, n, G)) {
        launch_degree_batch_win(edges, m, eo, vo, G, n, as<uint32_t>(ctx->tile_pairs), as<uint32_t>(ctx->deg), st,
                                ctx->bwin.p, ctx->num_sms, s, hook);
        return true;
    }
    launch_degree_batch(edges, m, eo, vo, G, as<uint32_t>(ctx->deg), st, ctx->grid, tile_queue(ctx), regions, s, hook);
    return false;
}

// Schedule tuner of the batched form. The hook passes over a batch map each
// tile of pairs to its graph, and how many pairs a thread carries per tile
// (amortising that lookup and keeping loads in flight) against how many
// blocks share the work depends on the mix of graph sizes. On the first
// call of a shape (log2 of the pairs and of the graph count) every
// candidate schedule times the first hook pass, which is idempotent after a
// parent reset (every vertex its own root), with CUDA events on the
// caller's stream; the fastest is kept for the context. Small batches keep
// the default (tuning would cost more than it saves).
cc_status ensure_tiles(cc_ctx *ctx, const int64_t *eo_dev, const int64_t *vo_dev, int G, long long m, long long n,
                       cudaStream_t s) {
    CC_TRY(buf_reserve(ctx, ctx->tile_pairs, (size_t)((m >> kTileShift) + 2) * 4));
    CC_TRY(buf_reserve(ctx, ctx->tile_verts, (size_t)((n >> kTileShift) + 2) * 4));
    launch_tile_graphs(eo_dev, G, m, as<uint32_t>(ctx->tile_pairs), ctx->grid, s);
    launch_tile_graphs(vo_dev, G, n, as<uint32_t>(ctx->tile_verts), ctx->grid, s);
    return CC_OK;
}

int ilog2_ceil(long long x) {
    int l = 0;
    while (l < 62 && (1LL << l) < x) l++;
    return l;
}

// options.batch_hook_regions overrides the tuned tile order of the hook passes
void hook_order(cc_ctx *ctx, BatchSchedule *sch) {
    const int k = ctx->opt.batch_hook_regions;
    if (k == 0) return;
    sch->sv_regions = k > 0 ? k : 0;
    sch->queue = counter_at<unsigned long long>(ctx->counters, kCtrSvQueue);
}

cc_status tune_batch(cc_ctx *ctx, const int32_t *edges, long long m, const int64_t *eo, const int64_t *vo, int G,
                     vid_t nt, cudaStream_t s, BatchSchedule *out) {
    *out = BatchSchedule();
    out->pair_tiles = as<uint32_t>(ctx->tile_pairs);
    out->queue = counter_at<unsigned long long>(ctx->counters, kCtrSvQueue);
    if (m < (1LL << 24)) return CC_OK;
    const int key = (ilog2_ceil(m) << 8) | ilog2_ceil(G);
    for (const auto &e : ctx->batch_tuned)
        if (e.first == key) {
            *out = e.second;
            return CC_OK;
        }
    // (unroll, grid multiple, regions): grid-stride schedules, and tiles in
    // region order from a counter (the grid multiple does not apply there)
    const int cand_spec[][3] = {{1, 1, 0}, {2, 1, 0}, {4, 1, 0}, {1, 2, 0}, {2, 2, 0},
                                {4, 2, 0}, {2, 1, 8}, {2, 1, 32}, {4, 1, 8}};
    std::vector<BatchSchedule> cand;
    for (const auto &c : cand_spec) {
        BatchSchedule b;
        b.unroll = c[0];
        b.grid_mult = c[1];
        b.sv_regions = c[2];
        b.queue = counter_at<unsigned long long>(ctx->counters, kCtrSvQueue);
        b.pair_tiles = as<uint32_t>(ctx->tile_pairs);
        cand.push_back(b);
    }
    DevState *st = as<DevState>(ctx->st);
    vid_t *parent = as<vid_t>(ctx->parent), *hooked = as<vid_t>(ctx->hooked);
    uint2 *eb0 = as<uint2>(ctx->ebuf0);
    cudaEvent_t a = pool_event(ctx), b = pool_event(ctx);
    if (!a || !b) return CC_OK;
    float best = 1e30f;
    // each candidate runs the first two passes of the route (idempotent after
    // a reset of the parents and the device state): the hook pass over all
    // pairs, the full shortcut and the gather pass that writes the survivors
    for (const BatchSchedule &c : cand) {
        launch_parent_init(parent, nt, nullptr, 0, ctx->grid, s);
        CU_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), s));
        CU_TRY(cudaEventRecord(a, s));
        launch_sv_pass_batch(0, edges, m, eo, vo, G, nt, parent, hooked, nullptr, st, 0, ctx->grid, s, c);
        launch_shortcut_all(parent, nt, st, 0, ctx->grid, s);
        launch_sv_pass_batch(2, edges, m, eo, vo, G, nt, parent, hooked, eb0, st, 1, ctx->grid, s, c);
        CU_TRY(cudaEventRecord(b, s));
        CU_TRY(cudaEventSynchronize(b));
        float ms = 0.f;
        CU_TRY(cudaEventElapsedTime(&ms, a, b));
        if (ms < best) {
            best = ms;
            *out = c;
        }
    }
    // the degree pass (idempotent after a reset of the counts): regions of
    // the pairs worked on side by side (the windowed pass has no regions: 0)
    if (batch_win(ctx, m, nt, G)) {
        out->deg_regions = 0;
    } else if (ctx->deg.p && ctx->deg.bytes >= (size_t)nt * 4) {
        float best_deg = 1e30f;
        for (int regions : {1, 8, 32}) {
            CU_TRY(cudaMemsetAsync(ctx->deg.p, 0, (size_t)nt * 4, s));
            CU_TRY(cudaEventRecord(a, s));
            launch_degree_batch(edges, m, eo, vo, G, as<uint32_t>(ctx->deg), st, ctx->grid, tile_queue(ctx), regions,
                                s);
            CU_TRY(cudaEventRecord(b, s));
            CU_TRY(cudaEventSynchronize(b));
            float ms = 0.f;
            CU_TRY(cudaEventElapsedTime(&ms, a, b));
            if (ms < best_deg) {
                best_deg = ms;
                out->deg_regions = regions;
            }
        }
    }
    CU_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), s));
    ctx->batch_tuned.push_back({key, *out});
    return CC_OK;
}

// ---------------------------------------------------------------------------
// Per-graph route prediction of the batched form (Algorithm 2 lines 1-3 for
// each graph): k_ks_batch fits every graph in one launch; a graph with more
// vertices of high degree than its shared-memory list holds takes the
// single-graph fit on its degree slice instead. Outputs stay on the device
// (kb_*), the routes and seeds are also returned on the host.
// blocks: scratch for this many k_ks_batch blocks (0 = a full grid, 3 per SM)
cc_status ensure_batch_route(cc_ctx *ctx, int G, int blocks) {
    const int want = blocks > 0 ? blocks : ctx->num_sms * 3;  // 3 blocks of k_ks_batch fit on an SM
    if (want > ctx->kb_blocks) ctx->kb_blocks = want;
    const size_t E = ks_batch_entries(), B = (size_t)ctx->kb_blocks;
    CC_TRY(buf_reserve(ctx, ctx->kb_xs, B * E * 4));
    CC_TRY(buf_reserve(ctx, ctx->kb_cnt, B * E * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_cum, B * (E + 1) * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_lnx, B * E * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_Dc, B * E * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_Ac, B * E * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_Zc, B * E * 8));
    const size_t g = (size_t)G + 1;
    CC_TRY(buf_reserve(ctx, ctx->kb_D, g * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_alpha, g * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_xmin, g * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_ntail, g * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_ncand, g * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_route, g * 4));
    CC_TRY(buf_reserve(ctx, ctx->kb_ovf, g * 4));
    CC_TRY(buf_reserve(ctx, ctx->kb_seed, g * 8));
    return CC_OK;
}

// deg holds the union degrees. Fills kb_* for every graph and returns the
// routes (1 = BFS first) in `route` (host, G entries).
// The batched route: the per-graph fits run on a highest-priority stream
// beside the first hook pass, which keeps its resident grid. Measured on
// 4,096 graphs while the fits took 25 ms: 107 ms with the fits after the
// pass, 105.7 beside a resident-grid pass, 103.2 beside a pass launched one
// block per tile (so that the fits get SMs as its blocks retire). Once the
// fits took 2.7 ms: 89.8 ms with the tile-block pass, 88.2 with the resident
// grid (the tile blocks cost more than the overlap saves).

// One K-S fit per graph on stream s (the degrees of every graph are in
// ctx->deg); the blocks take the graphs largest first.
cc_status enqueue_ks_batch(cc_ctx *ctx, const int64_t *vo_dev, const int64_t *vo_host, int G, cudaStream_t s) {
    CC_TRY(buf_reserve(ctx, ctx->kb_order, (size_t)(G > 0 ? G : 1) * 4));
    std::vector<int> order((size_t)G);
    for (int g = 0; g < G; g++) order[g] = g;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return vo_host[a + 1] - vo_host[a] > vo_host[b + 1] - vo_host[b];
    });
    // pageable source: the copy is staged before the call returns
    CU_TRY(cudaMemcpyAsync(ctx->kb_order.p, order.data(), (size_t)G * 4, cudaMemcpyHostToDevice, s));
    int *next = counter_at<int>(ctx->counters, kCtrKsQueue);
    KsBatchScratch sc{as<uint32_t>(ctx->kb_xs), as<unsigned long long>(ctx->kb_cnt), as<unsigned long long>(ctx->kb_cum),
                      as<double>(ctx->kb_lnx), as<double>(ctx->kb_Dc), as<double>(ctx->kb_Ac), as<double>(ctx->kb_Zc)};
    KsBatchOut out{as<double>(ctx->kb_D),     as<double>(ctx->kb_alpha), as<long long>(ctx->kb_xmin),
                   as<long long>(ctx->kb_ntail), as<long long>(ctx->kb_ncand), as<int>(ctx->kb_route),
                   as<int>(ctx->kb_ovf),      as<unsigned long long>(ctx->kb_seed)};
    Scope sc2(ctx, CC_K_KS, s, 1);
    launch_ks_batch(as<uint32_t>(ctx->deg), vo_dev, G, sc, out, ctx->opt.ks_min_tail, ctx->opt.ks_min_distinct,
                    ctx->opt.ks_min_span, ctx->opt.ks_tau, ctx->kb_blocks, as<int>(ctx->kb_order), next, s);
    return CC_OK;
}

// The per-graph routes of the fits enqueue_ks_batch queued before the work
// on s; graphs the batched fit flagged take the single-graph fit here.
cc_status batch_routes(cc_ctx *ctx, const int64_t *vo_host, int G, std::vector<int> &route, cudaStream_t s) {
    DevState *st = as<DevState>(ctx->st);
    route.assign((size_t)G, 0);
    std::vector<int> ovf((size_t)G, 0);
    CU_TRY(cudaMemcpyAsync(route.data(), ctx->kb_route.p, (size_t)G * 4, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaMemcpyAsync(ovf.data(), ctx->kb_ovf.p, (size_t)G * 4, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaMemcpyAsync(&ctx->h_st->err, &st->err, 4, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    if (ctx->h_st->err) return device_error(ctx->h_st->err);
    KsScratch ks{as<uint32_t>(ctx->ks_xs), as<unsigned long long>(ctx->ks_cnt), as<unsigned long long>(ctx->ks_cum),
                 as<double>(ctx->ks_lnx), as<double>(ctx->ks_Dc), as<double>(ctx->ks_Ac), as<double>(ctx->ks_Zc),
                 as<float>(ctx->ks_Df), as<unsigned long long>(ctx->chunk_nz), as<unsigned long long>(ctx->chunk_mass),
                 ctx->ks_cap};
    for (int g = 0; g < G; g++) {
        if (!ovf[g]) continue;
        // the single-graph histogram and fit on this graph's degree slice, copied
        // to the (idle, n-word) hooked-root buffer: k_hist reads 16-byte vectors
        const long long ng = vo_host[g + 1] - vo_host[g];
        uint32_t *slice = as<uint32_t>(ctx->hooked);
        CU_TRY(cudaMemsetAsync(st, 0, offsetof(DevState, kept), s));
        CU_TRY(cudaMemsetAsync(ctx->hist.p, 0, (size_t)kHistDense * 4, s));
        CU_TRY(cudaMemcpyAsync(slice, as<uint32_t>(ctx->deg) + vo_host[g], (size_t)ng * 4, cudaMemcpyDeviceToDevice, s));
        launch_hist(slice, (vid_t)ng, as<uint32_t>(ctx->hist), as<uint32_t>(ctx->ovf), ctx->ovf_cap, st, ctx->grid, s);
        launch_ks(as<uint32_t>(ctx->hist), as<uint32_t>(ctx->ovf), ctx->ovf_cap, ks, st, ctx->opt.ks_min_tail,
                  ctx->opt.ks_min_distinct, ctx->opt.ks_min_span, ctx->opt.ks_tau, ctx->ks_cap, ctx->grid, s);
        CU_TRY(cudaMemcpyAsync(ctx->h_st, st, offsetof(DevState, kept), cudaMemcpyDeviceToHost, s));
        CU_TRY(cudaStreamSynchronize(s));
        if (ctx->h_st->err) return device_error(ctx->h_st->err);
        const DevState *h = ctx->h_st;
        route[g] = h->route;
        const double D = h->ks_out[0], alpha = h->ks_out[1];
        const long long xmin = (long long)h->ks_out[2], ntail = (long long)h->ks_out[3],
                        ncand = (long long)h->ks_out[4];
        const unsigned long long seed = h->maxkey;
        CU_TRY(cudaMemcpyAsync(as<double>(ctx->kb_D) + g, &D, 8, cudaMemcpyHostToDevice, s));
        CU_TRY(cudaMemcpyAsync(as<double>(ctx->kb_alpha) + g, &alpha, 8, cudaMemcpyHostToDevice, s));
        CU_TRY(cudaMemcpyAsync(as<long long>(ctx->kb_xmin) + g, &xmin, 8, cudaMemcpyHostToDevice, s));
        CU_TRY(cudaMemcpyAsync(as<long long>(ctx->kb_ntail) + g, &ntail, 8, cudaMemcpyHostToDevice, s));
        CU_TRY(cudaMemcpyAsync(as<long long>(ctx->kb_ncand) + g, &ncand, 8, cudaMemcpyHostToDevice, s));
        CU_TRY(cudaMemcpyAsync(as<int>(ctx->kb_route) + g, &route[g], 4, cudaMemcpyHostToDevice, s));
        CU_TRY(cudaMemcpyAsync(as<unsigned long long>(ctx->kb_seed) + g, &seed, 8, cudaMemcpyHostToDevice, s));
        CU_TRY(cudaStreamSynchronize(s));  // the host values above go out of scope
    }
    return CC_OK;
}

// ---------------------------------------------------------------------------
// Stream-ordered batched form (options.profile == 0): the route prediction of
// every graph, the BFS step of the graphs routed to it and the SV over the
// union as one CUDA graph, decided on the device:
//   checked offsets and the tile tables of the batch; the degree pass; the
//   per-graph fits (largest first, sorted on the device) on a
//   highest-priority stream beside the first hook pass; a WHILE node over
//   the graphs whose large degrees overflow the per-graph fit (the
//   single-graph fit of each); an IF node for the BFS step when any graph
//   is routed to it; then the SV iterations (WHILE) and the labels.

cc_status ensure_batch_graph(cc_ctx *ctx, int G, long long n, long long m) {
    CC_TRY(ensure_batch_route(ctx, G));
    const size_t g1 = (size_t)G + 1;
    CC_TRY(buf_reserve(ctx, ctx->bo_e, g1 * 8));
    CC_TRY(buf_reserve(ctx, ctx->bo_v, g1 * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_keys, g1 * 4));
    CC_TRY(buf_reserve(ctx, ctx->kb_keys2, g1 * 4));
    CC_TRY(buf_reserve(ctx, ctx->kb_idx, g1 * 4));
    CC_TRY(buf_reserve(ctx, ctx->kb_order, g1 * 4));
    CC_TRY(buf_reserve(ctx, ctx->kb_rcnt, g1 * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_roff, g1 * 8));
    CC_TRY(buf_reserve(ctx, ctx->kb_cmin, g1 * 4));
    CC_TRY(buf_reserve(ctx, ctx->kb_cub, batch_cub_bytes(G > 0 ? G : 1)));
    CC_TRY(buf_reserve(ctx, ctx->tile_pairs, (size_t)((m >> kTileShift) + 2) * 4));
    CC_TRY(buf_reserve(ctx, ctx->tile_verts, (size_t)((n >> kTileShift) + 2) * 4));
    CC_TRY(ensure_feat(ctx, (size_t)n));
    // inside the caller's capture a missing window scratch means the L2 degree pass
    if (!ctx->capturing && ctx->opt.route_policy != CC_ROUTE_FORCE_SV) CC_TRY(ensure_batch_win(ctx, m, n, G));
    return CC_OK;
}

// checked offsets and the tile tables (also run before the schedule tuner)
void enqueue_batch_tables(cc_ctx *ctx, const int64_t *eo_u, const int64_t *vo_u, int G, long long m, long long n,
                          cudaStream_t cs) {
    int64_t *eo = as<int64_t>(ctx->bo_e), *vo = as<int64_t>(ctx->bo_v);
    launch_batch_offsets(eo_u, vo_u, G, m, n, eo, vo, as<DevState>(ctx->st), cs);
    launch_tile_graphs(eo, G, m, as<uint32_t>(ctx->tile_pairs), ctx->grid, cs);
    launch_tile_graphs(vo, G, n, as<uint32_t>(ctx->tile_verts), ctx->grid, cs);
}

// The first hook passes over a batch, every vertex its own root: one pass
// over all pairs, or with the front end (Section 3.1's joins over a sample
// first, so that the first gather pass finds most pairs inside one tree) a
// pass over the sampled tiles and the graphs that are not sampled, a full
// shortcut, and a gather pass over the sampled tiles. Returns the launches.
int enqueue_batch_first_hooks(cc_ctx *ctx, const int32_t *edges, long long m, const int64_t *eo, const int64_t *vo,
                              int G, vid_t nt, const BatchSchedule &sch, cudaStream_t cs) {
    DevState *st = as<DevState>(ctx->st);
    vid_t *parent = as<vid_t>(ctx->parent), *hooked = as<vid_t>(ctx->hooked);
    if (!sch.front) {
        launch_sv_pass_batch(0, edges, m, eo, vo, G, nt, parent, hooked, nullptr, st, 0, ctx->grid, cs, sch);
        return 1;
    }
    launch_sv_pass_batch(5, edges, m, eo, vo, G, nt, parent, hooked, nullptr, st, 0, ctx->grid, cs, sch);
    launch_shortcut_all(parent, nt, st, 0, ctx->grid, cs);
    launch_sv_pass_batch(6, edges, m, eo, vo, G, nt, parent, hooked, nullptr, st, 0, ctx->grid, cs, sch);
    return 3;
}

cc_status enqueue_batch_route(cc_ctx *ctx, const int32_t *edges, const int64_t *eo_u, const int64_t *vo_u, int G,
                              long long m, long long n, int32_t *labels, int cap, BatchSchedule sch, cudaStream_t cs,
                              cc_ctx::RouteGraph &rg) {
    DevState *st = as<DevState>(ctx->st);
    vid_t *parent = as<vid_t>(ctx->parent), *hooked = as<vid_t>(ctx->hooked);
    uint2 *eb0 = as<uint2>(ctx->ebuf0), *eb1 = as<uint2>(ctx->ebuf1);
    int64_t *eo = as<int64_t>(ctx->bo_e), *vo = as<int64_t>(ctx->bo_v);
    const vid_t nt = (vid_t)n;
    const int policy = ctx->opt.route_policy;
    const bool predict = policy != CC_ROUTE_FORCE_SV;
    const uint32_t *ptiles = as<uint32_t>(ctx->tile_pairs), *vtiles = as<uint32_t>(ctx->tile_verts);
    sch.pair_tiles = ptiles;
    const long long before = ctx->stats.launches;
    long long direct = 0;
    rg.edge_bfs = true;
    rg.batched = true;
    rg.degree_form = 0;
    rg.level_launches = 4;
    rg.bfs_launches = 0;
    rg.unsure_launches = 0;
    rg.sample_stride = sch.front ? -1 : 1;
    rg.batch_unroll = sch.unroll;
    rg.batch_grid_mult = sch.grid_mult;
    rg.batch_deg_regions = sch.deg_regions;
    rg.batch_sv_regions = sch.sv_regions;
    CU_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), cs));
    enqueue_batch_tables(ctx, eo_u, vo_u, G, m, n, cs);
    launch_parent_init(parent, nt, nullptr, 0, ctx->grid, cs);
    direct += 4;
    KsBatchScratch sc{as<uint32_t>(ctx->kb_xs), as<unsigned long long>(ctx->kb_cnt), as<unsigned long long>(ctx->kb_cum),
                      as<double>(ctx->kb_lnx), as<double>(ctx->kb_Dc), as<double>(ctx->kb_Ac), as<double>(ctx->kb_Zc)};
    KsBatchOut out{as<double>(ctx->kb_D),     as<double>(ctx->kb_alpha), as<long long>(ctx->kb_xmin),
                   as<long long>(ctx->kb_ntail), as<long long>(ctx->kb_ncand), as<int>(ctx->kb_route),
                   as<int>(ctx->kb_ovf),      as<unsigned long long>(ctx->kb_seed)};
    // without the front end the degree pass applies the first hook pass as well, and the fits
    // run beside the full shortcut that follows it
    const bool fused = predict && !sch.front;
    if (predict) {
        CU_TRY(cudaMemsetAsync(ctx->deg.p, 0, (size_t)n * 4, cs));
        enqueue_batch_degree(ctx, edges, m, eo, vo, G, n, sch.deg_regions, cs, fused ? parent : nullptr);
        // the fits (largest graph first) on the highest-priority stream beside the first hook pass
        CU_TRY(cudaEventRecord(ctx->ev_fork, cs));
        CU_TRY(cudaStreamWaitEvent(ctx->fit_s, ctx->ev_fork, 0));
        CU_TRY(launch_batch_order(vo, G, as<uint32_t>(ctx->kb_keys), as<uint32_t>(ctx->kb_keys2),
                                  as<int>(ctx->kb_idx), as<int>(ctx->kb_order), ctx->kb_cub.p, ctx->kb_cub.bytes,
                                  ctx->grid, ctx->fit_s));
        launch_ks_batch(as<uint32_t>(ctx->deg), vo, G, sc, out, ctx->opt.ks_min_tail, ctx->opt.ks_min_distinct,
                        ctx->opt.ks_min_span, ctx->opt.ks_tau, ctx->kb_blocks, as<int>(ctx->kb_order),
                        counter_at<int>(ctx->counters, kCtrKsQueue), ctx->fit_s);
        CU_TRY(cudaEventRecord(ctx->ev_fit, ctx->fit_s));
        if (fused) {
            launch_shortcut_all(parent, nt, st, 0, ctx->grid, cs);
            direct += 6;
        } else {
            direct += 5 + enqueue_batch_first_hooks(ctx, edges, m, eo, vo, G, nt, sch, cs);
        }
        CU_TRY(cudaStreamWaitEvent(cs, ctx->ev_fit, 0));
        // graphs with more large degrees than the per-graph fit holds: the single-graph fit, one per iteration
        KsScratch ks{as<uint32_t>(ctx->ks_xs), as<unsigned long long>(ctx->ks_cnt), as<unsigned long long>(ctx->ks_cum),
                     as<double>(ctx->ks_lnx), as<double>(ctx->ks_Dc), as<double>(ctx->ks_Ac), as<double>(ctx->ks_Zc),
                     as<float>(ctx->ks_Df), as<unsigned long long>(ctx->chunk_nz),
                     as<unsigned long long>(ctx->chunk_mass), ctx->ks_cap};
        cudaGraphConditionalHandle ho;
        CC_TRY(cond_handle(cs, &ho));
        launch_ovf_seek(as<int>(ctx->kb_ovf), G, vo, st, ho, 1, cs);
        direct += 1;
        CC_TRY(cond_node(cs, ctx->cap_s2, ho, cudaGraphCondTypeWhile, [&](cudaStream_t bs) -> cc_status {
            CU_TRY(cudaMemsetAsync(ctx->hist.p, 0, (size_t)kHistDense * 4, bs));
            launch_hist_slice(as<uint32_t>(ctx->deg), as<uint32_t>(ctx->hist), as<uint32_t>(ctx->ovf), ctx->ovf_cap, st,
                              ctx->grid, bs);
            launch_ks(as<uint32_t>(ctx->hist), as<uint32_t>(ctx->ovf), ctx->ovf_cap, ks, st, ctx->opt.ks_min_tail,
                      ctx->opt.ks_min_distinct, ctx->opt.ks_min_span, ctx->opt.ks_tau, ctx->ks_cap, ctx->grid, bs);
            launch_ovf_store(out, st, bs);
            launch_ovf_seek(as<int>(ctx->kb_ovf), G, vo, st, ho, 0, bs);
            return CC_OK;
        }));
        // the BFS step of the graphs routed to it (all of them under the forced-BFS policy)
        cudaGraphConditionalHandle hb;
        CC_TRY(cond_handle(cs, &hb));
        CU_TRY(launch_batch_bfs_plan(as<int>(ctx->kb_route), eo, vo, G, policy == CC_ROUTE_FORCE_BFS ? 1 : 0,
                                     as<unsigned long long>(ctx->kb_rcnt), as<unsigned long long>(ctx->kb_roff),
                                     ctx->kb_cub.p, ctx->kb_cub.bytes, st, hb, ctx->grid, cs));
        direct += 3;
        CC_TRY(cond_node(cs, ctx->cap_s2, hb, cudaGraphCondTypeIf, [&](cudaStream_t bs) -> cc_status {
            const long long nwords = (n + 31) / 32;
            uint32_t *fv = as<uint32_t>(ctx->f_vis), *f0 = as<uint32_t>(ctx->f_f0), *f1 = as<uint32_t>(ctx->f_f1);
            CU_TRY(cudaMemsetAsync(fv, 0, (size_t)nwords * 4, bs));
            CU_TRY(cudaMemsetAsync(f0, 0, (size_t)nwords * 4, bs));
            launch_batch_bfs_start(edges, m, eo, vo, G, ptiles, as<unsigned long long>(ctx->kb_rcnt),
                                   as<unsigned long long>(ctx->kb_roff), as<unsigned long long>(ctx->kb_seed), eb0, fv,
                                   f0, st, ctx->grid, bs);
            cudaGraphConditionalHandle hl;
            CC_TRY(cond_handle(bs, &hl));
            launch_set_cond(hl, 1u, bs);
            CC_TRY(cond_node(bs, ctx->cap_s3, hl, cudaGraphCondTypeWhile, [&](cudaStream_t ls) -> cc_status {
                launch_ebfsg_level<int32_t>(nullptr, 0, eb0, eb1, nt, fv, f0, f1, st, hl, ctx->grid, ls);
                return CC_OK;
            }));
            launch_batch_bfs_finish(fv, n, vo, G, vtiles, as<uint32_t>(ctx->kb_cmin), parent, ctx->grid, bs);
            rg.bfs_launches = 2 + 1 + 2;
            if (fused) {  // the merge left visited vertices two hops from their roots
                launch_shortcut_all(parent, nt, st, 0, ctx->grid, bs);
                rg.bfs_launches += 1;
            }
            return CC_OK;
        }));
    } else {
        direct += enqueue_batch_first_hooks(ctx, edges, m, eo, vo, G, nt, sch, cs);
    }
    if (!fused) {
        launch_shortcut_all(parent, nt, st, 0, ctx->grid, cs);
        direct += 1;
    }
    launch_sv_pass_batch(2, edges, m, eo, vo, G, nt, parent, hooked, eb0, st, 1, ctx->grid, cs, sch);
    launch_sv_shortcut(parent, hooked, st, 1, ctx->grid, cs);
    cudaGraphConditionalHandle hs;
    CC_TRY(cond_handle(cs, &hs));
    launch_sv_loop_init(st, 1, 0, cap, hs, cs);
    CC_TRY(cond_node(cs, ctx->cap_s2, hs, cudaGraphCondTypeWhile, [&](cudaStream_t bs) -> cc_status {
        launch_sv_loop_body(eb0, eb1, nt, parent, hooked, st, hs, ctx->grid, bs);
        return CC_OK;
    }));
    launch_finalize_batch(parent, nt, vo, G, labels, ctx->grid, cs, vtiles);
    direct += 4;
    CU_TRY(cudaMemcpyAsync(ctx->h_st, st, offsetof(DevState, hook_base), cudaMemcpyDeviceToHost, cs));
    rg.static_launches = ctx->stats.launches - before + direct;
    return CC_OK;
}

cc_status labels_batched_graph(cc_ctx *ctx, const int32_t *edges, const int64_t *eo_u, const int64_t *vo_u, int G,
                               long long m, long long n, int32_t *labels, cudaStream_t s) {
    cc_stats &S = ctx->stats;
    const int cap = ctx->opt.max_iters > 0 ? ctx->opt.max_iters : default_max_iters(n);
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    CU_TRY(cudaStreamIsCapturing(s, &cst));
    const bool user_capture = cst == cudaStreamCaptureStatusActive;
    cc_status prior = CC_OK;
    if (!user_capture && ctx->async_outstanding && cudaEventQuery(ctx->ev_done) == cudaSuccess) {
        prior = device_error(ctx->h_st->err);
        ctx->async_outstanding = false;
    }
    cudaGetLastError();
    memset(&S, 0, sizeof(S));
    prof_reset(ctx);
    for (int e = 0; e < EV_COUNT; e++) ctx->ev_used[e] = false;
    S.n = n;
    S.m = m;
    ctx->graph_last = true;
    ctx->capturing = user_capture;
    cc_status r = ensure_sv(ctx, (size_t)n, (size_t)m);
    if (r == CC_OK) r = ensure_batch_graph(ctx, G, n, m);
    ctx->capturing = false;
    CC_TRY(r);
    // the schedule of the hook passes: tuned on the first call of a shape (outside any capture)
    BatchSchedule sch;
    sch.pair_tiles = as<uint32_t>(ctx->tile_pairs);
    if (!user_capture && m >= (1LL << 24)) {
        const int key = (ilog2_ceil(m) << 8) | ilog2_ceil(G);
        bool known = false;
        for (const auto &e : ctx->batch_tuned) known |= e.first == key;
        if (!known) {
            CU_TRY(cudaMemsetAsync(ctx->st.p, 0, sizeof(DevState), s));
            enqueue_batch_tables(ctx, eo_u, vo_u, G, m, n, s);
        }
        CC_TRY(tune_batch(ctx, edges, m, as<int64_t>(ctx->bo_e), as<int64_t>(ctx->bo_v), G, (vid_t)n, s, &sch));
    } else if (m >= (1LL << 24)) {
        const int key = (ilog2_ceil(m) << 8) | ilog2_ceil(G);
        for (const auto &e : ctx->batch_tuned)
            if (e.first == key) sch = e.second;
    }
    sch.front = batch_front(ctx, m);
    hook_order(ctx, &sch);
    if (batch_win(ctx, m, n, G)) sch.deg_regions = 0;  // the windowed degree pass has no regions
    S.batch_unroll = sch.unroll;
    S.batch_grid_mult = sch.grid_mult;
    S.batch_deg_regions = sch.deg_regions;
    S.batch_sv_regions = sch.sv_regions;
    S.sv_sample_stride = sch.front ? -1 : 1;
    if (user_capture) {
        ctx->capturing = true;
        r = enqueue_batch_route(ctx, edges, eo_u, vo_u, G, m, n, labels, cap, sch, s, ctx->g_capture);
        ctx->capturing = false;
        ctx->rg_last = &ctx->g_capture;
        return r;
    }
    std::vector<unsigned char> key = route_key(ctx, 4, n, m, edges, labels, cap);
    const long long extra[] = {G, sch.unroll, sch.grid_mult, sch.deg_regions, sch.sv_regions, sch.front,
                               (long long)(uintptr_t)eo_u, (long long)(uintptr_t)vo_u,
                               (long long)(uintptr_t)ctx->bo_e.p, (long long)(uintptr_t)ctx->kb_route.p,
                               (long long)(uintptr_t)ctx->tile_pairs.p, (long long)(uintptr_t)ctx->kb_cub.p};
    key.insert(key.end(), reinterpret_cast<const unsigned char *>(extra),
               reinterpret_cast<const unsigned char *>(extra) + sizeof(extra));
    cc_ctx::RouteGraph &rg = ctx->g_batch_route;
    if (!rg.exec || rg.key != key) {
        if (rg.exec) cudaGraphExecDestroy(rg.exec);
        rg.exec = nullptr;
        CU_TRY(cudaStreamBeginCapture(ctx->cap_s, cudaStreamCaptureModeRelaxed));
        const cc_status rr = enqueue_batch_route(ctx, edges, eo_u, vo_u, G, m, n, labels, cap, sch, ctx->cap_s, rg);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ctx->cap_s, &g);
        if (rr != CC_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rr != CC_OK ? rr : CC_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&rg.exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            cudaGetLastError();
            rg.exec = nullptr;
            return CC_ERR_CUDA;
        }
        rg.key.swap(key);
    }
    ctx->rg_last = &rg;
    rec(ctx, EV_START, s);
    CU_TRY(cudaGraphLaunch(rg.exec, s));
    rec(ctx, EV_END, s);
    CU_TRY(cudaEventRecord(ctx->ev_done, s));
    ctx->async_outstanding = true;
    if (ctx->opt.debug_checks) {
        CU_TRY(cudaStreamSynchronize(s));
        ctx->async_outstanding = false;
        return device_error(ctx->h_st->err);
    }
    return prior;
}

// The caller's device offsets on the host (the profiled and the statistics
// entry points wait on the host anyway).
cc_status offsets_to_host(const int64_t *eo_dev, const int64_t *vo_dev, int G, long long m, long long n,
                          std::vector<int64_t> &eo, std::vector<int64_t> &vo, cudaStream_t s) {
    eo.assign((size_t)G + 1, 0);
    vo.assign((size_t)G + 1, 0);
    CU_TRY(cudaMemcpyAsync(eo.data(), eo_dev, ((size_t)G + 1) * 8, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaMemcpyAsync(vo.data(), vo_dev, ((size_t)G + 1) * 8, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    if (eo[0] != 0 || vo[0] != 0 || eo[G] != m || vo[G] != n) return CC_ERR_INVALID_ARG;
    for (int g = 0; g < G; g++)
        if (eo[g + 1] < eo[g] || vo[g + 1] < vo[g]) return CC_ERR_INVALID_ARG;
    for (int g = 0; g < G; g++)  // pairs in a graph without vertices cannot be valid
        if (vo[g + 1] == vo[g] && eo[g + 1] > eo[g]) return CC_ERR_INVALID_EDGE;
    return CC_OK;
}

}  // namespace

extern "C" {

cc_status cc_default_options(cc_options *opt) {
    if (!opt) return CC_ERR_INVALID_ARG;
    memset(opt, 0, sizeof(*opt));
    opt->id_bytes = 4;
    opt->route_policy = CC_ROUTE_AUTO;
    opt->ks_tau = 0.05;
    opt->ks_min_tail = 50;
    opt->ks_min_distinct = 3;
    opt->ks_min_span = 10.0;
    return CC_OK;
}

cc_status cc_create(cc_ctx **out, const cc_options *opt, int device) {
    if (!out) return CC_ERR_INVALID_ARG;
    *out = nullptr;
    cc_options o;
    if (opt) o = *opt;
    else cc_default_options(&o);
    CC_TRY(check_options(&o));
    int ndev = 0;
    CU_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return CC_ERR_INVALID_ARG;
    CU_TRY(cudaSetDevice(device));
    cc_ctx *ctx = new (std::nothrow) cc_ctx();
    if (!ctx) return CC_ERR_OOM;
    ctx->device = device;
    ctx->opt = o;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete ctx;
        return CC_ERR_CUDA;
    }
    ctx->num_sms = prop.multiProcessorCount;
    if (degree_part_setup() != cudaSuccess || degree_hubs_setup() != cudaSuccess || csr_kernels_setup() != cudaSuccess ||
        batch_win_setup() != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return CC_ERR_CUDA;
    }
    ctx->grid = ctx->num_sms * (prop.maxThreadsPerMultiProcessor / kBlock);
    if (cudaMallocHost(&ctx->h_st, sizeof(DevState)) != cudaSuccess) {
        delete ctx;
        return CC_ERR_OOM;
    }
    if (ensure_streams(ctx) != CC_OK) {  // every stream and event up front: none is created during a capture
        cudaGetLastError();
        cc_destroy(ctx);
        return CC_ERR_CUDA;
    }
    memset(ctx->h_st, 0, sizeof(DevState));
    for (int e = 0; e < EV_COUNT; e++) cudaEventCreate(&ctx->ev[e]);
    *out = ctx;
    return CC_OK;
}

cc_status cc_set_options(cc_ctx *ctx, const cc_options *opt) {
    if (!ctx || !opt) return CC_ERR_INVALID_ARG;
    CC_TRY(check_options(opt));
    ctx->opt = *opt;
    return CC_OK;
}

cc_status cc_destroy(cc_ctx *ctx) {
    if (!ctx) return CC_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    Buf *bufs[] = {&ctx->deg,    &ctx->parent,     &ctx->hooked, &ctx->ebuf0,   &ctx->ebuf1,  &ctx->hist,
                   &ctx->ovf,    &ctx->ks_xs,      &ctx->ks_cnt, &ctx->ks_cum,  &ctx->ks_lnx, &ctx->ks_Dc,
                   &ctx->ks_Ac,  &ctx->ks_Zc, &ctx->ks_Df, &ctx->chunk_nz,   &ctx->chunk_mass, &ctx->st,  &ctx->row_ptr, &ctx->col,
                   &ctx->vis,    &ctx->fb,         &ctx->nb,     &ctx->q0,      &ctx->q1,     &ctx->dq,
                   &ctx->off,    &ctx->tsum,       &ctx->counters, &ctx->bk_off, &ctx->csr_entries,
                   &ctx->dpart,  &ctx->f_sdeg,     &ctx->f_counts, &ctx->f_vis,
                   &ctx->f_f0,   &ctx->f_f1,       &ctx->f_x,    &ctx->pred_wb, &ctx->pred_bias, &ctx->pred_tmp,
                   &ctx->bfs_own, &ctx->bfs_tmin, &ctx->bwin};
    for (Buf *b : bufs) buf_free(*b);
    for (int e = 0; e < EV_COUNT; e++)
        if (ctx->ev[e]) cudaEventDestroy(ctx->ev[e]);
    for (cudaEvent_t e : ctx->evpool) cudaEventDestroy(e);
    graph_drop(ctx->g_single);
    graph_drop(ctx->g_batch);
    buf_free(ctx->hedges);
    buf_free(ctx->hlabels);
    buf_free(ctx->tile_pairs);
    buf_free(ctx->tile_verts);
    Buf *bg[] = {&ctx->bo_e, &ctx->bo_v, &ctx->kb_keys, &ctx->kb_keys2, &ctx->kb_idx,
                 &ctx->kb_rcnt, &ctx->kb_roff, &ctx->kb_cmin, &ctx->kb_cub};
    for (Buf *b : bg) buf_free(*b);
    if (ctx->g_batch_route.exec) cudaGraphExecDestroy(ctx->g_batch_route.exec);
    for (Buf &b : ctx->tsv_t32) buf_free(b);
    Buf *tsv[] = {&ctx->tsv_v0,    &ctx->tsv_v1, &ctx->tsv_val,  &ctx->tsv_val2, &ctx->tsv_uniq, &ctx->tsv_agg,
                  &ctx->tsv_dense, &ctx->tsv_pc, &ctx->tsv_done, &ctx->tsv_temp, &ctx->tsv_cnt};
    for (Buf *b : tsv) buf_free(*b);
    Buf *kb[] = {&ctx->kb_xs, &ctx->kb_cnt, &ctx->kb_cum, &ctx->kb_lnx, &ctx->kb_Dc, &ctx->kb_Ac, &ctx->kb_Zc,
                 &ctx->kb_D, &ctx->kb_alpha, &ctx->kb_xmin, &ctx->kb_ntail, &ctx->kb_ncand, &ctx->kb_route,
                 &ctx->kb_ovf, &ctx->kb_seed, &ctx->kb_order};
    for (Buf *b : kb) buf_free(*b);
    if (ctx->copy_s) cudaStreamDestroy(ctx->copy_s);
    for (cudaEvent_t e : ctx->ev_chunk) cudaEventDestroy(e);
    if (ctx->side_s) cudaStreamDestroy(ctx->side_s);
    if (ctx->fit_s) cudaStreamDestroy(ctx->fit_s);
    if (ctx->ev_fit) cudaEventDestroy(ctx->ev_fit);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->cap_s) cudaStreamDestroy(ctx->cap_s);
    if (ctx->cap_s2) cudaStreamDestroy(ctx->cap_s2);
    if (ctx->cap_s3) cudaStreamDestroy(ctx->cap_s3);
    if (ctx->g_route.exec) cudaGraphExecDestroy(ctx->g_route.exec);
    if (ctx->ev_done) cudaEventDestroy(ctx->ev_done);
    if (ctx->h_st) cudaFreeHost(ctx->h_st);
    delete ctx;
    return CC_OK;
}

cc_status cc_labels(cc_ctx *ctx, const void *edges_dev, int64_t n, int64_t m, void *labels_out_dev, void *stream) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    if (n < 0 || m < 0) return CC_ERR_INVALID_ARG;
    if (n >= 0xffffffffLL) return CC_ERR_UNSUPPORTED;
    if (m >= (1LL << 31)) return CC_ERR_UNSUPPORTED;
    if (n == 0) {
        if (m > 0) return CC_ERR_INVALID_EDGE;
        return CC_OK;
    }
    if (!labels_out_dev || (m > 0 && !edges_dev)) return CC_ERR_INVALID_ARG;
    if (((uintptr_t)edges_dev & 15) || ((uintptr_t)labels_out_dev & 15)) return CC_ERR_INVALID_ARG;
    CU_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    CU_TRY(cudaStreamIsCapturing(s, &cst));
    const bool user_capture = cst == cudaStreamCaptureStatusActive;
    if (user_capture && ctx->opt.profile) return CC_ERR_INVALID_ARG;  // profiling waits on the host
    if (ctx->opt.fault_inject & CC_FAULT_ALLOC) ctx->alloc_fail_pending = 1;
    ctx->capturing = user_capture;  // inside a capture the workspace must already fit
    cc_status st = ensure_sv(ctx, (size_t)n, (size_t)m);
    ctx->capturing = false;
    ctx->alloc_fail_pending = 0;
    if (st != CC_OK) {
        ctx->last_status = st;
        return st;
    }
    if (!ctx->opt.profile) {
        // stream-ordered: enqueued with no host wait (m = 0: every vertex its own label)
        if (m == 0) {
            memset(&ctx->stats, 0, sizeof(ctx->stats));
            ctx->stats.n = n;
            ctx->graph_last = false;
            launch_parent_init(as<vid_t>(ctx->parent), (vid_t)n, nullptr, 0, ctx->grid, s);
            if (ctx->opt.id_bytes == 4) launch_finalize<int32_t>(as<vid_t>(ctx->parent), (vid_t)n, labels_out_dev, ctx->grid, s);
            else launch_finalize<int64_t>(as<vid_t>(ctx->parent), (vid_t)n, labels_out_dev, ctx->grid, s);
            ctx->stats.launches = 2;
            st = cuda_status(cudaGetLastError());
        } else if (ctx->opt.id_bytes == 4) {
            st = labels_graph<int32_t>(ctx, edges_dev, (vid_t)n, m, labels_out_dev, s);
        } else {
            st = labels_graph<int64_t>(ctx, edges_dev, (vid_t)n, m, labels_out_dev, s);
        }
        ctx->last_status = st;
        ctx->stats.status = st;
        return st;
    }
    ctx->graph_last = false;
    if (ctx->opt.id_bytes == 4) st = labels_impl<int32_t>(ctx, edges_dev, (vid_t)n, m, labels_out_dev, s);
    else st = labels_impl<int64_t>(ctx, edges_dev, (vid_t)n, m, labels_out_dev, s);
    if (st == CC_OK || st == CC_ERR_INVALID_EDGE || st == CC_ERR_NO_CONVERGENCE) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
    }
    ctx->last_status = st;
    ctx->stats.status = st;
    return st;
}

cc_status cc_labels_tuple_sv(cc_ctx *ctx, const void *edges_dev, int64_t n, int64_t m, void *labels_out_dev,
                             void *stream) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    if (n < 0 || m < 0) return CC_ERR_INVALID_ARG;
    if (n >= (1LL << 31) || m >= (1LL << 31)) return CC_ERR_UNSUPPORTED;
    if (n == 0) return m > 0 ? CC_ERR_INVALID_EDGE : CC_OK;
    if (!labels_out_dev || (m > 0 && !edges_dev)) return CC_ERR_INVALID_ARG;
    CU_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    CC_TRY(ensure_sv(ctx, (size_t)n, (size_t)m));  // the device state and the events
    // tuples: n + 2m, plus up to one temporary per partition (at most n)
    const long long cap = 2 * n + 2 * m + 16;
    if (cap > ctx->tsv_cap) {
        for (Buf &b : ctx->tsv_t32) CC_TRY(buf_reserve(ctx, b, (size_t)cap * 4));
        CC_TRY(buf_reserve(ctx, ctx->tsv_v0, (size_t)cap * 8));
        CC_TRY(buf_reserve(ctx, ctx->tsv_v1, (size_t)cap * 8));
        CC_TRY(buf_reserve(ctx, ctx->tsv_val, (size_t)cap * 4));
        CC_TRY(buf_reserve(ctx, ctx->tsv_val2, (size_t)cap * 4));
        CC_TRY(buf_reserve(ctx, ctx->tsv_uniq, (size_t)cap * 4));
        CC_TRY(buf_reserve(ctx, ctx->tsv_agg, (size_t)cap * 4));
        CC_TRY(buf_reserve(ctx, ctx->tsv_cnt, 64));
        ctx->tsv_cap = cap;
    }
    CC_TRY(buf_reserve(ctx, ctx->tsv_dense, (size_t)(n + 4) * 4));
    CC_TRY(buf_reserve(ctx, ctx->tsv_pc, (size_t)(n + 4) * 4));
    CC_TRY(buf_reserve(ctx, ctx->tsv_done, (size_t)(n + 4) * 4));
    // the temporary storage the sorts need depends on the key bits (n) as well
    const size_t tb = tuple_sv_temp_bytes(ctx->tsv_cap, (vid_t)n);
    CC_TRY(buf_reserve(ctx, ctx->tsv_temp, tb));
    TupleSvBufs b;
    for (int k = 0; k < 4; k++) b.t32[k] = as<uint32_t>(ctx->tsv_t32[k]);
    b.v0 = as<unsigned long long>(ctx->tsv_v0);
    b.v1 = as<unsigned long long>(ctx->tsv_v1);
    b.val = as<uint32_t>(ctx->tsv_val);
    b.val2 = as<uint32_t>(ctx->tsv_val2);
    b.pc = as<uint32_t>(ctx->tsv_pc);
    b.done = as<uint32_t>(ctx->tsv_done);
    b.uniq = as<uint32_t>(ctx->tsv_uniq);
    b.agg = as<uint32_t>(ctx->tsv_agg);
    b.dense = as<uint32_t>(ctx->tsv_dense);
    b.counters = as<unsigned long long>(ctx->tsv_cnt);
    b.temp = ctx->tsv_temp.p;
    b.temp_bytes = ctx->tsv_temp.bytes;
    b.cap = ctx->tsv_cap;
    b.num_sms = ctx->num_sms;
    DevState *st = as<DevState>(ctx->st);
    cc_stats &S = ctx->stats;
    memset(&S, 0, sizeof(S));
    prof_reset(ctx);
    for (int e = 0; e < EV_COUNT; e++) ctx->ev_used[e] = false;
    S.n = n;
    S.m = m;
    S.route_source = 2;
    CU_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), s));
    rec(ctx, EV_START, s);
    const int cap_iters = ctx->opt.max_iters > 0 ? ctx->opt.max_iters : default_max_iters((vid_t)n);
    int iters = 0, sorts = 0;
    float sort_ms = 0.0f;
    float *sort_out = ctx->opt.profile ? &sort_ms : nullptr;
    long long active[CC_MAX_SV_ITERS_RECORDED] = {};
    const int rc = ctx->opt.id_bytes == 4
                       ? tuple_sv_run<int32_t>(edges_dev, m, (vid_t)n, labels_out_dev, b, st, cap_iters, &iters,
                                               active, CC_MAX_SV_ITERS_RECORDED, sort_out, &sorts, s)
                       : tuple_sv_run<int64_t>(edges_dev, m, (vid_t)n, labels_out_dev, b, st, cap_iters, &iters,
                                               active, CC_MAX_SV_ITERS_RECORDED, sort_out, &sorts, s);
    for (int i = 0; i < CC_MAX_SV_ITERS_RECORDED; i++) S.m_active[i] = active[i];
    S.kernel_ms[CC_K_TUPLE_SORT] = sort_ms;
    S.kernel_launches[CC_K_TUPLE_SORT] = sorts;
    rec(ctx, EV_SV, s);
    rec(ctx, EV_END, s);
    S.sv_iters = iters;
    cc_status out = rc == 0 ? CC_OK : rc == 2 ? CC_ERR_NO_CONVERGENCE : CC_ERR_CUDA;
    if (rc != 1) {
        CU_TRY(cudaMemcpyAsync(&ctx->h_st->err, &st->err, 4, cudaMemcpyDeviceToHost, s));
        CU_TRY(cudaStreamSynchronize(s));
        if (ctx->h_st->err) out = device_error(ctx->h_st->err);
    }
    ctx->last_status = out;
    S.status = out;
    return out;
}

cc_status cc_labels_host(cc_ctx *ctx, const void *edges_host, int64_t n, int64_t m, void *labels_out_host,
                         void *stream) {
    if (!ctx) return CC_ERR_INVALID_ARG;
    if (n < 0 || m < 0) return CC_ERR_INVALID_ARG;
    if (n >= 0xffffffffLL || m >= (1LL << 31)) return CC_ERR_UNSUPPORTED;
    if (n == 0) return m > 0 ? CC_ERR_INVALID_EDGE : CC_OK;
    if (!labels_out_host || (m > 0 && !edges_host)) return CC_ERR_INVALID_ARG;
    CU_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    const size_t w = (size_t)ctx->opt.id_bytes;
    if (ctx->opt.fault_inject & CC_FAULT_ALLOC) ctx->alloc_fail_pending = 1;
    cc_status st = ensure_sv(ctx, (size_t)n, (size_t)m);
    if (st == CC_OK) st = buf_reserve(ctx, ctx->hedges, (size_t)m * 2 * w + 16);
    if (st == CC_OK) st = buf_reserve(ctx, ctx->hlabels, round4((size_t)n) * w + 16);
    ctx->alloc_fail_pending = 0;
    if (st == CC_OK) {
        if (w == 4) st = labels_host_impl<int32_t>(ctx, edges_host, (vid_t)n, m, labels_out_host, s);
        else st = labels_host_impl<int64_t>(ctx, edges_host, (vid_t)n, m, labels_out_host, s);
    }
    if (st == CC_ERR_INVALID_EDGE || st == CC_ERR_NO_CONVERGENCE) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
    }
    ctx->last_status = st;
    ctx->stats.status = st;
    return st;
}

cc_status cc_ks_statistic_batched(cc_ctx *ctx, const void *edges_dev, const int64_t *edge_offsets_dev,
                                  const int64_t *vertex_offsets_dev, int G, int64_t m_total, int64_t n_total,
                                  double *D_host, double *alpha_host, int64_t *xmin_host, int64_t *ncand_host,
                                  int32_t *route_host, int64_t *seed_host, void *stream) {
    if (!ctx || G < 0 || m_total < 0 || n_total < 0) return CC_ERR_INVALID_ARG;
    if (G == 0) return m_total || n_total ? CC_ERR_INVALID_ARG : CC_OK;
    if (!edge_offsets_dev || !vertex_offsets_dev || !D_host || !alpha_host || !xmin_host || !ncand_host ||
        !route_host || !seed_host)
        return CC_ERR_INVALID_ARG;
    const long long m = m_total, n = n_total;
    if (n >= (1LL << 31) || m >= (1LL << 31)) return CC_ERR_UNSUPPORTED;
    if ((m > 0 && !edges_dev) || ((uintptr_t)edges_dev & 15)) return CC_ERR_INVALID_ARG;
    CU_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> eo_h, vo_h;  // the schedule is built on the host here: the call waits anyway
    CC_TRY(offsets_to_host(edge_offsets_dev, vertex_offsets_dev, G, m, n, eo_h, vo_h, s));
    const int64_t *edge_offsets_host = eo_h.data(), *vertex_offsets_host = vo_h.data();
    CC_TRY(ensure_sv(ctx, (size_t)(n > 0 ? n : 1), (size_t)m));
    CC_TRY(ensure_batch_route(ctx, G));
    CC_TRY(ensure_batch_win(ctx, m, n, G));
    DevState *st = as<DevState>(ctx->st);
    CU_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), s));
    CU_TRY(cudaMemsetAsync(ctx->deg.p, 0, (size_t)(n > 0 ? n : 1) * 4, s));
    CC_TRY(ensure_tiles(ctx, edge_offsets_dev, vertex_offsets_dev, G, m, n, s));
    enqueue_batch_degree(ctx, (const int32_t *)edges_dev, m, edge_offsets_dev, vertex_offsets_dev, G, n,
                         BatchSchedule().deg_regions, s, nullptr);
    std::vector<int> route;
    CC_TRY(enqueue_ks_batch(ctx, vertex_offsets_dev, vertex_offsets_host, G, s));
    CC_TRY(batch_routes(ctx, vertex_offsets_host, G, route, s));
    std::vector<long long> xmin((size_t)G), ncand((size_t)G);
    std::vector<unsigned long long> seed((size_t)G);
    CU_TRY(cudaMemcpyAsync(D_host, ctx->kb_D.p, (size_t)G * 8, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaMemcpyAsync(alpha_host, ctx->kb_alpha.p, (size_t)G * 8, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaMemcpyAsync(xmin.data(), ctx->kb_xmin.p, (size_t)G * 8, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaMemcpyAsync(ncand.data(), ctx->kb_ncand.p, (size_t)G * 8, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaMemcpyAsync(seed.data(), ctx->kb_seed.p, (size_t)G * 8, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    for (int g = 0; g < G; g++) {
        xmin_host[g] = xmin[g];
        ncand_host[g] = ncand[g];
        route_host[g] = route[g];
        seed_host[g] = seed[g] ? (int64_t)(0xffffffffull - (seed[g] & 0xffffffffull)) : 0;
    }
    return CC_OK;
}

// The profiled batched form (options.profile = 1): the same route driven
// from the host, with every kernel class timed; the offsets are on both sides.
static cc_status labels_batched_profiled(cc_ctx *ctx, const void *edges_dev, const int64_t *edge_offsets_dev,
                                         const int64_t *vertex_offsets_dev, const int64_t *edge_offsets_host,
                                         const int64_t *vertex_offsets_host, int G, void *labels_out_dev,
                                         cudaStream_t s) {
    const long long m = edge_offsets_host[G], n = vertex_offsets_host[G];
    ctx->graph_last = false;
    CC_TRY(ensure_sv(ctx, (size_t)n, (size_t)m));
    DevState *st = as<DevState>(ctx->st);
    cc_stats &S = ctx->stats;
    memset(&S, 0, sizeof(S));
    prof_reset(ctx);
    for (int e = 0; e < EV_COUNT; e++) ctx->ev_used[e] = false;
    S.n = n;
    S.m = m;
    S.route_source = 2;
    CU_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), s));
    rec(ctx, EV_START, s);
    vid_t *parent = as<vid_t>(ctx->parent), *hooked = as<vid_t>(ctx->hooked);
    const vid_t nt = (vid_t)n;
    const int cap = ctx->opt.max_iters > 0 ? ctx->opt.max_iters : default_max_iters(n);
    CC_TRY(ensure_tiles(ctx, edge_offsets_dev, vertex_offsets_dev, G, m, n, s));
    const uint32_t *vtiles = as<uint32_t>(ctx->tile_verts);
    if (m > 0 && ctx->opt.route_policy != CC_ROUTE_FORCE_SV) CC_TRY(ensure_batch_win(ctx, m, n, G));
    BatchSchedule sch;
    CC_TRY(tune_batch(ctx, (const int32_t *)edges_dev, m, edge_offsets_dev, vertex_offsets_dev, G, nt, s, &sch));
    sch.front = batch_front(ctx, m);
    hook_order(ctx, &sch);
    if (batch_win(ctx, m, n, G)) sch.deg_regions = 0;  // the windowed degree pass has no regions
    S.sv_sample_stride = sch.front ? -1 : 1;
    S.batch_unroll = sch.unroll;
    S.batch_grid_mult = sch.grid_mult;
    S.batch_deg_regions = sch.deg_regions;
    S.batch_sv_regions = sch.sv_regions;
    {
        Scope sc(ctx, CC_K_PARENT_INIT, s, 1);
        launch_parent_init(parent, nt, nullptr, 0, ctx->grid, s);
    }
    // Route prediction per graph (Algorithm 2 lines 1-3): the degree pass
    // (with the first hook pass fused in unless the SV front end runs: every
    // vertex starts as its own root, so that pass needs no route), one K-S fit
    // per graph, then the BFS step for the graphs routed to it (lines 5-7):
    // their visited vertices take the visited minimum as parent before the SV
    // passes continue.
    const int policy = ctx->opt.route_policy;
    const bool predict = m > 0 && policy != CC_ROUTE_FORCE_SV;
    if (predict) {
        CC_TRY(ensure_batch_route(ctx, G));
        CU_TRY(cudaMemsetAsync(ctx->deg.p, 0, (size_t)n * 4, s));
        {
            {
                Scope sc(ctx, CC_K_DEGREE, s, 1);
                enqueue_batch_degree(ctx, (const int32_t *)edges_dev, m, edge_offsets_dev, vertex_offsets_dev, G, n,
                                     sch.deg_regions, s, sch.front ? nullptr : parent);
            }
            // the fits on a highest-priority stream, overlapping the first hook
            // pass, which launches one block per tile so that the fits' blocks
            // get SMs as its blocks retire
            CC_TRY(ensure_fit_stream(ctx));
            CU_TRY(cudaEventRecord(ctx->ev_fork, s));
            CU_TRY(cudaStreamWaitEvent(ctx->fit_s, ctx->ev_fork, 0));
            CC_TRY(enqueue_ks_batch(ctx, vertex_offsets_dev, vertex_offsets_host, G, ctx->fit_s));
            CU_TRY(cudaEventRecord(ctx->ev_fit, ctx->fit_s));
            if (sch.front) {  // without the front end the degree pass applied the first hook pass
                Scope sc(ctx, CC_K_SV_FIRST, s, 1);
                enqueue_batch_first_hooks(ctx, (const int32_t *)edges_dev, m, edge_offsets_dev, vertex_offsets_dev, G,
                                          nt, sch, s);
            }
            CU_TRY(cudaStreamWaitEvent(s, ctx->ev_fit, 0));
        }
        rec(ctx, EV_DEGREE, s);
        std::vector<int> route;
        cc_status rs = batch_routes(ctx, vertex_offsets_host, G, route, s);
        if (rs != CC_OK) {
            ctx->last_status = rs;
            return rs;
        }
        if (policy == CC_ROUTE_FORCE_BFS) route.assign((size_t)G, 1);  // the opposite decision of Section 5
        rec(ctx, EV_PREDICT, s);
        long long nbfs = 0;
        for (int g = 0; g < G; g++) {
            const long long ng = vertex_offsets_host[g + 1] - vertex_offsets_host[g];
            const long long mg = edge_offsets_host[g + 1] - edge_offsets_host[g];
            if (!route[g] || ng == 0 || mg == 0) continue;
            nbfs++;
            // the graph's pairs, copied to a 16-byte aligned buffer for the vector loads
            CU_TRY(cudaMemcpyAsync(ctx->ebuf1.p, (const int32_t *)edges_dev + 2 * edge_offsets_host[g], (size_t)mg * 8,
                                   cudaMemcpyDeviceToDevice, s));
            int levels = 0, list_buf = -1;
            unsigned long long list_len = 0;
            CC_TRY(run_bfs_edges<int32_t>(ctx, ctx->ebuf1.p, (vid_t)ng, mg, s, ctx->opt.bfs_cutoff_levels,
                                          as<unsigned long long>(ctx->kb_seed) + g, &levels, &list_buf, &list_len));
            launch_merge_visited(as<uint32_t>(ctx->f_vis), ng, vertex_offsets_host[g], st, parent, ctx->grid, s);
            S.bfs_levels += levels;
        }
        S.route = nbfs;  // graphs that took the BFS step
        S.route_source = policy == CC_ROUTE_FORCE_BFS ? 2 : 0;
        rec(ctx, EV_BFS, s);
    }
    if (m > 0 && cap >= 2 && !ctx->opt.profile) {
        // one cached graph with a device-driven loop (the parent init above stays outside)
        uint2 *eb0 = as<uint2>(ctx->ebuf0);
        auto pre = [&](cudaStream_t cs) {
            if (!predict)
                enqueue_batch_first_hooks(ctx, (const int32_t *)edges_dev, m, edge_offsets_dev, vertex_offsets_dev, G,
                                          nt, sch, cs);
            launch_shortcut_all(parent, nt, st, 0, ctx->grid, cs);
            launch_sv_pass_batch(2, (const int32_t *)edges_dev, m, edge_offsets_dev, vertex_offsets_dev, G, nt, parent,
                                 hooked, eb0, st, 1, ctx->grid, cs, sch);
            launch_sv_shortcut(parent, hooked, st, 1, ctx->grid, cs);
        };
        auto post = [&](cudaStream_t cs) {
            launch_finalize_batch(parent, nt, vertex_offsets_dev, G, (int32_t *)labels_out_dev, ctx->grid, cs, vtiles);
        };
        const cc_ctx::GraphKey key =
            graph_key(ctx,
                      2 | (predict ? 4 : 0) | (sch.front ? 8 : 0) | (sch.unroll << 8) | (sch.grid_mult << 12) |
                          (sch.sv_regions << 16),
                      n, m, G, edges_dev, edge_offsets_dev, vertex_offsets_dev, labels_out_dev, cap);
        cc_status gs = launch_sv_graph(ctx, ctx->g_batch, key, nt, 1, 0, cap, pre, post, s);
        if (gs == CC_OK) {
            rec(ctx, EV_SV, s);
            rec(ctx, EV_END, s);
            S.m_active[0] = m;
            S.m_active[1] = m;
            gs = sv_graph_finish(ctx, 1, predict ? 3 : 4, s);
        }
        ctx->last_status = gs;
        S.status = gs;
        return gs;
    }
    unsigned long long m_cur = 0;
    int it = 0;
    if (m > 0) {
        if (!predict) {
            Scope sc(ctx, CC_K_SV_FIRST, s, 1);
            enqueue_batch_first_hooks(ctx, (const int32_t *)edges_dev, m, edge_offsets_dev, vertex_offsets_dev, G, nt,
                                      sch, s);
        }
        {
            Scope sc(ctx, CC_K_SV_SHORTCUT, s, 1);
            launch_shortcut_all(parent, nt, st, 0, ctx->grid, s);
        }
        S.m_active[0] = m;
        it = 1;
        {
            Scope sc(ctx, CC_K_SV_GATHER_INPUT, s, 1);
            launch_sv_pass_batch(2, (const int32_t *)edges_dev, m, edge_offsets_dev, vertex_offsets_dev, G, nt, parent,
                                 hooked, as<uint2>(ctx->ebuf0), st, 1, ctx->grid, s, sch);
        }
        {
            Scope sc(ctx, CC_K_SV_SHORTCUT, s, 1);
            launch_sv_shortcut(parent, hooked, st, 1, ctx->grid, s);
        }
        S.m_active[1] = m;
        CC_TRY(read_back(ctx, &st->err, 4, s));
        if (ctx->h_st->err) {
            ctx->last_status = device_error(ctx->h_st->err);
            return ctx->last_status;
        }
        CC_TRY(read_back(ctx, &st->kept[1], 8, s));
        m_cur = ctx->h_st->kept[1];
    }
    cc_status stt = sv_list_loop(ctx, nt, ctx->ebuf0.p, m_cur, it, cap, s);
    if (stt == CC_OK) {
        rec(ctx, EV_SV, s);
        {
            Scope sc(ctx, CC_K_FINALIZE, s, 1);
            launch_finalize_batch(parent, nt, vertex_offsets_dev, G, (int32_t *)labels_out_dev, ctx->grid, s, vtiles);
        }
        rec(ctx, EV_END, s);
        CU_TRY(cudaMemcpyAsync(&ctx->h_st->err, &st->err, 4, cudaMemcpyDeviceToHost, s));
        CU_TRY(cudaStreamSynchronize(s));
        CU_TRY(cudaGetLastError());
        prof_collect(ctx);
        stt = device_error(ctx->h_st->err);
    }
    ctx->last_status = stt;
    S.status = stt;
    return stt;
}

cc_status cc_labels_batched(cc_ctx *ctx, const void *edges_dev, const int64_t *edge_offsets_dev,
                            const int64_t *vertex_offsets_dev, int G, int64_t m_total, int64_t n_total,
                            void *labels_out_dev, void *stream) {
    if (!ctx || G < 0 || m_total < 0 || n_total < 0) return CC_ERR_INVALID_ARG;
    if (G == 0) return m_total || n_total ? CC_ERR_INVALID_ARG : CC_OK;
    if (!edge_offsets_dev || !vertex_offsets_dev) return CC_ERR_INVALID_ARG;
    if (n_total >= (1LL << 31) || m_total >= (1LL << 31)) return CC_ERR_UNSUPPORTED;
    if (n_total == 0) return m_total > 0 ? CC_ERR_INVALID_EDGE : CC_OK;
    if (!labels_out_dev || (m_total > 0 && !edges_dev) || ((uintptr_t)edges_dev & 15)) return CC_ERR_INVALID_ARG;
    if (ctx->opt.id_bytes != 4) return CC_ERR_INVALID_ARG;
    CU_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    ctx->last_stream = s;
    cc_status st;
    if (ctx->opt.profile) {
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        CU_TRY(cudaStreamIsCapturing(s, &cst));
        if (cst == cudaStreamCaptureStatusActive) return CC_ERR_INVALID_ARG;  // profiling waits on the host
        std::vector<int64_t> eo, vo;
        st = offsets_to_host(edge_offsets_dev, vertex_offsets_dev, G, m_total, n_total, eo, vo, s);
        if (st == CC_OK)
            st = labels_batched_profiled(ctx, edges_dev, edge_offsets_dev, vertex_offsets_dev, eo.data(), vo.data(), G,
                                         labels_out_dev, s);
    } else {
        st = labels_batched_graph(ctx, (const int32_t *)edges_dev, edge_offsets_dev, vertex_offsets_dev, G, m_total,
                                  n_total, (int32_t *)labels_out_dev, s);
    }
    ctx->last_status = st;
    ctx->stats.status = st;
    return st;
}

cc_status cc_degree_distribution(cc_ctx *ctx, const void *edges_dev, int64_t n, int64_t m, uint32_t *deg_out_dev,
                                 uint64_t *hist_out_dev, int64_t hist_len, void *stream) {
    if (!ctx || n < 0 || m < 0 || hist_len < 0) return CC_ERR_INVALID_ARG;
    if (n >= 0xffffffffLL || m >= (1LL << 31)) return CC_ERR_UNSUPPORTED;
    if (n == 0) return m > 0 ? CC_ERR_INVALID_EDGE : CC_OK;
    if ((m > 0 && !edges_dev) || ((uintptr_t)edges_dev & 15)) return CC_ERR_INVALID_ARG;
    CU_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    CC_TRY(ensure_sv(ctx, (size_t)n, (size_t)m));
    DevState *st = as<DevState>(ctx->st);
    CU_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), s));
    if (ctx->opt.id_bytes == 4) enqueue_degree<int32_t>(ctx, edges_dev, (vid_t)n, m, s);
    else enqueue_degree<int64_t>(ctx, edges_dev, (vid_t)n, m, s);
    if (deg_out_dev) CU_TRY(cudaMemcpyAsync(deg_out_dev, ctx->deg.p, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    CU_TRY(cudaMemcpyAsync(ctx->h_st, st, offsetof(DevState, kept), cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    if (ctx->h_st->err) return device_error(ctx->h_st->err);
    if (hist_out_dev && hist_len > 0)
        launch_hist_widen(as<uint32_t>(ctx->hist), as<uint32_t>(ctx->ovf), ctx->ovf_cap, st, hist_out_dev, hist_len,
                          ctx->grid, s);
    CU_TRY(cudaStreamSynchronize(s));
    CU_TRY(cudaGetLastError());
    return CC_OK;
}

cc_status cc_ks_statistic(cc_ctx *ctx, const uint64_t *hist_dev, int64_t hist_len, double *out_host, void *stream) {
    if (!ctx || !hist_dev || hist_len < 1 || !out_host) return CC_ERR_INVALID_ARG;
    if (hist_len > (int64_t)kHistDense) return CC_ERR_UNSUPPORTED;
    CU_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    // the distinct-degree scratch holds at most hist_len entries
    CC_TRY(ensure_sv(ctx, (size_t)hist_len, 1));
    DevState *st = as<DevState>(ctx->st);
    CU_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), s));
    CU_TRY(cudaMemsetAsync(ctx->hist.p, 0, (size_t)kHistDense * 4, s));
    launch_hist_narrow(hist_dev, hist_len, as<uint32_t>(ctx->hist), st, ctx->grid, s);
    enqueue_ks(ctx, s, distinct_degree_bound(ctx, hist_len, -1));
    CU_TRY(cudaMemcpyAsync(ctx->h_st, st, offsetof(DevState, kept), cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    CU_TRY(cudaGetLastError());
    if (ctx->h_st->err) return CC_ERR_UNSUPPORTED;
    for (int i = 0; i < 5; i++) out_host[i] = ctx->h_st->ks_out[i];
    return CC_OK;
}

cc_status cc_route_features(cc_ctx *ctx, const void *edges_dev, int64_t n, int64_t m, float *feat_out_dev,
                            void *stream) {
    if (!ctx || n <= 0 || m < 0 || !feat_out_dev) return CC_ERR_INVALID_ARG;
    if (n >= 0xffffffffLL || m >= (1LL << 31)) return CC_ERR_UNSUPPORTED;
    if ((m > 0 && !edges_dev) || ((uintptr_t)edges_dev & 15)) return CC_ERR_INVALID_ARG;
    CU_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    CC_TRY(ensure_sv(ctx, (size_t)n, (size_t)m));
    CC_TRY(ensure_feat(ctx, (size_t)n));
    DevState *st = as<DevState>(ctx->st);
    CU_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), s));
    if (ctx->opt.id_bytes == 4)
        launch_route_features<int32_t>(edges_dev, m, (vid_t)n, feat_scratch(ctx), st, feat_out_dev, ctx->grid, s);
    else
        launch_route_features<int64_t>(edges_dev, m, (vid_t)n, feat_scratch(ctx), st, feat_out_dev, ctx->grid, s);
    CU_TRY(cudaMemcpyAsync(&ctx->h_st->err, &st->err, 4, cudaMemcpyDeviceToHost, s));
    CU_TRY(cudaStreamSynchronize(s));
    CU_TRY(cudaGetLastError());
    return device_error(ctx->h_st->err);
}

cc_status cc_set_predictor(cc_ctx *ctx, const float *params_host, double min_confidence) {
    if (!ctx || !(min_confidence >= 0.0 && min_confidence <= 1.0)) return CC_ERR_INVALID_ARG;
    if (!params_host) {
        ctx->have_pred = false;
        return CC_OK;
    }
    CU_TRY(cudaSetDevice(ctx->device));
    const int np = mlp_num_params();
    CC_TRY(buf_reserve(ctx, ctx->pred_tmp, (size_t)np * 4));
    CC_TRY(buf_reserve(ctx, ctx->pred_wb, (size_t)np * 2));
    CC_TRY(buf_reserve(ctx, ctx->pred_bias, 512 * 4));
    CU_TRY(cudaMemcpy(ctx->pred_tmp.p, params_host, (size_t)np * 4, cudaMemcpyHostToDevice));
    mlp_prepare_inference(as<float>(ctx->pred_tmp), as<__nv_bfloat16>(ctx->pred_wb), as<float>(ctx->pred_bias), 0);
    CU_TRY(cudaDeviceSynchronize());
    CU_TRY(cudaGetLastError());
    ctx->have_pred = true;
    ctx->pred_min_conf = min_confidence;
    return CC_OK;
}

cc_status cc_mlp_forward(const float *params_dev, const float *X_dev, int B, float *act_dev, void *stream) {
    if (!params_dev || !X_dev || !act_dev || B <= 0) return CC_ERR_INVALID_ARG;
    mlp_forward(params_dev, X_dev, B, act_dev, (cudaStream_t)stream);
    return cuda_status(cudaGetLastError());
}

cc_status cc_mlp_backward(const float *params_dev, const float *X_dev, const int *y_dev, const float *t_dev,
                          const float *w_dev, int B, float lambda, const float *act_dev, float *grad_dev,
                          float *scratch_dev, float *loss_dev, void *stream) {
    if (!params_dev || !X_dev || !y_dev || !t_dev || !w_dev || !act_dev || !grad_dev || !scratch_dev || !loss_dev ||
        B <= 0)
        return CC_ERR_INVALID_ARG;
    mlp_backward(params_dev, X_dev, y_dev, t_dev, w_dev, B, lambda, act_dev, grad_dev, scratch_dev, loss_dev,
                 (cudaStream_t)stream);
    return cuda_status(cudaGetLastError());
}

cc_status cc_mlp_adam(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev, int count, float lr,
                      float beta1, float beta2, float eps, int t, void *stream) {
    if (!params_dev || !grad_dev || !m_dev || !v_dev || count <= 0 || t < 1) return CC_ERR_INVALID_ARG;
    mlp_adam(params_dev, grad_dev, m_dev, v_dev, count, lr, beta1, beta2, eps, t, (cudaStream_t)stream);
    return cuda_status(cudaGetLastError());
}

cc_status cc_measure_l2_rates(cc_ctx *ctx, cc_l2_rates *out, void *stream) {
    if (!ctx || !out) return CC_ERR_INVALID_ARG;
    CU_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const long long words = 1LL << 24, ops = 1LL << 28;
    const int reps = 3, grid = ctx->num_sms * 16;
    uint32_t *table = nullptr;
    CU_TRY(cudaMalloc(&table, (size_t)words * 4 + 64));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cc_status rc = CC_OK;
    double rate[4] = {0, 0, 0, 0};
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemsetAsync(table, 0xff, (size_t)words * 4 + 64, s) != cudaSuccess)
        rc = CC_ERR_CUDA;
    for (int kind = 0; kind < 4 && rc == CC_OK; kind++) {
        launch_l2_probe(kind, table, (uint32_t)(words - 1), ops, table + words, grid, s);  // warm-up
        for (int r = 0; r < reps && rc == CC_OK; r++) {
            float ms = 0.f;
            if (cudaEventRecord(e0, s) != cudaSuccess) rc = CC_ERR_CUDA;
            launch_l2_probe(kind, table, (uint32_t)(words - 1), ops, table + words, grid, s);
            if (rc != CC_OK || cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = CC_ERR_CUDA;
            else if (ms > 0.f && (double)ops / (ms * 1e-3) > rate[kind])
                rate[kind] = (double)ops / (ms * 1e-3);
        }
    }
    if (rc == CC_OK && cudaGetLastError() != cudaSuccess) rc = CC_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(table);
    if (rc != CC_OK) return rc;
    out->gather = rate[0];
    out->red_add = rate[1];
    out->red_min = rate[2];
    out->atom_min = rate[3];
    out->table_words = words;
    out->ops = ops;
    out->reps = reps;
    out->grid = grid;
    return CC_OK;
}

cc_status cc_get_stats(cc_ctx *ctx, cc_stats *out) {
    if (!ctx || !out) return CC_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->last_stream);
    cc_stats &S = ctx->stats;
    if (ctx->graph_last) {  // stream-ordered call: statistics and status from the device state
        const int64_t n = S.n, m = S.m;
        memset(&S, 0, sizeof(S));
        S.n = n;
        S.m = m;
        stats_from_device(ctx);
        ctx->async_outstanding = false;
        if (ctx->last_status == CC_OK) ctx->last_status = (cc_status)S.status;
    }
    S.ms_degree = ev_ms(ctx, EV_START, EV_DEGREE);
    S.ms_predict = ev_ms(ctx, EV_DEGREE, EV_PREDICT);
    S.ms_csr = ev_ms(ctx, EV_PREDICT, EV_CSR);
    S.ms_bfs = ev_ms(ctx, EV_CSR, EV_BFS);
    S.ms_sv = ctx->ev_used[EV_BFS] ? ev_ms(ctx, EV_BFS, EV_SV)
              : ctx->ev_used[EV_PREDICT] ? ev_ms(ctx, EV_PREDICT, EV_SV)
                                         : ev_ms(ctx, EV_START, EV_SV);
    S.ms_finalize = ev_ms(ctx, EV_SV, EV_END);
    S.ms_total = ev_ms(ctx, EV_START, EV_END);
    S.status = ctx->last_status;
    *out = S;
    return ctx->last_status;
}

const char *cc_strerror(cc_status s) {
    switch (s) {
        case CC_OK: return "ok";
        case CC_ERR_INVALID_ARG: return "invalid argument";
        case CC_ERR_INVALID_EDGE: return "edge id outside [0, n)";
        case CC_ERR_OOM: return "device workspace allocation failed";
        case CC_ERR_NO_CONVERGENCE: return "iteration cap exceeded";
        case CC_ERR_TIMEOUT: return "bounded device wait ran out";
        case CC_ERR_CUDA: return "CUDA runtime error";
        case CC_ERR_UNSUPPORTED: return "size outside the engine's limits";
    }
    return "unknown status";
}

}  // extern "C"

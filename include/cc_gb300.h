/*
 * cc_gb300.h - C ABI of the GB300 connected-components engine.
 *
 * The engine labels every vertex of an undirected graph G(V, E) with the
 * smallest vertex id of its connected component (Section 1, problem
 * statement; Section 3.1.1 and the Figure 1(b) caption: at termination every
 * tuple of a component carries the partition min(u, v1, v2)). It follows the
 * hybrid route of Algorithm 2 (Section 3.2):
 *   1. degree distribution of G,
 *   2. power-law fit + Kolmogorov-Smirnov statistic D; BFS runs iff D < tau,
 *   3. if so, a direction-optimizing BFS from the max-degree vertex claims
 *      its component and the visited pairs are filtered out,
 *   4. Shiloach-Vishkin iterations (Section 3.1, Algorithm 1 semantics: every
 *      partition joins its minimum neighbour, pointer doubling, completed
 *      partitions are excluded, Section 3.1.4) label the rest.
 * Labels are identical for every route; the route only changes the time.
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are device pointers (cudaMalloc / torch CUDA
 *    memory); pointers named *_host are host pointers. The caller owns all of
 *    them; the library never frees or retains them past the call and never
 *    writes to its inputs.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Work is enqueued on it in order. Unless noted otherwise the
 *    call returns after enqueueing; results are valid once the stream has
 *    reached that point.
 *  - Edge lists are [m][2] interleaved (u, v) pairs, row-major, of
 *    `id_bytes` (4: int32, 8: int64) each, vertex ids dense in [0, n).
 *    Self-loops and duplicate pairs are allowed. n must be < 2^32 - 1.
 *    Edge arrays must be 16-byte aligned (the kernels read them with 128-bit
 *    loads), and so must the label array of cc_labels (written with 128-bit
 *    stores); labels are written with the same id width as the edges.
 *  - Errors: argument errors are returned immediately and nothing is
 *    enqueued. Errors the device detects (an id outside [0, n), a run that
 *    exceeds the iteration cap) go to a device status word. cc_labels is
 *    stream-ordered: the word is copied to pinned host memory at the end of
 *    the call's stream work, and cc_get_stats() (which waits for the stream)
 *    returns it; the next cc_labels call returns it once if that work has
 *    finished by then; with options.debug_checks the call waits and returns
 *    it. The other labelling calls wait for their stream and return it. The
 *    contents of the outputs are then unspecified.
 *  - A context is not thread safe: use one context per host thread/stream.
 */
#ifndef CC_GB300_H
#define CC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cc_ctx cc_ctx;

typedef enum {
    CC_OK = 0,
    CC_ERR_INVALID_ARG = 1,     /* bad pointer, size, option or alignment */
    CC_ERR_INVALID_EDGE = 2,    /* an edge id lies outside [0, n) */
    CC_ERR_OOM = 3,             /* device workspace allocation failed */
    CC_ERR_NO_CONVERGENCE = 4,  /* SV iteration cap or BFS level cap exceeded */
    CC_ERR_TIMEOUT = 5,         /* a bounded device wait ran out */
    CC_ERR_CUDA = 6,            /* a CUDA runtime call failed */
    CC_ERR_UNSUPPORTED = 7      /* size outside the engine's limits */
} cc_status;

/* Route policies (Algorithm 2 and its variants). */
enum {
    CC_ROUTE_AUTO = 0,      /* K-S heuristic of Section 3.2: BFS iff D < ks_tau */
    CC_ROUTE_LEARNED = 1,   /* learned predictor (needs cc_set_predictor); K-S decides when unsure */
    CC_ROUTE_FORCE_BFS = 2, /* always BFS first (the "opposite decision" experiment of Section 5) */
    CC_ROUTE_FORCE_SV = 3   /* SV only, no prediction */
};

/* Host-side fault injection bits (tests only; no GPU fault is ever caused). */
enum {
    CC_FAULT_NONE = 0,
    CC_FAULT_ALLOC = 1,      /* the next workspace allocation fails -> CC_ERR_OOM */
    CC_FAULT_ITER_CAP = 2    /* SV iteration cap forced to 1 -> CC_ERR_NO_CONVERGENCE on any graph needing more */
};

typedef struct {
    int id_bytes;           /* 4 or 8; default 4 */
    int route_policy;       /* CC_ROUTE_*; default CC_ROUTE_AUTO */
    double ks_tau;          /* default 0.05 (Section 5, Table 2) */
    int ks_min_tail;        /* smallest tail (vertices) an xmin candidate may have; default 50 */
    int ks_min_distinct;    /* fewest distinct degrees in a candidate tail; default 3 */
    int max_iters;          /* SV iteration cap; 0 = default 64 + 4*ceil(log2 n) */
    int bfs_cutoff_levels;  /* stop BFS after this many levels; 0 = run to completion */
    int debug_checks;       /* 1: cc_labels waits for its stream and returns the device status */
    int fault_inject;       /* CC_FAULT_* bits */
    double ks_min_span;     /* a candidate tail must reach max degree >= ks_min_span * xmin; default 10 */
    int profile;            /* 1: time every kernel class with CUDA events (cc_stats.kernel_ms) */
    int bfs_mode;           /* BFS engine: 0 = direction-optimizing BFS on a CSR (default),
                               1 = edge-list BFS (each level one pass over the active pairs, no CSR);
                               the learned route always uses 1 */
    int sv_sample_stride;   /* SV front end: before the first pass over all pairs, hook passes over
                               one block of pairs in k (k = sv_sample_stride, 1..1024) join most of
                               every large component; 0 = default (from 2^22 pairs: k = the largest
                               power of two <= 2m/n, at most 64, none if that is below 4), 1 = none;
                               the batched form, when this is > 1, samples each graph by that rule on
                               its own m_g and n_g (off by default);
                               the labels are the same either way */
    int bfs_starts;         /* BFS starts: 0 or 1 = one tree from the max-degree vertex (Algorithm 2);
                               k in 2..4096 = the multi-start BFS: [0, n) is cut into k ranges
                               [j n / k, (j + 1) n / k) and each range's max-degree vertex (ties to
                               the smallest id) starts a tree unless its degree is 0; the trees grow
                               together on the edge-list engine, pairs inside one tree leave the
                               active list and each tree's vertices take its smallest vertex as
                               parent before SV. Used by the K-S heuristic and forced routes (the
                               learned route keeps one sampled start); the labels are the same */
    int batch_hook_regions; /* batched form, tile order of the hook passes over the pairs: 0 = the tuner's
                               choice (default), -1 = a grid stride, k > 0 = k contiguous regions of the
                               pairs worked on side by side, each in order */
    int reserved;
} cc_options;

/* Kernel classes reported in cc_stats.kernel_ms / kernel_launches. */
enum {
    CC_K_DEGREE = 0,        /* degree pass over the pairs */
    CC_K_HIST = 1,          /* degree histogram + argmax */
    CC_K_KS = 2,            /* distinct degrees + power-law fit + K-S (six small kernels) */
    CC_K_SCAN = 3,          /* prefix sums (CSR offsets, frontier offsets) */
    CC_K_CSR = 4,           /* CSR scatter */
    CC_K_BFS_TOPDOWN = 5,
    CC_K_BFS_BOTTOMUP = 6,
    CC_K_BFS_AUX = 7,       /* frontier conversions, degrees, visited count / minimum */
    CC_K_PARENT_INIT = 8,
    CC_K_SV_FIRST = 9,      /* first SV pass over the caller's pairs (no gathers) */
    CC_K_SV_GATHER_INPUT = 10, /* SV pass with parent gathers over the caller's pairs */
    CC_K_SV_GATHER_LIST = 11,  /* SV pass over the compacted active list */
    CC_K_SV_SHORTCUT = 12,
    CC_K_FINALIZE = 13,
    CC_K_PREDICT = 14,      /* sampled route features + network inference */
    CC_K_TUPLE_SORT = 15,   /* radix sorts of cc_labels_tuple_sv (the rest of its time is ms_total) */
    CC_K_COUNT = 16
};

#define CC_MAX_SV_ITERS_RECORDED 64

typedef struct {
    int status;             /* cc_status of the last call's device work */
    int route;              /* 1 = BFS then SV, 0 = SV only */
    int route_source;       /* 0 = K-S heuristic, 1 = learned predictor, 2 = forced */
    int bfs_levels;         /* BFS levels run */
    int sv_iters;           /* SV iterations run */
    int degree_form;        /* exact degree pass of a single-graph call: 0 = none ran, 1 = one L2
                               atomic per endpoint, 2 = hub table, 3 = windows of 2^23 vertices
                               counted in L2 (n > 2^25), 4 = windows counted in shared memory
                               (2^20 <= n <= 2^24) */
    double ks_d;            /* K-S statistic (min over xmin); 1.0 if no candidate */
    double ks_alpha;        /* power-law exponent at the chosen xmin */
    int64_t ks_xmin;        /* chosen xmin; 0 if no candidate */
    int64_t ks_ntail;       /* vertices in the chosen tail */
    int64_t ks_ncand;       /* number of xmin candidates */
    int64_t n, m;           /* problem size of the last call */
    int64_t max_degree;     /* largest vertex degree */
    int64_t seed_vertex;    /* BFS seed: max-degree vertex, ties to the smallest id */
    int64_t bfs_visited;    /* vertices claimed by BFS */
    int64_t comp_min;       /* smallest id among the BFS-visited vertices */
    int64_t bfs_edges_inspected; /* adjacency entries the BFS read */
    int64_t m_active[CC_MAX_SV_ITERS_RECORDED]; /* active pairs entering each SV iteration */
    float ms_degree, ms_predict, ms_csr, ms_bfs, ms_sv, ms_finalize, ms_total; /* device stage times */
    float pad1;
    int64_t launches;                   /* kernels this library launched in the call */
    float kernel_ms[CC_K_COUNT];        /* summed device time per kernel class (options.profile = 1) */
    int32_t kernel_launches[CC_K_COUNT];/* launches per kernel class (options.profile = 1) */
    int64_t sv_hooks[CC_MAX_SV_ITERS_RECORDED]; /* roots hooked in each SV iteration */
    float pred_confidence;              /* learned policy: probability of the predicted route */
    int pred_route;                     /* learned policy: predicted route (-1 if none) */
    int pred_cutoff;                    /* learned policy: predicted BFS cutoff (0 = none) */
    float ms_features;                  /* learned policy: device time of features + inference */
    int32_t batch_unroll;               /* batched form: tuned 16-byte vectors per thread per tile of the hook passes */
    int32_t batch_grid_mult;            /* batched form: tuned blocks per launch, in resident-grid multiples */
    int32_t sv_sample_stride;           /* SV front end: one block of pairs in this many was sampled (1 = no
                                           front end; 0 = no first pass over the input pairs in this call;
                                           -1 = batched form, each graph with its own stride) */
    int32_t batch_deg_regions;          /* batched form: tuned regions of the pairs the degree pass works on side by side;
                                           0 = the degree pass counted in shared-memory windows (2^20 pairs or more) */
    int32_t bfs_starts;                 /* BFS trees started (0 if the BFS did not run) */
    int32_t batch_sv_regions;           /* batched form: tuned tile order of the hook passes (0 = grid stride,
                                           else regions of the pairs worked on side by side) */
} cc_stats;

/* Fills *opt with the defaults listed above. */
cc_status cc_default_options(cc_options *opt);

/*
 * Creates a context bound to CUDA device `device`. opt == NULL takes the
 * defaults. The context owns a device workspace that grows on demand (the
 * first call at a new size allocates; later calls at that size or below do
 * not) and is freed by cc_destroy.
 */
cc_status cc_create(cc_ctx **out, const cc_options *opt, int device);

/* Replaces the context's options (same meaning as in cc_create). */
cc_status cc_set_options(cc_ctx *ctx, const cc_options *opt);

/* Frees the workspace and the context. NULL is accepted. */
cc_status cc_destroy(cc_ctx *ctx);

/*
 * Connected-component labels of one graph (Algorithm 2, Section 3.2).
 *   edges_dev      [m][2] pairs of id_bytes each (device, 16-byte aligned)
 *   n              vertices, 0 <= n < 2^32 - 1
 *   m              pairs, m >= 0 (m = 0 gives labels_out[v] = v)
 *   labels_out_dev [n] ids of id_bytes each (device, 16-byte aligned);
 *                  labels_out[v] = min id of v's component
 * Stream-ordered (options.profile = 0): every decision of the route - the
 * K-S route (or the learned one), the BFS levels and their direction, the
 * SV iterations - is taken on the device by conditional nodes of one CUDA
 * graph, which the context captures once per set of arguments, options and
 * workspace and then launches on `stream`. The call returns without waiting
 * for the device; the labels are complete when `stream` reaches that point.
 * If `stream` is being captured into a CUDA graph, the work is captured into
 * the caller's graph instead (replays may change the contents of edges_dev,
 * not n, m or the pointers); a capture needs a workspace already sized by an
 * earlier call of at least that size (else CC_ERR_UNSUPPORTED, nothing
 * enqueued) and options.profile = 0.
 * With options.profile = 1 the route is driven from the host (it waits on
 * `stream` to read the route and the active-pair counts) and every kernel
 * class is timed with CUDA events; the labels are the same.
 * Device-detected errors: see the conventions above.
 */
cc_status cc_labels(cc_ctx *ctx, const void *edges_dev, int64_t n, int64_t m, void *labels_out_dev, void *stream);

/*
 * cc_labels for a graph whose pairs and labels are in host memory (Algorithm
 * 2, Section 3.2). With the K-S route or forced SV, m >= 2^24 and no
 * iteration cap or fault injection set, the pairs are copied to the device
 * in at most 32 chunks (of at least 2^23 pairs) on a copy stream, and each
 * chunk is consumed as it lands: its degrees are counted (Section 3.2) and
 * one SV iteration (Section 3.1: hook on the current roots, shortcut)
 * runs over its pairs, keeping the pairs that crossed roots. After the copy
 * the route is predicted from the complete histogram; the SV route
 * continues with the kept pairs, the BFS route starts over from the device
 * copy. Otherwise the pairs are copied once and cc_labels runs.
 *   edges_host      [m][2] pairs of id_bytes each, host memory; page-locked
 *                   memory (cudaHostAlloc / cudaHostRegister) lets the copies
 *                   overlap the passes, pageable memory works but is slower
 *   n, m            as cc_labels
 *   labels_out_host [n] ids of id_bytes each, host memory
 *   stream          cudaStream_t as void*
 * The context keeps device copies of the pairs and labels (grown on demand,
 * freed by cc_destroy). The call returns with the labels in labels_out_host.
 * Errors as cc_labels; on an error labels_out_host is not written.
 */
cc_status cc_labels_host(cc_ctx *ctx, const void *edges_host, int64_t n, int64_t m, void *labels_out_host,
                         void *stream);

/*
 * Labels of G independent graphs in one call (the batched form). Under the
 * K-S policy (and the learned one, which the batch treats the same way)
 * every graph gets its own route prediction, as cc_ks_statistic_batched:
 * one degree pass over all graphs, then the per-graph fits (largest graph
 * first) beside the first SV hook pass over all graphs (which needs no
 * route: every vertex starts as its own root); the graphs routed to BFS take
 * the BFS step together (one edge-list BFS from all their seeds); then the
 * SV iterations run over the union of all graphs. CC_ROUTE_FORCE_SV skips
 * the prediction; CC_ROUTE_FORCE_BFS sends every graph to BFS.
 * cc_get_stats: route = number of graphs that took the BFS step.
 *   edges_dev          concatenated int32 pairs with ids local to each graph (16-byte aligned)
 *   edge_offsets_dev   [G+1] int64 (device): graph g owns pairs [eo[g], eo[g+1])
 *   vertex_offsets_dev [G+1] int64 (device): graph g owns vertices [vo[g], vo[g+1]) of labels_out
 *   m_total, n_total   eo[G] and vo[G] (the host sizes the workspace from them)
 *   labels_out_dev     [n_total] int32 (device): local labels, min local id of each component
 * Stream-ordered like cc_labels (options.profile = 0): the offsets stay on
 * the device; every decision (the routes, the overflow fallback of the fits,
 * the BFS levels, the SV iterations) is taken on the device by conditional
 * nodes of one CUDA graph, captured once per arguments and workspace and
 * launched on `stream` (or captured into the caller's graph). The offsets
 * are checked on the device: not non-decreasing from 0 to the totals gives
 * the device status CC_ERR_INVALID_ARG (no kernel reads unchecked offsets).
 * The first call of a shape (log2 of pairs and graphs) with m_total >= 2^24
 * tunes the schedule of the hook passes (it waits on `stream`). With
 * options.profile = 1 the offsets are read back and the route is driven from
 * the host. Works for id_bytes = 4 only; n_total < 2^31.
 */
cc_status cc_labels_batched(cc_ctx *ctx, const void *edges_dev, const int64_t *edge_offsets_dev,
                            const int64_t *vertex_offsets_dev, int G, int64_t m_total, int64_t n_total,
                            void *labels_out_dev, void *stream);

/*
 * Degree pass and degree distribution (Section 3.2, Algorithm 2 line 1):
 *   deg_out_dev  [n] uint32 (device): number of pair endpoints equal to v
 *                (a self-loop adds 2, duplicates count)
 *   hist_out_dev [hist_len] uint64 (device): hist[d] = #{v : deg[v] = d} for d < hist_len
 *                (degrees >= hist_len are not counted; pass NULL to skip)
 * Either output may be NULL. Returns CC_ERR_INVALID_EDGE (after a stream
 * synchronisation) if an id is outside [0, n).
 */
cc_status cc_degree_distribution(cc_ctx *ctx, const void *edges_dev, int64_t n, int64_t m, uint32_t *deg_out_dev,
                                 uint64_t *hist_out_dev, int64_t hist_len, void *stream);

/*
 * Power-law fit + K-S statistic of a degree histogram (Section 3.2, Table 2),
 * computed on the device:
 *   hist_dev [hist_len] uint64 (device) counts per degree
 *   out_host [5] doubles (host): D, alpha, xmin, tail size, candidates
 * Synchronises `stream`.
 */
cc_status cc_ks_statistic(cc_ctx *ctx, const uint64_t *hist_dev, int64_t hist_len, double *out_host, void *stream);

/*
 * Learned route predictor (the learned form of the route choice of Section
 * 3.2: it replaces the K-S threshold only in choosing BFS first vs SV only
 * and the BFS cutoff; labels never depend on it).
 *
 * Network 69 -> 128 (ReLU) -> 128 (ReLU) -> 3, parameters in one fp32 array
 * of CC_MLP_PARAMS floats: [W1 (128 x 69, row-major) | b1 (128) |
 * W2 (128 x 128) | b2 (128) | W3 (3 x 128) | b3 (3)]. Outputs: two route
 * logits (0 = SV only, 1 = BFS first) and the natural log of the BFS cutoff
 * in levels. Features (see cc_route_features) are CC_MLP_IN floats.
 */
#define CC_MLP_IN 69
#define CC_MLP_HIDDEN 128
#define CC_MLP_OUT 3
#define CC_MLP_PARAMS (128 * 69 + 128 + 128 * 128 + 128 + 3 * 128 + 3)

/*
 * Route features of a graph, computed on the device from samples:
 *   [0, 64)  log2-degree histogram (bucket 0: degree 0, bucket b: degrees in
 *            [2^(b-1), 2^b)) of the vertices whose id is a multiple of 16, as
 *            fractions of those vertices
 *   64, 65   ln(n) / 20, ln(m + 1) / 20
 *   66..68   ln(1 + vertices reached) / 20 at BFS levels 1, 2, 3 from the
 *            sampled vertex of highest degree, over the pairs of every 16th
 *            block of 256 pairs
 *   edges_dev, n, m as in cc_labels; feat_out_dev [CC_MLP_IN] floats (device).
 * Enqueued on `stream`; returns CC_ERR_INVALID_EDGE (after synchronising) for
 * an id outside [0, n).
 */
cc_status cc_route_features(cc_ctx *ctx, const void *edges_dev, int64_t n, int64_t m, float *feat_out_dev,
                            void *stream);

/*
 * Installs predictor parameters (host, CC_MLP_PARAMS floats) into the
 * context, converted to bf16 weights with fp32 biases for inference. With
 * route_policy CC_ROUTE_LEARNED, cc_labels then computes the features,
 * runs the network, and takes its route (and cutoff) when the predicted
 * route's softmax probability is at least min_confidence; otherwise the K-S
 * heuristic decides. params_host == NULL removes the predictor (the learned
 * policy then falls back to the heuristic on every call).
 */
cc_status cc_set_predictor(cc_ctx *ctx, const float *params_host, double min_confidence);

/*
 * Training kernels (fp32), all device pointers, nothing allocated:
 *   cc_mlp_forward:  X [B][CC_MLP_IN] -> act [B * (2 * CC_MLP_HIDDEN + CC_MLP_OUT)]
 *                    = [H1 (B x 128) | H2 (B x 128) | O (B x 3)]
 *   cc_mlp_backward: gradients of the batch-mean loss
 *                    CE(O[:, 0:2], y) + lambda * w * (O[:, 2] - t)^2
 *                    into grad [CC_MLP_PARAMS]; scratch holds
 *                    B * (3 + 2 * CC_MLP_HIDDEN) floats; the batch loss is
 *                    added into *loss_dev (one float)
 *   cc_mlp_adam:     one Adam step (step t >= 1, bias-corrected) on count floats
 */
cc_status cc_mlp_forward(const float *params_dev, const float *X_dev, int B, float *act_dev, void *stream);
cc_status cc_mlp_backward(const float *params_dev, const float *X_dev, const int *y_dev, const float *t_dev,
                          const float *w_dev, int B, float lambda, const float *act_dev, float *grad_dev,
                          float *scratch_dev, float *loss_dev, void *stream);
cc_status cc_mlp_adam(float *params_dev, const float *grad_dev, float *m_dev, float *v_dev, int count, float lr,
                      float beta1, float beta2, float eps, int t, void *stream);

/* Size limits of cc_labels_static: its scratch is compiled into the library. */
#define CC_STATIC_MAX_VERTICES (1 << 20)
#define CC_STATIC_MAX_PAIRS (1 << 21)

/*
 * Connected-component labels without any device allocation. The paper has no
 * counterpart: this entry point exists for callers that may not allocate
 * device memory themselves - a plugin inside an application whose memory
 * pool owns the whole device, or a latency-critical loop where cudaMalloc /
 * cudaFree (which can synchronise the device) are not allowed.
 *
 * It runs the SV-only route of cc_labels (no degree pass, no prediction, no
 * BFS; the labels are the same: min id of each component) on a scratch area
 * that is a file-scope __device__ array of the library, about 40 MB, held
 * by every GPU that loads the library until the process exits. It calls no
 * cudaMalloc, cudaFree or allocating library routine, and needs no context.
 *   edges_dev      [m][2] pairs of id_bytes (4 or 8) each, device, 16-byte aligned
 *   n, m           at most CC_STATIC_MAX_VERTICES vertices and CC_STATIC_MAX_PAIRS
 *                  pairs; larger sizes return CC_ERR_UNSUPPORTED before any work
 *   labels_out_dev [n] ids of id_bytes each, device, 16-byte aligned
 *   stream         cudaStream_t as void*
 * Errors as cc_labels (CC_ERR_INVALID_EDGE for an id outside [0, n)). The
 * call synchronises `stream` once per SV iteration (it reads the active-pair
 * count back) and returns with the labels complete.
 * Every call looks up the device address of the scratch array
 * (cudaGetSymbolAddress) on the current device, so it stays valid across a
 * device reset. Every call on a device shares the one scratch area and
 * clears the parts that must start at zero; calls that overlap on the GPU
 * (other streams or host threads) race and must be serialised by the
 * caller.
 */
cc_status cc_labels_static(const void *edges_dev, int id_bytes, int64_t n, int64_t m, void *labels_out_dev,
                           void *stream);

/*
 * The paper's own SV design on the GPU, for comparison with cc_labels
 * (Section 3.1): the bag of tuples of Section 3.1.1 (one (x, x) per vertex,
 * (u, v) and (v, u) per pair; a tuple holds a partition and a vertex),
 * grouped by radix sorts. Every iteration runs two join rounds: grouped by
 * vertex, each vertex nominates the smallest partition among its tuples;
 * grouped by partition, each partition moves to the smallest nomination of
 * its tuples. The second round carries one extra tuple (t, t) per target t
 * of the first, which moves t on as well (the pointer doubling of Fig. 3).
 * Completed partitions (Section 3.1.4: every vertex of the partition has
 * tuples of that partition only) are detected in the first round; their
 * labels are written and their tuples leave the working set after the
 * iteration. The run stops after the first iteration in which no partition
 * moved; a vertex's label is then its partition, the minimum id of its
 * component - the labels of cc_labels. No route prediction or BFS.
 *   edges_dev      [m][2] pairs of the context's id width, device
 *   n              vertices, n < 2^31 (else CC_ERR_UNSUPPORTED)
 *   labels_out_dev [n] ids of the context's id width, device
 *   stream         cudaStream_t as void*; the call synchronises it once per
 *                  iteration and returns with the labels complete
 * cc_get_stats reports the iterations (sv_iters), the tuples in the working
 * set entering each iteration (m_active[i - 1] for iteration i) and the time
 * (ms_sv, ms_total). The context keeps a workspace of 52 bytes per tuple
 * slot (2n + 2m slots: the n + 2m tuples and up to n extras) until
 * cc_destroy.
 * Errors: as cc_labels; CC_ERR_NO_CONVERGENCE past the iteration cap.
 */
cc_status cc_labels_tuple_sv(cc_ctx *ctx, const void *edges_dev, int64_t n, int64_t m, void *labels_out_dev,
                             void *stream);

/* Measured L2 random-access rates of the context's device: the ceiling of
 * the kernels whose cost is scattered 4-byte accesses to an L2-resident
 * array rather than streamed bytes (the degree pass of Section 3.2 and the
 * hook passes of Section 3.1, on the parent and degree arrays). Each rate is
 * operations per second of one grid-stride kernel that issues `ops` accesses
 * to a table of `table_words` 32-bit words at indices from a 64-bit mixing
 * hash of the operation number; the best of `reps` timed launches (CUDA
 * events on `stream`) counts.
 *   out     host struct, written on success
 *   stream  cudaStream_t as void*; the call synchronises it
 * The probe allocates and frees its own table (4 * table_words bytes).
 * Errors: CC_ERR_INVALID_ARG for a null pointer; CC_ERR_CUDA. */
typedef struct cc_l2_rates {
    double gather;       /* loads per second */
    double red_add;      /* atomicAdd with the result unused (RED) */
    double red_min;      /* atomicMin with the result unused (RED) */
    double atom_min;     /* atomicMin with the result used (ATOM) */
    int64_t table_words; /* 2^24 (64 MiB) */
    int64_t ops;         /* 2^28 per launch */
    int32_t reps;        /* 3 */
    int32_t grid;        /* blocks of 256 threads */
} cc_l2_rates;
cc_status cc_measure_l2_rates(cc_ctx *ctx, cc_l2_rates *out, void *stream);

/*
 * Route prediction of every graph of a batch (Algorithm 2 lines 1-3 and the
 * power-law fit of Section 3.2, per graph): the degrees of each graph, its
 * degree histogram, the K-S statistic D (minimum over candidate xmin, as
 * cc_ks_statistic), the route and the max-degree seed. cc_labels_batched
 * makes the same prediction under the K-S policy. Arguments as
 * cc_labels_batched, plus host output arrays of G entries each:
 *   D_host, alpha_host   statistic and exponent at the selected xmin (1, 0 without a candidate)
 *   xmin_host, ncand_host  selected xmin (0 without a candidate), number of candidates
 *   route_host           1 = BFS first (D < ks_tau), 0 = SV only
 *   seed_host            local id of the max-degree vertex (ties to the smallest id)
 * The call reads the offsets back, waits for `stream` and returns the
 * outputs. Errors as cc_labels_batched (offset errors returned directly).
 */
cc_status cc_ks_statistic_batched(cc_ctx *ctx, const void *edges_dev, const int64_t *edge_offsets_dev,
                                  const int64_t *vertex_offsets_dev, int G, int64_t m_total, int64_t n_total,
                                  double *D_host, double *alpha_host, int64_t *xmin_host, int64_t *ncand_host,
                                  int32_t *route_host, int64_t *seed_host, void *stream);

/* Statistics of the last cc_labels call; waits for its stream. Returns the device status of that call.
 * After a stream-ordered call the per-stage times other than ms_total are 0 (they need options.profile). */
cc_status cc_get_stats(cc_ctx *ctx, cc_stats *out);

/* Static, human-readable description of a status. */
const char *cc_strerror(cc_status s);

#ifdef __cplusplus
}
#endif

#endif /* CC_GB300_H */

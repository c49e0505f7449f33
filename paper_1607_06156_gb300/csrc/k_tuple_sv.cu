// The paper's sort-based Shiloach-Vishkin (Section 3.1) on the GPU: an
// ablation beside the atomic parent-array SV of the hot path.
//
// State: the bag of tuples of Section 3.1.1, one (x, x) per vertex and
// (u, v), (v, u) per pair, stored as two 32-bit words per tuple: the vertex
// r (never changes) and the partition p (bit 31 marks an extra tuple). The
// paper's unit of work is a sort of the bag by one key followed by a scan of
// each run of equal keys; here the sort is a radix sort and the scan a
// reduce-by-key.
//
// A join round moves every partition to its smallest candidate: grouped by
// vertex, each vertex r nominates the smallest partition among its tuples;
// grouped by partition, each partition moves to the smallest nomination of
// its tuples. An iteration is two join rounds: the plain one, then the
// pointer doubling of Fig. 3, where one extra tuple (t, t) per target t of
// the first round lets t itself move on to the smallest partition at vertex
// t; the extras are dropped after it. The run ends after the first
// iteration in which no partition moved; the label of r is then the
// partition of its tuples (Section 3.1.1).
//
// Completed partitions (Section 3.1.4) are found during the plain round: a
// vertex whose tuples all share one partition marks them "potentially
// completed" (the largest and the smallest partition at the vertex agree),
// and a partition all of whose tuples are so marked is completed, i.e. a
// whole component. After the iteration its labels are written and its
// tuples leave the bag, so the sorts shrink with the working set.
//
// The radix sort, reduce-by-key and select are CUB's (shipped with the CUDA
// toolkit): the comparison is between the sort-based design and the atomic
// one, not between sort implementations. Ids are below 2^31.
#include "cc_common.cuh"
#include "cc_kernels.h"

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_reduce.cuh>
#include <cub/device/device_select.cuh>

#include <vector>

namespace ccg {

constexpr uint32_t kTmpBit = 0x80000000u, kIdMask = 0x7fffffffu;

// The initial bag: R = vertex r, PT = partition p (| extra bit)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_tsv_init(const T *__restrict__ edges, long long m, vid_t n,
                                                     uint32_t *R, uint32_t *PT, DevState *st) {
    for (long long i = gtid(); i < (long long)n + m; i += gstride()) {
        if (i < (long long)n) {
            R[i] = (uint32_t)i;
            PT[i] = (uint32_t)i;
            continue;
        }
        const long long k = i - n;
        const long long u = (long long)edges[2 * k], v = (long long)edges[2 * k + 1];
        const bool ok = u >= 0 && v >= 0 && u < (long long)n && v < (long long)n;
        if (!ok) set_err(st, kErrInvalidEdge);
        const uint32_t a = ok ? (uint32_t)u : 0u, b = ok ? (uint32_t)v : 0u;
        const long long j = n + 2 * k;
        R[j] = b;  // (u, v): partition u at vertex v
        PT[j] = a;
        R[j + 1] = a;
        PT[j + 1] = b;
    }
}

__global__ void __launch_bounds__(kBlock) k_tsv_low31(const uint32_t *__restrict__ in, uint32_t *out, long long len) {
    for (long long i = gtid(); i < len; i += gstride()) out[i] = in[i] & kIdMask;
}

// Partition-grouped values: the nomination (31 bits) and, with `notpc`, the
// "not potentially completed" bit of the tuple (bit 63 of the packed value).
__global__ void __launch_bounds__(kBlock) k_tsv_split(const unsigned long long *__restrict__ in, uint32_t *nom,
                                                      uint32_t *notpc, long long len) {
    for (long long i = gtid(); i < len; i += gstride()) {
        const unsigned long long x = in[i];
        nom[i] = (uint32_t)(x >> 32) & kIdMask;
        if (notpc) notpc[i] = (uint32_t)(x >> 63);
    }
}

// dense[key] = the run's reduced value, for every run (runs: the reduce-by-key
// output); with `changed`, flags a run whose minimum differs from its key
__global__ void __launch_bounds__(kBlock) k_tsv_scatter(const uint32_t *__restrict__ keys,
                                                        const uint32_t *__restrict__ vals,
                                                        const unsigned long long *runs, uint32_t *dense,
                                                        unsigned long long *changed) {
    const long long nr = (long long)*runs;
    bool c = false;
    for (long long k = gtid(); k < nr; k += gstride()) {
        dense[keys[k]] = vals[k];
        c |= vals[k] != keys[k];
    }
    if (changed && __any_sync(0xffffffffu, c) && (threadIdx.x & 31) == 0) *changed = 1ull;
}

// pc[r] = 1 when every tuple at vertex r has the same partition: the largest
// partition at r (maxs) equals the smallest (umin[r])
__global__ void __launch_bounds__(kBlock) k_tsv_vertex_pc(const uint32_t *__restrict__ keys,
                                                          const uint32_t *__restrict__ maxs,
                                                          const unsigned long long *runs,
                                                          const uint32_t *__restrict__ umin, uint32_t *pc) {
    const long long nr = (long long)*runs;
    for (long long k = gtid(); k < nr; k += gstride()) pc[keys[k]] = maxs[k] == umin[keys[k]] ? 1u : 0u;
}

// done[p] = 1 when no tuple of partition p lacks the potentially-completed mark
__global__ void __launch_bounds__(kBlock) k_tsv_done(const uint32_t *__restrict__ keys,
                                                     const uint32_t *__restrict__ any_not,
                                                     const unsigned long long *runs, uint32_t *done) {
    const long long nr = (long long)*runs;
    for (long long k = gtid(); k < nr; k += gstride()) done[keys[k]] = any_not[k] == 0 ? 1u : 0u;
}

// vertex grouping -> partition grouping: key p, value
// (nomination | not-potentially-completed << 31) << 32 | (r | extra bit)
__global__ void __launch_bounds__(kBlock) k_tsv_to_partition(const uint32_t *__restrict__ R,
                                                             const uint32_t *__restrict__ PT,
                                                             const uint32_t *__restrict__ umin,
                                                             const uint32_t *__restrict__ pc, uint32_t *P,
                                                             unsigned long long *V, long long len) {
    for (long long i = gtid(); i < len; i += gstride()) {
        const uint32_t r = R[i], pt = PT[i];
        const uint32_t notpc = pc && !pc[r] ? kTmpBit : 0u;
        P[i] = pt & kIdMask;
        V[i] = ((unsigned long long)(umin[r] | notpc) << 32) | (unsigned long long)(r | (pt & kTmpBit));
    }
}

// partition grouping -> next vertex grouping: p <- its target, the vertex
// and the extra bit carried over
__global__ void __launch_bounds__(kBlock) k_tsv_to_vertex(const uint32_t *__restrict__ P,
                                                          const unsigned long long *__restrict__ V,
                                                          const uint32_t *__restrict__ target, uint32_t *R,
                                                          uint32_t *PT, long long len) {
    for (long long i = gtid(); i < len; i += gstride()) {
        const uint32_t rt = (uint32_t)V[i];
        R[i] = rt & kIdMask;
        PT[i] = target[P[i]] | (rt & kTmpBit);
    }
}

// one extra tuple (t, t) per partition of the round, t its target (appended)
__global__ void __launch_bounds__(kBlock) k_tsv_append(const uint32_t *__restrict__ targets,
                                                       const unsigned long long *runs, uint32_t *R, uint32_t *PT) {
    const long long nr = (long long)*runs;
    for (long long k = gtid(); k < nr; k += gstride()) {
        R[k] = targets[k];
        PT[k] = targets[k] | kTmpBit;
    }
}

__global__ void __launch_bounds__(kBlock) k_tsv_pack(const uint32_t *__restrict__ R, const uint32_t *__restrict__ PT,
                                                     unsigned long long *V, long long len) {
    for (long long i = gtid(); i < len; i += gstride())
        V[i] = ((unsigned long long)PT[i] << 32) | (unsigned long long)R[i];
}

__global__ void __launch_bounds__(kBlock) k_tsv_unpack(const unsigned long long *__restrict__ V, uint32_t *R,
                                                       uint32_t *PT, long long len) {
    for (long long i = gtid(); i < len; i += gstride()) {
        R[i] = (uint32_t)V[i];
        PT[i] = (uint32_t)(V[i] >> 32);
    }
}

// labels of the vertices of completed partitions (`done` non-null) or of
// every tuple (`done` null, at convergence); extra tuples are skipped
template <typename T>
__global__ void __launch_bounds__(kBlock) k_tsv_labels(const uint32_t *__restrict__ R, const uint32_t *__restrict__ PT,
                                                       const uint32_t *__restrict__ done, T *labels, long long len) {
    for (long long i = gtid(); i < len; i += gstride()) {
        const uint32_t pt = PT[i];
        if (pt & kTmpBit) continue;
        if (done && !done[pt]) continue;
        labels[R[i]] = (T)pt;
    }
}

// select predicate: neither an extra tuple nor in a completed partition
struct KeepActive {
    const uint32_t *done;
    __host__ __device__ bool operator()(const unsigned long long &x) const {
        const uint32_t pt = (uint32_t)(x >> 32);
        return (pt & kTmpBit) == 0 && !done[pt];
    }
};

struct MinU32 {
    __host__ __device__ uint32_t operator()(const uint32_t &a, const uint32_t &b) const { return b < a ? b : a; }
};
struct MaxU32 {
    __host__ __device__ uint32_t operator()(const uint32_t &a, const uint32_t &b) const { return b > a ? b : a; }
};

int tsv_key_bits(vid_t n) {
    int b = 1;
    while (b < 31 && (1ull << b) < (unsigned long long)n) b++;
    return b;
}

size_t tuple_sv_temp_bytes(long long cap, vid_t n) {
    const int bits = tsv_key_bits(n);
    size_t a = 0, b = 0, c = 0, c2 = 0, d = 0;
    cub::DoubleBuffer<uint32_t> k32(nullptr, nullptr), v32(nullptr, nullptr);
    cub::DoubleBuffer<unsigned long long> v64(nullptr, nullptr);
    cub::DeviceRadixSort::SortPairs(nullptr, a, k32, v32, cap, 0, bits);
    cub::DeviceRadixSort::SortPairs(nullptr, b, k32, v64, cap, 0, bits);
    cub::DeviceReduce::ReduceByKey(nullptr, c, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                   (const uint32_t *)nullptr, (uint32_t *)nullptr, (unsigned long long *)nullptr,
                                   MinU32(), cap);
    cub::DeviceReduce::ReduceByKey(nullptr, c2, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                   (const uint32_t *)nullptr, (uint32_t *)nullptr, (unsigned long long *)nullptr,
                                   MaxU32(), cap);
    cub::DeviceSelect::If(nullptr, d, (const unsigned long long *)nullptr, (unsigned long long *)nullptr,
                          (unsigned long long *)nullptr, cap, KeepActive{nullptr});
    size_t mx = a;
    for (size_t x : {b, c, c2, d})
        if (x > mx) mx = x;
    return mx + 256;
}

// Optional timing of the radix sorts (CUDA events around each sort).
struct SortTimer {
    std::vector<cudaEvent_t> ev;
    bool on = false;
    void mark(cudaStream_t s) {
        if (!on) return;
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            on = false;
            return;
        }
        cudaEventRecord(e, s);
        ev.push_back(e);
    }
    // sum of the (begin, end) pairs after the stream has finished
    float total_ms() {
        float t = 0.0f;
        for (size_t i = 0; i + 1 < ev.size(); i += 2) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) t += ms;
            else cudaGetLastError();
        }
        return t;
    }
    ~SortTimer() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

// One join round over the len tuples in (R, PT), two of the four 32-bit
// tuple buffers (the other two are scratch); on return R and PT point at the
// buffers holding the moved tuples. `extras`: the round's extra tuples
// (t, t) follow them and len grows by their count. `detect`: b.done marks
// the completed partitions. Sets counters[1] when a partition moved.
static cudaError_t tsv_join(const TupleSvBufs &b, uint32_t *&R, uint32_t *&PT, long long &len, vid_t n, bool extras,
                            bool detect, SortTimer &timer, cudaStream_t s) {
    const int bits = tsv_key_bits(n);
    const int grid = 8 * b.num_sms;
    uint32_t *free_a = nullptr, *free_b = nullptr;
    for (int k = 0; k < 4; k++) {
        uint32_t *x = b.t32[k];
        if (x == R || x == PT) continue;
        (free_a ? free_b : free_a) = x;
    }
    cudaError_t e;
    // grouped by vertex: every vertex nominates the smallest partition at it
    cub::DoubleBuffer<uint32_t> vk(R, free_a), vv(PT, free_b);
    size_t tb = b.temp_bytes;
    timer.mark(s);
    if ((e = cub::DeviceRadixSort::SortPairs(b.temp, tb, vk, vv, len, 0, bits, s)) != cudaSuccess) return e;
    timer.mark(s);
    uint32_t *Rs = vk.Current(), *Ra = vk.Alternate(), *PTs = vv.Current(), *PTa = vv.Alternate();
    k_tsv_low31<<<grid, kBlock, 0, s>>>(PTs, b.val, len);
    if (detect) {
        tb = b.temp_bytes;
        if ((e = cub::DeviceReduce::ReduceByKey(b.temp, tb, Rs, b.uniq, b.val, b.val2, b.counters, MaxU32(), len,
                                                s)) != cudaSuccess)
            return e;
    }
    tb = b.temp_bytes;
    if ((e = cub::DeviceReduce::ReduceByKey(b.temp, tb, Rs, b.uniq, b.val, b.agg, b.counters, MinU32(), len, s)) !=
        cudaSuccess)
        return e;
    k_tsv_scatter<<<grid, kBlock, 0, s>>>(b.uniq, b.agg, b.counters, b.dense, nullptr);
    if (detect) k_tsv_vertex_pc<<<grid, kBlock, 0, s>>>(b.uniq, b.val2, b.counters, b.dense, b.pc);
    k_tsv_to_partition<<<grid, kBlock, 0, s>>>(Rs, PTs, b.dense, detect ? b.pc : nullptr, Ra, b.v0, len);
    // grouped by partition: every partition moves to the smallest nomination
    cub::DoubleBuffer<uint32_t> pk(Ra, Rs);
    cub::DoubleBuffer<unsigned long long> pv(b.v0, b.v1);
    tb = b.temp_bytes;
    timer.mark(s);
    if ((e = cub::DeviceRadixSort::SortPairs(b.temp, tb, pk, pv, len, 0, bits, s)) != cudaSuccess) return e;
    timer.mark(s);
    uint32_t *P = pk.Current(), *Pa = pk.Alternate();
    unsigned long long *V = pv.Current();
    k_tsv_split<<<grid, kBlock, 0, s>>>(V, b.val, detect ? b.val2 : nullptr, len);
    if (detect) {
        tb = b.temp_bytes;
        if ((e = cub::DeviceReduce::ReduceByKey(b.temp, tb, P, b.uniq, b.val2, b.agg, b.counters, MaxU32(), len,
                                                s)) != cudaSuccess)
            return e;
        k_tsv_done<<<grid, kBlock, 0, s>>>(b.uniq, b.agg, b.counters, b.done);
    }
    tb = b.temp_bytes;
    if ((e = cub::DeviceReduce::ReduceByKey(b.temp, tb, P, b.uniq, b.val, b.agg, b.counters, MinU32(), len, s)) !=
        cudaSuccess)
        return e;
    k_tsv_scatter<<<grid, kBlock, 0, s>>>(b.uniq, b.agg, b.counters, b.dense, b.counters + 1);
    // the moved tuples go to the two buffers the partition sort left free (PTs and PTa were consumed)
    uint32_t *Rn = Pa, *PTn = PTa == P ? PTs : PTa;
    k_tsv_to_vertex<<<grid, kBlock, 0, s>>>(P, V, b.dense, Rn, PTn, len);
    if (extras) {
        unsigned long long runs = 0;
        if ((e = cudaMemcpyAsync(&runs, b.counters, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if (len + (long long)runs > b.cap) return cudaErrorInvalidValue;
        k_tsv_append<<<grid, kBlock, 0, s>>>(b.agg, b.counters, Rn + len, PTn + len);
        len += (long long)runs;
    }
    R = Rn;
    PT = PTn;
    return cudaGetLastError();
}

template <typename T>
static int tuple_sv_iterate(const void *edges, long long m, vid_t n, void *labels, const TupleSvBufs &b, DevState *st,
                            int max_iters, int *iters_out, long long *active_out, int active_cap, SortTimer &timer,
                            cudaStream_t s) {
    *iters_out = 0;
    const long long T0 = (long long)n + 2 * m;
    if (T0 + (long long)n > b.cap) return 1;
    const int grid = 8 * b.num_sms;
    uint32_t *R = b.t32[0], *PT = b.t32[1];
    if (cudaMemsetAsync(b.done, 0, (size_t)n * 4, s) != cudaSuccess) return 1;
    k_tsv_init<T><<<grid, kBlock, 0, s>>>((const T *)edges, m, n, R, PT, st);
    if (cudaGetLastError() != cudaSuccess) return 1;
    long long active = T0;
    for (int it = 1; it <= max_iters; it++) {
        *iters_out = it;
        if (it - 1 < active_cap) active_out[it - 1] = active;
        if (cudaMemsetAsync(b.counters, 0, 32, s) != cudaSuccess) return 1;
        long long len = active;
        if (tsv_join(b, R, PT, len, n, true, true, timer, s) != cudaSuccess) return 1;
        if (tsv_join(b, R, PT, len, n, false, false, timer, s) != cudaSuccess) return 1;
        // completed partitions: labels now; then drop them and the extra tuples
        k_tsv_labels<T><<<grid, kBlock, 0, s>>>(R, PT, b.done, (T *)labels, len);
        k_tsv_pack<<<grid, kBlock, 0, s>>>(R, PT, b.v0, len);
        size_t tb = b.temp_bytes;
        if (cub::DeviceSelect::If(b.temp, tb, b.v0, b.v1, b.counters + 2, len, KeepActive{b.done}, s) !=
            cudaSuccess)
            return 1;
        unsigned long long h[3] = {0, 0, 0};
        if (cudaMemcpyAsync(h, b.counters, 24, cudaMemcpyDeviceToHost, s) != cudaSuccess) return 1;
        if (cudaStreamSynchronize(s) != cudaSuccess) return 1;
        if ((long long)h[2] > active) return 1;
        active = (long long)h[2];
        k_tsv_unpack<<<grid, kBlock, 0, s>>>(b.v1, R, PT, active);
        if (h[1] == 0 || active == 0) {  // no partition moved in either round
            k_tsv_labels<T><<<grid, kBlock, 0, s>>>(R, PT, nullptr, (T *)labels, active);
            return cudaGetLastError() == cudaSuccess ? 0 : 1;
        }
    }
    return 2;
}

template <typename T>
int tuple_sv_run(const void *edges, long long m, vid_t n, void *labels, TupleSvBufs b, DevState *st, int max_iters,
                 int *iters_out, long long *active_out, int active_cap, float *sort_ms, int *sorts, cudaStream_t s) {
    SortTimer timer;
    timer.on = sort_ms != nullptr;
    const int rc =
        tuple_sv_iterate<T>(edges, m, n, labels, b, st, max_iters, iters_out, active_out, active_cap, timer, s);
    if (sort_ms) {
        cudaStreamSynchronize(s);
        *sort_ms = timer.total_ms();
        *sorts = (int)(timer.ev.size() / 2);
    }
    return rc;
}

template int tuple_sv_run<int32_t>(const void *, long long, vid_t, void *, TupleSvBufs, DevState *, int, int *,
                                   long long *, int, float *, int *, cudaStream_t);
template int tuple_sv_run<int64_t>(const void *, long long, vid_t, void *, TupleSvBufs, DevState *, int, int *,
                                   long long *, int, float *, int *, cudaStream_t);

}  // namespace ccg

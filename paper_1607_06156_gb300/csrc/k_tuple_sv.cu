// The paper's sort-based Shiloach-Vishkin (Section 3.1, Algorithm 1) on the
// GPU: an ablation of the atomic parent-array SV the hot path runs.
//
// The state is the tuple array of Section 3.1.1: <x,_,x> for every vertex x
// and <u,_,v>, <v,_,u> for every pair, written <p, q, r> (partition,
// candidate, vertex). One iteration is
//   vertex pass      sort by r; q <- min p over the tuples of r's bucket VB(r)
//   partition pass   sort by p; p_min <- min q over the tuples of p's bucket
//                    PB(p); p <- p_min; "not converged" if p != p_min for any p
//   temporaries      one <p_min,_,p_min> per partition of the first partition
//                    pass; both passes run again with them (pointer doubling,
//                    Fig. 3), then the temporaries are erased
// and the run ends when neither partition pass changed a partition. The
// label of vertex r is then the partition of its tuples (Section 3.1.1).
//
// Groups are formed the way the paper forms them, by sorting: a radix sort
// of the tuples by the bucket key, then a min over each run of equal keys.
// Both primitives are CUB's (the radix sort and reduce-by-key shipped with
// the CUDA toolkit): the comparison is between the sort-based design and the
// atomic one, not between sort implementations. Ids are below 2^31 (bit 31
// of a tuple word marks a temporary).
#include "cc_common.cuh"
#include "cc_kernels.h"

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_reduce.cuh>
#include <cub/device/device_select.cuh>

#include <vector>

namespace ccg {

constexpr uint32_t kTmpBit = 0x80000000u, kIdMask = 0x7fffffffu;

// A_0: R = vertex (r), PT = partition (p) | temporary bit
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
        R[j] = b;  // <u,_,v>
        PT[j] = a;
        R[j + 1] = a;  // <v,_,u>
        PT[j + 1] = b;
    }
}

__global__ void __launch_bounds__(kBlock) k_tsv_low31(const uint32_t *__restrict__ in, uint32_t *out, long long len) {
    for (long long i = gtid(); i < len; i += gstride()) out[i] = in[i] & kIdMask;
}

__global__ void __launch_bounds__(kBlock) k_tsv_high32(const unsigned long long *__restrict__ in, uint32_t *out,
                                                       long long len) {
    for (long long i = gtid(); i < len; i += gstride()) out[i] = (uint32_t)(in[i] >> 32);
}

// dense[key] = the run's minimum, for every run (runs: the reduce-by-key
// output); with `changed`, flags a run whose minimum differs from its key
__global__ void __launch_bounds__(kBlock) k_tsv_scatter(const uint32_t *__restrict__ keys,
                                                        const uint32_t *__restrict__ mins,
                                                        const unsigned long long *runs, uint32_t *dense,
                                                        unsigned long long *changed) {
    const long long nr = (long long)*runs;
    bool c = false;
    for (long long k = gtid(); k < nr; k += gstride()) {
        dense[keys[k]] = mins[k];
        c |= mins[k] != keys[k];
    }
    if (changed && __any_sync(0xffffffffu, c) && (threadIdx.x & 31) == 0) *changed = 1ull;
}

// vertex pass -> partition pass: key p, value q << 32 | (r | temporary bit)
__global__ void __launch_bounds__(kBlock) k_tsv_to_partition(const uint32_t *__restrict__ R,
                                                             const uint32_t *__restrict__ PT,
                                                             const uint32_t *__restrict__ umin, uint32_t *P,
                                                             unsigned long long *V, long long len) {
    for (long long i = gtid(); i < len; i += gstride()) {
        const uint32_t r = R[i], pt = PT[i];
        P[i] = pt & kIdMask;
        V[i] = ((unsigned long long)umin[r] << 32) | (unsigned long long)(r | (pt & kTmpBit));
    }
}

// partition pass -> next vertex pass: p <- p_min, the vertex and the
// temporary bit carried over
__global__ void __launch_bounds__(kBlock) k_tsv_to_vertex(const uint32_t *__restrict__ P,
                                                          const unsigned long long *__restrict__ V,
                                                          const uint32_t *__restrict__ pmin, uint32_t *R,
                                                          uint32_t *PT, long long len) {
    for (long long i = gtid(); i < len; i += gstride()) {
        const uint32_t rt = (uint32_t)V[i];
        R[i] = rt & kIdMask;
        PT[i] = pmin[P[i]] | (rt & kTmpBit);
    }
}

// one temporary <p_min,_,p_min> per partition of the pass (appended)
__global__ void __launch_bounds__(kBlock) k_tsv_append(const uint32_t *__restrict__ mins,
                                                       const unsigned long long *runs, uint32_t *R, uint32_t *PT) {
    const long long nr = (long long)*runs;
    for (long long k = gtid(); k < nr; k += gstride()) {
        R[k] = mins[k];
        PT[k] = mins[k] | kTmpBit;
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

template <typename T>
__global__ void __launch_bounds__(kBlock) k_tsv_labels(const uint32_t *__restrict__ R, const uint32_t *__restrict__ PT,
                                                       T *labels, long long len) {
    for (long long i = gtid(); i < len; i += gstride()) labels[R[i]] = (T)(PT[i] & kIdMask);
}

struct NotTemporary {
    __host__ __device__ bool operator()(const unsigned long long &x) const { return ((x >> 32) & kTmpBit) == 0; }
};

struct MinU32 {
    __host__ __device__ uint32_t operator()(const uint32_t &a, const uint32_t &b) const { return b < a ? b : a; }
};

int tsv_key_bits(vid_t n) {
    int b = 1;
    while (b < 31 && (1ull << b) < (unsigned long long)n) b++;
    return b;
}

size_t tuple_sv_temp_bytes(long long cap, vid_t n) {
    const int bits = tsv_key_bits(n);
    size_t a = 0, b = 0, c = 0, d = 0;
    cub::DoubleBuffer<uint32_t> k32(nullptr, nullptr), v32(nullptr, nullptr);
    cub::DoubleBuffer<unsigned long long> v64(nullptr, nullptr);
    cub::DeviceRadixSort::SortPairs(nullptr, a, k32, v32, cap, 0, bits);
    cub::DeviceRadixSort::SortPairs(nullptr, b, k32, v64, cap, 0, bits);
    cub::DeviceReduce::ReduceByKey(nullptr, c, (const uint32_t *)nullptr, (uint32_t *)nullptr,
                                   (const uint32_t *)nullptr, (uint32_t *)nullptr, (unsigned long long *)nullptr,
                                   MinU32(), cap);
    cub::DeviceSelect::If(nullptr, d, (const unsigned long long *)nullptr, (unsigned long long *)nullptr,
                          (unsigned long long *)nullptr, cap, NotTemporary());
    size_t mx = a;
    if (b > mx) mx = b;
    if (c > mx) mx = c;
    if (d > mx) mx = d;
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

// One vertex pass and one partition pass over the len tuples in (R, PT),
// two of the four 32-bit tuple buffers (the other two are scratch); on
// return R and PT point at the buffers holding the new tuples. With
// `append`, the pass's temporaries follow them and len grows by their count.
// Sets counters[1] when a partition changed.
static cudaError_t tsv_half(const TupleSvBufs &b, uint32_t *&R, uint32_t *&PT, long long &len, vid_t n, bool append,
                            SortTimer &timer, cudaStream_t s) {
    const int bits = tsv_key_bits(n);
    const int grid = 8 * b.num_sms;
    uint32_t *free_a = nullptr, *free_b = nullptr;
    for (int k = 0; k < 4; k++) {
        uint32_t *x = b.t32[k];
        if (x == R || x == PT) continue;
        (free_a ? free_b : free_a) = x;
    }
    cudaError_t e;
    // vertex pass: sort by r, q <- min p per run of equal r
    cub::DoubleBuffer<uint32_t> vk(R, free_a), vv(PT, free_b);
    size_t tb = b.temp_bytes;
    timer.mark(s);
    if ((e = cub::DeviceRadixSort::SortPairs(b.temp, tb, vk, vv, len, 0, bits, s)) != cudaSuccess) return e;
    timer.mark(s);
    uint32_t *Rs = vk.Current(), *Ra = vk.Alternate(), *PTs = vv.Current(), *PTa = vv.Alternate();
    k_tsv_low31<<<grid, kBlock, 0, s>>>(PTs, b.val, len);
    tb = b.temp_bytes;
    if ((e = cub::DeviceReduce::ReduceByKey(b.temp, tb, Rs, b.uniq, b.val, b.agg, b.counters, MinU32(), len, s)) !=
        cudaSuccess)
        return e;
    k_tsv_scatter<<<grid, kBlock, 0, s>>>(b.uniq, b.agg, b.counters, b.dense, nullptr);
    k_tsv_to_partition<<<grid, kBlock, 0, s>>>(Rs, PTs, b.dense, Ra, b.v0, len);
    // partition pass: sort by p, p_min <- min q per run of equal p, p <- p_min
    cub::DoubleBuffer<uint32_t> pk(Ra, Rs);
    cub::DoubleBuffer<unsigned long long> pv(b.v0, b.v1);
    tb = b.temp_bytes;
    timer.mark(s);
    if ((e = cub::DeviceRadixSort::SortPairs(b.temp, tb, pk, pv, len, 0, bits, s)) != cudaSuccess) return e;
    timer.mark(s);
    uint32_t *P = pk.Current(), *Pa = pk.Alternate();
    unsigned long long *V = pv.Current();
    k_tsv_high32<<<grid, kBlock, 0, s>>>(V, b.val, len);
    tb = b.temp_bytes;
    if ((e = cub::DeviceReduce::ReduceByKey(b.temp, tb, P, b.uniq, b.val, b.agg, b.counters, MinU32(), len, s)) !=
        cudaSuccess)
        return e;
    k_tsv_scatter<<<grid, kBlock, 0, s>>>(b.uniq, b.agg, b.counters, b.dense, b.counters + 1);
    // the new tuples go to the two buffers the partition sort left free (PTs and PTa were consumed)
    uint32_t *Rn = Pa, *PTn = PTa == P ? PTs : PTa;
    k_tsv_to_vertex<<<grid, kBlock, 0, s>>>(P, V, b.dense, Rn, PTn, len);
    if (append) {
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
                            int max_iters, int *iters_out, SortTimer &timer, cudaStream_t s) {
    *iters_out = 0;
    const long long T0 = (long long)n + 2 * m;
    if (T0 + (long long)n > b.cap) return 1;
    const int grid = 8 * b.num_sms;
    uint32_t *R = b.t32[0], *PT = b.t32[1];
    k_tsv_init<T><<<grid, kBlock, 0, s>>>((const T *)edges, m, n, R, PT, st);
    if (cudaGetLastError() != cudaSuccess) return 1;
    for (int it = 1; it <= max_iters; it++) {
        *iters_out = it;
        if (cudaMemsetAsync(b.counters, 0, 32, s) != cudaSuccess) return 1;
        long long len = T0;
        if (tsv_half(b, R, PT, len, n, true, timer, s) != cudaSuccess) return 1;
        if (tsv_half(b, R, PT, len, n, false, timer, s) != cudaSuccess) return 1;
        // erase the temporaries: pack (PT, R), keep the words without the bit
        k_tsv_pack<<<grid, kBlock, 0, s>>>(R, PT, b.v0, len);
        size_t tb = b.temp_bytes;
        if (cub::DeviceSelect::If(b.temp, tb, b.v0, b.v1, b.counters + 2, len, NotTemporary(), s) != cudaSuccess)
            return 1;
        k_tsv_unpack<<<grid, kBlock, 0, s>>>(b.v1, R, PT, T0);
        unsigned long long h[3] = {0, 0, 0};
        if (cudaMemcpyAsync(h, b.counters, 24, cudaMemcpyDeviceToHost, s) != cudaSuccess) return 1;
        if (cudaStreamSynchronize(s) != cudaSuccess) return 1;
        if ((long long)h[2] != T0) return 1;  // the real tuples must all survive
        if (h[1] == 0) {                       // no partition changed in either pass
            k_tsv_labels<T><<<grid, kBlock, 0, s>>>(R, PT, (T *)labels, T0);
            return cudaGetLastError() == cudaSuccess ? 0 : 1;
        }
    }
    return 2;
}
template <typename T>
int tuple_sv_run(const void *edges, long long m, vid_t n, void *labels, TupleSvBufs b, DevState *st, int max_iters,
                 int *iters_out, float *sort_ms, int *sorts, cudaStream_t s) {
    SortTimer timer;
    timer.on = sort_ms != nullptr;
    const int rc = tuple_sv_iterate<T>(edges, m, n, labels, b, st, max_iters, iters_out, timer, s);
    if (sort_ms) {
        cudaStreamSynchronize(s);
        *sort_ms = timer.total_ms();
        *sorts = (int)(timer.ev.size() / 2);
    }
    return rc;
}

template int tuple_sv_run<int32_t>(const void *, long long, vid_t, void *, TupleSvBufs, DevState *, int, int *,
                                   float *, int *, cudaStream_t);
template int tuple_sv_run<int64_t>(const void *, long long, vid_t, void *, TupleSvBufs, DevState *, int, int *,
                                   float *, int *, cudaStream_t);

}  // namespace ccg

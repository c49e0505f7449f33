// Degree distribution and route prediction (Section 3.2, Algorithm 2 lines 1-2).
//
//  k_degree        one streaming pass over the pairs: deg[v] = number of pair
//                  endpoints equal to v (both directions of every pair, so a
//                  self-loop adds 2); ids outside [0, n) raise kErrInvalidEdge.
//  k_hist          histogram of deg with shared-memory privatised bins for
//                  small degrees, dense global bins below kHistDense and an
//                  overflow list above; argmax degree (ties to the smallest id).
//  k_distinct_*    the distinct degrees >= 1 in increasing order with their
//                  counts, exclusive count prefix and natural logs.
//  k_ks_candidates one block per candidate xmin: discrete power-law exponent
//                  (Clauset et al. eq. 3.7), model CDF from the Hurwitz zeta,
//                  and the exact sup distance to the empirical CDF.
//  k_ks_select     min D over the candidates, route = D < tau.
#include "cc_common.cuh"
#include "cc_kernels.h"
#include "ks_math.cuh"

#include <math.h>

namespace ccg {

// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlock) k_degree(const T *__restrict__ edges, long long m, vid_t n,
                                                   uint32_t *__restrict__ deg, DevState *st) {
    constexpr int P = PairVec<T>::kPairs;
    constexpr int U = 4;  // vectors in flight per thread
    const long long nvec = m / P;
    const int4 *ev = reinterpret_cast<const int4 *>(edges);
    bool bad = false;
    const long long stride = gstride();
    for (long long base = gtid(); base < nvec; base += stride * U) {
        int4 q[U];
#pragma unroll
        for (int k = 0; k < U; k++) {
            const long long i = base + (long long)k * stride;
            if (i < nvec) q[k] = ld_stream(ev + i);
        }
#pragma unroll
        for (int k = 0; k < U; k++) {
            const long long i = base + (long long)k * stride;
            if (i >= nvec) break;
#pragma unroll
            for (int j = 0; j < P; j++) {
                long long u, v;
                vec_pair<T>(q[k], j, u, v);
                if ((unsigned long long)u >= n || (unsigned long long)v >= n) {
                    bad = true;
                    continue;
                }
                atomicAdd(&deg[u], 1u);
                atomicAdd(&deg[v], 1u);
            }
        }
    }
    if (P == 2 && (m & 1) && gtid() == 0) {
        long long u, v;
        scalar_pair<T>(edges, m - 1, u, v);
        if ((unsigned long long)u >= n || (unsigned long long)v >= n) bad = true;
        else {
            atomicAdd(&deg[u], 1u);
            atomicAdd(&deg[v], 1u);
        }
    }
    if (bad) set_err(st, kErrInvalidEdge);
}

// ---------------------------------------------------------------------------
// Hub-aware degree pass. Every pair endpoint costs one scattered L2 atomic in
// k_degree, and the L2 atomic rate, not HBM, bounds that kernel. In
// scale-free graphs a few thousand high-degree vertices (hubs) carry a large
// share of the endpoints (by the R-MAT degree law with a = 0.57, the 12K
// largest of scale 24 carry about a quarter), so the pass is split:
//   1. a prefix of kHubPrefix pairs is counted with plain global atomics;
//   2. the vertices with the largest prefix counts (at most half the table
//      slots: the count threshold is the smallest one that admits no more)
//      become hubs, placed in a global table of 4-slot buckets (a hub whose
//      bucket is full stays an ordinary vertex);
//   3. the rest of the pairs is streamed by blocks that hold the table in
//      shared memory: one 16-byte load of the endpoint's bucket decides; a
//      hub endpoint is counted with a shared-memory atomic, any other with a
//      global one; each block flushes its hub counts once at the end.
// Which vertices become hubs only changes the speed, never the counts.
constexpr int kHubBins = 4096;              // prefix-count histogram (last bin: >= 4095)
constexpr int kHubMinCount = 8;             // a hub needs at least this many prefix endpoints
constexpr int kHubSlotsMax = 24576;         // largest table (global scratch is sized for it)
constexpr uint32_t kEmptyKey = 0xffffffffu;
// scratch layout (32-bit words): bins[kHubBins], thr, nhubs, pad..., keys[kHubSlotsMax] at kHubKeysAt
constexpr int kHubThrAt = kHubBins, kHubCountAt = kHubBins + 1, kHubKeysAt = kHubBins + 32;

// bucket of vertex v among nb buckets (multiplicative hash, multiply-high range reduction)
__device__ __forceinline__ uint32_t hub_bucket(uint32_t v, uint32_t nb) {
    return (uint32_t)(((unsigned long long)(v * 2654435761u) * nb) >> 32);
}

// bins[min(c, kHubBins - 1)] += 1 for every prefix count c >= kHubMinCount
__global__ void __launch_bounds__(kBlock) k_hub_levels(const uint32_t *__restrict__ deg, vid_t n, unsigned *bins) {
    __shared__ unsigned sh[kHubBins];
    for (int i = threadIdx.x; i < kHubBins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (long long v = gtid(); v < (long long)n; v += gstride()) {
        const uint32_t d = deg[v];
        if (d >= (uint32_t)kHubMinCount) atomicAdd(&sh[d < (uint32_t)kHubBins ? d : kHubBins - 1], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHubBins; i += blockDim.x)
        if (sh[i]) atomicAdd(&bins[i], sh[i]);
}

// thr = the smallest count t >= kHubMinCount with at most hub_max vertices
// of count >= t (suffix sums of the bins; one block of 1024 threads, each
// owning kHubBins / 1024 consecutive bins)
__global__ void __launch_bounds__(1024) k_hub_threshold(unsigned *scr, unsigned hub_max) {
    constexpr int B = kHubBins / 1024;
    __shared__ unsigned warp_sum[32];
    __shared__ unsigned best;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    unsigned c[B], mine = 0;
#pragma unroll
    for (int k = 0; k < B; k++) mine += (c[k] = scr[t * B + k]);
    if (t == 0) best = kHubBins;
    // suffix sum over threads: the count of the bins of the threads above t
    unsigned incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_down_sync(0xffffffffu, incl, o);
        if (lane + o < 32) incl += y;
    }
    if (lane == 0) warp_sum[w] = incl;
    __syncthreads();
    unsigned above = incl - mine;
    for (int k = w + 1; k < 32; k++) above += warp_sum[k];
    unsigned suffix = above;  // vertices with count >= (t + 1) * B
    for (int k = B - 1; k >= 0; k--) {
        suffix += c[k];
        const int bin = t * B + k;
        if (bin >= kHubMinCount && suffix <= hub_max) atomicMin(&best, (unsigned)bin);
    }
    __syncthreads();
    if (t == 0) scr[kHubThrAt] = best;
}

// hubs: vertices with prefix count >= thr, each into a free slot of its
// bucket (nb buckets of 4 slots) if there is one
__global__ void __launch_bounds__(kBlock) k_hub_select(const uint32_t *__restrict__ deg, vid_t n, unsigned *scr,
                                                       uint32_t nb) {
    const unsigned thr = scr[kHubThrAt];
    if (thr >= (unsigned)kHubBins) return;
    uint32_t *keys = scr + kHubKeysAt;
    for (long long v = gtid(); v < (long long)n; v += gstride()) {
        const uint32_t d = deg[v];
        if ((d < (uint32_t)kHubBins ? d : kHubBins - 1) < thr) continue;
        const uint32_t b = hub_bucket((uint32_t)v, nb);
        for (int j = 0; j < 4; j++)
            if (atomicCAS(&keys[4 * b + j], kEmptyKey, (uint32_t)v) == kEmptyKey) {
                atomicAdd(&scr[kHubCountAt], 1u);
                break;
            }
    }
}

// SLOTS table slots (SLOTS / 4 buckets) in shared memory: keys then counts
template <typename T, int SLOTS, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_degree_hubs(const T *__restrict__ edges, long long m, vid_t n,
                                                               uint32_t *__restrict__ deg,
                                                               const unsigned *__restrict__ scr, DevState *st) {
    extern __shared__ uint4 hub_smem4[];
    uint4 *key4 = hub_smem4;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(hub_smem4 + SLOTS / 4);
    {
        const uint4 *gk = reinterpret_cast<const uint4 *>(scr + kHubKeysAt);
        for (int i = threadIdx.x; i < SLOTS / 4; i += THREADS) {
            key4[i] = gk[i];
            reinterpret_cast<uint4 *>(cnt)[i] = make_uint4(0, 0, 0, 0);
        }
    }
    __syncthreads();
    constexpr int P = PairVec<T>::kPairs;
    constexpr int U = MINB == 1 ? 4 : 2;  // vectors in flight per thread (register budget of MINB blocks)
    const long long nvec = m / P;
    const int4 *ev = reinterpret_cast<const int4 *>(edges);
    bool bad = false;
    const long long stride = gstride();
    auto count = [&](uint32_t x) {
        const uint32_t b = hub_bucket(x, SLOTS / 4);
        const uint4 k = key4[b];
        const int j = k.x == x ? 0 : k.y == x ? 1 : k.z == x ? 2 : k.w == x ? 3 : -1;
        if (j >= 0) atomicAdd(&cnt[4 * b + j], 1u);
        else atomicAdd(&deg[x], 1u);
    };
    for (long long base = gtid(); base < nvec; base += stride * U) {
        int4 q[U];
#pragma unroll
        for (int k = 0; k < U; k++) {
            const long long i = base + (long long)k * stride;
            if (i < nvec) q[k] = ld_stream(ev + i);
        }
#pragma unroll
        for (int k = 0; k < U; k++) {
            const long long i = base + (long long)k * stride;
            if (i >= nvec) break;
#pragma unroll
            for (int j = 0; j < P; j++) {
                long long u, v;
                vec_pair<T>(q[k], j, u, v);
                if ((unsigned long long)u >= n || (unsigned long long)v >= n) {
                    bad = true;
                    continue;
                }
                count((uint32_t)u);
                count((uint32_t)v);
            }
        }
    }
    if (P == 2 && (m & 1) && gtid() == 0) {
        long long u, v;
        scalar_pair<T>(edges, m - 1, u, v);
        if ((unsigned long long)u >= n || (unsigned long long)v >= n) bad = true;
        else {
            count((uint32_t)u);
            count((uint32_t)v);
        }
    }
    if (bad) set_err(st, kErrInvalidEdge);
    __syncthreads();
    const uint32_t *key = reinterpret_cast<const uint32_t *>(key4);
    for (int i = threadIdx.x; i < SLOTS; i += THREADS)
        if (cnt[i]) atomicAdd(&deg[key[i]], cnt[i]);
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ void hist_one(uint32_t d, vid_t v, uint32_t *sh, uint32_t *hist, uint32_t *ovf,
                                         unsigned long long ovf_cap, DevState *st, unsigned long long &best) {
    if (d < kHistSmem) atomicAdd(&sh[d], 1u);
    else if (d < kHistDense) atomicAdd(&hist[d], 1u);
    else {
        unsigned long long k = atomicAdd(&st->n_ovf, 1ull);
        if (k < ovf_cap) ovf[k] = d;
        else set_err(st, kErrOverflow);
    }
    const unsigned long long key = ((unsigned long long)d << 32) | (unsigned long long)(0xffffffffu - v);
    best = key > best ? key : best;
}

__global__ void __launch_bounds__(kBlock) k_hist(const uint32_t *__restrict__ deg, vid_t n, uint32_t *hist,
                                                 uint32_t *ovf, unsigned long long ovf_cap, DevState *st) {
    __shared__ uint32_t sh[kHistSmem];
    for (int i = threadIdx.x; i < (int)kHistSmem; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    unsigned long long best = 0;
    const long long nv4 = (long long)n / 4;
    const uint4 *d4 = reinterpret_cast<const uint4 *>(deg);
    for (long long i = gtid(); i < nv4; i += gstride()) {
        const uint4 q = d4[i];
        const vid_t v = (vid_t)(i * 4);
        hist_one(q.x, v, sh, hist, ovf, ovf_cap, st, best);
        hist_one(q.y, v + 1, sh, hist, ovf, ovf_cap, st, best);
        hist_one(q.z, v + 2, sh, hist, ovf, ovf_cap, st, best);
        hist_one(q.w, v + 3, sh, hist, ovf, ovf_cap, st, best);
    }
    for (long long v = nv4 * 4 + gtid(); v < (long long)n; v += gstride())
        hist_one(deg[v], (vid_t)v, sh, hist, ovf, ovf_cap, st, best);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long b = __shfl_xor_sync(0xffffffffu, best, o);
        best = b > best ? b : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&st->maxkey, best);
    __syncthreads();
    for (int i = threadIdx.x; i < (int)kHistSmem; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// k_hist over the degree slice of one graph of a batch (DevState::batch_base,
// batch_ng; ids local to that graph): the single-graph fit of a graph whose
// large degrees overflow the per-graph fit.
__global__ void __launch_bounds__(kBlock) k_hist_slice(const uint32_t *__restrict__ deg, uint32_t *hist, uint32_t *ovf,
                                                       unsigned long long ovf_cap, DevState *st) {
    if (st->batch_ng <= 0) return;
    __shared__ uint32_t sh[kHistSmem];
    for (int i = threadIdx.x; i < (int)kHistSmem; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint32_t *d = deg + st->batch_base;
    const long long n = st->batch_ng;
    unsigned long long best = 0;
    for (long long v = gtid(); v < n; v += gstride()) hist_one(d[v], (vid_t)v, sh, hist, ovf, ovf_cap, st, best);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long b = __shfl_xor_sync(0xffffffffu, best, o);
        best = b > best ? b : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&st->maxkey, best);
    __syncthreads();
    for (int i = threadIdx.x; i < (int)kHistSmem; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

void launch_hist_slice(const uint32_t *deg, uint32_t *hist, uint32_t *ovf, unsigned long long ovf_cap, DevState *st,
                       int grid, cudaStream_t s) {
    k_hist_slice<<<grid, kBlock, 0, s>>>(deg, hist, ovf, ovf_cap, st);
}

// ---------------------------------------------------------------------------
// Distinct degrees. The dense bins [1, min(maxdeg+1, kHistDense)) are split
// into chunks of kChunk; k_distinct_count counts nonzero bins and their mass
// per chunk, k_distinct_scan turns those into chunk offsets (one block),
// k_distinct_write writes the compacted arrays, k_distinct_overflow appends
// the (rare) degrees >= kHistDense in sorted order.
constexpr int kChunk = 4096;
constexpr int kNumChunks = (int)(kHistDense / kChunk);

__device__ __forceinline__ long long dense_limit(const DevState *st) {
    const unsigned long long maxdeg = st->maxkey >> 32;
    return maxdeg + 1 < kHistDense ? (long long)maxdeg + 1 : (long long)kHistDense;
}


__global__ void __launch_bounds__(1024) k_distinct_count(const uint32_t *hist, const DevState *st,
                                                         unsigned long long *chunk_nz, unsigned long long *chunk_mass) {
    __shared__ unsigned long long sm[33];
    const long long lim = dense_limit(st);
    const long long c0 = (long long)blockIdx.x * kChunk;
    unsigned long long nz = 0, mass = 0;
    for (long long d = c0 + threadIdx.x; d < c0 + kChunk && d < lim; d += blockDim.x) {
        if (d == 0) continue;
        const uint32_t h = hist[d];
        nz += h ? 1 : 0;
        mass += h;
    }
    unsigned long long tnz, tmass;
    block_exclusive_scan<unsigned long long>(nz, sm, tnz);
    block_exclusive_scan<unsigned long long>(mass, sm, tmass);
    if (threadIdx.x == 0) {
        chunk_nz[blockIdx.x] = tnz;
        chunk_mass[blockIdx.x] = tmass;
    }
}

__global__ void __launch_bounds__(1024) k_distinct_scan(unsigned long long *chunk_nz, unsigned long long *chunk_mass,
                                                        DevState *st, unsigned long long cap) {
    // kNumChunks = 256 <= blockDim: one element per thread.
    __shared__ unsigned long long sm[33];
    const int t = threadIdx.x;
    unsigned long long nz = t < kNumChunks ? chunk_nz[t] : 0, mass = t < kNumChunks ? chunk_mass[t] : 0;
    unsigned long long tnz, tmass;
    unsigned long long onz = block_exclusive_scan<unsigned long long>(nz, sm, tnz);
    unsigned long long omass = block_exclusive_scan<unsigned long long>(mass, sm, tmass);
    if (t < kNumChunks) {
        chunk_nz[t] = onz;
        chunk_mass[t] = omass;
    }
    if (t == 0) {
        chunk_nz[kNumChunks] = tnz;
        chunk_mass[kNumChunks] = tmass;
        st->nd = tnz < cap ? tnz : cap;
        if (tnz > cap) atomicOr(&st->err, kErrOverflow);
    }
}

__global__ void __launch_bounds__(1024) k_distinct_write(const uint32_t *hist, const DevState *st,
                                                         const unsigned long long *chunk_nz,
                                                         const unsigned long long *chunk_mass, uint32_t *xs,
                                                         unsigned long long *cnt, unsigned long long *cum, double *lnx,
                                                         unsigned long long cap) {
    __shared__ unsigned long long sm[33];
    const long long lim = dense_limit(st);
    const long long c0 = (long long)blockIdx.x * kChunk;
    if (c0 >= lim) return;  // uniform per block
    unsigned long long off = chunk_nz[blockIdx.x], moff = chunk_mass[blockIdx.x];
    // 4 rounds of 1024 bins, in increasing degree order
    for (long long r = 0; r < kChunk; r += blockDim.x) {
        const long long d = c0 + r + threadIdx.x;
        const uint32_t h = (d > 0 && d < lim) ? hist[d] : 0u;
        unsigned long long tnz, tmass;
        unsigned long long p = block_exclusive_scan<unsigned long long>(h ? 1ull : 0ull, sm, tnz);
        unsigned long long pm = block_exclusive_scan<unsigned long long>((unsigned long long)h, sm, tmass);
        if (h && off + p < cap) {
            const unsigned long long k = off + p;
            xs[k] = (uint32_t)d;
            cnt[k] = h;
            cum[k] = moff + pm;
            lnx[k] = log((double)d);
        }
        off += tnz;
        moff += tmass;
    }
}

// Appends the distinct overflow degrees (>= kHistDense) in increasing order:
// bitonic sort of the (at most kOvfMax) recorded degrees in shared memory,
// then one pass that keeps the first of each run of equal values.
constexpr int kOvfMax = 4096;

__global__ void __launch_bounds__(1024) k_distinct_overflow(const uint32_t *ovf, unsigned long long ovf_cap,
                                                            const unsigned long long *chunk_mass, DevState *st,
                                                            uint32_t *xs, unsigned long long *cnt,
                                                            unsigned long long *cum, double *lnx,
                                                            unsigned long long cap) {
    __shared__ uint32_t sv[kOvfMax];
    __shared__ unsigned long long sm[33];
    const unsigned long long rec = st->n_ovf < ovf_cap ? st->n_ovf : ovf_cap;
    const int k = (int)(rec < (unsigned long long)kOvfMax ? rec : (unsigned long long)kOvfMax);
    const unsigned long long base = st->nd, mass0 = chunk_mass[kNumChunks];
    int P = 1;
    while (P < k) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) sv[i] = i < k ? ovf[i] : 0xffffffffu;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const uint32_t a = sv[i], b = sv[j];
                    if ((a > b) == up) {
                        sv[i] = b;
                        sv[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    // runs of equal values: a run starts at i when sv[i] != sv[i-1]
    unsigned long long out = 0;
    for (int r = 0; r < P; r += blockDim.x) {
        const int i = r + threadIdx.x;
        const bool head = i < k && (i == 0 || sv[i] != sv[i - 1]);
        unsigned long long tot;
        const unsigned long long rank = block_exclusive_scan<unsigned long long>(head ? 1ull : 0ull, sm, tot);
        if (head && base + out + rank < cap) {
            int e = i + 1;
            while (e < k && sv[e] == sv[i]) e++;
            const unsigned long long o = base + out + rank;
            xs[o] = sv[i];
            cnt[o] = (unsigned long long)(e - i);
            cum[o] = mass0 + (unsigned long long)i;
            lnx[o] = log((double)sv[i]);
        }
        out += tot;
    }
    if (threadIdx.x == 0) {
        const unsigned long long nd = base + out < cap ? base + out : cap;
        if (base + out > cap) atomicOr(&st->err, kErrOverflow);
        st->nd = nd;
        cum[nd] = mass0 + (unsigned long long)k;  // total mass of degrees >= 1
        if (rec > (unsigned long long)kOvfMax) atomicOr(&st->err, kErrOverflow);
    }
}


// Candidate setup, one warp per candidate xmin: the tail rules, the
// exponent alpha (Clauset et al. eq. 3.7) and the normaliser Z = scaled
// zeta(alpha, xmin). Non-candidates get D = 2 (never selected).
__global__ void __launch_bounds__(256) k_ks_prep(const uint32_t *xs, const unsigned long long *cnt,
                                                 const unsigned long long *cum, const double *lnx, const DevState *st,
                                                 long long min_tail, long long min_distinct, double min_span,
                                                 double *Dc, double *Ac, double *Zc) {
    const long long nd = (long long)st->nd;
    if (nd == 0) return;
    const int lane = threadIdx.x & 31;
    const long long warp = gtid() >> 5, nwarps = gstride() >> 5;
    const double xmax = (double)xs[nd - 1];
    const unsigned long long total = cum[nd];
    for (long long i = warp; i < nd; i += nwarps) {
        const double xmin = (double)xs[i];
        const unsigned long long Nt = total - cum[i];
        if ((long long)Nt < min_tail || nd - i < min_distinct || xmax < min_span * xmin) {
            if (lane == 0) Dc[i] = 2.0;
            continue;
        }
        const double lshift = log(xmin - 0.5);
        double S = 0.0;
        for (long long j = i + lane; j < nd; j += 32) S += (double)cnt[j] * (lnx[j] - lshift);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
        if (lane == 0) {
            const double alpha = 1.0 + (double)Nt / S;
            Ac[i] = alpha;
            Zc[i] = zeta_scaled(alpha, xmin, lnx[i]);
            Dc[i] = 0.0;
        }
    }
}


template <bool REFINE>
__global__ void __launch_bounds__(256) k_ks_terms(const uint32_t *xs, const unsigned long long *cum,
                                                  const double *lnx, const DevState *st, double *Dc, const double *Ac,
                                                  const double *Zc, float *Df) {
    __shared__ float sf[8];
    __shared__ double sd[8];
    const long long nd = (long long)st->nd;
    for (long long i = blockIdx.y; i < nd; i += gridDim.y)
    for (long long j0 = i + (long long)blockIdx.x * kKsTerms; j0 < nd; j0 += (long long)gridDim.x * kKsTerms) {
        if (Dc[i] > 1.0) break;  // not a candidate (block-uniform)
        const double alpha = Ac[i], Z = Zc[i], lnc = lnx[i];
        const float alpha_f = (float)alpha, Z_f = (float)Z, lnc_f = (float)lnc;
        const unsigned long long ci = cum[i];
        const double N = (double)(cum[nd] - ci);
        const float invN_f = 1.0f / (float)(cum[nd] - ci);
        const float cut = REFINE ? Df[i] - kScreenSlack : 0.0f;
        float fmax_ = 0.0f;
        double dmax = 0.0;
        for (long long j = j0 + threadIdx.x; j < nd && j < j0 + kKsTerms; j += blockDim.x) {
            const double x = (double)xs[j];
            // the screen in fp32 throughout (CDF fractions included: an fp64
            // divide per term kept the fp64 pipe busy); fp64 only for the
            // terms the refinement keeps
            const float d32 = ks_term_f(alpha_f, Z_f, lnc_f, (float)x, (float)lnx[j], (float)(cum[j] - ci) * invN_f,
                                        (float)(cum[j + 1] - ci) * invN_f, j == i);
            fmax_ = fmaxf(fmax_, d32);
            if (REFINE && d32 >= cut) {
                const double before = (double)(cum[j] - ci) / N;
                const double at = (double)(cum[j + 1] - ci) / N;
                double zb, za;  // model mass at >= x and at >= x+1 (scaled by xmin^alpha)
                zeta_pair(alpha, x, lnx[j], lnc, zb, za);
                double d = fabs(at - (1.0 - za / Z));
                if (j > i) d = fmax(d, fabs(before - (1.0 - zb / Z)));
                dmax = fmax(dmax, d);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            fmax_ = fmaxf(fmax_, __shfl_xor_sync(0xffffffffu, fmax_, o));
            dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
            sf[threadIdx.x >> 5] = fmax_;
            sd[threadIdx.x >> 5] = dmax;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float bf = 0.0f;
            double bd = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
                bf = fmaxf(bf, sf[w]);
                bd = fmax(bd, sd[w]);
            }
            if (REFINE) atomicMax(reinterpret_cast<unsigned long long *>(&Dc[i]), (unsigned long long)__double_as_longlong(bd));
            else atomicMax(reinterpret_cast<unsigned int *>(&Df[i]), __float_as_uint(bf));
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_ks_select(const uint32_t *xs, const unsigned long long *cum,
                                                    const double *Dc, const double *Ac, DevState *st, double tau) {
    __shared__ double sD[1024];
    __shared__ long long sI[1024];
    __shared__ unsigned long long sC[1024];
    const long long nd = (long long)st->nd;
    double best = 2.0;
    long long bi = -1;
    unsigned long long nc = 0;
    for (long long i = threadIdx.x; i < nd; i += blockDim.x) {
        const double d = Dc[i];
        if (d <= 1.0) {
            nc++;
            if (d < best) {  // i increases per thread, so ties keep the smaller i
                best = d;
                bi = i;
            }
        }
    }
    sD[threadIdx.x] = best;
    sI[threadIdx.x] = bi;
    sC[threadIdx.x] = nc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double d2 = sD[threadIdx.x + o];
            const long long i2 = sI[threadIdx.x + o];
            if (i2 >= 0 && (d2 < sD[threadIdx.x] || (d2 == sD[threadIdx.x] && (sI[threadIdx.x] < 0 || i2 < sI[threadIdx.x])))) {
                sD[threadIdx.x] = d2;
                sI[threadIdx.x] = i2;
            }
            sC[threadIdx.x] += sC[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long i = sI[0];
        if (i < 0) {
            st->ks_out[0] = 1.0;
            st->ks_out[1] = 0.0;
            st->ks_out[2] = 0.0;
            st->ks_out[3] = 0.0;
        } else {
            st->ks_out[0] = sD[0];
            st->ks_out[1] = Ac[i];
            st->ks_out[2] = (double)xs[i];
            st->ks_out[3] = (double)(cum[nd] - cum[i]);
        }
        st->ks_out[4] = (double)sC[0];
        st->ncand = sC[0];
        st->route = st->ks_out[0] < tau ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// Host launchers

template <typename T>
void launch_degree(const void *edges, long long m, vid_t n, uint32_t *deg, DevState *st, int grid, cudaStream_t s) {
    if (m <= 0) return;
    k_degree<T><<<fit_grid((const void *)k_degree<T>, grid, kBlock), kBlock, 0, s>>>((const T *)edges, m, n, deg, st);
}
template void launch_degree<int32_t>(const void *, long long, vid_t, uint32_t *, DevState *, int, cudaStream_t);
template void launch_degree<int64_t>(const void *, long long, vid_t, uint32_t *, DevState *, int, cudaStream_t);

// prefix pairs counted plainly before the hubs are chosen
constexpr long long kHubPrefix = 1LL << 22;

bool degree_uses_hubs(long long m) { return m >= 4 * kHubPrefix; }

size_t degree_hubs_scratch_bytes() { return (size_t)(kHubKeysAt + kHubSlotsMax) * 4; }

// The table the shipped pass uses: 24,576 slots in 6,144 buckets (192 KB of
// keys and counts), one 1024-thread block per SM. On R-MAT scale 24 it
// holds about 11.8K hubs and the pass runs 24% faster than k_degree; the
// smaller tables that fit two blocks per SM were slower.
constexpr int kHubSlots = 24576, kHubThreads = 1024, kHubMinBlocks = 1;

// Steps 1-2 above (the hub table from the first kHubPrefix pairs) with a
// table of SLOTS slots (at most SLOTS / 2 hubs). deg must be zeroed;
// scratch: degree_hubs_scratch_bytes(), 16-byte aligned.
template <typename T, int SLOTS>
void launch_hub_prefix_cfg(const void *edges, vid_t n, uint32_t *deg, unsigned *scratch, DevState *st, int grid,
                           cudaStream_t s) {
    static_assert(SLOTS % 16 == 0 && SLOTS <= kHubSlotsMax, "table size");
    cudaMemsetAsync(scratch, 0, (size_t)kHubKeysAt * 4, s);
    cudaMemsetAsync(scratch + kHubKeysAt, 0xff, (size_t)SLOTS * 4, s);
    // the prefix ends on a 16-byte boundary of the pair array: kHubPrefix pairs of 8 or 16 bytes do
    k_degree<T><<<grid, kBlock, 0, s>>>((const T *)edges, kHubPrefix, n, deg, st);
    k_hub_levels<<<grid, kBlock, 0, s>>>(deg, n, scratch);
    k_hub_threshold<<<1, 1024, 0, s>>>(scratch, (unsigned)(SLOTS / 2));
    k_hub_select<<<grid, kBlock, 0, s>>>(deg, n, scratch, (uint32_t)(SLOTS / 4));
}

// Step 3 over m pairs at `edges` (blocks of THREADS threads, MINB per SM).
template <typename T, int SLOTS, int THREADS, int MINB>
void launch_hub_count_cfg(const void *edges, long long m, vid_t n, uint32_t *deg, const unsigned *scratch,
                          DevState *st, int num_sms, cudaStream_t s) {
    if (m <= 0) return;
    constexpr size_t smem = (size_t)SLOTS * 8;  // the attribute is set once, by degree_hubs_setup
    k_degree_hubs<T, SLOTS, THREADS, MINB><<<num_sms * MINB, THREADS, smem, s>>>((const T *)edges, m, n, deg, scratch,
                                                                                 st);
}

template <typename T, int SLOTS, int THREADS, int MINB>
void launch_degree_hubs_cfg(const void *edges, long long m, vid_t n, uint32_t *deg, unsigned *scratch,
                            DevState *st, int grid, int num_sms, cudaStream_t s) {
    launch_hub_prefix_cfg<T, SLOTS>(edges, n, deg, scratch, st, grid, s);
    launch_hub_count_cfg<T, SLOTS, THREADS, MINB>((const T *)edges + 2 * kHubPrefix, m - kHubPrefix, n, deg, scratch,
                                                  st, num_sms, s);
}

long long degree_hub_prefix() { return kHubPrefix; }

cudaError_t degree_hubs_setup() {
    const int smem = kHubSlots * 8;
    cudaError_t e = cudaFuncSetAttribute(k_degree_hubs<int32_t, kHubSlots, kHubThreads, kHubMinBlocks>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_degree_hubs<int64_t, kHubSlots, kHubThreads, kHubMinBlocks>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

template <typename T>
void launch_degree_hubs(const void *edges, long long m, vid_t n, uint32_t *deg, unsigned *scratch, DevState *st,
                        int grid, int num_sms, cudaStream_t s) {
    launch_degree_hubs_cfg<T, kHubSlots, kHubThreads, kHubMinBlocks>(edges, m, n, deg, scratch, st, grid, num_sms,
                                                                     s);
}

template <typename T>
void launch_degree_hub_prefix(const void *edges, vid_t n, uint32_t *deg, unsigned *scratch, DevState *st, int grid,
                              cudaStream_t s) {
    launch_hub_prefix_cfg<T, kHubSlots>(edges, n, deg, scratch, st, grid, s);
}

template <typename T>
void launch_degree_hub_count(const void *edges, long long m, vid_t n, uint32_t *deg, const unsigned *scratch,
                             DevState *st, int num_sms, cudaStream_t s) {
    launch_hub_count_cfg<T, kHubSlots, kHubThreads, kHubMinBlocks>(edges, m, n, deg, scratch, st, num_sms, s);
}
template void launch_degree_hub_prefix<int32_t>(const void *, vid_t, uint32_t *, unsigned *, DevState *, int,
                                                cudaStream_t);
template void launch_degree_hub_prefix<int64_t>(const void *, vid_t, uint32_t *, unsigned *, DevState *, int,
                                                cudaStream_t);
template void launch_degree_hub_count<int32_t>(const void *, long long, vid_t, uint32_t *, const unsigned *,
                                               DevState *, int, cudaStream_t);
template void launch_degree_hub_count<int64_t>(const void *, long long, vid_t, uint32_t *, const unsigned *,
                                               DevState *, int, cudaStream_t);
template void launch_degree_hubs<int32_t>(const void *, long long, vid_t, uint32_t *, unsigned *, DevState *, int,
                                          int, cudaStream_t);
template void launch_degree_hubs<int64_t>(const void *, long long, vid_t, uint32_t *, unsigned *, DevState *, int,
                                          int, cudaStream_t);

void launch_hist(const uint32_t *deg, vid_t n, uint32_t *hist, uint32_t *ovf, unsigned long long ovf_cap,
                 DevState *st, int grid, cudaStream_t s) {
    if (n == 0) return;
    k_hist<<<fit_grid((const void *)k_hist, grid, kBlock), kBlock, 0, s>>>(deg, n, hist, ovf, ovf_cap, st);
}

void launch_ks(const uint32_t *hist, const uint32_t *ovf, unsigned long long ovf_cap, KsScratch ks, DevState *st,
               long long min_tail, long long min_distinct, double min_span, double tau, long long nd_bound, int grid,
               cudaStream_t s) {
    k_distinct_count<<<kNumChunks, 1024, 0, s>>>(hist, st, ks.chunk_nz, ks.chunk_mass);
    k_distinct_scan<<<1, 1024, 0, s>>>(ks.chunk_nz, ks.chunk_mass, st, ks.cap);
    k_distinct_write<<<kNumChunks, 1024, 0, s>>>(hist, st, ks.chunk_nz, ks.chunk_mass, ks.xs, ks.cnt, ks.cum, ks.lnx,
                                                 ks.cap);
    k_distinct_overflow<<<1, 1024, 0, s>>>(ovf, ovf_cap, ks.chunk_mass, st, ks.xs, ks.cnt, ks.cum, ks.lnx, ks.cap);
    k_ks_prep<<<grid, 256, 0, s>>>(ks.xs, ks.cnt, ks.cum, ks.lnx, st, min_tail, min_distinct, min_span, ks.Dc,
                                   ks.Ac, ks.Zc);
    // blocks stride over candidates (y) and over chunks of kKsTerms terms (x);
    // nd_bound (an upper bound of the distinct degrees) keeps small graphs from
    // launching thousands of idle blocks
    const long long nb = nd_bound < 1 ? 1 : nd_bound;
    const dim3 tg((unsigned)(nb < 4 * kKsTerms ? (nb + kKsTerms - 1) / kKsTerms : 4), (unsigned)(nb < 2048 ? nb : 2048));
    cudaMemsetAsync(ks.Df, 0, sizeof(float) * (ks.cap + 1), s);
    k_ks_terms<false><<<tg, 256, 0, s>>>(ks.xs, ks.cum, ks.lnx, st, ks.Dc, ks.Ac, ks.Zc, ks.Df);
    k_ks_terms<true><<<tg, 256, 0, s>>>(ks.xs, ks.cum, ks.lnx, st, ks.Dc, ks.Ac, ks.Zc, ks.Df);
    k_ks_select<<<1, 1024, 0, s>>>(ks.xs, ks.cum, ks.Dc, ks.Ac, st, tau);
}

int ks_num_chunks() { return kNumChunks; }

// hist (uint32 dense bins + overflow list) -> uint64 histogram of length len
__global__ void __launch_bounds__(kBlock) k_hist_widen(const uint32_t *hist, const uint32_t *ovf,
                                                       unsigned long long ovf_cap, const DevState *st, uint64_t *out,
                                                       long long len) {
    for (long long d = gtid(); d < len; d += gstride()) out[d] = d < (long long)kHistDense ? hist[d] : 0ull;
}
__global__ void __launch_bounds__(kBlock) k_hist_widen_ovf(const uint32_t *ovf, unsigned long long ovf_cap,
                                                           const DevState *st, uint64_t *out, long long len) {
    const unsigned long long k = st->n_ovf < ovf_cap ? st->n_ovf : ovf_cap;
    for (long long i = gtid(); i < (long long)k; i += gstride())
        if ((long long)ovf[i] < len) atomicAdd((unsigned long long *)&out[ovf[i]], 1ull);
}
void launch_hist_widen(const uint32_t *hist, const uint32_t *ovf, unsigned long long ovf_cap, const DevState *st,
                       uint64_t *out, long long len, int grid, cudaStream_t s) {
    k_hist_widen<<<grid, kBlock, 0, s>>>(hist, ovf, ovf_cap, st, out, len);
    k_hist_widen_ovf<<<grid, kBlock, 0, s>>>(ovf, ovf_cap, st, out, len);
}

// uint64 histogram (len <= kHistDense, counts < 2^32) -> dense uint32 bins and
// the max degree (maxkey) the distinct-degree pass reads.
__global__ void __launch_bounds__(kBlock) k_hist_narrow(const uint64_t *in, long long len, uint32_t *hist,
                                                        DevState *st) {
    unsigned long long best = 0;
    for (long long d = gtid(); d < len; d += gstride()) {
        const uint64_t h = in[d];
        if (h > 0xffffffffull) set_err(st, kErrOverflow);
        hist[d] = (uint32_t)h;
        if (h) best = ((unsigned long long)d << 32) | 0xffffffffull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, best, o);
        best = b > best ? b : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&st->maxkey, best);
}
void launch_hist_narrow(const uint64_t *in, long long len, uint32_t *hist, DevState *st, int grid, cudaStream_t s) {
    k_hist_narrow<<<grid, kBlock, 0, s>>>(in, len, hist, st);
}

}  // namespace ccg

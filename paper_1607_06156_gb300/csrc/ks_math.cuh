// K-S fit arithmetic shared by the single-graph kernels (k_degree.cu) and
// the per-graph batched fit (k_batch_route.cu): the scaled Hurwitz zeta in
// fp64 and fp32, the fp32 screen term, and block-wide scans and reductions.
#pragma once

#include "cc_common.cuh"

#include <math.h>

namespace ccg {

template <typename V>
__device__ V block_exclusive_scan(V x, V *smem /* >= 32 */, V &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    V incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        V y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) smem[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        V w = lane < nw ? smem[lane] : (V)0;
        V wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            V y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) smem[lane] = wi - w;
        if (lane == nw - 1) smem[32] = wi;
    }
    __syncthreads();
    V r = smem[warp] + incl - x;
    total = smem[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Scaled Hurwitz zeta: c^s * zeta(s, q) = sum_{k>=0} ((q+k)/c)^-s, s > 1.
// Explicit terms until a = q + k reaches max(16, 2s); the remainder by the
// Euler-Maclaurin formula with six Bernoulli terms. With a >= 2s the ratio
// of consecutive correction terms is below (s / (2 pi a))^2 <= 1/(16 pi^2),
// so six terms leave a relative error near 1e-15.
// Euler-Maclaurin remainder sum_{k>=0} ((a+k)/c)^-s for a >= max(16, 2s),
// given A = (a/c)^-s.
__device__ __forceinline__ double zeta_tail(double s, double a, double A) {
    double acc = A * a / (s - 1.0) + 0.5 * A;
    const double ia2 = 1.0 / (a * a);
    // term_k = B_2k/(2k)! * s(s+1)...(s+2k-2) * A * a^-(2k-1)
    const double coef[6] = {1.0 / 12.0, -1.0 / 720.0, 1.0 / 30240.0, -1.0 / 1209600.0, 1.0 / 47900160.0,
                            -691.0 / 1307674368000.0};
    double t = A * s / a;
    acc += coef[0] * t;
#pragma unroll
    for (int k = 1; k < 6; k++) {
        t *= (s + 2 * k - 1) * (s + 2 * k) * ia2;
        acc += coef[k] * t;
    }
    return acc;
}

static __device__ double zeta_scaled(double s, double q, double lnc) {
    double acc = 0.0, a = q;
    const double thr = fmax(16.0, 2.0 * s);
    while (a < thr) {
        const double term = exp(-s * (log(a) - lnc));
        acc += term;
        a += 1.0;
        // the rest is below term * (1 + a/(s-1)) (integral bound); stop once it cannot matter
        if (term * (1.0 + a / (s - 1.0)) < 1e-18 * acc) return acc;
    }
    return acc + zeta_tail(s, a, exp(-s * (log(a) - lnc)));
}

// zeta_scaled at x and at x+1 for an observed degree x with ln x known.
// For x >= max(16, 2s) one evaluation serves both: the x+1 value is the x
// value minus its first term (x/c)^-s, and the tail is at least twice that
// term, so the subtraction loses under two bits.
__device__ __forceinline__ void zeta_pair(double s, double x, double lnx, double lnc, double &zx, double &zx1) {
    if (x >= fmax(16.0, 2.0 * s)) {
        const double A = exp(-s * (lnx - lnc));
        zx = zeta_tail(s, x, A);
        zx1 = zx - A;
    } else {
        zx = zeta_scaled(s, x, lnc);
        zx1 = zeta_scaled(s, x + 1.0, lnc);
    }
}

// The terms of the scaled zeta below its Euler-Maclaurin threshold, summed
// once per exponent by one warp: T is the first integer >= max(16, 2s);
// for integers q0 <= x < T, tab[x - q0] = sum_{t=x}^{T-1} (t/c)^-s (suffix
// sums), and `tail` = the remainder from T on. Then for q0 <= x < T
// zeta_scaled(s, x, lnc) = tab[x - q0] + tail (the same sum as the direct
// loop, summed in another order). Returns T, or -1 (warp-uniform) when the
// table would need more than cap entries. All lanes of the warp call it.
__device__ __forceinline__ long long zeta_table_warp(double s, long long q0, double lnc, double *tab, int cap,
                                                     double &tail) {
    const int lane = threadIdx.x & 31;
    const long long T = (long long)ceil(fmax(16.0, 2.0 * s));
    const long long span = T - q0;
    if (span > cap) return -1;
    tail = zeta_tail(s, (double)T, exp(-s * (log((double)T) - lnc)));
    double carry = 0.0;  // the sum of the entries above the current chunk
    for (long long c0 = span > 0 ? ((span - 1) / 32) * 32 : -1; c0 >= 0; c0 -= 32) {
        const long long k = c0 + lane;
        double v = k < span ? exp(-s * (log((double)(q0 + k)) - lnc)) : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {  // inclusive suffix sum over the lanes
            const double y = __shfl_down_sync(0xffffffffu, v, o);
            if (lane + o < 32) v += y;
        }
        if (k < span) tab[k] = v + carry;
        carry += __shfl_sync(0xffffffffu, v, 0);
    }
    __syncwarp();
    return T;
}

template <typename V>
__device__ V block_reduce_sum(V x, V *smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) smem[warp] = x;
    __syncthreads();
    V r = 0;
    for (int w = 0; w < nw; w++) r += smem[w];
    __syncthreads();
    return r;
}

// maximum over the block of non-negative values (all threads get it)
static __device__ double block_reduce_max(double x, double *smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) smem[warp] = x;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < nw; w++) r = fmax(r, smem[w]);
    __syncthreads();
    return r;
}

// minimum over the block (any sign; all threads get it)
static __device__ double block_reduce_min(double x, double *smem) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmin(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) smem[warp] = x;
    __syncthreads();
    double r = smem[0];
    for (int w = 1; w < nw; w++) r = fmin(r, smem[w]);
    __syncthreads();
    return r;
}

// The sup distance is taken in two passes over (candidate, chunk of
// kKsTerms terms) blocks. The screen evaluates every term in fp32 and keeps
// each candidate's fp32 maximum; the refine pass re-evaluates in fp64 only
// the terms whose fp32 value is within kScreenSlack of that maximum and
// folds them into D[i] (atomicMax on the bit pattern: non-negative doubles
// and floats order like their bits). The fp32 terms are within ~3e-6 of the
// fp64 ones (a few ulp on S, on the zeta ratio and on 1 - ratio), far inside
// the 1e-4 slack, so the term that attains the fp64 maximum always passes
// the screen and D[i] is the fp64 sup.
constexpr int kKsTerms = 1024;
constexpr float kScreenSlack = 1e-4f;

__device__ __forceinline__ float zeta_tail_f(float s, float a, float A) {
    float acc = A * a / (s - 1.0f) + 0.5f * A;
    const float ia2 = 1.0f / (a * a);
    float t = A * s / a;
    acc += t * (1.0f / 12.0f);
    t *= (s + 1.0f) * (s + 2.0f) * ia2;
    acc -= t * (1.0f / 720.0f);
    t *= (s + 3.0f) * (s + 4.0f) * ia2;
    acc += t * (1.0f / 30240.0f);
    return acc;
}

static __device__ float zeta_scaled_f(float s, float q, float lnc) {
    float acc = 0.0f, a = q;
    const float thr = fmaxf(16.0f, 2.0f * s);
    while (a < thr) {
        const float term = __expf(-s * (__logf(a) - lnc));
        acc += term;
        a += 1.0f;
        if (term * (1.0f + a / (s - 1.0f)) < 1e-9f * acc) return acc;
    }
    return acc + zeta_tail_f(s, a, __expf(-s * (__logf(a) - lnc)));
}

// fp32 distance of term j of candidate i
__device__ __forceinline__ float ks_term_f(float alpha, float Z, float lnc, float x, float lnxj, float before,
                                           float at, bool first) {
    float zb, za;
    if (x >= fmaxf(16.0f, 2.0f * alpha)) {
        const float A = __expf(-alpha * (lnxj - lnc));
        zb = zeta_tail_f(alpha, x, A);
        za = zb - A;
    } else {
        zb = zeta_scaled_f(alpha, x, lnc);
        za = zeta_scaled_f(alpha, x + 1.0f, lnc);
    }
    float d = fabsf(at - (1.0f - za / Z));
    if (!first) d = fmaxf(d, fabsf(before - (1.0f - zb / Z)));
    return d;
}

}  // namespace ccg

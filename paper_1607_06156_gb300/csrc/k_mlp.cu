// Learned route predictor: features, training kernels and bf16 inference.
//
// The predictor replaces the K-S threshold of Section 3.2 only in choosing
// BFS-then-SV vs SV only and the BFS cutoff; labels never depend on it.
//
// Network: 69 -> 128 (ReLU) -> 128 (ReLU) -> 3; parameters in one fp32
// buffer [W1 (128x69) | b1 | W2 (128x128) | b2 | W3 (3x128) | b3].
// Loss: mean over the batch of cross-entropy on the two route logits plus
// lambda * w * (o[2] - t)^2 on the log-cutoff output.
//
// Features (all from samples, so the learned route can skip the exact
// degree pass when it predicts SV):
//   [0, 64)  log2-degree histogram of the vertices with id % 16 == 0
//            (bucket 0: degree 0, bucket b: degrees in [2^(b-1), 2^b)),
//            as fractions of the sampled vertices
//   64, 65   ln(n) / 20, ln(m + 1) / 20
//   66..68   ln(1 + new vertices) / 20 at BFS levels 1, 2, 3 from the
//            highest-degree sampled vertex, over the pairs of every 16th
//            block of 256 pairs
#include <cuda_bf16.h>

#include "cc_common.cuh"
#include "cc_kernels.h"

namespace ccg {

constexpr int kIn = 69, kHid = 128, kOut = 3;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
              kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid, kNumParams = kOffB3 + kOut;

int mlp_num_params() { return kNumParams; }

// ---------------------------------------------------------------------------
// C[M,N] = op(A) op(B) (+ bias[N]) (relu) (* (mask > 0)); op(A) is A [M,K] or
// the transpose of A stored [K,M]; op(B) is B [K,N] or the transpose of B
// stored [N,K]. 16x16 shared-memory tiles.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(const float *A, const float *B, float *C, int M, int N, int K,
                                              const float *bias, int relu, const float *mask) {
    __shared__ float As[16][17], Bs[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    float acc = 0.0f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int ka = k0 + tx, kb = k0 + ty;
        // As[ty][tx] = opA[row][ka], Bs[ty][tx] = opB[kb][col]
        float a = 0.0f, b = 0.0f;
        if (row < M && ka < K) a = TA ? A[(long long)ka * M + row] : A[(long long)row * K + ka];
        if (kb < K && col < N) b = TB ? B[(long long)col * K + kb] : B[(long long)kb * N + col];
        As[ty][tx] = a;
        Bs[ty][tx] = b;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) acc += As[ty][k] * Bs[k][tx];
        __syncthreads();
    }
    if (row < M && col < N) {
        if (bias) acc += bias[col];
        if (relu) acc = fmaxf(acc, 0.0f);
        if (mask && !(mask[(long long)row * N + col] > 0.0f)) acc = 0.0f;
        C[(long long)row * N + col] = acc;
    }
}

template <bool TA, bool TB>
static void gemm(const float *A, const float *B, float *C, int M, int N, int K, const float *bias, int relu,
                 const float *mask, cudaStream_t s) {
    const dim3 g((N + 15) / 16, (M + 15) / 16);
    k_gemm<TA, TB><<<g, 256, 0, s>>>(A, B, C, M, N, K, bias, relu, mask);
}

// dO of the batch-mean loss; adds the batch loss into *loss
__global__ void k_loss_grad(const float *O, const int *y, const float *t, const float *w, int B, float lam,
                            float *dO, float *loss) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (b < B) {
        const float o0 = O[b * 3], o1 = O[b * 3 + 1], o2 = O[b * 3 + 2];
        const float mx = fmaxf(o0, o1);
        const float e0 = __expf(o0 - mx), e1 = __expf(o1 - mx), se = e0 + e1;
        const float p0 = e0 / se, p1 = e1 / se;
        const int yb = y[b];
        const float diff = o2 - t[b];
        dO[b * 3] = (p0 - (yb == 0 ? 1.0f : 0.0f)) / B;
        dO[b * 3 + 1] = (p1 - (yb == 1 ? 1.0f : 0.0f)) / B;
        dO[b * 3 + 2] = 2.0f * lam * w[b] * diff / B;
        l = (mx + __logf(se) - (yb == 0 ? o0 : o1) + lam * w[b] * diff * diff) / B;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// out[j] = sum_b X[b, j]
__global__ void k_colsum(const float *X, int B, int N, float *out) {
    const int j = blockIdx.x;
    float acc = 0.0f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) acc += X[(long long)b * N + j];
    __shared__ float s[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float r = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) r += s[w];
        out[j] = r;
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int count, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += blockDim.x * gridDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi, vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// act = [H1 (B x 128) | H2 (B x 128) | O (B x 3)]
void mlp_forward(const float *P, const float *X, int B, float *act, cudaStream_t s) {
    float *H1 = act, *H2 = act + (long long)B * kHid, *O = act + 2LL * B * kHid;
    gemm<false, true>(X, P + kOffW1, H1, B, kHid, kIn, P + kOffB1, 1, nullptr, s);
    gemm<false, true>(H1, P + kOffW2, H2, B, kHid, kHid, P + kOffB2, 1, nullptr, s);
    gemm<false, true>(H2, P + kOffW3, O, B, kOut, kHid, P + kOffB3, 0, nullptr, s);
}

// scratch = [dO (B x 3) | dZ2 (B x 128) | dZ1 (B x 128)]
void mlp_backward(const float *P, const float *X, const int *y, const float *t, const float *w, int B, float lam,
                  const float *act, float *G, float *scratch, float *loss, cudaStream_t s) {
    const float *H1 = act, *H2 = act + (long long)B * kHid, *O = act + 2LL * B * kHid;
    float *dO = scratch, *dZ2 = scratch + 3LL * B, *dZ1 = dZ2 + (long long)B * kHid;
    k_loss_grad<<<(B + 255) / 256, 256, 0, s>>>(O, y, t, w, B, lam, dO, loss);
    gemm<true, false>(dO, H2, G + kOffW3, kOut, kHid, B, nullptr, 0, nullptr, s);  // dW3 = dO^T H2
    k_colsum<<<kOut, 256, 0, s>>>(dO, B, kOut, G + kOffB3);
    gemm<false, false>(dO, P + kOffW3, dZ2, B, kHid, kOut, nullptr, 0, H2, s);      // dZ2 = (dO W3) . [H2 > 0]
    gemm<true, false>(dZ2, H1, G + kOffW2, kHid, kHid, B, nullptr, 0, nullptr, s);  // dW2 = dZ2^T H1
    k_colsum<<<kHid, 256, 0, s>>>(dZ2, B, kHid, G + kOffB2);
    gemm<false, false>(dZ2, P + kOffW2, dZ1, B, kHid, kHid, nullptr, 0, H1, s);     // dZ1 = (dZ2 W2) . [H1 > 0]
    gemm<true, false>(dZ1, X, G + kOffW1, kHid, kIn, B, nullptr, 0, nullptr, s);    // dW1 = dZ1^T X
    k_colsum<<<kHid, 256, 0, s>>>(dZ1, B, kHid, G + kOffB1);
}

void mlp_adam(float *P, const float *G, float *M, float *V, int count, float lr, float b1, float b2, float eps, int t,
              cudaStream_t s) {
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    k_adam<<<(count + 255) / 256, 256, 0, s>>>(P, G, M, V, count, lr, b1, b2, eps, c1, c2);
}

// ---------------------------------------------------------------------------
// bf16 inference of one feature vector (weights bf16, fp32 accumulation).
// Writes route (0 SV, 1 BFS), the chosen route's probability and the
// cutoff (levels; 0 = none) into DevState::pred.
__global__ void __launch_bounds__(kHid) k_mlp_infer(const __nv_bfloat16 *Wb, const float *bias, const float *x,
                                                   DevState *st) {
    __shared__ float xs[kIn], h1[kHid], h2[kHid], o[kOut];
    const int j = threadIdx.x;
    if (j < kIn) xs[j] = x[j];
    __syncthreads();
    float a = bias[kOffB1 - kOffB1 + j];
    for (int k = 0; k < kIn; k++) a += __bfloat162float(Wb[kOffW1 + j * kIn + k]) * xs[k];
    h1[j] = fmaxf(a, 0.0f);
    __syncthreads();
    a = bias[kHid + j];
    for (int k = 0; k < kHid; k++) a += __bfloat162float(Wb[kOffW2 + j * kHid + k]) * h1[k];
    h2[j] = fmaxf(a, 0.0f);
    __syncthreads();
    if (j < kOut) {
        a = bias[2 * kHid + j];
        for (int k = 0; k < kHid; k++) a += __bfloat162float(Wb[kOffW3 + j * kHid + k]) * h2[k];
        o[j] = a;
    }
    __syncthreads();
    if (j == 0) {
        const float mx = fmaxf(o[0], o[1]);
        const float e0 = __expf(o[0] - mx), e1 = __expf(o[1] - mx);
        const int r = o[1] > o[0] ? 1 : 0;
        st->pred_route = r;
        st->pred_conf = (r ? e1 : e0) / (e0 + e1);
        const float L = expf(fminf(fmaxf(o[2], 0.0f), 10.0f));
        const int lv = (int)(L + 0.5f);
        st->pred_cutoff = lv >= 64 ? 0 : (lv < 1 ? 1 : lv);
    }
}

__global__ void k_params_to_bf16(const float *P, __nv_bfloat16 *Wb, float *bias) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNumParams; i += blockDim.x * gridDim.x)
        Wb[i] = __float2bfloat16(P[i]);
    // biases kept in fp32: [b1 | b2 | b3]
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kHid) bias[i] = P[kOffB1 + i];
    else if (i < 2 * kHid) bias[i] = P[kOffB2 + i - kHid];
    else if (i < 2 * kHid + kOut) bias[i] = P[kOffB3 + i - 2 * kHid];
}

void mlp_prepare_inference(const float *P, __nv_bfloat16 *Wb, float *bias, cudaStream_t s) {
    k_params_to_bf16<<<(kNumParams + 255) / 256, 256, 0, s>>>(P, Wb, bias);
}

void mlp_infer(const __nv_bfloat16 *Wb, const float *bias, const float *x, DevState *st, cudaStream_t s) {
    k_mlp_infer<<<1, kHid, 0, s>>>(Wb, bias, x, st);
}

// ---------------------------------------------------------------------------
// Features. sdeg[v >> 4] counts the endpoints equal to a sampled vertex v
// (v % 16 == 0).
constexpr int kSampleShift = 4;
constexpr int kProbeTile = 256;  // pairs per probe block; every 16th block is sampled

template <typename T>
__global__ void __launch_bounds__(kBlock) k_sample_degree(const T *__restrict__ edges, long long m, vid_t n,
                                                          uint32_t *sdeg, DevState *st) {
    constexpr int P = PairVec<T>::kPairs;
    const long long nvec = m / P;
    const int4 *ev = reinterpret_cast<const int4 *>(edges);
    bool bad = false;
    for (long long i = gtid(); i < nvec; i += gstride()) {
        const int4 q = ld_stream(ev + i);
#pragma unroll
        for (int j = 0; j < P; j++) {
            long long u, v;
            vec_pair<T>(q, j, u, v);
            if ((unsigned long long)u >= n || (unsigned long long)v >= n) {
                bad = true;
                continue;
            }
            if (!(u & 15)) atomicAdd(&sdeg[u >> kSampleShift], 1u);
            if (!(v & 15)) atomicAdd(&sdeg[v >> kSampleShift], 1u);
        }
    }
    if (P == 2 && (m & 1) && gtid() == 0) {
        long long u, v;
        scalar_pair<T>(edges, m - 1, u, v);
        if ((unsigned long long)u >= n || (unsigned long long)v >= n) bad = true;
        else {
            if (!(u & 15)) atomicAdd(&sdeg[u >> kSampleShift], 1u);
            if (!(v & 15)) atomicAdd(&sdeg[v >> kSampleShift], 1u);
        }
    }
    if (bad) set_err(st, kErrInvalidEdge);
}

// log2 buckets of the sampled degrees (counts into feat_counts[64]) and the
// highest-degree sampled vertex (ties to the smallest id) into maxkey
__global__ void __launch_bounds__(kBlock) k_sample_hist(const uint32_t *sdeg, long long ns, unsigned *feat_counts,
                                                        DevState *st) {
    __shared__ unsigned sh[64];
    if (threadIdx.x < 64) sh[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long best = 0;
    for (long long i = gtid(); i < ns; i += gstride()) {
        const uint32_t d = sdeg[i];
        const int b = d == 0 ? 0 : (32 - __clz(d));
        atomicAdd(&sh[b < 63 ? b : 63], 1u);
        const vid_t v = (vid_t)(i << kSampleShift);
        const unsigned long long key = ((unsigned long long)d << 32) | (0xffffffffu - v);
        best = key > best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, best, o);
        best = b > best ? b : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(&st->pred_seedkey, best);
    __syncthreads();
    if (threadIdx.x < 64 && sh[threadIdx.x]) atomicAdd(&feat_counts[threadIdx.x], sh[threadIdx.x]);
}

__global__ void k_probe_seed(uint32_t *vis, uint32_t *cur, vid_t n, DevState *st) {
    vid_t s = 0xffffffffu - (vid_t)(st->pred_seedkey & 0xffffffffull);
    if (s >= n) s = 0;
    vis[s >> 5] |= 1u << (s & 31);
    cur[s >> 5] |= 1u << (s & 31);
}

// One BFS level over the sampled pairs: ends in the current frontier claim
// unvisited other ends into the next frontier; counts them into probe[level].
template <typename T>
__global__ void __launch_bounds__(kBlock) k_probe_level(const T *__restrict__ edges, long long m, vid_t n,
                                                        uint32_t *vis, const uint32_t *cur, uint32_t *next,
                                                        DevState *st, int level) {
    unsigned long long cnt = 0;
    const long long blocks = (m + kProbeTile - 1) / kProbeTile;
    for (long long b = (long long)blockIdx.x * 16; b < blocks; b += (long long)gridDim.x * 16) {
        const long long k = b * kProbeTile + threadIdx.x;
        if (threadIdx.x >= kProbeTile || k >= m) continue;
        const long long u = (long long)edges[2 * k], v = (long long)edges[2 * k + 1];
        if ((unsigned long long)u >= n || (unsigned long long)v >= n) continue;
        const bool cu = (cur[u >> 5] >> (u & 31)) & 1u, cv = (cur[v >> 5] >> (v & 31)) & 1u;
        if (cu && !((vis[v >> 5] >> (v & 31)) & 1u)) {
            const uint32_t old = atomicOr(&vis[v >> 5], 1u << (v & 31));
            if (!(old & (1u << (v & 31)))) {
                atomicOr(&next[v >> 5], 1u << (v & 31));
                cnt++;
            }
        }
        if (cv && !((vis[u >> 5] >> (u & 31)) & 1u)) {
            const uint32_t old = atomicOr(&vis[u >> 5], 1u << (u & 31));
            if (!(old & (1u << (u & 31)))) {
                atomicOr(&next[u >> 5], 1u << (u & 31));
                cnt++;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&st->pred_probe[level], cnt);
}

__global__ void k_features_finish(const unsigned *feat_counts, long long ns, vid_t n, long long m, const DevState *st,
                                  float *x) {
    const int j = threadIdx.x;
    if (j < 64) x[j] = ns > 0 ? (float)feat_counts[j] / (float)ns : 0.0f;
    if (j == 64) x[j] = logf((float)n) / 20.0f;
    if (j == 65) x[j] = logf((float)m + 1.0f) / 20.0f;
    if (j >= 66 && j < 69) x[j] = log1pf((float)st->pred_probe[j - 66]) / 20.0f;
}

template <typename T>
void launch_route_features(const void *edges, long long m, vid_t n, FeatScratch fs, DevState *st, float *x, int grid,
                           cudaStream_t s) {
    const long long ns = ((long long)n + 15) >> kSampleShift;
    const long long nwords = ((long long)n + 31) / 32;
    cudaMemsetAsync(fs.sdeg, 0, (size_t)ns * 4, s);
    cudaMemsetAsync(fs.counts, 0, 64 * 4, s);
    cudaMemsetAsync(fs.vis, 0, (size_t)nwords * 4, s);
    cudaMemsetAsync(fs.f0, 0, (size_t)nwords * 4, s);
    if (m > 0) k_sample_degree<T><<<grid, kBlock, 0, s>>>((const T *)edges, m, n, fs.sdeg, st);
    k_sample_hist<<<grid, kBlock, 0, s>>>(fs.sdeg, ns, fs.counts, st);
    k_probe_seed<<<1, 1, 0, s>>>(fs.vis, fs.f0, n, st);
    uint32_t *cur = fs.f0, *next = fs.f1;
    for (int l = 0; l < 3; l++) {
        cudaMemsetAsync(next, 0, (size_t)nwords * 4, s);
        if (m > 0) k_probe_level<T><<<grid, kBlock, 0, s>>>((const T *)edges, m, n, fs.vis, cur, next, st, l);
        uint32_t *t = cur;
        cur = next;
        next = t;
    }
    k_features_finish<<<1, 96, 0, s>>>(fs.counts, ns, n, m, st, x);
}
template void launch_route_features<int32_t>(const void *, long long, vid_t, FeatScratch, DevState *, float *, int,
                                             cudaStream_t);
template void launch_route_features<int64_t>(const void *, long long, vid_t, FeatScratch, DevState *, float *, int,
                                             cudaStream_t);

}  // namespace ccg

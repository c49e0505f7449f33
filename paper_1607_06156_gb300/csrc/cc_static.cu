// cc_labels_static: the SV-only labelling of cc_labels, run on a fixed
// scratch area that lives in the library itself instead of a workspace the
// library allocates.
//
// Some callers may not allocate device memory on their own: a plugin inside
// an application whose memory pool owns the whole device, or a latency
// critical loop where cudaMalloc / cudaFree (which can synchronise the
// device) are not allowed. This entry point serves them: the caller passes
// the input pairs and the output labels, and all scratch (parent array,
// hooked-root list, two active-pair lists, counters) comes from the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/cc_gb300.h"
#include "cc_common.cuh"
#include "cc_kernels.h"

using namespace ccg;

namespace {

constexpr long long kStaticMaxN = CC_STATIC_MAX_VERTICES;
constexpr long long kStaticMaxM = CC_STATIC_MAX_PAIRS;

// byte offsets inside the scratch array (each region 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffState = 0;
constexpr size_t kOffParent = align256(kOffState + sizeof(DevState));
constexpr size_t kOffHooked = align256(kOffParent + (kStaticMaxN + 4) * 4);
constexpr size_t kOffList0 = align256(kOffHooked + (kStaticMaxN + 4) * 4);
constexpr size_t kOffList1 = align256(kOffList0 + (kStaticMaxM + 4) * 8);
constexpr size_t kScratchBytes = align256(kOffList1 + (kStaticMaxM + 4) * 8);

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

namespace {

// Device address of the scratch array on the current device. The host-side
// symbol is only a stand-in, not a device address. The lookup is cheap and
// is repeated on every call, so a device reset (which reloads the module
// at another address) never leaves a stale pointer behind.
cc_status scratch_for_current_device(unsigned char **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return CC_ERR_CUDA;
    }
    *out = reinterpret_cast<unsigned char *>(p);
    return CC_OK;
}

cc_status cuda_ok(cudaError_t e) {
    if (e == cudaSuccess) return CC_OK;
    cudaGetLastError();
    return CC_ERR_CUDA;
}

template <typename T>
cc_status labels_static(const void *edges, vid_t n, long long m, void *labels, cudaStream_t s, unsigned char *base) {
    DevState *st = reinterpret_cast<DevState *>(base + kOffState);
    vid_t *parent = reinterpret_cast<vid_t *>(base + kOffParent);
    vid_t *hooked = reinterpret_cast<vid_t *>(base + kOffHooked);
    uint2 *list[2] = {reinterpret_cast<uint2 *>(base + kOffList0), reinterpret_cast<uint2 *>(base + kOffList1)};
    int dev = 0, sms = 0, threads = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaDeviceGetAttribute(&threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) {
        cudaGetLastError();
        return CC_ERR_CUDA;
    }
    const int grid = sms * (threads / kBlock);
    int lg = 0;
    while (lg < 62 && (1LL << lg) < (long long)n) lg++;
    const int cap = 64 + 4 * lg < kMaxIters - 1 ? 64 + 4 * lg : kMaxIters - 1;
    // the scratch keeps the previous call's contents: the counters must start at zero
    if (cudaMemsetAsync(st, 0, sizeof(DevState), s) != cudaSuccess) return cuda_ok(cudaGetLastError());
    launch_parent_init(parent, n, nullptr, 0, grid, s);
    unsigned long long kept = 0;
    int it = 0, cur = 0;
    if (m > 0) {
        launch_sv_pass<T>(0, false, false, edges, m, n, parent, nullptr, 0, hooked, nullptr, st, 0, grid, s);
        launch_shortcut_all(parent, n, st, 0, grid, s);
        it = 1;
        launch_sv_pass<T>(2, true, true, edges, m, n, parent, nullptr, 0, hooked, list[0], st, 1, grid, s);
        launch_sv_shortcut(parent, hooked, st, 1, grid, s);
        if (cudaMemcpyAsync(&kept, &st->kept[1], 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return cuda_ok(cudaGetLastError());
    }
    while (kept > 0) {
        if (++it >= cap) return CC_ERR_NO_CONVERGENCE;
        launch_sv_pass<uint32_t>(2, true, true, list[cur], (long long)kept, n, parent, nullptr, 0, hooked,
                                 list[1 - cur], st, it, grid, s);
        launch_sv_shortcut(parent, hooked, st, it, grid, s);
        cur = 1 - cur;
        if (cudaMemcpyAsync(&kept, &st->kept[it], 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return cuda_ok(cudaGetLastError());
    }
    launch_finalize<T>(parent, n, labels, grid, s);
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, &st->err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_ok(cudaGetLastError());
    if (cudaGetLastError() != cudaSuccess) return CC_ERR_CUDA;
    if (err & kErrInvalidEdge) return CC_ERR_INVALID_EDGE;
    if (err) return CC_ERR_CUDA;
    return CC_OK;
}

}  // namespace

extern "C" cc_status cc_labels_static(const void *edges_dev, int id_bytes, int64_t n, int64_t m,
                                      void *labels_out_dev, void *stream) {
    if (id_bytes != 4 && id_bytes != 8) return CC_ERR_INVALID_ARG;
    if (n < 0 || m < 0) return CC_ERR_INVALID_ARG;
    if (n > kStaticMaxN || m > kStaticMaxM) return CC_ERR_UNSUPPORTED;
    if (n == 0) return m > 0 ? CC_ERR_INVALID_EDGE : CC_OK;
    if (!labels_out_dev || (m > 0 && !edges_dev)) return CC_ERR_INVALID_ARG;
    if (((uintptr_t)edges_dev & 15) || ((uintptr_t)labels_out_dev & 15)) return CC_ERR_INVALID_ARG;
    unsigned char *base = nullptr;
    cc_status st = scratch_for_current_device(&base);
    if (st != CC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (id_bytes == 4) return labels_static<int32_t>(edges_dev, (vid_t)n, m, labels_out_dev, s, base);
    return labels_static<int64_t>(edges_dev, (vid_t)n, m, labels_out_dev, s, base);
}

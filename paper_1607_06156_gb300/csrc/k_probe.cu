// L2 random-access rate probe: the measured ceiling of the kernels whose cost
// is scattered 4-byte accesses (the degree pass, the SV hook passes).
//
// One grid-stride kernel per access kind; operation i touches word
// fmix64(i) & mask of the table (MurmurHash3's 64-bit finaliser), so every
// index is in bounds by construction and the pattern is uniform over the
// table, like the parent and degree accesses of a randomly labelled graph.
#include "cc_common.cuh"
#include "cc_kernels.h"

namespace ccg {

__device__ __forceinline__ uint32_t probe_index(unsigned long long x, uint32_t mask) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return (uint32_t)x & mask;
}

// kind 0: loads, 1: atomicAdd (result unused), 2: atomicMin (result unused),
// 3: atomicMin (result used). `sink` receives a value only if the folded
// results hit an impossible pattern, which keeps the loads live.
template <int KIND>
__global__ void __launch_bounds__(kBlock) k_l2_probe(uint32_t *table, uint32_t mask, long long ops, uint32_t *sink) {
    uint32_t acc = 0;
    for (long long i = gtid(); i < ops; i += gstride()) {
        uint32_t *p = table + probe_index((unsigned long long)i, mask);
        if (KIND == 0) acc += *p;
        else if (KIND == 1) atomicAdd(p, 1u);
        else if (KIND == 2) atomicMin(p, (uint32_t)i);
        else acc += atomicMin(p, (uint32_t)i);
    }
    if ((KIND == 0 || KIND == 3) && acc == 0x9e3779b9u) sink[0] = acc;
}

void launch_l2_probe(int kind, uint32_t *table, uint32_t mask, long long ops, uint32_t *sink, int grid,
                     cudaStream_t s) {
    switch (kind) {
    case 0: k_l2_probe<0><<<grid, kBlock, 0, s>>>(table, mask, ops, sink); break;
    case 1: k_l2_probe<1><<<grid, kBlock, 0, s>>>(table, mask, ops, sink); break;
    case 2: k_l2_probe<2><<<grid, kBlock, 0, s>>>(table, mask, ops, sink); break;
    default: k_l2_probe<3><<<grid, kBlock, 0, s>>>(table, mask, ops, sink); break;
    }
}

}  // namespace ccg

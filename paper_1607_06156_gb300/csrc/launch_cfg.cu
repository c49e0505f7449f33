// Launch configuration: grid-stride kernels get as many blocks as fit on
// the device at once (their occupancy times the SM count), so that no block
// waits for a second wave while the first wave works through the same
// number of tiles. Occupancy depends on each kernel's registers and shared
// memory, so it is queried once per kernel and device and cached.
#include "cc_kernels.h"

#include <mutex>
#include <vector>

namespace ccg {

namespace {
struct FitEntry {
    const void *kernel;
    int device, block;
    size_t smem;
    int resident;
};
std::mutex g_fit_mu;
std::vector<FitEntry> g_fit;
}  // namespace

int fit_grid(const void *kernel, int grid, int block, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return grid;
    }
    {
        std::lock_guard<std::mutex> lk(g_fit_mu);
        for (const FitEntry &e : g_fit)
            if (e.kernel == kernel && e.device == dev && e.block == block && e.smem == smem)
                return e.resident < grid ? e.resident : grid;
    }
    int occ = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || occ <= 0 || sms <= 0) {
        cudaGetLastError();
        return grid;
    }
    const int resident = occ * sms;
    std::lock_guard<std::mutex> lk(g_fit_mu);
    g_fit.push_back({kernel, dev, block, smem, resident});
    return resident < grid ? resident : grid;
}

}  // namespace ccg

// launch.h -- grid sizing of the persistent fragment kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace rt {

// Number of blocks of a persistent kernel: enough to cover `chunks` 32-fragment
// chunks with `warps` warps per block, at most (SMs x resident blocks per SM).
// The occupancy query is cached per kernel and device.
template <typename Kernel>
inline unsigned persistent_grid(Kernel kernel, int threads, int64_t chunks, size_t dynamic_smem = 0) {
    static std::mutex mu;
    static int cached_dev[64];
    static int cached_blocks[64];
    static bool init = false;
    int dev = 0;
    cudaGetDevice(&dev);
    int total = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!init) {
            for (int k = 0; k < 64; ++k) cached_dev[k] = -1;
            init = true;
        }
        if (dev >= 0 && dev < 64 && cached_dev[dev] == dev) total = cached_blocks[dev];
    }
    if (total == 0) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, dynamic_smem);
        total = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
        std::lock_guard<std::mutex> lock(mu);
        if (dev >= 0 && dev < 64) {
            cached_dev[dev] = dev;
            cached_blocks[dev] = total;
        }
    }
    const int warps = threads / 32;
    int64_t want = (chunks + warps - 1) / warps;
    if (want < 1) want = 1;
    return (unsigned)(want < total ? want : total);
}

}  // namespace rt

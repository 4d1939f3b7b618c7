// footprint_noalloc.cu -- rt_footprint_noalloc: the footprint counter without
// any device allocation.
//
// rt_footprint allocates its texel bitmap (and two small arrays) with
// cudaMalloc on every call and frees them afterwards.  Some callers cannot do
// that: a host application or framework that owns all device memory through
// its own allocator (a caching allocator, a fixed memory budget) and forbids
// allocations behind its back, or a per-frame render loop in which cudaMalloc /
// cudaFree would synchronise the device and stall the frame.  This entry point
// keeps its scratch in file-scope device arrays instead: every GPU that loads
// the library holds them (8 MiB + 8 KiB) until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "radtex.h"
#include "rt_device.cuh"
#include "rt_internal.h"

namespace {

// One bit per texel, summed over the context's objects (PLANES numbering).
constexpr int64_t kMaxTexels = RT_FOOTPRINT_NOALLOC_MAX_TEXELS;
constexpr int64_t kMaxWords = kMaxTexels / 32;
static __device__ __align__(256) uint32_t g_bitmap[kMaxWords];
// First bitmap word of each object.
static __device__ __align__(256) int64_t g_word_offset[RT_MAX_OBJECTS + 1];

// Device addresses of the two arrays, looked up once per device.  In host code
// the arrays' names stand for host-side shadows, not device addresses, so they
// are never passed to a kernel directly.
struct StaticScratch {
    bool ready = false;
    uint32_t* bitmap = nullptr;
    int64_t* word_offset = nullptr;
};
constexpr int kMaxDevices = 64;
std::mutex g_mu;
StaticScratch g_scratch[kMaxDevices];

// Called with `device` current.
cudaError_t scratch_for(int device, StaticScratch* out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    StaticScratch& s = g_scratch[device];
    if (!s.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_bitmap);
        if (e != cudaSuccess) return e;
        s.bitmap = static_cast<uint32_t*>(p);
        e = cudaGetSymbolAddress(&p, g_word_offset);
        if (e != cudaSuccess) return e;
        s.word_offset = static_cast<int64_t*>(p);
        s.ready = true;
    }
    *out = s;
    return cudaSuccess;
}

}  // namespace

extern "C" rt_status rt_footprint_noalloc(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj,
                                          int64_t F, rt_filter filter, uint64_t* counts_dev, int32_t n_counts,
                                          rt_stream_t stream) {
    if (!ctx || (filter != RT_NEAREST && filter != RT_ANGULAR_BILINEAR && filter != RT_QUADRILINEAR))
        return RT_ERR_INVALID_ARG;
    if (n_counts < 0 || n_counts > RT_MAX_OBJECTS || (n_counts > 0 && !counts_dev)) return RT_ERR_INVALID_ARG;
    if (F < 0 || (F > 0 && (!uv || !dir || !obj))) return RT_ERR_INVALID_ARG;
    if (((uintptr_t)uv | (uintptr_t)dir | (uintptr_t)obj) & 15u) return RT_ERR_INVALID_ARG;
    if (((uintptr_t)counts_dev) & 7u) return RT_ERR_INVALID_ARG;

    // Bitmap words of every object: the sum must fit the static bitmap.
    int n_obj = 0;
    int64_t offset[RT_MAX_OBJECTS + 1];
    offset[0] = 0;
    const rt::TexDesc* table = rt_internal_host_table(ctx, &n_obj);
    for (int o = 0; o < n_obj; ++o) {
        const rt::TexDesc& d = table[o];
        const int64_t texels = d.live ? d.plane * d.n * d.n : 0;
        offset[o + 1] = offset[o] + (texels + 31) / 32;
    }
    const int64_t words = offset[n_obj];
    if (words > kMaxWords) return RT_ERR_INVALID_ARG;  // more than RT_FOOTPRINT_NOALLOC_MAX_TEXELS texels

    int prev = -1, device = rt_internal_device(ctx);
    if (cudaGetDevice(&prev) != cudaSuccess) return RT_ERR_CUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return RT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    StaticScratch sc;
    cudaError_t e = scratch_for(device, &sc);
    // The arrays keep the previous call's contents: clear the outputs and the used words.
    if (e == cudaSuccess && n_counts > 0) e = cudaMemsetAsync(counts_dev, 0, sizeof(uint64_t) * n_counts, s);
    if (e == cudaSuccess && words > 0) e = cudaMemsetAsync(sc.bitmap, 0, sizeof(uint32_t) * (size_t)words, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sc.word_offset, offset, sizeof(int64_t) * (size_t)(n_obj + 1), cudaMemcpyHostToDevice,
                            s);
    if (e == cudaSuccess && F > 0)
        e = rt::launch_footprint_mark(rt_internal_device_table(ctx), n_obj, uv, dir, obj, F, filter, sc.bitmap,
                                      sc.word_offset, rt_internal_status(ctx), s);
    for (int o = 0; o < n_counts && o < n_obj && e == cudaSuccess; ++o)
        e = rt::launch_popcount(sc.bitmap + offset[o], offset[o + 1] - offset[o],
                                reinterpret_cast<unsigned long long*>(counts_dev) + o, s);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e == cudaSuccess) return RT_OK;
    return e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA;
}

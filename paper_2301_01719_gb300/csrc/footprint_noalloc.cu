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
//
// Nothing of a call is read from host memory on the GPU side: the per-object
// word offsets are computed on the device from the context's device-side
// descriptor table, and one popcount launch reads them from there.
#include <cuda.h>
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
// First bitmap word of each object, and the total after the last one.
static __device__ __align__(256) int64_t g_word_offset[RT_MAX_OBJECTS + 1];

// Word offsets of the objects 0 .. n_obj - 1 from the device table (a dead
// slot takes no words), and zeros in the caller's counts.  One block; the
// running sum is taken by thread 0 (at most RT_MAX_OBJECTS entries).
__global__ void noalloc_offsets_kernel(const rt::TexDesc* __restrict__ table, int n_obj, int64_t* word_offset,
                                       unsigned long long* counts, int n_counts) {
    for (int o = threadIdx.x; o < n_counts; o += blockDim.x) counts[o] = 0ull;
    if (threadIdx.x != 0) return;
    int64_t acc = 0;
    word_offset[0] = 0;
    for (int o = 0; o < n_obj; ++o) {
        const rt::TexDesc& d = table[o];
        const int64_t texels = d.live ? d.plane * d.n * d.n : 0;
        acc += (texels + 31) / 32;
        word_offset[o + 1] = acc;
    }
}

// Set bits of object blockIdx.y's words, added to counts[blockIdx.y].
__global__ void noalloc_popcount_kernel(const uint32_t* __restrict__ bitmap,
                                        const int64_t* __restrict__ word_offset, unsigned long long* counts) {
    const int o = blockIdx.y;
    const int64_t lo = word_offset[o], hi = word_offset[o + 1];
    unsigned long long local = 0;
    for (int64_t w = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < hi; w += (int64_t)gridDim.x * blockDim.x)
        local += __popc(bitmap[w]);
    for (int k = 16; k > 0; k >>= 1) local += __shfl_down_sync(0xFFFFFFFFu, local, k);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(counts + o, local);
}

// Device addresses of the two arrays.  In host code the arrays' names stand
// for host-side shadows, not device addresses, so they are never passed to a
// kernel directly.  The addresses are looked up once per device and context:
// a device reset (cudaDeviceReset, or a framework tearing its context down)
// makes a new primary context, whose module -- and arrays -- may sit
// elsewhere, so the cache is keyed on the current context's unique id.
struct StaticScratch {
    bool ready = false;
    unsigned long long ctx_id = 0;
    uint32_t* bitmap = nullptr;
    int64_t* word_offset = nullptr;
};
constexpr int kMaxDevices = 64;
std::mutex g_mu;
StaticScratch g_scratch[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// The current context's unique id, or false when the driver cannot tell.
bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
    });
    CUcontext c = nullptr;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

// Called with `device` current (the runtime has made its primary context
// current by then).
cudaError_t scratch_for(int device, StaticScratch* out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned long long id = 0;
    const bool keyed = current_context_id(&id);
    std::lock_guard<std::mutex> lock(g_mu);
    StaticScratch& s = g_scratch[device];
    if (!s.ready || !keyed || s.ctx_id != id) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_bitmap);
        if (e != cudaSuccess) return e;
        s.bitmap = static_cast<uint32_t*>(p);
        e = cudaGetSymbolAddress(&p, g_word_offset);
        if (e != cudaSuccess) return e;
        s.word_offset = static_cast<int64_t*>(p);
        s.ctx_id = id;
        s.ready = keyed;  // without a context id the addresses are looked up on every call
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
    // the G-buffer rules of every shading call (rt_footprint's included)
    if (F < 0 || (F > 0 && (!uv || !dir || !obj))) return RT_ERR_INVALID_ARG;
    if (F > 0 && (((uintptr_t)uv | (uintptr_t)dir | (uintptr_t)obj) & 15u)) return RT_ERR_INVALID_ARG;
    if (n_counts < 0 || (n_counts > 0 && !counts_dev) || (((uintptr_t)counts_dev) & 7u)) return RT_ERR_INVALID_ARG;

    // Bitmap words of every object: the sum must fit the static bitmap.
    int n_obj = 0;
    const rt::TexDesc* table = rt_internal_host_table(ctx, &n_obj);
    int64_t words = 0;
    for (int o = 0; o < n_obj; ++o) {
        const rt::TexDesc& d = table[o];
        const int64_t texels = d.live ? d.plane * d.n * d.n : 0;
        words += (texels + 31) / 32;
    }
    if (words > kMaxWords) return RT_ERR_INVALID_ARG;  // more than RT_FOOTPRINT_NOALLOC_MAX_TEXELS texels

    int prev = -1, device = rt_internal_device(ctx);
    if (cudaGetDevice(&prev) != cudaSuccess) return RT_ERR_CUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return RT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    StaticScratch sc;
    cudaError_t e = scratch_for(device, &sc);
    // The arrays keep the previous call's contents: the offsets are rewritten,
    // the counts zeroed (entries past the last object stay zero) and the used
    // bitmap words cleared before the marking pass.
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(counts_dev);
    if (e == cudaSuccess) {
        noalloc_offsets_kernel<<<1, 256, 0, s>>>(rt_internal_device_table(ctx), n_obj, sc.word_offset, counts,
                                                 n_counts);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && words > 0) e = cudaMemsetAsync(sc.bitmap, 0, sizeof(uint32_t) * (size_t)words, s);
    if (e == cudaSuccess && F > 0)
        e = rt::launch_footprint_mark(rt_internal_device_table(ctx), n_obj, uv, dir, obj, F, filter, sc.bitmap,
                                      sc.word_offset, rt_internal_status(ctx), s);
    const int n_pop = n_counts < n_obj ? n_counts : n_obj;
    if (e == cudaSuccess && n_pop > 0 && words > 0) {
        int64_t per = (words + 255) / 256;  // blocks to cover every word once, spread over the objects
        const unsigned gx = (unsigned)(per < 1024 ? per : 1024);
        noalloc_popcount_kernel<<<dim3(gx, (unsigned)n_pop), 256, 0, s>>>(sc.bitmap, sc.word_offset, counts);
        e = cudaGetLastError();
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e == cudaSuccess) return RT_OK;
    return e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA;
}

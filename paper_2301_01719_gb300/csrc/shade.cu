// shade.cu -- forward synthesis and lookup-coordinate kernels.
//
// One thread shades one fragment; each block stages its slice of the G-buffer
// through shared memory with 16-byte vector loads, and every thread writes its
// colour with one 16-byte store.  Texels are gathered through the
// read-only path; consecutive fragments of a scanline fall in neighbouring
// buckets, and in the PLANES layout neighbouring buckets at one in-bucket
// texel are neighbours in memory, so a warp's taps share cache lines.
#include "rt_device.cuh"
#include "rt_filter.cuh"
#include "rt_internal.h"

namespace rt {

constexpr int kShadeThreads = 256;

template <int FILTER>
__global__ void __launch_bounds__(kShadeThreads) shade_kernel(const TexDesc* __restrict__ table, int n_obj,
                                                              const float* __restrict__ uv,
                                                              const float* __restrict__ dir,
                                                              const int32_t* __restrict__ obj, int64_t F,
                                                              float* __restrict__ out, unsigned* status) {
    __shared__ GStage<kShadeThreads> S;
    const Frag q = stage_gbuffer<kShadeThreads>(uv, dir, obj, F, S);
    const int64_t f = (int64_t)blockIdx.x * kShadeThreads + threadIdx.x;
    if (f >= F) return;
    float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
    TexDesc d;
    if (fragment_valid(table, n_obj, q.o, q.u, q.v, q.x, q.y, q.z, status, d)) {
        Lookup<FILTER> L = locate<FILTER>(d, q.u, q.v, q.x, q.y, q.z);
        res = filter_any<FILTER>(d, L);
    }
    __stcs(reinterpret_cast<float4*>(out) + f, res);
}

template <int FILTER>
__global__ void __launch_bounds__(kShadeThreads) locate_kernel(const TexDesc* __restrict__ table, int n_obj,
                                                               const float* __restrict__ uv,
                                                               const float* __restrict__ dir,
                                                               const int32_t* __restrict__ obj, int64_t F,
                                                               int32_t* __restrict__ idx, float* __restrict__ coord,
                                                               unsigned* status) {
    __shared__ GStage<kShadeThreads> S;
    const Frag q = stage_gbuffer<kShadeThreads>(uv, dir, obj, F, S);
    const int64_t f = (int64_t)blockIdx.x * kShadeThreads + threadIdx.x;
    if (f >= F) return;
    int4 I = make_int4(0, 0, 0, 0);
    float4 C = make_float4(0.f, 0.f, 0.f, 0.f);
    TexDesc d;
    if (fragment_valid(table, n_obj, q.o, q.u, q.v, q.x, q.y, q.z, status, d)) {
        Lookup<FILTER> L = locate<FILTER>(d, q.u, q.v, q.x, q.y, q.z);
        I = make_int4(L.u.fl, L.v.fl, L.s.fl, L.t.fl);
        C = make_float4(L.u.c, L.v.c, L.s.c, L.t.c);
    }
    reinterpret_cast<int4*>(idx)[f] = I;
    reinterpret_cast<float4*>(coord)[f] = C;
}

static inline unsigned grid_for(int64_t F) { return (unsigned)((F + kShadeThreads - 1) / kShadeThreads); }

cudaError_t launch_shade(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                         int64_t F, int filter, float* out, unsigned* status, cudaStream_t stream) {
    dim3 grid(grid_for(F)), block(kShadeThreads);
    switch (filter) {
        case RT_NEAREST:
            shade_kernel<RT_NEAREST><<<grid, block, 0, stream>>>(table, n_obj, uv, dir, obj, F, out, status);
            break;
        case RT_ANGULAR_BILINEAR:
            shade_kernel<RT_ANGULAR_BILINEAR><<<grid, block, 0, stream>>>(table, n_obj, uv, dir, obj, F, out,
                                                                          status);
            break;
        default:
            shade_kernel<RT_QUADRILINEAR><<<grid, block, 0, stream>>>(table, n_obj, uv, dir, obj, F, out, status);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_locate(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                          int64_t F, int filter, int32_t* idx, float* coord, unsigned* status, cudaStream_t stream) {
    dim3 grid(grid_for(F)), block(kShadeThreads);
    switch (filter) {
        case RT_NEAREST:
            locate_kernel<RT_NEAREST><<<grid, block, 0, stream>>>(table, n_obj, uv, dir, obj, F, idx, coord, status);
            break;
        case RT_ANGULAR_BILINEAR:
            locate_kernel<RT_ANGULAR_BILINEAR><<<grid, block, 0, stream>>>(table, n_obj, uv, dir, obj, F, idx,
                                                                           coord, status);
            break;
        default:
            locate_kernel<RT_QUADRILINEAR><<<grid, block, 0, stream>>>(table, n_obj, uv, dir, obj, F, idx, coord,
                                                                       status);
            break;
    }
    return cudaGetLastError();
}

}  // namespace rt

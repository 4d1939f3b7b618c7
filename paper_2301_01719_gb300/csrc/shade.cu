// shade.cu -- forward synthesis and lookup-coordinate kernels.
//
// Persistent kernels: every warp walks 32-fragment chunks (a run of the flat
// stream, or a screen tile of a batch of frames) with the G-buffer of its next
// chunk prefetched into shared memory (rt_filter.cuh), one fragment per lane,
// and writes its colour with one 16-byte store.  Texels are gathered through
// the read-only path; fragments that are close on screen fall in neighbouring
// buckets, and in the PLANES layout neighbouring buckets at one in-bucket texel
// are neighbours in memory, so a warp's taps share cache lines.
#include "launch.h"
#include "rt_device.cuh"
#include "rt_filter.cuh"
#include "rt_internal.h"

namespace rt {

constexpr int kShadeThreads = 128;
constexpr int kShadeWarps = kShadeThreads / 32;

// The screen-tiled forward keeps three G-buffer chunks per warp (two in
// flight) and is held to 64 registers, 8 blocks (32 warps) per SM: measured 4%
// faster than two chunks at 72 registers.  The flat stream keeps two chunks
// (it would spill at 64 registers).
template <bool TILED>
constexpr int shade_stages() { return TILED ? 3 : 2; }

template <int FILTER, bool TILED>
__global__ void __launch_bounds__(kShadeThreads, TILED ? 8 : 1) shade_kernel(const TexDesc* __restrict__ table, int n_obj,
                                                              const float* __restrict__ uv,
                                                              const float* __restrict__ dir,
                                                              const int32_t* __restrict__ obj, int64_t F,
                                                              Tiling tiling, float* __restrict__ out,
                                                              unsigned* status) {
    __shared__ WarpStage<false, shade_stages<TILED>()> stages[kShadeWarps];
    for_each_fragment<kShadeWarps, false, TILED, shade_stages<TILED>()>(uv, dir, obj, nullptr, F, tiling, stages,
                                                               [&](int64_t f, const Frag& q, float4) {
        float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
        TexDesc d;
        if (fragment_valid(table, n_obj, q.o, q.u, q.v, q.x, q.y, q.z, status, d)) {
            Lookup<FILTER> L = locate<FILTER>(d, q.u, q.v, q.x, q.y, q.z);
            res = filter_any<FILTER>(d, L);
        }
        if (f >= 0) __stcs(reinterpret_cast<float4*>(out) + f, res);
    });
}

template <int FILTER, bool TILED>
__global__ void __launch_bounds__(kShadeThreads) locate_kernel(const TexDesc* __restrict__ table, int n_obj,
                                                               const float* __restrict__ uv,
                                                               const float* __restrict__ dir,
                                                               const int32_t* __restrict__ obj, int64_t F,
                                                               Tiling tiling, int32_t* __restrict__ idx,
                                                               float* __restrict__ coord, unsigned* status) {
    __shared__ WarpStage<false> stages[kShadeWarps];
    for_each_fragment<kShadeWarps, false, TILED, 2>(uv, dir, obj, nullptr, F, tiling, stages,
                                                    [&](int64_t f, const Frag& q, float4) {
        int4 I = make_int4(0, 0, 0, 0);
        float4 C = make_float4(0.f, 0.f, 0.f, 0.f);
        TexDesc d;
        if (fragment_valid(table, n_obj, q.o, q.u, q.v, q.x, q.y, q.z, status, d)) {
            Lookup<FILTER> L = locate<FILTER>(d, q.u, q.v, q.x, q.y, q.z);
            I = make_int4(L.u.fl, L.v.fl, L.s.fl, L.t.fl);
            C = make_float4(L.u.c, L.v.c, L.s.c, L.t.c);
        }
        if (f >= 0) {
            reinterpret_cast<int4*>(idx)[f] = I;
            reinterpret_cast<float4*>(coord)[f] = C;
        }
    });
}

// World-space forward and lookup (Eq. 1a with a per-fragment normal): one
// fragment per thread, grid-stride; the G-buffer has a fourth stream, the
// normal, and no screen tiling.
template <int FILTER>
__global__ void __launch_bounds__(kShadeThreads) world_shade_kernel(const TexDesc* __restrict__ table, int n_obj,
                                                                    const float* __restrict__ uv,
                                                                    const float* __restrict__ dir,
                                                                    const float* __restrict__ nrm,
                                                                    const int32_t* __restrict__ obj, int64_t F,
                                                                    float* __restrict__ out, int32_t* __restrict__ idx,
                                                                    float* __restrict__ coord, unsigned* status) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        const float2 q = reinterpret_cast<const float2*>(uv)[f];
        const float3 I = make_float3(dir[3 * f], dir[3 * f + 1], dir[3 * f + 2]);
        const float3 N = make_float3(nrm[3 * f], nrm[3 * f + 1], nrm[3 * f + 2]);
        float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
        int4 Ix = make_int4(0, 0, 0, 0);
        float4 C = make_float4(0.f, 0.f, 0.f, 0.f);
        TexDesc d;
        if (fragment_valid(table, n_obj, obj[f], q.x, q.y, I.x, I.y, I.z, status, d) && normal_valid(N, status)) {
            const Lookup<FILTER> L = locate_world<FILTER>(d, q.x, q.y, I, N);
            if (out) res = filter_any<FILTER>(d, L);
            Ix = make_int4(L.u.fl, L.v.fl, L.s.fl, L.t.fl);
            C = make_float4(L.u.c, L.v.c, L.s.c, L.t.c);
        }
        if (out) __stcs(reinterpret_cast<float4*>(out) + f, res);
        if (idx) {
            reinterpret_cast<int4*>(idx)[f] = Ix;
            reinterpret_cast<float4*>(coord)[f] = C;
        }
    }
}

// S lookups per fragment, averaged (area lights over a shadow texture, Section
// 5: "more than one sample per bucket"): dirs holds S directions per fragment.
template <int FILTER>
__global__ void __launch_bounds__(kShadeThreads) multi_shade_kernel(const TexDesc* __restrict__ table, int n_obj,
                                                                    const float* __restrict__ uv,
                                                                    const float* __restrict__ dirs, int S,
                                                                    const int32_t* __restrict__ obj, int64_t F,
                                                                    float* __restrict__ out, unsigned* status) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        const float2 q = reinterpret_cast<const float2*>(uv)[f];
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        bool ok = true;
        for (int k = 0; k < S && ok; ++k) {
            const float* I = dirs + 3 * (f * S + k);
            TexDesc d;
            ok = fragment_valid(table, n_obj, obj[f], q.x, q.y, I[0], I[1], I[2], status, d);
            if (!ok) break;
            const float4 c = filter_any<FILTER>(d, locate<FILTER>(d, q.x, q.y, I[0], I[1], I[2]));
            acc.x += c.x;
            acc.y += c.y;
            acc.z += c.z;
            acc.w += c.w;
        }
        const float inv = 1.0f / (float)S;
        const float4 res = ok ? make_float4(acc.x * inv, acc.y * inv, acc.z * inv, acc.w * inv)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        __stcs(reinterpret_cast<float4*>(out) + f, res);
    }
}

cudaError_t launch_multi_shade(const TexDesc* table, int n_obj, const float* uv, const float* dirs, int S,
                               const int32_t* obj, int64_t F, int filter, float* out, unsigned* status,
                               cudaStream_t stream) {
    const int64_t items = (F + kShadeThreads - 1) / kShadeThreads;
    switch (filter) {
        case RT_NEAREST: {
            const unsigned grid = persistent_grid(multi_shade_kernel<RT_NEAREST>, kShadeThreads, items);
            multi_shade_kernel<RT_NEAREST><<<grid, kShadeThreads, 0, stream>>>(table, n_obj, uv, dirs, S, obj, F,
                                                                               out, status);
            break;
        }
        case RT_ANGULAR_BILINEAR: {
            const unsigned grid = persistent_grid(multi_shade_kernel<RT_ANGULAR_BILINEAR>, kShadeThreads, items);
            multi_shade_kernel<RT_ANGULAR_BILINEAR><<<grid, kShadeThreads, 0, stream>>>(table, n_obj, uv, dirs, S,
                                                                                        obj, F, out, status);
            break;
        }
        default: {
            const unsigned grid = persistent_grid(multi_shade_kernel<RT_QUADRILINEAR>, kShadeThreads, items);
            multi_shade_kernel<RT_QUADRILINEAR><<<grid, kShadeThreads, 0, stream>>>(table, n_obj, uv, dirs, S, obj,
                                                                                    F, out, status);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_world_shade(const TexDesc* table, int n_obj, const float* uv, const float* dir, const float* nrm,
                               const int32_t* obj, int64_t F, int filter, float* out, int32_t* idx, float* coord,
                               unsigned* status, cudaStream_t stream) {
    const int64_t items = (F + kShadeThreads - 1) / kShadeThreads;
    switch (filter) {
        case RT_NEAREST: {
            const unsigned grid = persistent_grid(world_shade_kernel<RT_NEAREST>, kShadeThreads, items);
            world_shade_kernel<RT_NEAREST><<<grid, kShadeThreads, 0, stream>>>(table, n_obj, uv, dir, nrm, obj, F,
                                                                               out, idx, coord, status);
            break;
        }
        case RT_ANGULAR_BILINEAR: {
            const unsigned grid = persistent_grid(world_shade_kernel<RT_ANGULAR_BILINEAR>, kShadeThreads, items);
            world_shade_kernel<RT_ANGULAR_BILINEAR><<<grid, kShadeThreads, 0, stream>>>(
                table, n_obj, uv, dir, nrm, obj, F, out, idx, coord, status);
            break;
        }
        default: {
            const unsigned grid = persistent_grid(world_shade_kernel<RT_QUADRILINEAR>, kShadeThreads, items);
            world_shade_kernel<RT_QUADRILINEAR><<<grid, kShadeThreads, 0, stream>>>(table, n_obj, uv, dir, nrm, obj,
                                                                                    F, out, idx, coord, status);
        }
    }
    return cudaGetLastError();
}

template <int FILTER, bool TILED>
static cudaError_t launch_shade_t(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                  const int32_t* obj, int64_t F, const Tiling& T, float* out, unsigned* status,
                                  cudaStream_t stream) {
    const unsigned grid = persistent_grid(shade_kernel<FILTER, TILED>, kShadeThreads,
                                          chunk_count_host(T, F, kShadeWarps));
    shade_kernel<FILTER, TILED><<<grid, kShadeThreads, 0, stream>>>(table, n_obj, uv, dir, obj, F, T, out, status);
    return cudaGetLastError();
}

template <bool TILED>
static cudaError_t launch_shade_f(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                  const int32_t* obj, int64_t F, int filter, const Tiling& T, float* out,
                                  unsigned* status, cudaStream_t stream) {
    switch (filter) {
        case RT_NEAREST:
            return launch_shade_t<RT_NEAREST, TILED>(table, n_obj, uv, dir, obj, F, T, out, status, stream);
        case RT_ANGULAR_BILINEAR:
            return launch_shade_t<RT_ANGULAR_BILINEAR, TILED>(table, n_obj, uv, dir, obj, F, T, out, status, stream);
        default:
            return launch_shade_t<RT_QUADRILINEAR, TILED>(table, n_obj, uv, dir, obj, F, T, out, status, stream);
    }
}

cudaError_t launch_shade(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                         int64_t F, int filter, const Tiling& T, float* out, unsigned* status, cudaStream_t stream) {
    if (T.W > 0) return launch_shade_f<true>(table, n_obj, uv, dir, obj, F, filter, T, out, status, stream);
    return launch_shade_f<false>(table, n_obj, uv, dir, obj, F, filter, T, out, status, stream);
}

template <int FILTER, bool TILED>
static cudaError_t launch_locate_t(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                   const int32_t* obj, int64_t F, const Tiling& T, int32_t* idx, float* coord,
                                   unsigned* status, cudaStream_t stream) {
    const unsigned grid = persistent_grid(locate_kernel<FILTER, TILED>, kShadeThreads,
                                          chunk_count_host(T, F, kShadeWarps));
    locate_kernel<FILTER, TILED><<<grid, kShadeThreads, 0, stream>>>(table, n_obj, uv, dir, obj, F, T, idx, coord,
                                                                     status);
    return cudaGetLastError();
}

cudaError_t launch_locate(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                          int64_t F, int filter, int32_t* idx, float* coord, unsigned* status, cudaStream_t stream) {
    const Tiling T = flat_tiling();
    switch (filter) {
        case RT_NEAREST:
            return launch_locate_t<RT_NEAREST, false>(table, n_obj, uv, dir, obj, F, T, idx, coord, status, stream);
        case RT_ANGULAR_BILINEAR:
            return launch_locate_t<RT_ANGULAR_BILINEAR, false>(table, n_obj, uv, dir, obj, F, T, idx, coord, status,
                                                               stream);
        default:
            return launch_locate_t<RT_QUADRILINEAR, false>(table, n_obj, uv, dir, obj, F, T, idx, coord, status,
                                                           stream);
    }
}

}  // namespace rt

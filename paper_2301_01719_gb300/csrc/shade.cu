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

template <int FILTER, bool TILED, int SPEC>
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
            Lookup<FILTER> L = locate<FILTER, (SPEC < 0)>(d, q.u, q.v, q.x, q.y, q.z);
            res = filter_spec<FILTER, SPEC>(d, L);
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

// World-space forward and lookup (Eq. 1a with a per-fragment normal): the
// streamer of the tangent-space kernels with a fourth staged stream, the
// normal, over the flat fragment stream or, TILED, over screen tiles of a batch
// of frames.
template <int FILTER, bool TILED>
__global__ void __launch_bounds__(kShadeThreads) world_shade_kernel(const TexDesc* __restrict__ table, int n_obj,
                                                                    const float* __restrict__ uv,
                                                                    const float* __restrict__ dir,
                                                                    const float* __restrict__ nrm,
                                                                    const int32_t* __restrict__ obj, int64_t F,
                                                                    Tiling tiling, float* __restrict__ out,
                                                                    int32_t* __restrict__ idx,
                                                                    float* __restrict__ coord, unsigned* status) {
    __shared__ WarpStage<false, 2, true> stages[kShadeWarps];
    for_each_fragment<kShadeWarps, false, TILED, 2, true>(uv, dir, obj, nullptr, F, tiling, stages,
                                                          [&](int64_t f, const Frag& q, float4) {
        float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
        int4 Ix = make_int4(0, 0, 0, 0);
        float4 C = make_float4(0.f, 0.f, 0.f, 0.f);
        TexDesc d;
        const float3 N = make_float3(q.nx, q.ny, q.nz);
        if (fragment_valid(table, n_obj, q.o, q.u, q.v, q.x, q.y, q.z, status, d) && normal_valid(N, status)) {
            const Lookup<FILTER> L = locate_world<FILTER>(d, q.u, q.v, make_float3(q.x, q.y, q.z), N);
            if (out) res = filter_any<FILTER>(d, L);
            Ix = make_int4(L.u.fl, L.v.fl, L.s.fl, L.t.fl);
            C = make_float4(L.u.c, L.v.c, L.s.c, L.t.c);
        }
        if (f < 0) return;
        if (out) __stcs(reinterpret_cast<float4*>(out) + f, res);
        if (idx) {
            reinterpret_cast<int4*>(idx)[f] = Ix;
            reinterpret_cast<float4*>(coord)[f] = C;
        }
    }, nrm);
}

template <int FILTER, bool TILED>
static cudaError_t launch_world_shade_t(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                        const float* nrm, const int32_t* obj, int64_t F, const Tiling& T, float* out,
                                        int32_t* idx, float* coord, unsigned* status, cudaStream_t stream) {
    const unsigned grid = persistent_grid(world_shade_kernel<FILTER, TILED>, kShadeThreads,
                                          chunk_count_host(T, F, kShadeWarps));
    world_shade_kernel<FILTER, TILED><<<grid, kShadeThreads, 0, stream>>>(table, n_obj, uv, dir, nrm, obj, F, T,
                                                                          out, idx, coord, status);
    return cudaGetLastError();
}

template <bool TILED>
static cudaError_t launch_world_shade_f(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                        const float* nrm, const int32_t* obj, int64_t F, int filter, const Tiling& T,
                                        float* out, int32_t* idx, float* coord, unsigned* status,
                                        cudaStream_t stream) {
    switch (filter) {
        case RT_NEAREST:
            return launch_world_shade_t<RT_NEAREST, TILED>(table, n_obj, uv, dir, nrm, obj, F, T, out, idx, coord,
                                                           status, stream);
        case RT_ANGULAR_BILINEAR:
            return launch_world_shade_t<RT_ANGULAR_BILINEAR, TILED>(table, n_obj, uv, dir, nrm, obj, F, T, out, idx,
                                                                    coord, status, stream);
        default:
            return launch_world_shade_t<RT_QUADRILINEAR, TILED>(table, n_obj, uv, dir, nrm, obj, F, T, out, idx,
                                                                coord, status, stream);
    }
}

cudaError_t launch_world_shade(const TexDesc* table, int n_obj, const float* uv, const float* dir, const float* nrm,
                               const int32_t* obj, int64_t F, int filter, const Tiling& T, float* out, int32_t* idx,
                               float* coord, unsigned* status, cudaStream_t stream) {
    if (T.W > 0)
        return launch_world_shade_f<true>(table, n_obj, uv, dir, nrm, obj, F, filter, T, out, idx, coord, status,
                                          stream);
    return launch_world_shade_f<false>(table, n_obj, uv, dir, nrm, obj, F, filter, T, out, idx, coord, status,
                                       stream);
}

// S lookups per fragment, averaged (area lights over a shadow texture, Section
// 5: "more than one sample per bucket"): dirs holds S directions per fragment.
// General S: one fragment per thread, the samples in a loop.
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

// S a power of two <= 32: one lookup per lane, lanes f S .. f S + S - 1 of a
// warp share fragment f (coalesced direction loads, 32 lookups in flight per
// warp) and sum by butterfly shuffles.  Each lane loads the inputs of its next
// lookup before filtering the current one, so their DRAM latency overlaps the
// gathers (which hit L1 and L2: a bit texture is small).
template <int FILTER>
__global__ void __launch_bounds__(kShadeThreads) multi_shade_lanes_kernel(const TexDesc* __restrict__ table,
                                                                          int n_obj, const float* __restrict__ uv,
                                                                          const float* __restrict__ dirs, int S,
                                                                          const int32_t* __restrict__ obj, int64_t F,
                                                                          float* __restrict__ out, unsigned* status) {
    const int lane = threadIdx.x & 31;
    const int lg = __ffs(S) - 1;  // S = 2^lg
    const int64_t total = F * S;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t stride = (((int64_t)gridDim.x * blockDim.x) >> 5) * 32;
    float2 q = make_float2(0.f, 0.f);
    float ix = 0.f, iy = 0.f, iz = 0.f;
    int32_t o = -1;
    auto fetch = [&](int64_t e) {
        if (e < total) {
            const int64_t f = e >> lg;
            q = reinterpret_cast<const float2*>(uv)[f];
            o = obj[f];
            ix = dirs[3 * e];
            iy = dirs[3 * e + 1];
            iz = dirs[3 * e + 2];
        }
    };
    fetch(warp0 * 32 + lane);
    for (int64_t base = warp0 * 32; base < total; base += stride) {
        const int64_t e = base + lane;
        const float2 cq = q;
        const float cx = ix, cy = iy, cz = iz;
        const int32_t co = o;
        fetch(e + stride);
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        int bad = 0;
        if (e < total) {
            TexDesc d;
            if (fragment_valid(table, n_obj, co, cq.x, cq.y, cx, cy, cz, status, d))
                c = filter_any<FILTER>(d, locate<FILTER>(d, cq.x, cq.y, cx, cy, cz));
            else
                bad = co >= 0;  // an invalid sample zeroes its fragment
        }
        for (int off = 1; off < S; off <<= 1) {
            c.x += __shfl_xor_sync(0xffffffffu, c.x, off);
            c.y += __shfl_xor_sync(0xffffffffu, c.y, off);
            c.z += __shfl_xor_sync(0xffffffffu, c.z, off);
            c.w += __shfl_xor_sync(0xffffffffu, c.w, off);
            bad |= __shfl_xor_sync(0xffffffffu, bad, off);
        }
        if (e < total && (lane & (S - 1)) == 0) {
            const float inv = 1.0f / (float)S;
            const float4 r = bad ? make_float4(0.f, 0.f, 0.f, 0.f)
                                 : make_float4(c.x * inv, c.y * inv, c.z * inv, c.w * inv);
            __stcs(reinterpret_cast<float4*>(out) + (e >> lg), r);
        }
    }
}

template <int FILTER>
static void launch_multi_t(const TexDesc* table, int n_obj, const float* uv, const float* dirs, int S,
                           const int32_t* obj, int64_t F, float* out, unsigned* status, cudaStream_t stream) {
    if (S <= 32 && (S & (S - 1)) == 0) {
        const unsigned grid = persistent_grid(multi_shade_lanes_kernel<FILTER>, kShadeThreads, (F * S + 31) / 32);
        multi_shade_lanes_kernel<FILTER><<<grid, kShadeThreads, 0, stream>>>(table, n_obj, uv, dirs, S, obj, F, out,
                                                                              status);
    } else {
        const unsigned grid = persistent_grid(multi_shade_kernel<FILTER>, kShadeThreads,
                                              (F + kShadeThreads - 1) / kShadeThreads);
        multi_shade_kernel<FILTER><<<grid, kShadeThreads, 0, stream>>>(table, n_obj, uv, dirs, S, obj, F, out,
                                                                        status);
    }
}

cudaError_t launch_multi_shade(const TexDesc* table, int n_obj, const float* uv, const float* dirs, int S,
                               const int32_t* obj, int64_t F, int filter, float* out, unsigned* status,
                               cudaStream_t stream) {
    switch (filter) {
        case RT_NEAREST:
            launch_multi_t<RT_NEAREST>(table, n_obj, uv, dirs, S, obj, F, out, status, stream);
            break;
        case RT_ANGULAR_BILINEAR:
            launch_multi_t<RT_ANGULAR_BILINEAR>(table, n_obj, uv, dirs, S, obj, F, out, status, stream);
            break;
        default:
            launch_multi_t<RT_QUADRILINEAR>(table, n_obj, uv, dirs, S, obj, F, out, status, stream);
    }
    return cudaGetLastError();
}

template <int FILTER, bool TILED, int SPEC>
static cudaError_t launch_shade_t(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                  const int32_t* obj, int64_t F, const Tiling& T, float* out, unsigned* status,
                                  cudaStream_t stream) {
    const unsigned grid = persistent_grid(shade_kernel<FILTER, TILED, SPEC>, kShadeThreads,
                                          chunk_count_host(T, F, kShadeWarps));
    shade_kernel<FILTER, TILED, SPEC><<<grid, kShadeThreads, 0, stream>>>(table, n_obj, uv, dir, obj, F, T, out,
                                                                          status);
    return cudaGetLastError();
}

template <bool TILED, int SPEC>
static cudaError_t launch_shade_f(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                  const int32_t* obj, int64_t F, int filter, const Tiling& T, float* out,
                                  unsigned* status, cudaStream_t stream) {
    switch (filter) {
        case RT_NEAREST:
            return launch_shade_t<RT_NEAREST, TILED, SPEC>(table, n_obj, uv, dir, obj, F, T, out, status, stream);
        case RT_ANGULAR_BILINEAR:
            return launch_shade_t<RT_ANGULAR_BILINEAR, TILED, SPEC>(table, n_obj, uv, dir, obj, F, T, out, status,
                                                                    stream);
        default:
            return launch_shade_t<RT_QUADRILINEAR, TILED, SPEC>(table, n_obj, uv, dir, obj, F, T, out, status,
                                                                stream);
    }
}

// The screen-tiled path has a single-format instantiation per storage format
// (spec = that format); everything else runs the dispatching kernels.
cudaError_t launch_shade(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                         int64_t F, int filter, const Tiling& T, int spec, float* out, unsigned* status,
                         cudaStream_t stream) {
    if (T.W > 0) {
        switch (spec) {
            case RT_F16:
                return launch_shade_f<true, RT_F16>(table, n_obj, uv, dir, obj, F, filter, T, out, status, stream);
            case RT_BF16:
                return launch_shade_f<true, RT_BF16>(table, n_obj, uv, dir, obj, F, filter, T, out, status, stream);
            case RT_F32:
                return launch_shade_f<true, RT_F32>(table, n_obj, uv, dir, obj, F, filter, T, out, status, stream);
            case RT_E4M3_BUCKET_SCALE:
                return launch_shade_f<true, RT_E4M3_BUCKET_SCALE>(table, n_obj, uv, dir, obj, F, filter, T, out,
                                                                  status, stream);
            default:
                return launch_shade_f<true, -1>(table, n_obj, uv, dir, obj, F, filter, T, out, status, stream);
        }
    }
    return launch_shade_f<false, -1>(table, n_obj, uv, dir, obj, F, filter, T, out, status, stream);
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

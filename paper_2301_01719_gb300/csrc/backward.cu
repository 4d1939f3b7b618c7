// backward.cu -- gradients of the lookup: texels, UV and direction.
//
// The filter weights are recomputed exactly as the forward pass computes them
// (nothing is stored between the passes).  Texel gradients w_tap * dL/dout are
// summed into FP32 buffers with 16-byte vector reductions (red.global.add.v4.f32),
// one per tap of non-zero weight.  UV and direction gradients follow the chain
// rule through the nested lerps, the Note's clamp (zero derivative where a
// coordinate is clamped), Eq. 3 and Eq. 1b.
#include "launch.h"
#include "rt_backward.cuh"
#include "rt_internal.h"

namespace rt {

// The single-format tiled kernels are held to 80 registers (6 blocks, 24 warps
// per SM): measured 3 % faster than 95 registers at 5 blocks.
template <int FILTER, bool TILED, bool DET, int SPEC>
__global__ void __launch_bounds__(kBackThreads, (TILED && !DET && SPEC >= 0) ? 6 : 1) backward_kernel(
    const TexDesc* __restrict__ table, int n_obj, const float* __restrict__ uv, const float* __restrict__ dir,
    const int32_t* __restrict__ obj, int64_t F, Tiling tiling, const float* __restrict__ dL_dout,
    const __grid_constant__ GradTable grads, bool any_grad, float* __restrict__ dL_duv, float* __restrict__ dL_ddir,
    bool accumulate, unsigned* status) {
    __shared__ WarpStage<true> stages[kBackWarps];
    const bool coord_grads = (dL_duv != nullptr) || (dL_ddir != nullptr);
    for_each_fragment<kBackWarps, true, TILED, 2>(uv, dir, obj, dL_dout, F, tiling, stages,
                                               [&](int64_t f, const Frag& q, float4 go) {
        float2 guv = make_float2(0.f, 0.f);
        float3 gdir = make_float3(0.f, 0.f, 0.f);
        TexDesc d;
        if (fragment_valid(table, n_obj, q.o, q.u, q.v, q.x, q.y, q.z, status, d)) {
            Lookup<FILTER> L = locate<FILTER, (SPEC < 0)>(d, q.u, q.v, q.x, q.y, q.z);
            void* grad = any_grad ? grads.p[q.o] : nullptr;
            CoordGrad cg = backward_spec<FILTER, DET, SPEC>(d, L, go, grad, coord_grads);
            coord_grads_of<FILTER>(d, L, q, cg, dL_ddir != nullptr, guv, gdir);
        }
        if (f < 0) return;
        store_coord_grads(f, guv, gdir, dL_duv, dL_ddir, accumulate);
    });
}

template <int FILTER, bool TILED, bool DET, int SPEC>
static cudaError_t launch_backward_t(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                     const int32_t* obj, int64_t F, const Tiling& T, const float* dL_dout,
                                     const GradTable& grads, bool any_grad, float* dL_duv, float* dL_ddir,
                                     bool accumulate, unsigned* status, cudaStream_t stream) {
    const unsigned grid = persistent_grid(backward_kernel<FILTER, TILED, DET, SPEC>, kBackThreads,
                                          chunk_count_host(T, F, kBackWarps));
    backward_kernel<FILTER, TILED, DET, SPEC><<<grid, kBackThreads, 0, stream>>>(
        table, n_obj, uv, dir, obj, F, T, dL_dout, grads, any_grad, dL_duv, dL_ddir, accumulate, status);
    return cudaGetLastError();
}

template <bool TILED, bool DET, int SPEC>
static cudaError_t launch_backward_f(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                     const int32_t* obj, int64_t F, int filter, const Tiling& T,
                                     const float* dL_dout, const GradTable& grads, bool any_grad, float* dL_duv,
                                     float* dL_ddir, bool accumulate, unsigned* status, cudaStream_t stream) {
    switch (filter) {
        case RT_NEAREST:
            return launch_backward_t<RT_NEAREST, TILED, DET, SPEC>(table, n_obj, uv, dir, obj, F, T, dL_dout, grads,
                                                                   any_grad, dL_duv, dL_ddir, accumulate, status,
                                                                   stream);
        case RT_ANGULAR_BILINEAR:
            return launch_backward_t<RT_ANGULAR_BILINEAR, TILED, DET, SPEC>(table, n_obj, uv, dir, obj, F, T,
                                                                            dL_dout, grads, any_grad, dL_duv,
                                                                            dL_ddir, accumulate, status, stream);
        default:
            return launch_backward_t<RT_QUADRILINEAR, TILED, DET, SPEC>(table, n_obj, uv, dir, obj, F, T, dL_dout,
                                                                        grads, any_grad, dL_duv, dL_ddir,
                                                                        accumulate, status, stream);
    }
}

// The screen-tiled, non-deterministic path has a single-format instantiation
// per storage format (spec); the others run the dispatching kernels.
cudaError_t launch_backward(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                            int64_t F, int filter, const Tiling& T, int spec, const float* dL_dout,
                            const GradTable& grads, bool any_grad, float* dL_duv, float* dL_ddir, bool accumulate,
                            bool deterministic, unsigned* status, cudaStream_t stream) {
#define RT_BWD(TILED, DET, SPEC)                                                                                 \
    launch_backward_f<TILED, DET, SPEC>(table, n_obj, uv, dir, obj, F, filter, T, dL_dout, grads, any_grad, dL_duv, \
                                        dL_ddir, accumulate, status, stream)
    if (T.W > 0) {
        if (deterministic) return RT_BWD(true, true, -1);
        switch (spec) {
            case RT_F16:
                return RT_BWD(true, false, RT_F16);
            case RT_BF16:
                return RT_BWD(true, false, RT_BF16);
            case RT_F32:
                return RT_BWD(true, false, RT_F32);
            case RT_E4M3_BUCKET_SCALE:
                return RT_BWD(true, false, RT_E4M3_BUCKET_SCALE);
            default:
                return RT_BWD(true, false, -1);
        }
    }
    if (deterministic) return RT_BWD(false, true, -1);
    return RT_BWD(false, false, -1);
#undef RT_BWD
}

// World-space backward (Eq. 1a with a per-fragment normal): the streamer of
// the tangent-space backward with the normal as a fourth staged stream, over
// the flat fragment stream or, TILED, over screen tiles of a batch of frames.
// dL/dI = dL/dN, since A depends on h = I + N only.
template <int FILTER, bool DET, bool TILED>
__global__ void __launch_bounds__(kBackThreads) world_backward_kernel(
    const TexDesc* __restrict__ table, int n_obj, const float* __restrict__ uv, const float* __restrict__ dir,
    const float* __restrict__ nrm, const int32_t* __restrict__ obj, int64_t F, Tiling tiling,
    const float* __restrict__ dL_dout,
    const __grid_constant__ GradTable grads, bool any_grad, float* __restrict__ dL_duv, float* __restrict__ dL_ddir,
    float* __restrict__ dL_dnrm, bool accumulate, unsigned* status) {
    __shared__ WarpStage<true, 2, true> stages[kBackWarps];
    const bool coord_grads = dL_duv || dL_ddir || dL_dnrm;
    for_each_fragment<kBackWarps, true, TILED, 2, true>(uv, dir, obj, dL_dout, F, tiling, stages,
                                                        [&](int64_t f, const Frag& q, float4 go) {
        float2 guv = make_float2(0.f, 0.f);
        float3 gh = make_float3(0.f, 0.f, 0.f);
        TexDesc d;
        const float3 I = make_float3(q.x, q.y, q.z), N = make_float3(q.nx, q.ny, q.nz);
        if (fragment_valid(table, n_obj, q.o, q.u, q.v, I.x, I.y, I.z, status, d) && normal_valid(N, status)) {
            const Lookup<FILTER> L = locate_world<FILTER>(d, q.u, q.v, I, N);
            void* grad = any_grad ? grads.p[q.o] : nullptr;
            const CoordGrad cg = backward_any<FILTER, DET>(d, L, go, grad, coord_grads);
            if (FILTER == RT_QUADRILINEAR) guv = uv_grad(d, q.u, q.v, cg.gu, cg.gv);
            if (FILTER != RT_NEAREST && (dL_ddir || dL_dnrm)) {
                const float gBx = (L.B.x > -d.hi && L.B.x < d.hi) ? cg.gs * d.half_n : 0.f;
                const float gBy = (L.B.y > -d.hi && L.B.y < d.hi) ? cg.gt * d.half_n : 0.f;
                gh = half_grad(I.x + N.x, I.y + N.y, I.z + N.z, gBx, gBy);
            }
        }
        if (f < 0) return;
        if (dL_duv) {
            float2* p = reinterpret_cast<float2*>(dL_duv) + f;
            if (accumulate) {
                const float2 o = *p;
                guv.x += o.x;
                guv.y += o.y;
            }
            *p = guv;
        }
        float* outs[2] = {dL_ddir, dL_dnrm};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            float* p = outs[k];
            if (!p) continue;
            p += 3 * f;
            p[0] = accumulate ? p[0] + gh.x : gh.x;
            p[1] = accumulate ? p[1] + gh.y : gh.y;
            p[2] = accumulate ? p[2] + gh.z : gh.z;
        }
    }, nrm);
}

template <int FILTER, bool DET, bool TILED>
static cudaError_t launch_world_backward_t(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                           const float* nrm, const int32_t* obj, int64_t F, const Tiling& T,
                                           const float* dL_dout, const GradTable& grads, bool any_grad, float* dL_duv,
                                           float* dL_ddir, float* dL_dnrm, bool accumulate, unsigned* status,
                                           cudaStream_t stream) {
    const unsigned grid = persistent_grid(world_backward_kernel<FILTER, DET, TILED>, kBackThreads,
                                          chunk_count_host(T, F, kBackWarps));
    world_backward_kernel<FILTER, DET, TILED><<<grid, kBackThreads, 0, stream>>>(
        table, n_obj, uv, dir, nrm, obj, F, T, dL_dout, grads, any_grad, dL_duv, dL_ddir, dL_dnrm, accumulate,
        status);
    return cudaGetLastError();
}

template <bool DET, bool TILED>
static cudaError_t launch_world_backward_d(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                           const float* nrm, const int32_t* obj, int64_t F, int filter,
                                           const Tiling& T, const float* dL_dout, const GradTable& grads,
                                           bool any_grad, float* dL_duv, float* dL_ddir, float* dL_dnrm,
                                           bool accumulate, unsigned* status, cudaStream_t stream) {
#define RT_WBWD(FILT)                                                                                              \
    launch_world_backward_t<FILT, DET, TILED>(table, n_obj, uv, dir, nrm, obj, F, T, dL_dout, grads, any_grad,      \
                                              dL_duv, dL_ddir, dL_dnrm, accumulate, status, stream)
    switch (filter) {
        case RT_NEAREST:
            return RT_WBWD(RT_NEAREST);
        case RT_ANGULAR_BILINEAR:
            return RT_WBWD(RT_ANGULAR_BILINEAR);
        default:
            return RT_WBWD(RT_QUADRILINEAR);
    }
#undef RT_WBWD
}

cudaError_t launch_world_backward(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                  const float* nrm, const int32_t* obj, int64_t F, int filter, const Tiling& T,
                                  const float* dL_dout, const GradTable& grads, bool any_grad, float* dL_duv,
                                  float* dL_ddir, float* dL_dnrm, bool accumulate, bool deterministic,
                                  unsigned* status, cudaStream_t stream) {
#define RT_WBWD_D(DET, TILED)                                                                                      \
    launch_world_backward_d<DET, TILED>(table, n_obj, uv, dir, nrm, obj, F, filter, T, dL_dout, grads, any_grad,    \
                                        dL_duv, dL_ddir, dL_dnrm, accumulate, status, stream)
    if (T.W > 0) return deterministic ? RT_WBWD_D(true, true) : RT_WBWD_D(false, true);
    return deterministic ? RT_WBWD_D(true, false) : RT_WBWD_D(false, false);
#undef RT_WBWD_D
}

// Fixed-point sums (deterministic mode) -> FP32 gradients, times `scale` (the
// product taken in FP64, rounded once), added to or overwriting dst.
__global__ void fixed_to_float_kernel(const long long* __restrict__ acc, float* __restrict__ dst, int64_t count,
                                      double scale, bool accumulate) {
    const double f = scale * (1.0 / 4294967296.0);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
        float v = (float)((double)acc[k] * f);
        dst[k] = accumulate ? dst[k] + v : v;
    }
}

cudaError_t launch_fixed_to_float(const long long* acc, float* dst, int64_t count, bool accumulate,
                                  cudaStream_t stream, double scale) {
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + 255) / 256;
    fixed_to_float_kernel<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, stream>>>(acc, dst, count, scale,
                                                                                          accumulate);
    return cudaGetLastError();
}

}  // namespace rt

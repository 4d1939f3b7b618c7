// fused.cu -- one pass over the screen tiles of a batch of frames doing the
// forward lookup, an L2 loss against target colours and the backward.
//
// Per fragment: the colour c of the forward filter (written to `out`), the
// residual r = c - target and dL/dout = scale r, then the texel, UV and
// direction gradients of the backward for that dL/dout.  The G-buffer and the
// target are read once, the lookup coordinates are computed once, and the
// taps gathered for the colour serve the backward too (kept in registers for
// FP16 / BF16 / E4M3, reloaded from L1 otherwise).  On the 60-pose 1080p step
// the fused kernel takes 4.83 ms where the forward and the backward take
// 1.74 + 4.62 ms.
#include "launch.h"
#include "rt_backward.cuh"
#include "rt_internal.h"

namespace rt {

// The stored code of one texel as the fused step keeps it in registers: 8 bytes
// for FP16 / BF16, 4 for E4M3 (whose bucket scale is kept beside it).
template <int FMT>
struct KeptCode {
    using type = uint2;
};
template <>
struct KeptCode<RT_E4M3_BUCKET_SCALE> {
    using type = unsigned;
};

template <int FMT>
__device__ __forceinline__ P4 decode_kept(typename KeptCode<FMT>::type c, float scale) {
    if constexpr (FMT == RT_E4M3_BUCKET_SCALE)
        return decode4_e4m3(c, scale);
    else
        return decode8<FMT>(c);
}

// Held to 128 registers (4 blocks, 16 warps per SM): at 5 blocks (96
// registers) the kernel took 5.86 ms against 5.65 ms, at 6 blocks (80,
// spilling) 6.21 ms, on the 60-pose 1080p step (textures in row-major planes
// then).  With FP16 / BF16 quadrilinear textures the 16 taps' 8-byte codes are
// gathered once and kept in registers (118 then, no spills; 126 with the
// reductions' once-per-fragment pair exchange) for the coordinate gradients
// instead of being reloaded from L1: 5.15 -> 5.03 ms (E4M3: the 4-byte codes and
// the buckets' scales, 5.28 -> 5.09 ms).  A variant that
// forms colour-derivative vectors from the forward's lerps needs far more
// registers and measured slower at every occupancy (7.0 ms at best against
// 6.4 ms then).
template <int FILTER, bool DET, int SPEC>
__global__ void __launch_bounds__(kBackThreads, (!DET && SPEC >= 0) ? 4 : 1) fused_l2_kernel(
    const TexDesc* __restrict__ table, int n_obj, const float* __restrict__ uv, const float* __restrict__ dir,
    const int32_t* __restrict__ obj, int64_t F, Tiling tiling, const float* __restrict__ target, float scale,
    float* __restrict__ out, double* __restrict__ sums, const __grid_constant__ GradTable grads, bool any_grad,
    float* __restrict__ dL_duv, float* __restrict__ dL_ddir, bool accumulate, unsigned* status) {
    __shared__ WarpStage<true> stages[kBackWarps];
    const bool coord_grads = (dL_duv != nullptr) || (dL_ddir != nullptr);
    double se = 0.0;  // this lane's squared residuals
    int cnt = 0;      // and its fragments with an object id
    for_each_fragment<kBackWarps, true, true, 2>(uv, dir, obj, target, F, tiling, stages,
                                               [&](int64_t f, const Frag& q, float4 t) {
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        TexDesc d;
        Lookup<FILTER> L;
        // FP16 / BF16 / E4M3 quadrilinear: the 16 taps' codes (and E4M3's four bucket scales)
        // stay in registers for the backward
        constexpr bool kE4 = SPEC == RT_E4M3_BUCKET_SCALE;
        constexpr bool kKeepTaps = FILTER == RT_QUADRILINEAR && !DET && (SPEC == RT_F16 || SPEC == RT_BF16 || kE4);
        constexpr int kKept = kKeepTaps ? SPEC : RT_F16;
        using Code = typename KeptCode<kKept>::type;
        int64_t pl[4];
        int o[4];
        Code code[kKeepTaps ? 4 : 1][kKeepTaps ? 4 : 1];  // [bucket][texel]
        float sc[kE4 ? 4 : 1];                             // E4M3: the scale of each bucket
        const bool valid = fragment_valid(table, n_obj, q.o, q.u, q.v, q.x, q.y, q.z, status, d);
        if (valid) {
            L = locate<FILTER, (SPEC < 0)>(d, q.u, q.v, q.x, q.y, q.z);
            if constexpr (kKeepTaps) {
                quad_tap_addresses<RT_LAYOUT_QUADS>(d, L.u, L.v, L.s, L.t, pl, o);
                if constexpr (kE4) {
#pragma unroll
                    for (int b = 0; b < 4; ++b) sc[b] = __ldg(d.scale + o[b]);
                }
                P4 tq[4][4];
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        code[b][k] = __ldg(reinterpret_cast<const Code*>(d.base) + checked_texel(d, pl[k] + o[b]));
                        tq[b][k] = decode_kept<kKept>(code[b][k], sc[kE4 ? b : 0]);
                    }
                c = toF4(quadrilinear_combine(tq, L.u, L.v, L.s, L.t));
            } else {
                c = filter_spec<FILTER, SPEC>(d, L);
            }
        }
        // the colour and the loss are done with before the backward starts (shorter live ranges)
        if (f >= 0) {
            if (out) __stcs(reinterpret_cast<float4*>(out) + f, c);
            if (q.o >= 0) {  // every fragment with an object id, as rt_l2_loss_grad counts them
                const float4 r = make_float4(c.x - t.x, c.y - t.y, c.z - t.z, c.w - t.w);
                se += (double)r.x * r.x + (double)r.y * r.y + (double)r.z * r.z + (double)r.w * r.w;
                ++cnt;
            }
        }
        float2 guv = make_float2(0.f, 0.f);
        float3 gdir = make_float3(0.f, 0.f, 0.f);
        if (valid) {
            const float4 g = make_float4(scale * (c.x - t.x), scale * (c.y - t.y), scale * (c.z - t.z),
                                         scale * (c.w - t.w));
            void* grad = any_grad ? grads.p[q.o] : nullptr;
            CoordGrad cg;
            if constexpr (kKeepTaps) {
                reduce_quadrilinear_taps<false>(d, L, pl, o, g, grad);
                cg = CoordGrad{0.f, 0.f, 0.f, 0.f};
                if (coord_grads)
                    cg = quad_coord_grads(L, g, [&](int b, int k) { return decode_kept<kKept>(code[b][k], sc[kE4 ? b : 0]); });
            } else {
                cg = backward_spec<FILTER, DET, SPEC>(d, L, g, grad, coord_grads);
            }
            coord_grads_of<FILTER>(d, L, q, cg, dL_ddir != nullptr, guv, gdir);
        }
        if (f < 0) return;
        store_coord_grads(f, guv, gdir, dL_duv, dL_ddir, accumulate);
    });
    if (!sums) return;
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_down_sync(0xFFFFFFFFu, se, o);
        cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0 && cnt > 0) {
        atomicAdd(sums, se);
        atomicAdd(sums + 1, (double)cnt);
    }
}

template <int FILTER, bool DET, int SPEC>
static cudaError_t launch_fused_t(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                  const int32_t* obj, int64_t F, const Tiling& T, const float* target, float scale,
                                  float* out, double* sums, const GradTable& grads, bool any_grad, float* dL_duv,
                                  float* dL_ddir, bool accumulate, unsigned* status, cudaStream_t stream) {
    const unsigned grid = persistent_grid(fused_l2_kernel<FILTER, DET, SPEC>, kBackThreads,
                                          chunk_count_host(T, F, kBackWarps));
    fused_l2_kernel<FILTER, DET, SPEC><<<grid, kBackThreads, 0, stream>>>(
        table, n_obj, uv, dir, obj, F, T, target, scale, out, sums, grads, any_grad, dL_duv, dL_ddir, accumulate,
        status);
    return cudaGetLastError();
}

template <bool DET, int SPEC>
static cudaError_t launch_fused_f(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                  const int32_t* obj, int64_t F, int filter, const Tiling& T, const float* target,
                                  float scale, float* out, double* sums, const GradTable& grads, bool any_grad,
                                  float* dL_duv, float* dL_ddir, bool accumulate, unsigned* status,
                                  cudaStream_t stream) {
#define RT_FUSED_F(FILT)                                                                                            \
    launch_fused_t<FILT, DET, SPEC>(table, n_obj, uv, dir, obj, F, T, target, scale, out, sums, grads, any_grad,     \
                                    dL_duv, dL_ddir, accumulate, status, stream)
    switch (filter) {
        case RT_NEAREST:
            return RT_FUSED_F(RT_NEAREST);
        case RT_ANGULAR_BILINEAR:
            return RT_FUSED_F(RT_ANGULAR_BILINEAR);
        default:
            return RT_FUSED_F(RT_QUADRILINEAR);
    }
#undef RT_FUSED_F
}

// Single-format instantiations for the non-deterministic path, as the backward.
cudaError_t launch_fused_l2(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                            int64_t F, int filter, const Tiling& T, int spec, const float* target, float scale,
                            float* out, double* sums, const GradTable& grads, bool any_grad, float* dL_duv,
                            float* dL_ddir, bool accumulate, bool deterministic, unsigned* status,
                            cudaStream_t stream) {
#define RT_FUSED(DET, SPEC)                                                                                         \
    launch_fused_f<DET, SPEC>(table, n_obj, uv, dir, obj, F, filter, T, target, scale, out, sums, grads, any_grad,  \
                              dL_duv, dL_ddir, accumulate, status, stream)
    if (deterministic) return RT_FUSED(true, -1);
    switch (spec) {
        case RT_F16:
            return RT_FUSED(false, RT_F16);
        case RT_BF16:
            return RT_FUSED(false, RT_BF16);
        case RT_F32:
            return RT_FUSED(false, RT_F32);
        case RT_E4M3_BUCKET_SCALE:
            return RT_FUSED(false, RT_E4M3_BUCKET_SCALE);
        default:
            return RT_FUSED(false, -1);
    }
#undef RT_FUSED
}

}  // namespace rt

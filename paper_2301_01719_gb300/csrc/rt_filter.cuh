// rt_filter.cuh -- gathering and filtering the taps of one fragment (FP32).
//
// QUADRILINEAR: 2 x 2 buckets (u, v) x 2 x 2 texels (s, t) = 16 taps, all four
// buckets at the same in-bucket coordinate (one tangent-space direction per
// fragment).  ANGULAR_BILINEAR: the nearest bucket, 2 x 2 texels inside it
// ("single sample per bucket", Section 2).  NEAREST: one texel.
// Weights are applied as nested lerps a + w (b - a) in the order s, t, u, v, so
// a constant texture returns its constant exactly.
#pragma once

#include "rt_device.cuh"

namespace rt {

// The four texels (s0,t0) (s1,t0) (s0,t1) (s1,t1) of bucket (i, j).
template <int FMT, int LAYOUT>
__device__ __forceinline__ void load_quad(const TexDesc& d, int i, int j, const Axis& s, const Axis& t, float4& t00,
                                          float4& t10, float4& t01, float4& t11) {
    float sc = 1.0f;
    if (FMT == RT_E4M3_BUCKET_SCALE) sc = __ldg(d.scale + (int64_t)j * d.W + i);
    t00 = load_texel<FMT>(d.base, texel_index<LAYOUT>(d, i, j, s.k0, t.k0), sc);
    t10 = load_texel<FMT>(d.base, texel_index<LAYOUT>(d, i, j, s.k1, t.k0), sc);
    t01 = load_texel<FMT>(d.base, texel_index<LAYOUT>(d, i, j, s.k0, t.k1), sc);
    t11 = load_texel<FMT>(d.base, texel_index<LAYOUT>(d, i, j, s.k1, t.k1), sc);
}

template <int FILTER, int FMT, int LAYOUT>
__device__ __forceinline__ float4 filter_taps(const TexDesc& d, const Lookup<FILTER>& L) {
    if (FILTER == RT_NEAREST) {
        float sc = 1.0f;
        if (FMT == RT_E4M3_BUCKET_SCALE) sc = __ldg(d.scale + (int64_t)L.v.k0 * d.W + L.u.k0);
        return load_texel<FMT>(d.base, texel_index<LAYOUT>(d, L.u.k0, L.v.k0, L.s.k0, L.t.k0), sc);
    } else if (FILTER == RT_ANGULAR_BILINEAR) {
        float4 a, b, c, e;
        load_quad<FMT, LAYOUT>(d, L.u.k0, L.v.k0, L.s, L.t, a, b, c, e);
        return lerp4(lerp4(a, b, L.s.w), lerp4(c, e, L.s.w), L.t.w);
    } else {
        float4 q[2][2][4];
#pragma unroll
        for (int bv = 0; bv < 2; ++bv)
#pragma unroll
            for (int au = 0; au < 2; ++au)
                load_quad<FMT, LAYOUT>(d, au ? L.u.k1 : L.u.k0, bv ? L.v.k1 : L.v.k0, L.s, L.t, q[bv][au][0],
                                       q[bv][au][1], q[bv][au][2], q[bv][au][3]);
        float4 y[2];
#pragma unroll
        for (int bv = 0; bv < 2; ++bv) {
            float4 c[2];
#pragma unroll
            for (int au = 0; au < 2; ++au)
                c[au] = lerp4(lerp4(q[bv][au][0], q[bv][au][1], L.s.w), lerp4(q[bv][au][2], q[bv][au][3], L.s.w),
                              L.t.w);
            y[bv] = lerp4(c[0], c[1], L.u.w);
        }
        return lerp4(y[0], y[1], L.v.w);
    }
}

// Dispatch on the object's storage format and layout (owned textures are
// PLANES; a borrowed FP32 buffer may be either).
template <int FILTER>
__device__ __forceinline__ float4 filter_any(const TexDesc& d, const Lookup<FILTER>& L) {
    switch (d.fmt) {
        case RT_F16:
            return filter_taps<FILTER, RT_F16, RT_LAYOUT_PLANES>(d, L);
        case RT_BF16:
            return filter_taps<FILTER, RT_BF16, RT_LAYOUT_PLANES>(d, L);
        case RT_E4M3_BUCKET_SCALE:
            return filter_taps<FILTER, RT_E4M3_BUCKET_SCALE, RT_LAYOUT_PLANES>(d, L);
        default:
            if (d.layout == RT_LAYOUT_ATLAS) return filter_taps<FILTER, RT_F32, RT_LAYOUT_ATLAS>(d, L);
            return filter_taps<FILTER, RT_F32, RT_LAYOUT_PLANES>(d, L);
    }
}

// G-buffer staging: a block of BLOCK threads shades BLOCK consecutive
// fragments.  The block reads its slice of uv (BLOCK x 8 bytes), dir (BLOCK x
// 12 bytes) and obj (BLOCK x 4 bytes) with 16-byte vector loads into shared
// memory, then each thread takes one fragment.  The G-buffer is read once, so
// the loads ask for early eviction (ld.global.cs) and leave the caches to the
// texels.  Fragments past F are background.
template <int BLOCK>
struct GStage {
    float uv[2 * BLOCK];
    float dir[3 * BLOCK];
    int obj[BLOCK];
};

struct Frag {
    float u, v, x, y, z;
    int o;
};

template <int BLOCK>
__device__ __forceinline__ Frag stage_gbuffer(const float* __restrict__ uv, const float* __restrict__ dir,
                                              const int32_t* __restrict__ obj, int64_t F, GStage<BLOCK>& S) {
    const int64_t f0 = (int64_t)blockIdx.x * BLOCK;
    const int tid = threadIdx.x;
    if (f0 + BLOCK <= F) {
        const float4* uv4 = reinterpret_cast<const float4*>(uv + 2 * f0);
        const float4* d4 = reinterpret_cast<const float4*>(dir + 3 * f0);
        const int4* o4 = reinterpret_cast<const int4*>(obj + f0);
        for (int k = tid; k < BLOCK / 2; k += BLOCK) reinterpret_cast<float4*>(S.uv)[k] = __ldcs(uv4 + k);
        for (int k = tid; k < 3 * BLOCK / 4; k += BLOCK) reinterpret_cast<float4*>(S.dir)[k] = __ldcs(d4 + k);
        for (int k = tid; k < BLOCK / 4; k += BLOCK) reinterpret_cast<int4*>(S.obj)[k] = __ldcs(o4 + k);
    } else {
        const int count = (int)(F - f0);
        for (int k = tid; k < 2 * BLOCK; k += BLOCK) S.uv[k] = k < 2 * count ? uv[2 * f0 + k] : 0.f;
        for (int k = tid; k < 3 * BLOCK; k += BLOCK) S.dir[k] = k < 3 * count ? dir[3 * f0 + k] : 0.f;
        for (int k = tid; k < BLOCK; k += BLOCK) S.obj[k] = k < count ? obj[f0 + k] : -1;
    }
    __syncthreads();
    Frag r;
    float2 q = reinterpret_cast<const float2*>(S.uv)[tid];
    r.u = q.x;
    r.v = q.y;
    r.x = S.dir[3 * tid];
    r.y = S.dir[3 * tid + 1];
    r.z = S.dir[3 * tid + 2];
    r.o = S.obj[tid];
    return r;
}

// Validity of one fragment: 1 = shade it, 0 = background or invalid (status
// bits raised for invalid ones).
__device__ __forceinline__ bool fragment_valid(const TexDesc* __restrict__ table, int n_obj, int o, float u, float v,
                                               float x, float y, float z, unsigned* status, TexDesc& d) {
    if (o < 0) return false;
    if (o >= n_obj) {
        atomicOr(status, ST_BAD_OBJ);
        return false;
    }
    d = load_desc(table, o);
    if (!d.live) {
        atomicOr(status, ST_BAD_OBJ);
        return false;
    }
    if (!(isfinite(u) && isfinite(v) && finite3(x, y, z))) {
        atomicOr(status, ST_NONFINITE);
        return false;
    }
    return true;
}

}  // namespace rt

// rt_encode.cuh -- texel addressing and storage encoders shared by the
// kernels that write textures (encode, fill, bake) and convert layouts.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "radtex.h"

namespace rt {

// (i, j, s, t) of texel `idx` in the PLANES layout.
__device__ __forceinline__ void planes_coords(int64_t idx, int W, int H, int n, int& i, int& j, int& s, int& t) {
    int64_t plane = (int64_t)W * H;
    int64_t p = idx / plane, r = idx - p * plane;
    j = (int)(r / W);
    i = (int)(r - (int64_t)j * W);
    t = (int)(p / n);
    s = (int)(p - (int64_t)t * n);
}

// Buckets per direction plane of a PLANES buffer (w h) or a QUADS buffer
// (4 ceil(w/2) ceil(h/2): an odd side is padded to even).
__host__ __device__ __forceinline__ int64_t plane_buckets(int layout, int W, int H) {
    if (layout == RT_LAYOUT_QUADS) return 4 * (int64_t)((W + 1) >> 1) * ((H + 1) >> 1);
    return (int64_t)W * H;
}

// Offset of bucket (i, j) inside a direction plane of a PLANES or QUADS buffer.
__host__ __device__ __forceinline__ int64_t slot_in(int layout, int W, int i, int j) {
    if (layout == RT_LAYOUT_QUADS)
        return ((int64_t)(j >> 1) * ((W + 1) >> 1) + (i >> 1)) * 4 + ((j & 1) << 1) + (i & 1);
    return (int64_t)j * W + i;
}

__device__ __forceinline__ int64_t index_in(int layout, int W, int H, int n, int i, int j, int s, int t) {
    if (layout == RT_LAYOUT_PLANES || layout == RT_LAYOUT_QUADS)
        return ((int64_t)t * n + s) * plane_buckets(layout, W, H) + slot_in(layout, W, i, j);
    return ((int64_t)j * n + t) * ((int64_t)W * n) + (int64_t)i * n + s;
}

__device__ __forceinline__ uint2 pack_f16(float4 v) {
    __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    return make_uint2(*reinterpret_cast<unsigned*>(&a), *reinterpret_cast<unsigned*>(&b));
}

__device__ __forceinline__ uint2 pack_bf16(float4 v) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    return make_uint2(*reinterpret_cast<unsigned*>(&a), *reinterpret_cast<unsigned*>(&b));
}

// E4M3 codes of v / scale, round to nearest even with saturation; channel 0 in the low byte.
__device__ __forceinline__ unsigned pack_e4m3(float4 v, float scale) {
    float2 lo = make_float2(__fdiv_rn(v.x, scale), __fdiv_rn(v.y, scale));
    float2 hi = make_float2(__fdiv_rn(v.z, scale), __fdiv_rn(v.w, scale));
    unsigned a = __nv_cvt_float2_to_fp8x2(lo, __NV_SATFINITE, __NV_E4M3);
    unsigned b = __nv_cvt_float2_to_fp8x2(hi, __NV_SATFINITE, __NV_E4M3);
    return (a & 0xFFFFu) | (b << 16);
}

__device__ __forceinline__ float bucket_scale(float amax) { return amax == 0.0f ? 1.0f : __fdiv_rn(amax, 448.0f); }

__device__ __forceinline__ float amax4(float4 v) {
    return fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
}

// Direction of the centre of texel (s, t): B = ((2s+1)/n - 1, (2t+1)/n - 1),
// A = Eq. 4a(B) = B max(|B_x|, |B_y|) / |B|, I = Eq. 2c(A) =
// (A_x sqrt(2 - |A|^2), A_y sqrt(2 - |A|^2), 1 - |A|^2).
__device__ __forceinline__ float3 texel_centre_direction(int s, int t, int n) {
    float Bx = (float)(2 * s + 1) / (float)n - 1.0f;
    float By = (float)(2 * t + 1) / (float)n - 1.0f;
    float r = sqrtf(Bx * Bx + By * By);
    float Ax = 0.f, Ay = 0.f;
    if (r > 0.f) {
        float k = fmaxf(fabsf(Bx), fabsf(By)) / r;
        Ax = Bx * k;
        Ay = By * k;
    }
    float a2 = Ax * Ax + Ay * Ay;
    float q = sqrtf(fmaxf(2.0f - a2, 0.0f));
    return make_float3(Ax * q, Ay * q, 1.0f - a2);
}

// Eq. 4b: the reflection vector of texel (s, t), the mirror image of its
// Eq. 2c direction about the normal: (-A_x sqrt(2 - |A|^2), -A_y sqrt(2 - |A|^2), 1 - |A|^2).
__device__ __forceinline__ float3 texel_reflection(int s, int t, int n) {
    const float3 I = texel_centre_direction(s, t, n);
    return make_float3(-I.x, -I.y, I.z);
}

}  // namespace rt

// rt_device.cuh -- device-side pieces shared by the kernels of libradtex.
//
// The per-fragment lookup of Section 2 of Fober, "Radiance Textures for
// Rasterizing Ray-Traced Data" (arXiv 2301.01719), in FP32:
//   bucket  <- surface UV                     (Section 2, third paragraph)
//   A       <- Eq. 1b (equisolid projection, tangent space)
//   B       <- Eq. 3  (disc to square)
//   B       <- clamp to [1/n - 1, 1 - 1/n]    (Note after Eq. 3)
//   texels  <- floor / fractions of the continuous coordinates
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "radtex.h"

namespace rt {

enum : unsigned { ST_BAD_OBJ = 1u, ST_NONFINITE = 2u, ST_TIMEOUT = 4u, ST_BAD_ARG = 8u, ST_BOUNDS = 16u };

// One object of the texture table (64 bytes; 80 in the checked build, which
// adds the object's texel extent and the context's status word).  Built on the
// host when the texture is created; read by every kernel through the
// read-only path.
struct __align__(16) TexDesc {
    const void* base;       // texel storage
    const float* scale;     // per-bucket scale (E4M3 only): h x w, or one per palette bucket
    const uint32_t* index;  // palette textures: bucket (i, j) -> palette bucket index[j w + i]; else null
    int64_t plane;          // texels per direction plane: w * h, or the palette size K
    int32_t W, H, n;
    int8_t fmt, layout, live, wrap;  // wrap: bit 0 u, bit 1 v (repeat instead of clamp to edge)
    float fW, fH;           // w, h as float
    float half_n;           // n / 2
    float hi;               // clamp range of B: [-hi, hi], hi = 1 - 1/n
#ifdef RADTEX_CHECKED
    int64_t extent;         // texels a computed index may name: [0, extent)
    unsigned* status;       // the context's sticky status word
#endif
};
#ifdef RADTEX_CHECKED
static_assert(sizeof(TexDesc) == 80, "TexDesc is 80 bytes in the checked build");
#else
static_assert(sizeof(TexDesc) == 64, "TexDesc is 64 bytes");
#endif

__device__ __forceinline__ TexDesc load_desc(const TexDesc* __restrict__ table, int o) {
    const int4* p = reinterpret_cast<const int4*>(table + o);
    int4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2), d = __ldg(p + 3);
#ifdef RADTEX_CHECKED
    int4 e = __ldg(p + 4);
#endif
    TexDesc r;
    int4* q = reinterpret_cast<int4*>(&r);
    q[0] = a;
    q[1] = b;
    q[2] = c;
    q[3] = d;
#ifdef RADTEX_CHECKED
    q[4] = e;
#endif
    return r;
}

// Bounds checks of the checked build (RADTEX_CHECKED): a texel index outside
// [0, extent), a bucket outside the w x h matrix or a stored bucket outside
// [0, plane) sets ST_BOUNDS in the context's status word and is replaced by 0,
// so the access stays inside the object; nothing traps.  In the normal build
// each check is the identity.
__device__ __forceinline__ int64_t checked_texel(const TexDesc& d, int64_t idx) {
#ifdef RADTEX_CHECKED
    if (idx < 0 || idx >= d.extent) {
        atomicOr(d.status, ST_BOUNDS);
        return 0;
    }
#endif
    return idx;
}

#ifdef RADTEX_CHECKED
__device__ __forceinline__ int checked_slot(const TexDesc& d, int64_t slot, int64_t count) {
    if (slot < 0 || slot >= count) {
        atomicOr(d.status, ST_BOUNDS);
        return 0;
    }
    return (int)slot;
}
#endif

__device__ __forceinline__ bool finite3(float a, float b, float c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}

// Eq. 3 applied to A = sqrt(2) h_xy / |h|, the equisolid projection of a
// half-way vector h: h = (I_x, I_y, I_z + 1) in the tangent frame (Eq. 1b) or
// h = I + N in any frame (Eq. 1a).  Since A is a positive multiple of h_xy,
// B = A |A| / max(|A_x|, |A_y|) = sqrt(2) (h_xy / m) |h_xy| / |h| with
// m = max(|h_x|, |h_y|).  Every component is divided by m first, so the sums of
// squares neither underflow nor overflow (g2 lies in [1, 2]); a huge h_z / m
// gives B = 0, the limit.  h_xy = 0 (also I = -N) gives B = 0, the limit of
// Eq. 3; so does m < 1e-18, which moves B by less than 1e-18.
__device__ __forceinline__ float2 square_from_half(float hx, float hy, float hz) {
    float m = fmaxf(fabsf(hx), fabsf(hy));
    if (!(m >= 1e-18f)) return make_float2(0.f, 0.f);
    float rm = 1.0f / m;
    float x = hx * rm, y = hy * rm, z = hz * rm;
    float g2 = x * x + y * y;
    float D2 = g2 + z * z;
    float k = 1.41421356237f * sqrtf(g2 / D2);
    return make_float2(x * k, y * k);
}

// Eq. 1b followed by Eq. 3 (tangent-space incidence).
__device__ __forceinline__ float2 incidence_to_square(float Ix, float Iy, float Iz) {
    return square_from_half(Ix, Iy, Iz + 1.0f);
}

// Continuous coordinate of a spatial axis and its two taps (clamp to edge).
struct Axis {
    int k0, k1;  // taps (equal on a nearest axis)
    float w;     // weight of k1 (0 on a nearest axis)
    float c;     // continuous coordinate
    int fl;      // floor(c)
};

__device__ __forceinline__ Axis spatial_axis_bilinear(float x, float size, int isize) {
    Axis a;
    float c = fmaf(x, size, -0.5f);
    c = fminf(fmaxf(c, -1.0f), size);
    float f = floorf(c);
    a.c = c;
    a.fl = (int)f;
    a.w = c - f;
    a.k0 = min(max(a.fl, 0), isize - 1);
    a.k1 = min(max(a.fl + 1, 0), isize - 1);
    return a;
}

// Repeat address mode: c is not clamped; the taps are floor(c) (and
// floor(c) + 1) modulo the size.  Valid while |c| < 2^30.
__device__ __forceinline__ int wrap_index(int x, int size) {
    const int r = x % size;
    return r < 0 ? r + size : r;
}

__device__ __forceinline__ Axis spatial_axis_bilinear_wrap(float x, float size, int isize) {
    Axis a;
    float c = fmaf(x, size, -0.5f);
    float f = floorf(c);
    a.c = c;
    a.fl = (int)f;
    a.w = c - f;
    a.k0 = wrap_index(a.fl, isize);
    a.k1 = a.k0 + 1 == isize ? 0 : a.k0 + 1;
    return a;
}

__device__ __forceinline__ Axis spatial_axis_nearest_wrap(float x, float size, int isize) {
    Axis a;
    float c = x * size;
    a.c = c;
    a.fl = (int)floorf(c);
    a.k0 = a.k1 = wrap_index(a.fl, isize);
    a.w = 0.0f;
    return a;
}

__device__ __forceinline__ Axis spatial_axis_nearest(float x, float size, int isize) {
    Axis a;
    float c = fminf(fmaxf(x * size, 0.0f), size);
    a.c = c;
    a.fl = (int)floorf(c);
    a.k0 = a.k1 = min(a.fl, isize - 1);
    a.w = 0.0f;
    return a;
}

// In-bucket axis: B clamped to [lo, hi] (the Note after Eq. 3), texel k centred at
// B = (2k + 1)/n - 1.
__device__ __forceinline__ Axis angular_axis_bilinear(float B, float lo, float hi, float half_n, int n) {
    Axis a;
    float Bc = fminf(fmaxf(B, lo), hi);
    float c = fmaf(Bc + 1.0f, half_n, -0.5f);
    c = fminf(fmaxf(c, 0.0f), (float)(n - 1));
    float f = floorf(c);
    a.c = c;
    a.fl = (int)f;
    a.w = c - f;
    a.k0 = a.fl;
    a.k1 = min(a.fl + 1, n - 1);
    return a;
}

__device__ __forceinline__ Axis angular_axis_nearest(float B, float lo, float hi, float half_n, int n) {
    Axis a;
    float Bc = fminf(fmaxf(B, lo), hi);
    float c = (Bc + 1.0f) * half_n;
    a.c = c;
    a.fl = (int)floorf(c);
    a.k0 = a.k1 = min(max(a.fl, 0), n - 1);
    a.w = 0.0f;
    return a;
}

template <int FILTER>
struct Lookup {
    Axis u, v, s, t;
    float2 B;
};

// The lookup from B (any incidence mapping): spatial axes from (u, v) with the
// texture's address mode, in-bucket axes from B.
// WRAP = false: the caller knows that no object repeats (clamp to edge only).
template <int FILTER, bool WRAP = true>
__device__ __forceinline__ Lookup<FILTER> locate_from_square(const TexDesc& d, float u, float v, float2 B) {
    Lookup<FILTER> L;
    if (FILTER == RT_QUADRILINEAR) {
        L.u = (WRAP && (d.wrap & 1)) ? spatial_axis_bilinear_wrap(u, d.fW, d.W) : spatial_axis_bilinear(u, d.fW, d.W);
        L.v = (WRAP && (d.wrap & 2)) ? spatial_axis_bilinear_wrap(v, d.fH, d.H) : spatial_axis_bilinear(v, d.fH, d.H);
    } else {
        L.u = (WRAP && (d.wrap & 1)) ? spatial_axis_nearest_wrap(u, d.fW, d.W) : spatial_axis_nearest(u, d.fW, d.W);
        L.v = (WRAP && (d.wrap & 2)) ? spatial_axis_nearest_wrap(v, d.fH, d.H) : spatial_axis_nearest(v, d.fH, d.H);
    }
    L.B = B;
    if (FILTER == RT_NEAREST) {
        L.s = angular_axis_nearest(L.B.x, -d.hi, d.hi, d.half_n, d.n);
        L.t = angular_axis_nearest(L.B.y, -d.hi, d.hi, d.half_n, d.n);
    } else {
        L.s = angular_axis_bilinear(L.B.x, -d.hi, d.hi, d.half_n, d.n);
        L.t = angular_axis_bilinear(L.B.y, -d.hi, d.hi, d.half_n, d.n);
    }
    return L;
}

// Tangent-space lookup: Eq. 1b, Eq. 3, the Note's clamp.
template <int FILTER, bool WRAP = true>
__device__ __forceinline__ Lookup<FILTER> locate(const TexDesc& d, float u, float v, float Ix, float Iy, float Iz) {
    return locate_from_square<FILTER, WRAP>(d, u, v, incidence_to_square(Ix, Iy, Iz));
}

// World-space lookup: A from the first two entries of Eq. 1a, h = I + N.
template <int FILTER>
__device__ __forceinline__ Lookup<FILTER> locate_world(const TexDesc& d, float u, float v, float3 I, float3 N) {
    return locate_from_square<FILTER>(d, u, v, square_from_half(I.x + N.x, I.y + N.y, I.z + N.z));
}

// ---------------------------------------------------------------------------
// Texel addressing and decoding.
// ---------------------------------------------------------------------------

// Internal layout of palette textures: PLANES storage of K palette buckets
// (plane = K) reached through the index map, bucket (i, j) -> index[j w + i].
constexpr int kLayoutPalette = 2;

// Offset of bucket (i, j) in the 2 x 2 quad order of RT_LAYOUT_QUADS: a plane
// holds ceil(w/2) x ceil(h/2) quads (an odd side is padded).
__device__ __forceinline__ int quad_slot(int W, int i, int j) {
    return (((j >> 1) * ((W + 1) >> 1) + (i >> 1)) << 2) + ((j & 1) << 1) + (i & 1);
}

// Spatial offset of bucket (i, j) inside a direction plane.
template <int LAYOUT>
__device__ __forceinline__ int bucket_slot(const TexDesc& d, int i, int j) {
#ifdef RADTEX_CHECKED
    const int b = checked_slot(d, (int64_t)j * d.W + i, (int64_t)d.W * d.H);
    if (LAYOUT == kLayoutPalette) return checked_slot(d, __ldg(d.index + b), d.plane);
    if (LAYOUT == RT_LAYOUT_QUADS) {
        const int jb = b / d.W;
        return quad_slot(d.W, b - jb * d.W, jb);
    }
#else
    if (LAYOUT == RT_LAYOUT_QUADS) return quad_slot(d.W, i, j);
    const int b = j * d.W + i;
    if (LAYOUT == kLayoutPalette) return (int)__ldg(d.index + b);
#endif
    return b;
}

// The spatial offsets of the 2 x 2 buckets (u0,v0) (u1,v0) (u0,v1) (u1,v1) of a
// quadrilinear lookup.  The quad order is separable, slot(i, j) = a(j) + b(i)
// with b(i) = 2 i - (i mod 2) and a(j) = 4 (j / 2) ceil(w / 2) + 2 (j mod 2), so
// the four offsets cost two terms per axis and four additions.
template <int LAYOUT>
__device__ __forceinline__ void bucket_slots4(const TexDesc& d, int u0, int u1, int v0, int v1, int (&o)[4]) {
#ifndef RADTEX_CHECKED
    if constexpr (LAYOUT == RT_LAYOUT_QUADS) {
        const int wq4 = ((d.W + 1) >> 1) << 2;
        const int b0 = 2 * u0 - (u0 & 1), b1 = 2 * u1 - (u1 & 1);
        const int a0 = (v0 >> 1) * wq4 + ((v0 & 1) << 1), a1 = (v1 >> 1) * wq4 + ((v1 & 1) << 1);
        o[0] = a0 + b0;
        o[1] = a0 + b1;
        o[2] = a1 + b0;
        o[3] = a1 + b1;
        return;
    }
#endif
    o[0] = bucket_slot<LAYOUT>(d, u0, v0);
    o[1] = bucket_slot<LAYOUT>(d, u1, v0);
    o[2] = bucket_slot<LAYOUT>(d, u0, v1);
    o[3] = bucket_slot<LAYOUT>(d, u1, v1);
}

template <int LAYOUT>
__device__ __forceinline__ int64_t texel_index(const TexDesc& d, int i, int j, int s, int t) {
    if (LAYOUT == RT_LAYOUT_ATLAS)
        return checked_texel(d, ((int64_t)j * d.n + t) * ((int64_t)d.W * d.n) + (int64_t)i * d.n + s);
    return checked_texel(d, (int64_t)(t * d.n + s) * d.plane + bucket_slot<LAYOUT>(d, i, j));
}

template <int FMT>
__device__ __forceinline__ float4 load_texel(const void* base, int64_t idx, float scale);

// 1-bit texels: bit idx of the packed words.
__device__ __forceinline__ float bit_texel(const void* base, int64_t idx) {
    const unsigned w = __ldg(reinterpret_cast<const unsigned*>(base) + (idx >> 5));
    return (float)((w >> (unsigned)(idx & 31)) & 1u);
}

template <>
__device__ __forceinline__ float4 load_texel<RT_BIT1>(const void* base, int64_t idx, float) {
    const float v = bit_texel(base, idx);
    return make_float4(v, v, v, v);
}

template <>
__device__ __forceinline__ float4 load_texel<RT_F32>(const void* base, int64_t idx, float) {
    return __ldg(reinterpret_cast<const float4*>(base) + idx);
}

template <>
__device__ __forceinline__ float4 load_texel<RT_F16>(const void* base, int64_t idx, float) {
    uint2 r = __ldg(reinterpret_cast<const uint2*>(base) + idx);
    __half2 a = *reinterpret_cast<__half2*>(&r.x);
    __half2 b = *reinterpret_cast<__half2*>(&r.y);
    float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

template <>
__device__ __forceinline__ float4 load_texel<RT_BF16>(const void* base, int64_t idx, float) {
    uint2 r = __ldg(reinterpret_cast<const uint2*>(base) + idx);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&r.x);
    __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&r.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

__device__ __forceinline__ float2 e4m3x2_to_float2(unsigned short v) {
    __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)v, __NV_E4M3);
    __half2 hh = *reinterpret_cast<__half2*>(&h);
    return __half22float2(hh);
}

template <>
__device__ __forceinline__ float4 load_texel<RT_E4M3_BUCKET_SCALE>(const void* base, int64_t idx, float scale) {
    unsigned r = __ldg(reinterpret_cast<const unsigned*>(base) + idx);
    float2 a = e4m3x2_to_float2((unsigned short)(r & 0xFFFFu));
    float2 b = e4m3x2_to_float2((unsigned short)(r >> 16));
    return make_float4(a.x * scale, a.y * scale, b.x * scale, b.y * scale);
}

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float w) {
    return make_float4(fmaf(w, b.x - a.x, a.x), fmaf(w, b.y - a.y, a.y), fmaf(w, b.z - a.z, a.z),
                       fmaf(w, b.w - a.w, a.w));
}

__device__ __forceinline__ float4 sub4(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}

__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }

// RGBA held as two packed FP32 pairs, filtered with the paired FP32 FMA of
// sm_100+ (fma.rn.f32x2 / sub.rn.f32x2): the same roundings as the scalar
// lerp a + w (b - a), at half the instruction count.
typedef unsigned long long f32x2;
struct P4 {
    f32x2 rg, ba;
};

__device__ __forceinline__ f32x2 pack2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 unpack2(f32x2 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f32x2 lerp2(f32x2 a, f32x2 b, f32x2 w) {
    f32x2 d, r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(b), "l"(a));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(w), "l"(d), "l"(a));
    return r;
}
__device__ __forceinline__ P4 lerpP(const P4& a, const P4& b, f32x2 w) { return {lerp2(a.rg, b.rg, w), lerp2(a.ba, b.ba, w)}; }
__device__ __forceinline__ float4 toF4(const P4& p) {
    float2 a = unpack2(p.rg), b = unpack2(p.ba);
    return make_float4(a.x, a.y, b.x, b.y);
}

template <int FMT>
__device__ __forceinline__ P4 load_texelP(const void* base, int64_t idx, float scale);

template <>
__device__ __forceinline__ P4 load_texelP<RT_F32>(const void* base, int64_t idx, float) {
    float4 v = __ldg(reinterpret_cast<const float4*>(base) + idx);
    return {pack2(v.x, v.y), pack2(v.z, v.w)};
}

// The four channels of an 8-byte FP16 / BF16 code, widened to FP32 (exact).
template <int FMT>
__device__ __forceinline__ P4 decode8(uint2 r);

template <>
__device__ __forceinline__ P4 decode8<RT_F16>(uint2 r) {
    float2 fa = __half22float2(*reinterpret_cast<__half2*>(&r.x));
    float2 fb = __half22float2(*reinterpret_cast<__half2*>(&r.y));
    return {pack2(fa.x, fa.y), pack2(fb.x, fb.y)};
}

// BF16 is the upper half of an FP32: widening is a 16-bit shift (exact).
template <>
__device__ __forceinline__ P4 decode8<RT_BF16>(uint2 r) {
    return {pack2(__uint_as_float(r.x << 16), __uint_as_float(r.x & 0xFFFF0000u)),
            pack2(__uint_as_float(r.y << 16), __uint_as_float(r.y & 0xFFFF0000u))};
}

template <>
__device__ __forceinline__ P4 load_texelP<RT_F16>(const void* base, int64_t idx, float) {
    return decode8<RT_F16>(__ldg(reinterpret_cast<const uint2*>(base) + idx));
}

template <>
__device__ __forceinline__ P4 load_texelP<RT_BIT1>(const void* base, int64_t idx, float) {
    const float v = bit_texel(base, idx);
    return {pack2(v, v), pack2(v, v)};
}

template <>
__device__ __forceinline__ P4 load_texelP<RT_BF16>(const void* base, int64_t idx, float) {
    return decode8<RT_BF16>(__ldg(reinterpret_cast<const uint2*>(base) + idx));
}

// The four channels of a 4-byte E4M3 code times its bucket's scale, in FP32.
__device__ __forceinline__ P4 decode4_e4m3(unsigned r, float scale) {
    float2 a = e4m3x2_to_float2((unsigned short)(r & 0xFFFFu));
    float2 b = e4m3x2_to_float2((unsigned short)(r >> 16));
    return {pack2(a.x * scale, a.y * scale), pack2(b.x * scale, b.y * scale)};
}

template <>
__device__ __forceinline__ P4 load_texelP<RT_E4M3_BUCKET_SCALE>(const void* base, int64_t idx, float scale) {
    return decode4_e4m3(__ldg(reinterpret_cast<const unsigned*>(base) + idx), scale);
}

// Vector reduction of four floats into global memory (one 16-byte atomic).
__device__ __forceinline__ void red_add_v4(float* addr, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

}  // namespace rt

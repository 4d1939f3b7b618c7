// bake.cu -- baking a radiance texture from a ray-traced analytic scene
// (Section 2.2, Eq. 4a and Eq. 4b).
//
// One thread per bucket.  A block covers 128 consecutive buckets (bucket
// b = j w + i), so at every in-bucket texel (s, t) its stores fall in one
// direction plane: consecutive texels (PLANES) or pairs of them (QUADS).  The grid's y dimension
// splits the n^2 planes of a bucket among blocks when there are too few
// buckets to fill the GPU; FP8 E4M3 keeps a bucket in one thread, which
// evaluates the bucket twice (its amax sets the bucket's scale, then the
// codes).  The per-texel work is the reflection vector (Eq. 4a, Eq. 4b), its
// rotation to world space, one ray against the sphere and the plane, and the
// sky and shading functions: ALU work, about 150 instructions per texel.
#include <math.h>

#include "rt_encode.cuh"
#include "rt_internal.h"

namespace rt {

constexpr int kBakeThreads = 128;

struct Ray {
    float3 P, T, B, N;  // surface point and tangent frame
    float3 base;        // the surface's own lit colour
    float refl;
};

__device__ __forceinline__ float3 mk(const float* a) { return make_float3(a[0], a[1], a[2]); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 axpy(float a, float3 x, float3 y) {
    return make_float3(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z));
}
__device__ __forceinline__ float3 scale3(float a, float3 x) { return make_float3(a * x.x, a * x.y, a * x.z); }

__device__ __forceinline__ float lit(const rt_bake_scene& S, float3 N) {
    return S.ambient + (1.0f - S.ambient) * fmaxf(dot3(N, mk(S.sun_direction)), 0.0f);
}

__device__ __forceinline__ float3 sky(const rt_bake_scene& S, float3 d) {
    const float h = 0.5f + 0.5f * d.y;
    const float c = dot3(d, mk(S.sun_direction));
    const float sun = c > 0.0f ? powf(c, S.sun_exponent) : 0.0f;
    float3 r;
    r.x = S.sky_horizon[0] + (S.sky_zenith[0] - S.sky_horizon[0]) * h + S.sun_rgb[0] * sun;
    r.y = S.sky_horizon[1] + (S.sky_zenith[1] - S.sky_horizon[1]) * h + S.sun_rgb[1] * sun;
    r.z = S.sky_horizon[2] + (S.sky_zenith[2] - S.sky_horizon[2]) * h + S.sun_rgb[2] * sun;
    return r;
}

__device__ __forceinline__ float3 plane_albedo(const rt_bake_scene& S, float x, float z) {
    const float m = 0.75f + 0.25f * cosf(S.plane_frequency * x) * cosf(S.plane_frequency * z);
    return scale3(m, mk(S.plane_albedo));
}

// Radiance along P + t d and its fog transmittance (0 for a miss).
__device__ __forceinline__ float4 trace(const rt_bake_scene& S, float3 P, float3 d) {
    const float3 c = mk(S.sphere_centre);
    const float3 o = make_float3(P.x - c.x, P.y - c.y, P.z - c.z);
    const float b = dot3(o, d);
    const float q = dot3(o, o) - S.sphere_radius * S.sphere_radius;
    const float disc = b * b - q;
    float tb = INFINITY;
    int hit = -1;
    if (disc > 0.0f) {
        const float t = -b - sqrtf(disc);  // entering root
        if (t > S.ray_offset) {
            tb = t;
            hit = RT_SURFACE_SPHERE;
        }
    }
    if (d.y != 0.0f) {
        const float t = (S.plane_height - P.y) / d.y;
        if (t > S.ray_offset && t < tb) {
            tb = t;
            hit = RT_SURFACE_PLANE;
        }
    }
    const float3 K = sky(S, d);
    if (hit < 0) return make_float4(K.x, K.y, K.z, 0.0f);
    const float3 X = axpy(tb, d, P);
    float3 C;
    if (hit == RT_SURFACE_SPHERE) {
        const float ir = 1.0f / S.sphere_radius;
        const float3 Nh = make_float3((X.x - c.x) * ir, (X.y - c.y) * ir, (X.z - c.z) * ir);
        C = scale3(lit(S, Nh), mk(S.sphere_albedo));
    } else {
        C = scale3(lit(S, make_float3(0.0f, 1.0f, 0.0f)), plane_albedo(S, X.x, X.z));
    }
    const float g = expf(-S.fog * tb);
    return make_float4(g * C.x + (1.0f - g) * K.x, g * C.y + (1.0f - g) * K.y, g * C.z + (1.0f - g) * K.z, g);
}

// The sphere's entering root or the plane crossing at t > ray_offset.
__device__ __forceinline__ bool occluded(const rt_bake_scene& S, float3 P, float3 d) {
    const float3 c = mk(S.sphere_centre);
    const float3 o = make_float3(P.x - c.x, P.y - c.y, P.z - c.z);
    const float b = dot3(o, d);
    const float q = dot3(o, o) - S.sphere_radius * S.sphere_radius;
    const float disc = b * b - q;
    if (disc > 0.0f && -b - sqrtf(disc) > S.ray_offset) return true;
    return d.y != 0.0f && (S.plane_height - P.y) / d.y > S.ray_offset;
}

// Deferred payload (Section 1: ambient occlusion and reflections for deferred
// rendering): the first hit X of the reflected ray, its unlit albedo and the
// share of the K local directions (frame of the hit normal facing the ray, x
// and y from the orthonormal basis of Duff et al., JCGT 6(1) 2017) that leave
// X unblocked; (0, 0, 0, 1) when the ray reaches the sky.  An AO ray is tested
// against the other surface only: leaving the plane into its normal's
// half-space it cannot meet the plane again, nor leaving the convex sphere
// outward the sphere.
__device__ __forceinline__ float4 deferred_payload(const rt_bake_scene& S, float3 P, float3 d, const float4* dirs,
                                                   int K) {
    const float3 c = mk(S.sphere_centre);
    const float3 o = make_float3(P.x - c.x, P.y - c.y, P.z - c.z);
    const float b = dot3(o, d);
    const float q = dot3(o, o) - S.sphere_radius * S.sphere_radius;
    const float disc = b * b - q;
    float tb = INFINITY;
    int hit = -1;
    if (disc > 0.0f) {
        const float t = -b - sqrtf(disc);
        if (t > S.ray_offset) {
            tb = t;
            hit = RT_SURFACE_SPHERE;
        }
    }
    if (d.y != 0.0f) {
        const float t = (S.plane_height - P.y) / d.y;
        if (t > S.ray_offset && t < tb) {
            tb = t;
            hit = RT_SURFACE_PLANE;
        }
    }
    if (hit < 0) return make_float4(0.0f, 0.0f, 0.0f, 1.0f);
    const float3 X = axpy(tb, d, P);
    float3 N, alb;
    if (hit == RT_SURFACE_SPHERE) {
        const float ir = 1.0f / S.sphere_radius;
        N = make_float3((X.x - c.x) * ir, (X.y - c.y) * ir, (X.z - c.z) * ir);
        alb = mk(S.sphere_albedo);
    } else {
        N = make_float3(0.0f, d.y < 0.0f ? 1.0f : -1.0f, 0.0f);
        alb = plane_albedo(S, X.x, X.z);
    }
    // basis (b1, b2, N), right-handed
    const float sg = copysignf(1.0f, N.z);
    const float a = -1.0f / (sg + N.z);
    const float bb = N.x * N.y * a;
    const float3 b1 = make_float3(fmaf(sg * N.x * N.x, a, 1.0f), sg * bb, -sg * N.x);
    const float3 b2 = make_float3(bb, fmaf(N.y * N.y, a, sg), -N.y);
    // Each test needs one component of the world direction b1 w.x + b2 w.y + N w.z
    // along a fixed vector, so that vector is projected on the basis once per hit
    // and a direction costs three FMAs; the tests are written without division
    // or square root (the same decisions up to rounding at the threshold).
    const float eps = S.ray_offset;
    int vis = 0;
    if (hit == RT_SURFACE_SPHERE) {
        // only the plane can block: the crossing t = h / w_y lies beyond eps
        const float h = S.plane_height - X.y;
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
            const float4 w = dirs[k];
            const float wy = fmaf(w.z, N.y, fmaf(w.y, b2.y, w.x * b1.y));
            const float e = eps * wy;
            vis += ((wy > 0.0f && h > e) || (wy < 0.0f && h < e)) ? 0 : 1;
        }
    } else {
        // only the sphere can block: b = (X - c).w, entering root -b - sqrt(b^2 - q) > eps
        const float3 oX = make_float3(X.x - c.x, X.y - c.y, X.z - c.z);
        const float qX = dot3(oX, oX) - S.sphere_radius * S.sphere_radius;
        const float o1 = dot3(oX, b1), o2 = dot3(oX, b2), o3 = dot3(oX, N);
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
            const float4 w = dirs[k];
            const float bw = fmaf(w.z, o3, fmaf(w.y, o2, w.x * o1));
            const float dw = fmaf(bw, bw, -qX);  // the ray meets the sphere when dw > 0
            const float m = -bw - eps;            // and enters ahead when m > sqrt(dw)
            vis += (dw > 0.0f && m > 0.0f && m * m > dw) ? 0 : 1;
        }
    }
    return make_float4(alb.x, alb.y, alb.z, (float)vis / (float)K);
}

// Surface point, frame and own colour at the centre of bucket (i, j).
__device__ __forceinline__ Ray bucket_ray(const rt_bake_scene& S, int surface, int i, int j, int W, int H) {
    const float u = ((float)i + 0.5f) / (float)W, v = ((float)j + 0.5f) / (float)H;
    Ray r;
    if (surface == RT_SURFACE_SPHERE) {
        float sp, cp, st, ct;
        sincospif(2.0f * u - 1.0f, &sp, &cp);  // phi = 2 pi u - pi
        sincospif(v, &st, &ct);                // theta = pi v
        r.N = make_float3(st * cp, ct, st * sp);
        r.T = make_float3(-sp, 0.0f, cp);
        r.B = make_float3(ct * cp, -st, ct * sp);
        r.P = axpy(S.sphere_radius, r.N, mk(S.sphere_centre));
        r.base = scale3(lit(S, r.N), mk(S.sphere_albedo));
        r.refl = S.sphere_reflectance;
    } else {
        const float e = S.plane_half_extent;
        r.P = make_float3(2.0f * e * u - e, S.plane_height, 2.0f * e * v - e);
        r.T = make_float3(1.0f, 0.0f, 0.0f);
        r.B = make_float3(0.0f, 0.0f, 1.0f);
        r.N = make_float3(0.0f, 1.0f, 0.0f);
        r.base = scale3(lit(S, r.N), plane_albedo(S, r.P.x, r.P.z));
        r.refl = S.plane_reflectance;
    }
    return r;
}

// Texel p of the bucket with tangent-space reflection vector R (Eq. 4a then
// Eq. 4b at the texel centre, from the block's table); d = R in world space.
// The radiance payload, or with K > 0 the deferred one over the K directions.
__device__ __forceinline__ float4 bake_texel(const rt_bake_scene& S, const Ray& r, float3 R, const float4* dirs,
                                             int K) {
    const float3 d = axpy(R.z, r.N, axpy(R.y, r.B, scale3(R.x, r.T)));
    if (K > 0) return deferred_payload(S, r.P, d, dirs, K);
    const float4 tr = trace(S, r.P, d);
    return make_float4(fmaf(r.refl, tr.x, r.base.x), fmaf(r.refl, tr.y, r.base.y), fmaf(r.refl, tr.z, r.base.z),
                       tr.w);
}

// The n^2 tangent-space vectors of the in-bucket texels (Eq. 4a, then Eq. 4b or
// Eq. 2c), computed once per block into shared memory (n <= 64: at most 48 KiB).
template <bool REFLECT>
__device__ __forceinline__ void texel_vector_table(float3* tab, int n) {
    for (int p = threadIdx.x; p < n * n; p += blockDim.x)
        tab[p] = REFLECT ? texel_reflection(p % n, p / n, n) : texel_centre_direction(p % n, p / n, n);
    __syncthreads();
}

// K = 0: radiance texels; K > 0: deferred payloads over the K local
// directions ao_dirs (device, K x 3 floats), staged after the vector table.
template <int FMT, int LAYOUT>
__global__ void __launch_bounds__(kBakeThreads) bake_kernel(rt_bake_scene S, int surface, void* __restrict__ dst,
                                                            float* __restrict__ scale, int W, int H, int n,
                                                            const float* __restrict__ ao_dirs, int K) {
    extern __shared__ float3 Rtab[];
    // the directions as float4 (one 16-byte shared load each), after the vector table
    float4* dirs = reinterpret_cast<float4*>(Rtab + ((n * n + 3) & ~3));
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        dirs[k] = make_float4(ao_dirs[3 * k], ao_dirs[3 * k + 1], ao_dirs[3 * k + 2], 0.0f);
    texel_vector_table<true>(Rtab, n);  // ends with the block barrier
    const int64_t b = (int64_t)blockIdx.x * kBakeThreads + threadIdx.x;
    if (b >= (int64_t)W * H) return;
    const int j = (int)(b / W), i = (int)(b - (int64_t)j * W);
    const Ray r = bucket_ray(S, surface, i, j, W, H);
    const int planes = n * n;
    const int p0 = (int)((int64_t)blockIdx.y * planes / gridDim.y);
    const int p1 = (int)((int64_t)(blockIdx.y + 1) * planes / gridDim.y);
    float sc = 1.0f;
    if (FMT == RT_E4M3_BUCKET_SCALE) {
        float amax = 0.0f;
        for (int p = 0; p < planes; ++p) amax = fmaxf(amax, amax4(bake_texel(S, r, Rtab[p], dirs, K)));
        sc = bucket_scale(amax);
        scale[slot_in(LAYOUT, W, i, j)] = sc;
    }
    for (int p = p0; p < p1; ++p) {
        const int t = p / n, s = p - t * n;
        const float4 v = bake_texel(S, r, Rtab[p], dirs, K);
        const int64_t idx = index_in(LAYOUT, W, H, n, i, j, s, t);
        if (FMT == RT_F32)
            reinterpret_cast<float4*>(dst)[idx] = v;
        else if (FMT == RT_F16)
            reinterpret_cast<uint2*>(dst)[idx] = pack_f16(v);
        else if (FMT == RT_BF16)
            reinterpret_cast<uint2*>(dst)[idx] = pack_bf16(v);
        else
            reinterpret_cast<unsigned*>(dst)[idx] = pack_e4m3(v, sc);
    }
}

template <int FMT, int LAYOUT>
static cudaError_t launch_bake_t(const rt_bake_scene& S, int surface, void* dst, float* scale, int W, int H, int n,
                                 const float* ao_dirs, int K, cudaStream_t stream) {
    const int64_t buckets = (int64_t)W * H;
    const unsigned gx = (unsigned)((buckets + kBakeThreads - 1) / kBakeThreads);
    // enough blocks for 8 per SM; E4M3 needs the whole bucket in one thread
    unsigned gy = 1;
    if (FMT != RT_E4M3_BUCKET_SCALE) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t want = (int64_t)sms * 8;
        if ((int64_t)gx < want) gy = (unsigned)((want + gx - 1) / gx);
        if (gy > (unsigned)(n * n)) gy = (unsigned)(n * n);
    }
    const size_t smem = sizeof(float3) * (((size_t)n * n + 3) & ~(size_t)3) + sizeof(float4) * (size_t)K;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(bake_kernel<FMT, LAYOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    bake_kernel<FMT, LAYOUT><<<dim3(gx, gy), kBakeThreads, smem, stream>>>(S, surface, dst, scale, W, H, n, ao_dirs,
                                                                            K);
    return cudaGetLastError();
}

template <int LAYOUT>
static cudaError_t launch_bake_l(const rt_bake_scene& S, int surface, void* dst, float* scale, int W, int H, int n,
                                 int fmt, const float* ao_dirs, int K, cudaStream_t stream) {
    switch (fmt) {
        case RT_F32:
            return launch_bake_t<RT_F32, LAYOUT>(S, surface, dst, scale, W, H, n, ao_dirs, K, stream);
        case RT_F16:
            return launch_bake_t<RT_F16, LAYOUT>(S, surface, dst, scale, W, H, n, ao_dirs, K, stream);
        case RT_BF16:
            return launch_bake_t<RT_BF16, LAYOUT>(S, surface, dst, scale, W, H, n, ao_dirs, K, stream);
        default:
            return launch_bake_t<RT_E4M3_BUCKET_SCALE, LAYOUT>(S, surface, dst, scale, W, H, n, ao_dirs, K, stream);
    }
}

cudaError_t launch_bake(const rt_bake_scene& S, int surface, void* dst, float* scale, int W, int H, int n, int fmt,
                        int layout, const float* ao_dirs, int K, cudaStream_t stream) {
    if (layout == RT_LAYOUT_ATLAS) {
        if (fmt != RT_F32) return cudaErrorInvalidValue;
        return launch_bake_t<RT_F32, RT_LAYOUT_ATLAS>(S, surface, dst, scale, W, H, n, ao_dirs, K, stream);
    }
    if (layout == RT_LAYOUT_QUADS) return launch_bake_l<RT_LAYOUT_QUADS>(S, surface, dst, scale, W, H, n, fmt, ao_dirs,
                                                                         K, stream);
    return launch_bake_l<RT_LAYOUT_PLANES>(S, surface, dst, scale, W, H, n, fmt, ao_dirs, K, stream);
}

// ---------------------------------------------------------------------------
// Shadow bake (Section 5, "Shadowing"): a 1-bit texture keyed by the light
// direction.  Bit (i, j, s, t) = the ray from bucket (i, j)'s surface point
// towards texel (s, t)'s direction (Eq. 4a, Eq. 2c, in world space) reaches
// the sky.  One thread per 32-bit word of the PLANES bit numbering, so every
// word is written once, whole.
// ---------------------------------------------------------------------------

// Surface point and frame of bucket (i, j) (the geometry of bucket_ray).
__device__ __forceinline__ void bucket_frame(const rt_bake_scene& S, int surface, int i, int j, int W, int H,
                                             float3& P, float3& T, float3& B, float3& N) {
    const float u = ((float)i + 0.5f) / (float)W, v = ((float)j + 0.5f) / (float)H;
    if (surface == RT_SURFACE_SPHERE) {
        float sp, cp, st, ct;
        sincospif(2.0f * u - 1.0f, &sp, &cp);
        sincospif(v, &st, &ct);
        N = make_float3(st * cp, ct, st * sp);
        T = make_float3(-sp, 0.0f, cp);
        B = make_float3(ct * cp, -st, ct * sp);
        P = axpy(S.sphere_radius, N, mk(S.sphere_centre));
    } else {
        const float e = S.plane_half_extent;
        P = make_float3(2.0f * e * u - e, S.plane_height, 2.0f * e * v - e);
        T = make_float3(1.0f, 0.0f, 0.0f);
        B = make_float3(0.0f, 0.0f, 1.0f);
        N = make_float3(0.0f, 1.0f, 0.0f);
    }
}

__global__ void __launch_bounds__(kBakeThreads) shadow_bake_kernel(rt_bake_scene S, int surface,
                                                                   unsigned* __restrict__ dst, int W, int H, int n) {
    const int64_t plane = (int64_t)W * H, total = plane * n * n;
    const int64_t w = (int64_t)blockIdx.x * kBakeThreads + threadIdx.x;
    if (w * 32 >= total) return;
    unsigned word = 0;
    for (int k = 0; k < 32; ++k) {
        const int64_t e = w * 32 + k;
        if (e >= total) break;
        const int p = (int)(e / plane);
        const int64_t b = e - (int64_t)p * plane;
        const int j = (int)(b / W), i = (int)(b - (int64_t)j * W);
        const int t = p / n, s = p - t * n;
        float3 P, T, B, N;
        bucket_frame(S, surface, i, j, W, H, P, T, B, N);
        const float3 I = texel_centre_direction(s, t, n);
        const float3 d = axpy(I.z, N, axpy(I.y, B, scale3(I.x, T)));
        if (!occluded(S, P, d)) word |= 1u << k;
    }
    dst[w] = word;
}

// w h a multiple of 32: a warp takes 32 consecutive buckets (one 32-bit word
// of every plane), computes each bucket's frame once, and forms every plane's
// word with a ballot of the lanes' visibility bits.
__global__ void __launch_bounds__(kBakeThreads) shadow_bake_ballot_kernel(rt_bake_scene S, int surface,
                                                                          unsigned* __restrict__ dst, int W, int H,
                                                                          int n) {
    extern __shared__ float3 Dtab[];
    texel_vector_table<false>(Dtab, n);
    const int64_t plane = (int64_t)W * H;
    const int64_t b = (int64_t)blockIdx.x * kBakeThreads + threadIdx.x;  // plane % 32 == 0: warps stay in range
    if (b - (threadIdx.x & 31) >= plane) return;                        // whole warps only
    const int lane = threadIdx.x & 31;
    const bool valid = b < plane;
    float3 P, T, B, N;
    const int j = valid ? (int)(b / W) : 0, i = valid ? (int)(b - (int64_t)j * W) : 0;
    bucket_frame(S, surface, i, j, W, H, P, T, B, N);
    for (int p = 0; p < n * n; ++p) {
        const float3 I = Dtab[p];
        const float3 d = axpy(I.z, N, axpy(I.y, B, scale3(I.x, T)));
        const unsigned word = __ballot_sync(0xffffffffu, valid && !occluded(S, P, d));
        if (lane == 0) dst[(p * plane + b) >> 5] = word;
    }
}

cudaError_t launch_bake_shadow(const rt_bake_scene& S, int surface, void* dst, int W, int H, int n,
                               cudaStream_t stream) {
    const int64_t plane = (int64_t)W * H;
    if (plane % 32 == 0) {
        const size_t smem = sizeof(float3) * (size_t)n * n;
        shadow_bake_ballot_kernel<<<(unsigned)((plane + kBakeThreads - 1) / kBakeThreads), kBakeThreads, smem,
                                    stream>>>(S, surface, static_cast<unsigned*>(dst), W, H, n);
        return cudaGetLastError();
    }
    const int64_t words = ((int64_t)W * H * n * n + 31) / 32;
    shadow_bake_kernel<<<(unsigned)((words + kBakeThreads - 1) / kBakeThreads), kBakeThreads, 0, stream>>>(
        S, surface, static_cast<unsigned*>(dst), W, H, n);
    return cudaGetLastError();
}

}  // namespace rt

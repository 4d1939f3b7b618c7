// rt_backward.cuh -- device code of the lookup's gradients, shared by the
// backward kernels (backward.cu) and the fused forward + L2 + backward step
// (fused.cu): texel gradients w_tap * dL/dout summed into FP32 buffers with
// 16-byte vector reductions (or 64-bit fixed point in the deterministic mode),
// and the chain rule of the UV and direction gradients through the nested
// lerps, the Note's clamp, Eq. 3 and Eq. 1b.
#pragma once

#include "rt_device.cuh"
#include "rt_filter.cuh"

namespace rt {

constexpr int kBackThreads = 128;
constexpr int kBackWarps = kBackThreads / 32;

struct CoordGrad {
    float gu, gv, gs, gt;  // dL/d(weight coordinate) of the u, v, s, t axes
};

// Deterministic mode: each contribution w g_c is rounded once to a signed
// 64-bit fixed-point number with 32 fractional bits and added with integer
// atomics, which are associative, so the sums do not depend on the order in
// which fragments arrive.
constexpr float kFixedScale = 4294967296.0f;  // 2^32

__device__ __forceinline__ void red_add_fixed4(unsigned long long* addr, float4 v) {
    atomicAdd(addr + 0, (unsigned long long)__float2ll_rn(v.x * kFixedScale));
    atomicAdd(addr + 1, (unsigned long long)__float2ll_rn(v.y * kFixedScale));
    atomicAdd(addr + 2, (unsigned long long)__float2ll_rn(v.z * kFixedScale));
    atomicAdd(addr + 3, (unsigned long long)__float2ll_rn(v.w * kFixedScale));
}

// The weights a lane whose axis has taps pk0, pk0 + 1 and weight pw (of pk0 + 1)
// puts on coordinates k0 and k0 + 1: 1 - pw on pk0, pw on pk0 + 1, 0 elsewhere --
// the values that lane uses for its own taps, bit for bit.
__device__ __forceinline__ void partner_axis_weights(int k0, int pk0, float pw, float (&out)[2]) {
    const int dk = k0 - pk0;
    const float w0 = 1.f - pw;
    out[0] = dk == 0 ? w0 : (dk == 1 ? pw : 0.f);
    out[1] = dk == -1 ? w0 : (dk == 0 ? pw : 0.f);
}

// QUADRILINEAR on the PLANES / QUADS / palette layouts: the four in-bucket
// texels select four planes (64-bit bases), the four buckets four spatial
// offsets (32-bit), shared by the 16 reductions and the 16 loads.  The 16
// texel-gradient contributions w_tap g of a lookup: planes pl[k] (k = (s0,t0)
// (s1,t0) (s0,t1) (s1,t1)), spatial offsets o[b] (b = (u0,v0) (u1,v0) (u0,v1)
// (u1,v1)).
template <bool DET>
__device__ __forceinline__ void reduce_quadrilinear_taps(const TexDesc& d, const Lookup<RT_QUADRILINEAR>& L,
                                                         const int64_t (&pl)[4], const int (&o)[4], float4 g,
                                                         void* grad) {
    const float wu[2] = {1.f - L.u.w, L.u.w}, wv[2] = {1.f - L.v.w, L.v.w};
    const float ws[2] = {1.f - L.s.w, L.s.w}, wt[2] = {1.f - L.t.w, L.t.w};
    if (DET) {
        if (grad) {
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float w = wu[b & 1] * wv[b >> 1] * ws[k & 1] * wt[k >> 1];
                    if (w == 0.f) continue;
                    const int64_t idx = checked_texel(d, pl[k] + o[b]);
                    red_add_fixed4(static_cast<unsigned long long*>(grad) + 4 * idx,
                                   make_float4(w * g.x, w * g.y, w * g.z, w * g.w));
                }
        }
    } else {
        // Neighbouring fragments often update the same texels: lanes 2m and
        // 2m + 1 (horizontal neighbours on screen) exchange, once per fragment,
        // their texture's addressing (gradient buffer, plane size, width, n,
        // layout), their four axes' floors k0 and weights, and dL/dout.  Each
        // lane then knows the other's weight on each of its own taps -- the same
        // tap or one a bucket or texel over -- as the same product of the same
        // axis weights the other lane forms, so both decide alike: for a texel
        // both reduce into, the even lane adds the odd lane's contribution to its
        // own and issues one reduction, and the odd lane issues none.  Only pairs
        // whose four axes each have the two taps k0, k0 + 1 merge (not at a
        // clamped edge or a wrapped seam).  A lane without a gradient buffer
        // leaves before the exchange (its partner sees it inactive).
        if (!grad) return;
        const unsigned active = __activemask();
        const int lane = threadIdx.x & 31;
        const bool partner = (active >> (lane ^ 1)) & 1u;
        const bool plain = L.u.k1 == L.u.k0 + 1 && L.v.k1 == L.v.k0 + 1 && L.s.k1 == L.s.k0 + 1 &&
                           L.t.k1 == L.t.k0 + 1 && d.plane < ((int64_t)1 << 32) && d.W < (1 << 17) && d.n < 256;
        // the texel index of given coordinates depends on (plane, W, n, layout) only
        // (the layouts are 0 to 3)
        const uint64_t gp = (uint64_t)grad;
        const unsigned geo = plain ? ((unsigned)d.W | ((unsigned)d.n << 17) | ((unsigned)(d.layout & 3) << 25))
                                   : (0x80000000u | (unsigned)lane);  // matches no other lane
        const unsigned id[4] = {(unsigned)gp, (unsigned)(gp >> 32), (unsigned)d.plane, geo};
        bool merge = partner;
#pragma unroll
        for (int m = 0; m < 4; ++m) merge &= __shfl_xor_sync(active, id[m], 1) == id[m];
        const int pk[4] = {__shfl_xor_sync(active, L.u.k0, 1), __shfl_xor_sync(active, L.v.k0, 1),
                           __shfl_xor_sync(active, L.s.k0, 1), __shfl_xor_sync(active, L.t.k0, 1)};
        const float pwk[4] = {__shfl_xor_sync(active, L.u.w, 1), __shfl_xor_sync(active, L.v.w, 1),
                              __shfl_xor_sync(active, L.s.w, 1), __shfl_xor_sync(active, L.t.w, 1)};
        const float4 pg = make_float4(__shfl_xor_sync(active, g.x, 1), __shfl_xor_sync(active, g.y, 1),
                                      __shfl_xor_sync(active, g.z, 1), __shfl_xor_sync(active, g.w, 1));
        // the partner's weight on this lane's coordinates k0 and k0 + 1 of each axis
        float pu[2], pv[2], ps[2], pt[2];
        partner_axis_weights(L.u.k0, pk[0], pwk[0], pu);
        partner_axis_weights(L.v.k0, pk[1], pwk[1], pv);
        partner_axis_weights(L.s.k0, pk[2], pwk[2], ps);
        partner_axis_weights(L.t.k0, pk[3], pwk[3], pt);
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float w = wu[b & 1] * wv[b >> 1] * ws[k & 1] * wt[k >> 1];
                if (w == 0.f) continue;
                const float pw = pu[b & 1] * pv[b >> 1] * ps[k & 1] * pt[k >> 1];
                const bool shared = merge && pw != 0.f;
                if (shared && (lane & 1)) continue;  // the even lane reduces it for both
                float4 c = make_float4(w * g.x, w * g.y, w * g.z, w * g.w);
                if (shared) {
                    c.x += pw * pg.x;
                    c.y += pw * pg.y;
                    c.z += pw * pg.z;
                    c.w += pw * pg.w;
                }
                red_add_v4(static_cast<float*>(grad) + 4 * checked_texel(d, pl[k] + o[b]), c);
            }
    }
}

// UV and in-bucket coordinate gradients of a quadrilinear lookup from its 16
// taps, texel(b, k) giving tap (bucket b, texel k): each tap is projected on g
// as it arrives and the lerps run on scalars.
template <typename Texel>
__device__ __forceinline__ CoordGrad quad_coord_grads(const Lookup<RT_QUADRILINEAR>& L, float4 g, Texel texel) {
    CoordGrad cg;
    const f32x2 g_rg = pack2(g.x, g.y), g_ba = pack2(g.z, g.w);
    auto lerpf = [](float a, float b, float w) { return fmaf(w, b - a, a); };
    float c[4], cs[4], ct[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        float p[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const P4 T = texel(b, k);
            f32x2 q;
            asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(q) : "l"(T.rg), "l"(g_rg));
            asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(q) : "l"(T.ba), "l"(g_ba), "l"(q));
            const float2 h = unpack2(q);
            p[k] = h.x + h.y;
        }
        const float x0 = lerpf(p[0], p[1], L.s.w), x1 = lerpf(p[2], p[3], L.s.w);
        c[b] = lerpf(x0, x1, L.t.w);
        cs[b] = lerpf(p[1] - p[0], p[3] - p[2], L.t.w);
        ct[b] = x1 - x0;
    }
    cg.gu = lerpf(c[1] - c[0], c[3] - c[2], L.v.w);
    cg.gv = lerpf(c[2], c[3], L.u.w) - lerpf(c[0], c[1], L.u.w);
    cg.gs = lerpf(lerpf(cs[0], cs[1], L.u.w), lerpf(cs[2], cs[3], L.u.w), L.v.w);
    cg.gt = lerpf(lerpf(ct[0], ct[1], L.u.w), lerpf(ct[2], ct[3], L.u.w), L.v.w);
    return cg;
}

template <int FMT, int LAYOUT, bool DET>
__device__ __forceinline__ CoordGrad backward_quadrilinear_planes(const TexDesc& d, const Lookup<RT_QUADRILINEAR>& L,
                                                                  float4 g, void* grad, bool coord_grads) {
    int64_t pl[4];  // (s0,t0) (s1,t0) (s0,t1) (s1,t1)
    int o[4];       // (u0,v0) (u1,v0) (u0,v1) (u1,v1)
    quad_tap_addresses<LAYOUT>(d, L.u, L.v, L.s, L.t, pl, o);
    reduce_quadrilinear_taps<DET>(d, L, pl, o, g, grad);
    if (!coord_grads) return CoordGrad{0.f, 0.f, 0.f, 0.f};
    return quad_coord_grads(L, g, [&](int b, int k) {
        const float sc = FMT == RT_E4M3_BUCKET_SCALE ? __ldg(d.scale + o[b]) : 1.0f;
        return load_texelP<FMT>(d.base, checked_texel(d, pl[k] + o[b]), sc);
    });
}

template <int FILTER, int FMT, int LAYOUT, bool DET>
__device__ __forceinline__ CoordGrad backward_taps(const TexDesc& d, const Lookup<FILTER>& L, float4 g, void* grad,
                                                   bool coord_grads) {
    CoordGrad cg = {0.f, 0.f, 0.f, 0.f};
    const float wu[2] = {1.f - L.u.w, L.u.w}, wv[2] = {1.f - L.v.w, L.v.w};
    const float ws[2] = {1.f - L.s.w, L.s.w}, wt[2] = {1.f - L.t.w, L.t.w};
    if (grad) {
        const int nu = FILTER == RT_QUADRILINEAR ? 2 : 1;
        const int ns = FILTER == RT_NEAREST ? 1 : 2;
        for (int b = 0; b < nu; ++b)
            for (int a = 0; a < nu; ++a)
                for (int q = 0; q < ns; ++q)
                    for (int p = 0; p < ns; ++p) {
                        float w = (nu == 2 ? wu[a] * wv[b] : 1.f) * (ns == 2 ? ws[p] * wt[q] : 1.f);
                        if (w == 0.f) continue;
                        int64_t idx = texel_index<LAYOUT>(d, a ? L.u.k1 : L.u.k0, b ? L.v.k1 : L.v.k0,
                                                          p ? L.s.k1 : L.s.k0, q ? L.t.k1 : L.t.k0);
                        const float4 c = make_float4(w * g.x, w * g.y, w * g.z, w * g.w);
                        if (DET)
                            red_add_fixed4(static_cast<unsigned long long*>(grad) + 4 * idx, c);
                        else
                            red_add_v4(static_cast<float*>(grad) + 4 * idx, c);
                    }
    }
    if (FILTER == RT_NEAREST || !coord_grads) return cg;
    // Coordinate gradients need only g . T per texel: every derivative of the
    // colour is a weighted sum of texels, so each texel is projected onto g as
    // soon as it is loaded and the lerps run on scalars.
    const f32x2 g_rg = pack2(g.x, g.y), g_ba = pack2(g.z, g.w);
    auto proj = [&](const P4& T) {
        f32x2 p;
        asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(p) : "l"(T.rg), "l"(g_rg));
        asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(p) : "l"(T.ba), "l"(g_ba), "l"(p));
        const float2 q = unpack2(p);
        return q.x + q.y;
    };
    auto lerpf = [](float a, float b, float w) { return fmaf(w, b - a, a); };
    if constexpr (FILTER == RT_ANGULAR_BILINEAR) {
        P4 t00, t10, t01, t11;
        load_quadP<FMT, LAYOUT>(d, L.u.k0, L.v.k0, L.s, L.t, t00, t10, t01, t11);
        const float p00 = proj(t00), p10 = proj(t10), p01 = proj(t01), p11 = proj(t11);
        cg.gs = lerpf(p10 - p00, p11 - p01, L.t.w);
        cg.gt = lerpf(p01, p11, L.s.w) - lerpf(p00, p10, L.s.w);
        return cg;
    } else {
        // bucket (a, b) of the 2 x 2 spatial footprint: value c_ab, d/ds, d/dt (all projected on g)
        float c[2][2], cs[2][2], ct[2][2];
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                P4 t00, t10, t01, t11;
                load_quadP<FMT, LAYOUT>(d, a ? L.u.k1 : L.u.k0, b ? L.v.k1 : L.v.k0, L.s, L.t, t00, t10, t01, t11);
                const float p00 = proj(t00), p10 = proj(t10), p01 = proj(t01), p11 = proj(t11);
                const float x0 = lerpf(p00, p10, L.s.w), x1 = lerpf(p01, p11, L.s.w);
                c[b][a] = lerpf(x0, x1, L.t.w);
                cs[b][a] = lerpf(p10 - p00, p11 - p01, L.t.w);
                ct[b][a] = x1 - x0;
            }
        cg.gu = lerpf(c[0][1] - c[0][0], c[1][1] - c[1][0], L.v.w);
        cg.gv = lerpf(c[1][0], c[1][1], L.u.w) - lerpf(c[0][0], c[0][1], L.u.w);
        cg.gs = lerpf(lerpf(cs[0][0], cs[0][1], L.u.w), lerpf(cs[1][0], cs[1][1], L.u.w), L.v.w);
        cg.gt = lerpf(lerpf(ct[0][0], ct[0][1], L.u.w), lerpf(ct[1][0], ct[1][1], L.u.w), L.v.w);
        return cg;
    }
}

template <int FILTER, int FMT, int LAYOUT, bool DET>
__device__ __forceinline__ CoordGrad backward_layout(const TexDesc& d, const Lookup<FILTER>& L, float4 g, void* grad,
                                                     bool coord_grads) {
    if constexpr (FILTER == RT_QUADRILINEAR && LAYOUT != RT_LAYOUT_ATLAS)
        return backward_quadrilinear_planes<FMT, LAYOUT, DET>(d, L, g, grad, coord_grads);
    else
        return backward_taps<FILTER, FMT, LAYOUT, DET>(d, L, g, grad, coord_grads);
}

template <int FILTER, int FMT, bool DET>
__device__ __forceinline__ CoordGrad backward_dense(const TexDesc& d, const Lookup<FILTER>& L, float4 g, void* grad,
                                                    bool coord_grads) {
    // as filter_dense: owned textures QUADS (bits PLANES), borrowed FP32 buffers QUADS or PLANES
    if (d.layout == kLayoutPalette) return backward_layout<FILTER, FMT, kLayoutPalette, DET>(d, L, g, grad, coord_grads);
    if (FMT == RT_BIT1) return backward_layout<FILTER, FMT, RT_LAYOUT_PLANES, DET>(d, L, g, grad, coord_grads);
    if (FMT != RT_F32 || d.layout == RT_LAYOUT_QUADS)
        return backward_layout<FILTER, FMT, RT_LAYOUT_QUADS, DET>(d, L, g, grad, coord_grads);
    return backward_layout<FILTER, FMT, RT_LAYOUT_PLANES, DET>(d, L, g, grad, coord_grads);
}

template <int FILTER, bool DET>
__device__ __forceinline__ CoordGrad backward_any(const TexDesc& d, const Lookup<FILTER>& L, float4 g, void* grad,
                                                  bool coord_grads) {
    switch (d.fmt) {
        case RT_F16:
            return backward_dense<FILTER, RT_F16, DET>(d, L, g, grad, coord_grads);
        case RT_BF16:
            return backward_dense<FILTER, RT_BF16, DET>(d, L, g, grad, coord_grads);
        case RT_BIT1:  // no texel gradients (rejected on the host); coordinate gradients only
            return backward_dense<FILTER, RT_BIT1, DET>(d, L, g, nullptr, coord_grads);
        case RT_E4M3_BUCKET_SCALE:
            return backward_dense<FILTER, RT_E4M3_BUCKET_SCALE, DET>(d, L, g, grad, coord_grads);
        default:
            if (d.layout == RT_LAYOUT_ATLAS)
                return backward_layout<FILTER, RT_F32, RT_LAYOUT_ATLAS, DET>(d, L, g, grad, coord_grads);
            return backward_dense<FILTER, RT_F32, DET>(d, L, g, grad, coord_grads);
    }
}


// dL/dI from dL/dB through Eq. 3 and Eq. 1b.
//  Eq. 3 (x branch, |A_x| >= |A_y|, q = A_y / A_x = I_y / I_x):
//    dB/dA = [[1, q], [-q^3, 1 + 2 q^2]] / sqrt(1 + q^2)   (rows B_x, B_y)
//  and symmetrically on the y branch; the identity at A = 0.
//  Eq. 1b: dA_r/dI_c = sqrt(2) (delta_rc / D - I_r g_c / D^3), g = (I_x, I_y, I_z + 1), D = |g|.
//  The same holds for any half-way vector h in place of g (Eq. 1a: h = I + N,
//  and dA/dI = dA/dN = dA/dh).  Every product and sum is an explicit rounded
//  multiply or fused multiply-add, so that every kernel that inlines this
//  (the backward, the fused step) rounds it the same way.
__device__ __forceinline__ float3 half_grad(float Ix, float Iy, float zp, float gBx, float gBy) {
    float ax = fabsf(Ix), ay = fabsf(Iy);
    float gAx, gAy;
    if (!(fmaxf(ax, ay) >= 1e-30f)) {
        gAx = gBx;
        gAy = gBy;
    } else if (ax >= ay) {
        float q = Iy / Ix;
        float r = 1.0f / sqrtf(fmaf(q, q, 1.0f));
        gAx = __fmul_rn(fmaf(-gBy, __fmul_rn(__fmul_rn(q, q), q), gBx), r);
        gAy = __fmul_rn(fmaf(gBx, q, __fmul_rn(gBy, fmaf(2.0f * q, q, 1.0f))), r);
    } else {
        float p = Ix / Iy;
        float r = 1.0f / sqrtf(fmaf(p, p, 1.0f));
        gAy = __fmul_rn(fmaf(-gBx, __fmul_rn(__fmul_rn(p, p), p), gBy), r);
        gAx = __fmul_rn(fmaf(gBy, p, __fmul_rn(gBx, fmaf(2.0f * p, p, 1.0f))), r);
    }
    float D2 = fmaf(Ix, Ix, fmaf(Iy, Iy, __fmul_rn(zp, zp)));
    if (!(D2 > 1e-30f)) return make_float3(0.f, 0.f, 0.f);
    float invD = 1.0f / sqrtf(D2);
    float k = __fmul_rn(1.41421356237f, invD);
    float k3 = __fmul_rn(__fmul_rn(k, invD), invD);
    float m = __fmul_rn(k3, fmaf(gAx, Ix, __fmul_rn(gAy, Iy)));
    return make_float3(fmaf(-m, Ix, __fmul_rn(k, gAx)), fmaf(-m, Iy, __fmul_rn(k, gAy)), __fmul_rn(-m, zp));
}

__device__ __forceinline__ float3 direction_grad(float Ix, float Iy, float Iz, float gBx, float gBy) {
    return half_grad(Ix, Iy, Iz + 1.0f, gBx, gBy);
}

// dL/du, dL/dv of a bilinear spatial lookup: zero where clamp to edge holds c fixed.
__device__ __forceinline__ float2 uv_grad(const TexDesc& d, float u, float v, float gu, float gv) {
    const float cu = fmaf(u, d.fW, -0.5f), cv = fmaf(v, d.fH, -0.5f);
    float2 r;
    r.x = ((d.wrap & 1) || (cu > -1.0f && cu < d.fW)) ? gu * d.fW : 0.f;
    r.y = ((d.wrap & 2) || (cv > -1.0f && cv < d.fH)) ? gv * d.fH : 0.f;
    return r;
}

// SPEC as in filter_spec: one format for every object, or -1 (dispatch).
template <int FILTER, bool DET, int SPEC>
__device__ __forceinline__ CoordGrad backward_spec(const TexDesc& d, const Lookup<FILTER>& L, float4 g, void* grad,
                                                   bool coord_grads) {
    if constexpr (SPEC < 0)
        return backward_any<FILTER, DET>(d, L, g, grad, coord_grads);
    else
        return backward_layout<FILTER, SPEC, RT_LAYOUT_QUADS, DET>(d, L, g, grad, coord_grads);
}

// UV and direction gradients of one fragment from its weight-coordinate
// gradients: through u w - 1/2 (uv_grad), and through the Note's clamp (zero
// where a coordinate is clamped), Eq. 3 and Eq. 1b (direction_grad).
template <int FILTER>
__device__ __forceinline__ void coord_grads_of(const TexDesc& d, const Lookup<FILTER>& L, const Frag& q,
                                               const CoordGrad& cg, bool want_dir, float2& guv, float3& gdir) {
    if (FILTER == RT_QUADRILINEAR) guv = uv_grad(d, q.u, q.v, cg.gu, cg.gv);
    if (FILTER != RT_NEAREST && want_dir) {
        float gBx = (L.B.x > -d.hi && L.B.x < d.hi) ? cg.gs * d.half_n : 0.f;
        float gBy = (L.B.y > -d.hi && L.B.y < d.hi) ? cg.gt * d.half_n : 0.f;
        gdir = direction_grad(q.x, q.y, q.z, gBx, gBy);
    }
}

// Writes, or with `accumulate` adds to, fragment f's UV and direction gradients
// (either buffer may be absent).
__device__ __forceinline__ void store_coord_grads(int64_t f, float2 guv, float3 gdir, float* dL_duv, float* dL_ddir,
                                                  bool accumulate) {
    if (dL_duv) {
        float2* p = reinterpret_cast<float2*>(dL_duv) + f;
        if (accumulate) {
            float2 o = *p;
            guv.x += o.x;
            guv.y += o.y;
        }
        *p = guv;
    }
    if (dL_ddir) {
        float* p = dL_ddir + 3 * f;
        if (accumulate) {
            gdir.x += p[0];
            gdir.y += p[1];
            gdir.z += p[2];
        }
        p[0] = gdir.x;
        p[1] = gdir.y;
        p[2] = gdir.z;
    }
}

}  // namespace rt

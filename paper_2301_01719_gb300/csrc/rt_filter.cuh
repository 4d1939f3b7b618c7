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

// G-buffer staging.  Kernels that walk fragments are persistent: each warp
// takes 32-fragment chunks c, c + (warps in the grid), ...  and double-buffers
// them in its own slice of shared memory.  While the warp filters chunk c, the
// G-buffer of its next chunk (uv 256 B, dir 384 B, obj 128 B, and optionally a
// 16-byte-per-fragment extra stream such as dL/dout) is already in flight with
// 16-byte cp.async copies that bypass L1 -- so the DRAM latency of the
// G-buffer overlaps the texel gather, and no block-wide barrier is needed.
// Only __syncwarp orders the warp's own copies and reads.
constexpr int kChunk = 32;

template <bool EXTRA>
struct WarpStage {
    float uv[2][2 * kChunk];
    float dir[2][3 * kChunk];
    int obj[2][kChunk];
    float4 extra[EXTRA ? 2 : 1][EXTRA ? kChunk : 1];
};

struct Frag {
    float u, v, x, y, z;
    int o;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Issues the copies of chunk `c` into buffer `b` (a partial last chunk is read
// with plain bounded loads instead; fragments past F become background).
template <bool EXTRA>
__device__ __forceinline__ void stage_chunk(const float* __restrict__ uv, const float* __restrict__ dir,
                                            const int32_t* __restrict__ obj, const float* __restrict__ extra,
                                            int64_t F, int64_t c, int b, WarpStage<EXTRA>& S, int lane) {
    const int64_t f0 = c * kChunk;
    if (f0 + kChunk <= F) {
        // 16 + 24 + 8 (+ 32) sixteen-byte pieces spread over the 32 lanes
        if (lane < 16) cp_async16(&S.uv[b][4 * lane], uv + 2 * f0 + 4 * lane);
        if (lane < 24) cp_async16(&S.dir[b][4 * lane], dir + 3 * f0 + 4 * lane);
        if (lane < 8) cp_async16(&S.obj[b][4 * lane], obj + f0 + 4 * lane);
        if (EXTRA) cp_async16(&S.extra[b][lane], extra + 4 * (f0 + lane));
    } else {
        const int count = (int)(F - f0);
        for (int k = lane; k < 2 * kChunk; k += 32) S.uv[b][k] = k < 2 * count ? uv[2 * f0 + k] : 0.f;
        for (int k = lane; k < 3 * kChunk; k += 32) S.dir[b][k] = k < 3 * count ? dir[3 * f0 + k] : 0.f;
        S.obj[b][lane] = lane < count ? obj[f0 + lane] : -1;
        if (EXTRA)
            S.extra[b][lane] = lane < count ? reinterpret_cast<const float4*>(extra)[f0 + lane]
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <bool EXTRA>
__device__ __forceinline__ Frag read_frag(const WarpStage<EXTRA>& S, int b, int lane) {
    Frag r;
    float2 q = reinterpret_cast<const float2*>(S.uv[b])[lane];
    r.u = q.x;
    r.v = q.y;
    r.x = S.dir[b][3 * lane];
    r.y = S.dir[b][3 * lane + 1];
    r.z = S.dir[b][3 * lane + 2];
    r.o = S.obj[b][lane];
    return r;
}

// Runs body(f, frag, extra) with all 32 lanes of the warp, one fragment per
// lane, persistent over the grid, with the G-buffer of the next chunk
// prefetched.  Lanes past F get a background fragment and f >= F: the body
// must not store for them.  WARPS = warps per block; the block's shared memory
// holds WARPS stages.
template <int WARPS, bool EXTRA, typename Body>
__device__ __forceinline__ void for_each_fragment(const float* __restrict__ uv, const float* __restrict__ dir,
                                                  const int32_t* __restrict__ obj, const float* __restrict__ extra,
                                                  int64_t F, WarpStage<EXTRA>* stages, Body body) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpStage<EXTRA>& S = stages[w];
    const int64_t nchunks = (F + kChunk - 1) / kChunk;
    const int64_t step = (int64_t)gridDim.x * WARPS;
    int64_t c = (int64_t)blockIdx.x * WARPS + w;
    int b = 0;
    if (c < nchunks) stage_chunk<EXTRA>(uv, dir, obj, extra, F, c, 0, S, lane);
    cp_async_commit();
    for (; c < nchunks; c += step, b ^= 1) {
        const int64_t next = c + step;
        if (next < nchunks) stage_chunk<EXTRA>(uv, dir, obj, extra, F, next, b ^ 1, S, lane);
        cp_async_commit();
        cp_async_wait<1>();  // chunk c has landed (the newest group may still be in flight)
        __syncwarp();
        const Frag q = read_frag<EXTRA>(S, b, lane);
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
        if (EXTRA) e = S.extra[EXTRA ? b : 0][EXTRA ? lane : 0];
        __syncwarp();  // every lane has read buffer b before it is refilled
        body(c * kChunk + lane, q, e);
    }
    cp_async_wait<0>();
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

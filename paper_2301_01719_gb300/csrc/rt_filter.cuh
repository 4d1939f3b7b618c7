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
    if (FMT == RT_E4M3_BUCKET_SCALE) sc = __ldg(d.scale + bucket_slot<LAYOUT>(d, i, j));
    t00 = load_texel<FMT>(d.base, texel_index<LAYOUT>(d, i, j, s.k0, t.k0), sc);
    t10 = load_texel<FMT>(d.base, texel_index<LAYOUT>(d, i, j, s.k1, t.k0), sc);
    t01 = load_texel<FMT>(d.base, texel_index<LAYOUT>(d, i, j, s.k0, t.k1), sc);
    t11 = load_texel<FMT>(d.base, texel_index<LAYOUT>(d, i, j, s.k1, t.k1), sc);
}

// Addresses of the taps.  PLANES / QUADS: the four in-bucket texels (s0|s1,
// t0|t1) select four planes (64-bit base indices), the (up to) four buckets
// select spatial offsets inside a plane (32-bit, w h < 2^31).
template <int FMT, int LAYOUT>
__device__ __forceinline__ void load_quadP(const TexDesc& d, int i, int j, const Axis& s, const Axis& t, P4& t00,
                                           P4& t10, P4& t01, P4& t11) {
    float sc = 1.0f;
    if (FMT == RT_E4M3_BUCKET_SCALE) sc = __ldg(d.scale + bucket_slot<LAYOUT>(d, i, j));
    t00 = load_texelP<FMT>(d.base, texel_index<LAYOUT>(d, i, j, s.k0, t.k0), sc);
    t10 = load_texelP<FMT>(d.base, texel_index<LAYOUT>(d, i, j, s.k1, t.k0), sc);
    t01 = load_texelP<FMT>(d.base, texel_index<LAYOUT>(d, i, j, s.k0, t.k1), sc);
    t11 = load_texelP<FMT>(d.base, texel_index<LAYOUT>(d, i, j, s.k1, t.k1), sc);
}

// The planes (64-bit bases, k = (s0,t0) (s1,t0) (s0,t1) (s1,t1)) and the spatial
// offsets (b = (u0,v0) (u1,v0) (u0,v1) (u1,v1)) of a quadrilinear lookup's 16 taps
// on a PLANES / QUADS / palette texture: tap (b, k) is texel pl[k] + o[b].
template <int LAYOUT>
__device__ __forceinline__ void quad_tap_addresses(const TexDesc& d, const Axis& U, const Axis& V, const Axis& S,
                                                   const Axis& T, int64_t (&pl)[4], int (&o)[4]) {
    const int64_t P = d.plane;
    const int64_t p00 = (int64_t)(T.k0 * d.n + S.k0) * P;
    const int64_t ds = (int64_t)(S.k1 - S.k0) * P, dt = (int64_t)(T.k1 - T.k0) * d.n * P;
    pl[0] = p00;
    pl[1] = p00 + ds;
    pl[2] = p00 + dt;
    pl[3] = p00 + dt + ds;
    bucket_slots4<LAYOUT>(d, U.k0, U.k1, V.k0, V.k1, o);
}

// The colour of 16 taps q[bucket][texel]: lerps in s, t, then u, v.
__device__ __forceinline__ P4 quadrilinear_combine(const P4 (&q)[4][4], const Axis& U, const Axis& V, const Axis& S,
                                                   const Axis& T) {
    const f32x2 ws = pack2(S.w, S.w), wt = pack2(T.w, T.w), wu = pack2(U.w, U.w), wv = pack2(V.w, V.w);
    P4 c[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) c[b] = lerpP(lerpP(q[b][0], q[b][1], ws), lerpP(q[b][2], q[b][3], ws), wt);
    return lerpP(lerpP(c[0], c[1], wu), lerpP(c[2], c[3], wu), wv);
}

template <int FMT, int LAYOUT>
__device__ __forceinline__ P4 quadrilinear_planes(const TexDesc& d, const Axis& U, const Axis& V, const Axis& S,
                                                  const Axis& T) {
    int64_t pl[4];
    int o[4];
    quad_tap_addresses<LAYOUT>(d, U, V, S, T, pl, o);
    float sc[4] = {1.f, 1.f, 1.f, 1.f};
    if (FMT == RT_E4M3_BUCKET_SCALE) {
#pragma unroll
        for (int k = 0; k < 4; ++k) sc[k] = __ldg(d.scale + o[k]);
    }
    P4 q[4][4];  // [bucket][texel]
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int k = 0; k < 4; ++k) q[b][k] = load_texelP<FMT>(d.base, checked_texel(d, pl[k] + o[b]), sc[b]);
    return quadrilinear_combine(q, U, V, S, T);
}

template <int FILTER, int FMT, int LAYOUT>
__device__ __forceinline__ float4 filter_taps(const TexDesc& d, const Lookup<FILTER>& L) {
    if (FILTER == RT_NEAREST) {
        float sc = 1.0f;
        if (FMT == RT_E4M3_BUCKET_SCALE) sc = __ldg(d.scale + bucket_slot<LAYOUT>(d, L.u.k0, L.v.k0));
        return toF4(load_texelP<FMT>(d.base, texel_index<LAYOUT>(d, L.u.k0, L.v.k0, L.s.k0, L.t.k0), sc));
    } else if (FILTER == RT_ANGULAR_BILINEAR) {
        P4 a, b, c, e;
        load_quadP<FMT, LAYOUT>(d, L.u.k0, L.v.k0, L.s, L.t, a, b, c, e);
        const f32x2 ws = pack2(L.s.w, L.s.w), wt = pack2(L.t.w, L.t.w);
        return toF4(lerpP(lerpP(a, b, ws), lerpP(c, e, ws), wt));
    } else if (LAYOUT != RT_LAYOUT_ATLAS) {
        return toF4(quadrilinear_planes<FMT, LAYOUT>(d, L.u, L.v, L.s, L.t));
    } else {
        P4 q[2][2][4];
#pragma unroll
        for (int bv = 0; bv < 2; ++bv)
#pragma unroll
            for (int au = 0; au < 2; ++au)
                load_quadP<FMT, LAYOUT>(d, au ? L.u.k1 : L.u.k0, bv ? L.v.k1 : L.v.k0, L.s, L.t, q[bv][au][0],
                                        q[bv][au][1], q[bv][au][2], q[bv][au][3]);
        const f32x2 ws = pack2(L.s.w, L.s.w), wt = pack2(L.t.w, L.t.w), wu = pack2(L.u.w, L.u.w),
                    wv = pack2(L.v.w, L.v.w);
        P4 y[2];
#pragma unroll
        for (int bv = 0; bv < 2; ++bv) {
            P4 c[2];
#pragma unroll
            for (int au = 0; au < 2; ++au)
                c[au] = lerpP(lerpP(q[bv][au][0], q[bv][au][1], ws), lerpP(q[bv][au][2], q[bv][au][3], ws), wt);
            y[bv] = lerpP(c[0], c[1], wu);
        }
        return toF4(lerpP(y[0], y[1], wv));
    }
}

// Dispatch on the object's storage format and layout: owned textures are
// QUADS (bit textures PLANES) or palettes; only a borrowed buffer, always
// FP32, may also be ATLAS or PLANES.
template <int FILTER, int FMT>
__device__ __forceinline__ float4 filter_dense(const TexDesc& d, const Lookup<FILTER>& L) {
    if (d.layout == kLayoutPalette) return filter_taps<FILTER, FMT, kLayoutPalette>(d, L);
    if (FMT == RT_BIT1) return filter_taps<FILTER, FMT, RT_LAYOUT_PLANES>(d, L);
    if (FMT != RT_F32 || d.layout == RT_LAYOUT_QUADS) return filter_taps<FILTER, FMT, RT_LAYOUT_QUADS>(d, L);
    return filter_taps<FILTER, FMT, RT_LAYOUT_PLANES>(d, L);
}

template <int FILTER>
__device__ __forceinline__ float4 filter_any(const TexDesc& d, const Lookup<FILTER>& L) {
    switch (d.fmt) {
        case RT_F16:
            return filter_dense<FILTER, RT_F16>(d, L);
        case RT_BF16:
            return filter_dense<FILTER, RT_BF16>(d, L);
        case RT_E4M3_BUCKET_SCALE:
            return filter_dense<FILTER, RT_E4M3_BUCKET_SCALE>(d, L);
        case RT_BIT1:
            return filter_dense<FILTER, RT_BIT1>(d, L);
        default:
            if (d.layout == RT_LAYOUT_ATLAS) return filter_taps<FILTER, RT_F32, RT_LAYOUT_ATLAS>(d, L);
            return filter_dense<FILTER, RT_F32>(d, L);
    }
}

// SPEC: -1 = any objects (format, layout, palette and repeat mode dispatched
// per fragment); a format = every object of the table is a dense QUADS
// texture of that format in clamp mode, so the fragment code is one path
// (the host picks the instantiation from the table).
template <int FILTER, int SPEC>
__device__ __forceinline__ float4 filter_spec(const TexDesc& d, const Lookup<FILTER>& L) {
    if constexpr (SPEC < 0)
        return filter_any<FILTER>(d, L);
    else
        return filter_taps<FILTER, SPEC, RT_LAYOUT_QUADS>(d, L);
}

// G-buffer staging.  Kernels that walk fragments are persistent: each warp
// takes 32-fragment chunks c, c + (warps in the grid), ...  and double-buffers
// them in its own slice of shared memory.  While the warp filters chunk c, the
// G-buffer of its next chunk (uv 256 B, dir 384 B, obj 128 B, and optionally a
// 16-byte-per-fragment extra stream such as dL/dout) is already in flight with
// 16-byte cp.async copies that bypass L1 -- so the DRAM latency of the
// G-buffer overlaps the texel gather, and no block-wide barrier is needed.
// Only __syncwarp orders the warp's own copies and reads.
//
// A chunk is either 32 consecutive fragments of the flat stream (rt_shade), or
// a tw x th screen tile of a batch of frames (rt_shade_batched): fragment
// (view, y, x) of views x H x W frames.  A block's warps take the tw x th
// sub-tiles of one bx x by block tile, so the warps that share an SM's L1 work
// on one compact screen region: vertically adjacent fragments read the same
// bucket rows.  Block tiles are visited in raster order, frame after frame.
constexpr int kChunk = 32;

// Division of a non-negative 31-bit integer by a fixed divisor d >= 1 with a
// multiply and a shift (the divisor's "magic" reciprocal is prepared on the
// host): q = umulhi(n, mul) >> shift, with shift = ceil(log2 d) and
// mul = ceil(2^(32 + shift) / d) - 2^32 handled as below for d = 1.
struct FastDiv {
    uint32_t d, mul, shift;
    __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const {
        // q = (umulhi(n, mul) + n) >> shift, with the 33-bit sum taken in 64 bits
#ifdef __CUDA_ARCH__
        const uint32_t hi = __umulhi(n, mul);
#else
        const uint32_t hi = (uint32_t)(((uint64_t)n * mul) >> 32);
#endif
        return (uint32_t)(((uint64_t)hi + n) >> shift);
    }
};

// Prepares a FastDiv for divisor d >= 1 (exact for every n < 2^31).
__host__ __device__ inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    uint32_t s = 0;
    while (s < 32 && (1ull << s) < d) ++s;
    f.shift = s;
    // mul = floor(2^32 (2^s - d) / d) + 1
    f.mul = (uint32_t)((((1ull << s) - d) << 32) / d + 1);
    return f;
}

struct Tiling {
    int32_t W, H, views;  // frame size and count; W = H = 0 selects the flat stream
    int32_t tw, th;       // warp tile, tw * th = 32, tw a multiple of 4
    int32_t bx, by;       // block tile in warp tiles, bx * by = warps per block
    int32_t btx, bty;     // block tiles per frame row / column
    int32_t tw_log2, bx_log2;
    FastDiv div_btx, div_frame;  // by btx, by btx * bty
    int64_t frame;        // W * H
};

// A warp's G-buffer buffers: the chunk being processed plus STAGES - 1
// prefetched ones.
// NRM adds a second three-float stream (the per-fragment normal of the
// world-space lookup), staged like dir.
template <bool EXTRA, int STAGES = 2, bool NRM = false>
struct WarpStage {
    float uv[STAGES][2 * kChunk];
    float dir[STAGES][3 * kChunk];
    int obj[STAGES][kChunk];
    float4 extra[EXTRA ? STAGES : 1][EXTRA ? kChunk : 1];
    float nrm[NRM ? STAGES : 1][NRM ? 3 * kChunk : 1];
};

struct Frag {
    float u, v, x, y, z;
    int o;
    float nx, ny, nz;  // NRM streams only
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

// Geometry of one chunk: the first fragment of each of its rows, whether the
// whole chunk can be copied with aligned 16-byte pieces, and this lane's
// fragment (-1 = none).
struct ChunkGeom {
    int64_t row0;    // fragment index of (x0, y0)
    int64_t pitch;   // fragment stride between rows
    int tw, th, tw_log2;
    bool fast;
    int64_t f;       // this lane's fragment, -1 outside the frame / stream
};

template <int WARPS, bool TILED>
__device__ __forceinline__ ChunkGeom chunk_geom(const Tiling& T, int64_t F, int64_t c, int lane) {
    ChunkGeom g;
    if (!TILED) {
        g.row0 = c * kChunk;
        g.pitch = kChunk;
        g.tw = kChunk;
        g.th = 1;
        g.tw_log2 = 5;
        g.fast = g.row0 + kChunk <= F;
        g.f = g.row0 + lane < F ? g.row0 + lane : -1;
        return g;
    }
    // block tile bt, sub-tile w; chunk indices of the tiled walk fit 31 bits
    const uint32_t cc = (uint32_t)c;
    const uint32_t bt = cc / WARPS, w = cc % WARPS;
    const uint32_t view = T.div_frame.div(bt);
    const uint32_t r = bt - view * T.div_frame.d;
    const uint32_t tyb = T.div_btx.div(r), txb = r - tyb * T.div_btx.d;
    const int x0 = (int)((txb * T.bx + (w & (T.bx - 1))) << T.tw_log2);
    const int y0 = (int)((tyb * T.by + (w >> T.bx_log2)) * T.th);
    g.tw = T.tw;
    g.th = T.th;
    g.tw_log2 = T.tw_log2;
    g.pitch = T.W;
    g.row0 = (int64_t)view * T.frame + (int64_t)y0 * T.W + x0;
    g.fast = (x0 + T.tw <= T.W) && (y0 + T.th <= T.H) && ((T.W & 3) == 0);
    const int ly = lane >> T.tw_log2, lx = lane & (T.tw - 1);
    g.f = (x0 + lx < T.W && y0 + ly < T.H) ? g.row0 + (int64_t)ly * T.W + lx : -1;
    return g;
}

// Issues the copies of one chunk into buffer `b` (a chunk that is not entirely
// inside the frame or not 16-byte aligned is read with plain bounded loads
// instead; lanes without a fragment become background).
template <bool EXTRA, int STAGES, bool NRM>
__device__ __forceinline__ void stage_chunk(const float* __restrict__ uv, const float* __restrict__ dir,
                                            const int32_t* __restrict__ obj, const float* __restrict__ extra,
                                            const float* __restrict__ nrm, const ChunkGeom& g, int b,
                                            WarpStage<EXTRA, STAGES, NRM>& S, int lane) {
    if (g.fast) {
        // 24 pieces of dir, 16 of uv, 8 of obj: lanes 0-23 take dir, 16-31 uv,
        // 24-31 obj.  Shared memory holds the chunk in lane order (lane = row
        // tw + column), so piece q covers shared floats 4q..4q+3 of its stream,
        // all in one row: row k = (first lane of the piece) >> log2(tw).
        const int lg = g.tw_log2;
        if (lane < 24) {
            const int m = 4 * lane, k = (m / 3) >> lg;
            const int64_t src = 3 * (g.row0 + (int64_t)k * g.pitch) + (m - 3 * (k << lg));
            cp_async16(&S.dir[b][m], dir + src);
            if (NRM) cp_async16(&S.nrm[NRM ? b : 0][NRM ? m : 0], nrm + src);
        }
        if (lane >= 16) {
            const int m = 4 * (lane - 16), k = (m >> 1) >> lg;
            cp_async16(&S.uv[b][m], uv + 2 * (g.row0 + (int64_t)k * g.pitch) + (m - 2 * (k << lg)));
        }
        if (lane >= 24) {
            const int m = 4 * (lane - 24), k = m >> lg;
            cp_async16(&S.obj[b][m], obj + (g.row0 + (int64_t)k * g.pitch) + (m - (k << lg)));
        }
        if (EXTRA) cp_async16(&S.extra[b][lane], extra + 4 * g.f);
    } else {
        const int64_t f = g.f;
        if (f >= 0) {
            S.uv[b][2 * lane] = uv[2 * f];
            S.uv[b][2 * lane + 1] = uv[2 * f + 1];
            S.dir[b][3 * lane] = dir[3 * f];
            S.dir[b][3 * lane + 1] = dir[3 * f + 1];
            S.dir[b][3 * lane + 2] = dir[3 * f + 2];
            S.obj[b][lane] = obj[f];
            if (NRM) {
                S.nrm[NRM ? b : 0][NRM ? 3 * lane : 0] = nrm[3 * f];
                S.nrm[NRM ? b : 0][NRM ? 3 * lane + 1 : 0] = nrm[3 * f + 1];
                S.nrm[NRM ? b : 0][NRM ? 3 * lane + 2 : 0] = nrm[3 * f + 2];
            }
        } else {
            S.uv[b][2 * lane] = S.uv[b][2 * lane + 1] = 0.f;
            S.dir[b][3 * lane] = S.dir[b][3 * lane + 1] = S.dir[b][3 * lane + 2] = 0.f;
            S.obj[b][lane] = -1;
            if (NRM)
                S.nrm[NRM ? b : 0][NRM ? 3 * lane : 0] = S.nrm[NRM ? b : 0][NRM ? 3 * lane + 1 : 0] =
                    S.nrm[NRM ? b : 0][NRM ? 3 * lane + 2 : 0] = 0.f;
        }
        if (EXTRA)
            S.extra[b][lane] = f >= 0 ? reinterpret_cast<const float4*>(extra)[f] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <bool EXTRA, int STAGES, bool NRM>
__device__ __forceinline__ Frag read_frag(const WarpStage<EXTRA, STAGES, NRM>& S, int b, int lane) {
    Frag r;
    float2 q = reinterpret_cast<const float2*>(S.uv[b])[lane];
    r.u = q.x;
    r.v = q.y;
    r.x = S.dir[b][3 * lane];
    r.y = S.dir[b][3 * lane + 1];
    r.z = S.dir[b][3 * lane + 2];
    r.o = S.obj[b][lane];
    r.nx = r.ny = r.nz = 0.f;
    if (NRM) {
        r.nx = S.nrm[NRM ? b : 0][NRM ? 3 * lane : 0];
        r.ny = S.nrm[NRM ? b : 0][NRM ? 3 * lane + 1 : 0];
        r.nz = S.nrm[NRM ? b : 0][NRM ? 3 * lane + 2 : 0];
    }
    return r;
}

template <bool TILED>
__device__ __forceinline__ int64_t chunk_count(const Tiling& T, int64_t F, int warps) {
    if (!TILED) return (F + kChunk - 1) / kChunk;
    return (int64_t)T.btx * T.bty * T.views * warps;
}

// Runs body(f, frag, extra) with all 32 lanes of the warp, one fragment per
// lane, persistent over the grid, with the G-buffer of the next STAGES - 1
// chunks prefetched.  Lanes without a fragment get a background fragment and
// f = -1: the body must not store for them.  WARPS = warps per block; the
// block's shared memory holds WARPS stages.
template <int WARPS, bool EXTRA, bool TILED, int STAGES, bool NRM = false, typename Body>
__device__ __forceinline__ void for_each_fragment(const float* __restrict__ uv, const float* __restrict__ dir,
                                                  const int32_t* __restrict__ obj, const float* __restrict__ extra,
                                                  int64_t F, const Tiling& T, WarpStage<EXTRA, STAGES, NRM>* stages,
                                                  Body body, const float* __restrict__ nrm = nullptr) {
    constexpr int kStages = STAGES;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    WarpStage<EXTRA, STAGES, NRM>& S = stages[w];
    const int64_t nchunks = chunk_count<TILED>(T, F, WARPS);
    const int64_t step = (int64_t)gridDim.x * WARPS;
    int64_t c = (int64_t)blockIdx.x * WARPS + w;
    // fk[k]: this lane's fragment of chunk c + k * step, staged in buffer (b + k) % kStages
    int64_t fk[kStages];
#pragma unroll
    for (int k = 0; k < kStages - 1; ++k) {
        const ChunkGeom g = chunk_geom<WARPS, TILED>(T, F, c + k * step, lane);
        if (c + k * step < nchunks) stage_chunk<EXTRA, STAGES, NRM>(uv, dir, obj, extra, nrm, g, k, S, lane);
        cp_async_commit();
        fk[k] = g.f;
    }
    int b = 0;
    for (; c < nchunks; c += step) {
        const int64_t ahead = c + (kStages - 1) * step;
        const int bl = b + kStages - 1 >= kStages ? b - 1 : b + kStages - 1;  // (b + kStages - 1) % kStages
        const ChunkGeom g = chunk_geom<WARPS, TILED>(T, F, ahead, lane);
        if (ahead < nchunks) stage_chunk<EXTRA, STAGES, NRM>(uv, dir, obj, extra, nrm, g, bl, S, lane);
        cp_async_commit();
        fk[kStages - 1] = g.f;
        cp_async_wait<kStages - 1>();  // chunk c has landed (newer groups may still be in flight)
        __syncwarp();
        const Frag q = read_frag<EXTRA, STAGES, NRM>(S, b, lane);
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
        if (EXTRA) e = S.extra[EXTRA ? b : 0][EXTRA ? lane : 0];
        __syncwarp();  // every lane has read buffer b before it is refilled
        body(fk[0], q, e);
#pragma unroll
        for (int k = 0; k < kStages - 1; ++k) fk[k] = fk[k + 1];
        b = b + 1 == kStages ? 0 : b + 1;
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
    // 0 * t is 0 for finite t and NaN for an infinity or a NaN: one test covers all five inputs
    const float probe = fmaf(z, 0.f, fmaf(y, 0.f, fmaf(x, 0.f, fmaf(v, 0.f, u * 0.f))));
    if (probe != 0.f) {
        atomicOr(status, ST_NONFINITE);
        return false;
    }
    return true;
}

// A world-space fragment's normal must be finite (status bit otherwise).
__device__ __forceinline__ bool normal_valid(float3 N, unsigned* status) {
    const float probe = fmaf(N.z, 0.f, fmaf(N.y, 0.f, N.x * 0.f));
    if (probe != 0.f) {
        atomicOr(status, ST_NONFINITE);
        return false;
    }
    return true;
}

}  // namespace rt

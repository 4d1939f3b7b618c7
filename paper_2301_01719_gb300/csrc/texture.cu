// texture.cu -- texture set-up kernels: encoding, read-back, lobe fill, layout
// conversion, and the footprint counter used to compute algorithmic bytes.
#include "launch.h"
#include "rt_device.cuh"
#include "rt_filter.cuh"
#include "rt_encode.cuh"
#include "rt_internal.h"

namespace rt {

constexpr int kThreads = 256;

static inline unsigned blocks_for(int64_t items) { return (unsigned)((items + kThreads - 1) / kThreads); }

// FP32 source (any layout) -> FP32 / FP16 / BF16 storage in dst_layout (PLANES
// or QUADS), one thread per texel (the padding of a QUADS buffer is not written).
__global__ void encode_elementwise(const float4* __restrict__ src, int src_layout, void* __restrict__ dst,
                                   int dst_layout, int W, int H, int n, int fmt, int64_t total) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int i, j, s, t;
    planes_coords(idx, W, H, n, i, j, s, t);
    const float4 v = src[index_in(src_layout, W, H, n, i, j, s, t)];
    const int64_t o = index_in(dst_layout, W, H, n, i, j, s, t);
    if (fmt == RT_F32)
        reinterpret_cast<float4*>(dst)[o] = v;
    else if (fmt == RT_F16)
        reinterpret_cast<uint2*>(dst)[o] = pack_f16(v);
    else
        reinterpret_cast<uint2*>(dst)[o] = pack_bf16(v);
}

// FP32 source -> E4M3 + per-bucket scale (stored at the bucket's slot of
// dst_layout), one thread per bucket (amax pass, then encode pass).
__global__ void encode_e4m3_buckets(const float4* __restrict__ src, int src_layout, unsigned* __restrict__ dst,
                                    float* __restrict__ scale, int dst_layout, int W, int H, int n) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)W * H) return;
    int j = (int)(b / W), i = (int)(b - (int64_t)j * W);
    float amax = 0.0f;
    for (int t = 0; t < n; ++t)
        for (int s = 0; s < n; ++s) amax = fmaxf(amax, amax4(src[index_in(src_layout, W, H, n, i, j, s, t)]));
    float sc = bucket_scale(amax);
    scale[slot_in(dst_layout, W, i, j)] = sc;
    for (int t = 0; t < n; ++t)
        for (int s = 0; s < n; ++s)
            dst[index_in(dst_layout, W, H, n, i, j, s, t)] = pack_e4m3(src[index_in(src_layout, W, H, n, i, j, s, t)], sc);
}

// FP32 source -> 1-bit storage: bit = (channel 0 >= 1/2); one thread per 32-bit word.
__global__ void encode_bits(const float4* __restrict__ src, int src_layout, unsigned* __restrict__ dst, int W, int H,
                            int n, int64_t total) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w * 32 >= total) return;
    unsigned word = 0;
    for (int k = 0; k < 32; ++k) {
        const int64_t idx = w * 32 + k;
        if (idx >= total) break;
        int i, j, s, t;
        planes_coords(idx, W, H, n, i, j, s, t);
        if (src[index_in(src_layout, W, H, n, i, j, s, t)].x >= 0.5f) word |= 1u << k;
    }
    dst[w] = word;
}

cudaError_t launch_encode(const float* src, int src_layout, void* dst, float* scale, int W, int H, int n, int fmt,
                          int dst_layout, cudaStream_t stream) {
    if (fmt == RT_BIT1) {
        const int64_t total = (int64_t)W * H * n * n;
        encode_bits<<<blocks_for((total + 31) / 32), kThreads, 0, stream>>>(
            reinterpret_cast<const float4*>(src), src_layout, reinterpret_cast<unsigned*>(dst), W, H, n, total);
    } else if (fmt == RT_E4M3_BUCKET_SCALE) {
        int64_t buckets = (int64_t)W * H;
        encode_e4m3_buckets<<<blocks_for(buckets), kThreads, 0, stream>>>(
            reinterpret_cast<const float4*>(src), src_layout, reinterpret_cast<unsigned*>(dst), scale, dst_layout, W,
            H, n);
    } else {
        int64_t total = (int64_t)W * H * n * n;
        encode_elementwise<<<blocks_for(total), kThreads, 0, stream>>>(reinterpret_cast<const float4*>(src),
                                                                       src_layout, dst, dst_layout, W, H, n, fmt,
                                                                       total);
    }
    return cudaGetLastError();
}

// Stored codes (src_layout: PLANES or QUADS) -> codes in dst_layout; T is the
// per-texel code type; one thread per texel (padding is not written).
template <typename T>
__global__ void read_codes(const T* __restrict__ src, int src_layout, T* __restrict__ dst, int W, int H, int n,
                           int dst_layout, int64_t total) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int i, j, s, t;
    planes_coords(idx, W, H, n, i, j, s, t);
    dst[index_in(dst_layout, W, H, n, i, j, s, t)] = src[index_in(src_layout, W, H, n, i, j, s, t)];
}

// Per-bucket scales stored at their slots of src_layout -> row-major h x w.
__global__ void read_scales(const float* __restrict__ src, int src_layout, float* __restrict__ dst, int W, int H) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)W * H) return;
    const int j = (int)(b / W), i = (int)(b - (int64_t)j * W);
    dst[b] = src[slot_in(src_layout, W, i, j)];
}

// 1-bit storage -> one byte (0 or 1) per texel in dst_layout.
__global__ void read_bits(const unsigned* __restrict__ src, uint8_t* __restrict__ dst, int W, int H, int n,
                          int dst_layout, int64_t total) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int i, j, s, t;
    planes_coords(idx, W, H, n, i, j, s, t);
    int64_t o = index_in(dst_layout, W, H, n, i, j, s, t);
    dst[o] = (uint8_t)((src[idx >> 5] >> (unsigned)(idx & 31)) & 1u);
}

cudaError_t launch_read(const void* src, int src_layout, const float* scale, int fmt, int W, int H, int n,
                        int dst_layout, void* dst, float* scale_dst, cudaStream_t stream) {
    int64_t total = (int64_t)W * H * n * n;
    unsigned g = blocks_for(total);
    if (fmt == RT_BIT1)  // bit textures are always PLANES
        read_bits<<<g, kThreads, 0, stream>>>(reinterpret_cast<const unsigned*>(src), reinterpret_cast<uint8_t*>(dst),
                                              W, H, n, dst_layout, total);
    else if (fmt == RT_F32)
        read_codes<float4><<<g, kThreads, 0, stream>>>(reinterpret_cast<const float4*>(src), src_layout,
                                                       reinterpret_cast<float4*>(dst), W, H, n, dst_layout, total);
    else if (fmt == RT_E4M3_BUCKET_SCALE)
        read_codes<unsigned><<<g, kThreads, 0, stream>>>(reinterpret_cast<const unsigned*>(src), src_layout,
                                                         reinterpret_cast<unsigned*>(dst), W, H, n, dst_layout, total);
    else
        read_codes<uint2><<<g, kThreads, 0, stream>>>(reinterpret_cast<const uint2*>(src), src_layout,
                                                      reinterpret_cast<uint2*>(dst), W, H, n, dst_layout, total);
    if (scale && scale_dst)
        read_scales<<<blocks_for((int64_t)W * H), kThreads, 0, stream>>>(scale, src_layout, scale_dst, W, H);
    return cudaGetLastError();
}

__device__ __forceinline__ float4 lobe_value(const float* P, float3 I) {
    float c = I.x * P[3] + I.y * P[4] + I.z * P[5];
    float l = c > 0.f ? powf(c, P[6]) : 0.f;
    return make_float4(P[0] * l, P[1] * l, P[2] * l, l);
}

__global__ void fill_lobes_kernel(const float* __restrict__ params, void* __restrict__ dst, float* __restrict__ scale,
                                  int layout, int W, int H, int n, int fmt) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (int64_t)W * H) return;
    int j = (int)(b / W), i = (int)(b - (int64_t)j * W);
    float P[8];
    const float4* p4 = reinterpret_cast<const float4*>(params) + 2 * b;
    float4 a = p4[0], c = p4[1];
    P[0] = a.x; P[1] = a.y; P[2] = a.z; P[3] = a.w;
    P[4] = c.x; P[5] = c.y; P[6] = c.z; P[7] = c.w;
    float sc = 1.0f;
    if (fmt == RT_E4M3_BUCKET_SCALE) {
        float amax = 0.f;
        for (int t = 0; t < n; ++t)
            for (int s = 0; s < n; ++s) amax = fmaxf(amax, amax4(lobe_value(P, texel_centre_direction(s, t, n))));
        sc = bucket_scale(amax);
        scale[slot_in(layout, W, i, j)] = sc;
    }
    for (int t = 0; t < n; ++t)
        for (int s = 0; s < n; ++s) {
            float4 v = lobe_value(P, texel_centre_direction(s, t, n));
            int64_t idx = index_in(layout, W, H, n, i, j, s, t);
            if (fmt == RT_F32)
                reinterpret_cast<float4*>(dst)[idx] = v;
            else if (fmt == RT_F16)
                reinterpret_cast<uint2*>(dst)[idx] = pack_f16(v);
            else if (fmt == RT_BF16)
                reinterpret_cast<uint2*>(dst)[idx] = pack_bf16(v);
            else
                reinterpret_cast<unsigned*>(dst)[idx] = pack_e4m3(v, sc);
        }
}

cudaError_t launch_fill_lobes(const float* params, void* dst, float* scale, int layout, int W, int H, int n, int fmt,
                              cudaStream_t stream) {
    int64_t buckets = (int64_t)W * H;
    fill_lobes_kernel<<<blocks_for(buckets), kThreads, 0, stream>>>(params, dst, scale, layout, W, H, n, fmt);
    return cudaGetLastError();
}

__global__ void convert_kernel(const float4* __restrict__ src, int src_layout, float4* __restrict__ dst,
                               int dst_layout, int W, int H, int n, int64_t total) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int i, j, s, t;
    planes_coords(idx, W, H, n, i, j, s, t);
    dst[index_in(dst_layout, W, H, n, i, j, s, t)] = src[index_in(src_layout, W, H, n, i, j, s, t)];
}

__global__ void check_index_kernel(const uint32_t* __restrict__ index, int64_t count, uint32_t K, unsigned* bad) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count && index[k] >= K) atomicOr(bad, 1u);
}

cudaError_t launch_check_index(const uint32_t* index, int64_t count, uint32_t K, unsigned* bad, cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    check_index_kernel<<<blocks_for(count), kThreads, 0, stream>>>(index, count, K, bad);
    return cudaGetLastError();
}

cudaError_t launch_convert(const float* src, int src_layout, float* dst, int dst_layout, int W, int H, int n,
                           cudaStream_t stream) {
    int64_t total = (int64_t)W * H * n * n;
    convert_kernel<<<blocks_for(total), kThreads, 0, stream>>>(reinterpret_cast<const float4*>(src), src_layout,
                                                               reinterpret_cast<float4*>(dst), dst_layout, W, H, n,
                                                               total);
    return cudaGetLastError();
}

// Footprint: one bit per texel of every object (PLANES numbering), set for
// every tap the forward kernel reads.
template <int FILTER>
__global__ void __launch_bounds__(kThreads) footprint_kernel(const TexDesc* __restrict__ table, int n_obj,
                                                            const float* __restrict__ uv,
                                                            const float* __restrict__ dir,
                                                            const int32_t* __restrict__ obj, int64_t F,
                                                            uint32_t* __restrict__ bitmap,
                                                            const int64_t* __restrict__ word_offset,
                                                            unsigned* status) {
    __shared__ WarpStage<false> stages[kThreads / 32];
    const Tiling flat = flat_tiling();
    for_each_fragment<kThreads / 32, false, false, 2>(uv, dir, obj, nullptr, F, flat, stages,
                                                   [&](int64_t, const Frag& q, float4) {
        TexDesc d;
        if (!fragment_valid(table, n_obj, q.o, q.u, q.v, q.x, q.y, q.z, status, d)) return;
        Lookup<FILTER> L = locate<FILTER>(d, q.u, q.v, q.x, q.y, q.z);
        const int64_t base = word_offset[q.o] * 32;
        const int nu = FILTER == RT_QUADRILINEAR ? 2 : 1;
        const int ns = FILTER == RT_NEAREST ? 1 : 2;
        for (int b = 0; b < nu; ++b)
            for (int a = 0; a < nu; ++a)
                for (int t = 0; t < ns; ++t)
                    for (int p = 0; p < ns; ++p) {
                        const int i = a ? L.u.k1 : L.u.k0, j = b ? L.v.k1 : L.v.k0;
                        const int s = p ? L.s.k1 : L.s.k0, tt = t ? L.t.k1 : L.t.k0;
                        int64_t bit = base + (d.layout == kLayoutPalette
                                                  ? texel_index<kLayoutPalette>(d, i, j, s, tt)
                                                  : texel_index<RT_LAYOUT_PLANES>(d, i, j, s, tt));
                        atomicOr(bitmap + (bit >> 5), 1u << (bit & 31));
                    }
    });
}

template <int FILTER>
static cudaError_t launch_footprint_t(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                      const int32_t* obj, int64_t F, uint32_t* bitmap, const int64_t* word_offset,
                                      unsigned* status, cudaStream_t stream) {
    const unsigned grid = persistent_grid(footprint_kernel<FILTER>, kThreads, (F + kChunk - 1) / kChunk);
    footprint_kernel<FILTER><<<grid, kThreads, 0, stream>>>(table, n_obj, uv, dir, obj, F, bitmap, word_offset,
                                                            status);
    return cudaGetLastError();
}

cudaError_t launch_footprint_mark(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                  const int32_t* obj, int64_t F, int filter, uint32_t* bitmap,
                                  const int64_t* word_offset, unsigned* status, cudaStream_t stream) {
    if (filter == RT_NEAREST)
        return launch_footprint_t<RT_NEAREST>(table, n_obj, uv, dir, obj, F, bitmap, word_offset, status, stream);
    if (filter == RT_ANGULAR_BILINEAR)
        return launch_footprint_t<RT_ANGULAR_BILINEAR>(table, n_obj, uv, dir, obj, F, bitmap, word_offset, status,
                                                       stream);
    return launch_footprint_t<RT_QUADRILINEAR>(table, n_obj, uv, dir, obj, F, bitmap, word_offset, status, stream);
}

__global__ void popcount_kernel(const uint32_t* __restrict__ bitmap, int64_t words, unsigned long long* count) {
    unsigned long long local = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x)
        local += __popc(bitmap[w]);
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xFFFFFFFFu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

cudaError_t launch_popcount(const uint32_t* bitmap, int64_t words, unsigned long long* count, cudaStream_t stream) {
    if (words <= 0) return cudaSuccess;
    int64_t b = (words + kThreads - 1) / kThreads;
    unsigned grid = (unsigned)(b < 4096 ? b : 4096);
    popcount_kernel<<<grid, kThreads, 0, stream>>>(bitmap, words, count);
    return cudaGetLastError();
}

}  // namespace rt

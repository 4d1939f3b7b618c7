// kmeans.cu -- the encoder of palette textures: Lloyd's k-means over the
// buckets of a dense texture, each bucket a vector of n^2 x 4 values.
//
// Centroids are stored like a K x 1 texture in PLANES order: centroid k,
// texel (s, t) at float4 index (t n + s) K + k.
//
// Assignment is a distance matrix contraction (w h buckets x K centroids over
// n^2 x 4 values) with an argmin epilogue, in FP32 on the CUDA cores: a block
// holds 128 buckets and sweeps the centroids 64 at a time, 4 texels of each per
// shared-memory stage; each thread accumulates 8 x 4 dot products and keeps
// the running (distance, index) minimum of its 8 rows, ties to the lower
// index.  |x - c|^2 is ranked as |c|^2 - 2 x.c (|x|^2 is added for the
// reported distance only).
//
// Update: per-centroid counts, their prefix sums and a scatter of the bucket
// numbers group every cluster's members; one block per centroid then sums its
// members in FP64 (one thread per texel) and writes the mean rounded to FP32.
// Empty clusters keep their centroid.
#include "rt_device.cuh"
#include "rt_internal.h"

namespace rt {

constexpr int kAM = 128;  // buckets per block
constexpr int kAN = 64;   // centroids per sweep step
constexpr int kAP = 4;    // texels per shared-memory stage
constexpr int kAThreads = 256;

// Texel p = t n + s of bucket (i, j) of a dense texture (ATLAS, PLANES or QUADS).
template <int FMT, int LAYOUT>
__device__ __forceinline__ float4 bucket_texel(const TexDesc& d, int i, int j, int p, float sc) {
    if (LAYOUT == RT_LAYOUT_ATLAS)
        return load_texel<FMT>(d.base, texel_index<RT_LAYOUT_ATLAS>(d, i, j, p % d.n, p / d.n), sc);
    return load_texel<FMT>(d.base, checked_texel(d, (int64_t)p * d.plane + bucket_slot<LAYOUT>(d, i, j)), sc);
}

// The E4M3 scale of bucket (i, j) (1 for the other formats).
template <int FMT, int LAYOUT>
__device__ __forceinline__ float bucket_scale_of(const TexDesc& d, int i, int j) {
    return FMT == RT_E4M3_BUCKET_SCALE ? __ldg(d.scale + bucket_slot<LAYOUT>(d, i, j)) : 1.0f;
}

__device__ __forceinline__ float dot4f(float4 a, float4 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

template <int FMT, int LAYOUT>
__global__ void __launch_bounds__(kAThreads, 2) kmeans_assign_kernel(TexDesc d, int K, const float4* __restrict__ C,
                                                                  uint32_t* __restrict__ index,
                                                                  float* __restrict__ dist) {
    __shared__ float4 Xs[kAP][kAM];
    __shared__ float4 Cs[kAP][kAN];
    __shared__ float cnp[kAP][kAN];
    __shared__ float cn[kAN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t B = (int64_t)d.W * d.H;
    const int64_t b0 = (int64_t)blockIdx.x * kAM;
    const int planes = d.n * d.n;
    // loader role for X: bucket b0 + lb, stages q = tid / 128 and q + 2
    const int lb = tid & (kAM - 1);
    const int64_t bb = b0 + lb;
    const bool bvalid = bb < B;
    int bi = 0, bj = 0;
    float sc = 1.0f;
    if (bvalid) {
        bj = (int)(bb / d.W);
        bi = (int)(bb - (int64_t)bj * d.W);
        sc = bucket_scale_of<FMT, LAYOUT>(d, bi, bj);
    }
    // loader role for C: stage cq, centroid ck of the sweep step
    const int cq = tid >> 6, ck = tid & (kAN - 1);

    float best[8], xn[8];
    int bestk[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        best[r] = INFINITY;
        bestk[r] = 0;
        xn[r] = 0.0f;
    }
    for (int k0 = 0; k0 < K; k0 += kAN) {
        float acc[8][4];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0.0f;
        float cnorm = 0.0f;  // |c|^2 partial of centroid k0 + ck over stages cq
        for (int p0 = 0; p0 < planes; p0 += kAP) {
            __syncthreads();
            for (int q = tid >> 7; q < kAP; q += 2) {
                const int p = p0 + q;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (bvalid && p < planes) v = bucket_texel<FMT, LAYOUT>(d, bi, bj, p, sc);
                Xs[q][lb] = v;
            }
            {
                const int p = p0 + cq, k = k0 + ck;
                float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
                if (p < planes && k < K) c = __ldg(C + (int64_t)p * K + k);
                Cs[cq][ck] = c;
                cnorm += dot4f(c, c);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kAP; ++q) {
                float4 c[4];
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) c[cc] = Cs[q][tx + 16 * cc];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float4 x = Xs[q][ty * 8 + r];
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) acc[r][cc] += dot4f(x, c[cc]);
                    if (k0 == 0 && tx == 0) xn[r] += dot4f(x, x);
                }
            }
        }
        __syncthreads();
        cnp[cq][ck] = cnorm;
        __syncthreads();
        if (tid < kAN) cn[tid] = (cnp[0][tid] + cnp[1][tid]) + (cnp[2][tid] + cnp[3][tid]);
        __syncthreads();
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int k = k0 + tx + 16 * cc;
            if (k >= K) continue;
            const float c2 = cn[tx + 16 * cc];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float dd = fmaf(-2.0f, acc[r][cc], c2);
                if (dd < best[r]) {  // k grows within a thread: equal distances keep the lower index
                    best[r] = dd;
                    bestk[r] = k;
                }
            }
        }
    }
    // reduce over the 16 threads (tx) of each row group; they share a half-warp
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
        for (int off = 8; off >= 1; off >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best[r], off);
            const int ok = __shfl_xor_sync(0xffffffffu, bestk[r], off);
            if (ob < best[r] || (ob == best[r] && ok < bestk[r])) {
                best[r] = ob;
                bestk[r] = ok;
            }
        }
    }
    if (tx == 0) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int64_t b = b0 + ty * 8 + r;
            if (b >= B) continue;
            index[b] = (uint32_t)bestk[r];
            if (dist) dist[b] = fmaxf(best[r] + xn[r], 0.0f);
        }
    }
}

template <int FMT, int LAYOUT>
__global__ void kmeans_init_kernel(TexDesc d, int K, const int32_t* __restrict__ buckets, float4* __restrict__ C,
                                   unsigned* status) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int planes = d.n * d.n;
    if (e >= (int64_t)K * planes) return;
    const int p = (int)(e / K), k = (int)(e - (int64_t)p * K);
    const int64_t B = (int64_t)d.W * d.H;
    int64_t b = buckets[k];
    if (b < 0 || b >= B) {
        atomicOr(status, ST_BAD_ARG);
        b = b < 0 ? 0 : B - 1;
    }
    const int j = (int)(b / d.W), i = (int)(b - (int64_t)j * d.W);
    C[(int64_t)p * K + k] = bucket_texel<FMT, LAYOUT>(d, i, j, p, bucket_scale_of<FMT, LAYOUT>(d, i, j));
}

__global__ void kmeans_count_kernel(const uint32_t* __restrict__ index, int64_t B, int K, uint32_t* counts,
                                    unsigned* status) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const uint32_t k = index[b];
    if (k >= (uint32_t)K) {
        atomicOr(status, ST_BAD_ARG);
        return;
    }
    atomicAdd(counts + k, 1u);
}

// Exclusive prefix sum of counts[0..K) into offsets[0..K] (one block).
__global__ void __launch_bounds__(1024) kmeans_scan_kernel(const uint32_t* __restrict__ counts, int K,
                                                           uint32_t* __restrict__ offsets) {
    __shared__ uint32_t part[1024];
    const int t = threadIdx.x;
    const int per = (K + 1023) / 1024;
    const int lo = t * per, hi = min(K, lo + per);
    uint32_t s = 0;
    for (int k = lo; k < hi; ++k) s += counts[k];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // inclusive scan of the partial sums
        const uint32_t v = t >= off ? part[t - off] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = t ? part[t - 1] : 0u;
    for (int k = lo; k < hi; ++k) {
        offsets[k] = run;
        run += counts[k];
    }
    if (t == 1023) offsets[K] = part[1023];
}

__global__ void kmeans_scatter_kernel(const uint32_t* __restrict__ index, int64_t B, int K,
                                      const uint32_t* __restrict__ offsets, uint32_t* cursor,
                                      uint32_t* __restrict__ members) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const uint32_t k = index[b];
    if (k >= (uint32_t)K) return;
    members[offsets[k] + atomicAdd(cursor + k, 1u)] = (uint32_t)b;
}

template <int FMT, int LAYOUT>
__global__ void __launch_bounds__(256) kmeans_mean_kernel(TexDesc d, int K, const uint32_t* __restrict__ offsets,
                                                          const uint32_t* __restrict__ members,
                                                          float4* __restrict__ C) {
    const int k = blockIdx.x;
    const uint32_t m0 = offsets[k], m1 = offsets[k + 1];
    if (m1 == m0) return;  // empty: keep the centroid
    const int planes = d.n * d.n;
    const double inv = 1.0 / (double)(m1 - m0);
    for (int p = threadIdx.x; p < planes; p += blockDim.x) {
        double sx = 0.0, sy = 0.0, sz = 0.0, sw = 0.0;
        for (uint32_t m = m0; m < m1; ++m) {
            const int64_t b = members[m];
            const int j = (int)(b / d.W), i = (int)(b - (int64_t)j * d.W);
            const float4 v = bucket_texel<FMT, LAYOUT>(d, i, j, p, bucket_scale_of<FMT, LAYOUT>(d, i, j));
            sx += v.x;
            sy += v.y;
            sz += v.z;
            sw += v.w;
        }
        C[(int64_t)p * K + k] = make_float4((float)(sx * inv), (float)(sy * inv), (float)(sz * inv), (float)(sw * inv));
    }
}

static unsigned blocks(int64_t items, int threads) { return (unsigned)((items + threads - 1) / threads); }

template <template <int, int> class Launch, int LAYOUT, typename... Args>
static cudaError_t dispatch_format(const TexDesc& d, Args... args) {
    switch (d.fmt) {
        case RT_F16:
            return Launch<RT_F16, LAYOUT>::run(d, args...);
        case RT_BF16:
            return Launch<RT_BF16, LAYOUT>::run(d, args...);
        case RT_E4M3_BUCKET_SCALE:
            return Launch<RT_E4M3_BUCKET_SCALE, LAYOUT>::run(d, args...);
        default:
            return Launch<RT_F32, LAYOUT>::run(d, args...);
    }
}

// Calls Launch<FMT, LAYOUT>::run(args...) for the texture's format and layout (dense textures only).
template <template <int, int> class Launch, typename... Args>
static cudaError_t dispatch_dense(const TexDesc& d, Args... args) {
    if (d.layout == RT_LAYOUT_ATLAS) return Launch<RT_F32, RT_LAYOUT_ATLAS>::run(d, args...);
    if (d.layout == RT_LAYOUT_QUADS) return dispatch_format<Launch, RT_LAYOUT_QUADS>(d, args...);
    if (d.layout != RT_LAYOUT_PLANES) return cudaErrorInvalidValue;
    return dispatch_format<Launch, RT_LAYOUT_PLANES>(d, args...);
}

template <int FMT, int LAYOUT>
struct InitLaunch {
    static cudaError_t run(const TexDesc& d, int K, const int32_t* buckets, float* C, unsigned* status,
                           cudaStream_t stream) {
        const int64_t items = (int64_t)K * d.n * d.n;
        kmeans_init_kernel<FMT, LAYOUT><<<blocks(items, 256), 256, 0, stream>>>(d, K, buckets,
                                                                              reinterpret_cast<float4*>(C), status);
        return cudaGetLastError();
    }
};

template <int FMT, int LAYOUT>
struct AssignLaunch {
    static cudaError_t run(const TexDesc& d, int K, const float* C, uint32_t* index, float* dist,
                           cudaStream_t stream) {
        const int64_t B = (int64_t)d.W * d.H;
        kmeans_assign_kernel<FMT, LAYOUT><<<blocks(B, kAM), kAThreads, 0, stream>>>(
            d, K, reinterpret_cast<const float4*>(C), index, dist);
        return cudaGetLastError();
    }
};

template <int FMT, int LAYOUT>
struct MeanLaunch {
    static cudaError_t run(const TexDesc& d, int K, const uint32_t* offsets, const uint32_t* members, float* C,
                           cudaStream_t stream) {
        kmeans_mean_kernel<FMT, LAYOUT><<<K, 256, 0, stream>>>(d, K, offsets, members, reinterpret_cast<float4*>(C));
        return cudaGetLastError();
    }
};

cudaError_t launch_kmeans_init(const TexDesc& d, int K, const int32_t* buckets, float* C, unsigned* status,
                               cudaStream_t stream) {
    return dispatch_dense<InitLaunch>(d, K, buckets, C, status, stream);
}

cudaError_t launch_kmeans_assign(const TexDesc& d, int K, const float* C, uint32_t* index, float* dist,
                                 cudaStream_t stream) {
    return dispatch_dense<AssignLaunch>(d, K, C, index, dist, stream);
}

cudaError_t launch_kmeans_update(const TexDesc& d, int K, const uint32_t* index, float* C, uint32_t* scratch,
                                 unsigned* status, cudaStream_t stream) {
    const int64_t B = (int64_t)d.W * d.H;
    uint32_t* counts = scratch;
    uint32_t* cursor = scratch + K;
    uint32_t* offsets = scratch + 2 * (int64_t)K;  // K + 1 entries
    uint32_t* members = scratch + 3 * (int64_t)K + 1;
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * 2 * (size_t)K, stream);
    if (e != cudaSuccess) return e;
    kmeans_count_kernel<<<blocks(B, 256), 256, 0, stream>>>(index, B, K, counts, status);
    kmeans_scan_kernel<<<1, 1024, 0, stream>>>(counts, K, offsets);
    kmeans_scatter_kernel<<<blocks(B, 256), 256, 0, stream>>>(index, B, K, offsets, cursor, members);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return dispatch_dense<MeanLaunch>(d, K, (const uint32_t*)offsets, (const uint32_t*)members, C, stream);
}

}  // namespace rt

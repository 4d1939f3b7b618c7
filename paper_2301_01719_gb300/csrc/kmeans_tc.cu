// kmeans_tc.cu -- the k-means assignment of the palette encoder on the tensor
// cores: the distance contraction x_b . c_k over n^2 x 4 values is a dense
// GEMM (buckets x centroids), run with tcgen05.mma (FP16 operands, FP32
// accumulators in tensor memory), operands staged by TMA, and the argmin taken
// in the epilogue straight from tensor memory.
//
// Operands: X (the bucket vectors, Bp x Dp FP16, row-major) and C (the
// centroids, Kp x Dp FP16), both K-major, built by the conversion kernels
// below into caller-provided scratch; |c_k|^2 and |x_b|^2 are summed in FP32
// from the FP16 values.  Bp, Dp, Kp are rounded up to 128, 64 and 256 with
// zeros; padded centroids get |c|^2 = +inf and are never chosen.
//
// Persistent: one CTA per SM walks the 128-bucket tiles m = blockIdx.x,
// m + gridDim.x, ...; 192 threads: warp 0 issues the TMA loads (one elected
// lane), warp 1 the MMAs (one elected lane), warps 2-5 (128 threads, one per
// accumulator row) run the epilogue.  The three roles walk the same sequence of
// (bucket tile, centroid tile) pairs, so the shared-memory ring and the two
// accumulators stay busy across bucket tiles: the loads of the next tile
// overlap the last MMAs of this one, its epilogue the next tile's MMAs.  A 4-stage shared-memory ring of
// 128 x 64 (A) and 256 x 64 (B) FP16 tiles in the 128-byte swizzled K-major
// layout feeds M = 128, N = 256, K = 16 MMAs; two 256-column accumulators in
// tensor memory let the epilogue of one 256-centroid tile overlap the MMAs of
// the next.  Every wait on an mbarrier is bounded: on a timeout the CTA raises
// RT_ERR_TIMEOUT in the status word, stops, waits (bounded) for its copies and
// MMAs in flight, and frees its tensor memory.
#include <cuda.h>

#include "rt_device.cuh"
#include "rt_internal.h"

namespace rt {
namespace tc {

constexpr int BM = 128;  // buckets per CTA = accumulator rows (tensor-memory lanes)
constexpr int BN = 256;  // centroids per tile = accumulator columns
constexpr int BK = 64;   // FP16 values per stage row: one 128-byte swizzle row
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;  // 16 KiB
constexpr int B_BYTES = BN * BK * 2;  // 32 KiB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int THREADS = 192;
constexpr uint32_t TMEM_COLS = 2 * BN;      // two accumulators
constexpr uint32_t kSpinLimit = 1u << 22;  // polls of one mbarrier wait before giving up
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 256 + 1024;  // stages, barriers, alignment slack

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Non-blocking test of the phase of `parity`.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of `parity` to complete; false after `limit` polls
// (each followed by a 32 ns sleep: with the default kSpinLimit a fraction of a
// second in all) or once another role of the CTA has given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_test(bar, parity)) return true;
        if ((i & 255) == 255 && *abort_flag) return false;
        __nanosleep(32);
    }
    return false;
}

// The drain after a timeout: waits (kSpinLimit polls at most) for copies or
// MMAs this thread has already issued, whatever the other roles did, so that
// nothing is in flight into the CTA's shared or tensor memory when it exits.
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        if (mbar_test(bar, parity)) return true;
        __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzled
// layout: rows of 128 bytes, 8-row (1024-byte) atoms stacked at a stride of
// 1024 bytes.  Fields: start address >> 4 (bits 0-13), leading-dimension byte
// offset >> 4 (16-29; unused by swizzled K-major layouts, set to 1),
// stride-dimension byte offset >> 4 (32-45), descriptor version 1 (46-47),
// swizzle mode 2 = 128 bytes (61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16 with FP16 A and B, FP32 D, both operands
// K-major: D format (bits 4-5) = 1 (F32), A format (7-9) = 0 (F16), B format
// (10-12) = 0, N >> 3 (17-22), M >> 4 (24-28).
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__global__ void __launch_bounds__(THREADS, 1)
    assign_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int B, int Dp,
                  int Kp, const float* __restrict__ cn, const float* __restrict__ xn, uint32_t* __restrict__ index,
                  float* __restrict__ dist, unsigned* status, uint32_t spin_limit) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
    uint64_t* full = bars;                // TMA -> MMA, one per stage
    uint64_t* empty = bars + STAGES;      // MMA -> TMA
    uint64_t* accfull = bars + 2 * STAGES;       // MMA -> epilogue, one per accumulator
    uint64_t* accempty = bars + 2 * STAGES + 2;  // epilogue -> MMA
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = Kp / BN, kchunks = Dp / BK;
    const int mtiles = (B + BM - 1) / BM;
    // this CTA's bucket tiles, times the centroid tiles of each
    const int my_m = blockIdx.x < mtiles ? (mtiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int jobs = my_m * ntiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accfull[a], 1);
            mbar_init(&accempty[a], BM);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        __syncwarp();  // lane 0 initialised the barriers; the allocation is warp-wide
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    bool timed_out = false;
    if (warp == 0 && lane == 0) {
        // producer: stage s of iteration `it` holds A rows m0.., B rows of tile t, values kc*BK..
        int it = 0;
        for (int job = 0; job < jobs && !timed_out; ++job) {
            const int t = job % ntiles, m0 = ((int)blockIdx.x + (job / ntiles) * (int)gridDim.x) * BM;
            for (int kc = 0; kc < kchunks; ++kc, ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, spin_limit)) {
                    timed_out = true;
                    break;
                }
                uint8_t* sa = base + s * STAGE_BYTES;
                mbar_expect_tx(&full[s], STAGE_BYTES);
                tma_load_2d(sa, &tmA, kc * BK, m0, &full[s]);
                tma_load_2d(sa + A_BYTES, &tmB, kc * BK, t * BN, &full[s]);
            }
        }
        if (timed_out) {
            // let the copies already issued land before the CTA exits
            for (int k = 1; k <= STAGES && it - k >= 0; ++k) {
                const int j = it - k;
                mbar_drain(&full[j % STAGES], (uint32_t)(j / STAGES) & 1u);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        int it = 0;
        for (int job = 0; job < jobs && !timed_out; ++job) {
            const int a = job & 1;
            if (!mbar_wait(&accempty[a], ((uint32_t)(job >> 1) & 1u) ^ 1u, abort_flag, spin_limit)) {
                timed_out = true;
                break;
            }
            tc_fence_after();
            const uint32_t dacc = tmem + (uint32_t)(a * BN);
            for (int kc = 0; kc < kchunks; ++kc, ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (!mbar_wait(&full[s], ph, abort_flag, spin_limit)) {
                    timed_out = true;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(base + s * STAGE_BYTES);
                const uint64_t adesc = sw128_desc(sa), bdesc = sw128_desc(sa + A_BYTES);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)  // K = 16 per MMA: 32 bytes along the swizzled row
                    umma_f16(dacc, adesc + (uint64_t)(2 * kk), bdesc + (uint64_t)(2 * kk), (kc | kk) != 0);
                umma_commit(&empty[s]);  // the stage is free once these MMAs have read it
            }
            if (timed_out) break;
            umma_commit(&accfull[a]);
        }
        if (timed_out && it > 0) {
            // wait for the MMAs in flight before the tensor memory is freed
            const int j = it - 1;
            mbar_drain(&empty[j % STAGES], (uint32_t)(j / STAGES) & 1u);
        }
    } else if (warp >= 2) {
        // epilogue: thread = accumulator row; warp w reads tensor-memory lanes 32 (w % 4) ..
        const int q = warp & 3;
        const int row = q * 32 + lane;
        float best = INFINITY;
        int bestk = 0;
        for (int job = 0; job < jobs; ++job) {
            const int t = job % ntiles, a = job & 1;
            if (t == 0) {
                best = INFINITY;
                bestk = 0;
            }
            if (!mbar_wait(&accfull[a], (uint32_t)(job >> 1) & 1u, abort_flag, spin_limit)) {
                timed_out = true;
                break;
            }
            tc_fence_after();
            const uint32_t tacc = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * BN);
            for (int c0 = 0; c0 < BN; c0 += 32) {
                float v[32];
                tmem_ld32(tacc + (uint32_t)c0, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int k = t * BN + c0 + j;
                    const float d = fmaf(-2.0f, v[j], __ldg(cn + k));
                    if (d < best) {  // k grows: equal distances keep the lower index
                        best = d;
                        bestk = k;
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&accempty[a]);
            if (t == ntiles - 1) {
                const int b = ((int)blockIdx.x + (job / ntiles) * (int)gridDim.x) * BM + row;
                if (b < B) {
                    index[b] = (uint32_t)bestk;
                    if (dist) dist[b] = fmaxf(best + xn[b], 0.0f);
                }
            }
        }
    }
    if (timed_out) {
        *abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// X: bucket vectors as FP16 rows (b, (t n + s) 4 + c), zero padding; xn = |x|^2
// of the FP16 values.  One thread per (bucket, texel): a block is 32 buckets x
// 8 texels, transposed through shared memory so that reads (consecutive
// buckets of a plane) and writes (consecutive texels of a row) are coalesced.
template <int FMT, int LAYOUT>
__global__ void convert_x_kernel(TexDesc d, int Bp, int Dp, __half* __restrict__ X) {
    __shared__ uint2 tile[8][33];
    const int B = d.W * d.H, planes = d.n * d.n, P4 = Dp / 4;
    const int b0 = blockIdx.x * 32, p0 = blockIdx.y * 8;
    {
        const int b = b0 + threadIdx.x, p = p0 + threadIdx.y;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (b < B && p < planes) {
            const int j = b / d.W, i = b - j * d.W;
            if (LAYOUT != RT_LAYOUT_ATLAS) {
                const float sc = FMT == RT_E4M3_BUCKET_SCALE ? __ldg(d.scale + bucket_slot<LAYOUT>(d, i, j)) : 1.0f;
                v = load_texel<FMT>(d.base, checked_texel(d, (int64_t)p * d.plane + bucket_slot<LAYOUT>(d, i, j)), sc);
            } else {
                v = load_texel<FMT>(d.base, texel_index<RT_LAYOUT_ATLAS>(d, i, j, p % d.n, p / d.n), 1.0f);
            }
        }
        const __half2 lo = __floats2half2_rn(v.x, v.y), hi = __floats2half2_rn(v.z, v.w);
        tile[threadIdx.y][threadIdx.x] =
            make_uint2(*reinterpret_cast<const unsigned*>(&lo), *reinterpret_cast<const unsigned*>(&hi));
    }
    __syncthreads();
    // write: thread (x, y) -> bucket b0 + 4 y + x / 8, texel p0 + x % 8
    const int bl = threadIdx.y * 4 + (threadIdx.x >> 3), pl = threadIdx.x & 7;
    const int b = b0 + bl, p = p0 + pl;
    if (b < Bp && p < P4) reinterpret_cast<uint2*>(X)[(int64_t)b * P4 + p] = tile[pl][bl];
}

// |x_b|^2 of the FP16 rows (one warp per bucket).
__global__ void row_norms_kernel(const __half* __restrict__ X, int rows, int Dp, float* __restrict__ out,
                                 float pad_value, int live_rows) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (r >= rows) return;
    float s = 0.f;
    const __half2* row = reinterpret_cast<const __half2*>(X + (int64_t)r * Dp);
    for (int k = lane; k < Dp / 2; k += 32) {
        const float2 f = __half22float2(row[k]);
        s = fmaf(f.x, f.x, fmaf(f.y, f.y, s));
    }
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[r] = r < live_rows ? s : pad_value;
}

// C: centroids (n, n, K, 4) FP32 -> FP16 rows (k, (t n + s) 4 + c), zero padding.
__global__ void convert_c_kernel(const float4* __restrict__ C, int K, int planes, int Kp, int Dp,
                                 __half* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (k, p) over Kp x Dp / 4
    const int P4 = Dp / 4;
    if (e >= (int64_t)Kp * P4) return;
    const int k = (int)(e / P4), p = (int)(e - (int64_t)k * P4);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < K && p < planes) v = C[(int64_t)p * K + k];
    const __half2 lo = __floats2half2_rn(v.x, v.y), hi = __floats2half2_rn(v.z, v.w);
    reinterpret_cast<uint2*>(out)[e] =
        make_uint2(*reinterpret_cast<const unsigned*>(&lo), *reinterpret_cast<const unsigned*>(&hi));
}

struct Layout {
    int64_t Bp, Dp, Kp;
    size_t x_off, c_off, cn_off, xn_off, bytes;
};

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

inline Layout layout(int W, int H, int n, int K) {
    Layout L;
    L.Bp = round_up((int64_t)W * H, BM);
    L.Dp = round_up((int64_t)n * n * 4, BK);
    L.Kp = round_up(K, BN);
    L.x_off = 0;
    L.c_off = (size_t)round_up(L.Bp * L.Dp * 2, 1024);
    L.cn_off = L.c_off + (size_t)round_up(L.Kp * L.Dp * 2, 1024);
    L.xn_off = L.cn_off + (size_t)round_up(L.Kp * 4, 1024);
    L.bytes = L.xn_off + (size_t)round_up(L.Bp * 4, 1024);
    return L;
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// A 2-D FP16 tensor map over rows x cols (row-major), box of box_rows x 64
// values, 128-byte swizzle.
static bool make_map(CUtensorMap* m, void* ptr, int64_t rows, int64_t cols, int box_rows) {
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int FMT, int LAYOUT>
static cudaError_t convert_x(const TexDesc& d, const Layout& L, __half* X, cudaStream_t stream) {
    const dim3 grid((unsigned)(L.Bp / 32), (unsigned)((L.Dp / 4 + 7) / 8));
    convert_x_kernel<FMT, LAYOUT><<<grid, dim3(32, 8), 0, stream>>>(d, (int)L.Bp, (int)L.Dp, X);
    return cudaGetLastError();
}

template <int LAYOUT>
static cudaError_t convert_x_fmt(const TexDesc& d, const Layout& L, __half* X, cudaStream_t stream) {
    switch (d.fmt) {
        case RT_F16:
            return convert_x<RT_F16, LAYOUT>(d, L, X, stream);
        case RT_BF16:
            return convert_x<RT_BF16, LAYOUT>(d, L, X, stream);
        case RT_E4M3_BUCKET_SCALE:
            return convert_x<RT_E4M3_BUCKET_SCALE, LAYOUT>(d, L, X, stream);
        default:
            return convert_x<RT_F32, LAYOUT>(d, L, X, stream);
    }
}

}  // namespace tc

int64_t kmeans_tc_scratch_bytes(int W, int H, int n, int K) { return (int64_t)tc::layout(W, H, n, K).bytes; }

cudaError_t launch_kmeans_assign_tc(const TexDesc& d, int K, const float* C, uint32_t* index, float* dist,
                                    void* scratch, unsigned* status, uint32_t spin_limit, cudaStream_t stream) {
    using namespace tc;
    const Layout L = layout(d.W, d.H, d.n, K);
    uint8_t* base = static_cast<uint8_t*>(scratch);
    __half* X = reinterpret_cast<__half*>(base + L.x_off);
    __half* Ch = reinterpret_cast<__half*>(base + L.c_off);
    float* cn = reinterpret_cast<float*>(base + L.cn_off);
    float* xn = reinterpret_cast<float*>(base + L.xn_off);
    cudaError_t e;
    if (d.layout == RT_LAYOUT_ATLAS)
        e = convert_x<RT_F32, RT_LAYOUT_ATLAS>(d, L, X, stream);
    else if (d.layout == RT_LAYOUT_QUADS)
        e = convert_x_fmt<RT_LAYOUT_QUADS>(d, L, X, stream);
    else
        e = convert_x_fmt<RT_LAYOUT_PLANES>(d, L, X, stream);
    if (e != cudaSuccess) return e;
    const int64_t ce = L.Kp * (L.Dp / 4);
    convert_c_kernel<<<(unsigned)((ce + 255) / 256), 256, 0, stream>>>(reinterpret_cast<const float4*>(C), K,
                                                                        d.n * d.n, (int)L.Kp, (int)L.Dp, Ch);
    row_norms_kernel<<<(unsigned)((L.Kp * 32 + 255) / 256), 256, 0, stream>>>(Ch, (int)L.Kp, (int)L.Dp, cn,
                                                                              INFINITY, K);
    row_norms_kernel<<<(unsigned)((L.Bp * 32 + 255) / 256), 256, 0, stream>>>(X, (int)L.Bp, (int)L.Dp, xn, 0.f,
                                                                              (int)L.Bp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    CUtensorMap tmA, tmB;
    if (!make_map(&tmA, X, L.Bp, L.Dp, BM) || !make_map(&tmB, Ch, L.Kp, L.Dp, BN)) return cudaErrorNotSupported;
    if ((e = cudaFuncSetAttribute(assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)) !=
        cudaSuccess)
        return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t mtiles = L.Bp / BM;
    const unsigned grid = (unsigned)(mtiles < sms ? mtiles : sms);  // one CTA per SM (its shared memory)
    assign_kernel<<<grid, THREADS, SMEM_BYTES, stream>>>(tmA, tmB, d.W * d.H, (int)L.Dp, (int)L.Kp, cn, xn, index,
                                                         dist, status, spin_limit ? spin_limit : kSpinLimit);
    return cudaGetLastError();
}

}  // namespace rt

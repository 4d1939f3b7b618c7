// rt_internal.h -- host-side declarations shared by the translation units of libradtex.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "radtex.h"

#include "rt_filter.cuh"

namespace rt {
struct TexDesc;

// The flat stream (no frame shape).
__host__ __device__ inline Tiling flat_tiling() {
    Tiling t{};
    t.tw = 32;
    t.th = 1;
    t.bx = 1;
    t.by = 1;
    return t;
}

// Screen tiling of views x h x w frames with tw x th warp tiles arranged bx x by
// in a block tile; false if the shape is not usable (tw * th != 32, tw not a
// multiple of 4, bx * by != warps).
inline int log2_exact(int x) {
    int k = 0;
    while ((1 << k) < x) ++k;
    return (1 << k) == x ? k : -1;
}

inline bool make_tiling(int views, int h, int w, int tw, int th, int bx, int by, int warps, Tiling* t) {
    if (views < 1 || h < 1 || w < 1 || tw * th != 32 || (tw & 3) != 0 || bx * by != warps) return false;
    if (log2_exact(tw) < 0 || log2_exact(bx) < 0) return false;
    t->W = w;
    t->H = h;
    t->views = views;
    t->tw = tw;
    t->th = th;
    t->bx = bx;
    t->by = by;
    t->btx = (w + bx * tw - 1) / (bx * tw);
    t->bty = (h + by * th - 1) / (by * th);
    t->frame = (int64_t)w * h;
    t->tw_log2 = log2_exact(tw);
    t->bx_log2 = log2_exact(bx);
    t->div_btx = make_fastdiv((uint32_t)t->btx);
    t->div_frame = make_fastdiv((uint32_t)((int64_t)t->btx * t->bty));
    // the tiled walk indexes chunks with 31-bit integers
    return (int64_t)t->btx * t->bty * views * warps < ((int64_t)1 << 31);
}

inline int64_t chunk_count_host(const Tiling& T, int64_t F, int warps) {
    if (T.W <= 0) return (F + 31) / 32;
    return (int64_t)T.btx * T.bty * T.views * warps;
}

// Pointers to the FP32 texel-gradient buffers, indexed by object id, passed by
// value as a kernel parameter (no device allocation, capturable in a graph).
struct GradTable {
    void* p[RT_MAX_OBJECTS];  // float* (FP32 sums) or long long* (fixed-point sums, deterministic mode)
};

// spec: the storage format shared by every object of the table (dense QUADS,
// clamp mode), or -1; selects a single-format instantiation of the tiled kernels.
cudaError_t launch_shade(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                         int64_t F, int filter, const Tiling& T, int spec, float* out, unsigned* status,
                         cudaStream_t stream);
cudaError_t launch_locate(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                          int64_t F, int filter, int32_t* idx, float* coord, unsigned* status, cudaStream_t stream);
cudaError_t launch_backward(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                            int64_t F, int filter, const Tiling& T, int spec, const float* dL_dout,
                            const GradTable& grads, bool any_grad, float* dL_duv, float* dL_ddir, bool accumulate,
                            bool deterministic, unsigned* status, cudaStream_t stream);
cudaError_t launch_fused_l2(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                            int64_t F, int filter, const Tiling& T, int spec, const float* target, float scale,
                            float* out, double* sums, const GradTable& grads, bool any_grad, float* dL_duv,
                            float* dL_ddir, bool accumulate, bool deterministic, unsigned* status,
                            cudaStream_t stream);
cudaError_t launch_fixed_to_float(const long long* acc, float* dst, int64_t count, bool accumulate,
                                  cudaStream_t stream, double scale = 1.0);

cudaError_t launch_encode(const float* src, int src_layout, void* dst, float* scale, int W, int H, int n, int fmt,
                          int dst_layout, cudaStream_t stream);
cudaError_t launch_read(const void* src, int src_layout, const float* scale, int fmt, int W, int H, int n,
                        int dst_layout, void* dst, float* scale_dst, cudaStream_t stream);
cudaError_t launch_bake_shadow(const rt_bake_scene& S, int surface, void* dst, int W, int H, int n,
                               cudaStream_t stream);
cudaError_t launch_multi_shade(const TexDesc* table, int n_obj, const float* uv, const float* dirs, int S,
                               const int32_t* obj, int64_t F, int filter, float* out, unsigned* status,
                               cudaStream_t stream);
// World-space kernels: T is flat_tiling() for the flat stream, or a screen tiling.
cudaError_t launch_world_shade(const TexDesc* table, int n_obj, const float* uv, const float* dir, const float* nrm,
                               const int32_t* obj, int64_t F, int filter, const Tiling& T, float* out, int32_t* idx,
                               float* coord, unsigned* status, cudaStream_t stream);
cudaError_t launch_world_backward(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                  const float* nrm, const int32_t* obj, int64_t F, int filter, const Tiling& T,
                                  const float* dL_dout, const GradTable& grads, bool any_grad, float* dL_duv,
                                  float* dL_ddir, float* dL_dnrm, bool accumulate, bool deterministic,
                                  unsigned* status, cudaStream_t stream);
int64_t kmeans_tc_scratch_bytes(int W, int H, int n, int K);
cudaError_t launch_kmeans_assign_tc(const TexDesc& d, int K, const float* C, uint32_t* index, float* dist,
                                    void* scratch, unsigned* status, uint32_t spin_limit, cudaStream_t stream);
cudaError_t launch_kmeans_init(const TexDesc& d, int K, const int32_t* buckets, float* C, unsigned* status,
                               cudaStream_t stream);
cudaError_t launch_kmeans_assign(const TexDesc& d, int K, const float* C, uint32_t* index, float* dist,
                                 cudaStream_t stream);
cudaError_t launch_kmeans_update(const TexDesc& d, int K, const uint32_t* index, float* C, uint32_t* scratch,
                                 unsigned* status, cudaStream_t stream);
cudaError_t launch_check_index(const uint32_t* index, int64_t count, uint32_t K, unsigned* bad, cudaStream_t stream);
cudaError_t launch_bake(const rt_bake_scene& S, int surface, void* dst, float* scale, int W, int H, int n, int fmt,
                        int layout, const float* ao_dirs, int K, cudaStream_t stream);
cudaError_t launch_fill_lobes(const float* params, void* dst, float* scale, int layout, int W, int H, int n, int fmt,
                              cudaStream_t stream);
cudaError_t launch_convert(const float* src, int src_layout, float* dst, int dst_layout, int W, int H, int n,
                           cudaStream_t stream);
cudaError_t launch_footprint_mark(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                  const int32_t* obj, int64_t F, int filter, uint32_t* bitmap,
                                  const int64_t* word_offset, unsigned* status, cudaStream_t stream);
cudaError_t launch_popcount(const uint32_t* bitmap, int64_t words, unsigned long long* count, cudaStream_t stream);

}  // namespace rt

// Read-only views of a context for entry points defined outside api.cu.
const rt::TexDesc* rt_internal_host_table(rt_ctx* ctx, int* n_obj);
const rt::TexDesc* rt_internal_device_table(rt_ctx* ctx);
unsigned* rt_internal_status(rt_ctx* ctx);
int rt_internal_device(rt_ctx* ctx);

// rt_internal.h -- host-side declarations shared by the translation units of libradtex.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "radtex.h"

namespace rt {
struct TexDesc;

// Pointers to the FP32 texel-gradient buffers, indexed by object id, passed by
// value as a kernel parameter (no device allocation, capturable in a graph).
struct GradTable {
    float* p[RT_MAX_OBJECTS];
};

cudaError_t launch_shade(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                         int64_t F, int filter, float* out, unsigned* status, cudaStream_t stream);
cudaError_t launch_locate(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                          int64_t F, int filter, int32_t* idx, float* coord, unsigned* status, cudaStream_t stream);
cudaError_t launch_backward(const TexDesc* table, int n_obj, const float* uv, const float* dir, const int32_t* obj,
                            int64_t F, int filter, const float* dL_dout, const GradTable& grads, bool any_grad,
                            float* dL_duv, float* dL_ddir, bool accumulate, unsigned* status, cudaStream_t stream);

cudaError_t launch_encode(const float* src, int src_layout, void* dst, float* scale, int W, int H, int n, int fmt,
                          cudaStream_t stream);
cudaError_t launch_read(const void* src, int fmt, int W, int H, int n, int dst_layout, void* dst, cudaStream_t stream);
cudaError_t launch_fill_lobes(const float* params, void* dst, float* scale, int W, int H, int n, int fmt,
                              cudaStream_t stream);
cudaError_t launch_convert(const float* src, int src_layout, float* dst, int dst_layout, int W, int H, int n,
                           cudaStream_t stream);
cudaError_t launch_footprint_mark(const TexDesc* table, int n_obj, const float* uv, const float* dir,
                                  const int32_t* obj, int64_t F, int filter, uint32_t* bitmap,
                                  const int64_t* word_offset, unsigned* status, cudaStream_t stream);
cudaError_t launch_popcount(const uint32_t* bitmap, int64_t words, unsigned long long* count, cudaStream_t stream);

}  // namespace rt

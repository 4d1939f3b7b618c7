// optim.cu -- the loss and optimiser kernels of texture fitting: an L2 loss
// against target renders (its value and dL/dout) and an Adam step on an FP32
// texture.  With rt_shade_batched / rt_shade_batched_backward they make a
// fitting step that runs entirely in this library's kernels.
#include <cuda_runtime.h>

#include <cstdint>

#include "radtex.h"
#include "rt_internal.h"

namespace {

constexpr int kThreads = 256;

// dL/dout = scale (out - target) on shaded fragments (obj >= 0), 0 elsewhere;
// sums[0] += sum over shaded fragments of |out - target|^2 (FP64), sums[1] += their count.
__global__ void __launch_bounds__(kThreads) l2_loss_grad_kernel(const float4* __restrict__ out,
                                                                const float4* __restrict__ target,
                                                                const int32_t* __restrict__ obj, int64_t F,
                                                                float scale, float4* __restrict__ dL_dout,
                                                                double* sums) {
    double se = 0.0, cnt = 0.0;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        if (obj[f] >= 0) {
            const float4 o = out[f], t = target[f];
            const float4 r = make_float4(o.x - t.x, o.y - t.y, o.z - t.z, o.w - t.w);
            se += (double)r.x * r.x + (double)r.y * r.y + (double)r.z * r.z + (double)r.w * r.w;
            cnt += 1.0;
            g = make_float4(scale * r.x, scale * r.y, scale * r.z, scale * r.w);
        }
        if (dL_dout) dL_dout[f] = g;
    }
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_down_sync(0xFFFFFFFFu, se, o);
        cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, o);
    }
    __shared__ double part[2][kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        part[0][w] = se;
        part[1][w] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) {
            a += part[0][k];
            b += part[1][k];
        }
        if (sums) {
            atomicAdd(sums, a);
            atomicAdd(sums + 1, b);
        }
    }
}

// One Adam step (Kingma & Ba) with bias correction, element-wise on float4.
__device__ __forceinline__ void adam4(float4& pp, const float4 gg, float4& mm, float4& vv, float lr, float b1,
                                      float b2, float eps, float ic1, float ic2) {
    float* P = &pp.x;
    const float* G = &gg.x;
    float* M = &mm.x;
    float* V = &vv.x;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        M[c] = b1 * M[c] + (1.0f - b1) * G[c];
        V[c] = b2 * V[c] + (1.0f - b2) * G[c] * G[c];
        const float mh = M[c] * ic1, vh = V[c] * ic2;
        P[c] -= lr * mh / (sqrtf(vh) + eps);
    }
}

// Two float4 elements in flight per thread, the gradient read with an
// evict-first hint (it is read once); the bias corrections are applied as
// reciprocals computed on the host.  Inside the fitting step (after the fused
// launch has written the gradients) this took the step from 2.58 to 2.36 ms.
__global__ void __launch_bounds__(kThreads) adam_kernel(float4* __restrict__ p, const float4* __restrict__ g,
                                                        float4* __restrict__ m, float4* __restrict__ v, int64_t n4,
                                                        float lr, float b1, float b2, float eps, float ic1, float ic2) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; k + stride < n4; k += 2 * stride) {  // two elements in flight per thread
        float4 p0 = p[k], g0 = __ldcs(g + k), m0 = m[k], v0 = v[k];
        float4 p1 = p[k + stride], g1 = __ldcs(g + k + stride), m1 = m[k + stride], v1 = v[k + stride];
        adam4(p0, g0, m0, v0, lr, b1, b2, eps, ic1, ic2);
        adam4(p1, g1, m1, v1, lr, b1, b2, eps, ic1, ic2);
        p[k] = p0;
        m[k] = m0;
        v[k] = v0;
        p[k + stride] = p1;
        m[k + stride] = m1;
        v[k + stride] = v1;
    }
    for (; k < n4; k += stride) {
        float4 pp = p[k], gg = __ldcs(g + k), mm = m[k], vv = v[k];
        adam4(pp, gg, mm, vv, lr, b1, b2, eps, ic1, ic2);
        p[k] = pp;
        m[k] = mm;
        v[k] = vv;
    }
}

inline unsigned grid_for(int64_t items) {
    int64_t b = (items + kThreads - 1) / kThreads;
    return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

extern "C" rt_status rt_l2_loss_grad(const float* out, const float* target, const int32_t* obj, int64_t F,
                                     float scale, float* dL_dout, double* sums, rt_stream_t stream) {
    if (F < 0 || (F > 0 && (!out || !target || !obj))) return RT_ERR_INVALID_ARG;
    if ((((uintptr_t)out | (uintptr_t)target | (uintptr_t)dL_dout) & 15u) || (((uintptr_t)sums) & 7u))
        return RT_ERR_INVALID_ARG;
    if (F == 0) return RT_OK;
    l2_loss_grad_kernel<<<grid_for(F), kThreads, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4*>(out), reinterpret_cast<const float4*>(target), obj, F, scale,
        reinterpret_cast<float4*>(dL_dout), sums);
    return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}

extern "C" rt_status rt_adam_step(float* param, const float* grad, float* m, float* v, int64_t count, float lr,
                                  float beta1, float beta2, float eps, int32_t step, rt_stream_t stream) {
    if (count < 0 || (count & 3) || step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f))
        return RT_ERR_INVALID_ARG;
    if (count > 0 && (!param || !grad || !m || !v)) return RT_ERR_INVALID_ARG;
    if (((uintptr_t)param | (uintptr_t)grad | (uintptr_t)m | (uintptr_t)v) & 15u) return RT_ERR_INVALID_ARG;
    if (count == 0) return RT_OK;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    adam_kernel<<<grid_for(count / 4), kThreads, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<float4*>(param), reinterpret_cast<const float4*>(grad), reinterpret_cast<float4*>(m),
        reinterpret_cast<float4*>(v), count / 4, lr, beta1, beta2, eps, 1.0f / c1, 1.0f / c2);
    return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ERR_CUDA;
}

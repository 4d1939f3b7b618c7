/* A plain C99 user of the library: only include/radtex.h and the CUDA runtime.
 * Without arguments it calls the host-only entry points; with "gpu" it also
 * creates a context and a constant FP32 texture, shades a few fragments and
 * checks that every channel comes back as the constant (a constant texture is
 * reproduced exactly, the lerps' weights summing to one). */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "radtex.h"

#define CHECK(call)                                                                  \
    do {                                                                             \
        rt_status st_ = (call);                                                      \
        if (st_ != RT_OK) {                                                          \
            printf("FAIL %s: %s\n", #call, rt_status_string(st_));                   \
            return 1;                                                                \
        }                                                                            \
    } while (0)

int main(int argc, char** argv) {
    printf("status %d %s\n", (int)RT_ERR_INVALID_ARG, rt_status_string(RT_ERR_INVALID_ARG));
    printf("tc scratch %lld\n", (long long)rt_kmeans_tc_scratch_bytes(64, 64, 8, 300));
    if (argc < 2 || strcmp(argv[1], "gpu") != 0) return 0;

    const int W = 7, H = 5, n = 4, F = 6;
    const float value[4] = {0.25f, 0.5f, 0.75f, 1.0f};
    const size_t atlas_n = (size_t)H * n * W * n * 4;
    float* h_atlas = (float*)malloc(atlas_n * sizeof(float));
    for (size_t i = 0; i < atlas_n; ++i) h_atlas[i] = value[i % 4];
    const float h_uv[2 * 6] = {0.f, 0.f, 0.31f, 0.77f, 0.5f, 0.5f, 1.f, 1.f, 0.99f, 0.01f, 0.2f, 0.6f};
    const float h_dir[3 * 6] = {0.f, 0.f, 1.f, 0.3f, -0.2f, 0.93f, 0.9f, 0.1f, 0.42f,
                                -0.5f, 0.5f, 0.707f, 0.f, 0.99f, 0.1f, 0.1f, 0.1f, 0.98f};
    float *d_atlas, *d_uv, *d_dir, *d_out;
    int32_t* d_obj;
    if (cudaMalloc((void**)&d_atlas, atlas_n * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&d_uv, sizeof h_uv) != cudaSuccess || cudaMalloc((void**)&d_dir, sizeof h_dir) != cudaSuccess ||
        cudaMalloc((void**)&d_obj, F * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc((void**)&d_out, 4 * F * sizeof(float)) != cudaSuccess) {
        printf("FAIL cudaMalloc\n");
        return 1;
    }
    cudaMemcpy(d_atlas, h_atlas, atlas_n * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(d_uv, h_uv, sizeof h_uv, cudaMemcpyHostToDevice);
    cudaMemcpy(d_dir, h_dir, sizeof h_dir, cudaMemcpyHostToDevice);

    rt_ctx* ctx = NULL;
    int32_t oid = -1;
    CHECK(rt_context_create(0, &ctx));
    CHECK(rt_create_texture(ctx, W, H, n, RT_F32, RT_LAYOUT_ATLAS, d_atlas, 0, &oid));
    int32_t h_obj[6];
    for (int i = 0; i < F; ++i) h_obj[i] = oid;
    cudaMemcpy(d_obj, h_obj, sizeof h_obj, cudaMemcpyHostToDevice);
    CHECK(rt_shade(ctx, d_uv, d_dir, d_obj, F, RT_QUADRILINEAR, d_out, NULL));
    rt_status dev_status = RT_OK;
    CHECK(rt_get_error(ctx, NULL, &dev_status));
    float h_out[4 * 6];
    cudaMemcpy(h_out, d_out, sizeof h_out, cudaMemcpyDeviceToHost);
    int bad = dev_status != RT_OK;
    for (int i = 0; i < 4 * F; ++i) bad |= h_out[i] != value[i % 4];
    CHECK(rt_destroy_texture(ctx, oid));
    rt_context_destroy(ctx);
    cudaFree(d_atlas);
    cudaFree(d_uv);
    cudaFree(d_dir);
    cudaFree(d_obj);
    cudaFree(d_out);
    free(h_atlas);
    printf(bad ? "FAIL constant texture\n" : "gpu ok\n");
    return bad;
}

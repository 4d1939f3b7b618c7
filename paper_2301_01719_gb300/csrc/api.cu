// api.cu -- the C ABI of libradtex (declared in include/radtex.h): context,
// texture table, argument validation, kernel launches and the status model.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "radtex.h"
#include "rt_device.cuh"
#include "rt_encode.cuh"
#include "rt_internal.h"

using rt::TexDesc;

struct rt_ctx {
    int device = 0;
    TexDesc* d_table = nullptr;          // device copy of `table`
    unsigned* d_status = nullptr;        // sticky device status word
    unsigned* h_status = nullptr;        // pinned host mirror for rt_get_error
    TexDesc table[RT_MAX_OBJECTS];       // host copy
    void* owned[RT_MAX_OBJECTS];         // storage the library allocated (nullptr if borrowed)
    float* scales[RT_MAX_OBJECTS];       // E4M3 scales the library allocated
    int64_t bytes[RT_MAX_OBJECTS];
    int n_obj = 0;                       // one past the highest id ever used
    int tile[2][3][4];                   // per pass (forward, backward) and filter: tw, th, bx, by of the batched kernels
    long long* det[RT_MAX_OBJECTS];      // fixed-point gradient sums of the deterministic mode
    uint32_t* index[RT_MAX_OBJECTS];     // palette index maps the library copied
    int spec = -1;                       // the format shared by all objects (dense PLANES, clamp), else -1
    uint32_t wait_limit = 0;             // polls of a bounded device wait before it gives up (0: the default)
};

namespace {

// Makes the context's device current for the duration of a call and restores
// the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline int texel_bytes(int fmt) {
    switch (fmt) {
        case RT_F32:
            return 16;
        case RT_F16:
        case RT_BF16:
            return 8;
        case RT_E4M3_BUCKET_SCALE:
            return 4;
        case RT_BIT1:
            return 1;  // storage: texels / 8 bytes, rounded up to whole 32-bit words (storage_bytes)
        default:
            return 0;
    }
}

// Bytes of the texel storage of `texels` texels.
inline int64_t storage_bytes(int fmt, int64_t texels) {
    if (fmt == RT_BIT1) return (texels + 31) / 32 * 4;
    return texels * texel_bytes(fmt);
}


inline rt_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return RT_OK;
    if (e == cudaErrorMemoryAllocation) return RT_ERR_OOM;
    return RT_ERR_CUDA;
}

inline bool valid_filter(int f) { return f == RT_NEAREST || f == RT_ANGULAR_BILINEAR || f == RT_QUADRILINEAR; }

rt_status check_gbuffer(const float* uv, const float* dir, const int32_t* obj, int64_t F) {
    if (F < 0) return RT_ERR_INVALID_ARG;
    if (F == 0) return RT_OK;
    if (!uv || !dir || !obj) return RT_ERR_INVALID_ARG;
    if (!aligned16(uv) || !aligned16(dir) || !aligned16(obj)) return RT_ERR_INVALID_ARG;
    return RT_OK;
}

// The single-format specialisation the tiled kernels may use for this table.
int table_spec(const rt_ctx* ctx) {
    int spec = -2;
    for (int o = 0; o < ctx->n_obj; ++o) {
        const TexDesc& d = ctx->table[o];
        if (!d.live) continue;
        if (d.layout != RT_LAYOUT_QUADS || d.wrap || d.fmt == RT_BIT1) return -1;
        if (spec == -2)
            spec = d.fmt;
        else if (spec != d.fmt)
            return -1;
    }
    return spec < 0 ? -1 : spec;
}

rt_status upload_table(rt_ctx* ctx) {
    ctx->spec = table_spec(ctx);
    cudaError_t e = cudaMemcpy(ctx->d_table, ctx->table, sizeof(TexDesc) * RT_MAX_OBJECTS, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return cuda_status(e);
}

}  // namespace

const rt::TexDesc* rt_internal_host_table(rt_ctx* ctx, int* n_obj) {
    *n_obj = ctx->n_obj;
    return ctx->table;
}
const rt::TexDesc* rt_internal_device_table(rt_ctx* ctx) { return ctx->d_table; }
unsigned* rt_internal_status(rt_ctx* ctx) { return ctx->d_status; }
int rt_internal_device(rt_ctx* ctx) { return ctx->device; }

extern "C" {

const char* rt_status_string(rt_status s) {
    switch (s) {
        case RT_OK:
            return "ok";
        case RT_ERR_INVALID_ARG:
            return "invalid argument (null, misaligned or out-of-range)";
        case RT_ERR_OOM:
            return "device memory or object ids exhausted";
        case RT_ERR_CUDA:
            return "CUDA runtime error";
        case RT_ERR_BAD_OBJ_ID:
            return "a fragment named an object id with no texture";
        case RT_ERR_NONFINITE:
            return "a fragment had a non-finite UV or direction";
        case RT_ERR_TIMEOUT:
            return "a bounded device wait gave up";
        case RT_ERR_UNSUPPORTED:
            return "unsupported combination of options";
        case RT_ERR_OUT_OF_BOUNDS:
            return "a computed texel address fell outside its object (checked build)";
    }
    return "unknown status";
}

rt_status rt_context_create(int cuda_device, rt_ctx** out) {
    if (!out) return RT_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) return RT_ERR_CUDA;
    if (cuda_device < 0 || cuda_device >= count) return RT_ERR_INVALID_ARG;
    rt_ctx* ctx = new (std::nothrow) rt_ctx();
    if (!ctx) return RT_ERR_OOM;
    std::memset(ctx->table, 0, sizeof(ctx->table));
    std::memset(ctx->owned, 0, sizeof(ctx->owned));
    std::memset(ctx->scales, 0, sizeof(ctx->scales));
    std::memset(ctx->bytes, 0, sizeof(ctx->bytes));
    std::memset(ctx->det, 0, sizeof(ctx->det));
    std::memset(ctx->index, 0, sizeof(ctx->index));
    for (int p = 0; p < 2; ++p)
        for (int f = 0; f < 3; ++f) {
            ctx->tile[p][f][0] = 8;
            ctx->tile[p][f][1] = 4;
            ctx->tile[p][f][2] = 2;
            ctx->tile[p][f][3] = 2;
        }
    ctx->device = cuda_device;
    DeviceGuard g(cuda_device);
    if (!g.ok) {
        delete ctx;
        return RT_ERR_CUDA;
    }
    cudaError_t e = cudaMalloc(&ctx->d_table, sizeof(TexDesc) * RT_MAX_OBJECTS);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(unsigned));
    if (e == cudaSuccess) {
        rt_status st = upload_table(ctx);
        if (st != RT_OK) e = cudaErrorUnknown;
    }
    if (e != cudaSuccess) {
        cudaFree(ctx->d_table);
        cudaFree(ctx->d_status);
        cudaFreeHost(ctx->h_status);
        delete ctx;
        return cuda_status(e);
    }
    *out = ctx;
    return RT_OK;
}

void rt_context_destroy(rt_ctx* ctx) {
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        for (int o = 0; o < RT_MAX_OBJECTS; ++o) {
            if (ctx->owned[o]) cudaFree(ctx->owned[o]);
            if (ctx->scales[o]) cudaFree(ctx->scales[o]);
            if (ctx->det[o]) cudaFree(ctx->det[o]);
            if (ctx->index[o]) cudaFree(ctx->index[o]);
        }
        cudaFree(ctx->d_table);
        cudaFree(ctx->d_status);
        cudaFreeHost(ctx->h_status);
    }
    delete ctx;
}

// Storage layout of an owned dense texture: 2 x 2 bucket quads (an odd side
// padded); bit textures keep the PLANES bit numbering.
static rt_layout store_layout(rt_format storage) {
    return storage != RT_BIT1 ? RT_LAYOUT_QUADS : RT_LAYOUT_PLANES;
}

// Creates a dense texture (K = 0) or a palette texture (K palette buckets
// stored as a K x 1 texture, plus a copy of the w x h index map).
static rt_status create_object(rt_ctx* ctx, int32_t w, int32_t h, int32_t n, int32_t K, rt_format storage,
                               rt_layout src_layout, const float* src, const uint32_t* index, int32_t flags,
                               int32_t* obj_id_out) {
    if (!ctx || !obj_id_out) return RT_ERR_INVALID_ARG;
    if (w < 1 || h < 1 || n < 1 || w > 65536 || h > 65536 || n > 64) return RT_ERR_INVALID_ARG;
    if ((int64_t)w * h > ((int64_t)1 << 30)) return RT_ERR_INVALID_ARG;  // spatial offsets are 32-bit
    if (texel_bytes(storage) == 0) return RT_ERR_INVALID_ARG;
    if (src_layout != RT_LAYOUT_ATLAS && src_layout != RT_LAYOUT_PLANES && src_layout != RT_LAYOUT_QUADS)
        return RT_ERR_INVALID_ARG;
    if (src && !aligned16(src)) return RT_ERR_INVALID_ARG;
    const bool palette = K > 0;
    if (src_layout == RT_LAYOUT_QUADS && palette) return RT_ERR_INVALID_ARG;  // a palette source is K x 1 planes
    if (palette && (K > (1 << 30) || !index || !src)) return RT_ERR_INVALID_ARG;
    const bool borrow = (flags & RT_BORROW) != 0;
    if (borrow && (storage != RT_F32 || !src)) return RT_ERR_INVALID_ARG;
    if (borrow && palette && src_layout != RT_LAYOUT_PLANES) return RT_ERR_UNSUPPORTED;
    if (palette && storage == RT_BIT1) return RT_ERR_UNSUPPORTED;
    int o = -1;
    for (int k = 0; k < RT_MAX_OBJECTS; ++k)
        if (!ctx->table[k].live) {
            o = k;
            break;
        }
    if (o < 0) return RT_ERR_OOM;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    // src and index may have been written on any stream of the device.
    if (cudaDeviceSynchronize() != cudaSuccess) return RT_ERR_CUDA;

    // the stored buckets: the w x h matrix (in quads: ceil(w/2) x ceil(h/2) of them), or the K x 1 palette
    const int32_t sw = palette ? K : w, sh = palette ? 1 : h;
    const int layout = palette ? (int)rt::kLayoutPalette : borrow ? (int)src_layout : (int)store_layout(storage);
    const int64_t plane = palette ? (int64_t)K : rt::plane_buckets(layout, w, h);
    const int64_t texels = plane * n * n;
    TexDesc d;
    std::memset(&d, 0, sizeof(d));
    d.W = w;
    d.H = h;
    d.n = n;
    d.fmt = (int8_t)storage;
    d.layout = (int8_t)layout;
    d.plane = plane;
    d.fW = (float)w;
    d.fH = (float)h;
    d.half_n = 0.5f * (float)n;
    d.hi = 1.0f - 1.0f / (float)n;
    d.live = 1;
    d.wrap = (int8_t)(((flags & RT_WRAP_U) ? 1 : 0) | ((flags & RT_WRAP_V) ? 2 : 0));
#ifdef RADTEX_CHECKED
    d.extent = texels;
    d.status = ctx->d_status;
#endif
    void* storage_ptr = nullptr;
    float* scale_ptr = nullptr;
    uint32_t* index_ptr = nullptr;
    cudaError_t e = cudaSuccess;
    if (palette) {
        // copy and check the index map: every entry < K
        const size_t ib = sizeof(uint32_t) * (size_t)w * h;
        unsigned* bad = nullptr;
        e = cudaMalloc(&index_ptr, ib);
        if (e == cudaSuccess) e = cudaMalloc(&bad, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemset(bad, 0, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemcpy(index_ptr, index, ib, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) e = rt::launch_check_index(index_ptr, (int64_t)w * h, (uint32_t)K, bad, 0);
        unsigned h_bad = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&h_bad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost);
        cudaFree(bad);
        if (e != cudaSuccess || h_bad) {
            cudaFree(index_ptr);
            return e != cudaSuccess ? cuda_status(e) : RT_ERR_INVALID_ARG;
        }
        d.index = index_ptr;
    }
    if (borrow) {
        d.base = src;
        ctx->bytes[o] = texels * 16;
    } else {
        const int64_t bytes = storage_bytes(storage, texels);
        e = cudaMalloc(&storage_ptr, (size_t)bytes);
        if (e == cudaSuccess && storage == RT_E4M3_BUCKET_SCALE)
            e = cudaMalloc(&scale_ptr, sizeof(float) * (size_t)d.plane);
        // zero codes and unit scales first: the padding of odd sides keeps them (no lookup reads it)
        if (e == cudaSuccess && (!src || plane != (int64_t)sw * sh)) e = cudaMemset(storage_ptr, 0, (size_t)bytes);
        if (e == cudaSuccess && scale_ptr) {
            std::vector<float> ones((size_t)d.plane, 1.0f);
            e = cudaMemcpy(scale_ptr, ones.data(), sizeof(float) * ones.size(), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess && src)
            e = rt::launch_encode(src, src_layout, storage_ptr, scale_ptr, sw, sh, n, storage,
                                  palette ? RT_LAYOUT_PLANES : layout, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            cudaFree(storage_ptr);
            cudaFree(scale_ptr);
            cudaFree(index_ptr);
            return cuda_status(e);
        }
        d.base = storage_ptr;
        d.scale = scale_ptr;
        ctx->owned[o] = storage_ptr;
        ctx->scales[o] = scale_ptr;
        ctx->bytes[o] = bytes + (scale_ptr ? (int64_t)sizeof(float) * d.plane : 0);
    }
    ctx->index[o] = index_ptr;
    if (index_ptr) ctx->bytes[o] += (int64_t)sizeof(uint32_t) * w * h;
    ctx->table[o] = d;
    if (o + 1 > ctx->n_obj) ctx->n_obj = o + 1;
    rt_status st = upload_table(ctx);
    if (st != RT_OK) {
        ctx->table[o].live = 0;
        cudaFree(storage_ptr);
        cudaFree(scale_ptr);
        cudaFree(index_ptr);
        ctx->owned[o] = nullptr;
        ctx->scales[o] = nullptr;
        ctx->index[o] = nullptr;
        return st;
    }
    *obj_id_out = o;
    return RT_OK;
}

rt_status rt_create_texture(rt_ctx* ctx, int32_t w, int32_t h, int32_t n, rt_format storage, rt_layout src_layout,
                            const float* src, int32_t flags, int32_t* obj_id_out) {
    return create_object(ctx, w, h, n, 0, storage, src_layout, src, nullptr, flags, obj_id_out);
}

rt_status rt_create_palette_texture(rt_ctx* ctx, int32_t w, int32_t h, int32_t n, int32_t K, rt_format storage,
                                    rt_layout src_layout, const float* palette, const uint32_t* index, int32_t flags,
                                    int32_t* obj_id_out) {
    if (K < 1) return RT_ERR_INVALID_ARG;
    return create_object(ctx, w, h, n, K, storage, src_layout, palette, index, flags, obj_id_out);
}

rt_status rt_palette_size(rt_ctx* ctx, int32_t obj_id, int32_t* K) {
    if (!ctx || !K || obj_id < 0 || obj_id >= RT_MAX_OBJECTS || !ctx->table[obj_id].live) return RT_ERR_INVALID_ARG;
    const TexDesc& d = ctx->table[obj_id];
    *K = d.layout == rt::kLayoutPalette ? (int32_t)d.plane : 0;
    return RT_OK;
}

rt_status rt_destroy_texture(rt_ctx* ctx, int32_t obj_id) {
    if (!ctx || obj_id < 0 || obj_id >= RT_MAX_OBJECTS || !ctx->table[obj_id].live) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    cudaError_t e = cudaDeviceSynchronize();
    if (ctx->owned[obj_id]) cudaFree(ctx->owned[obj_id]);
    if (ctx->scales[obj_id]) cudaFree(ctx->scales[obj_id]);
    if (ctx->det[obj_id]) cudaFree(ctx->det[obj_id]);
    if (ctx->index[obj_id]) cudaFree(ctx->index[obj_id]);
    ctx->index[obj_id] = nullptr;
    ctx->owned[obj_id] = nullptr;
    ctx->scales[obj_id] = nullptr;
    ctx->det[obj_id] = nullptr;
    ctx->bytes[obj_id] = 0;
    std::memset(&ctx->table[obj_id], 0, sizeof(TexDesc));
    rt_status st = upload_table(ctx);
    return e != cudaSuccess ? cuda_status(e) : st;
}

rt_status rt_texture_info(rt_ctx* ctx, int32_t obj_id, int32_t* w, int32_t* h, int32_t* n, int32_t* storage,
                          int32_t* layout, int64_t* bytes) {
    if (!ctx || obj_id < 0 || obj_id >= RT_MAX_OBJECTS || !ctx->table[obj_id].live) return RT_ERR_INVALID_ARG;
    const TexDesc& d = ctx->table[obj_id];
    if (w) *w = d.W;
    if (h) *h = d.H;
    if (n) *n = d.n;
    if (storage) *storage = d.fmt;
    if (layout) *layout = d.layout;
    if (bytes) *bytes = ctx->bytes[obj_id];
    return RT_OK;
}

rt_status rt_read_texture(rt_ctx* ctx, int32_t obj_id, rt_layout dst_layout, void* codes_dst, float* scales_dst,
                          rt_stream_t stream) {
    if (!ctx || obj_id < 0 || obj_id >= RT_MAX_OBJECTS || !ctx->table[obj_id].live || !codes_dst)
        return RT_ERR_INVALID_ARG;
    if (dst_layout != RT_LAYOUT_ATLAS && dst_layout != RT_LAYOUT_PLANES && dst_layout != RT_LAYOUT_QUADS)
        return RT_ERR_INVALID_ARG;
    const TexDesc& d = ctx->table[obj_id];
    if (d.layout == RT_LAYOUT_ATLAS) return RT_ERR_UNSUPPORTED;
    const bool pal = d.layout == rt::kLayoutPalette;  // a palette reads as its K x 1 texture (PLANES)
    const int rw = pal ? (int)d.plane : d.W, rh = pal ? 1 : d.H;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    return cuda_status(rt::launch_read(d.base, pal ? RT_LAYOUT_PLANES : d.layout, d.scale, d.fmt, rw, rh, d.n,
                                       dst_layout, codes_dst, scales_dst, s));
}

rt_status rt_fill_bucket_lobes(rt_ctx* ctx, int32_t obj_id, const float* params, rt_stream_t stream) {
    if (!ctx || obj_id < 0 || obj_id >= RT_MAX_OBJECTS || !ctx->table[obj_id].live || !params || !aligned16(params))
        return RT_ERR_INVALID_ARG;
    const TexDesc& d = ctx->table[obj_id];
    if (!ctx->owned[obj_id] || d.layout == rt::kLayoutPalette || d.fmt == RT_BIT1) return RT_ERR_UNSUPPORTED;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_fill_lobes(params, ctx->owned[obj_id], ctx->scales[obj_id], d.layout, d.W, d.H, d.n,
                                             d.fmt,
                                             (cudaStream_t)stream));
}

static bool valid_scene(const rt_bake_scene* S) {
    const float* f = reinterpret_cast<const float*>(S);
    for (size_t k = 0; k < sizeof(rt_bake_scene) / sizeof(float); ++k)
        if (!std::isfinite(f[k])) return false;
    return S->sphere_radius > 0.f && S->plane_half_extent > 0.f && S->fog >= 0.f && S->sun_exponent >= 0.f &&
           S->ray_offset >= 0.f;
}

rt_status rt_bake(rt_ctx* ctx, int32_t obj_id, rt_surface surface, const rt_bake_scene* scene, rt_stream_t stream) {
    if (!ctx || obj_id < 0 || obj_id >= RT_MAX_OBJECTS || !ctx->table[obj_id].live || !scene ||
        (surface != RT_SURFACE_SPHERE && surface != RT_SURFACE_PLANE) || !valid_scene(scene))
        return RT_ERR_INVALID_ARG;
    const TexDesc& d = ctx->table[obj_id];
    if (d.layout == rt::kLayoutPalette || d.fmt == RT_BIT1) return RT_ERR_UNSUPPORTED;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_bake(*scene, (int)surface, const_cast<void*>(d.base), ctx->scales[obj_id], d.W, d.H,
                                       d.n, d.fmt, d.layout, nullptr, 0, (cudaStream_t)stream));
}

rt_status rt_bake_deferred(rt_ctx* ctx, int32_t obj_id, rt_surface surface, const rt_bake_scene* scene,
                           const float* ao_dirs, int32_t K, rt_stream_t stream) {
    if (!ctx || obj_id < 0 || obj_id >= RT_MAX_OBJECTS || !ctx->table[obj_id].live || !scene ||
        (surface != RT_SURFACE_SPHERE && surface != RT_SURFACE_PLANE) || !valid_scene(scene) || !ao_dirs ||
        K < 1 || K > RT_MAX_AO_DIRECTIONS || (reinterpret_cast<uintptr_t>(ao_dirs) & 3))
        return RT_ERR_INVALID_ARG;
    const TexDesc& d = ctx->table[obj_id];
    if (d.layout == rt::kLayoutPalette || d.fmt == RT_BIT1) return RT_ERR_UNSUPPORTED;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_bake(*scene, (int)surface, const_cast<void*>(d.base), ctx->scales[obj_id], d.W, d.H,
                                       d.n, d.fmt, d.layout, ao_dirs, K, (cudaStream_t)stream));
}

static bool kmeans_source(rt_ctx* ctx, int32_t obj_id, int32_t K) {
    if (!ctx || obj_id < 0 || obj_id >= RT_MAX_OBJECTS || !ctx->table[obj_id].live) return false;
    const TexDesc& d = ctx->table[obj_id];
    return K >= 1 && K <= (1 << 24) && d.fmt != RT_BIT1 &&
           (d.layout == RT_LAYOUT_PLANES || d.layout == RT_LAYOUT_QUADS || d.layout == RT_LAYOUT_ATLAS);
}

rt_status rt_kmeans_init(rt_ctx* ctx, int32_t obj_id, int32_t K, const int32_t* buckets, float* centroids,
                         rt_stream_t stream) {
    if (!kmeans_source(ctx, obj_id, K) || !buckets || !centroids || !aligned16(centroids)) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_kmeans_init(ctx->table[obj_id], K, buckets, centroids, ctx->d_status,
                                              (cudaStream_t)stream));
}

rt_status rt_kmeans_assign(rt_ctx* ctx, int32_t obj_id, int32_t K, const float* centroids, uint32_t* index,
                           float* dist, rt_stream_t stream) {
    if (!kmeans_source(ctx, obj_id, K) || !centroids || !aligned16(centroids) || !index) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_kmeans_assign(ctx->table[obj_id], K, centroids, index, dist, (cudaStream_t)stream));
}

int64_t rt_kmeans_tc_scratch_bytes(int32_t w, int32_t h, int32_t n, int32_t K) {
    if (w < 1 || h < 1 || n < 1 || n > 64 || K < 1) return -1;
    return rt::kmeans_tc_scratch_bytes(w, h, n, K);
}

rt_status rt_kmeans_assign_tc(rt_ctx* ctx, int32_t obj_id, int32_t K, const float* centroids, uint32_t* index,
                              float* dist, void* scratch, int64_t scratch_bytes, rt_stream_t stream) {
    if (!kmeans_source(ctx, obj_id, K) || !centroids || !aligned16(centroids) || !index || !scratch ||
        (reinterpret_cast<uintptr_t>(scratch) & 1023u) != 0)
        return RT_ERR_INVALID_ARG;
    const TexDesc& d = ctx->table[obj_id];
    if (scratch_bytes < rt::kmeans_tc_scratch_bytes(d.W, d.H, d.n, K)) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    cudaError_t e = rt::launch_kmeans_assign_tc(d, K, centroids, index, dist, scratch, ctx->d_status,
                                                ctx->wait_limit, (cudaStream_t)stream);
    return e == cudaErrorNotSupported ? RT_ERR_UNSUPPORTED : cuda_status(e);
}

rt_status rt_set_wait_limit(rt_ctx* ctx, uint32_t polls) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    ctx->wait_limit = polls;
    return RT_OK;
}

rt_status rt_kmeans_update(rt_ctx* ctx, int32_t obj_id, int32_t K, const uint32_t* index, float* centroids,
                           uint32_t* scratch, rt_stream_t stream) {
    if (!kmeans_source(ctx, obj_id, K) || !index || !centroids || !aligned16(centroids) || !scratch)
        return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_kmeans_update(ctx->table[obj_id], K, index, centroids, scratch, ctx->d_status,
                                                (cudaStream_t)stream));
}

rt_status rt_shade(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int64_t F, rt_filter filter,
                   float* out, rt_stream_t stream) {
    if (!ctx || !valid_filter(filter)) return RT_ERR_INVALID_ARG;
    rt_status st = check_gbuffer(uv, dir, obj, F);
    if (st != RT_OK) return st;
    if (F == 0) return RT_OK;
    if (!out || !aligned16(out)) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_shade(ctx->d_table, ctx->n_obj, uv, dir, obj, F, filter, rt::flat_tiling(), ctx->spec, out,
                                        ctx->d_status, (cudaStream_t)stream));
}

rt_status rt_locate(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int64_t F, rt_filter filter,
                    int32_t* idx, float* coord, rt_stream_t stream) {
    if (!ctx || !valid_filter(filter)) return RT_ERR_INVALID_ARG;
    rt_status st = check_gbuffer(uv, dir, obj, F);
    if (st != RT_OK) return st;
    if (F == 0) return RT_OK;
    if (!idx || !coord || !aligned16(idx) || !aligned16(coord)) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_locate(ctx->d_table, ctx->n_obj, uv, dir, obj, F, filter, idx, coord,
                                         ctx->d_status, (cudaStream_t)stream));
}

}  // extern "C"

// nrm == NULL: tangent-space backward on tiling T; otherwise world-space
// (Eq. 1a) on the flat stream, with dL/dN into dL_dnrm.
// The L2 step's extra arguments: with them the backward pass is the fused
// forward + loss + backward kernel, which forms dL/dout itself.
struct FusedL2 {
    const float* target;
    float scale;
    float* out;
    double* sums;
};

static rt_status shade_backward_impl(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int64_t F,
                                     rt_filter filter, const rt::Tiling& T, const float* dL_dout,
                                     float* const* dL_dtex, int32_t n_dtex, float* dL_duv, float* dL_ddir,
                                     int32_t flags, rt_stream_t stream, const float* nrm = nullptr,
                                     float* dL_dnrm = nullptr, const FusedL2* fused = nullptr) {
    if (!ctx || !valid_filter(filter)) return RT_ERR_INVALID_ARG;
    rt_status st = check_gbuffer(uv, dir, obj, F);
    if (st != RT_OK) return st;
    if (nrm == nullptr && dL_dnrm != nullptr) return RT_ERR_INVALID_ARG;
    if (F > 0 && nrm && !aligned16(nrm)) return RT_ERR_INVALID_ARG;
    if (dL_dnrm && !aligned16(dL_dnrm)) return RT_ERR_INVALID_ARG;
    if (n_dtex < 0 || n_dtex > RT_MAX_OBJECTS || (n_dtex > 0 && !dL_dtex)) return RT_ERR_INVALID_ARG;
    if ((dL_duv && !aligned16(dL_duv)) || (dL_ddir && !aligned16(dL_ddir))) return RT_ERR_INVALID_ARG;
    if (fused) {
        if (F > 0 && (!fused->target || !aligned16(fused->target))) return RT_ERR_INVALID_ARG;
        if ((fused->out && !aligned16(fused->out)) || (reinterpret_cast<uintptr_t>(fused->sums) & 7) ||
            !std::isfinite(fused->scale))
            return RT_ERR_INVALID_ARG;
    } else if (F > 0 && (!dL_dout || !aligned16(dL_dout))) {
        return RT_ERR_INVALID_ARG;
    }
    const bool accumulate = (flags & RT_ACCUMULATE) != 0;                       // every output adds
    const bool accumulate_tex = accumulate || (flags & RT_ACCUMULATE_TEXELS) != 0;  // the texel gradients add
    const bool fixed_out = (flags & RT_FIXED_POINT_GRADS) != 0;  // the caller's buffers hold the fixed-point sums
    const bool deterministic = (flags & RT_DETERMINISTIC) != 0 || fixed_out;
    rt::GradTable grads;
    std::memset(&grads, 0, sizeof(grads));
    bool any = false;
    for (int o = 0; o < n_dtex; ++o) {
        if (!dL_dtex[o]) continue;
        if (o >= RT_MAX_OBJECTS || !ctx->table[o].live || !aligned16(dL_dtex[o])) return RT_ERR_INVALID_ARG;
        if (deterministic && !fixed_out && !ctx->det[o]) return RT_ERR_INVALID_ARG;  // rt_prepare_deterministic first
        if (ctx->table[o].fmt == RT_BIT1) return RT_ERR_UNSUPPORTED;   // bits have no texel gradient
        grads.p[o] = (deterministic && !fixed_out) ? static_cast<void*>(ctx->det[o]) : static_cast<void*>(dL_dtex[o]);
        any = true;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    for (int o = 0; o < n_dtex && e == cudaSuccess; ++o) {
        if (!grads.p[o]) continue;
        const TexDesc& d = ctx->table[o];
        const size_t texels = (size_t)d.plane * d.n * d.n;
        if (fixed_out) {
            if (!accumulate_tex) e = cudaMemsetAsync(dL_dtex[o], 0, 32 * texels, s);
        } else if (deterministic)
            e = cudaMemsetAsync(ctx->det[o], 0, 32 * texels, s);
        else if (!accumulate_tex)
            e = cudaMemsetAsync(dL_dtex[o], 0, 16 * texels, s);
    }
    if (e == cudaSuccess && F > 0) {
        if (nrm)
            e = rt::launch_world_backward(ctx->d_table, ctx->n_obj, uv, dir, nrm, obj, F, filter, T, dL_dout, grads,
                                          any, dL_duv, dL_ddir, dL_dnrm, accumulate, deterministic, ctx->d_status, s);
        else if (fused)
            e = rt::launch_fused_l2(ctx->d_table, ctx->n_obj, uv, dir, obj, F, filter, T, ctx->spec, fused->target,
                                    fused->scale, fused->out, fused->sums, grads, any, dL_duv, dL_ddir, accumulate,
                                    deterministic, ctx->d_status, s);
        else
            e = rt::launch_backward(ctx->d_table, ctx->n_obj, uv, dir, obj, F, filter, T, ctx->spec, dL_dout, grads, any,
                                    dL_duv, dL_ddir, accumulate, deterministic, ctx->d_status, s);
    }
    if (deterministic && !fixed_out)
        for (int o = 0; o < n_dtex && e == cudaSuccess; ++o)
            if (grads.p[o]) {
                const TexDesc& d = ctx->table[o];
                e = rt::launch_fixed_to_float(ctx->det[o], dL_dtex[o], (int64_t)d.plane * d.n * d.n * 4,
                                              accumulate_tex, s);
            }
    return cuda_status(e);
}

enum { kForward = 0, kBackward = 1 };

static bool frames_tiling(rt_ctx* ctx, int pass, int32_t views, int32_t height, int32_t width, rt_filter filter,
                          rt::Tiling* T) {
    const int* t = ctx->tile[pass][filter];
    return rt::make_tiling(views, height, width, t[0], t[1], t[2], t[3], 4, T);
}

static rt_status set_tile(rt_ctx* ctx, int pass, rt_filter filter, int32_t tw, int32_t th, int32_t bx, int32_t by) {
    if (!ctx || !valid_filter(filter)) return RT_ERR_INVALID_ARG;
    rt::Tiling T;
    if (!rt::make_tiling(1, 1, 1, tw, th, bx, by, 4, &T)) return RT_ERR_INVALID_ARG;
    for (int p = 0; p < 2; ++p) {
        if (pass >= 0 && p != pass) continue;
        ctx->tile[p][filter][0] = tw;
        ctx->tile[p][filter][1] = th;
        ctx->tile[p][filter][2] = bx;
        ctx->tile[p][filter][3] = by;
    }
    return RT_OK;
}

// Times `run` (one launch of a batched pass) with each candidate tile written
// into `tile`, `reps` launches after one warm-up, and keeps the fastest.
template <class Run>
static rt_status tune_tile(int (&tile)[4], Run run, int reps, cudaStream_t s, int32_t* tile4, float* best_ms) {
    static const int kCand[][4] = {{32, 1, 4, 1}, {32, 1, 2, 2}, {32, 1, 1, 4}, {16, 2, 4, 1}, {16, 2, 2, 2},
                                   {16, 2, 1, 4}, {8, 4, 4, 1},  {8, 4, 2, 2},  {8, 4, 1, 4},  {4, 8, 4, 1},
                                   {4, 8, 2, 2},  {4, 8, 1, 4}};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return RT_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return RT_ERR_CUDA;
    }
    int saved[4];
    for (int k = 0; k < 4; ++k) saved[k] = tile[k];
    float best = 1e30f;
    int best_k = -1;
    rt_status st = RT_OK;
    for (int c = 0; c < (int)(sizeof(kCand) / sizeof(kCand[0])) && st == RT_OK; ++c) {
        for (int k = 0; k < 4; ++k) tile[k] = kCand[c][k];
        st = run();  // warm-up
        if (st != RT_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == RT_OK; ++r) st = run();
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = RT_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st == RT_OK && ms < best) {
            best = ms;
            best_k = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RT_OK || best_k < 0) {
        for (int k = 0; k < 4; ++k) tile[k] = saved[k];
        return st != RT_OK ? st : RT_ERR_CUDA;
    }
    for (int k = 0; k < 4; ++k) tile[k] = kCand[best_k][k];
    if (tile4)
        for (int k = 0; k < 4; ++k) tile4[k] = kCand[best_k][k];
    if (best_ms) *best_ms = best / (float)reps;
    return RT_OK;
}

extern "C" {

rt_status rt_shade_backward(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int64_t F,
                            rt_filter filter, const float* dL_dout, float* const* dL_dtex, int32_t n_dtex,
                            float* dL_duv, float* dL_ddir, int32_t flags, rt_stream_t stream) {
    return shade_backward_impl(ctx, uv, dir, obj, F, filter, rt::flat_tiling(), dL_dout, dL_dtex, n_dtex, dL_duv,
                               dL_ddir, flags, stream);
}

rt_status rt_bake_shadow(rt_ctx* ctx, int32_t obj_id, rt_surface surface, const rt_bake_scene* scene,
                         rt_stream_t stream) {
    if (!ctx || obj_id < 0 || obj_id >= RT_MAX_OBJECTS || !ctx->table[obj_id].live || !scene ||
        (surface != RT_SURFACE_SPHERE && surface != RT_SURFACE_PLANE) || !valid_scene(scene))
        return RT_ERR_INVALID_ARG;
    const TexDesc& d = ctx->table[obj_id];
    if (d.fmt != RT_BIT1 || !ctx->owned[obj_id] || d.layout != RT_LAYOUT_PLANES) return RT_ERR_UNSUPPORTED;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_bake_shadow(*scene, (int)surface, ctx->owned[obj_id], d.W, d.H, d.n,
                                              (cudaStream_t)stream));
}

rt_status rt_shade_multi(rt_ctx* ctx, const float* uv, const float* dirs, int32_t samples, const int32_t* obj,
                         int64_t F, rt_filter filter, float* out, rt_stream_t stream) {
    if (!ctx || !valid_filter(filter) || samples < 1) return RT_ERR_INVALID_ARG;
    rt_status st = check_gbuffer(uv, dirs, obj, F);
    if (st != RT_OK) return st;
    if (F == 0) return RT_OK;
    if (!out || !aligned16(out)) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_multi_shade(ctx->d_table, ctx->n_obj, uv, dirs, samples, obj, F, filter, out,
                                              ctx->d_status, (cudaStream_t)stream));
}

rt_status rt_shade_world(rt_ctx* ctx, const float* uv, const float* dir, const float* nrm, const int32_t* obj,
                         int64_t F, rt_filter filter, float* out, rt_stream_t stream) {
    if (!ctx || !valid_filter(filter)) return RT_ERR_INVALID_ARG;
    rt_status st = check_gbuffer(uv, dir, obj, F);
    if (st != RT_OK) return st;
    if (F == 0) return RT_OK;
    if (!nrm || !aligned16(nrm) || !out || !aligned16(out)) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_world_shade(ctx->d_table, ctx->n_obj, uv, dir, nrm, obj, F, filter,
                                              rt::flat_tiling(), out, nullptr, nullptr, ctx->d_status,
                                              (cudaStream_t)stream));
}

rt_status rt_locate_world(rt_ctx* ctx, const float* uv, const float* dir, const float* nrm, const int32_t* obj,
                          int64_t F, rt_filter filter, int32_t* idx, float* coord, rt_stream_t stream) {
    if (!ctx || !valid_filter(filter)) return RT_ERR_INVALID_ARG;
    rt_status st = check_gbuffer(uv, dir, obj, F);
    if (st != RT_OK) return st;
    if (F == 0) return RT_OK;
    if (!nrm || !aligned16(nrm) || !idx || !coord || !aligned16(idx) || !aligned16(coord)) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_world_shade(ctx->d_table, ctx->n_obj, uv, dir, nrm, obj, F, filter,
                                              rt::flat_tiling(), nullptr, idx, coord, ctx->d_status,
                                              (cudaStream_t)stream));
}

rt_status rt_shade_world_backward(rt_ctx* ctx, const float* uv, const float* dir, const float* nrm,
                                  const int32_t* obj, int64_t F, rt_filter filter, const float* dL_dout,
                                  float* const* dL_dtex, int32_t n_dtex, float* dL_duv, float* dL_ddir,
                                  float* dL_dnrm, int32_t flags, rt_stream_t stream) {
    if (F > 0 && !nrm) return RT_ERR_INVALID_ARG;
    static const float kNone[4] = {0.f, 0.f, 0.f, 0.f};  // an unused non-null marker for F = 0
    return shade_backward_impl(ctx, uv, dir, obj, F, filter, rt::flat_tiling(), dL_dout, dL_dtex, n_dtex, dL_duv,
                               dL_ddir, flags, stream, nrm ? nrm : kNone, dL_dnrm);
}

rt_status rt_shade_batched(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int32_t views,
                           int32_t height, int32_t width, rt_filter filter, float* out, rt_stream_t stream) {
    if (!ctx || !valid_filter(filter) || views < 0 || height < 0 || width < 0 || height > 65536 || width > 65536)
        return RT_ERR_INVALID_ARG;
    const int64_t F = (int64_t)views * height * width;
    rt_status st = check_gbuffer(uv, dir, obj, F);
    if (st != RT_OK) return st;
    if (F == 0) return RT_OK;
    if (!out || !aligned16(out)) return RT_ERR_INVALID_ARG;
    rt::Tiling T;
    if (!frames_tiling(ctx, kForward, views, height, width, filter, &T)) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_shade(ctx->d_table, ctx->n_obj, uv, dir, obj, F, filter, T, ctx->spec, out, ctx->d_status,
                                        (cudaStream_t)stream));
}

rt_status rt_shade_batched_backward(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int32_t views,
                                    int32_t height, int32_t width, rt_filter filter, const float* dL_dout,
                                    float* const* dL_dtex, int32_t n_dtex, float* dL_duv, float* dL_ddir,
                                    int32_t flags, rt_stream_t stream) {
    if (!ctx || !valid_filter(filter) || views < 0 || height < 0 || width < 0 || height > 65536 || width > 65536)
        return RT_ERR_INVALID_ARG;
    const int64_t F = (int64_t)views * height * width;
    rt::Tiling T = rt::flat_tiling();
    if (F > 0 && !frames_tiling(ctx, kBackward, views, height, width, filter, &T)) return RT_ERR_INVALID_ARG;
    return shade_backward_impl(ctx, uv, dir, obj, F, filter, T, dL_dout, dL_dtex, n_dtex, dL_duv, dL_ddir, flags,
                               stream);
}

rt_status rt_shade_batched_l2_step(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int32_t views,
                                   int32_t height, int32_t width, rt_filter filter, const float* target, float scale,
                                   float* out, double* sums, float* const* dL_dtex, int32_t n_dtex, float* dL_duv,
                                   float* dL_ddir, int32_t flags, rt_stream_t stream) {
    if (!ctx || !valid_filter(filter) || views < 0 || height < 0 || width < 0 || height > 65536 || width > 65536)
        return RT_ERR_INVALID_ARG;
    const int64_t F = (int64_t)views * height * width;
    rt::Tiling T = rt::flat_tiling();
    if (F > 0 && !frames_tiling(ctx, kBackward, views, height, width, filter, &T)) return RT_ERR_INVALID_ARG;
    const FusedL2 fused = {target, scale, out, sums};
    return shade_backward_impl(ctx, uv, dir, obj, F, filter, T, nullptr, dL_dtex, n_dtex, dL_duv, dL_ddir, flags,
                               stream, nullptr, nullptr, &fused);
}

rt_status rt_shade_world_batched(rt_ctx* ctx, const float* uv, const float* dir, const float* nrm,
                                 const int32_t* obj, int32_t views, int32_t height, int32_t width, rt_filter filter,
                                 float* out, rt_stream_t stream) {
    if (!ctx || !valid_filter(filter) || views < 0 || height < 0 || width < 0 || height > 65536 || width > 65536)
        return RT_ERR_INVALID_ARG;
    const int64_t F = (int64_t)views * height * width;
    rt_status st = check_gbuffer(uv, dir, obj, F);
    if (st != RT_OK) return st;
    if (F == 0) return RT_OK;
    if (!nrm || !aligned16(nrm) || !out || !aligned16(out)) return RT_ERR_INVALID_ARG;
    rt::Tiling T;
    if (!frames_tiling(ctx, kForward, views, height, width, filter, &T)) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    return cuda_status(rt::launch_world_shade(ctx->d_table, ctx->n_obj, uv, dir, nrm, obj, F, filter, T, out, nullptr,
                                              nullptr, ctx->d_status, (cudaStream_t)stream));
}

rt_status rt_shade_world_batched_backward(rt_ctx* ctx, const float* uv, const float* dir, const float* nrm,
                                          const int32_t* obj, int32_t views, int32_t height, int32_t width,
                                          rt_filter filter, const float* dL_dout, float* const* dL_dtex,
                                          int32_t n_dtex, float* dL_duv, float* dL_ddir, float* dL_dnrm,
                                          int32_t flags, rt_stream_t stream) {
    if (!ctx || !valid_filter(filter) || views < 0 || height < 0 || width < 0 || height > 65536 || width > 65536)
        return RT_ERR_INVALID_ARG;
    const int64_t F = (int64_t)views * height * width;
    if (F > 0 && !nrm) return RT_ERR_INVALID_ARG;
    rt::Tiling T = rt::flat_tiling();
    if (F > 0 && !frames_tiling(ctx, kBackward, views, height, width, filter, &T)) return RT_ERR_INVALID_ARG;
    static const float kNone[4] = {0.f, 0.f, 0.f, 0.f};  // an unused non-null marker for F = 0
    return shade_backward_impl(ctx, uv, dir, obj, F, filter, T, dL_dout, dL_dtex, n_dtex, dL_duv, dL_ddir, flags,
                               stream, nrm ? nrm : kNone, dL_dnrm);
}

rt_status rt_fixed_to_float(const int64_t* acc, float* dst, int64_t count, double scale, int32_t flags,
                            rt_stream_t stream) {
    if (count < 0 || (count > 0 && (!acc || !dst)) || !aligned16(acc) || !aligned16(dst) || !std::isfinite(scale))
        return RT_ERR_INVALID_ARG;
    return cuda_status(rt::launch_fixed_to_float(reinterpret_cast<const long long*>(acc), dst, count,
                                                 (flags & RT_ACCUMULATE) != 0, (cudaStream_t)stream, scale));
}

rt_status rt_zero_texture_grads(rt_ctx* ctx, float* const* dL_dtex, int32_t n_dtex, rt_stream_t stream) {
    if (!ctx || n_dtex < 0 || n_dtex > RT_MAX_OBJECTS || (n_dtex > 0 && !dL_dtex)) return RT_ERR_INVALID_ARG;
    for (int o = 0; o < n_dtex; ++o)
        if (dL_dtex[o] && (!ctx->table[o].live || !aligned16(dL_dtex[o]))) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    for (int o = 0; o < n_dtex && e == cudaSuccess; ++o) {
        if (!dL_dtex[o]) continue;
        const TexDesc& d = ctx->table[o];
        e = cudaMemsetAsync(dL_dtex[o], 0, (size_t)16 * d.plane * d.n * d.n, (cudaStream_t)stream);
    }
    return cuda_status(e);
}

rt_status rt_prepare_deterministic(rt_ctx* ctx) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    for (int o = 0; o < ctx->n_obj; ++o) {
        const TexDesc& d = ctx->table[o];
        if (!d.live || ctx->det[o]) continue;
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, (size_t)32 * d.plane * d.n * d.n);
        if (e != cudaSuccess) return cuda_status(e);
        ctx->det[o] = static_cast<long long*>(p);
    }
    return RT_OK;
}

rt_status rt_set_tile(rt_ctx* ctx, rt_filter filter, int32_t tw, int32_t th, int32_t bx, int32_t by) {
    return set_tile(ctx, -1, filter, tw, th, bx, by);
}

rt_status rt_set_backward_tile(rt_ctx* ctx, rt_filter filter, int32_t tw, int32_t th, int32_t bx, int32_t by) {
    return set_tile(ctx, kBackward, filter, tw, th, bx, by);
}

rt_status rt_get_tile(rt_ctx* ctx, rt_filter filter, int32_t* tile4) {
    if (!ctx || !valid_filter(filter) || !tile4) return RT_ERR_INVALID_ARG;
    for (int k = 0; k < 4; ++k) tile4[k] = ctx->tile[kForward][filter][k];
    return RT_OK;
}

rt_status rt_get_backward_tile(rt_ctx* ctx, rt_filter filter, int32_t* tile4) {
    if (!ctx || !valid_filter(filter) || !tile4) return RT_ERR_INVALID_ARG;
    for (int k = 0; k < 4; ++k) tile4[k] = ctx->tile[kBackward][filter][k];
    return RT_OK;
}

rt_status rt_autotune(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int32_t views,
                      int32_t height, int32_t width, rt_filter filter, float* out, int32_t reps, rt_stream_t stream,
                      int32_t* tile4, float* best_ms) {
    if (!ctx || !valid_filter(filter) || views < 1 || height < 1 || width < 1 || reps < 1) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    auto run = [&]() { return rt_shade_batched(ctx, uv, dir, obj, views, height, width, filter, out, stream); };
    return tune_tile(ctx->tile[kForward][filter], run, reps, (cudaStream_t)stream, tile4, best_ms);
}

rt_status rt_autotune_backward(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int32_t views,
                               int32_t height, int32_t width, rt_filter filter, const float* dL_dout,
                               float* const* dL_dtex, int32_t n_dtex, float* dL_duv, float* dL_ddir, int32_t flags,
                               int32_t reps, rt_stream_t stream, int32_t* tile4, float* best_ms) {
    if (!ctx || !valid_filter(filter) || views < 1 || height < 1 || width < 1 || reps < 1) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    auto run = [&]() {
        return rt_shade_batched_backward(ctx, uv, dir, obj, views, height, width, filter, dL_dout, dL_dtex, n_dtex,
                                         dL_duv, dL_ddir, flags, stream);
    };
    return tune_tile(ctx->tile[kBackward][filter], run, reps, (cudaStream_t)stream, tile4, best_ms);
}

rt_status rt_footprint(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int64_t F,
                       rt_filter filter, uint64_t* counts_host, int32_t n_counts, rt_stream_t stream) {
    if (!ctx || !valid_filter(filter) || !counts_host || n_counts < 0) return RT_ERR_INVALID_ARG;
    rt_status st = check_gbuffer(uv, dir, obj, F);
    if (st != RT_OK) return st;
    for (int o = 0; o < n_counts; ++o) counts_host[o] = 0;
    if (F == 0) return RT_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> offset(ctx->n_obj + 1, 0);
    for (int o = 0; o < ctx->n_obj; ++o) {
        const TexDesc& d = ctx->table[o];
        int64_t texels = d.live ? d.plane * d.n * d.n : 0;
        offset[o + 1] = offset[o] + (texels + 31) / 32;
    }
    const int64_t words = offset[ctx->n_obj];
    uint32_t* bitmap = nullptr;
    int64_t* d_offset = nullptr;
    unsigned long long* d_count = nullptr;
    cudaError_t e = cudaMalloc(&bitmap, sizeof(uint32_t) * (size_t)(words > 0 ? words : 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_offset, sizeof(int64_t) * offset.size());
    if (e == cudaSuccess) e = cudaMalloc(&d_count, sizeof(unsigned long long) * (size_t)(ctx->n_obj + 1));
    if (e == cudaSuccess) e = cudaMemsetAsync(bitmap, 0, sizeof(uint32_t) * (size_t)(words > 0 ? words : 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long) * (size_t)(ctx->n_obj + 1), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_offset, offset.data(), sizeof(int64_t) * offset.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = rt::launch_footprint_mark(ctx->d_table, ctx->n_obj, uv, dir, obj, F, filter, bitmap, d_offset,
                                      ctx->d_status, s);
    for (int o = 0; o < ctx->n_obj && e == cudaSuccess; ++o)
        e = rt::launch_popcount(bitmap + offset[o], offset[o + 1] - offset[o], d_count + o, s);
    std::vector<unsigned long long> h((size_t)ctx->n_obj + 1, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d_count, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(bitmap);
    cudaFree(d_offset);
    cudaFree(d_count);
    if (e != cudaSuccess) return cuda_status(e);
    for (int o = 0; o < n_counts && o < ctx->n_obj; ++o) counts_host[o] = h[o];
    return RT_OK;
}

rt_status rt_convert_layout(const float* src, rt_layout src_layout, float* dst, rt_layout dst_layout, int32_t w,
                            int32_t h, int32_t n, rt_stream_t stream) {
    if (!src || !dst || !aligned16(src) || !aligned16(dst) || w < 1 || h < 1 || n < 1) return RT_ERR_INVALID_ARG;
    auto ok = [](rt_layout l) { return l == RT_LAYOUT_ATLAS || l == RT_LAYOUT_PLANES || l == RT_LAYOUT_QUADS; };
    if (!ok(src_layout) || !ok(dst_layout))
        return RT_ERR_INVALID_ARG;
    return cuda_status(rt::launch_convert(src, src_layout, dst, dst_layout, w, h, n, (cudaStream_t)stream));
}

rt_status rt_checked_limit_extent(rt_ctx* ctx, int32_t obj_id, int64_t texels) {
#ifdef RADTEX_CHECKED
    if (!ctx || obj_id < 0 || obj_id >= ctx->n_obj || !ctx->table[obj_id].live) return RT_ERR_INVALID_ARG;
    TexDesc& d = ctx->table[obj_id];
    if (texels < 0 || texels > d.plane * d.n * d.n) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    d.extent = texels;
    return upload_table(ctx);
#else
    (void)ctx;
    (void)obj_id;
    (void)texels;
    return RT_ERR_UNSUPPORTED;
#endif
}

rt_status rt_get_error(rt_ctx* ctx, rt_stream_t stream, rt_status* device_status) {
    if (!ctx || !device_status) return RT_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return RT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    unsigned bits = *ctx->h_status;
    *device_status = (bits & rt::ST_BOUNDS)      ? RT_ERR_OUT_OF_BOUNDS
                     : (bits & rt::ST_BAD_OBJ)   ? RT_ERR_BAD_OBJ_ID
                     : (bits & rt::ST_NONFINITE) ? RT_ERR_NONFINITE
                     : (bits & rt::ST_TIMEOUT)   ? RT_ERR_TIMEOUT
                     : (bits & rt::ST_BAD_ARG)   ? RT_ERR_INVALID_ARG
                                                 : RT_OK;
    return RT_OK;
}

}  // extern "C"

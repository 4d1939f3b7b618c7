/*
 * radtex.h -- C ABI of libradtex, GPU radiance-texture synthesis for GB300 (sm_103a).
 *
 * The method (J. M. Fober, "Radiance Textures for Rasterizing Ray-Traced Data",
 * arXiv 2301.01719, Section 2): every texel of an ordinary w x h texture is
 * replaced by a "bucket", an n x n discrete hemispherical radiance map.  A
 * fragment's surface UV selects the bucket, and its incidence vector, mapped by
 * the equisolid projection (Eq. 1b) and the disc-to-square mapping (Eq. 3) and
 * clamped to the texel-centre range (Note after Eq. 3), selects the texels
 * inside the bucket.  The texels are filtered in FP32 into the output colour.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named "device" are CUDA device pointers of the context's device;
 *   the caller owns them.  "host" pointers are ordinary host memory.
 * - All compute calls are asynchronous on the given stream (a cudaStream_t; NULL
 *   is the legacy default stream), neither allocate nor synchronise, and may be
 *   captured in a CUDA graph, unless their comment says otherwise.  Texture
 *   creation and destruction are synchronous set-up calls.
 * - Errors are returned as rt_status; nothing is thrown across the ABI.
 *   Problems found on the device (an object id with no texture, a non-finite
 *   UV or direction) make that fragment's outputs zero and set a sticky status
 *   word that rt_get_error reads and clears.
 * - G-buffer: F fragments, structure of arrays: uv (F x 2 float: u, v),
 *   dir (F x 3 float: the tangent-space unit vector from the surface to the
 *   eye, x along dP/du, y along dP/dv, z along the normal), obj (F int32:
 *   object id, < 0 = background, whose outputs are zero and which reads no
 *   texel).  uv, dir, obj and every F x k output must start on a 16-byte
 *   boundary (RT_ERR_INVALID_ARG otherwise).
 * - Texel (i, j, s, t) of an object is bucket column i (0..w-1, from u), bucket
 *   row j (0..h-1, from v), in-bucket column s (0..n-1, from B_x) and row t
 *   (from B_y); each texel holds 4 channels (RGBA).  Layouts:
 *     RT_LAYOUT_ATLAS : the paper's texture, row-major (h n) x (w n) texels,
 *                       texel (i, j, s, t) at row j n + t, column i n + s.
 *     RT_LAYOUT_PLANES: n x n planes of w x h texels, texel (i, j, s, t) at
 *                       index ((t n + s) h + j) w + i: fragments that are close
 *                       on screen read texels that are close in memory.
 *     RT_LAYOUT_QUADS : the planes of RT_LAYOUT_PLANES with each plane's
 *                       buckets in 2 x 2 quads: a plane holds wq x hq quads,
 *                       wq = ceil(w / 2), hq = ceil(h / 2) (an odd side is
 *                       padded; P = 4 wq hq buckets per plane), texel
 *                       (i, j, s, t) at index (t n + s) P + 4 q + 2 (j mod 2)
 *                       + (i mod 2), quad q = (j / 2) wq + i / 2.  The 2 x 2
 *                       buckets of a quadrilinear lookup at one in-bucket texel
 *                       then lie in one quad more often, and a warp's taps and
 *                       texel-gradient reductions in fewer cache lines.  A
 *                       QUADS buffer holds P n^2 texels; the padding is never
 *                       read by a lookup, is zero in owned textures and is not
 *                       written by rt_convert_layout or rt_read_texture.
 *   Textures the library owns are stored in RT_LAYOUT_QUADS, bit textures
 *   (RT_BIT1) in RT_LAYOUT_PLANES (rt_texture_info reports the layout).
 */
#ifndef RADTEX_H
#define RADTEX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* rt_stream_t; /* identical to cudaStream_t */
typedef struct rt_ctx rt_ctx;

typedef enum {
    RT_OK = 0,
    RT_ERR_INVALID_ARG = 1,  /* a null, misaligned or out-of-range argument */
    RT_ERR_OOM = 2,          /* device allocation failed (set-up calls only) */
    RT_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    RT_ERR_BAD_OBJ_ID = 4,   /* device: an object id names no texture */
    RT_ERR_NONFINITE = 5,    /* device: a UV or direction was NaN or infinite */
    RT_ERR_TIMEOUT = 6,      /* device: a bounded wait gave up */
    RT_ERR_UNSUPPORTED = 7,  /* the combination of options is not implemented */
    RT_ERR_OUT_OF_BOUNDS = 8 /* device, checked build only: a computed texel address fell outside its object */
} rt_status;

typedef enum {
    RT_F32 = 0,              /* 16 bytes per texel */
    RT_F16 = 1,              /* 8 bytes per texel, round to nearest even */
    RT_BF16 = 2,             /* 8 bytes per texel, round to nearest even */
    RT_E4M3_BUCKET_SCALE = 3, /* 4 bytes per texel: OCP FP8 E4M3 codes of v / s, s = (bucket amax) / 448 */
    RT_BIT1 = 4               /* 1 bit per texel (shadow textures, Section 5): bit k of 32-bit word k >> 5 holds
                                 texel k of the PLANES numbering (always the storage layout of bit
                                 textures); the value (0 or 1) fills every channel.
                                 Created from FP32 by channel 0 >= 1/2, or by rt_bake_shadow */
} rt_format;

typedef enum {
    RT_NEAREST = 0,          /* nearest bucket, nearest texel: 1 tap */
    RT_ANGULAR_BILINEAR = 1, /* nearest bucket, bilinear inside it ("single sample per bucket", Section 2): 4 taps */
    RT_QUADRILINEAR = 2      /* bilinear over u, v and over s, t: 16 taps */
} rt_filter;

typedef enum { RT_LAYOUT_ATLAS = 0, RT_LAYOUT_PLANES = 1, RT_LAYOUT_QUADS = 3 } rt_layout;
/* (2 is reported by rt_texture_info for a palette texture) */

/* rt_create_texture / rt_create_palette_texture flags */
#define RT_BORROW 1          /* use the caller's FP32 buffer in place; no copy */
#define RT_WRAP_U 2          /* repeat in u: taps floor(c) mod w instead of clamp to edge (|u| w < 2^30) */
#define RT_WRAP_V 4          /* repeat in v likewise */
/* rt_shade_backward flags */
#define RT_ACCUMULATE 1      /* add into dL_dtex / dL_duv / dL_ddir instead of overwriting */
#define RT_DETERMINISTIC 2   /* bit-reproducible texel gradients (fixed-point sums; see rt_prepare_deterministic) */
#define RT_FIXED_POINT_GRADS 4 /* dL_dtex entries are int64 buffers that receive the raw fixed-point sums (below) */
#define RT_ACCUMULATE_TEXELS 8 /* add into dL_dtex (no clear first) but overwrite dL_duv / dL_ddir / dL_dnrm */

#define RT_MAX_OBJECTS 1024

/* Creates a context on CUDA device `cuda_device`: a texture table and a sticky
 * device status word.  *out receives the context; RT_ERR_INVALID_ARG for a bad
 * device index, RT_ERR_OOM / RT_ERR_CUDA on failure. */
rt_status rt_context_create(int cuda_device, rt_ctx** out);

/* Destroys the context and frees every texture it owns (synchronises the device). */
void rt_context_destroy(rt_ctx* ctx);

/* Creates a radiance texture of w x h buckets of n x n texels (Section 2: the
 * bucket matrix, stored as w n x h n texels).  1 <= w, h <= 65536, w h <= 2^30, 1 <= n <= 64.
 * src (device, FP32, 4 channels per texel, layout src_layout; a QUADS buffer
 * holds P n^2 texels, see above) gives the texel values; NULL leaves an owned
 * texture zero (fill it with rt_fill_bucket_lobes).  Without RT_BORROW the
 * library allocates storage (RT_LAYOUT_QUADS, or RT_LAYOUT_PLANES for RT_BIT1)
 * and encodes src into `storage` (E4M3: one FP32 scale per bucket,
 * s = amax / 448, s = 1 for an all-zero bucket; codes =
 * round-to-nearest-even-satfinite(v / s)).
 * With RT_BORROW, `storage` must be RT_F32 and src non-NULL: the library reads
 * src in place, in src_layout, for as long as the texture lives; the caller
 * keeps it alive and may update its values between calls (texture fitting).
 * *obj_id_out receives the object id used in the G-buffer's obj array.
 * Synchronous.  RT_ERR_INVALID_ARG for bad sizes/pointers, RT_ERR_OOM when the
 * storage or the RT_MAX_OBJECTS ids are exhausted. */
rt_status rt_create_texture(rt_ctx* ctx, int32_t w, int32_t h, int32_t n, rt_format storage, rt_layout src_layout,
                            const float* src, int32_t flags, int32_t* obj_id_out);

/* Releases an object id and the storage the library owns for it (synchronises
 * the device).  Fragments that still name the id read no texel and set
 * RT_ERR_BAD_OBJ_ID. */
rt_status rt_destroy_texture(rt_ctx* ctx, int32_t obj_id);

/* Properties of an object (any output pointer may be NULL).  bytes = texel
 * storage plus scales (plus the index map of a palette texture); layout is the
 * storage layout (an rt_layout; that of the caller's buffer for a borrowed
 * texture), or 2 for a palette texture (w, h are then its bucket matrix; its
 * K x 1 palette is stored in RT_LAYOUT_PLANES).  Texel gradients
 * (rt_shade_backward's dL_dtex) use the same layout. */
rt_status rt_texture_info(rt_ctx* ctx, int32_t obj_id, int32_t* w, int32_t* h, int32_t* n, int32_t* storage,
                          int32_t* layout, int64_t* bytes);

/* Copies the stored codes of an object into codes_dst (device; w n h n x 4
 * elements of the storage type: float, uint16 (FP16/BF16 bits) or uint8
 * (E4M3 codes)) in dst_layout (a QUADS buffer holds P n^2 texels, its padding
 * not written), and for E4M3 the per-bucket scales into scales_dst (device, h x w floats in row-major
 * bucket order, may be NULL).  Used to check the encoders. */
rt_status rt_read_texture(rt_ctx* ctx, int32_t obj_id, rt_layout dst_layout, void* codes_dst, float* scales_dst,
                          rt_stream_t stream);

/* Fills an owned texture from one cosine-power lobe per bucket, evaluated at
 * every texel centre's direction: B_k = (2k + 1)/n - 1, A = Eq. 4a(B),
 * I = Eq. 2c(A); T_c = rho_c max(0, I . d)^p (c < 3), T_3 = max(0, I . d)^p;
 * then encodes as rt_create_texture does.  params (device): h x w x 8 floats
 * per bucket (rho_r, rho_g, rho_b, d_x, d_y, d_z, p, unused), row-major.
 * RT_ERR_UNSUPPORTED for a borrowed texture. */
rt_status rt_fill_bucket_lobes(rt_ctx* ctx, int32_t obj_id, const float* params, rt_stream_t stream);

/* Palette textures: bucket compression.  Section 2 notes that buckets are
 * highly repetitive and change only slightly from one to another, which
 * suits a simple compression.  A palette texture stores K palette buckets of
 * n x n texels plus a w x h index map; bucket (i, j) reads palette bucket
 * index[j w + i].  Shading, lookup, footprint and backward accept palette
 * textures unchanged.  Their texel gradients are per palette texel: dL_dtex
 * holds K n^2 texels in PLANES order (n, n, K, 4).  rt_fill_bucket_lobes and
 * rt_bake return RT_ERR_UNSUPPORTED for them.
 * palette (device, FP32): the K buckets as a K x 1 texture in src_layout,
 * i.e. n x K n texels (ATLAS) or (n, n, K, 4) (PLANES), encoded into
 * `storage`.  E4M3 has one scale per palette bucket.
 * index (device, h x w uint32): every entry must be < K, else
 * RT_ERR_INVALID_ARG.  The map is copied.
 * RT_BORROW (FP32, PLANES only) uses the caller's palette buffer in place.
 * 1 <= K <= 2^30.  Synchronous; allocates the palette (unless borrowed) and
 * the index map. */
rt_status rt_create_palette_texture(rt_ctx* ctx, int32_t w, int32_t h, int32_t n, int32_t K, rt_format storage,
                                    rt_layout src_layout, const float* palette, const uint32_t* index, int32_t flags,
                                    int32_t* obj_id_out);

/* *K = the palette size of obj_id, 0 for a dense texture.  rt_read_texture of
 * a palette texture returns its palette as a K x 1 texture. */
rt_status rt_palette_size(rt_ctx* ctx, int32_t obj_id, int32_t* K);

/* The palette encoder: Lloyd's k-means over the buckets of a dense texture
 * (owned, or borrowed FP32), each bucket a vector x_b of n^2 x 4 decoded
 * texel values, b = j w + i.  Centroids are FP32 in a K x 1 texture's PLANES
 * order: centroid k, texel (s, t) at float4 (t n + s) K + k.  So a centroid
 * buffer is a valid `palette` for rt_create_palette_texture with
 * RT_LAYOUT_PLANES, and the assignment is its index map.  1 <= K <= 2^24.
 * All three calls are asynchronous on `stream` and allocate nothing.
 *
 * rt_kmeans_init: centroid k = x_{buckets[k]}.  buckets is device int32 x K.
 * An entry outside [0, w h) is clamped and raises RT_ERR_INVALID_ARG in
 * rt_get_error.
 *
 * rt_kmeans_assign: index[b] = argmin_k |x_b - c_k|^2, ties to the lower k.
 * Computed in FP32 as |c_k|^2 - 2 x_b . c_k.  dist (device FP32 x w h, may
 * be NULL) receives that squared distance.
 *
 * rt_kmeans_update: c_k = mean of the x_b with index[b] = k, summed in FP64.
 * A centroid with no member keeps its value.  scratch: device uint32,
 * w h + 3 K + 1 entries. */
/* rt_kmeans_assign on the tensor cores: the distance contraction x_b . c_k is
 * a dense FP16 GEMM (tcgen05.mma, FP32 accumulation in tensor memory, TMA
 * operand staging) and the argmin is taken in its epilogue.  The bucket
 * vectors and centroids are rounded to FP16 (exact for FP16 textures), |c_k|^2
 * and |x_b|^2 are summed in FP32 from those values, so a chosen centroid is a
 * nearest one up to about 2^-10 (|x|^2 + |c|^2).  scratch: device,
 * 1024-byte aligned, at least rt_kmeans_tc_scratch_bytes(w, h, n, K) bytes
 * (the FP16 operands and the norms).  Ties go to the lower k.  Asynchronous;
 * allocates nothing; RT_ERR_UNSUPPORTED when the driver lacks tensor-map
 * encoding; a stalled pipeline raises RT_ERR_TIMEOUT in rt_get_error. */
int64_t rt_kmeans_tc_scratch_bytes(int32_t w, int32_t h, int32_t n, int32_t K);
rt_status rt_kmeans_assign_tc(rt_ctx* ctx, int32_t obj_id, int32_t K, const float* centroids, uint32_t* index,
                              float* dist, void* scratch, int64_t scratch_bytes, rt_stream_t stream);

/* The number of polls (each followed by a 32 ns sleep) after which a bounded
 * wait of the library's kernels -- the mbarrier waits of the tensor-core
 * k-means assignment's pipeline -- gives up: the kernel then raises
 * RT_ERR_TIMEOUT (read by rt_get_error), lets the copies and MMAs it has
 * already issued finish (with the default limit), frees its tensor memory and
 * returns, and the context stays usable.  0 restores the default, 2^22 polls
 * (a fraction of a second).  A setting of the context; no counterpart in the
 * paper. */
rt_status rt_set_wait_limit(rt_ctx* ctx, uint32_t polls);

rt_status rt_kmeans_init(rt_ctx* ctx, int32_t obj_id, int32_t K, const int32_t* buckets, float* centroids,
                         rt_stream_t stream);
rt_status rt_kmeans_assign(rt_ctx* ctx, int32_t obj_id, int32_t K, const float* centroids, uint32_t* index,
                           float* dist, rt_stream_t stream);
rt_status rt_kmeans_update(rt_ctx* ctx, int32_t obj_id, int32_t K, const uint32_t* index, float* centroids,
                           uint32_t* scratch, rt_stream_t stream);

/* Baking (Section 2.2, Eq. 4a and Eq. 4b).  The scene that is ray traced into
 * a texture: a sphere, the ground plane y = plane_height and a sky.  The paper
 * names only the reflection vector; the shading below is this library's
 * (smooth everywhere but at the hit decisions):
 *   lit(N)     = ambient + (1 - ambient) max(0, N . sun_direction)
 *   sky(d)     = sky_horizon + (sky_zenith - sky_horizon)(1/2 + d_y/2)
 *                + sun_rgb max(0, d . sun_direction)^sun_exponent
 *   albedo     = sphere_albedo on the sphere; on the plane
 *                plane_albedo (3/4 + cos(f x) cos(f z) / 4), f = plane_frequency
 *   trace(P,d) = nearest hit at t > ray_offset of the sphere's entering root
 *                and the plane: (g C + (1 - g) sky(d), g) with g = exp(-fog t),
 *                C = albedo lit(normal at the hit); a miss gives (sky(d), 0).
 * All values are plain floats; the struct is read on the host during the call. */
typedef struct rt_bake_scene {
    float sphere_centre[3];
    float sphere_radius;      /* > 0 */
    float plane_height;       /* the plane y = plane_height */
    float plane_half_extent;  /* > 0: the plane's UV square is x, z in [-e, e] */
    float sphere_albedo[3];
    float sphere_reflectance;
    float plane_albedo[3];
    float plane_reflectance;
    float plane_frequency;
    float sun_direction[3];   /* unit, towards the sun */
    float sun_rgb[3];
    float sun_exponent;       /* >= 0 */
    float sky_zenith[3];
    float sky_horizon[3];
    float ambient;
    float fog;                /* >= 0 */
    float ray_offset;         /* >= 0: hits at t <= ray_offset are ignored */
} rt_bake_scene;

/* The surface that carries a baked texture, and its UV parametrisation.
 * SPHERE: lat-long, phi = 2 pi u - pi, theta = pi v (polar angle from +y),
 *   P = c + r (sin theta cos phi, cos theta, sin theta sin phi); tangent frame
 *   x = (-sin phi, 0, cos phi) (along dP/du), y = (cos theta cos phi,
 *   -sin theta, cos theta sin phi) (along dP/dv), z = outward normal.
 * PLANE: P = (2 e u - e, plane_height, 2 e v - e); frame (+x, +z, +y). */
typedef enum { RT_SURFACE_SPHERE = 0, RT_SURFACE_PLANE = 1 } rt_surface;

/* Bakes object obj_id from the scene (Section 2.2): for every texel (i, j, s, t)
 * the bucket centre (u, v) = ((i + 1/2)/w, (j + 1/2)/h) gives the surface point
 * P and frame; the texel centre B = ((2s+1)/n - 1, (2t+1)/n - 1) goes to A by
 * Eq. 4a and to the reflection vector R by Eq. 4b; d = R in world space; the
 * texel is (albedo(P) lit(N) + reflectance trace_rgb(P, d), trace_alpha(P, d)),
 * with the albedo and reflectance of `surface`.  Computed in FP32 and encoded
 * as rt_create_texture does (owned textures, any format), or written as FP32
 * into a borrowed buffer in its layout.  scene (host) is validated: finite
 * values, radius and extent > 0, fog, exponent and offset >= 0, else
 * RT_ERR_INVALID_ARG.  Asynchronous on `stream`; allocates nothing. */
rt_status rt_bake(rt_ctx* ctx, int32_t obj_id, rt_surface surface, const rt_bake_scene* scene, rt_stream_t stream);

/* Largest direction count of rt_bake_deferred. */
#define RT_MAX_AO_DIRECTIONS 1024

/* Bakes a deferred payload into object obj_id (Section 1: a texel may hold
 * data for deferred rendering, such as ambient occlusion or reflections,
 * instead of the final colour).  The ray of each texel is rt_bake's (Eq. 4a,
 * Eq. 4b); at its first hit X (the sphere's entering root or the plane, at
 * t > ray_offset) the texel holds (albedo(X) unlit, AO(X)), AO = the fraction
 * of the K directions for which the ray from X meets neither occluder at
 * t > ray_offset.  ao_dirs (device, K x 3 floats, row-major, 4-byte aligned,
 * caller-owned, read during the call only) are unit vectors in the local frame
 * of the hit: z along the normal facing the arriving ray (the sphere's outward
 * normal; +y or -y on the plane), x and y the orthonormal basis of Duff et al.,
 * "Building an Orthonormal Basis, Revisited" (JCGT 6(1), 2017) built from it;
 * cosine-distributed directions make AO the usual cosine-weighted estimate.
 * A ray that reaches the sky gives (0, 0, 0, 1).  1 <= K <=
 * RT_MAX_AO_DIRECTIONS; scene, format and layout rules and errors as rt_bake.
 * Asynchronous on `stream`; allocates nothing. */
rt_status rt_bake_deferred(rt_ctx* ctx, int32_t obj_id, rt_surface surface, const rt_bake_scene* scene,
                           const float* ao_dirs, int32_t K, rt_stream_t stream);

/* Forward synthesis of F >= 0 fragments (Section 2, Eq. 1b, Eq. 3, the Note's
 * clamp), filtered with `filter` in FP32: out (device, F x 4 float, RGBA).
 * Spatial addressing clamps to the edge; nearest indices take floor (an exact
 * boundary goes to the higher index). */
rt_status rt_shade(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int64_t F, rt_filter filter,
                   float* out, rt_stream_t stream);

/* The lookup coordinates of every fragment, for index checks: coord (device,
 * F x 4 float) = the continuous coordinates (c_u, c_v, c_s, c_t) whose floors
 * select the taps, idx (device, F x 4 int32) = those floors.  Spatial:
 * c = u w (nearest) or u w - 1/2 clamped to [-1, w] (bilinear).  In-bucket:
 * c = (B + 1) n / 2 (nearest) or (B + 1) n / 2 - 1/2 (bilinear), B clamped to
 * [1/n - 1, 1 - 1/n].  Background and invalid fragments give zeros. */
rt_status rt_locate(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int64_t F, rt_filter filter,
                    int32_t* idx, float* coord, rt_stream_t stream);

/* Gradients of a loss L given dL_dout (device, F x 4):
 *   dL_dtex: host array of n_dtex device pointers indexed by object id (the
 *            array itself may be NULL, and so may any entry): FP32 gradient of
 *            the object's decoded texel values, 4 channels per texel, in the
 *            object's storage layout (rt_texture_info: RT_LAYOUT_QUADS for
 *            owned textures, P n^2 texels with the padding left untouched; the
 *            borrowed buffer's layout otherwise; rt_convert_layout turns it
 *            into another).  Summed with vector atomics.
 *   dL_duv:  device F x 2 or NULL; dL_ddir: device F x 3 or NULL, through
 *            the filter weights, the Note's clamp, Eq. 3 and Eq. 1b.
 * Without RT_ACCUMULATE the per-fragment outputs are overwritten and each
 * dL_dtex buffer is zeroed first (a full write of the buffer); with it, all
 * outputs are added to.  With RT_ACCUMULATE_TEXELS alone the texel gradients
 * are added to (a caller that clears them itself, rt_zero_texture_grads) and
 * the per-fragment outputs are overwritten (not read).  With RT_DETERMINISTIC the texel gradients are summed
 * in fixed point (rt_prepare_deterministic, which must have been called after
 * the objects were created) and are bit-identical from run to run; the UV and
 * direction gradients are per fragment and always deterministic.  Subgradients: the floor branch at integer
 * coordinates, zero where a coordinate is clamped, the |A_x| >= |A_y| branch
 * of Eq. 3 on its diagonal, the identity at A = 0. */
rt_status rt_shade_backward(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int64_t F,
                            rt_filter filter, const float* dL_dout, float* const* dL_dtex, int32_t n_dtex,
                            float* dL_duv, float* dL_ddir, int32_t flags, rt_stream_t stream);

/* With RT_FIXED_POINT_GRADS (any backward or fused step), each non-NULL
 * dL_dtex[o] is a device buffer of 4 int64 per texel (the object's layout,
 * 16-byte aligned) that receives the texel gradients as the deterministic mode
 * sums them -- signed 64-bit fixed point with 32 fractional bits, each
 * contribution w * dL/dout rounded once to nearest -- without converting them
 * to FP32: zeroed first unless RT_ACCUMULATE is set.  Integer sums are
 * associative, so buffers filled from disjoint sets of fragments (views split
 * across calls, streams or processes) add up, in any order, to exactly the
 * buffer one call over all the fragments gives; rt_fixed_to_float converts
 * the total.  No rt_prepare_deterministic is needed.  Range |sum| < 2^31. */

/* FP32 values from fixed-point sums (RT_FIXED_POINT_GRADS): dst[k] =
 * (float)(acc[k] * 2^-32 * scale) (the product taken in FP64, rounded once),
 * for k < count; with RT_ACCUMULATE in flags added to dst[k] instead.  A loss
 * whose dL/dout carries a small constant factor (a mean over many fragments)
 * keeps its resolution when the sums are taken without it (a fused step with
 * scale 1) and the factor is applied here.  acc and dst device, 16-byte
 * aligned; scale finite. */
rt_status rt_fixed_to_float(const int64_t* acc, float* dst, int64_t count, double scale, int32_t flags,
                            rt_stream_t stream);

/* Zeroes texel-gradient buffers on `stream` (asynchronous, no allocation): for
 * every non-NULL entry o < n_dtex of dL_dtex (host array of device pointers
 * indexed by object id, as in rt_shade_backward), the object's full extent in
 * its storage layout, (P, w h or K) x n^2 texels of 4 FP32 values.  The clear that a step which
 * accumulates gradients (RT_ACCUMULATE) runs first; rt_shade_backward without
 * RT_ACCUMULATE does the same itself.  RT_ERR_INVALID_ARG for a dead object, a
 * buffer that is not 16-byte aligned or n_dtex outside [0, RT_MAX_OBJECTS]. */
rt_status rt_zero_texture_grads(rt_ctx* ctx, float* const* dL_dtex, int32_t n_dtex, rt_stream_t stream);

/* Prepares the deterministic backward mode (RT_DETERMINISTIC): allocates, for
 * every live object that has none yet, a buffer of 32 bytes per texel in which
 * rt_shade_backward sums texel gradients as signed 64-bit fixed-point numbers
 * with 32 fractional bits (each contribution w * dL/dout rounded once to
 * nearest; integer addition is associative, so the sums -- and the FP32
 * gradients converted from them -- do not depend on the order in which the
 * GPU schedules fragments).  Range |sum| < 2^31, resolution 2^-32.  A
 * synchronous set-up call; RT_ERR_OOM when the buffers do not fit. */
rt_status rt_prepare_deterministic(rt_ctx* ctx);

/* Shadow bake (Section 5, "Shadowing"): fills an owned RT_BIT1 texture with
 * the visibility of the sky from the bucket centre's surface point (the
 * parametrisations of rt_bake) towards every texel's direction:
 * B_k = (2k+1)/n - 1, A = Eq. 4a(B), L = Eq. 2c(A), rotated to world space.
 * The bit is 1 when the ray P + t L meets neither the sphere (entering root)
 * nor the plane at t > ray_offset.  At shading time the light direction, in
 * the tangent frame, takes the place of the view direction.  Asynchronous;
 * RT_ERR_UNSUPPORTED for textures that are not owned RT_BIT1. */
rt_status rt_bake_shadow(rt_ctx* ctx, int32_t obj_id, rt_surface surface, const rt_bake_scene* scene,
                         rt_stream_t stream);

/* Several lookups per fragment, averaged: out[f] = (1/S) sum_k lookup(uv[f],
 * dirs[f S + k]), with dirs F x S x 3 (16-byte aligned) and S = samples >= 1.
 * With a shadow texture and S light directions spread over an area light this
 * gives area (soft) shadows ("more than one sample per bucket", Section 5).
 * Flat fragment stream. */
rt_status rt_shade_multi(rt_ctx* ctx, const float* uv, const float* dirs, int32_t samples, const int32_t* obj,
                         int64_t F, rt_filter filter, float* out, rt_stream_t stream);

/* World-space variant (Eq. 1a).  The incidence I (dir, F x 3) and a
 * per-fragment normal N (nrm, F x 3, 16-byte aligned) are given in one frame,
 * with no tangent transform.  A is the first two entries of
 * sqrt(2) (I + N) / |I + N|.  With N = +z this is Eq. 1b, the tangent-space
 * form.  Eq. 3, the Note's clamp and the filter follow as in rt_shade.  A
 * non-finite normal raises RT_ERR_NONFINITE and gives a zero fragment.
 * rt_locate_world is rt_locate for this lookup.  rt_shade_world_backward is
 * rt_shade_backward for it: dL_dnrm (F x 3 or NULL) receives dL/dN, which
 * equals dL/dI.  These run on the flat fragment stream; rt_shade_world_batched
 * and rt_shade_world_batched_backward (below) walk screen tiles. */
rt_status rt_shade_world(rt_ctx* ctx, const float* uv, const float* dir, const float* nrm, const int32_t* obj,
                         int64_t F, rt_filter filter, float* out, rt_stream_t stream);
rt_status rt_locate_world(rt_ctx* ctx, const float* uv, const float* dir, const float* nrm, const int32_t* obj,
                          int64_t F, rt_filter filter, int32_t* idx, float* coord, rt_stream_t stream);
rt_status rt_shade_world_backward(rt_ctx* ctx, const float* uv, const float* dir, const float* nrm,
                                  const int32_t* obj, int64_t F, rt_filter filter, const float* dL_dout,
                                  float* const* dL_dtex, int32_t n_dtex, float* dL_duv, float* dL_ddir,
                                  float* dL_dnrm, int32_t flags, rt_stream_t stream);

/* Batched synthesis of views x height x width fragments: the same arrays as
 * rt_shade with F = views * height * width, fragment (view, y, x) at index
 * (view * height + y) * width + x (for instance every pose of a camera path,
 * row-major images).  The frame shape lets the kernel walk screen tiles: each
 * warp shades a tw x th tile, the warps of a block a compact block tile, so
 * fragments that read the same buckets run together (Section 2: neighbouring
 * fragments map to neighbouring buckets).  The tile shape is the context's
 * current one for `filter` (rt_set_tile / rt_autotune); every shape gives
 * bit-identical results.  0 <= height, width <= 65536. */
rt_status rt_shade_batched(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int32_t views,
                           int32_t height, int32_t width, rt_filter filter, float* out, rt_stream_t stream);

/* Gradients of the batched synthesis; arguments and semantics as in
 * rt_shade_backward, fragments laid out as in rt_shade_batched. */
rt_status rt_shade_batched_backward(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int32_t views,
                                    int32_t height, int32_t width, rt_filter filter, const float* dL_dout,
                                    float* const* dL_dtex, int32_t n_dtex, float* dL_duv, float* dL_ddir,
                                    int32_t flags, rt_stream_t stream);

/* One fused training step of the batched synthesis under an L2 loss: for every
 * fragment, the colour of rt_shade_batched (written to `out` when non-NULL),
 * dL/dout = scale (out - target) on fragments with obj >= 0 as rt_l2_loss_grad
 * forms it (the same FP32 roundings), sums (device, 2 doubles, 8-byte aligned,
 * may be NULL) accumulating the sum of |out - target|^2 and the count of those
 * fragments (the caller zeroes it), and the gradients of
 * rt_shade_batched_backward for that dL/dout (dL_dtex ... flags as there).
 * Equivalent to rt_shade_batched, rt_l2_loss_grad and
 * rt_shade_batched_backward in sequence (colours and UV / direction gradients
 * bit-identical, texel gradients up to the order of FP32 atomic additions,
 * sums up to the order of FP64 additions), in one pass: the G-buffer and target
 * are read once and each fragment's taps are gathered once.  target (device,
 * views x height x width x 4 floats, 16-byte aligned) is required when there
 * are fragments; scale finite.  Uses the backward's tile (rt_set_backward_tile,
 * rt_autotune_backward).  Asynchronous on `stream`. */
rt_status rt_shade_batched_l2_step(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int32_t views,
                                   int32_t height, int32_t width, rt_filter filter, const float* target, float scale,
                                   float* out, double* sums, float* const* dL_dtex, int32_t n_dtex, float* dL_duv,
                                   float* dL_ddir, int32_t flags, rt_stream_t stream);

/* The world-space lookup (Eq. 1a, rt_shade_world) over a batch of frames:
 * uv, dir, nrm (views x height x width x 2, 3, 3 floats) and obj laid out as
 * in rt_shade_batched, walked in screen tiles of the context's forward tile
 * for `filter` (the backward's tile for the gradients).  Results equal
 * rt_shade_world / rt_shade_world_backward on the same arrays: colours and
 * UV / direction / normal gradients bit for bit, texel gradients up to the
 * order of FP32 atomic additions.  Arguments, alignment, flags and errors as
 * there; 0 <= height, width <= 65536. */
rt_status rt_shade_world_batched(rt_ctx* ctx, const float* uv, const float* dir, const float* nrm,
                                 const int32_t* obj, int32_t views, int32_t height, int32_t width, rt_filter filter,
                                 float* out, rt_stream_t stream);
rt_status rt_shade_world_batched_backward(rt_ctx* ctx, const float* uv, const float* dir, const float* nrm,
                                          const int32_t* obj, int32_t views, int32_t height, int32_t width,
                                          rt_filter filter, const float* dL_dout, float* const* dL_dtex,
                                          int32_t n_dtex, float* dL_duv, float* dL_ddir, float* dL_dnrm,
                                          int32_t flags, rt_stream_t stream);

/* Sets the screen tile of the batched kernels for `filter`, forward and
 * backward: warp tiles of tw x th fragments (tw * th = 32, tw a multiple of 4)
 * arranged bx x by in a block tile (bx * by = 4).  The default is 8 x 4,
 * 2 x 2.  RT_ERR_INVALID_ARG for other shapes.  Not a device call. */
rt_status rt_set_tile(rt_ctx* ctx, rt_filter filter, int32_t tw, int32_t th, int32_t bx, int32_t by);

/* As rt_set_tile, for the backward (rt_shade_batched_backward) only. */
rt_status rt_set_backward_tile(rt_ctx* ctx, rt_filter filter, int32_t tw, int32_t th, int32_t bx, int32_t by);

/* The current forward tile of `filter`: tile4 = (tw, th, bx, by) (host, 4 ints). */
rt_status rt_get_tile(rt_ctx* ctx, rt_filter filter, int32_t* tile4);

/* The current backward tile of `filter`, as rt_get_tile. */
rt_status rt_get_backward_tile(rt_ctx* ctx, rt_filter filter, int32_t* tile4);

/* Autotuner: times rt_shade_batched with each of the twelve tile shapes
 * (tw, th) in {32x1, 16x2, 8x4, 4x8} x (bx, by) in {4x1, 2x2, 1x4}, `reps`
 * launches each after one warm-up, on the caller's representative inputs
 * (writing `out`), keeps the fastest for `filter` in the context and returns
 * it in tile4 (host, 4 ints, may be NULL) with its mean launch time in best_ms
 * (host, may be NULL).  Synchronises the stream; not capturable. */
rt_status rt_autotune(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int32_t views,
                      int32_t height, int32_t width, rt_filter filter, float* out, int32_t reps, rt_stream_t stream,
                      int32_t* tile4, float* best_ms);

/* The autotuner of the backward: times rt_shade_batched_backward with the same
 * twelve tiles and keeps the fastest as the backward tile of `filter`
 * (rt_shade_batched's tile is left alone).  The arguments from dL_dout to
 * flags are those of rt_shade_batched_backward, and the gradient buffers end
 * up holding the results of the timed launches (with RT_ACCUMULATE, their
 * sum), so a caller clears them before real use.  tile4, best_ms, reps and
 * the synchronisation as in rt_autotune. */
rt_status rt_autotune_backward(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int32_t views,
                               int32_t height, int32_t width, rt_filter filter, const float* dL_dout,
                               float* const* dL_dtex, int32_t n_dtex, float* dL_duv, float* dL_ddir, int32_t flags,
                               int32_t reps, rt_stream_t stream, int32_t* tile4, float* best_ms);

/* Counts the distinct texels read by the F fragments (any tap of non-zero or
 * zero weight of the filter's footprint), per object: counts_host (host,
 * n_counts entries indexed by object id).  A measurement utility: it allocates
 * a bitmap of one bit per texel of every object and synchronises the stream. */
rt_status rt_footprint(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int64_t F,
                       rt_filter filter, uint64_t* counts_host, int32_t n_counts, rt_stream_t stream);

/* Largest texel count, summed over a context's objects, that
 * rt_footprint_noalloc accepts (its bitmap holds one bit per texel: 8 MiB). */
#define RT_FOOTPRINT_NOALLOC_MAX_TEXELS (1ll << 26)

/* rt_footprint without any device allocation.  The paper has no counterpart:
 * this is a service of the library.  It is meant for callers that must not
 * allocate device memory themselves: an application or framework that owns all
 * device memory through its own allocator or budget, or a per-frame loop in
 * which cudaMalloc / cudaFree would synchronise the device.  The scratch bitmap
 * (and a table of per-object offsets) lives in file-scope device arrays that
 * every GPU loading the library keeps until the process exits; the contexts'
 * objects may hold at most RT_FOOTPRINT_NOALLOC_MAX_TEXELS texels in total
 * (RT_ERR_INVALID_ARG otherwise).  counts_dev (device, n_counts uint64 entries,
 * 8-byte aligned, indexed by object id; any n_counts >= 0, entries past the
 * last object are set to zero) receives the distinct-texel counts,
 * asynchronously on `stream`; nothing is read back to the host, and the
 * per-object offsets are computed on the device from the context's own
 * descriptor table (no host-to-device copy).  The G-buffer rules are
 * rt_footprint's.  The first call on a device (and again after the device's
 * context is reset) looks the arrays' device addresses up on the host.  All
 * calls share the arrays, and each clears what it uses first, so calls whose
 * work overlaps on the GPU (other streams, other threads) race and must be
 * ordered by the caller. */
rt_status rt_footprint_noalloc(rt_ctx* ctx, const float* uv, const float* dir, const int32_t* obj, int64_t F,
                               rt_filter filter, uint64_t* counts_dev, int32_t n_counts, rt_stream_t stream);

/* Texture fitting (no counterpart in the paper, which fills textures by ray
 * tracing, Eq. 4b; here a texture is fitted to target renders by gradient
 * descent).  L2 loss of F output colours against targets: dL_dout (device,
 * F x 4, may be NULL) = scale (out - target) on fragments with obj >= 0 and 0
 * on background; sums (device, 2 doubles, may be NULL) accumulates the sum of
 * |out - target|^2 over shaded fragments and their count (the caller zeroes
 * it).  out, target, dL_dout 16-byte aligned. */
rt_status rt_l2_loss_grad(const float* out, const float* target, const int32_t* obj, int64_t F, float scale,
                          float* dL_dout, double* sums, rt_stream_t stream);

/* One Adam step (bias-corrected; step >= 1 is the 1-based step number) on
 * `count` FP32 values (a multiple of 4): m = b1 m + (1 - b1) g,
 * v = b2 v + (1 - b2) g^2, param -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * All four arrays device, 16-byte aligned. */
rt_status rt_adam_step(float* param, const float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                       float beta2, float eps, int32_t step, rt_stream_t stream);


/* Converts an FP32 4-channel texture buffer of w x h buckets of n x n texels
 * between layouts (device src and dst, which must not overlap; the padding of
 * a QUADS dst is not written): for instance a texel-gradient buffer of an
 * owned texture into the atlas. */
rt_status rt_convert_layout(const float* src, rt_layout src_layout, float* dst, rt_layout dst_layout, int32_t w,
                            int32_t h, int32_t n, rt_stream_t stream);

/* Synchronises `stream`, then reads and clears the context's sticky status
 * word: *device_status = RT_OK, or the first of RT_ERR_OUT_OF_BOUNDS,
 * RT_ERR_BAD_OBJ_ID, RT_ERR_NONFINITE, RT_ERR_TIMEOUT, RT_ERR_INVALID_ARG raised
 * since the last call. */
rt_status rt_get_error(rt_ctx* ctx, rt_stream_t stream, rt_status* device_status);

/* The checked build (libradtex_checked.so, compiled with RADTEX_CHECKED; no
 * counterpart in the paper).  Every texel index the lookups and the texel-
 * gradient reductions compute (Section 2's bucket and in-bucket texels), every
 * bucket of the w x h matrix and every stored bucket a palette's index map
 * names is checked against its object's extent on the device.  A failed check
 * sets a sticky bit that rt_get_error reports as RT_ERR_OUT_OF_BOUNDS, and the
 * access goes to texel 0 (bucket 0) of the same object instead: it stays
 * inside the object's storage and nothing traps.  The outputs of a call that
 * raised it are not meaningful.
 *
 * rt_checked_limit_extent lowers the extent that those checks allow for object
 * obj_id to `texels` (0 <= texels <= the object's stored texel count, P n^2 in
 * quads; larger values, a bad id or a dead object give RT_ERR_INVALID_ARG)
 * without touching the storage, so that in-bounds accesses past it raise the
 * error; it exists to test the checks.  Synchronous.  The normal build returns
 * RT_ERR_UNSUPPORTED and checks nothing. */
rt_status rt_checked_limit_extent(rt_ctx* ctx, int32_t obj_id, int64_t texels);

/* A static English description of a status code. */
const char* rt_status_string(rt_status status);

#ifdef __cplusplus
}
#endif

#endif /* RADTEX_H */

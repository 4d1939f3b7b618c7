/*
 * radtex_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision CPU oracle for per-fragment radiance-texture
 * synthesis, written from J. M. Fober, "Radiance Textures for Rasterizing
 * Ray-Traced Data" (arXiv 2301.01719).  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg load this library.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * What it computes, per fragment (Section 2, "Methodology"):
 *   - the surface UV selects a bucket of the w x h bucket matrix;
 *   - the tangent-space incidence I is projected with the equisolid mapping
 *     (Eq. 1b), made square with the disc-to-square mapping (Eq. 3) and
 *     clamped to the texel-centre range of the Note after Eq. 3;
 *   - the selected texels are filtered: NEAREST, ANGULAR_BILINEAR (one bucket,
 *     bilinear inside it: "single sample per bucket"), or QUADRILINEAR
 *     (separable tent filter over u, v and the two in-bucket axes).
 * The colour is the plain weighted sum over the taps, sum(w_u w_v w_s w_t T),
 * evaluated in FP64 on texels decoded exactly from their stored codes.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *   R1  I points from the surface to the eye, in the tangent frame (x along
 *       dP/du, y along dP/dv, z = N).  Eq. 1b is applied literally, without
 *       renormalising I; I = -N (zero denominator) maps to A = 0.
 *   R2  Eq. 3 is singular only at A = 0, which maps to B = 0 (the limit); the
 *       printed condition "A_x and A_y != 0" is read as "A != 0".
 *   R3  Texel k of an n-texel bucket axis has its centre at B = (2k+1)/n - 1;
 *       the clamp range [1/n - 1, 1 - 1/n] of the Note is then exactly the
 *       first and last centre.  B_x selects the column s, B_y the row t;
 *       u selects the bucket column i, v the bucket row j, no flip.
 *   R4  Atlas layout: row-major (h n) x (w n) texels of 4 channels (RGBA),
 *       texel (i, j, s, t) at row j n + t, column i n + s (Section 1.3
 *       naming convention, Section 2 first paragraph).
 *   R5  Spatial filtering: nearest bucket i = clamp(floor(u w), 0, w-1); the
 *       bilinear coordinate is c = u w - 1/2 clamped to [-1, w], taps
 *       clamp(floor(c)) and clamp(floor(c)+1) (clamp to edge).  Angular axes
 *       use c = (B+1) n/2 (nearest) or (B+1) n/2 - 1/2 (bilinear) with the
 *       same floor-and-clamp rule.  An exact boundary goes to the higher
 *       index (floor).
 *   R6  Gradients: at an integer coordinate the floor branch is taken; a
 *       clamped coordinate has zero derivative; at |A_x| = |A_y| Eq. 3 uses
 *       the x branch; at A = 0 the Jacobian of Eq. 3 is the identity.
 *   R7  Storage formats: FP32, FP16 and BF16 round to nearest-even from FP32;
 *       FP8 E4M3 (OCP 8-bit floating point, max finite 448, no infinities)
 *       rounds to nearest-even with saturation, on v / s where s is one FP32
 *       scale per bucket, s = amax / 448 (s = 1 if amax = 0).  The quantising
 *       decision is taken in FP32, like the device encoder.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fopenmp -shared -fPIC.
 * FP contraction stays off so the results do not depend on the host ISA.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_F32 0
#define OR_F16 1
#define OR_BF16 2
#define OR_E4M3 3
#define OR_F64 4  /* oracle-only exact format, used by the pins */
#define OR_BIT1 5 /* 1-bit payload (reading R13): code 0 or 1, the texel value in every channel */
/* Oracle-only procedural texels, for textures too large to hold as an atlas in
 * host memory: `codes` points at 13 int64 parameters a[4], b[4], k[4], m, and
 * channel c of atlas texel (X, Y) is the triangle wave
 * |((a_c X + b_c Y + k_c) mod 2m) - m| / m  (a value j / m, 0 <= j <= m). */
#define OR_PATTERN 6

#define OR_NEAREST 0
#define OR_ANGULAR_BILINEAR 1
#define OR_QUADRILINEAR 2

#define OR_FLAG_BAD_OBJ 1u
#define OR_FLAG_NONFINITE 2u

static const double SQRT2 = 1.41421356237309504880168872420969808;

/* ------------------------------------------------------------------------ */
/* Section 2.1: the incidence-to-bucket mapping and its inverses.           */
/* ------------------------------------------------------------------------ */

/* Eq. 1b: tangent-space equisolid projection (N_z = 1),
 * A = sqrt(2) (I_x, I_y) / |(I_x, I_y, I_z + 1)|. */
static void equisolid_ts(const double I[3], double A[2]) {
    double zp = I[2] + 1.0;
    double D = sqrt(I[0] * I[0] + I[1] * I[1] + zp * zp);
    if (D == 0.0) {
        A[0] = 0.0;
        A[1] = 0.0;
        return;
    }
    A[0] = SQRT2 * I[0] / D;
    A[1] = SQRT2 * I[1] / D;
}

/* Eq. 1a: general normal.  The vector sqrt(2) * (I + N) / |I + N| whose first
 * two entries are A (in a frame where N is the z axis) and whose last entry is
 * sqrt(2) cos(theta/2).  The double bar of the equation is read as "normalise". */
static void equisolid_normal(const double I[3], const double N[3], double A3[3]) {
    double h[3] = {I[0] + N[0], I[1] + N[1], I[2] + N[2]};
    double L = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    if (L == 0.0) {
        A3[0] = A3[1] = A3[2] = 0.0;
        return;
    }
    for (int k = 0; k < 3; ++k) A3[k] = SQRT2 * h[k] / L;
}

/* Eq. 3: disc to square, B = A |A| / max(|A_x|, |A_y|); A = 0 gives B = 0. */
static void squarify(const double A[2], double B[2]) {
    double m = fmax(fabs(A[0]), fabs(A[1]));
    if (m == 0.0) {
        B[0] = 0.0;
        B[1] = 0.0;
        return;
    }
    double r = sqrt(A[0] * A[0] + A[1] * A[1]);
    B[0] = A[0] * r / m;
    B[1] = A[1] * r / m;
}

/* Eq. 4a: square to disc, A = B max(|B_x|, |B_y|) / |B|; B = 0 gives A = 0. */
static void unsquarify(const double B[2], double A[2]) {
    double r = sqrt(B[0] * B[0] + B[1] * B[1]);
    if (r == 0.0) {
        A[0] = 0.0;
        A[1] = 0.0;
        return;
    }
    double m = fmax(fabs(B[0]), fabs(B[1]));
    A[0] = B[0] * m / r;
    A[1] = B[1] * m / r;
}

/* Eq. 2c: tangent-space inverse equisolid mapping,
 * I = (A_x sqrt(2 - |A|^2), A_y sqrt(2 - |A|^2), 1 - |A|^2). */
static void equisolid_inverse_ts(const double A[2], double I[3]) {
    double a2 = A[0] * A[0] + A[1] * A[1];
    double s = sqrt(2.0 - a2);
    I[0] = A[0] * s;
    I[1] = A[1] * s;
    I[2] = 1.0 - a2;
}

/* Eq. 2a then Eq. 2b: the half vector A' = (A_x / sqrt 2, A_y / sqrt 2,
 * sqrt(1 - |A|^2 / 2)), then I = 2((A' . N) A' - N) + N. */
static void equisolid_inverse_normal(const double A[2], const double N[3], double I[3]) {
    double Ap[3];
    Ap[0] = A[0] * sqrt(0.5);
    Ap[1] = A[1] * sqrt(0.5);
    Ap[2] = sqrt(1.0 - A[0] * A[0] / 2.0 - A[1] * A[1] / 2.0);
    double d = Ap[0] * N[0] + Ap[1] * N[1] + Ap[2] * N[2];
    for (int k = 0; k < 3; ++k) I[k] = 2.0 * (d * Ap[k] - N[k]) + N[k];
}

/* Eq. 4b: equisolid reflection vector,
 * R = (-A_x sqrt(2 - |A|^2), -A_y sqrt(2 - |A|^2), 1 - |A|^2). */
static void reflection(const double A[2], double R[3]) {
    double a2 = A[0] * A[0] + A[1] * A[1];
    double s = sqrt(2.0 - a2);
    R[0] = -A[0] * s;
    R[1] = -A[1] * s;
    R[2] = 1.0 - a2;
}

/* Reading R3: centre of texel k on an n-texel bucket axis, in B units. */
static double texel_centre(int64_t k, int64_t n) { return (2.0 * (double)k + 1.0) / (double)n - 1.0; }

/* Direction of the texel centre (s, t): Eq. 4a then Eq. 2c. */
static void texel_direction(int64_t s, int64_t t, int64_t n, double I[3]) {
    double B[2] = {texel_centre(s, n), texel_centre(t, n)};
    double A[2];
    unsquarify(B, A);
    equisolid_inverse_ts(A, I);
}

/* Batched entry points of the mapping functions (rows of 2 or 3 doubles). */
void oracle_equisolid(int64_t count, const double* I, double* A) {
    for (int64_t k = 0; k < count; ++k) equisolid_ts(I + 3 * k, A + 2 * k);
}
void oracle_equisolid_normal(int64_t count, const double* I, const double* N, double* A3) {
    for (int64_t k = 0; k < count; ++k) equisolid_normal(I + 3 * k, N + 3 * k, A3 + 3 * k);
}
void oracle_squarify(int64_t count, const double* A, double* B) {
    for (int64_t k = 0; k < count; ++k) squarify(A + 2 * k, B + 2 * k);
}
void oracle_unsquarify(int64_t count, const double* B, double* A) {
    for (int64_t k = 0; k < count; ++k) unsquarify(B + 2 * k, A + 2 * k);
}
void oracle_equisolid_inverse(int64_t count, const double* A, double* I) {
    for (int64_t k = 0; k < count; ++k) equisolid_inverse_ts(A + 2 * k, I + 3 * k);
}
void oracle_equisolid_inverse_normal(int64_t count, const double* A, const double* N, double* I) {
    for (int64_t k = 0; k < count; ++k) equisolid_inverse_normal(A + 2 * k, N + 3 * k, I + 3 * k);
}
void oracle_reflection(int64_t count, const double* A, double* R) {
    for (int64_t k = 0; k < count; ++k) reflection(A + 2 * k, R + 3 * k);
}
/* Directions of all n x n texel centres of a bucket, row t major: dirs[(t n + s) 3 + c]. */
void oracle_texel_directions(int32_t n, double* dirs) {
    for (int64_t t = 0; t < n; ++t)
        for (int64_t s = 0; s < n; ++s) texel_direction(s, t, n, dirs + 3 * (t * n + s));
}

/* ------------------------------------------------------------------------ */
/* Storage formats (reading R7), written from the format definitions.       */
/* ------------------------------------------------------------------------ */

/* A binary floating-point format with `mbits` stored mantissa bits, minimum
 * normal exponent `emin`, exponent bias `bias`, and largest finite value
 * `maxf`.  Rounds |x| to nearest, ties to even; overflow gives +-infinity
 * (FP16, BF16) or saturates to maxf (E4M3 "satfinite"). */
typedef struct {
    int mbits, emin, bias, ebits;
    double maxf;
    int saturate;
} fmt_t;

static const fmt_t FMT_F16 = {10, -14, 15, 5, 65504.0, 0};
static const fmt_t FMT_BF16 = {7, -126, 127, 8, 3.38953138925153547590470800371487867e38, 0};
static const fmt_t FMT_E4M3 = {3, -6, 7, 4, 448.0, 1};

/* Round a finite non-negative double to the format's value set. */
static double round_to_format(double a, const fmt_t* f) {
    if (a == 0.0) return 0.0;
    int e;
    (void)frexp(a, &e); /* a = m 2^e, m in [0.5, 1): floor(log2 a) = e - 1 */
    int ex = e - 1;
    if (ex < f->emin) ex = f->emin; /* subnormal quantum */
    double quantum = ldexp(1.0, ex - f->mbits);
    double q = rint(a / quantum) * quantum; /* exact scaling; rint = ties to even */
    if (q > f->maxf) {
        if (f->saturate) return f->maxf;
        /* IEEE overflow threshold: values that round above maxf become inf. */
        return INFINITY;
    }
    return q;
}

/* Pack a value of the format's value set (or +-inf / NaN) into its code. */
static uint32_t pack_format(double v, int negative, const fmt_t* f) {
    uint32_t sign = negative ? (1u << (f->ebits + f->mbits)) : 0u;
    uint32_t emask = (1u << f->ebits) - 1u;
    if (isnan(v)) return sign | (emask << f->mbits) | ((1u << f->mbits) - 1u);
    if (isinf(v)) return sign | (emask << f->mbits);
    if (v == 0.0) return sign;
    int e;
    (void)frexp(v, &e);
    int ex = e - 1;
    if (ex < f->emin) { /* subnormal: exponent field 0, mantissa v / 2^(emin - mbits) */
        uint32_t mant = (uint32_t)ldexp(v, f->mbits - f->emin);
        return sign | mant;
    }
    uint32_t mant = (uint32_t)ldexp(ldexp(v, -ex) - 1.0, f->mbits);
    uint32_t field = (uint32_t)(ex + f->bias);
    return sign | (field << f->mbits) | mant;
}

static double unpack_format(uint32_t code, const fmt_t* f, int has_inf) {
    uint32_t mmask = (1u << f->mbits) - 1u;
    uint32_t emask = (1u << f->ebits) - 1u;
    int negative = (code >> (f->ebits + f->mbits)) & 1u;
    uint32_t field = (code >> f->mbits) & emask;
    uint32_t mant = code & mmask;
    double v;
    if (field == emask && has_inf) {
        v = mant ? NAN : INFINITY;
    } else if (field == emask && !has_inf && mant == mmask) {
        v = NAN; /* E4M3: S.1111.111 is the only NaN */
    } else if (field == 0) {
        v = ldexp((double)mant, f->emin - f->mbits);
    } else {
        v = ldexp(1.0 + ldexp((double)mant, -f->mbits), (int)field - f->bias);
    }
    return negative ? -v : v;
}

static uint32_t encode_float(float x, const fmt_t* f) {
    double a = fabs((double)x);
    int neg = signbit(x) ? 1 : 0;
    if (isnan(x)) return pack_format(NAN, neg, f);
    if (isinf(x)) return f->saturate ? pack_format(f->maxf, neg, f) : pack_format(INFINITY, neg, f);
    return pack_format(round_to_format(a, f), neg, f);
}

static double decode_f16(uint16_t c) { return unpack_format(c, &FMT_F16, 1); }
static double decode_bf16(uint16_t c) { return unpack_format(c, &FMT_BF16, 1); }
static double decode_e4m3(uint8_t c) { return unpack_format(c, &FMT_E4M3, 0); }

/* Encode `count` FP32 values to F32 (copy), F16 or BF16 codes. */
void oracle_encode(int32_t fmt, int64_t count, const float* x, void* codes) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k) {
        if (fmt == OR_F32)
            ((float*)codes)[k] = x[k];
        else if (fmt == OR_F16)
            ((uint16_t*)codes)[k] = (uint16_t)encode_float(x[k], &FMT_F16);
        else if (fmt == OR_BF16)
            ((uint16_t*)codes)[k] = (uint16_t)encode_float(x[k], &FMT_BF16);
        else if (fmt == OR_E4M3)
            ((uint8_t*)codes)[k] = (uint8_t)encode_float(x[k], &FMT_E4M3);
    }
}

/* Decode `count` codes of a format to FP64, exactly. */
void oracle_decode(int32_t fmt, int64_t count, const void* codes, double* out) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k) {
        if (fmt == OR_F32)
            out[k] = (double)((const float*)codes)[k];
        else if (fmt == OR_F16)
            out[k] = decode_f16(((const uint16_t*)codes)[k]);
        else if (fmt == OR_BF16)
            out[k] = decode_bf16(((const uint16_t*)codes)[k]);
        else if (fmt == OR_E4M3)
            out[k] = decode_e4m3(((const uint8_t*)codes)[k]);
        else
            out[k] = ((const double*)codes)[k];
    }
}

/* E4M3 with one FP32 scale per bucket (reading R7).  `atlas` is the FP32
 * atlas of reading R4; codes have the same layout, scales are row-major w x h. */
void oracle_encode_e4m3_buckets(int32_t W, int32_t H, int32_t n, const float* atlas, uint8_t* codes,
                                float* scales) {
    int64_t row = (int64_t)W * n * 4;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < (int64_t)W * H; ++b) {
        int64_t i = b % W, j = b / W;
        float amax = 0.0f;
        for (int64_t t = 0; t < n; ++t)
            for (int64_t s = 0; s < n; ++s)
                for (int c = 0; c < 4; ++c) {
                    float v = fabsf(atlas[(j * n + t) * row + (i * n + s) * 4 + c]);
                    if (v > amax) amax = v;
                }
        float sc = (amax == 0.0f) ? 1.0f : amax / 448.0f;
        scales[b] = sc;
        for (int64_t t = 0; t < n; ++t)
            for (int64_t s = 0; s < n; ++s)
                for (int c = 0; c < 4; ++c) {
                    int64_t e = (j * n + t) * row + (i * n + s) * 4 + c;
                    float q = atlas[e] / sc; /* the decision is taken in FP32 */
                    codes[e] = (uint8_t)encode_float(q, &FMT_E4M3);
                }
    }
}

/* ------------------------------------------------------------------------ */
/* Texture access (readings R4 and R7).                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t W, H, n;
    int32_t fmt;
    int32_t wrap; /* reading R12: bit 0 repeats u, bit 1 repeats v (else clamp to edge) */
    const void* codes;
    const float* scale;
} tex_t;

static int64_t atlas_offset(const tex_t* T, int64_t i, int64_t j, int64_t s, int64_t t, int c) {
    int64_t X = i * T->n + s, Y = j * T->n + t;
    return (Y * T->W * T->n + X) * 4 + c;
}

/* The stored texel (i, j, s, t), channel c, decoded exactly to FP64. */
static double texel(const tex_t* T, int64_t i, int64_t j, int64_t s, int64_t t, int c) {
    int64_t e = atlas_offset(T, i, j, s, t, c);
    switch (T->fmt) {
        case OR_F32:
            return (double)((const float*)T->codes)[e];
        case OR_F16:
            return decode_f16(((const uint16_t*)T->codes)[e]);
        case OR_BF16:
            return decode_bf16(((const uint16_t*)T->codes)[e]);
        case OR_E4M3:
            return decode_e4m3(((const uint8_t*)T->codes)[e]) * (double)T->scale[j * T->W + i];
        case OR_BIT1:
            return (double)(((const uint8_t*)T->codes)[e] & 1u);
        case OR_PATTERN: {
            const int64_t* p = (const int64_t*)T->codes;
            const int64_t X = i * T->n + s, Y = j * T->n + t, m = p[12];
            const int64_t q = (p[c] * X + p[4 + c] * Y + p[8 + c]) % (2 * m);
            return (double)llabs(q - m) / (double)m;
        }
        default:
            return ((const double*)T->codes)[e];
    }
}

/* ------------------------------------------------------------------------ */
/* Per-fragment lookup: Eq. 1b, Eq. 3, the Note's clamp, the filter.        */
/* ------------------------------------------------------------------------ */

/* One filter axis: two taps (equal for a nearest axis), their weights, the
 * continuous coordinate c, its floor, and dc/d(input) for the gradient. */
typedef struct {
    int64_t tap[2];
    double w[2];
    double c;
    int64_t fl;
    double dc; /* derivative of c with respect to the axis input (u, v, B_x or B_y) */
} axis_t;

static int64_t clampi(int64_t x, int64_t lo, int64_t hi) { return x < lo ? lo : (x > hi ? hi : x); }

static int64_t wrapi(int64_t x, int64_t size) {
    int64_t r = x % size;
    return r < 0 ? r + size : r;
}

/* Spatial axis (reading R5, and R12 for the repeat address mode); size = w or
 * h, x = u or v.  Repeat: c = x size (- 1/2 when bilinear) is not clamped;
 * the taps are its floor (and floor + 1) modulo size. */
static void spatial_axis(double x, int64_t size, int bilinear, int wrap, axis_t* a) {
    if (wrap) {
        double c = x * (double)size - (bilinear ? 0.5 : 0.0);
        double f = floor(c);
        a->c = c;
        a->fl = (int64_t)f;
        a->tap[0] = wrapi(a->fl, size);
        a->tap[1] = bilinear ? wrapi(a->fl + 1, size) : a->tap[0];
        a->w[1] = bilinear ? c - f : 0.0;
        a->w[0] = 1.0 - a->w[1];
        a->dc = bilinear ? (double)size : 0.0;
        return;
    }
    if (bilinear) {
        double c = x * (double)size - 0.5;
        a->dc = (c > -1.0 && c < (double)size) ? (double)size : 0.0;
        if (c < -1.0) c = -1.0;
        if (c > (double)size) c = (double)size;
        double f = floor(c);
        a->c = c;
        a->fl = (int64_t)f;
        a->tap[0] = clampi(a->fl, 0, size - 1);
        a->tap[1] = clampi(a->fl + 1, 0, size - 1);
        a->w[1] = c - f;
        a->w[0] = 1.0 - a->w[1];
    } else {
        double c = x * (double)size;
        if (c < 0.0) c = 0.0;
        if (c > (double)size) c = (double)size;
        a->c = c;
        a->fl = (int64_t)floor(c);
        a->tap[0] = a->tap[1] = clampi(a->fl, 0, size - 1);
        a->w[0] = 1.0;
        a->w[1] = 0.0;
        a->dc = 0.0;
    }
}

/* In-bucket axis (Note after Eq. 3, readings R3 and R5); B is one component of Eq. 3's output. */
static void angular_axis(double B, int64_t n, int bilinear, axis_t* a) {
    double lo = 1.0 / (double)n - 1.0, hi = 1.0 - 1.0 / (double)n;
    double inside = (B > lo && B < hi) ? 1.0 : 0.0;
    double Bc = B < lo ? lo : (B > hi ? hi : B);
    if (bilinear) {
        double c = (Bc + 1.0) * (double)n / 2.0 - 0.5;
        double f = floor(c);
        a->c = c;
        a->fl = (int64_t)f;
        a->tap[0] = clampi(a->fl, 0, n - 1);
        a->tap[1] = clampi(a->fl + 1, 0, n - 1);
        a->w[1] = c - f;
        a->w[0] = 1.0 - a->w[1];
        a->dc = inside * (double)n / 2.0;
    } else {
        double c = (Bc + 1.0) * (double)n / 2.0;
        a->c = c;
        a->fl = (int64_t)floor(c);
        a->tap[0] = a->tap[1] = clampi(a->fl, 0, n - 1);
        a->w[0] = 1.0;
        a->w[1] = 0.0;
        a->dc = 0.0;
    }
}

typedef struct {
    axis_t u, v, s, t;
    double A[2], B[2];
} lookup_t;

/* N == NULL: I is in the tangent frame, Eq. 1b.  Otherwise I and N are in one
 * (world) frame and A is the first two entries of Eq. 1a. */
static void locate_one(const tex_t* T, double u, double v, const double I[3], const double* N, int filter,
                       lookup_t* L) {
    int spatial_bilinear = (filter == OR_QUADRILINEAR);
    int angular_bilinear = (filter != OR_NEAREST);
    spatial_axis(u, T->W, spatial_bilinear, T->wrap & 1, &L->u);
    spatial_axis(v, T->H, spatial_bilinear, (T->wrap >> 1) & 1, &L->v);
    if (N) {
        double A3[3];
        equisolid_normal(I, N, A3); /* Eq. 1a */
        L->A[0] = A3[0];
        L->A[1] = A3[1];
    } else {
        equisolid_ts(I, L->A); /* Eq. 1b */
    }
    squarify(L->A, L->B);   /* Eq. 3 */
    angular_axis(L->B[0], T->n, angular_bilinear, &L->s);
    angular_axis(L->B[1], T->n, angular_bilinear, &L->t);
}

/* Colour of one fragment: the plain sum over the 16 (u, v, s, t) taps. */
static void colour_one(const tex_t* T, const lookup_t* L, double out[4]) {
    for (int c = 0; c < 4; ++c) {
        double acc = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q) {
                        double w = L->u.w[a] * L->v.w[b] * L->s.w[p] * L->t.w[q];
                        if (w == 0.0) continue; /* zero-weight tap: no texel read */
                        acc += w * texel(T, L->u.tap[a], L->v.tap[b], L->s.tap[p], L->t.tap[q], c);
                    }
        out[c] = acc;
    }
}

static void make_tex(const int32_t* dims, const void* const* codes, const float* const* scales, int32_t o,
                     tex_t* T) {
    T->W = dims[4 * o + 0];
    T->H = dims[4 * o + 1];
    T->n = dims[4 * o + 2];
    T->fmt = dims[4 * o + 3] & 0xff;
    T->wrap = (dims[4 * o + 3] >> 8) & 3;
    T->codes = codes[o];
    T->scale = scales ? scales[o] : NULL;
}

/* Validity of a fragment: 0 = background, 1 = shade, otherwise an error flag. */
static uint32_t classify(int32_t o, int32_t n_obj, const void* const* codes, double u, double v,
                         const double I[3], const double* N, int* shade) {
    *shade = 0;
    if (o < 0) return 0;
    if (o >= n_obj || codes[o] == NULL) return OR_FLAG_BAD_OBJ;
    if (!isfinite(u) || !isfinite(v) || !isfinite(I[0]) || !isfinite(I[1]) || !isfinite(I[2]))
        return OR_FLAG_NONFINITE;
    if (N && (!isfinite(N[0]) || !isfinite(N[1]) || !isfinite(N[2]))) return OR_FLAG_NONFINITE;
    *shade = 1;
    return 0;
}

/* Continuous coordinates and floors of every fragment (for index parity).
 * coord[4f..4f+3] = (c_u, c_v, c_s, c_t), idx likewise (floors); background
 * and invalid fragments get zeros. */
static uint32_t locate_core(const int32_t* dims, const void* const* codes, int32_t n_obj, int64_t F,
                            const float* uv, const float* dir, const float* nrm, const int32_t* obj, int32_t filter,
                            int32_t* idx, double* coord) {
    uint32_t flags = 0;
#pragma omp parallel for schedule(static) reduction(| : flags)
    for (int64_t f = 0; f < F; ++f) {
        double u = uv[2 * f], v = uv[2 * f + 1];
        double I[3] = {dir[3 * f], dir[3 * f + 1], dir[3 * f + 2]};
        double Nw[3] = {0.0, 0.0, 0.0};
        if (nrm)
            for (int k = 0; k < 3; ++k) Nw[k] = nrm[3 * f + k];
        const double* N = nrm ? Nw : NULL;
        int shade;
        flags |= classify(obj[f], n_obj, codes, u, v, I, N, &shade);
        for (int k = 0; k < 4; ++k) {
            idx[4 * f + k] = 0;
            coord[4 * f + k] = 0.0;
        }
        if (!shade) continue;
        tex_t T;
        make_tex(dims, codes, NULL, obj[f], &T);
        lookup_t L;
        locate_one(&T, u, v, I, N, filter, &L);
        const axis_t* ax[4] = {&L.u, &L.v, &L.s, &L.t};
        for (int k = 0; k < 4; ++k) {
            idx[4 * f + k] = (int32_t)ax[k]->fl;
            coord[4 * f + k] = ax[k]->c;
        }
    }
    return flags;
}

uint32_t oracle_locate(const int32_t* dims, const void* const* codes, int32_t n_obj, int64_t F, const float* uv,
                       const float* dir, const int32_t* obj, int32_t filter, int32_t* idx, double* coord) {
    return locate_core(dims, codes, n_obj, F, uv, dir, NULL, obj, filter, idx, coord);
}

/* The taps of every fragment and their weights, as the colour sums them: 16
 * entries per fragment in (u, v, s, t) tap order, each the atlas texel index
 * Y (w n) + X of texel (X, Y) = (i n + s, j n + t) and the weight
 * w_u w_v w_s w_t.  Zero-weight entries (the second tap of a nearest axis) and
 * fragments that are not shaded have index -1 and weight 0.  The texel
 * gradient of a loss is the sum over entries of weight x dL/dout. */
uint32_t oracle_taps(const int32_t* dims, const void* const* codes, int32_t n_obj, int64_t F, const float* uv,
                     const float* dir, const int32_t* obj, int32_t filter, int64_t* index, double* weight) {
    uint32_t flags = 0;
#pragma omp parallel for schedule(static) reduction(| : flags)
    for (int64_t f = 0; f < F; ++f) {
        double u = uv[2 * f], v = uv[2 * f + 1];
        double I[3] = {dir[3 * f], dir[3 * f + 1], dir[3 * f + 2]};
        int shade;
        flags |= classify(obj[f], n_obj, codes, u, v, I, NULL, &shade);
        for (int e = 0; e < 16; ++e) {
            index[16 * f + e] = -1;
            weight[16 * f + e] = 0.0;
        }
        if (!shade) continue;
        tex_t T;
        make_tex(dims, codes, NULL, obj[f], &T);
        lookup_t L;
        locate_one(&T, u, v, I, NULL, filter, &L);
        int e = 0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q, ++e) {
                        double w = L.u.w[a] * L.v.w[b] * L.s.w[p] * L.t.w[q];
                        if (w == 0.0) continue;
                        int64_t X = L.u.tap[a] * T.n + L.s.tap[p], Y = L.v.tap[b] * T.n + L.t.tap[q];
                        index[16 * f + e] = Y * T.W * T.n + X;
                        weight[16 * f + e] = w;
                    }
    }
    return flags;
}

/* The world-space lookup (Eq. 1a with a per-fragment normal nrm, F x 3). */
uint32_t oracle_locate_world(const int32_t* dims, const void* const* codes, int32_t n_obj, int64_t F,
                             const float* uv, const float* dir, const float* nrm, const int32_t* obj, int32_t filter,
                             int32_t* idx, double* coord) {
    return locate_core(dims, codes, n_obj, F, uv, dir, nrm, obj, filter, idx, coord);
}

/* Reads fragment f of an FP32 or FP64 G-buffer; returns the normal pointer
 * (NULL without a normal stream). */
static const double* read_fragment(int64_t f, const float* uv32, const float* dir32, const float* nrm32,
                                   const double* uv64, const double* dir64, const double* nrm64, double* u, double* v,
                                   double I[3], double N[3]) {
    if (uv64) {
        *u = uv64[2 * f];
        *v = uv64[2 * f + 1];
        for (int k = 0; k < 3; ++k) I[k] = dir64[3 * f + k];
        if (!nrm64) return NULL;
        for (int k = 0; k < 3; ++k) N[k] = nrm64[3 * f + k];
        return N;
    }
    *u = uv32[2 * f];
    *v = uv32[2 * f + 1];
    for (int k = 0; k < 3; ++k) I[k] = dir32[3 * f + k];
    if (!nrm32) return NULL;
    for (int k = 0; k < 3; ++k) N[k] = nrm32[3 * f + k];
    return N;
}

static uint32_t shade_core(const int32_t* dims, const void* const* codes, const float* const* scales,
                           int32_t n_obj, int64_t F, const float* uv32, const float* dir32, const float* nrm32,
                           const double* uv64, const double* dir64, const double* nrm64, const int32_t* obj,
                           int32_t filter, double* out) {
    uint32_t flags = 0;
#pragma omp parallel for schedule(static) reduction(| : flags)
    for (int64_t f = 0; f < F; ++f) {
        double u, v, I[3], Nb[3];
        const double* N = read_fragment(f, uv32, dir32, nrm32, uv64, dir64, nrm64, &u, &v, I, Nb);
        int shade;
        flags |= classify(obj[f], n_obj, codes, u, v, I, N, &shade);
        for (int c = 0; c < 4; ++c) out[4 * f + c] = 0.0;
        if (!shade) continue;
        tex_t T;
        make_tex(dims, codes, scales, obj[f], &T);
        lookup_t L;
        locate_one(&T, u, v, I, N, filter, &L);
        colour_one(&T, &L, out + 4 * f);
    }
    return flags;
}

/* Forward synthesis of F fragments with an FP32 G-buffer (uv: F x 2, dir: F x 3,
 * obj: F; obj < 0 is background and gives 0).  dims: n_obj x (w, h, n, format);
 * codes[o]: the stored atlas of object o (NULL: no such object); scales[o]: its
 * per-bucket E4M3 scales.  out: F x 4 FP64.  Returns OR_FLAG_* bits. */
uint32_t oracle_shade(const int32_t* dims, const void* const* codes, const float* const* scales, int32_t n_obj,
                      int64_t F, const float* uv, const float* dir, const int32_t* obj, int32_t filter,
                      double* out) {
    return shade_core(dims, codes, scales, n_obj, F, uv, dir, NULL, NULL, NULL, NULL, obj, filter, out);
}

/* The same with an FP64 G-buffer (finite-difference pins). */
uint32_t oracle_shade64(const int32_t* dims, const void* const* codes, const float* const* scales, int32_t n_obj,
                        int64_t F, const double* uv, const double* dir, const int32_t* obj, int32_t filter,
                        double* out) {
    return shade_core(dims, codes, scales, n_obj, F, NULL, NULL, NULL, uv, dir, NULL, obj, filter, out);
}

/* World-space synthesis: dir (I) and nrm (N) in one frame, A from Eq. 1a. */
uint32_t oracle_shade_world(const int32_t* dims, const void* const* codes, const float* const* scales,
                            int32_t n_obj, int64_t F, const float* uv, const float* dir, const float* nrm,
                            const int32_t* obj, int32_t filter, double* out) {
    return shade_core(dims, codes, scales, n_obj, F, uv, dir, nrm, NULL, NULL, NULL, obj, filter, out);
}

uint32_t oracle_shade_world64(const int32_t* dims, const void* const* codes, const float* const* scales,
                              int32_t n_obj, int64_t F, const double* uv, const double* dir, const double* nrm,
                              const int32_t* obj, int32_t filter, double* out) {
    return shade_core(dims, codes, scales, n_obj, F, NULL, NULL, NULL, uv, dir, nrm, obj, filter, out);
}

/* ------------------------------------------------------------------------ */
/* Gradients (reading R6).                                                  */
/* ------------------------------------------------------------------------ */

/* Jacobian of Eq. 3, J[r][c] = dB_r / dA_c. */
static void squarify_jacobian(const double A[2], double J[2][2]) {
    double ax = fabs(A[0]), ay = fabs(A[1]);
    if (ax == 0.0 && ay == 0.0) {
        J[0][0] = 1.0;
        J[0][1] = 0.0;
        J[1][0] = 0.0;
        J[1][1] = 1.0;
        return;
    }
    double r = sqrt(A[0] * A[0] + A[1] * A[1]);
    if (ax >= ay) { /* B = A r / |A_x| */
        double sx = A[0] > 0.0 ? 1.0 : -1.0;
        J[0][0] = ax / r;
        J[0][1] = sx * A[1] / r;
        J[1][0] = sx * A[1] * (1.0 / r - r / (A[0] * A[0]));
        J[1][1] = (r * r + A[1] * A[1]) / (r * ax);
    } else { /* B = A r / |A_y| */
        double sy = A[1] > 0.0 ? 1.0 : -1.0;
        J[1][1] = ay / r;
        J[1][0] = sy * A[0] / r;
        J[0][1] = sy * A[0] * (1.0 / r - r / (A[1] * A[1]));
        J[0][0] = (r * r + A[0] * A[0]) / (r * ay);
    }
}

/* Jacobian of Eq. 1b, J[r][c] = dA_r / dI_c. */
static void equisolid_jacobian(const double I[3], double J[2][3]) {
    double zp = I[2] + 1.0;
    double D = sqrt(I[0] * I[0] + I[1] * I[1] + zp * zp);
    if (D == 0.0) {
        memset(J, 0, sizeof(double) * 6);
        return;
    }
    double D3 = D * D * D;
    double g[3] = {I[0], I[1], zp}; /* dD/dI = g / D */
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) J[r][c] = SQRT2 * ((r == c ? 1.0 / D : 0.0) - I[r] * g[c] / D3);
}

/* Jacobian of Eq. 1a's first two entries with respect to I (and equally N):
 * with h = I + N, L = |h|: dA_r/dh_c = sqrt(2) (delta_rc / L - h_r h_c / L^3). */
static void equisolid_normal_jacobian(const double I[3], const double N[3], double J[2][3]) {
    double h[3] = {I[0] + N[0], I[1] + N[1], I[2] + N[2]};
    double L = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    if (L == 0.0) {
        memset(J, 0, sizeof(double) * 6);
        return;
    }
    double L3 = L * L * L;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) J[r][c] = SQRT2 * ((r == c ? 1.0 / L : 0.0) - h[r] * h[c] / L3);
}

static uint32_t backward_core(const int32_t* dims, const void* const* codes, const float* const* scales,
                              int32_t n_obj, int64_t F, const float* uv32, const float* dir32, const float* nrm32,
                              const double* uv64, const double* dir64, const double* nrm64, const int32_t* obj,
                              int32_t filter, const double* dL_dout, double* const* dL_dtex, double* dL_duv,
                              double* dL_ddir, double* dL_dnrm) {
    uint32_t flags = 0;
    /* Texel gradients are summed serially, in fragment order. */
    for (int64_t f = 0; f < F; ++f) {
        double u, v, I[3], Nb[3];
        const double* N = read_fragment(f, uv32, dir32, nrm32, uv64, dir64, nrm64, &u, &v, I, Nb);
        if (dL_duv) dL_duv[2 * f] = dL_duv[2 * f + 1] = 0.0;
        if (dL_ddir) dL_ddir[3 * f] = dL_ddir[3 * f + 1] = dL_ddir[3 * f + 2] = 0.0;
        if (dL_dnrm) dL_dnrm[3 * f] = dL_dnrm[3 * f + 1] = dL_dnrm[3 * f + 2] = 0.0;
        int shade;
        flags |= classify(obj[f], n_obj, codes, u, v, I, N, &shade);
        if (!shade) continue;
        tex_t T;
        make_tex(dims, codes, scales, obj[f], &T);
        lookup_t L;
        locate_one(&T, u, v, I, N, filter, &L);
        const double* g = dL_dout + 4 * f;
        const double dw[2] = {-1.0, 1.0}; /* d(weight of tap k)/dc for a bilinear axis */
        double gu = 0.0, gv = 0.0, gs = 0.0, gt = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q) {
                        int64_t i = L.u.tap[a], j = L.v.tap[b], s = L.s.tap[p], t = L.t.tap[q];
                        double w = L.u.w[a] * L.v.w[b] * L.s.w[p] * L.t.w[q];
                        double gT = 0.0; /* sum over channels of g_c T_c */
                        for (int c = 0; c < 4; ++c) gT += g[c] * texel(&T, i, j, s, t, c);
                        gu += dw[a] * L.v.w[b] * L.s.w[p] * L.t.w[q] * gT;
                        gv += L.u.w[a] * dw[b] * L.s.w[p] * L.t.w[q] * gT;
                        gs += L.u.w[a] * L.v.w[b] * dw[p] * L.t.w[q] * gT;
                        gt += L.u.w[a] * L.v.w[b] * L.s.w[p] * dw[q] * gT;
                        if (dL_dtex && dL_dtex[obj[f]] && w != 0.0)
                            for (int c = 0; c < 4; ++c) dL_dtex[obj[f]][atlas_offset(&T, i, j, s, t, c)] += w * g[c];
                    }
        if (dL_duv) {
            dL_duv[2 * f] = gu * L.u.dc;
            dL_duv[2 * f + 1] = gv * L.v.dc;
        }
        if (dL_ddir || dL_dnrm) {
            double gB[2] = {gs * L.s.dc, gt * L.t.dc};
            double J3[2][2], J1[2][3];
            squarify_jacobian(L.A, J3);
            if (N)
                equisolid_normal_jacobian(I, N, J1); /* dA/dI = dA/dN */
            else
                equisolid_jacobian(I, J1);
            double gA[2] = {gB[0] * J3[0][0] + gB[1] * J3[1][0], gB[0] * J3[0][1] + gB[1] * J3[1][1]};
            for (int c = 0; c < 3; ++c) {
                double gI = gA[0] * J1[0][c] + gA[1] * J1[1][c];
                if (dL_ddir) dL_ddir[3 * f + c] = gI;
                if (dL_dnrm && N) dL_dnrm[3 * f + c] = gI;
            }
        }
    }
    return flags;
}

/* Gradients of L with respect to the texels (accumulated into the FP64 atlas
 * dL_dtex[o], which the caller zeroes; NULL to skip), the UVs (F x 2) and the
 * directions (F x 3), given dL/dout (F x 4).  NULL outputs are skipped. */
uint32_t oracle_shade_backward(const int32_t* dims, const void* const* codes, const float* const* scales,
                               int32_t n_obj, int64_t F, const float* uv, const float* dir, const int32_t* obj,
                               int32_t filter, const double* dL_dout, double* const* dL_dtex, double* dL_duv,
                               double* dL_ddir) {
    return backward_core(dims, codes, scales, n_obj, F, uv, dir, NULL, NULL, NULL, NULL, obj, filter, dL_dout, dL_dtex,
                         dL_duv, dL_ddir, NULL);
}

uint32_t oracle_shade_backward64(const int32_t* dims, const void* const* codes, const float* const* scales,
                                 int32_t n_obj, int64_t F, const double* uv, const double* dir, const int32_t* obj,
                                 int32_t filter, const double* dL_dout, double* const* dL_dtex, double* dL_duv,
                                 double* dL_ddir) {
    return backward_core(dims, codes, scales, n_obj, F, NULL, NULL, NULL, uv, dir, NULL, obj, filter, dL_dout, dL_dtex,
                         dL_duv, dL_ddir, NULL);
}

/* World-space gradients: additionally dL/dN (F x 3; equal to dL/dI, since A
 * depends on I + N only). */
uint32_t oracle_shade_world_backward(const int32_t* dims, const void* const* codes, const float* const* scales,
                                     int32_t n_obj, int64_t F, const float* uv, const float* dir, const float* nrm,
                                     const int32_t* obj, int32_t filter, const double* dL_dout,
                                     double* const* dL_dtex, double* dL_duv, double* dL_ddir, double* dL_dnrm) {
    return backward_core(dims, codes, scales, n_obj, F, uv, dir, nrm, NULL, NULL, NULL, obj, filter, dL_dout, dL_dtex,
                         dL_duv, dL_ddir, dL_dnrm);
}

uint32_t oracle_shade_world_backward64(const int32_t* dims, const void* const* codes, const float* const* scales,
                                       int32_t n_obj, int64_t F, const double* uv, const double* dir,
                                       const double* nrm, const int32_t* obj, int32_t filter, const double* dL_dout,
                                       double* const* dL_dtex, double* dL_duv, double* dL_ddir, double* dL_dnrm) {
    return backward_core(dims, codes, scales, n_obj, F, NULL, NULL, NULL, uv, dir, nrm, obj, filter, dL_dout,
                         dL_dtex, dL_duv, dL_ddir, dL_dnrm);
}

/* ------------------------------------------------------------------------ */
/* Texture fills (the paper gives no field; these are the synthetic ones).  */
/* Fill rule: T[i, j, s, t] = f((i + 1/2)/w, (j + 1/2)/h, Eq. 2c(Eq. 4a(B_s, B_t))). */
/* ------------------------------------------------------------------------ */

/* Analytic field with L lobes; lobe k has 11 parameters
 * (a_0..a_3, alpha, beta, gamma, d_x, d_y, d_z, p):
 * f_c(u, v, I) = sum_k a_kc (1/2 + 1/2 cos(2 pi (alpha u + beta v) + gamma)) max(0, I . d)^p. */
static void field_eval(const double* lobes, int32_t L, double u, double v, const double I[3], double out[4]) {
    static const double TWO_PI = 6.28318530717958647692528676655900577;
    for (int c = 0; c < 4; ++c) out[c] = 0.0;
    for (int k = 0; k < L; ++k) {
        const double* P = lobes + 11 * k;
        double spatial = 0.5 + 0.5 * cos(TWO_PI * (P[4] * u + P[5] * v) + P[6]);
        double cosang = I[0] * P[7] + I[1] * P[8] + I[2] * P[9];
        double lobe = cosang > 0.0 ? pow(cosang, P[10]) : 0.0;
        for (int c = 0; c < 4; ++c) out[c] += P[c] * spatial * lobe;
    }
}

/* Field values at arbitrary (uv, I) in FP64 (fitting targets): out count x 4. */
void oracle_eval_field(const double* lobes, int32_t L, int64_t count, const double* uv, const double* dir,
                       double* out) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k) field_eval(lobes, L, uv[2 * k], uv[2 * k + 1], dir + 3 * k, out + 4 * k);
}

/* FP32 atlas (reading R4) filled from the analytic field by the fill rule. */
void oracle_fill_field(int32_t W, int32_t H, int32_t n, const double* lobes, int32_t L, float* atlas) {
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < (int64_t)W * H; ++b) {
        int64_t i = b % W, j = b / W;
        double u = ((double)i + 0.5) / W, v = ((double)j + 0.5) / H;
        for (int64_t t = 0; t < n; ++t)
            for (int64_t s = 0; s < n; ++s) {
                double I[3], val[4];
                texel_direction(s, t, n, I);
                field_eval(lobes, L, u, v, I, val);
                int64_t e = ((j * n + t) * (int64_t)W * n + (i * n + s)) * 4;
                for (int c = 0; c < 4; ++c) atlas[e + c] = (float)val[c];
            }
    }
}

/* FP32 atlas filled from one cosine-power lobe per bucket.  params: w h x 8
 * floats per bucket (rho_r, rho_g, rho_b, d_x, d_y, d_z, p, unused):
 * T_c = rho_c max(0, I . d)^p for c < 3 and T_3 = max(0, I . d)^p. */
void oracle_fill_bucket_lobes(int32_t W, int32_t H, int32_t n, const float* params, float* atlas) {
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < (int64_t)W * H; ++b) {
        int64_t i = b % W, j = b / W;
        const float* P = params + 8 * b;
        for (int64_t t = 0; t < n; ++t)
            for (int64_t s = 0; s < n; ++s) {
                double I[3];
                texel_direction(s, t, n, I);
                double cosang = I[0] * (double)P[3] + I[1] * (double)P[4] + I[2] * (double)P[5];
                double lobe = cosang > 0.0 ? pow(cosang, (double)P[6]) : 0.0;
                int64_t e = ((j * n + t) * (int64_t)W * n + (i * n + s)) * 4;
                atlas[e + 0] = (float)((double)P[0] * lobe);
                atlas[e + 1] = (float)((double)P[1] * lobe);
                atlas[e + 2] = (float)((double)P[2] * lobe);
                atlas[e + 3] = (float)lobe;
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Baking (Section 2.2, Eq. 4a and Eq. 4b).  Each texel centre B of a bucket  */
/* goes back to the equisolid vector A (Eq. 4a) and to the reflection vector  */
/* R (Eq. 4b); the ray from the bucket's surface point along R, taken to      */
/* world space with the surface's tangent frame, is traced through an        */
/* analytic scene and the radiance it brings back is stored.  The paper       */
/* fixes only the direction; reading R10 fixes the scene and its shading, all */
/* smooth so that the hit decisions are the only discontinuities:             */
/*   lit(N)    = a + (1 - a) max(0, N . L)                                     */
/*   sky(d)    = K_h + (K_z - K_h)(1/2 + d_y/2) + S max(0, d . L)^p            */
/*   albedo    : sphere rho_s; plane rho_p (3/4 + cos(w x) cos(w z) / 4)       */
/*   trace(P,d): nearest of the sphere's entering root and the plane hit with  */
/*               t > eps; a miss gives (sky(d), 0), a hit at t gives          */
/*               (f C + (1 - f) sky(d), f), f = exp(-k t), C = albedo lit(N_h) */
/*   texel     = (albedo(P) lit(N(P)) + rho_r trace_rgb(P, R), trace_alpha).   */
/* The bucket's surface point is the bucket centre ((i+1/2)/w, (j+1/2)/h) on  */
/* the sphere (lat-long: phi = 2 pi u - pi, theta = pi v, frame T along       */
/* dP/dphi, B along dP/dtheta, N outward) or on the plane y = h_p (x = 2 e u  */
/* - e, z = 2 e v - e, frame (+x, +z, +y)).                                    */
/* ------------------------------------------------------------------------ */

/* Scene parameters, one flat array of doubles. */
enum {
    BK_SPHERE_C = 0, BK_SPHERE_R = 3, BK_PLANE_Y = 4, BK_PLANE_E = 5, BK_SPHERE_ALB = 6, BK_SPHERE_REFL = 9,
    BK_PLANE_ALB = 10, BK_PLANE_REFL = 13, BK_PLANE_FREQ = 14, BK_SUN_DIR = 15, BK_SUN_RGB = 18, BK_SUN_EXP = 21,
    BK_SKY_ZEN = 22, BK_SKY_HOR = 25, BK_AMBIENT = 28, BK_FOG = 29, BK_EPS = 30, BK_COUNT = 31
};
#define OR_SURFACE_SPHERE 0
#define OR_SURFACE_PLANE 1

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static double lit(const double* S, const double N[3]) {
    double c = dot3(N, S + BK_SUN_DIR);
    return S[BK_AMBIENT] + (1.0 - S[BK_AMBIENT]) * (c > 0.0 ? c : 0.0);
}

static void sky(const double* S, const double d[3], double out[3]) {
    double h = 0.5 + 0.5 * d[1];
    double c = dot3(d, S + BK_SUN_DIR);
    double sun = c > 0.0 ? pow(c, S[BK_SUN_EXP]) : 0.0;
    for (int k = 0; k < 3; ++k)
        out[k] = S[BK_SKY_HOR + k] + (S[BK_SKY_ZEN + k] - S[BK_SKY_HOR + k]) * h + S[BK_SUN_RGB + k] * sun;
}

static void plane_albedo(const double* S, const double x[3], double out[3]) {
    double w = S[BK_PLANE_FREQ];
    double m = 0.75 + 0.25 * cos(w * x[0]) * cos(w * x[2]);
    for (int k = 0; k < 3; ++k) out[k] = S[BK_PLANE_ALB + k] * m;
}

/* Surface point and tangent frame F = (T, B, N) of bucket coordinate (u, v). */
static void surface_frame(const double* S, int surface, double u, double v, double P[3], double F[3][3]) {
    static const double PI = 3.14159265358979323846264338327950288;
    if (surface == OR_SURFACE_SPHERE) {
        double phi = 2.0 * PI * u - PI, theta = PI * v;
        double r = S[BK_SPHERE_R];
        double N[3] = {sin(theta) * cos(phi), cos(theta), sin(theta) * sin(phi)};
        double T[3] = {-sin(phi), 0.0, cos(phi)};
        double B[3] = {cos(theta) * cos(phi), -sin(theta), cos(theta) * sin(phi)};
        for (int k = 0; k < 3; ++k) {
            P[k] = S[BK_SPHERE_C + k] + r * N[k];
            F[0][k] = T[k];
            F[1][k] = B[k];
            F[2][k] = N[k];
        }
    } else {
        double e = S[BK_PLANE_E];
        P[0] = 2.0 * e * u - e;
        P[1] = S[BK_PLANE_Y];
        P[2] = 2.0 * e * v - e;
        double T[3] = {1.0, 0.0, 0.0}, B[3] = {0.0, 0.0, 1.0}, N[3] = {0.0, 1.0, 0.0};
        for (int k = 0; k < 3; ++k) {
            F[0][k] = T[k];
            F[1][k] = B[k];
            F[2][k] = N[k];
        }
    }
}

/* Own (view-independent) colour of a surface point. */
static void surface_base(const double* S, int surface, const double P[3], const double N[3], double out[3]) {
    double l = lit(S, N);
    if (surface == OR_SURFACE_SPHERE) {
        for (int k = 0; k < 3; ++k) out[k] = S[BK_SPHERE_ALB + k] * l;
    } else {
        plane_albedo(S, P, out);
        for (int k = 0; k < 3; ++k) out[k] *= l;
    }
}

/* Radiance along the ray P + t d (d unit), and its fog transmittance. */
static void trace(const double* S, const double P[3], const double d[3], double out[4]) {
    double eps = S[BK_EPS];
    double t_best = INFINITY;
    int hit = -1;
    /* sphere: |P + t d - c|^2 = r^2, entering root t = -b - sqrt(b^2 - q) */
    double o[3] = {P[0] - S[BK_SPHERE_C], P[1] - S[BK_SPHERE_C + 1], P[2] - S[BK_SPHERE_C + 2]};
    double b = dot3(o, d);
    double q = dot3(o, o) - S[BK_SPHERE_R] * S[BK_SPHERE_R];
    double disc = b * b - q;
    if (disc > 0.0) {
        double t = -b - sqrt(disc);
        if (t > eps) {
            t_best = t;
            hit = OR_SURFACE_SPHERE;
        }
    }
    /* plane y = h_p, from above or below */
    if (d[1] != 0.0) {
        double t = (S[BK_PLANE_Y] - P[1]) / d[1];
        if (t > eps && t < t_best) {
            t_best = t;
            hit = OR_SURFACE_PLANE;
        }
    }
    double K[3];
    sky(S, d, K);
    if (hit < 0) {
        for (int k = 0; k < 3; ++k) out[k] = K[k];
        out[3] = 0.0;
        return;
    }
    double X[3] = {P[0] + t_best * d[0], P[1] + t_best * d[1], P[2] + t_best * d[2]};
    double C[3];
    if (hit == OR_SURFACE_SPHERE) {
        double r = S[BK_SPHERE_R];
        double Nh[3] = {(X[0] - S[BK_SPHERE_C]) / r, (X[1] - S[BK_SPHERE_C + 1]) / r, (X[2] - S[BK_SPHERE_C + 2]) / r};
        double l = lit(S, Nh);
        for (int k = 0; k < 3; ++k) C[k] = S[BK_SPHERE_ALB + k] * l;
    } else {
        double up[3] = {0.0, 1.0, 0.0};
        double l = lit(S, up);
        plane_albedo(S, X, C);
        for (int k = 0; k < 3; ++k) C[k] *= l;
    }
    double f = exp(-S[BK_FOG] * t_best);
    for (int k = 0; k < 3; ++k) out[k] = f * C[k] + (1.0 - f) * K[k];
    out[3] = f;
}

static void normalize3(double v[3]) {
    double m = sqrt(dot3(v, v));
    v[0] /= m;
    v[1] /= m;
    v[2] /= m;
}

/* One texel (i, j, s, t) of a w x h x n x n bake: value out[4] and, with lo
 * non-NULL, the range lo[4], hi[4] of the value over ten perturbed rays
 * (origin moved by +-delta along T and B, direction tilted by +-delta along
 * T, B and N and renormalised): the spread of the exact value over inputs one
 * FP32 rounding chain away, which marks rays that graze a hit decision. */
static void bake_texel(const double* S, int surface, int64_t W, int64_t H, int64_t n, int64_t i, int64_t j,
                       int64_t s, int64_t t, double delta, double out[4], double* lo, double* hi) {
    double u = ((double)i + 0.5) / W, v = ((double)j + 0.5) / H;
    double P[3], F[3][3], base[3];
    surface_frame(S, surface, u, v, P, F);
    surface_base(S, surface, P, F[2], base);
    double refl = surface == OR_SURFACE_SPHERE ? S[BK_SPHERE_REFL] : S[BK_PLANE_REFL];
    double B[2] = {texel_centre(s, n), texel_centre(t, n)};
    double A[2], R[3];
    unsquarify(B, A); /* Eq. 4a */
    reflection(A, R); /* Eq. 4b, tangent space */
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = R[0] * F[0][k] + R[1] * F[1][k] + R[2] * F[2][k];
    double tr[4];
    trace(S, P, d, tr);
    for (int k = 0; k < 3; ++k) out[k] = base[k] + refl * tr[k];
    out[3] = tr[3];
    if (!lo) return;
    for (int c = 0; c < 4; ++c) lo[c] = hi[c] = out[c];
    for (int m = 0; m < 10; ++m) {
        double Pp[3] = {P[0], P[1], P[2]}, dp[3] = {d[0], d[1], d[2]};
        double sg = (m & 1) ? -delta : delta;
        if (m < 4) {
            for (int k = 0; k < 3; ++k) Pp[k] += sg * F[m >> 1][k];
        } else {
            for (int k = 0; k < 3; ++k) dp[k] += sg * F[(m - 4) >> 1][k];
            normalize3(dp);
        }
        double tp[4];
        trace(S, Pp, dp, tp);
        double o4[4] = {base[0] + refl * tp[0], base[1] + refl * tp[1], base[2] + refl * tp[2], tp[3]};
        for (int c = 0; c < 4; ++c) {
            if (o4[c] < lo[c]) lo[c] = o4[c];
            if (o4[c] > hi[c]) hi[c] = o4[c];
        }
    }
}

/* Bakes one object into val (atlas order of reading R4, 4 doubles a texel);
 * lo / hi (same shape, or NULL) receive the perturbed-ray range. */
void oracle_bake(int32_t W, int32_t H, int32_t n, int32_t surface, const double* S, double delta, double* val,
                 double* lo, double* hi) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t bk = 0; bk < (int64_t)W * H; ++bk) {
        int64_t i = bk % W, j = bk / W;
        for (int64_t t = 0; t < n; ++t)
            for (int64_t s = 0; s < n; ++s) {
                int64_t e = ((j * n + t) * (int64_t)W * n + (i * n + s)) * 4;
                bake_texel(S, surface, W, H, n, i, j, s, t, delta, val + e, lo ? lo + e : NULL, hi ? hi + e : NULL);
            }
    }
}

/* The same for a list of texels ijst (count x 4 int32: i, j, s, t): rows of 4
 * doubles in val / lo / hi. */
void oracle_bake_texels(int32_t W, int32_t H, int32_t n, int32_t surface, const double* S, double delta,
                        int64_t count, const int32_t* ijst, double* val, double* lo, double* hi) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k) {
        const int32_t* q = ijst + 4 * k;
        bake_texel(S, surface, W, H, n, q[0], q[1], q[2], q[3], delta, val + 4 * k, lo ? lo + 4 * k : NULL,
                   hi ? hi + 4 * k : NULL);
    }
}

/* ------------------------------------------------------------------------ */
/* Shadow textures (Section 5, "Shadowing"; reading R13): a 1-bit radiance   */
/* texture keyed by the light direction.  The bit of texel (i, j, s, t) says  */
/* whether the ray from the bucket's surface point towards the direction of  */
/* texel (s, t) -- Eq. 4a then Eq. 2c, taken to world space -- reaches the   */
/* sky (1) or is blocked by the sphere or the plane at t > eps (0).           */
/* ------------------------------------------------------------------------ */

/* Occlusion of the ray P + t d (d unit), written geometrically: the sphere
 * blocks it when the ray passes within r of the centre and its entry point
 * lies ahead (t > eps); the plane when it is crossed at t > eps. */
static int occluded(const double* S, const double P[3], const double d[3]) {
    double eps = S[BK_EPS], r = S[BK_SPHERE_R];
    double oc[3] = {S[BK_SPHERE_C] - P[0], S[BK_SPHERE_C + 1] - P[1], S[BK_SPHERE_C + 2] - P[2]};
    double tc = dot3(oc, d); /* closest approach along the ray */
    double x[3] = {oc[0] - tc * d[0], oc[1] - tc * d[1], oc[2] - tc * d[2]};
    double m2 = dot3(x, x);
    if (m2 < r * r && tc - sqrt(r * r - m2) > eps) return 1;
    if (d[1] != 0.0 && (S[BK_PLANE_Y] - P[1]) / d[1] > eps) return 1;
    return 0;
}

/* Visibility bit of one texel, and whether it changes under the ten perturbed
 * rays of bake_texel (a ray grazing an occluder: either bit is correct). */
static void shadow_texel(const double* S, int surface, int64_t W, int64_t H, int64_t n, int64_t i, int64_t j,
                         int64_t s, int64_t t, double delta, uint8_t* vis, uint8_t* band) {
    double u = ((double)i + 0.5) / W, v = ((double)j + 0.5) / H;
    double P[3], F[3][3], I[3];
    surface_frame(S, surface, u, v, P, F);
    texel_direction(s, t, n, I); /* Eq. 4a then Eq. 2c */
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = I[0] * F[0][k] + I[1] * F[1][k] + I[2] * F[2][k];
    int o = occluded(S, P, d);
    *vis = (uint8_t)(o ? 0 : 1);
    if (!band) return;
    *band = 0;
    for (int m = 0; m < 10 && !*band; ++m) {
        double Pp[3] = {P[0], P[1], P[2]}, dp[3] = {d[0], d[1], d[2]};
        double sg = (m & 1) ? -delta : delta;
        if (m < 4) {
            for (int k = 0; k < 3; ++k) Pp[k] += sg * F[m >> 1][k];
        } else {
            for (int k = 0; k < 3; ++k) dp[k] += sg * F[(m - 4) >> 1][k];
            normalize3(dp);
        }
        if (occluded(S, Pp, dp) != o) *band = 1;
    }
}

/* Shadow bake of a w x h x n x n texture: vis and band (NULL to skip), one
 * byte per texel in the atlas order of reading R4. */
void oracle_bake_shadow(int32_t W, int32_t H, int32_t n, int32_t surface, const double* S, double delta,
                        uint8_t* vis, uint8_t* band) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t bk = 0; bk < (int64_t)W * H; ++bk) {
        int64_t i = bk % W, j = bk / W;
        for (int64_t t = 0; t < n; ++t)
            for (int64_t s = 0; s < n; ++s) {
                int64_t e = (j * n + t) * (int64_t)W * n + (i * n + s);
                shadow_texel(S, surface, W, H, n, i, j, s, t, delta, vis + e, band ? band + e : NULL);
            }
    }
}

/* The same for a list of texels ijst (count x 4 int32). */
void oracle_bake_shadow_texels(int32_t W, int32_t H, int32_t n, int32_t surface, const double* S, double delta,
                               int64_t count, const int32_t* ijst, uint8_t* vis, uint8_t* band) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k) {
        const int32_t* q = ijst + 4 * k;
        shadow_texel(S, surface, W, H, n, q[0], q[1], q[2], q[3], delta, vis + k, band ? band + k : NULL);
    }
}

/* ------------------------------------------------------------------------ */
/* Deferred payloads (Section 1: a texel may hold data for deferred          */
/* rendering, such as ambient occlusion or reflections, instead of the final */
/* colour; reading R15).  Texel (i, j, s, t) follows the ray of the radiance */
/* bake (Eq. 4a, Eq. 4b) to its first hit X and stores                       */
/*     (albedo(X), AO(X)),   AO(X) = (1/K) sum_k [ray X + t w_k unblocked],  */
/* the AO rays tested against the other surface than the one X lies on.      */
/* the albedo unlit; a ray that reaches the sky stores (0, 0, 0, 1).  The K  */
/* directions w_k are given in the local frame of the hit: z along the       */
/* surface normal that faces the arriving ray, x and y the orthonormal basis */
/* of Duff et al., "Building an Orthonormal Basis, Revisited" (JCGT 6(1),    */
/* 2017) built from that normal.                                             */
/* ------------------------------------------------------------------------ */

/* Orthonormal b1, b2 with (b1, b2, N) right-handed, for unit N (Duff et al.,
 * the branch-free form) with the sign choice sg = +-1 (either is a valid
 * basis when N_z is not -sg). */
static void onb_signed(const double N[3], double sg, double b1[3], double b2[3]) {
    double a = -1.0 / (sg + N[2]);
    double b = N[0] * N[1] * a;
    b1[0] = 1.0 + sg * N[0] * N[0] * a;
    b1[1] = sg * b;
    b1[2] = -sg * N[0];
    b2[0] = b;
    b2[1] = sg + N[1] * N[1] * a;
    b2[2] = -N[1];
}

/* The basis Duff et al. take: sg = the sign of N_z, +1 for +0. */
static void onb_duff(const double N[3], double b1[3], double b2[3]) { onb_signed(N, copysign(1.0, N[2]), b1, b2); }

/* World direction of local w in the frame (b1, b2, N). */
static void local_to_world(const double b1[3], const double b2[3], const double N[3], const double w[3],
                           double out[3]) {
    for (int k = 0; k < 3; ++k) out[k] = w[0] * b1[k] + w[1] * b2[k] + w[2] * N[k];
}

/* occluded() by the other surface than `self` only: a ray leaving a point of
 * the plane into the half-space of its normal cannot meet the plane again, nor
 * one leaving the convex sphere outward meet the sphere, so the AO rays skip
 * the surface they start on (exact, and free of the ray offset there). */
static int occluded_by_other(const double* S, int self, const double P[3], const double d[3]) {
    double eps = S[BK_EPS], r = S[BK_SPHERE_R];
    if (self != OR_SURFACE_SPHERE) {
        double oc[3] = {S[BK_SPHERE_C] - P[0], S[BK_SPHERE_C + 1] - P[1], S[BK_SPHERE_C + 2] - P[2]};
        double tc = dot3(oc, d);
        double x[3] = {oc[0] - tc * d[0], oc[1] - tc * d[1], oc[2] - tc * d[2]};
        double m2 = dot3(x, x);
        if (m2 < r * r && tc - sqrt(r * r - m2) > eps) return 1;
    }
    if (self != OR_SURFACE_PLANE && d[1] != 0.0 && (S[BK_PLANE_Y] - P[1]) / d[1] > eps) return 1;
    return 0;
}

/* Unblocked directions among the K at X with normal N, given the basis.
 * With amb non-NULL, *amb counts the directions whose test changes when X is
 * moved by +-delta along b1, b2, N or the direction is tilted by +-delta
 * along b1, b2 (grazing an occluder), and *amb_vis how many of those were
 * unblocked. */
static int visible_count(const double* S, int self, const double X[3], const double N[3], const double b1[3],
                         const double b2[3], int K, const double* dirs, double delta, int* amb, int* amb_vis) {
    int vis = 0;
    if (amb) *amb = *amb_vis = 0;
    for (int k = 0; k < K; ++k) {
        double w[3];
        local_to_world(b1, b2, N, dirs + 3 * k, w);
        int o = occluded_by_other(S, self, X, w);
        vis += !o;
        if (!amb) continue;
        const double* ax[3] = {b1, b2, N};
        int flips = 0;
        for (int m = 0; m < 10 && !flips; ++m) {
            double sg = (m & 1) ? -delta : delta;
            double Xp[3] = {X[0], X[1], X[2]}, wp[3] = {w[0], w[1], w[2]};
            if (m < 6) {
                for (int c = 0; c < 3; ++c) Xp[c] += sg * ax[m >> 1][c];
            } else {
                for (int c = 0; c < 3; ++c) wp[c] += sg * ax[(m - 6) >> 1][c];
                normalize3(wp);
            }
            flips = occluded_by_other(S, self, Xp, wp) != o;
        }
        if (flips) {
            ++*amb;
            *amb_vis += !o;
        }
    }
    return vis;
}

/* First hit of the ray P + t d (t > eps): surface (-1 for the sky), point X,
 * the normal N facing the ray and the unlit albedo. */
static int first_hit(const double* S, const double P[3], const double d[3], double X[3], double N[3],
                     double alb[3]) {
    double eps = S[BK_EPS], r = S[BK_SPHERE_R];
    double t_best = INFINITY;
    int hit = -1;
    double o[3] = {P[0] - S[BK_SPHERE_C], P[1] - S[BK_SPHERE_C + 1], P[2] - S[BK_SPHERE_C + 2]};
    double b = dot3(o, d), q = dot3(o, o) - r * r, disc = b * b - q;
    if (disc > 0.0) {
        double t = -b - sqrt(disc);
        if (t > eps) {
            t_best = t;
            hit = OR_SURFACE_SPHERE;
        }
    }
    if (d[1] != 0.0) {
        double t = (S[BK_PLANE_Y] - P[1]) / d[1];
        if (t > eps && t < t_best) {
            t_best = t;
            hit = OR_SURFACE_PLANE;
        }
    }
    if (hit < 0) return hit;
    for (int k = 0; k < 3; ++k) X[k] = P[k] + t_best * d[k];
    if (hit == OR_SURFACE_SPHERE) {
        for (int k = 0; k < 3; ++k) {
            N[k] = (X[k] - S[BK_SPHERE_C + k]) / r;
            alb[k] = S[BK_SPHERE_ALB + k];
        }
    } else {
        N[0] = N[2] = 0.0;
        N[1] = d[1] < 0.0 ? 1.0 : -1.0;
        plane_albedo(S, X, alb);
    }
    return hit;
}

/* The deferred payload of the ray P + d; with lo / hi non-NULL, widened by its
 * ambiguous AO directions and, on the sphere, by the basis of the opposite
 * sign choice when the hit normal's z lies within 2^-16 of 0. */
static void deferred_ray(const double* S, const double P[3], const double d[3], int K, const double* dirs,
                         double delta, double out[4], double* lo, double* hi) {
    double X[3], N[3], alb[3];
    int hit = first_hit(S, P, d, X, N, alb);
    if (hit < 0) {
        out[0] = out[1] = out[2] = 0.0;
        out[3] = 1.0;
        if (lo)
            for (int c = 0; c < 4; ++c) lo[c] = hi[c] = out[c];
        return;
    }
    double b1[3], b2[3];
    onb_duff(N, b1, b2);
    int amb = 0, amb_vis = 0;
    int vis = visible_count(S, hit, X, N, b1, b2, K, dirs, delta, lo ? &amb : NULL, &amb_vis);
    for (int k = 0; k < 3; ++k) out[k] = alb[k];
    out[3] = (double)vis / K;
    if (!lo) return;
    for (int c = 0; c < 3; ++c) lo[c] = hi[c] = out[c];
    lo[3] = (double)(vis - amb_vis) / K;
    hi[3] = (double)(vis + (amb - amb_vis)) / K;
    if (hit == OR_SURFACE_PLANE) {
        /* A grazing ray meets the plane far away: a direction error of 2^-20 (a
         * few FP32 roundings) moves the hit by t 2^-20 / |d_y| along the plane.
         * Past a tenth of a radian of the pattern's phase the albedo is not
         * determined by FP32 inputs: the range becomes the pattern's whole
         * range, albedo x [1/2, 1]. */
        double t = sqrt((X[0] - P[0]) * (X[0] - P[0]) + (X[1] - P[1]) * (X[1] - P[1]) +
                        (X[2] - P[2]) * (X[2] - P[2]));
        if (S[BK_PLANE_FREQ] * t * 0x1p-20 / fabs(d[1]) > 0.1)
            for (int c = 0; c < 3; ++c) {
                lo[c] = fmin(lo[c], 0.5 * S[BK_PLANE_ALB + c]);
                hi[c] = fmax(hi[c], S[BK_PLANE_ALB + c]);
            }
    }
    if (hit == OR_SURFACE_SPHERE && fabs(N[2]) < 0x1p-16) {
        /* a computed N_z this small may have the other sign in FP32, hence the other basis (the
         * plane's normal has an exact zero z on both sides) */
        double c1[3], c2[3];
        onb_signed(N, -copysign(1.0, N[2]), c1, c2);
        double other = (double)visible_count(S, hit, X, N, c1, c2, K, dirs, delta, NULL, NULL) / K;
        if (other < lo[3]) lo[3] = other;
        if (other > hi[3]) hi[3] = other;
    }
}

/* One deferred texel: value, and with lo non-NULL the range over the ten
 * perturbed primary rays of bake_texel and the ambiguous AO directions. */
static void deferred_texel(const double* S, int surface, int64_t W, int64_t H, int64_t n, int64_t i, int64_t j,
                           int64_t s, int64_t t, int K, const double* dirs, double delta, double out[4], double* lo,
                           double* hi) {
    double u = ((double)i + 0.5) / W, v = ((double)j + 0.5) / H;
    double P[3], F[3][3];
    surface_frame(S, surface, u, v, P, F);
    double B[2] = {texel_centre(s, n), texel_centre(t, n)};
    double A[2], R[3];
    unsquarify(B, A); /* Eq. 4a */
    reflection(A, R); /* Eq. 4b */
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = R[0] * F[0][k] + R[1] * F[1][k] + R[2] * F[2][k];
    deferred_ray(S, P, d, K, dirs, delta, out, lo, hi);
    if (!lo) return;
    for (int m = 0; m < 10; ++m) {
        double Pp[3] = {P[0], P[1], P[2]}, dp[3] = {d[0], d[1], d[2]};
        double sg = (m & 1) ? -delta : delta;
        if (m < 4) {
            for (int k = 0; k < 3; ++k) Pp[k] += sg * F[m >> 1][k];
        } else {
            for (int k = 0; k < 3; ++k) dp[k] += sg * F[(m - 4) >> 1][k];
            normalize3(dp);
        }
        double o4[4];
        deferred_ray(S, Pp, dp, K, dirs, delta, o4, NULL, NULL);
        for (int c = 0; c < 4; ++c) {
            if (o4[c] < lo[c]) lo[c] = o4[c];
            if (o4[c] > hi[c]) hi[c] = o4[c];
        }
    }
}

/* Deferred bake of a w x h x n x n texture (atlas order of reading R4, 4
 * doubles a texel); lo / hi as in oracle_bake. dirs: K local directions. */
void oracle_bake_deferred(int32_t W, int32_t H, int32_t n, int32_t surface, const double* S, int32_t K,
                          const double* dirs, double delta, double* val, double* lo, double* hi) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t bk = 0; bk < (int64_t)W * H; ++bk) {
        int64_t i = bk % W, j = bk / W;
        for (int64_t t = 0; t < n; ++t)
            for (int64_t s = 0; s < n; ++s) {
                int64_t e = ((j * n + t) * (int64_t)W * n + (i * n + s)) * 4;
                deferred_texel(S, surface, W, H, n, i, j, s, t, K, dirs, delta, val + e, lo ? lo + e : NULL,
                               hi ? hi + e : NULL);
            }
    }
}

/* The same for a list of texels ijst (count x 4 int32). */
void oracle_bake_deferred_texels(int32_t W, int32_t H, int32_t n, int32_t surface, const double* S, int32_t K,
                                 const double* dirs, double delta, int64_t count, const int32_t* ijst, double* val,
                                 double* lo, double* hi) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k) {
        const int32_t* q = ijst + 4 * k;
        deferred_texel(S, surface, W, H, n, q[0], q[1], q[2], q[3], K, dirs, delta, val + 4 * k,
                       lo ? lo + 4 * k : NULL, hi ? hi + 4 * k : NULL);
    }
}

/* AO at given points X (rows of 3) of surface `self` (the surface the rays
 * leave, or -1 to test both) with unit normals N: out[count]. */
void oracle_ambient_occlusion(const double* S, int32_t self, int64_t count, const double* X, const double* N,
                              int32_t K, const double* dirs, double* out) {
    for (int64_t k = 0; k < count; ++k) {
        double b1[3], b2[3];
        onb_duff(N + 3 * k, b1, b2);
        out[k] = (double)visible_count(S, self, X + 3 * k, N + 3 * k, b1, b2, K, dirs, 0.0, NULL, NULL) / K;
    }
}

/* The basis of onb_duff for given unit normals (rows of 3): b1, b2. */
void oracle_onb(int64_t count, const double* N, double* b1, double* b2) {
    for (int64_t k = 0; k < count; ++k) onb_duff(N + 3 * k, b1 + 3 * k, b2 + 3 * k);
}

/* The world-space reflection ray of texel (s, t) at bucket coordinate (u, v):
 * origin P, direction d and the frame rows T, B, N (9 doubles), for the pins. */
void oracle_bake_ray(int32_t n, int32_t surface, const double* S, double u, double v, int32_t s, int32_t t,
                     double* P, double* d, double* frame) {
    double F[3][3];
    surface_frame(S, surface, u, v, P, F);
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) frame[3 * r + k] = F[r][k];
    double B[2] = {texel_centre(s, n), texel_centre(t, n)};
    double A[2], R[3];
    unsquarify(B, A);
    reflection(A, R);
    for (int k = 0; k < 3; ++k) d[k] = R[0] * F[0][k] + R[1] * F[1][k] + R[2] * F[2][k];
}

/* trace() for given rays (rows of 3): out count x 4. */
void oracle_trace(const double* S, int64_t count, const double* P, const double* d, double* out) {
    for (int64_t k = 0; k < count; ++k) trace(S, P + 3 * k, d + 3 * k, out + 4 * k);
}

/* ------------------------------------------------------------------------ */
/* Bucket compression (Section 2: buckets are highly repetitive and change  */
/* only slightly from one to another, "a great case for a simple            */
/* compression").  Reading R11: a palette of K buckets and an index map;    */
/* bucket (i, j) holds palette bucket index[j w + i].  The encoder is        */
/* k-means over the buckets as vectors of n^2 x 4 values (Lloyd's steps).   */
/* ------------------------------------------------------------------------ */

/* The dense texture a palette texture stands for (its definition): codes of
 * bucket (i, j) = codes of palette bucket index[j w + i].  Palette codes are a
 * K x 1 atlas (n rows of K n texels), elem_bytes per channel code; E4M3
 * scales follow their palette bucket. */
void oracle_palette_expand(int32_t W, int32_t H, int32_t n, int32_t K, int32_t elem_bytes, const void* palette,
                           const float* palette_scales, const uint32_t* index, void* dense, float* dense_scales) {
    const uint8_t* P = (const uint8_t*)palette;
    uint8_t* D = (uint8_t*)dense;
    int64_t texel = 4 * (int64_t)elem_bytes;
    for (int64_t j = 0; j < H; ++j)
        for (int64_t i = 0; i < W; ++i) {
            int64_t k = index[j * W + i];
            if (dense_scales) dense_scales[j * W + i] = palette_scales[k];
            for (int64_t t = 0; t < n; ++t)
                for (int64_t s = 0; s < n; ++s) {
                    int64_t src = (t * (int64_t)K * n + k * n + s) * texel;
                    int64_t dst = ((j * n + t) * (int64_t)W * n + i * n + s) * texel;
                    memcpy(D + dst, P + src, (size_t)texel);
                }
        }
}

/* k-means assignment: for every row x_b of X (B x D), the nearest centroid
 * index[b] = argmin_k |x_b - c_k|^2 (ties to the lowest k) and that squared
 * distance; all distances in dist_all (B x K) when non-NULL. */
void oracle_kmeans_assign(int64_t B, int64_t D, const double* X, int64_t K, const double* C, uint32_t* index,
                          double* dist, double* dist_all) {
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < B; ++b) {
        double best = INFINITY;
        int64_t arg = 0;
        for (int64_t k = 0; k < K; ++k) {
            double acc = 0.0;
            for (int64_t d = 0; d < D; ++d) {
                double e = X[b * D + d] - C[k * D + d];
                acc += e * e;
            }
            if (dist_all) dist_all[b * K + k] = acc;
            if (acc < best) {
                best = acc;
                arg = k;
            }
        }
        index[b] = (uint32_t)arg;
        if (dist) dist[b] = best;
    }
}

/* k-means update: c_k = mean of the rows assigned to k; a centroid with no
 * rows keeps its previous value (C holds the previous centroids on entry). */
void oracle_kmeans_update(int64_t B, int64_t D, const double* X, int64_t K, const uint32_t* index, double* C,
                          int64_t* counts) {
    double* sum = (double*)calloc((size_t)(K * D), sizeof(double));
    for (int64_t k = 0; k < K; ++k) counts[k] = 0;
    for (int64_t b = 0; b < B; ++b) {
        int64_t k = index[b];
        counts[k] += 1;
        for (int64_t d = 0; d < D; ++d) sum[k * D + d] += X[b * D + d];
    }
    for (int64_t k = 0; k < K; ++k)
        if (counts[k] > 0)
            for (int64_t d = 0; d < D; ++d) C[k * D + d] = sum[k * D + d] / (double)counts[k];
    free(sum);
}

int32_t oracle_num_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int32_t k) {
#ifdef _OPENMP
    omp_set_num_threads(k);
#else
    (void)k;
#endif
}

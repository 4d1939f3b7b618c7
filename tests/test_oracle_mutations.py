"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source: a sign, an
index, a swapped operand, an off-by-half-texel centre, a missing clamp, a
wrong tie rule, a wrong constant.  The copy is built on the CPU, and the pin
files that cover that part of the oracle run against it in a subprocess.  At
least one pin must fail; a mutant that passes every pin would mean its part
of the oracle is not pinned."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "radtex_oracle.c")

PINS = "tests/test_oracle_pins.py"
BAKE = "tests/test_oracle_bake.py"
PALETTE = "tests/test_oracle_palette.py"
WORLD = "tests/test_oracle_world.py"
SHADOW = "tests/test_oracle_shadow.py"
DEFERRED = "tests/test_oracle_deferred.py"
PATTERN = "tests/test_oracle_pattern.py"

# (name, original text, mutated text, pin files expected to catch it)
MUTATIONS = [
    ("eq1b_sign", "double zp = I[2] + 1.0;", "double zp = I[2] - 1.0;", [PINS]),
    ("eq3_inverted_ratio", "B[0] = A[0] * r / m;", "B[0] = A[0] * m / r;", [PINS]),
    ("texel_centre_half_off", "return (2.0 * (double)k + 1.0) / (double)n - 1.0;",
     "return (2.0 * (double)k) / (double)n - 1.0;", [PINS]),
    ("spatial_half_texel", "double c = x * (double)size - 0.5;", "double c = x * (double)size;", [PINS]),
    ("missing_note_clamp", "double lo = 1.0 / (double)n - 1.0, hi = 1.0 - 1.0 / (double)n;",
     "double lo = -1.0, hi = 1.0;", [PINS]),
    ("atlas_s_t_swapped", "int64_t X = i * T->n + s, Y = j * T->n + t;",
     "int64_t X = i * T->n + t, Y = j * T->n + s;", [PINS]),
    ("e4m3_wrong_max", "amax / 448.0f", "amax / 240.0f", [PINS]),
    ("grad_wrong_index", "gu += dw[a] * L.v.w[b]", "gu += dw[b] * L.v.w[b]", [PINS]),
    ("eq4b_sign", "R[2] = 1.0 - a2;", "R[2] = a2 - 1.0;", [PINS, BAKE]),
    ("bake_fog", "double f = exp(-S[BK_FOG] * t_best);", "double f = exp(-0.5 * S[BK_FOG] * t_best);", [BAKE]),
    ("bake_sun_exponent", "double sun = c > 0.0 ? pow(c, S[BK_SUN_EXP]) : 0.0;",
     "double sun = c > 0.0 ? pow(c, S[BK_SUN_EXP] + 1.0) : 0.0;", [BAKE]),
    ("kmeans_tie_to_higher", "if (acc < best) {", "if (acc <= best) {", [PALETTE]),
    ("palette_index_transposed", "int64_t k = index[j * W + i];", "int64_t k = index[(i * H + j) % (W * H)];",
     [PALETTE]),
    ("shadow_shrunk_occluder", "if (m2 < r * r && tc - sqrt(r * r - m2) > eps) return 1;",
     "if (m2 < 0.81 * r * r && tc - sqrt(r * r - m2) > eps) return 1;", [SHADOW]),
    ("shadow_plane_sign", "if (d[1] != 0.0 && (S[BK_PLANE_Y] - P[1]) / d[1] > eps) return 1;",
     "if (d[1] != 0.0 && (P[1] - S[BK_PLANE_Y]) / d[1] > eps) return 1;", [SHADOW]),
    ("eq1a_minus_normal", "double h[3] = {I[0] + N[0], I[1] + N[1], I[2] + N[2]};",
     "double h[3] = {I[0] - N[0], I[1] - N[1], I[2] + N[2]};", [PINS, WORLD]),
    ("repeat_negative_modulo", "return r < 0 ? r + size : r;", "return r < 0 ? -r : r;", [WORLD]),
    ("deferred_wrong_albedo", "alb[k] = S[BK_SPHERE_ALB + k];", "alb[k] = S[BK_PLANE_ALB + k];", [DEFERRED]),
    ("deferred_plane_normal_side", "N[1] = d[1] < 0.0 ? 1.0 : -1.0;", "N[1] = d[1] < 0.0 ? -1.0 : 1.0;",
     [DEFERRED]),
    ("onb_flipped_b2", "    b2[2] = -N[1];", "    b2[2] = N[1];", [DEFERRED]),
    ("ao_counts_blocked", "vis += !o;", "vis += o;", [DEFERRED]),
    ("deferred_sky_occluded", "out[3] = 1.0;\n        if (lo)", "out[3] = 0.0;\n        if (lo)", [DEFERRED]),
    ("deferred_from_origin_side", "for (int k = 0; k < 3; ++k) X[k] = P[k] + t_best * d[k];",
     "for (int k = 0; k < 3; ++k) X[k] = P[k] + 0.5 * t_best * d[k];", [DEFERRED]),
    ("nearest_angular_half_off", "double c = (Bc + 1.0) * (double)n / 2.0;",
     "double c = (Bc + 1.0) * (double)n / 2.0 - 0.5;", [PINS]),
    ("bf16_mantissa_bits", "static const fmt_t FMT_BF16 = {7, -126, 127, 8,",
     "static const fmt_t FMT_BF16 = {8, -126, 127, 8,", [PINS]),
    ("eq1a_without_sqrt2", "for (int k = 0; k < 3; ++k) A3[k] = SQRT2 * h[k] / L;",
     "for (int k = 0; k < 3; ++k) A3[k] = h[k] / L;", [PINS, WORLD]),
    ("kmeans_mean_off_by_one", "C[k * D + d] = sum[k * D + d] / (double)counts[k];",
     "C[k * D + d] = sum[k * D + d] / (double)(counts[k] + 1);", [PALETTE]),
    ("rounding_half_up", "double q = rint(a / quantum) * quantum;", "double q = floor(a / quantum + 0.5) * quantum;",
     [PINS]),
    ("subnormal_quantum_lost", "if (ex < f->emin) ex = f->emin; /* subnormal quantum */",
     "if (ex < f->emin - 1) ex = f->emin - 1; /* subnormal quantum */", [PINS]),
    ("clamp_passes_gradient", "double inside = (B > lo && B < hi) ? 1.0 : 0.0;", "double inside = 1.0;", [PINS]),
    ("sky_gradient_inverted", "double h = 0.5 + 0.5 * d[1];", "double h = 0.5 - 0.5 * d[1];", [BAKE]),
    ("lit_ambient_unscaled", "return S[BK_AMBIENT] + (1.0 - S[BK_AMBIENT]) * (c > 0.0 ? c : 0.0);",
     "return S[BK_AMBIENT] + (c > 0.0 ? c : 0.0);", [BAKE]),
    ("plane_pattern_axis", "cos(w * x[0]) * cos(w * x[2])", "cos(w * x[0]) * cos(w * x[1])", [BAKE, DEFERRED]),
    ("eq1b_jacobian_sign", "J[r][c] = SQRT2 * ((r == c ? 1.0 / D : 0.0) - I[r] * g[c] / D3);",
     "J[r][c] = SQRT2 * ((r == c ? 1.0 / D : 0.0) + I[r] * g[c] / D3);", [PINS]),
    ("spatial_derivative_scale", "a->dc = (c > -1.0 && c < (double)size) ? (double)size : 0.0;",
     "a->dc = (c > -1.0 && c < (double)size) ? (double)(size - 1) : 0.0;", [PINS]),
    ("eq1a_jacobian_power", "J[r][c] = SQRT2 * ((r == c ? 1.0 / L : 0.0) - h[r] * h[c] / L3);",
     "J[r][c] = SQRT2 * ((r == c ? 1.0 / L : 0.0) - h[r] * h[c] / (L * L));", [WORLD]),
    ("eq3_tie_takes_y_branch", "if (ax >= ay) { /* B = A r / |A_x| */", "if (ax > ay) { /* B = A r / |A_x| */",
     [PINS]),
    ("bit_texel_inverted", "return (double)(((const uint8_t*)T->codes)[e] & 1u);",
     "return (double)((((const uint8_t*)T->codes)[e] & 1u) ^ 1u);", [SHADOW]),
    ("repeat_v_reads_u_flag", "spatial_axis(v, T->H, spatial_bilinear, (T->wrap >> 1) & 1, &L->v);",
     "spatial_axis(v, T->H, spatial_bilinear, T->wrap & 1, &L->v);", [WORLD]),
    ("bucket_lobe_exponent", "double lobe = cosang > 0.0 ? pow(cosang, (double)P[6]) : 0.0;",
     "double lobe = cosang > 0.0 ? pow(cosang, (double)P[6] + 1.0) : 0.0;", [PINS]),
    ("pattern_x_y_swapped", "const int64_t q = (p[c] * X + p[4 + c] * Y + p[8 + c]) % (2 * m);",
     "const int64_t q = (p[c] * Y + p[4 + c] * X + p[8 + c]) % (2 * m);", [PATTERN]),
    ("taps_s_t_swapped", "int64_t X = L.u.tap[a] * T.n + L.s.tap[p], Y = L.v.tap[b] * T.n + L.t.tap[q];",
     "int64_t X = L.u.tap[a] * T.n + L.t.tap[q], Y = L.v.tap[b] * T.n + L.s.tap[p];", [PATTERN]),
]


@pytest.mark.parametrize("name,old,new,files", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_the_mutation(tmp_path, name, old, new, files):
    text = open(SRC).read()
    assert text.count(old) >= 1, f"{name}: the original text is not in the oracle"
    mutated = text.replace(old, new, 1)
    src = tmp_path / "mutant.c"
    src.write_text(mutated)
    lib = oracle.compile_oracle(str(src), str(tmp_path / "libmutant.so"))
    env = dict(os.environ, RADTEX_ORACLE_LIB=lib)
    run = subprocess.run([sys.executable, "-m", "pytest", *files, "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert run.returncode == 1 and " failed" in run.stdout, (
        f"mutation {name} was not caught by {files}:\n{run.stdout[-1500:]}\n{run.stderr[-500:]}")

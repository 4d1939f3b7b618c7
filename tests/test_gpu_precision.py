"""GPU: error of each stored texel format against the FP64 oracle (the tiny quad
workload, 64^2 buckets x 8^2 directions).

The reference is the oracle shading the FP32 texture exactly (FP64 arithmetic);
each format's GPU output is compared with it, so the error is storage rounding
plus kernel rounding.  Filtering is a convex combination, so the filtered
error is bounded by the largest texel error: 2^-11 (FP16), 2^-8 (BF16) and
2^-4 (E4M3 with a per-bucket scale) relative to the largest texel, plus the
1e-5 kernel tolerance.  Prints the table (max-abs, PSNR with peak 1.0)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_01719_gb300 import api
from parity_util import gbuffer_to_dev, quad_workload, to_dev

pytestmark = pytest.mark.gpu

BOUND = {api.RT_F32: 0.0, api.RT_F16: 2.0 ** -11, api.RT_BF16: 2.0 ** -8, api.RT_E4M3_BUCKET_SCALE: 2.0 ** -4}
NAMES = {api.RT_F32: "FP32", api.RT_F16: "FP16", api.RT_BF16: "BF16", api.RT_E4M3_BUCKET_SCALE: "FP8 E4M3 + bucket scale"}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    c = api.Context(0)
    yield c
    c.close()


def psnr(err2_mean):
    return float("inf") if err2_mean == 0 else 10 * np.log10(1.0 / err2_mean)


@pytest.mark.parametrize("filt", [api.RT_NEAREST, api.RT_QUADRILINEAR])
def test_storage_format_error_vs_fp64_oracle(ctx, filt):
    W, H, n = 64, 64, 8
    atlas, g, _ = quad_workload(api.RT_F32, W, H, n)
    exact = oracle.Texture(W, H, n, oracle.F64, atlas.astype(np.float64))
    ref, _ = oracle.shade([exact], g.uv, g.dir, g.obj, filt)
    hit = g.obj >= 0
    tmax = float(np.abs(atlas).max())
    uv, d, o = gbuffer_to_dev(g)
    rows = []
    for fmt in (api.RT_F32, api.RT_F16, api.RT_BF16, api.RT_E4M3_BUCKET_SCALE):
        oid = api.rt_create_texture(ctx, W, H, n, fmt, api.RT_LAYOUT_ATLAS, to_dev(atlas))
        obj = torch.where(o >= 0, torch.full_like(o, oid), o)
        out = api.rt_shade(ctx, uv, d, obj, filt).cpu().numpy()
        err = np.abs(out - ref)[hit]
        rows.append((NAMES[fmt], float(err.max()), psnr(float((err ** 2).mean())),
                     api.rt_texture_info(ctx, oid)["bytes"]))
        if filt == api.RT_QUADRILINEAR:
            assert err.max() <= BOUND[fmt] * tmax + 1e-5, (NAMES[fmt], err.max())
        else:  # nearest: a floor that flips inside the FP32 band picks a neighbouring texel
            assert np.quantile(err, 0.999) <= BOUND[fmt] * tmax + 1e-5
        api.rt_destroy_texture(ctx, oid)
    name = {api.RT_NEAREST: "nearest", api.RT_QUADRILINEAR: "quadrilinear"}[filt]
    print(f"\n| format ({name}, 64^2 x 8^2, quad 256^2) | max abs error | PSNR (dB) | texture bytes |")
    print("|---|---:|---:|---:|")
    for r in rows:
        print(f"| {r[0]} | {r[1]:.3e} | {r[2]:.1f} | {r[3]} |")
    # coarser storage never beats finer storage here
    assert rows[0][2] >= rows[1][2] >= rows[3][2] and rows[1][2] >= rows[2][2]

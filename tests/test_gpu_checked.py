"""The bounds-checked build, libradtex_checked.so (compiled with RADTEX_CHECKED).

A process loads one of the two libraries, chosen by RADTEX_CHECKED when the
binding first loads it.  So the outer test runs the whole GPU suite again in a
child pytest with RADTEX_CHECKED=1: there every case must pass against the
checked build with no bounds error raised (conftest.py reads the status of
every live context after each test), and the checked-only tests below run.

The failure path is exercised without a bad address.  rt_checked_limit_extent
lowers the extent the checks allow below the object's real size (here to the
median of the oracle's weighted taps), so in-bounds accesses past it raise
RT_ERR_OUT_OF_BOUNDS and go to texel 0 instead.  The expected results follow
from the oracle: the colours are those of a texture whose texels past the limit
hold texel 0's codes; the texel gradients are the oracle's below the limit,
zero past it (nothing is written there), and texel 0 also receives the sum of
the gradients past the limit."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_2301_01719_gb300 import _lib, api
from parity_util import COLOUR_TOL, atlas_to_storage, quad_workload, storage_index, storage_to_atlas, to_dev

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build(checked=_lib.CHECKED)
    c = api.Context(0)
    yield c
    c.close()


def test_parity_suites_pass_on_the_checked_build():
    if _lib.CHECKED:
        pytest.skip("this process already runs the checked build")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build(checked=True)
    env = dict(os.environ, RADTEX_CHECKED="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider", HERE]
    r = subprocess.run(cmd, env=env, cwd=ROOT, capture_output=True, text=True, timeout=1800)
    tail = r.stdout[-6000:] + "\n" + r.stderr[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and " failed" not in r.stdout, tail


def test_normal_build_checks_nothing(ctx):
    if _lib.CHECKED:
        pytest.skip("the normal build only")
    oid = api.rt_create_texture(ctx, 4, 4, 2, api.RT_F16)
    assert api.rt_checked_limit_extent(ctx, oid, 0) == api.RT_ERR_UNSUPPORTED
    api.rt_destroy_texture(ctx, oid)


def _checked_only():
    if not _lib.CHECKED:
        pytest.skip("runs in the checked build's child process")


def test_checked_library_is_the_one_loaded(ctx):
    _checked_only()
    assert os.path.basename(_lib.LIB_PATH) == "libradtex_checked.so"
    assert os.path.samefile(_lib.lib()._name, _lib.LIB_PATH)


def test_limit_rejects_bad_arguments(ctx):
    _checked_only()
    W, H, n = 8, 6, 4
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F32)
    texels = W * H * n * n
    assert api.rt_checked_limit_extent(ctx, oid, texels + 1) == api.RT_ERR_INVALID_ARG
    assert api.rt_checked_limit_extent(ctx, oid, -1) == api.RT_ERR_INVALID_ARG
    assert api.rt_checked_limit_extent(ctx, oid + 1, 0) == api.RT_ERR_INVALID_ARG
    assert api.rt_checked_limit_extent(ctx, -1, 0) == api.RT_ERR_INVALID_ARG
    assert api.rt_checked_limit_extent(ctx, oid, texels) == api.RT_OK
    api.rt_destroy_texture(ctx, oid)
    assert api.rt_checked_limit_extent(ctx, oid, 0) == api.RT_ERR_INVALID_ARG  # dead object


def _substituted(T, layout, W, H, n, limit):
    """The oracle texture whose texels at storage index >= limit hold texel 0's codes."""
    P = atlas_to_storage(T.codes, layout, W, H, n).reshape(-1, 4)
    P[limit:] = P[0]
    return oracle.Texture(W, H, n, T.fmt, storage_to_atlas(P, layout, W, H, n))


def _median_tap(table, g, obj_np, filt, layout, W, H, n):
    """The median storage index of the taps with a non-zero weight (the
    oracle's taps are atlas indices (j n + t) w n + i n + s)."""
    idx, weight, _ = oracle.taps(table, g.uv, g.dir, obj_np, filt)
    keep = (idx >= 0) & (weight > 0)
    Y, X = np.divmod(idx[keep], W * n)
    j, t = np.divmod(Y, n)
    i, s = np.divmod(X, n)
    return int(np.median(storage_index(layout, W, H, n, i, j, s, t)))


@pytest.mark.parametrize("path", ["flat", "batched", "fused"])
@pytest.mark.parametrize("filt", [api.RT_ANGULAR_BILINEAR, api.RT_QUADRILINEAR])
def test_accesses_past_the_limit_are_redirected_and_reported(ctx, path, filt):
    _checked_only()
    W, H, n = 32, 32, 8
    width = height = 256
    atlas, g, T = quad_workload(api.RT_F16, W, H, n, width=width, height=height)
    oid = api.rt_create_texture(ctx, W, H, n, api.RT_F16, api.RT_LAYOUT_ATLAS, to_dev(atlas))
    assert api.rt_get_error(ctx) == api.RT_OK
    obj_np = np.where(g.obj >= 0, oid, -1).astype(np.int32)
    table = [None] * (oid + 1)
    table[oid] = T
    texels = W * H * n * n
    layout = api.rt_texture_info(ctx, oid)["layout"]
    assert layout == api.RT_LAYOUT_QUADS
    limit = _median_tap(table, g, obj_np, filt, layout, W, H, n)  # about half the weighted taps lie past it
    assert 0 < limit < texels
    assert api.rt_checked_limit_extent(ctx, oid, limit) == api.RT_OK
    T2 = _substituted(T, layout, W, H, n, limit)
    table2 = [None] * (oid + 1)
    table2[oid] = T2

    uv, d, o = to_dev(g.uv), to_dev(g.dir), to_dev(obj_np)
    frame = (1, height, width)
    uvb, db, ob = uv.reshape(*frame, 2), d.reshape(*frame, 3), o.reshape(frame)
    dtex = torch.zeros((n, n, H, W, 4), dtype=torch.float32, device=uv.device)
    if path == "fused":
        target = torch.zeros((*frame, 4), dtype=torch.float32, device=uv.device)
        out = torch.empty_like(target)
        api.rt_shade_batched_l2_step(ctx, uvb, db, ob, filt, target, 1.0, out=out, dL_dtex={oid: dtex})
        out = out.reshape(-1, 4)
        gout = out.cpu().numpy().astype(np.float64)  # dL/dout = scale (out - 0)
    else:
        out = api.rt_shade(ctx, uv, d, o, filt) if path == "flat" else \
            api.rt_shade_batched(ctx, uvb, db, ob, filt).reshape(-1, 4)
        gout = np.random.default_rng(5).normal(size=(g.F, 4)).astype(np.float32)
        if path == "flat":
            api.rt_shade_backward(ctx, uv, d, o, filt, to_dev(gout), {oid: dtex})
        else:
            api.rt_shade_batched_backward(ctx, uvb, db, ob, filt, to_dev(gout).reshape(*frame, 4), {oid: dtex})
    assert api.rt_get_error(ctx) == api.RT_ERR_OUT_OF_BOUNDS
    assert api.rt_get_error(ctx) == api.RT_OK  # read and cleared

    # colours: the lookup of the substituted texture
    ref, flags = oracle.shade(table2, g.uv, g.dir, obj_np, filt)
    assert flags == 0
    got = out.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= COLOUR_TOL
    # and some fragments did reach past the limit
    ref_full, _ = oracle.shade(table, g.uv, g.dir, obj_np, filt)
    assert np.sum(np.any(np.abs(ref_full - ref) > 1e-3, axis=1)) > 100

    # texel gradients: redirected to texel 0, nothing written past the limit
    gt, _, _, _ = oracle.shade_backward(table, g.uv, g.dir, obj_np, filt, gout, want_uv=False, want_dir=False)
    gabs, _, _, _ = oracle.shade_backward(table, g.uv, g.dir, obj_np, filt, np.abs(gout), want_uv=False,
                                          want_dir=False)
    G = atlas_to_storage(gt[oid], layout, W, H, n).reshape(-1, 4)
    A = atlas_to_storage(gabs[oid], layout, W, H, n).reshape(-1, 4)
    want = G.copy()
    want[0] += G[limit:].sum(axis=0)
    want[limit:] = 0.0
    tol = 1e-4 * A + 2e-5 * np.abs(gout).max()
    tol[0] += tol[limit:].sum(axis=0)
    got_t = dtex.reshape(-1, 4).cpu().numpy()
    assert np.all(got_t[limit:] == 0.0)
    assert np.all(np.abs(got_t - want) <= tol)
    assert np.abs(G[limit:]).sum() > 0

    # the full extent again: no error, the original colours
    assert api.rt_checked_limit_extent(ctx, oid, texels) == api.RT_OK
    out = api.rt_shade(ctx, uv, d, o, filt)
    assert api.rt_get_error(ctx) == api.RT_OK
    assert np.max(np.abs(out.cpu().numpy() - ref_full)) <= COLOUR_TOL
    api.rt_destroy_texture(ctx, oid)

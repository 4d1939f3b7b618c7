"""GPU parity at the benchmark's full size and launch configuration: the sphere +
ground plane, 1920x1080 x 60 poses (124.4 M fragments), two 1024^2 x 16^2 FP16
textures, quadrilinear, through rt_shade_batched / rt_shade_batched_backward
with the autotuned tile -- exactly what bench.py times.

The oracle cannot shade 124 M fragments in a test, so it checks samples one by
one: 200 000 random fragments plus every fragment of a few 64 x 64 screen tiles.
Properties that hold at any size are checked on the whole step: the texel
gradients of every channel sum to the sum of dL/dout over shaded fragments, and
background fragments get zero colour and zero gradients.  The fused step and
the world-space variant run on the same frames and textures."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import api
from parity_util import COLOUR_TOL, compare_indices, index_taus, storage_index

pytestmark = pytest.mark.gpu

VIEWS, HEIGHT, WIDTH, BUCKETS, N = 60, 1080, 1920, 1024, 16
SCENE_SEED, TEX_SEEDS = 1002, (2001, 2002)


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    dev = torch.device("cuda", 0)
    ctx = api.Context(0)
    textures, oids = [], []
    for seed in TEX_SEEDS:
        atlas = oracle.fill_bucket_lobes(BUCKETS, BUCKETS, N, synth.bucket_lobe_params(seed, BUCKETS, BUCKETS))
        src = torch.from_numpy(atlas).to(dev)
        oids.append(api.rt_create_texture(ctx, BUCKETS, BUCKETS, N, api.RT_F16, api.RT_LAYOUT_ATLAS, src))
        del src
        textures.append(oracle.Texture.from_f32(atlas, BUCKETS, BUCKETS, N, oracle.F16))
        del atlas
    assert oids == [0, 1]
    g = synth.sphere_plane_scene(SCENE_SEED, views=VIEWS, width=WIDTH, height=HEIGHT)
    shape = (VIEWS, HEIGHT, WIDTH)
    uv = torch.from_numpy(g.uv).to(dev).view(*shape, 2)
    d = torch.from_numpy(g.dir).to(dev).view(*shape, 3)
    o = torch.from_numpy(g.obj).to(dev).view(*shape)
    out = torch.empty((*shape, 4), device=dev)
    tile, _ = api.rt_autotune(ctx, uv, d, o, api.RT_QUADRILINEAR, out, reps=2)
    api.rt_shade_batched(ctx, uv, d, o, api.RT_QUADRILINEAR, out)
    assert api.rt_get_error(ctx) == api.RT_OK
    rng = np.random.default_rng(7)
    sel = [rng.choice(g.F, 200000, replace=False)]
    per = HEIGHT * WIDTH
    for view, y0, x0 in ((0, 500, 900), (17, 700, 300), (33, 100, 1700), (59, 1016, 1856)):
        yy, xx = np.meshgrid(np.arange(y0, y0 + 64), np.arange(x0, x0 + 64), indexing="ij")
        sel.append(view * per + (yy * WIDTH + xx).reshape(-1))
    sel = np.unique(np.concatenate(sel))
    yield dict(ctx=ctx, textures=textures, g=g, uv=uv, d=d, o=o, out=out, sel=sel, tile=tile)
    ctx.close()


def test_fullsize_colours_and_indices(full):
    g, sel = full["g"], full["sel"]
    out = full["out"].view(-1, 4)[torch.from_numpy(sel).to(full["out"].device)].cpu().numpy()
    ref, flags = oracle.shade(full["textures"], g.uv[sel], g.dir[sel], g.obj[sel], oracle.QUADRILINEAR)
    assert flags == 0
    assert np.abs(out - ref).max() <= COLOUR_TOL
    # indices of the sample through rt_locate, against the oracle's
    uv = torch.from_numpy(g.uv[sel]).to(full["out"].device)
    d = torch.from_numpy(g.dir[sel]).to(full["out"].device)
    o = torch.from_numpy(g.obj[sel]).to(full["out"].device)
    idx, coord = api.rt_locate(full["ctx"], uv, d, o, api.RT_QUADRILINEAR)
    oi, oc, _ = oracle.locate(full["textures"], g.uv[sel], g.dir[sel], g.obj[sel], oracle.QUADRILINEAR)
    _, band = compare_indices(idx.cpu().numpy(), coord.cpu().numpy().astype(np.float64), oi, oc,
                              index_taus(BUCKETS, BUCKETS, N), mask=g.obj[sel] >= 0)
    assert band <= 0.01 * int((g.obj[sel] >= 0).sum())  # about 0.4 % expected from the band widths
    # background fragments of the whole step are exactly zero
    bg = full["o"] < 0
    assert torch.count_nonzero(full["out"][bg]) == 0


def test_fullsize_backward(full):
    ctx, g, sel = full["ctx"], full["g"], full["sel"]
    uv, d, o, out = full["uv"], full["d"], full["o"], full["out"]
    dev = out.device
    dtex = {k: torch.empty((N, N, BUCKETS, BUCKETS, 4), device=dev) for k in (0, 1)}
    duv = torch.empty_like(uv)
    ddir = torch.empty_like(d)
    api.rt_shade_batched_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, out, dtex, duv, ddir)
    assert api.rt_get_error(ctx) == api.RT_OK
    # sum rule over the whole step: sum over texels == sum of dL/dout (= out) over shaded fragments
    shaded = (o >= 0).unsqueeze(-1)
    for k in (0, 1):
        lhs = dtex[k].double().sum(dim=(0, 1, 2, 3))
        rhs = (out.double() * (o == k).unsqueeze(-1)).sum(dim=(0, 1, 2))
        torch.testing.assert_close(lhs, rhs, rtol=1e-4, atol=1e-3)
    assert torch.count_nonzero(duv * ~shaded) == 0 and torch.count_nonzero(ddir * ~shaded) == 0
    # per-fragment UV and direction gradients of the sample, against the oracle
    gout = out.view(-1, 4)[torch.from_numpy(sel).to(dev)].cpu().numpy().astype(np.float64)
    _, guv, gdir, _ = oracle.shade_backward(full["textures"], g.uv[sel], g.dir[sel], g.obj[sel],
                                            oracle.QUADRILINEAR, gout, want_tex=False)
    got_uv = duv.view(-1, 2)[torch.from_numpy(sel).to(dev)].cpu().numpy()
    got_dir = ddir.view(-1, 3)[torch.from_numpy(sel).to(dev)].cpu().numpy()
    _, oc, _ = oracle.locate(full["textures"], g.uv[sel], g.dir[sel], g.obj[sel], oracle.QUADRILINEAR)
    far = (np.abs(oc - np.round(oc)) > 1e-3).all(axis=1) & (g.obj[sel] >= 0)
    B = oracle.squarify(oracle.equisolid(g.dir[sel].astype(np.float64)))
    far &= (np.abs(np.abs(B) - (1 - 1.0 / N)) > 1e-3).all(axis=1)
    assert far.sum() > 50000
    for got_c, ref_c in ((got_uv, guv), (got_dir, gdir)):
        scale = np.abs(ref_c[far]).max()
        assert np.all(np.abs(got_c[far] - ref_c[far]) <= 1e-3 * np.abs(ref_c[far]) + 1e-5 * scale)


def test_fullsize_texel_gradients_per_texel(full):
    """Texel gradients one by one at the benchmark's size and launch: dL/dout is
    zero except on the sampled fragments (the 200 000 random ones and the four
    screen tiles, minus those whose floors lie inside the FP32/FP64 band), so
    every touched texel's gradient is the sum of w_tap dL/dout over exactly
    those fragments -- the oracle's taps and weights, summed in FP64 -- and
    every other texel stays zero."""
    ctx, g, sel = full["ctx"], full["g"], full["sel"]
    uv, d, o, out = full["uv"], full["d"], full["o"], full["out"]
    dev = out.device
    _, oc, _ = oracle.locate(full["textures"], g.uv[sel], g.dir[sel], g.obj[sel], oracle.QUADRILINEAR)
    near = np.abs(oc - np.round(oc))
    keep = (g.obj[sel] >= 0) & ~((near < index_taus(BUCKETS, BUCKETS, N)) & (near > 0)).any(axis=1)
    fs = sel[keep]
    assert fs.size > 100000
    rng = np.random.default_rng(8)
    gsel = rng.uniform(-1.0, 1.0, (fs.size, 4)).astype(np.float32)
    gout = torch.zeros_like(out).view(-1, 4)
    gout[torch.from_numpy(fs).to(dev)] = torch.from_numpy(gsel).to(dev)
    dtex = {k: torch.empty((N, N, BUCKETS, BUCKETS, 4), device=dev) for k in (0, 1)}
    api.rt_shade_batched_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, gout.view_as(out), dtex)
    assert api.rt_get_error(ctx) == api.RT_OK
    index, weight, flags = oracle.taps(full["textures"], g.uv[fs], g.dir[fs], g.obj[fs], oracle.QUADRILINEAR)
    assert flags == 0
    W = BUCKETS * N
    touched_total = 0
    for k in (0, 1):
        mine = g.obj[fs] == k
        tap = index[mine] >= 0  # -1: no tap
        idx, w = index[mine][tap], weight[mine][tap]
        gk = np.repeat(gsel[mine], 16, axis=0).reshape(-1, 16, 4)[tap]
        keys, inv = np.unique(idx, return_inverse=True)
        ref = np.zeros((keys.size, 4))
        bound = np.zeros(keys.size)
        np.add.at(ref, inv, w[:, None] * gk.astype(np.float64))
        np.add.at(bound, inv, w * np.abs(gk.astype(np.float64)).max(axis=1))
        Y, X = keys // W, keys % W
        flat = storage_index(api.rt_texture_info(ctx, k)["layout"], BUCKETS, BUCKETS, N, X // N, Y // N, X % N,
                             Y % N)
        got = dtex[k].view(-1, 4)[torch.from_numpy(flat).to(dev)].double().cpu().numpy()
        err = np.abs(got - ref)
        tol = 1e-4 * bound[:, None] + 2e-5 * np.abs(gsel).max()
        assert (err <= tol).all(), (f"object {k}: {(err > tol).sum()} texel channels off, worst "
                                    f"{(err - tol).max():.3e}")
        # nothing outside the touched texels
        total = dtex[k].abs().double().sum().item()
        assert abs(total - np.abs(got).sum()) <= 1e-6 * max(total, 1.0)
        touched_total += keys.size
    assert touched_total > 1000000


def test_fullsize_fused_l2_step(full):
    """The benchmark's fused step (forward, L2 loss against a zero target and
    backward in one kernel) at full size: its colours are rt_shade_batched's bit
    for bit, its UV and direction gradients the unfused backward's for the
    same dL/dout, its texel gradients satisfy the sum rule and the loss is the
    sum of squared colours."""
    ctx, uv, d, o, out = full["ctx"], full["uv"], full["d"], full["o"], full["out"]
    dev = out.device
    api.rt_autotune_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, out, None, torch.empty_like(uv), None, 0, reps=1)
    target = torch.zeros_like(out)
    out2 = torch.empty_like(out)
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    dtex = {k: torch.zeros((N, N, BUCKETS, BUCKETS, 4), device=dev) for k in (0, 1)}
    duv, ddir = torch.zeros_like(uv), torch.zeros_like(d)  # RT_ACCUMULATE adds to them
    api.rt_shade_batched_l2_step(ctx, uv, d, o, api.RT_QUADRILINEAR, target, 1.0, out2, sums, dtex, duv, ddir,
                                 api.RT_ACCUMULATE)
    assert api.rt_get_error(ctx) == api.RT_OK
    assert torch.equal(out2, out)
    shaded = (o >= 0).unsqueeze(-1)
    ref_se = (out.double() ** 2 * shaded).sum().item()
    assert abs(sums[0].item() - ref_se) <= 1e-9 * ref_se
    assert sums[1].item() == shaded.sum().item()
    for k in (0, 1):
        lhs = dtex[k].double().sum(dim=(0, 1, 2, 3))
        rhs = (out.double() * (o == k).unsqueeze(-1)).sum(dim=(0, 1, 2))
        torch.testing.assert_close(lhs, rhs, rtol=1e-4, atol=1e-3)
    del dtex
    duv_ref, ddir_ref = torch.empty_like(uv), torch.empty_like(d)
    api.rt_shade_batched_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, out, None, duv_ref, ddir_ref)
    assert torch.equal(duv, duv_ref) and torch.equal(ddir, ddir_ref)


def test_fullsize_world_step(full):
    """The world-space variant as the benchmark's world workload runs it: the same
    frames with its bumpy per-fragment normals (bench.variant_inputs), one
    rt_shade_world_batched and one rt_shade_world_batched_backward (screen
    tiles) over all 124.4 M fragments.
    The sample against the oracle's Eq. 1a lookup (colours, UV, direction and
    normal gradients away from kinks), the texel-gradient sum rule on the whole
    step."""
    import bench

    ctx, g, sel, textures = full["ctx"], full["g"], full["sel"], full["textures"]
    dev = full["out"].device
    uv4, d4, o3 = full["uv"], full["d"], full["o"]
    nrm4 = bench.variant_inputs(None, torch, dev, uv4.view(-1, 2), d4.view(-1, 3), 0, 0).view(d4.shape)
    out4 = api.rt_shade_world_batched(ctx, uv4, d4, nrm4, o3, api.RT_QUADRILINEAR)
    dtex = {k: torch.empty((N, N, BUCKETS, BUCKETS, 4), device=dev) for k in (0, 1)}
    duv4, ddir4, dnrm4 = torch.empty_like(uv4), torch.empty_like(d4), torch.empty_like(d4)
    api.rt_shade_world_batched_backward(ctx, uv4, d4, nrm4, o3, api.RT_QUADRILINEAR, out4, dtex, duv4, ddir4, dnrm4)
    assert api.rt_get_error(ctx) == api.RT_OK
    o, out, nrm = o3.view(-1), out4.view(-1, 4), nrm4.view(-1, 3)
    duv, ddir, dnrm = duv4.view(-1, 2), ddir4.view(-1, 3), dnrm4.view(-1, 3)
    for k in (0, 1):
        lhs = dtex[k].double().sum(dim=(0, 1, 2, 3))
        rhs = (out.double() * (o == k).unsqueeze(-1)).sum(dim=0)
        torch.testing.assert_close(lhs, rhs, rtol=1e-4, atol=1e-3)
    del dtex
    t_sel = torch.from_numpy(sel).to(dev)
    N_sel = nrm[t_sel].cpu().numpy()
    got = out[t_sel].cpu().numpy()
    ref, flags = oracle.shade_world(textures, g.uv[sel], g.dir[sel], N_sel, g.obj[sel], oracle.QUADRILINEAR)
    assert flags == 0
    assert np.abs(got - ref).max() <= COLOUR_TOL
    gout = got.astype(np.float64)
    _, guv, gdir, gnrm, _ = oracle.shade_world_backward(textures, g.uv[sel], g.dir[sel], N_sel, g.obj[sel],
                                                        oracle.QUADRILINEAR, gout, want_tex=False)
    _, oc, _ = oracle.locate_world(textures, g.uv[sel], g.dir[sel], N_sel, g.obj[sel], oracle.QUADRILINEAR)
    far = (np.abs(oc - np.round(oc)) > 1e-3).all(axis=1) & (g.obj[sel] >= 0)
    lo = 1.0 / N - 1.0
    far &= (np.abs(np.abs((oc[:, 2:] + 0.5) * 2 / N - 1) - abs(lo)) > 1e-3).all(axis=1)
    assert far.sum() > 50000
    for got_c, ref_c in ((duv[t_sel].cpu().numpy(), guv), (ddir[t_sel].cpu().numpy(), gdir),
                         (dnrm[t_sel].cpu().numpy(), gnrm)):
        scale = np.abs(ref_c[far]).max()
        assert np.all(np.abs(got_c[far] - ref_c[far]) <= 1e-3 * np.abs(ref_c[far]) + 1e-5 * scale)

"""GPU: differentiation and fitting -- deterministic texel gradients, the loss and
Adam kernels, finite-difference and FP64-oracle checks of the texel gradients,
and a small fit with checkpoint/resume."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import api
from paper_2301_01719_gb300.fit import TextureFit
from parity_util import storage_to_atlas, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    c = api.Context(0)
    yield c
    c.close()


def for_object(o, oid):
    """The quad scene names object 0; point its fragments at `oid`."""
    return torch.where(o >= 0, torch.full_like(o, oid), o)


def small_fit_scene(views=4, size=96, seed=5000):
    g = synth.quad_views(seed, views, size, size)
    lobes = synth.field_lobes(seed + 777)  # the hidden field
    target = np.zeros((g.F, 4), np.float32)
    hit = g.obj >= 0
    target[hit] = synth.eval_field_lobes(lobes, g.uv[hit], g.dir[hit]).astype(np.float32)
    shape = (views, size, size)
    uv = to_dev(g.uv).view(*shape, 2)
    d = to_dev(g.dir).view(*shape, 3)
    o = to_dev(g.obj).view(*shape)
    t = to_dev(target).view(*shape, 4)
    return g, uv, d, o, t


def test_loss_and_adam_kernels_match_torch(ctx):
    dev = torch.device("cuda", 0)
    g = torch.Generator(device="cpu").manual_seed(0)
    F = 10003
    out = torch.rand((F, 4), generator=g).to(dev)
    tgt = torch.rand((F, 4), generator=g).to(dev)
    obj = torch.where(torch.rand(F, generator=g) < 0.3, -1, 0).to(torch.int32).to(dev)
    dL = torch.empty_like(out)
    sums = torch.zeros(2, dtype=torch.float64, device=dev)
    api.rt_l2_loss_grad(out, tgt, obj, 0.25, dL, sums)
    mask = (obj >= 0).unsqueeze(1).float()
    torch.testing.assert_close(dL, 0.25 * (out - tgt) * mask, rtol=1e-6, atol=1e-7)
    ref = (((out - tgt).double() ** 2) * mask.double()).sum()
    assert abs(sums[0].item() - ref.item()) <= 1e-9 * ref.item()
    assert sums[1].item() == mask.sum().item()
    # Adam against the textbook update in plain PyTorch FP32
    p = torch.rand(4096, generator=g).to(dev)
    gr = torch.randn(4096, generator=g).to(dev)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    pr, mr, vr = p.clone(), m.clone(), v.clone()
    for step in (1, 2, 3):
        api.rt_adam_step(p, gr, m, v, 1e-2, 0.9, 0.999, 1e-8, step)
        mr = 0.9 * mr + 0.1 * gr
        vr = 0.999 * vr + 0.001 * gr * gr
        pr = pr - 1e-2 * (mr / (1 - 0.9 ** step)) / (torch.sqrt(vr / (1 - 0.999 ** step)) + 1e-8)
    torch.testing.assert_close(p, pr, rtol=1e-5, atol=1e-6)
    torch.testing.assert_close(m, mr, rtol=1e-6, atol=1e-7)


def test_deterministic_texel_gradients_are_bitwise_reproducible(ctx):
    g, uv, d, o, t = small_fit_scene()
    fit = TextureFit(ctx, 16, 16, 8, init=0.3)
    o = for_object(o, fit.oid)
    fit.tex.uniform_(0, 1)
    out = api.rt_shade_batched(ctx, uv, d, o, api.RT_QUADRILINEAR)
    dL = torch.empty_like(out)
    api.rt_l2_loss_grad(out, t, o, 1.0, dL, None)
    with pytest.raises(api.RadtexError):
        api.rt_shade_batched_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, dL, {fit.oid: fit.grad}, None, None,
                                      api.RT_DETERMINISTIC)
    api.rt_prepare_deterministic(ctx)
    runs = []
    for _ in range(3):
        gr = torch.empty_like(fit.tex)
        api.rt_shade_batched_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, dL, {fit.oid: gr}, None, None,
                                      api.RT_DETERMINISTIC)
        runs.append(gr.cpu().numpy())
    assert np.array_equal(runs[0], runs[1]) and np.array_equal(runs[0], runs[2])
    fast = torch.empty_like(fit.tex)
    api.rt_shade_batched_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, dL, {fit.oid: fast}, None, None, 0)
    scale = np.abs(runs[0]).max()
    assert np.abs(runs[0] - fast.cpu().numpy()).max() <= 1e-5 * scale
    # accumulate in deterministic mode doubles
    acc = torch.from_numpy(runs[0]).to(uv.device)
    api.rt_shade_batched_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, dL, {fit.oid: acc}, None, None,
                                  api.RT_DETERMINISTIC | api.RT_ACCUMULATE)
    assert np.array_equal(acc.cpu().numpy(), 2 * runs[0])
    api.rt_destroy_texture(ctx, fit.oid)


def test_texel_gradients_vs_fd_and_oracle(ctx):
    """1000 sampled texels: central differences (eps 1e-3) of the loss, summed in FP64
    on the device, against the kernel's gradient; all texels against the FP64 oracle."""
    g, uv, d, o, t = small_fit_scene()
    W = H = 16
    n = 8
    fit = TextureFit(ctx, W, H, n)
    o = for_object(o, fit.oid)
    torch.manual_seed(1)
    fit.tex.copy_(torch.rand_like(fit.tex))
    count = fit.shaded_count(o)
    scale = 1.0 / (4.0 * count)
    out = api.rt_shade_batched(ctx, uv, d, o, api.RT_QUADRILINEAR)
    dL = torch.empty_like(out)
    api.rt_l2_loss_grad(out, t, o, scale, dL, None)
    grad = torch.empty_like(fit.tex)
    api.rt_shade_batched_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, dL, {fit.oid: grad}, None, None, 0)
    grad_np = grad.cpu().numpy()
    mask = (o >= 0).unsqueeze(-1).double()

    def loss():
        oo = api.rt_shade_batched(ctx, uv, d, o, api.RT_QUADRILINEAR)
        return (0.5 * scale * ((oo.double() - t.double()) ** 2 * mask).sum()).item()

    flat = fit.tex.view(-1)
    rng = np.random.default_rng(2)
    touched = np.flatnonzero(np.abs(grad_np.reshape(-1)) > 0)
    sel = rng.choice(touched, size=min(1000, touched.size), replace=False)
    eps = 1e-3
    fd = np.empty(len(sel))
    for k, e in enumerate(sel):
        v0 = flat[e].item()
        flat[e] = v0 + eps
        lp = loss()
        flat[e] = v0 - eps
        lm = loss()
        flat[e] = v0
        fd[k] = (lp - lm) / (2 * eps)
    ana = grad_np.reshape(-1)[sel]
    # L is quadratic in the texels: the central difference is exact up to the rounding of the
    # FP32 colours it changes, about (fragments) * scale * |c - t| * 2^-24 / eps ~ 1e-8 here
    assert np.all(np.abs(fd - ana) <= 2e-3 * np.abs(ana) + 2e-8)
    # against the FP64 oracle on the same texels and dL/dout
    atlas = storage_to_atlas(fit.tex.cpu().numpy(), fit.layout, W, H, n)
    T = oracle.Texture(W, H, n, oracle.F64, atlas.astype(np.float64))
    table = [None] * (fit.oid + 1)
    table[fit.oid] = T
    obj_np = o.reshape(-1).cpu().numpy()
    gt, _, _, _ = oracle.shade_backward(table, g.uv, g.dir, obj_np, oracle.QUADRILINEAR,
                                        dL.reshape(-1, 4).cpu().numpy().astype(np.float64), want_uv=False,
                                        want_dir=False)
    got = storage_to_atlas(grad_np, fit.layout, W, H, n)
    assert np.abs(got - gt[fit.oid]).max() <= 1e-4 * np.abs(gt[fit.oid]).max()
    api.rt_destroy_texture(ctx, fit.oid)


def test_fit_converges_and_resumes_bitwise(ctx, tmp_path):
    g, uv, d, o, t = small_fit_scene(views=6, size=128)
    fit = TextureFit(ctx, 16, 16, 8, init=0.0, lr=2e-2, deterministic=True)
    o = for_object(o, fit.oid)
    count = fit.shaded_count(o)
    p0 = TextureFit.psnr(fit.render(uv, d, o), t, o)
    losses = []
    for k in range(40):
        losses.append(float(fit.step(uv, d, o, t, count)))
        if k == 14:
            fit.save(str(tmp_path / "ck.pt"))
            mid_tex = fit.tex.clone()
    p1 = TextureFit.psnr(fit.render(uv, d, o), t, o)
    assert losses[-1] < 0.2 * losses[0]
    assert p1 > p0 + 10.0
    final = fit.tex.clone()
    # resume from the checkpoint in a fresh fitter (own borrowed texture): identical result
    fit2 = TextureFit(ctx, 16, 16, 8, init=0.5, lr=2e-2, deterministic=True)
    o = for_object(o, fit2.oid)
    fit2.load(str(tmp_path / "ck.pt"))
    assert torch.equal(fit2.tex, mid_tex) and fit2.step_count == 15
    for _ in range(25):
        fit2.step(uv, d, o, t, count)
    assert torch.equal(fit2.tex, final)
    # a checkpoint of a different configuration is refused
    fit3 = TextureFit(ctx, 16, 16, 8, lr=1e-3)
    with pytest.raises(ValueError):
        fit3.load(str(tmp_path / "ck.pt"))
    for f in (fit, fit2, fit3):
        api.rt_destroy_texture(ctx, f.oid)


def test_fixed_point_gradients_add_up_over_view_shards(ctx):
    """RT_FIXED_POINT_GRADS: the int64 sums of two view shards (separate calls, as
    two data-parallel ranks would compute them) add up bit for bit to one call
    over all views, and accumulating the second shard into the first's buffer
    gives the same; converted by rt_fixed_to_float they are the deterministic
    mode's FP32 gradient bit for bit."""
    g, uv, d, o, t = small_fit_scene(views=4, size=64)
    fit = TextureFit(ctx, 16, 16, 8, init=0.3)
    o = for_object(o, fit.oid)
    fit.tex.uniform_(0, 1)
    F = lambda: torch.zeros(fit.tex.shape, dtype=torch.int64, device=uv.device)  # noqa: E731
    flags = api.RT_FIXED_POINT_GRADS
    every, half_a, half_b, acc = F(), F(), F(), F()
    api.rt_shade_batched_l2_step(ctx, uv, d, o, api.RT_QUADRILINEAR, t, 0.5, None, None, {fit.oid: every},
                                 flags=flags)
    api.rt_shade_batched_l2_step(ctx, uv[:2], d[:2], o[:2], api.RT_QUADRILINEAR, t[:2], 0.5, None, None,
                                 {fit.oid: half_a}, flags=flags)
    api.rt_shade_batched_l2_step(ctx, uv[2:], d[2:], o[2:], api.RT_QUADRILINEAR, t[2:], 0.5, None, None,
                                 {fit.oid: half_b}, flags=flags)
    api.rt_shade_batched_l2_step(ctx, uv[2:], d[2:], o[2:], api.RT_QUADRILINEAR, t[2:], 0.5, None, None,
                                 {fit.oid: acc}, flags=flags)
    api.rt_shade_batched_l2_step(ctx, uv[:2], d[:2], o[:2], api.RT_QUADRILINEAR, t[:2], 0.5, None, None,
                                 {fit.oid: acc}, flags=flags | api.RT_ACCUMULATE)
    assert int(half_a.abs().sum()) > 0 and int(half_b.abs().sum()) > 0
    assert torch.equal(half_a + half_b, every)
    assert torch.equal(acc, every)
    # the same sums through the separate backward over the same dL/dout
    out = api.rt_shade_batched(ctx, uv, d, o, api.RT_QUADRILINEAR)
    dL = torch.empty_like(out)
    api.rt_l2_loss_grad(out, t, o, 0.5, dL, None)
    sep = F()
    api.rt_shade_batched_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, dL, {fit.oid: sep}, None, None, flags)
    assert int(sep.abs().sum()) > 0
    # converted: the deterministic mode's FP32 gradient of the separate backward, bit for bit
    api.rt_prepare_deterministic(ctx)
    det = torch.empty_like(fit.tex)
    api.rt_shade_batched_backward(ctx, uv, d, o, api.RT_QUADRILINEAR, dL, {fit.oid: det}, None, None,
                                  api.RT_DETERMINISTIC)
    conv = api.rt_fixed_to_float(sep)
    assert torch.equal(conv, det)
    twice = conv.clone()
    api.rt_fixed_to_float(sep, twice, api.RT_ACCUMULATE)
    assert torch.equal(twice, det + det)
    api.rt_destroy_texture(ctx, fit.oid)


def test_deterministic_fit_steps_match_the_fixed_point_reduction(ctx):
    """Deterministic fitting steps (fixed-point texel sums, converted once, then
    Adam) give a bit-identical texture from run to run and move the loss down
    (the loss itself is an FP64 atomic sum, equal to rounding)."""
    g, uv, d, o, t = small_fit_scene(views=4, size=64)
    losses, texs = [], []
    for _ in range(2):
        fit = TextureFit(ctx, 16, 16, 8, init=0.3, deterministic=True)
        oo = for_object(o, fit.oid)
        count = fit.shaded_count(oo)
        ls = [float(fit.step(uv, d, oo, t, count)) for _ in range(5)]
        losses.append(ls)
        texs.append(fit.tex.clone())
        api.rt_destroy_texture(ctx, fit.oid)
    assert torch.equal(texs[0], texs[1])
    np.testing.assert_allclose(losses[0], losses[1], rtol=1e-12)
    assert losses[0][-1] < losses[0][0]


def test_deterministic_fit_gradient_matches_the_fast_one(ctx):
    """The deterministic fit sums w (out - target) in fixed point and applies the
    loss's 1 / (4 count) in the conversion: its texel gradient equals the fast
    one to FP32 summation accuracy.  The same at a loss scale of 1e-9, where each
    scaled contribution w * 1e-9 (out - target) would lie below the fixed point's
    2^-32 resolution if it were summed with the scale."""
    g, uv, d, o, t = small_fit_scene(views=4, size=64)
    grads = []
    for det in (False, True):
        fit = TextureFit(ctx, 16, 16, 8, init=0.3, deterministic=det)
        oo = for_object(o, fit.oid)
        fit.step(uv, d, oo, t, fit.shaded_count(oo))
        torch.cuda.synchronize()
        grads.append(fit.grad.clone())  # the step's gradient (Adam leaves it in place)
        api.rt_destroy_texture(ctx, fit.oid)
    fast, det = grads
    m = float(fast.abs().max())
    err = float((det - fast).abs().max())
    print(f"deterministic vs fast fit gradient: max |diff| {err:.3e}, max |g| {m:.3e}")
    assert m > 0 and err <= 1e-4 * m
    # a loss scale of 1e-9: the unscaled fixed-point sums, scaled in the conversion
    fit = TextureFit(ctx, 16, 16, 8, init=0.3)
    oo = for_object(o, fit.oid)
    tiny = 1e-9
    fast = torch.empty_like(fit.tex)
    api.rt_shade_batched_l2_step(ctx, uv, d, oo, api.RT_QUADRILINEAR, t, tiny, None, None, {fit.oid: fast})
    acc = torch.zeros(fit.tex.shape, dtype=torch.int64, device=uv.device)
    api.rt_shade_batched_l2_step(ctx, uv, d, oo, api.RT_QUADRILINEAR, t, 1.0, None, None, {fit.oid: acc},
                                 flags=api.RT_FIXED_POINT_GRADS)
    det = api.rt_fixed_to_float(acc, scale=tiny)
    m = float(fast.abs().max())
    assert m > 0 and float((det - fast).abs().max()) <= 1e-4 * m
    # summed with the scale, the contributions round away
    coarse = torch.zeros_like(acc)
    api.rt_shade_batched_l2_step(ctx, uv, d, oo, api.RT_QUADRILINEAR, t, tiny, None, None, {fit.oid: coarse},
                                 flags=api.RT_FIXED_POINT_GRADS)
    assert float((api.rt_fixed_to_float(coarse) - fast).abs().max()) > 1e-3 * m
    api.rt_destroy_texture(ctx, fit.oid)

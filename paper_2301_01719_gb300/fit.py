"""Fitting a radiance texture to target renders by gradient descent.

The paper fills radiance textures from ray-traced data (Eq. 4b); this module
fits one to a set of target views instead, which is what the differentiable
lookup is for.  A step is: forward synthesis of every view, the L2 loss and its
gradient and the backward pass into the texel gradients, fused into one launch
(rt_shade_batched_l2_step), then an Adam update (rt_adam_step) -- all in
libradtex's kernels, on the FP32 texture the context borrows (RT_BORROW) in
the layout the library gives owned textures (2 x 2 bucket quads).  Checkpoints
hold the texture, the Adam moments, the step count and a hash of the
configuration; with deterministic=True (fixed-point texel gradients) a run
resumed from a checkpoint is bit-identical to an uninterrupted one.

Data-parallel fitting: with a torch.distributed process group, every rank
holds the whole texture (replicated) and a shard of the target views
(shard_views); after each rank's fused step the texel gradients and the loss
sums are all-reduced (all_reduce_gradients) before the same Adam update runs
on every rank, so the textures stay identical.  The loss is normalised by the
shaded fragments of all ranks.  In the deterministic mode the ranks reduce the
64-bit fixed-point sums (RT_FIXED_POINT_GRADS): integer addition is exact, so
the gradient -- and the whole run -- is bit-identical for any number of ranks
and any split of the views.
"""
from __future__ import annotations

import hashlib
import json

import torch

from . import api


def shard_views(views: int, rank: int, world: int) -> slice:
    """The contiguous block of views rank `rank` of `world` fits: views r V / N to (r + 1) V / N."""
    if not (0 <= rank < world):
        raise ValueError("rank must lie in [0, world)")
    return slice(rank * views // world, (rank + 1) * views // world)


def all_reduce_gradients(grad: torch.Tensor, sums: torch.Tensor | None = None, group=None) -> None:
    """Sums the texel gradient (FP32, or the int64 fixed-point sums of
    RT_FIXED_POINT_GRADS) and the loss sums over the ranks of `group`, in place;
    nothing without an initialised process group of more than one rank."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return
    dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    if sums is not None:
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)


def global_count(count: int, device, group=None) -> int:
    """The shaded fragments of all ranks (the loss normaliser of a data-parallel fit)."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return int(count)
    t = torch.tensor([int(count)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return int(t.item())


class TextureFit:
    def __init__(self, ctx: api.Context, w: int, h: int, n: int, init: float = 0.0, lr: float = 1e-2,
                 betas=(0.9, 0.999), eps: float = 1e-8, filt: int = api.RT_QUADRILINEAR, deterministic: bool = False,
                 group=None):
        dev = torch.device("cuda", ctx.device)
        self.ctx = ctx
        self.group = group  # torch.distributed group of the data-parallel ranks (None: the default, if any)
        self.w, self.h, self.n = int(w), int(h), int(n)
        self.lr, self.betas, self.eps, self.filt = float(lr), tuple(betas), float(eps), int(filt)
        self.deterministic = bool(deterministic)
        # the owned textures' layout: 2 x 2 bucket quads (an odd side padded)
        self.layout = api.RT_LAYOUT_QUADS
        self.tex = torch.full(api.layout_shape(self.layout, w, h, n), float(init), dtype=torch.float32, device=dev)
        self.oid = api.rt_create_texture(ctx, w, h, n, api.RT_F32, self.layout, self.tex, api.RT_BORROW)
        self.grad = torch.zeros_like(self.tex)
        self.m = torch.zeros_like(self.tex)
        self.v = torch.zeros_like(self.tex)
        self.step_count = 0
        self.sums = torch.zeros(2, dtype=torch.float64, device=dev)
        # deterministic mode: the fixed-point texel sums (4 int64 per texel), reduced over ranks as integers
        self.grad_fixed = torch.zeros(self.tex.shape, dtype=torch.int64, device=dev) if self.deterministic else None

    def config(self) -> dict:
        return {"w": self.w, "h": self.h, "n": self.n, "lr": self.lr, "betas": list(self.betas), "eps": self.eps,
                "filter": self.filt, "deterministic": self.deterministic}

    def config_hash(self) -> str:
        return hashlib.sha256(json.dumps(self.config(), sort_keys=True).encode()).hexdigest()[:16]

    def shaded_count(self, obj: torch.Tensor) -> int:
        """Number of fragments with an object (the loss's normaliser), counted by the loss
        kernel, summed over the data-parallel ranks."""
        s = torch.zeros(2, dtype=torch.float64, device=obj.device)
        z = torch.zeros((*obj.shape, 4), dtype=torch.float32, device=obj.device)
        api.rt_l2_loss_grad(z, z, obj, 0.0, None, s)
        return global_count(int(s[1].item()), obj.device, self.group)

    def step(self, uv, dirs, obj, target, count: int, out=None):
        """One fitting step over a batch of views (tensors shaped (V, H, W, k)): this
        rank's shard in a data-parallel fit; the G-buffer's object ids name this
        fitter's texture (self.oid) or background.  count = the shaded fragments of
        all ranks (shaded_count).
        L = 1/(2 * 4 count) sum over shaded fragments and channels of (out - target)^2.
        `out` (optional) receives the rendered colours.  Returns the loss as a device
        tensor (no synchronisation)."""
        self.sums.zero_()
        scale = 1.0 / (4.0 * max(count, 1))
        if self.deterministic:
            # the fixed-point sums are taken of w (out - target), unscaled (resolution 2^-32 against
            # residuals of order one), and the loss's 1 / (4 count) is applied in the conversion
            api.rt_shade_batched_l2_step(self.ctx, uv, dirs, obj, self.filt, target, 1.0, out, self.sums,
                                         {self.oid: self.grad_fixed}, None, None, api.RT_FIXED_POINT_GRADS)
            all_reduce_gradients(self.grad_fixed, self.sums, self.group)
            api.rt_fixed_to_float(self.grad_fixed, self.grad, scale=scale)
        else:
            api.rt_shade_batched_l2_step(self.ctx, uv, dirs, obj, self.filt, target, scale, out, self.sums,
                                         {self.oid: self.grad}, None, None, 0)
            all_reduce_gradients(self.grad, self.sums, self.group)
        self.step_count += 1
        api.rt_adam_step(self.tex, self.grad, self.m, self.v, self.lr, self.betas[0], self.betas[1], self.eps,
                         self.step_count)
        return 0.5 * self.sums[0] * scale

    def render(self, uv, dirs, obj):
        return api.rt_shade_batched(self.ctx, uv, dirs, obj, self.filt)

    @staticmethod
    def psnr(out: torch.Tensor, target: torch.Tensor, obj: torch.Tensor, peak: float = 1.0) -> float:
        mask = (obj >= 0).unsqueeze(-1)
        se = ((out.double() - target.double()) ** 2 * mask).sum().item()
        cnt = 4 * mask.sum().item()
        mse = se / max(cnt, 1)
        return float("inf") if mse == 0 else 10.0 * torch.log10(torch.tensor(peak * peak / mse)).item()

    def state_dict(self) -> dict:
        return {"tex": self.tex.detach().cpu().clone(), "m": self.m.cpu().clone(), "v": self.v.cpu().clone(),
                "step": self.step_count, "config": self.config(), "config_hash": self.config_hash()}

    def save(self, path: str) -> None:
        torch.save(self.state_dict(), path)

    def load(self, path: str) -> None:
        st = torch.load(path, map_location="cpu", weights_only=False)
        if st["config_hash"] != self.config_hash():
            raise ValueError("checkpoint was written by a different fitting configuration")
        # the context keeps reading self.tex in place: copy into it, do not rebind it
        self.tex.copy_(st["tex"])
        self.m.copy_(st["m"])
        self.v.copy_(st["v"])
        self.step_count = int(st["step"])


def main(argv=None):
    """The fitting workload: a w x h x n^2 FP32 texture fitted to `views` target
    renders of the quad from a hidden multi-lobe field; prints one JSON line with
    the step throughput and the PSNR before and after."""
    import argparse
    import time

    import numpy as np

    import synth

    p = argparse.ArgumentParser(description=main.__doc__.split(";")[0])
    p.add_argument("--buckets", type=int, default=512)
    p.add_argument("--n", type=int, default=16)
    p.add_argument("--views", type=int, default=32)
    p.add_argument("--size", type=int, default=1024)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--lr", type=float, default=1e-2)
    p.add_argument("--seed", type=int, default=5005)
    p.add_argument("--deterministic", action="store_true")
    a = p.parse_args(argv)
    import os

    import torch.distributed as dist

    # data-parallel when launched by torchrun: one rank per GPU, views sharded, texture replicated
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    t0 = time.perf_counter()
    g = synth.quad_views(a.seed, a.views, a.size, a.size)
    mine = shard_views(a.views, rank, world)
    per = a.size * a.size
    g = synth.GBuffer(g.uv[mine.start * per:mine.stop * per], g.dir[mine.start * per:mine.stop * per],
                      g.obj[mine.start * per:mine.stop * per], a.size, a.size, mine.stop - mine.start)
    lobes = synth.field_lobes(a.seed + 777)
    target = np.zeros((g.F, 4), np.float32)
    hit = g.obj >= 0
    target[hit] = synth.eval_field_lobes(lobes, g.uv[hit], g.dir[hit]).astype(np.float32)
    shape = (mine.stop - mine.start, a.size, a.size)
    uv = torch.from_numpy(g.uv).to(dev).view(*shape, 2)
    d = torch.from_numpy(g.dir).to(dev).view(*shape, 3)
    o = torch.from_numpy(g.obj).to(dev).view(*shape)
    t = torch.from_numpy(target).to(dev).view(*shape, 4)
    setup_s = time.perf_counter() - t0
    ctx = api.Context(dev.index)
    fit = TextureFit(ctx, a.buckets, a.buckets, a.n, lr=a.lr, deterministic=a.deterministic)
    o = torch.where(o >= 0, torch.full_like(o, fit.oid), o)
    count = fit.shaded_count(o)
    out = torch.empty((*shape, 4), dtype=torch.float32, device=dev)
    psnr0 = TextureFit.psnr(fit.render(uv, d, o), t, o)
    fit.step(uv, d, o, t, count, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps - 1):
        loss = fit.step(uv, d, o, t, count, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(a.steps - 1, 1)
    psnr1 = TextureFit.psnr(fit.render(uv, d, o), t, o)
    F = a.views * per
    if rank == 0:
        print(json.dumps({"workload": f"fit {a.buckets}^2 x {a.n}^2 FP32 texture to {a.views} views of {a.size}^2",
                          "ranks": world, "steps": a.steps, "ms_per_step": ms,
                          "gfrag_per_s_fwd_bwd": F / (ms * 1e-3) / 1e9, "fragments_per_step": F,
                          "shaded_fragments": count, "loss": float(loss), "psnr_start_db_rank0": psnr0,
                          "psnr_end_db_rank0": psnr1, "deterministic": a.deterministic, "setup_s": setup_s}))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Throughput of per-fragment radiance-texture synthesis on GB300.

Workload (default): a unit sphere and a ground plane rendered from 60 orbit
poses at 1920x1080 (124,416,000 fragments per step); each object carries a
radiance texture of 1024 x 1024 buckets x 16 x 16 directions stored as FP16
(2 GiB), filled from one seeded cosine-power lobe per bucket; quadrilinear
filtering.  One step = the forward synthesis of every fragment plus the
backward pass (texel, UV and direction gradients of L = 1/2 sum out^2, texel
gradients zeroed first), all through the C ABI of libradtex.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "radiance lookups/s (Gfrag/s), forward + backward step"
FALLBACK_HBM_GBS = 6800.0
SCENE_SEED = 1002
TEX_SEEDS = (2001, 2002)
NOMINAL_HBM_GBS = 8000.0  # the 8 TB/s that HBM fractions are also quoted against


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["radtex", "reference"], default="radtex")
    p.add_argument("--views", type=int, default=60)
    p.add_argument("--width", type=int, default=1920)
    p.add_argument("--height", type=int, default=1080)
    p.add_argument("--buckets", type=int, default=1024)
    p.add_argument("--n", type=int, default=16)
    p.add_argument("--storage", choices=["f32", "f16", "bf16", "e4m3"], default="f16")
    p.add_argument("--filter", choices=["nearest", "angular_bilinear", "quadrilinear"], default="quadrilinear")
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--e2e-chunk", type=int, default=4, help="views per pipeline chunk of the end-to-end step")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle baseline")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-other-step", "--no-fused-line", dest="no_other_step", action="store_true",
                   help="skip timing the other form of the step (fused or separate) beside the timed one")
    p.add_argument("--no-precision", action="store_true",
                   help="skip the storage formats' error against FP32 storage on the step's frames")
    p.add_argument("--samples", type=int, default=4, help="shadow: light samples per fragment")
    p.add_argument("--separate", action="store_true",
                   help="time the step as three launches (forward, gradient clear, backward) instead of the "
                        "default: the clear and one fused forward + L2 loss (zero target) + backward launch")
    p.add_argument("--fused", action="store_true", help="the fused step (the default)")
    p.add_argument("--deferred", type=int, default=0,
                   help="bake: the deferred payload (albedo + ambient occlusion) over this many AO directions")
    p.add_argument("--workload", choices=["sphere-plane", "voronoi64", "bake", "world", "shadow"],
                   default="sphere-plane",
                   help="voronoi64: 64 objects of uneven sizes, 4 views of 3840x2160, forward in a CUDA graph; "
                        "bake: rt_bake of the sphere-plane workload's two textures")
    p.add_argument("--objects", type=int, default=64)
    p.add_argument("--palette", type=int, default=0,
                   help="sphere-plane: compress each texture to a K-bucket palette (k-means) before timing")
    p.add_argument("--palette-iters", type=int, default=4, help="Lloyd steps of the palette encoder")
    p.add_argument("--palette-fp32", action="store_true",
                   help="palette encoder: assign on the CUDA cores in FP32 instead of the tensor cores")
    p.add_argument("--voronoi-backward", action="store_true",
                   help="voronoi64: time the fused forward + loss + backward launch in the graph (the clear apart)")
    p.add_argument("--mem-fraction", type=float, default=0.7,
                   help="voronoi64: largest share of free device memory the textures may take")
    a = p.parse_args(argv)
    if a.fused and a.separate:
        p.error("--fused and --separate exclude each other")
    a.fused = not a.separate
    return a


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_scene_seed(rank: int) -> int:
    """Every rank renders its own orbit batch of the same size (weak scaling)."""
    return SCENE_SEED + rank


def max_over_ranks(x: float, device=None) -> float:
    """Max of a per-rank scalar (the step time) over all ranks; identity without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(fragments_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput in Gfrag/s: all ranks' fragments over the slowest rank's time."""
    return world * fragments_per_rank / (ms * 1e-3) / 1e9


def workload_name(a) -> str:
    pal = f", palette K={a.palette}" if getattr(a, "palette", 0) else ""
    return (f"sphere+plane {a.width}x{a.height} x {a.views} poses, 2 objects x {a.buckets}^2 buckets x {a.n}^2 "
            f"directions {a.storage.upper()}{pal}, {a.filter}")


def encode_palettes(a, api, ctx, oids, uv, dirs, obj, dev, h_obj):
    """k-means palettes of the dense textures (timed), the palette textures that
    replace them, and the PSNR of their shading against the dense textures' on
    the first pose."""
    import torch

    K = a.palette
    B = a.buckets * a.buckets
    D = a.n * a.n * 4
    new_ids, sse, times = [], [], []
    ref = api.rt_shade(ctx, uv[0].reshape(-1, 2), dirs[0].reshape(-1, 3), obj[0].reshape(-1),
                       api.FILTER_NAMES[a.filter])
    assign_ms = []
    for k, oid in enumerate(oids):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tc = not a.palette_fp32
        C, index, e = api.palette_encode(ctx, oid, K, a.palette_iters, seed=k, tensor_cores=tc)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        sse.append(e)
        scratch = api.TcScratch(api.rt_kmeans_tc_scratch_bytes(a.buckets, a.buckets, a.n, K), dev) if tc else None
        for rep_ in range(2):  # warm, then timed
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            if tc:
                api.rt_kmeans_assign_tc(ctx, oid, K, C, index, scratch=scratch)
            else:
                api.rt_kmeans_assign(ctx, oid, K, C, index)
            s1.record()
            torch.cuda.synchronize()
        assign_ms.append(s0.elapsed_time(s1))
        del scratch
        pid = api.rt_create_palette_texture(ctx, a.buckets, a.buckets, a.n, K, api.FORMAT_NAMES[a.storage],
                                            api.RT_LAYOUT_PLANES, C, index)
        new_ids.append(pid)
    # the palette ids replace the dense ones in the G-buffer (ids 0, 1 -> the new ids)
    remap = torch.full((max(oids) + 1,), -1, dtype=torch.int32, device=dev)
    for o, p in zip(oids, new_ids):
        remap[o] = p
    valid = obj >= 0
    obj.copy_(torch.where(valid, remap[obj.clamp(min=0).long()], obj))
    h_obj.copy_(obj.reshape(-1).cpu())
    for o in oids:
        api.rt_destroy_texture(ctx, o)
    out = api.rt_shade(ctx, uv[0].reshape(-1, 2), dirs[0].reshape(-1, 3), obj[0].reshape(-1),
                       api.FILTER_NAMES[a.filter])
    mse = float(((out - ref) ** 2)[obj[0].reshape(-1) >= 0].mean())
    ms = float(np.mean(assign_ms))
    info = {"K": K, "iterations": a.palette_iters, "encode_s": [round(t, 3) for t in times],
            "sse_first_last": [[x[0], x[-1]] for x in sse],
            "assign_ms": ms, "assign_tflops": 2.0 * B * K * D / (ms * 1e-3) / 1e12,
            "assign_path": "CUDA cores, FP32" if a.palette_fp32 else "tensor cores (tcgen05, FP16 operands, FP32 accumulation; includes the FP16 operand conversion)",
            "texture_bytes": int(sum(api.rt_texture_info(ctx, p)["bytes"] for p in new_ids)),
            "psnr_vs_dense_db": float(10 * np.log10(1.0 / mse)) if mse > 0 else None}
    return info, new_ids


def bytes_per_texel(storage: str) -> int:
    return {"f32": 16, "f16": 8, "bf16": 8, "e4m3": 4}[storage]


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# The sources the forward and backward shading kernels are compiled from.
SHADING_SOURCES = ("backward.cu", "fused.cu", "launch.h", "rt_backward.cuh", "rt_device.cuh", "rt_filter.cuh",
                   "rt_internal.h", "shade.cu")


def _code_only(text: str) -> str:
    """C/C++ source without its comments and with whitespace collapsed: edits to
    comments or layout do not change what the kernels compile to."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2301_01719_gb300", "csrc")
    paths = [os.path.join(csrc, f) for f in SHADING_SOURCES] + [os.path.join(ROOT, "include", "radtex.h")]
    for path in paths:
        with open(path, encoding="utf-8") as fh:
            h.update(os.path.basename(path).encode() + _code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, algorithmic_bytes: float):
    """DRAM bytes per launch of `kernel` at this launch's size, scaled from the committed
    ncu capture of a small case (profiles/traffic.md: DRAM read + write bytes and the
    algorithmic bytes of that launch) by the ratio of the algorithmic bytes -- if the
    capture was taken on the current kernel sources; else (None, None)."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None, None
    src = kernel_source_hash()
    with open(path) as fh:
        for line in fh:
            parts = [x.strip() for x in line.strip().strip("|").split("|")]
            if len(parts) >= 5 and parts[0] == kernel and parts[4] == src:
                try:
                    dram, alg = float(parts[2]), float(parts[3])
                except ValueError:
                    return None, None
                ratio = dram / alg
                return ratio * algorithmic_bytes, (f"ncu DRAM bytes of {parts[1]} ({ratio:.3f} x its algorithmic "
                                                   "bytes), scaled to this launch's algorithmic bytes")
    return None, None


# ---------------------------------------------------------------------------
# Clock sampling during the timed region.
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.5)  # let the sampler start before the timed region
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        import datetime

        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    ts = None
                # keep the samples taken inside the timed region (with a 0.2 s margin)
                if ts is not None and self.t0 is not None and not (self.t0 - 0.2 <= ts <= self.t1 + 0.2):
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle baseline.
# ---------------------------------------------------------------------------

def oracle_textures(a):
    import oracle
    import synth

    fmt = {"f32": oracle.F32, "f16": oracle.F16, "bf16": oracle.BF16, "e4m3": oracle.E4M3}[a.storage]
    texs = []
    for seed in TEX_SEEDS:
        params = synth.bucket_lobe_params(seed, a.buckets, a.buckets)
        atlas = oracle.fill_bucket_lobes(a.buckets, a.buckets, a.n, params)
        texs.append(oracle.Texture.from_f32(atlas, a.buckets, a.buckets, a.n, fmt))
        del atlas
    return texs


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline lines."""
    import subprocess

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample(a, g, seconds: float, texs, filt):
    """A bounded, evenly spread sample of the workload's fragments: every k-th
    fragment of all its poses, k chosen so the oracle's forward over the sample
    takes about `seconds` on all host cores (probed on 1/500 of the fragments)."""
    import oracle

    F = g.obj.shape[0]
    stride = max(1, F // 200000)
    t0 = time.perf_counter()
    oracle.shade(texs, g.uv[::stride], g.dir[::stride], g.obj[::stride], filt)
    rate = g.obj[::stride].shape[0] / max(time.perf_counter() - t0, 1e-6)
    count = int(min(F, max(20000, rate * seconds)))
    stride = max(1, F // count)
    return stride, g.uv[::stride], g.dir[::stride], g.obj[::stride]


def single_thread_rate(texs, uv, d, o, filt, seconds: float = 1.0) -> float:
    """The oracle's forward rate (fragments/s) on one host thread, on a part of the sample."""
    import oracle

    cores = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        k = max(1, o.shape[0] // 4000)
        t0 = time.perf_counter()
        oracle.shade(texs, uv[::k], d[::k], o[::k], filt)
        probe = o[::k].shape[0] / max(time.perf_counter() - t0, 1e-6)
        k = max(1, int(o.shape[0] // max(probe * seconds, 1)))
        t0 = time.perf_counter()
        oracle.shade(texs, uv[::k], d[::k], o[::k], filt)
        return o[::k].shape[0] / max(time.perf_counter() - t0, 1e-9)
    finally:
        oracle.set_num_threads(cores)


BACKWARD_SUBSAMPLE = 10  # the oracle's backward sums texel gradients serially: it runs on a tenth of the sample


def cpu_baseline(a, g, seconds: float):
    """The oracle as it stands, on a bounded sample of the workload's fragments:
    the forward on the sample, the backward on every tenth of its fragments, both
    on all host cores; the step rate combines the two per-fragment times.  The
    forward's rate on one thread is reported beside it."""
    import oracle

    filt = {"nearest": oracle.NEAREST, "angular_bilinear": oracle.ANGULAR_BILINEAR,
            "quadrilinear": oracle.QUADRILINEAR}[a.filter]
    texs = oracle_textures(a)
    F = g.obj.shape[0]
    stride, uv, d, o = oracle_sample(a, g, seconds, texs, filt)
    t0 = time.perf_counter()
    oracle.shade(texs, uv, d, o, filt)
    fwd = o.shape[0] / (time.perf_counter() - t0)
    sub = BACKWARD_SUBSAMPLE
    gout = np.ones((o[::sub].shape[0], 4))
    t0 = time.perf_counter()
    oracle.shade_backward(texs, uv[::sub], d[::sub], o[::sub], filt, gout)
    bwd = o[::sub].shape[0] / max(time.perf_counter() - t0, 1e-9)
    step = 1.0 / (1.0 / fwd + 1.0 / bwd)
    one = single_thread_rate(texs, uv, d, o, filt)
    return {"value": step / 1e9, "unit": "Gfrag/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": ((f"every {stride}th fragment" if stride > 1 else "every fragment") +
                       f" of the {F}-fragment step ({o.shape[0]} forward, every {sub}th of those backward: "
                       f"{o[::sub].shape[0]}), same textures"),
            "fwd_gfrag_s": fwd / 1e9, "bwd_gfrag_s": bwd / 1e9,
            "fwd_gfrag_s_1_thread": one / 1e9, "cpu_model": cpu_model()}


def run_reference(a):
    """--impl reference: the FP64 CPU oracle on host cores, rank 0 only.  Each
    step is the oracle's forward over a bounded sample of the workload (every
    k-th fragment of all its poses) and its backward over every tenth fragment
    of that sample; ms_per_step is the time those two calls took, and the rate
    divides the sample by the time of a forward + backward over all of it (the
    backward's time scaled by ten), reported as ms_per_step_normalised."""
    import synth

    rank, world, _ = dist_info()
    if rank != 0:
        return
    g = synth.sphere_plane_scene(SCENE_SEED, views=a.views, width=a.width, height=a.height)
    import oracle

    filt = {"nearest": oracle.NEAREST, "angular_bilinear": oracle.ANGULAR_BILINEAR,
            "quadrilinear": oracle.QUADRILINEAR}[a.filter]
    texs = oracle_textures(a)
    sub = BACKWARD_SUBSAMPLE
    # about a minute of oracle work over the whole run, between 0.3 and 3 s per step: probe the
    # forward and backward rates, then size the forward's share of a step so that the forward
    # over the sample and the backward over every tenth fragment of it fit the step's time
    per_step = min(3.0, max(0.3, 60.0 / max(a.steps + a.warmup, 1)))
    k = max(1, g.F // 20000)
    t0 = time.perf_counter()
    oracle.shade(texs, g.uv[::k], g.dir[::k], g.obj[::k], filt)
    t_fwd = (time.perf_counter() - t0) / g.obj[::k].shape[0]
    kb = max(1, g.F // 2000)
    t0 = time.perf_counter()
    oracle.shade_backward(texs, g.uv[::kb], g.dir[::kb], g.obj[::kb], filt, np.ones((g.obj[::kb].shape[0], 4)))
    t_bwd = (time.perf_counter() - t0) / g.obj[::kb].shape[0]
    fwd_share = t_fwd / (t_fwd + t_bwd / sub)
    stride, uv, d, o = oracle_sample(a, g, per_step * fwd_share, texs, filt)
    gout = np.ones((o.shape[0], 4))
    run_ms, norm_ms = [], []
    for k in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        oracle.shade(texs, uv, d, o, filt)
        t1 = time.perf_counter()
        oracle.shade_backward(texs, uv[::sub], d[::sub], o[::sub], filt, gout[::sub])
        t2 = time.perf_counter()
        run_ms.append((t2 - t0) * 1e3)
        norm_ms.append(((t1 - t0) + (t2 - t1) * (o.shape[0] / max(o[::sub].shape[0], 1))) * 1e3)
    ms = float(np.mean(run_ms[a.warmup:]))
    ms_norm = float(np.mean(norm_ms[a.warmup:]))
    value = o.shape[0] / (ms_norm * 1e-3) / 1e9
    one = single_thread_rate(texs, uv, d, o, filt)
    config = {"workload": workload_name(a), "fragments_per_step": int(g.F), "views": a.views, "width": a.width,
              "height": a.height, "buckets": a.buckets, "n": a.n, "storage": a.storage, "filter": a.filter,
              "objects": len(texs)}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gfrag/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "ms_per_step_normalised": ms_norm,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": "Gfrag/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": (f"every {stride}th fragment of the {g.F}-fragment step ({o.shape[0]} "
                                        f"forward, every {sub}th of those backward: {o[::sub].shape[0]}); "
                                        "the rate scales the backward's time to the whole sample"),
                             "fwd_gfrag_s_1_thread": one / 1e9, "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "Gfrag/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm.
# ---------------------------------------------------------------------------

def run_radtex(a):
    import torch

    import synth
    from paper_2301_01719_gb300 import api, build

    rank, world, local = dist_info()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device; libradtex has no CPU path")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    fmt = api.FORMAT_NAMES[a.storage]
    filt = api.FILTER_NAMES[a.filter]

    # Scene: every rank renders its own 60-pose orbit (weak scaling), in pinned host memory.
    per = a.width * a.height
    F = a.views * per
    h_uv = torch.empty((F, 2), dtype=torch.float32, pin_memory=True)
    h_dir = torch.empty((F, 3), dtype=torch.float32, pin_memory=True)
    h_obj = torch.empty((F,), dtype=torch.int32, pin_memory=True)
    t0 = time.perf_counter()
    g = synth.sphere_plane_scene(rank_scene_seed(rank), views=a.views, width=a.width, height=a.height,
                                 out=(h_uv.numpy(), h_dir.numpy(), h_obj.numpy()))
    scene_s = time.perf_counter() - t0
    shape = (a.views, a.height, a.width)
    uv = h_uv.to(dev).view(*shape, 2)
    dirs = h_dir.to(dev).view(*shape, 3)
    obj = h_obj.to(dev).view(*shape)

    ctx = api.Context(local)
    oids = []
    for seed in TEX_SEEDS:
        oid = api.rt_create_texture(ctx, a.buckets, a.buckets, a.n, fmt)
        params = torch.from_numpy(synth.bucket_lobe_params(seed, a.buckets, a.buckets)).to(dev)
        api.rt_fill_bucket_lobes(ctx, oid, params)
        oids.append(oid)
    torch.cuda.synchronize()
    palette = None
    if a.palette:
        palette, oids = encode_palettes(a, api, ctx, oids, uv, dirs, obj, dev, h_obj)
    out = torch.empty((*shape, 4), dtype=torch.float32, device=dev)
    duv = torch.empty((*shape, 2), dtype=torch.float32, device=dev)
    ddir = torch.empty((*shape, 3), dtype=torch.float32, device=dev)
    dtex = {o: torch.empty(api.storage_numel(ctx, o), dtype=torch.float32, device=dev) for o in oids}

    # Algorithmic bytes: distinct texels per frame (counted outside the timed region).
    distinct = 0
    for v in range(a.views):
        counts = api.rt_footprint(ctx, uv[v].reshape(-1, 2), dirs[v].reshape(-1, 3), obj[v].reshape(-1), filt,
                                  len(oids))
        distinct += sum(counts)
    tb = bytes_per_texel(a.storage)
    scale_bytes = 0  # E4M3 scales: 4 B per distinct bucket, counted as at most one per texel quad below
    if a.storage == "e4m3":
        scale_bytes = distinct // (a.n * a.n) * 4
    index_bytes = sum(4 * a.buckets * a.buckets for _ in oids) if a.palette else 0  # whole index maps, an upper bound
    fwd_bytes = 40 * F + distinct * tb + scale_bytes + index_bytes
    bwd_bytes = (24 + 16 + 8 + 12) * F + distinct * (tb + 32) + scale_bytes + index_bytes
    # the fused step: G-buffer and target in, colour and UV / direction gradients out, each texel read and its
    # gradient read-modified-written once
    fused_bytes = (24 + 16 + 16 + 8 + 12) * F + distinct * (tb + 32) + scale_bytes + index_bytes
    target = torch.zeros_like(out)  # the fused step's L2 target: dL/dout = out - 0 = out, as the separate step
    sums = torch.zeros(2, dtype=torch.float64, device=dev)

    stream = torch.cuda.current_stream(dev)
    # screen tile of the batched kernels, picked by the library's autotuner on this workload
    tile, tile_ms = api.rt_autotune(ctx, uv, dirs, obj, filt, out, reps=3)
    # and of the backward (the fused step uses it too), timed as the step runs it (the gradients it
    # leaves are cleared by every step)
    api.rt_zero_texture_grads(ctx, dtex)
    btile, btile_ms = api.rt_autotune_backward(ctx, uv, dirs, obj, filt, out, dtex, duv, ddir, api.RT_ACCUMULATE,
                                               reps=2)

    # The two forms of the step, as lists of (part name, launch).  Fused: the clear and one
    # launch doing the forward, dL/dout = out - 0 and the backward.  Separate: the forward, the
    # clear and the backward with dL/dout = out.  Both leave the same colours and gradients.
    fused_parts = [("zero", lambda: api.rt_zero_texture_grads(ctx, dtex)),
                   ("fused", lambda: api.rt_shade_batched_l2_step(ctx, uv, dirs, obj, filt, target, 1.0, out, sums,
                                                                  dtex, duv, ddir, api.RT_ACCUMULATE_TEXELS))]
    separate_parts = [("fwd", lambda: api.rt_shade_batched(ctx, uv, dirs, obj, filt, out)),
                      ("zero", lambda: api.rt_zero_texture_grads(ctx, dtex)),
                      ("bwd", lambda: api.rt_shade_batched_backward(ctx, uv, dirs, obj, filt, out, dtex, duv, ddir,
                                                                    api.RT_ACCUMULATE))]
    main_parts, other_parts = (fused_parts, separate_parts) if a.fused else (separate_parts, fused_parts)

    def run_steps(parts, n, warmup, barrier):
        """warmup untimed steps, then n steps between CUDA events on the launching stream
        (one event before each part and one after the step) with the SM clocks sampled.
        Returns the total ms, the mean ms of each part and the clock summary."""
        for _ in range(warmup):
            for _, fn in parts:
                fn()
        torch.cuda.synchronize()
        st = api.rt_get_error(ctx)
        if st != api.RT_OK:
            raise RuntimeError(f"device status after warm-up: {api.rt_status_string(st)}")
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(parts) + 1)] for _ in range(n)]
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        if barrier and world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            clk.mark_start()
            start.record(stream)
            for k in range(n):
                for i, (_, fn) in enumerate(parts):
                    ev[k][i].record(stream)
                    fn()
                ev[k][-1].record(stream)
            end.record(stream)
            torch.cuda.synchronize()
            clk.mark_end()
        if barrier and world > 1:
            torch.distributed.barrier()
        st = api.rt_get_error(ctx)
        if st != api.RT_OK:
            raise RuntimeError(f"device status after timing: {api.rt_status_string(st)}")
        part_ms = {name: float(np.mean([e[i].elapsed_time(e[i + 1]) for e in ev])) for i, (name, _) in
                   enumerate(parts)}
        return start.elapsed_time(end), part_ms, clk.summary()

    total_ms, part_ms, clocks = run_steps(main_parts, a.steps, a.warmup, barrier=True)
    total_ms = max_over_ranks(total_ms, dev)
    ms_per_step = total_ms / a.steps
    value = whole_job_rate(F, world, ms_per_step)

    # The other form of the step, timed after the main one on the same inputs: reported beside it
    # (and it gives the forward and backward kernels' own times, or the fused kernel's).
    other = None
    if not a.no_other_step:
        o_steps = min(a.steps, 20)
        o_total, o_parts, o_clocks = run_steps(other_parts, o_steps, a.warmup, barrier=False)
        o_ms = max_over_ranks(o_total / o_steps, dev)
        other = {"value": whole_job_rate(F, world, o_ms), "unit": "Gfrag/s", "ms_per_step": o_ms,
                 "steps": o_steps, "part_ms": o_parts, "clocks": o_clocks}
    times = dict(part_ms)
    if other is not None:
        for k, v in other["part_ms"].items():
            times.setdefault(k, v)
    zero_ms = part_ms["zero"]
    fwd_ms, bwd_ms, fused_ms = times.get("fwd"), times.get("bwd"), times.get("fused")

    # End to end through the public API with host buffers: every step copies the
    # G-buffer from pinned host memory and the image back.  The step is pipelined
    # over chunks of views on three streams: the copy of chunk k+1 in, the shading
    # (forward + backward) of chunk k and the copy of chunk k-1 out overlap.
    e2e = None
    if not a.no_e2e:
        h_out = torch.empty((*shape, 4), dtype=torch.float32, pin_memory=True)
        hv_uv, hv_dir, hv_obj = h_uv.view(*shape, 2), h_dir.view(*shape, 3), h_obj.view(*shape)
        d_uv = torch.empty_like(uv)
        d_dir = torch.empty_like(dirs)
        d_obj = torch.empty_like(obj)
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        chunk = max(1, a.e2e_chunk)
        bounds = [(v, min(a.views, v + chunk)) for v in range(0, a.views, chunk)]

        consumed = [None] * len(bounds)  # the last step's kernels are done with chunk j's inputs

        def e2e_step():
            comp = torch.cuda.current_stream(dev)
            api.rt_zero_texture_grads(ctx, dtex)
            for j, (lo, hi) in enumerate(bounds):
                with torch.cuda.stream(s_in):
                    if consumed[j] is not None:
                        s_in.wait_event(consumed[j])  # do not overwrite inputs still being read
                    d_uv[lo:hi].copy_(hv_uv[lo:hi], non_blocking=True)
                    d_dir[lo:hi].copy_(hv_dir[lo:hi], non_blocking=True)
                    d_obj[lo:hi].copy_(hv_obj[lo:hi], non_blocking=True)
                    arrived = torch.cuda.Event()
                    arrived.record(s_in)
                comp.wait_event(arrived)
                if a.fused:
                    api.rt_shade_batched_l2_step(ctx, d_uv[lo:hi], d_dir[lo:hi], d_obj[lo:hi], filt, target[lo:hi],
                                                 1.0, out[lo:hi], sums, dtex, duv[lo:hi], ddir[lo:hi],
                                                 api.RT_ACCUMULATE_TEXELS)
                else:
                    api.rt_shade_batched(ctx, d_uv[lo:hi], d_dir[lo:hi], d_obj[lo:hi], filt, out[lo:hi])
                    api.rt_shade_batched_backward(ctx, d_uv[lo:hi], d_dir[lo:hi], d_obj[lo:hi], filt, out[lo:hi],
                                                  dtex, duv[lo:hi], ddir[lo:hi], api.RT_ACCUMULATE)
                shaded = torch.cuda.Event()
                shaded.record(comp)
                consumed[j] = shaded
                with torch.cuda.stream(s_out):
                    s_out.wait_event(shaded)
                    h_out[lo:hi].copy_(out[lo:hi], non_blocking=True)
            comp.wait_stream(s_out)
            comp.wait_stream(s_in)

        for _ in range(2):  # the first steps also page in the pinned buffers' mappings
            e2e_step()
        torch.cuda.synchronize()
        # each step between its own events: the host link is shared with the machine's other
        # jobs, so the median step is reported (every step's time beside it)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(a.e2e_steps + 1)]
        ev[0].record(stream)
        for k in range(a.e2e_steps):
            e2e_step()
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        steps_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(a.e2e_steps)]
        e_ms = max_over_ranks(float(np.median(steps_ms)), dev)
        e2e = {"value": whole_job_rate(F, world, e_ms), "unit": "Gfrag/s", "ms_per_step": e_ms,
               "ms_per_step_each": [round(t, 3) for t in steps_ms], "statistic": "median step",
               "h2d_bytes_per_step": int(h_uv.nbytes + h_dir.nbytes + h_obj.nbytes),
               "d2h_bytes_per_step": int(h_out.nbytes),
               "pipeline": f"{len(bounds)} chunks of {chunk} views on 3 streams"}
        del h_out

    peak, peak_kind = measured_peak()
    wl = workload_name(a)

    def roof(ms, kernel, nbytes):
        if ms is None:
            return None
        achieved = nbytes / (ms * 1e-3) / 1e9
        traffic, traffic_source = recorded_traffic(kernel, nbytes)
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS,
                "traffic": traffic, "traffic_source": traffic_source, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": int(nbytes), "kernel": kernel}

    r_fwd = roof(fwd_ms, f"shade_kernel<{a.filter}, tiled>", fwd_bytes)
    r_bwd = roof(bwd_ms, f"backward_kernel<{a.filter}, tiled>", bwd_bytes)
    r_fused = roof(fused_ms, f"fused_l2_kernel<{a.filter}, tiled>", fused_bytes)
    # the dominant kernel of the timed step
    dominant = r_fused if a.fused else (r_bwd if bwd_ms >= fwd_ms else r_fwd)
    fused_desc = ("rt_zero_texture_grads + rt_shade_batched_l2_step(target 0, scale 1, RT_ACCUMULATE_TEXELS): "
                  "forward, dL/dout = out, backward in one launch")
    separate_desc = ("rt_shade_batched + rt_zero_texture_grads + rt_shade_batched_backward(RT_ACCUMULATE, "
                     "dL/dout = out)")
    if other is not None:
        other["step"] = separate_desc if a.fused else fused_desc

    def rate(ms):
        return None if ms is None else F / (ms * 1e-3) / 1e9

    result = {
        "metric": METRIC, "value": value, "unit": "Gfrag/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl, "fragments_per_step": F * world, "views": a.views, "width": a.width,
                   "height": a.height, "buckets": a.buckets, "n": a.n, "storage": a.storage, "filter": a.filter,
                   "objects": len(oids), "texture_bytes": int(sum(api.rt_texture_info(ctx, o)["bytes"] for o in oids)),
                   "l2": "inputs larger than L2 (G-buffer %.1f GB, textures %.1f GB per rank)" % (
                       24 * F / 1e9, sum(api.rt_texture_info(ctx, o)["bytes"] for o in oids) / 1e9),
                   "step": fused_desc if a.fused else separate_desc,
                   "tile": {"tw": tile[0], "th": tile[1], "bx": tile[2], "by": tile[3], "autotune_ms": tile_ms},
                   "backward_tile": {"tw": btile[0], "th": btile[1], "bx": btile[2], "by": btile[3],
                                     "autotune_ms": btile_ms},
                   "distinct_texels_per_step": int(distinct), "scene_gen_s": round(scene_s, 2),
                   "palette": palette},
        "fused_ms": fused_ms, "fused_gfrag_s": rate(fused_ms),
        "fwd_ms": fwd_ms, "fwd_gfrag_s": rate(fwd_ms), "bwd_ms": bwd_ms, "bwd_gfrag_s": rate(bwd_ms),
        "zero_grad_ms": zero_ms,
        "part_times": ("kernel times from per-step CUDA events: those of the timed step, the others from "
                       "the other form of the step timed after it (%s)" % ("separate_step" if a.fused else
                                                                        "fused_step")),
        "roofline": dominant, "roofline_fwd": r_fwd, "roofline_bwd": r_bwd, "roofline_fused": r_fused,
        "gpu_launches": (1 if a.fused else 2) * a.steps,
        "clocks": clocks,
        "e2e": e2e,
    }
    if other is not None:
        result["separate_step" if a.fused else "fused_step"] = other
    if not a.no_precision and not a.palette:
        result["precision_vs_fp32"] = precision_vs_fp32(a, api, local, uv, dirs, obj, filt, dev)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(a, g, a.cpu_seconds)
    if rank == 0:
        print(json.dumps(result), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def precision_vs_fp32(a, api, device, uv, dirs, obj, filt, dev, reps=5):
    """The stored formats against FP32 storage of the same lobe fill, shading the
    step's frames (a context of its own): the largest difference of a colour
    channel over the shaded fragments, the PSNR of the colours (peak 1: the lobe
    colours lie in [0, 1]) and each format's forward rate (CUDA events, `reps`
    launches after one warm-up)."""
    import torch

    import synth

    ctx = api.Context(device)
    shaded = (obj >= 0).unsqueeze(-1)
    count = int(shaded.sum()) * 4
    F = obj.numel()
    outs, rows = {}, {}
    for name in ("f32", "f16", "bf16", "e4m3"):
        oids = []
        for seed in TEX_SEEDS:
            oid = api.rt_create_texture(ctx, a.buckets, a.buckets, a.n, api.FORMAT_NAMES[name])
            api.rt_fill_bucket_lobes(ctx, oid, torch.from_numpy(synth.bucket_lobe_params(seed, a.buckets,
                                                                                         a.buckets)).to(dev))
            oids.append(oid)
        o_ids = torch.where(obj >= 0, torch.as_tensor(oids, dtype=torch.int32, device=dev)[obj.clamp(min=0).long()],
                            obj)
        out = api.rt_shade_batched(ctx, uv, dirs, o_ids, filt)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            api.rt_shade_batched(ctx, uv, dirs, o_ids, filt, out)
        e1.record()
        torch.cuda.synchronize()
        if api.rt_get_error(ctx) != api.RT_OK:
            raise RuntimeError("device status set while measuring the storage formats")
        ms = e0.elapsed_time(e1) / reps
        rows[name] = {"fwd_gfrag_s": F / (ms * 1e-3) / 1e9}
        if name == "f32":
            outs["f32"] = out
        else:
            d = torch.where(shaded, out - outs["f32"], torch.zeros_like(out))
            mse = float((d.double() ** 2).sum()) / count
            rows[name].update({"max_abs": float(d.abs().max()),
                               "psnr_db": float(10 * np.log10(1.0 / mse)) if mse > 0 else None})
            del out
        for oid in oids:
            api.rt_destroy_texture(ctx, oid)
    ctx.close()
    return {"frames": f"the step's {a.views} views, every shaded fragment; forward {a.filter}",
            "reference": "the same lobe fill stored in FP32 (the FP64 oracle comparison is in the tests)", **rows}


# ---------------------------------------------------------------------------
# Bake workload: rt_bake of the sphere-plane workload's two textures.
# ---------------------------------------------------------------------------

BAKE_METRIC = "baked texels/s (Gtexel/s), sphere + plane textures"
BAKE_SCENE_SEED = 2001
# FP32 operations per texel of the bake, counted from its formulas (add, mul,
# compare = 1, FMA = 2, each sqrt / divide / pow / exp / cos = 1): Eq. 4a and
# Eq. 2c/4b 21, rotation to world space 15, the traced ray 86 (sphere and plane
# tests 26, sky 24, hit point and its shading 26, fog and blend 10), final
# combination 6.
BAKE_FLOPS_PER_TEXEL = 128
# Deferred payload, counted from its formulas.  Every texel: Eq. 4a/4b 21, world
# rotation 15, first hit with its normal and albedo 45.  A texel whose ray hits
# a surface adds the hit's basis 12, the projections of the test's fixed vector
# on it 15 and the AO divide 1; then per direction, from a plane hit (the sphere
# object's texels) the projected dot product 5 and the sphere test 7, from a
# sphere hit (the plane object's) the dot product 5 and the plane test 3.  Sky
# texels end after the first hit.
DEFERRED_FLOPS_TEXEL, DEFERRED_FLOPS_HIT = 81, 28
DEFERRED_FLOPS_DIR = {"sphere": 12, "plane": 8}
AO_DIRS_SEED = 4242
SMS, FP32_LANES_PER_SM, NOMINAL_SM_MHZ = 152, 128, 2070.0


def bake_name(a) -> str:
    what = f"deferred payload (albedo + AO over {a.deferred} directions)" if a.deferred else "radiance"
    return (f"bake {what}, 2 objects (sphere, plane) x {a.buckets}^2 buckets x {a.n}^2 directions "
            f"{a.storage.upper()}")


def deferred_flops(K: int, hit_fraction: dict) -> float:
    """Formula flops of the deferred payload per texel, averaged over the two
    objects given each object's share of texels whose ray hits a surface."""
    per = [DEFERRED_FLOPS_TEXEL + h * (DEFERRED_FLOPS_HIT + K * DEFERRED_FLOPS_DIR[obj])
           for obj, h in hit_fraction.items()]
    return float(np.mean(per))


def bake_cpu_baseline(a, scene, seconds: float, steps: int | None = None):
    """The oracle's bake on a bounded random sample of texels of both objects."""
    import oracle

    rng = np.random.default_rng(9)
    W = H = a.buckets
    n = a.n

    def sample(k):
        return np.stack([rng.integers(0, W, k), rng.integers(0, H, k), rng.integers(0, n, k),
                         rng.integers(0, n, k)], 1).astype(np.int32)

    if a.deferred:
        import synth

        dirs = synth.ao_directions(AO_DIRS_SEED, a.deferred)

        def bake(surf, q):
            oracle.bake_deferred_texels(W, H, n, surf, scene, dirs, q, None)
    else:
        def bake(surf, q):
            oracle.bake_texels(W, H, n, surf, scene, q, None)

    probe = sample(20000)
    t0 = time.perf_counter()
    bake(oracle.SURFACE_SPHERE, probe)
    rate = probe.shape[0] / max(time.perf_counter() - t0, 1e-6)
    k = int(max(20000, rate * seconds / 2))
    q = sample(k)
    times = []
    for _ in range(steps or 1):
        t0 = time.perf_counter()
        for surf in (oracle.SURFACE_SPHERE, oracle.SURFACE_PLANE):
            bake(surf, q)
        times.append(time.perf_counter() - t0)
    return 2 * k, times, oracle.num_threads()


def run_bake(a):
    import torch

    import synth
    from paper_2301_01719_gb300 import api, build

    rank, world, local = dist_info()
    if a.impl == "reference":
        if rank != 0:
            return
        scene = synth.bake_scene(BAKE_SCENE_SEED)
        count, times, cores = bake_cpu_baseline(a, scene, 2.0, a.warmup + a.steps)
        mean = float(np.mean(times[a.warmup:]))
        value = count / mean / 1e9
        print(json.dumps({
            "impl": "reference", "metric": BAKE_METRIC, "value": value, "unit": "Gtexel/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": bake_name(a), "sample_texels": count},
            "cpu_baseline": {"value": value, "unit": "Gtexel/s", "cores": cores, "kind": "oracle",
                             "sample": f"{count} random texels of the two textures per step"},
            "e2e": {"value": value, "unit": "Gtexel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
            flush=True)
        return
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device; libradtex has no CPU path")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    fmt = api.FORMAT_NAMES[a.storage]
    W = H = a.buckets
    n = a.n
    scene = synth.bake_scene(BAKE_SCENE_SEED + rank)
    ctx = api.Context(local)
    oids = [api.rt_create_texture(ctx, W, H, n, fmt) for _ in range(2)]
    surfaces = (api.RT_SURFACE_SPHERE, api.RT_SURFACE_PLANE)
    stream = torch.cuda.current_stream(dev)
    if a.deferred:
        ao_dirs = torch.from_numpy(synth.ao_directions(AO_DIRS_SEED, a.deferred)).to(dev)

        def bake_one(oid, surf):
            api.rt_bake_deferred(ctx, oid, surf, scene, ao_dirs, stream)
    else:
        def bake_one(oid, surf):
            api.rt_bake(ctx, oid, surf, scene, stream)

    def step():
        for oid, surf in zip(oids, surfaces):
            bake_one(oid, surf)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(a.steps)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        clk.mark_start()
        start.record(stream)
        for k in range(a.steps):
            e = ev[k]
            e[0].record(stream)
            bake_one(oids[0], surfaces[0])
            e[1].record(stream)
            bake_one(oids[1], surfaces[1])
            e[2].record(stream)
        end.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
    if world > 1:
        torch.distributed.barrier()
    st = api.rt_get_error(ctx)
    if st != api.RT_OK:
        raise RuntimeError(f"device status after timing: {api.rt_status_string(st)}")
    ms_per_step = max_over_ranks(start.elapsed_time(end) / a.steps, dev)
    texels = W * H * n * n
    value = 2 * texels * world / (ms_per_step * 1e-3) / 1e9
    sphere_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    plane_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    launch_ms = (sphere_ms + plane_ms) / 2
    clocks = clk.summary()
    sm_max = clocks.get("sm_max_mhz") or NOMINAL_SM_MHZ
    peak_tflops = SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    hit_fraction = None
    if a.deferred:
        # sky texels hold (0, 0, 0, 1) and every hit a positive albedo: count the hits on the device
        hit_fraction = {}
        for name, oid in zip(("sphere", "plane"), oids):
            codes, _ = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_PLANES, stream)
            hit_fraction[name] = float((codes[..., :3] != 0).any(-1).float().mean())
            del codes
        flops_per_texel = deferred_flops(a.deferred, hit_fraction)
    else:
        flops_per_texel = BAKE_FLOPS_PER_TEXEL
    achieved = flops_per_texel * texels / (launch_ms * 1e-3) / 1e12
    tb = bytes_per_texel(a.storage)
    write_gbs = texels * tb / (launch_ms * 1e-3) / 1e9
    hbm_peak, hbm_kind = measured_peak()

    # End to end through the public API: the baked textures are read back to
    # pinned host memory every step (the scene struct is the only input).
    e2e = None
    if not a.no_e2e:
        info = api.rt_texture_info(ctx, oids[0])
        host = [torch.empty((n, n, H, W, 4), dtype=api.CODE_DTYPE[fmt], pin_memory=True) for _ in oids]

        def e2e_step():
            for k, (oid, surf) in enumerate(zip(oids, surfaces)):
                bake_one(oid, surf)
                codes, _ = api.rt_read_texture(ctx, oid, api.RT_LAYOUT_PLANES, stream)
                host[k].copy_(codes, non_blocking=True)
            torch.cuda.current_stream(dev).synchronize()

        e2e_step()
        s0 = time.perf_counter()
        for _ in range(a.e2e_steps):
            e2e_step()
        e_ms = max_over_ranks((time.perf_counter() - s0) * 1e3 / a.e2e_steps, dev)
        e2e = {"value": 2 * texels * world / (e_ms * 1e-3) / 1e9, "unit": "Gtexel/s", "ms_per_step": e_ms,
               "h2d_bytes_per_step": 2 * int(ctypes_sizeof_scene()),
               "d2h_bytes_per_step": int(sum(h.nbytes for h in host)),
               "texture_bytes_per_object": int(info["bytes"])}
        del host

    result = {
        "metric": BAKE_METRIC, "value": value, "unit": "Gtexel/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": bake_name(a), "texels_per_step": 2 * texels * world, "buckets": a.buckets, "n": n,
                   "storage": a.storage, "l2": "outputs larger than L2 (%.1f GB written per step per rank)" % (
                       2 * texels * tb / 1e9)},
        "sphere_ms": sphere_ms, "plane_ms": plane_ms,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": None,
                     "peak_source": f"{SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz",
                     "algorithmic_flops_per_texel": flops_per_texel, "hit_fraction": hit_fraction,
                     "kernel": "bake_kernel",
                     "write_gbs": write_gbs, "write_frac_of_hbm": write_gbs / hbm_peak, "hbm_peak_source": hbm_kind},
        "gpu_launches": 2 * a.steps,
        "clocks": clocks,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        count, times, cores = bake_cpu_baseline(a, scene, a.cpu_seconds)
        result["cpu_baseline"] = {"value": count / times[0] / 1e9, "unit": "Gtexel/s", "cores": cores,
                                  "kind": "oracle", "sample": f"{count} random texels of the two textures"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def ctypes_sizeof_scene() -> int:
    import ctypes

    from paper_2301_01719_gb300 import _lib

    return ctypes.sizeof(_lib.BakeScene)


# ---------------------------------------------------------------------------
# Variant workloads on the sphere-plane G-buffer: world-space lookups with a
# per-fragment normal, and area shadows over 1-bit shadow textures.
# ---------------------------------------------------------------------------

def variant_inputs(a, torch, dev, g_uv, g_dir, samples: int, seed: int):
    """Seeded per-fragment extra inputs made on the device (input synthesis
    only).  World-space workload: unit normals tilted from +z by a smooth
    bump pattern of the surface UV (a normal-mapped surface).  Shadow
    workload: `samples` light directions per fragment, the G-buffer direction
    plus one of `samples` fixed seeded offsets (an area light seen through the
    same sample pattern at every fragment)."""
    F = g_dir.shape[0]
    if samples == 0:
        two_pi = 6.283185307179586
        N = torch.stack([0.3 * torch.sin(two_pi * 8.0 * g_uv[:, 0]), 0.3 * torch.cos(two_pi * 8.0 * g_uv[:, 1]),
                         torch.ones(F, device=dev)], dim=1)
        return (N / N.norm(dim=1, keepdim=True)).contiguous()
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    offsets = 0.1 * torch.randn((1, samples, 3), generator=gen, device=dev)
    L = g_dir[:, None, :] + offsets
    L[..., 2] = L[..., 2].abs()
    return (L / L.norm(dim=2, keepdim=True)).contiguous()


def run_variant(a):
    """--workload world | shadow on the sphere-plane G-buffer (flat fragment stream)."""
    import torch

    import synth
    from paper_2301_01719_gb300 import api, build

    rank, world, local = dist_info()
    if a.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the oracle on the "
                              "default workload; the variant workloads report their oracle baseline inline"}))
        return
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device; libradtex has no CPU path")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    filt = api.FILTER_NAMES[a.filter]
    F = a.views * a.width * a.height
    g = synth.sphere_plane_scene(rank_scene_seed(rank), views=a.views, width=a.width, height=a.height)
    uv = torch.from_numpy(g.uv).to(dev)
    dirs = torch.from_numpy(g.dir).to(dev)
    ctx = api.Context(local)
    oids = []
    shadow = a.workload == "shadow"
    scene = synth.bake_scene(BAKE_SCENE_SEED + rank)
    bake_ms = None
    if shadow:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for surf in (api.RT_SURFACE_SPHERE, api.RT_SURFACE_PLANE):
            oids.append(api.rt_create_texture(ctx, a.buckets, a.buckets, a.n, api.RT_BIT1))
        for _ in range(2):  # warm, then timed
            ev0.record()
            for oid, surf in zip(oids, (api.RT_SURFACE_SPHERE, api.RT_SURFACE_PLANE)):
                api.rt_bake_shadow(ctx, oid, surf, scene)
            ev1.record()
            torch.cuda.synchronize()
        bake_ms = ev0.elapsed_time(ev1)
    else:
        for seed in TEX_SEEDS:
            oid = api.rt_create_texture(ctx, a.buckets, a.buckets, a.n, api.FORMAT_NAMES[a.storage])
            api.rt_fill_bucket_lobes(ctx, oid, torch.from_numpy(synth.bucket_lobe_params(seed, a.buckets,
                                                                                          a.buckets)).to(dev))
            oids.append(oid)
    remap = torch.tensor(oids, dtype=torch.int32, device=dev)
    obj_np = torch.from_numpy(g.obj).to(dev)
    obj = torch.where(obj_np >= 0, remap[obj_np.clamp(min=0).long()], obj_np).contiguous()
    del g
    extra = variant_inputs(a, torch, dev, uv, dirs, a.samples if shadow else 0, 77 + rank)
    out = torch.empty((F, 4), dtype=torch.float32, device=dev)
    duv = torch.empty_like(uv)
    ddir = torch.empty_like(dirs)
    dnrm = torch.empty_like(dirs)
    stream = torch.cuda.current_stream(dev)

    frames = (a.views, a.height, a.width)
    fv = [t.view(*frames, -1) for t in (uv, dirs, extra, out, duv, ddir, dnrm)] if not shadow else None
    o_v = obj.view(*frames)

    def step():
        if shadow:
            api.rt_shade_multi(ctx, uv, extra, obj, filt, out)
        else:  # the screen-tiled world-space calls
            api.rt_shade_world_batched(ctx, fv[0], fv[1], fv[2], o_v, filt, fv[3])
            api.rt_shade_world_batched_backward(ctx, fv[0], fv[1], fv[2], o_v, filt, fv[3], None, fv[4], fv[5],
                                                fv[6])

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        clk.mark_start()
        start.record(stream)
        for _ in range(a.steps):
            step()
        end.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
    st = api.rt_get_error(ctx)
    if st != api.RT_OK:
        raise RuntimeError(f"device status after timing: {api.rt_status_string(st)}")
    ms = max_over_ranks(start.elapsed_time(end) / a.steps, dev)
    value = whole_job_rate(F, world, ms)
    peak, peak_kind = measured_peak()
    if shadow:
        nbytes = F * (8 + 12 * a.samples + 4 + 16)  # uv, S directions, obj, colour; the bits stay in L2
        kernel, metric = "multi_shade_kernel", "area-shadow lookups (Gfrag/s, S light samples per fragment)"
    else:
        nbytes = F * ((8 + 12 + 12 + 4 + 16) + (8 + 12 + 12 + 4 + 16 + 8 + 12 + 12))  # fwd + bwd streams
        kernel = "world_shade_kernel<tiled> + world_backward_kernel<tiled>"
        metric = "world-space lookups (Gfrag/s), fwd + bwd"
    achieved = nbytes / (ms * 1e-3) / 1e9
    result = {
        "metric": metric, "value": value, "unit": "Gfrag/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{a.workload}: sphere+plane {a.width}x{a.height} x {a.views} poses, 2 objects x "
                               f"{a.buckets}^2 x {a.n}^2 " + (f"BIT1, S={a.samples}" if shadow else
                                                             f"{a.storage.upper()}, bumpy normals"),
                   "filter": a.filter, "fragments_per_step": F * world,
                   "l2": "inputs larger than L2 (G-buffer %.1f GB per rank)" % (nbytes / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS,
                     "traffic": None, "peak_source": peak_kind, "algorithmic_bytes_per_step": int(nbytes),
                     "kernel": kernel},
        "gpu_launches": (1 if shadow else 2) * a.steps,
        "clocks": clk.summary(),
        "e2e": None,
    }
    if shadow:
        result["lookups_per_s"] = value * a.samples
        result["shadow_bake_ms"] = bake_ms
        result["shadow_bake_gtexel_s"] = 2 * a.buckets * a.buckets * a.n * a.n / (bake_ms * 1e-3) / 1e9
    if rank == 0:
        print(json.dumps(result), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


VORONOI_SCENE_SEED, VORONOI_SIZE_SEED = 7007, 4004


def voronoi_objects(n_objects: int, seed: int = VORONOI_SIZE_SEED):
    """Bucket-matrix sizes (log-uniform in [128, 2048]) and direction resolutions
    (from {8, 12, 16, 24, 32}) of the many-object workload."""
    rng = np.random.default_rng(seed)
    sizes = np.round(np.exp(rng.uniform(np.log(128.0), np.log(2048.0), n_objects))).astype(np.int64)
    ns = rng.choice(np.array([8, 12, 16, 24, 32]), n_objects)
    return sizes, ns


def run_voronoi(a):
    """Many objects in one launch: --objects textures of seeded uneven sizes, FP16,
    4 views of 3840x2160 whose pixels show the objects in Voronoi regions; the
    forward synthesis of all 33 M fragments is one persistent launch, captured in
    a CUDA graph and replayed.  With --voronoi-backward the graph holds the fused
    forward + L2 loss (zero target) + backward launch instead, adding into FP32
    gradient buffers for every object (the textures shrink to leave room for
    them); the clear of those buffers, dense and far larger than the texels one
    step touches, is timed apart and reported beside it."""
    import torch
    from concurrent.futures import ThreadPoolExecutor

    import synth
    from paper_2301_01719_gb300 import api, build

    rank, world, local = dist_info()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device; libradtex has no CPU path")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    views, height, width = 4, 2160, 3840
    filt = api.FILTER_NAMES[a.filter]
    backward = a.voronoi_backward
    sizes, ns = voronoi_objects(a.objects)
    need = int((sizes ** 2 * ns.astype(np.int64) ** 2 * 8).sum())
    if backward:  # FP16 codes plus an FP32 gradient per texel
        need *= 3
    free, total = torch.cuda.mem_get_info(dev)
    budget = a.mem_fraction * free
    scale = min(1.0, float(np.sqrt(budget / need)))
    if scale < 1.0:  # state the cap: every bucket matrix shrinks by the same factor
        sizes = np.maximum(16, np.floor(sizes * scale)).astype(np.int64)
    t0 = time.perf_counter()
    g = synth.voronoi_planes_scene(VORONOI_SCENE_SEED, a.objects, views=views, width=width, height=height)
    scene_s = time.perf_counter() - t0
    shape = (views, height, width)
    uv = torch.from_numpy(g.uv).to(dev).view(*shape, 2)
    dirs = torch.from_numpy(g.dir).to(dev).view(*shape, 3)
    obj = torch.from_numpy(g.obj).to(dev).view(*shape)
    ctx = api.Context(local)
    oids = [api.rt_create_texture(ctx, int(sz), int(sz), int(n), api.RT_F16) for sz, n in zip(sizes, ns)]
    assert oids == list(range(a.objects))
    t0 = time.perf_counter()
    with ThreadPoolExecutor(8) as ex:
        params = list(ex.map(lambda k: synth.bucket_lobe_params(9000 + k, int(sizes[k]), int(sizes[k])),
                             range(a.objects)))
    for o, p in zip(oids, params):
        api.rt_fill_bucket_lobes(ctx, o, torch.from_numpy(p).to(dev))
    del params
    torch.cuda.synchronize()
    fill_s = time.perf_counter() - t0
    F = views * height * width
    out = torch.empty((*shape, 4), dtype=torch.float32, device=dev)
    distinct = 0
    for v in range(views):
        distinct += sum(api.rt_footprint(ctx, uv[v].reshape(-1, 2), dirs[v].reshape(-1, 3), obj[v].reshape(-1),
                                         filt, a.objects))
    fwd_bytes = 40 * F + distinct * 8
    # the fused step: G-buffer and target in, colour and UV / direction gradients out, each texel
    # read and its gradient read-modified-written once
    step_bytes = (24 + 16 + 16 + 8 + 12) * F + distinct * (8 + 32) if backward else fwd_bytes
    tile, tile_ms = api.rt_autotune(ctx, uv, dirs, obj, filt, out, reps=3)
    btile = None
    if backward:
        dtex = {o: torch.empty(api.storage_numel(ctx, o), dtype=torch.float32, device=dev) for o in oids}
        duv = torch.empty((*shape, 2), dtype=torch.float32, device=dev)
        ddir = torch.empty((*shape, 3), dtype=torch.float32, device=dev)
        target = torch.zeros_like(out)
        sums = torch.zeros(2, dtype=torch.float64, device=dev)
        api.rt_zero_texture_grads(ctx, dtex)
        btile, btile_ms = api.rt_autotune_backward(ctx, uv, dirs, obj, filt, out, dtex, duv, ddir,
                                                   api.RT_ACCUMULATE, reps=2)

    def launch(s):
        if backward:
            api.rt_shade_batched_l2_step(ctx, uv, dirs, obj, filt, target, 1.0, out, sums, dtex, duv, ddir,
                                         api.RT_ACCUMULATE_TEXELS, stream=s)
        else:
            api.rt_shade_batched(ctx, uv, dirs, obj, filt, out, stream=s)

    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        launch(stream)  # warm the launch path
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            launch(stream)
    for _ in range(a.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if api.rt_get_error(ctx) != api.RT_OK:
        raise RuntimeError("device status after warm-up is not RT_OK")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream(dev)
    with ClockSampler(local) as clk:
        clk.mark_start()
        e0.record(cur)
        for _ in range(a.steps):
            graph.replay()
        e1.record(cur)
        torch.cuda.synchronize()
        clk.mark_end()
    ms = e0.elapsed_time(e1) / a.steps
    if api.rt_get_error(ctx) != api.RT_OK:
        raise RuntimeError("device status after timing is not RT_OK")
    clear_ms = None
    if backward:  # the dense clear of every gradient buffer, as a step that clears would run it
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(cur)
        for _ in range(3):
            api.rt_zero_texture_grads(ctx, dtex)
        c1.record(cur)
        torch.cuda.synchronize()
        clear_ms = c0.elapsed_time(c1) / 3
    peak, peak_kind = measured_peak()
    achieved = step_bytes / (ms * 1e-3) / 1e9
    tex_bytes = int(sum(api.rt_texture_info(ctx, o)["bytes"] for o in oids))
    result = {
        "metric": "radiance lookups/s (Gfrag/s), " + ("forward + backward launch" if backward else "forward"),
        "value": F / (ms * 1e-3) / 1e9, "unit": "Gfrag/s",
        "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": (f"voronoi {a.objects} objects (buckets log-uniform 128..2048, n in 8..32, FP16), "
                                f"4 x 3840x2160, {a.filter}, CUDA graph"
                                + (": fused forward, L2 loss, backward (texel gradients added)" if backward else "")),
                   **({"backward_tile": {"tw": btile[0], "th": btile[1], "bx": btile[2], "by": btile[3]},
                       "gradient_bytes": int(sum(t.numel() * 4 for t in dtex.values())),
                       "gradient_clear_ms": clear_ms, "step_with_clear_ms": ms + clear_ms} if backward else {}),
                   "fragments_per_step": F, "objects": a.objects, "texture_bytes": tex_bytes,
                   "texture_bytes_uncapped": need, "bucket_scale_cap": scale,
                   "buckets_min_max": [int(sizes.min()), int(sizes.max())],
                   "l2": "inputs larger than L2 (G-buffer %.2f GB, textures %.1f GB)" % (24 * F / 1e9, tex_bytes / 1e9),
                   "tile": {"tw": tile[0], "th": tile[1], "bx": tile[2], "by": tile[3], "autotune_ms": tile_ms},
                   "distinct_texels_per_step": int(distinct), "scene_gen_s": round(scene_s, 2),
                   "fill_s": round(fill_s, 2), "free_bytes_before": int(free)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "frac_of_nominal_8tbs": achieved / NOMINAL_HBM_GBS,
                     "traffic": None, "peak_source": peak_kind, "algorithmic_bytes_per_launch": int(step_bytes),
                     "kernel": (f"fused_l2_kernel<{a.filter}, tiled>" if backward
                                else f"shade_kernel<{a.filter}, tiled>")},
        "gpu_launches": a.steps, "clocks": clk.summary(), "e2e": None,
    }
    print(json.dumps(result), flush=True)
    del graph
    ctx.close()


def main(argv=None):
    a = parse_args(argv)
    if a.workload == "bake":
        run_bake(a)
    elif a.workload in ("world", "shadow"):
        run_variant(a)
    elif a.impl == "reference":
        run_reference(a)
    elif a.workload == "voronoi64":
        run_voronoi(a)
    else:
        run_radtex(a)


if __name__ == "__main__":
    main()

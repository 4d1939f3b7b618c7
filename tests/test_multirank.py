"""The multi-rank logic of bench.py on CPU: two gloo ranks (one process per rank,
as torchrun launches them).  Fragments are independent, so ranks shard by
rendering their own batches (weak scaling) and exchange only the step time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth

    r, w, local = bench.dist_info()
    t = 10.0 + 5.0 * r  # rank 1 is the slower one
    mx = bench.max_over_ranks(t)
    seed = bench.rank_scene_seed(r)
    g = synth.sphere_plane_scene(seed, views=2, width=64, height=32)
    rate = bench.whole_job_rate(g.F, w, mx)
    # the reference arm runs on rank 0 only; the others return without work
    ref = None
    if r != 0:
        ref = bench.run_reference(bench.parse_args(["--impl", "reference"]))
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, mx, seed, g.F, rate, ref, float(g.uv.sum())))


@pytest.mark.timeout(300)
def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    (r0, w0, l0, mx0, s0, F0, rate0, ref0, sum0), (r1, w1, l1, mx1, s1, F1, rate1, ref1, sum1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert mx0 == mx1 == 15.0  # max over ranks
    assert s0 != s1 and sum0 != sum1  # each rank renders its own batch
    assert F0 == F1  # of the same size
    assert rate0 == pytest.approx(2 * F0 / 15e-3 / 1e9)
    assert ref1 is None


def _dp_worker(rank, world, port, q):
    """One data-parallel fitting rank on CPU: its shard of the views, its texel
    gradient from the FP64 oracle's backward (the test's stand-in for the
    library's fused step), then the product's reduction over the gloo group."""
    import sys

    sys.path.insert(0, ROOT)
    import numpy as np

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    from paper_2301_01719_gb300 import fit

    V, S, W, H, n = 6, 24, 8, 6, 4
    g = synth.quad_views(3003, V, S, S)
    rng = np.random.default_rng(11)
    atlas = rng.uniform(0, 1, (H * n, W * n, 4))
    T = oracle.Texture.from_f32(atlas, W, H, n, oracle.F64)
    target = rng.uniform(0, 1, (g.F, 4))
    sl = fit.shard_views(V, rank, world)
    lo, hi = sl.start * S * S, sl.stop * S * S
    uv, d, o, tg = g.uv[lo:hi], g.dir[lo:hi], g.obj[lo:hi], target[lo:hi]
    count = fit.global_count(int((o >= 0).sum()), "cpu")
    scale = 1.0 / (4.0 * count)
    out, _ = oracle.shade([T], uv, d, o, oracle.QUADRILINEAR)
    gout = np.where((o >= 0)[:, None], scale * (out - tg), 0.0)
    gtex, _, _, _ = oracle.shade_backward([T], uv, d, o, oracle.QUADRILINEAR, gout, want_uv=False, want_dir=False)
    sums = torch.tensor([float((((out - tg) ** 2) * (o >= 0)[:, None]).sum()), float((o >= 0).sum())],
                        dtype=torch.float64)
    g64 = torch.from_numpy(np.ascontiguousarray(gtex[0]))
    fixed = torch.from_numpy(np.rint(gtex[0] * 2.0 ** 32).astype(np.int64))  # this shard's fixed-point sums
    mine_fixed = fixed.clone()
    fit.all_reduce_gradients(g64, sums)
    fit.all_reduce_gradients(fixed)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, (sl.start, sl.stop), count, g64.numpy(), fixed.numpy(), mine_fixed.numpy(), sums.numpy()))


@pytest.mark.timeout(300)
def test_data_parallel_fit_gradients_two_gloo_ranks(orc):
    """Views sharded over two ranks, texture replicated: the all-reduced texel
    gradient equals the single-process gradient over all views (FP64 to rounding;
    the fixed-point sums bit for bit), the shards cover every view once, and the
    loss is normalised by the shaded fragments of both ranks."""
    import numpy as np

    import synth
    from paper_2301_01719_gb300 import fit

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dp_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=240) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    (r0, sl0, c0, g0, f0, m0, s0), (r1, sl1, c1, g1, f1, m1, s1) = res
    assert sl0 == (0, 3) and sl1 == (3, 6)
    V, S, W, H, n = 6, 24, 8, 6, 4
    g = synth.quad_views(3003, V, S, S)
    rng = np.random.default_rng(11)
    atlas = rng.uniform(0, 1, (H * n, W * n, 4))
    T = orc.Texture.from_f32(atlas, W, H, n, orc.F64)
    target = rng.uniform(0, 1, (g.F, 4))
    hit = g.obj >= 0
    assert c0 == c1 == int(hit.sum())  # the global normaliser
    out, _ = orc.shade([T], g.uv, g.dir, g.obj, orc.QUADRILINEAR)
    gout = np.where(hit[:, None], (out - target) / (4.0 * hit.sum()), 0.0)
    full, _, _, _ = orc.shade_backward([T], g.uv, g.dir, g.obj, orc.QUADRILINEAR, gout, want_uv=False, want_dir=False)
    np.testing.assert_array_equal(g0, g1)  # every rank holds the same reduced gradient
    np.testing.assert_allclose(g0, full[0], rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(f0, f1)
    np.testing.assert_array_equal(f0, m0 + m1)  # integer sums: exact, in any order
    assert np.abs(m0).sum() > 0 and np.abs(m1).sum() > 0  # both shards contribute
    np.testing.assert_allclose(s0, [float((((out - target) ** 2) * hit[:, None]).sum()), hit.sum()], rtol=1e-12)
    np.testing.assert_array_equal(s0, s1)
    with pytest.raises(ValueError):
        fit.shard_views(4, 2, 2)
    assert [fit.shard_views(7, r, 3) for r in range(3)] == [slice(0, 2), slice(2, 4), slice(4, 7)]

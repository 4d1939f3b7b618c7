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

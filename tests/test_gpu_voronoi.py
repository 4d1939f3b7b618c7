"""GPU parity of the many-object workload (64 objects in one launch): the
benchmark's 64 seeded objects (bucket matrices of uneven sizes, direction
resolutions from {8, 12, 16, 24, 32}, FP16), the first 3840 x 2160 view of its
Voronoi scene, and the benchmark's launch configuration -- the autotuned tile
and one persistent rt_shade_batched launch captured in a CUDA graph and
replayed.

Every bucket matrix side is a sixteenth of the benchmark's (118 M texels instead
of the benchmark's 207 GB of textures, which the oracle's host copy could not
hold); the fragments, objects, direction resolutions and launch are the
benchmark's.  The oracle checks 100 000 random fragments and every fragment of
two 64 x 64 screen tiles one by one."""
import numpy as np
import pytest
import torch

import bench
import oracle
import synth
from paper_2301_01719_gb300 import api
from parity_util import COLOUR_TOL

pytestmark = pytest.mark.gpu

OBJECTS, WIDTH, HEIGHT = 64, 3840, 2160


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    c = api.Context(0)
    yield c
    c.close()


def test_many_objects_graph_replay_matches_oracle(ctx):
    sizes, ns = bench.voronoi_objects(OBJECTS)
    sizes = np.maximum(8, sizes // 16)
    dev = torch.device("cuda", 0)
    textures, oids = [], []
    for k in range(OBJECTS):
        sz, n = int(sizes[k]), int(ns[k])
        atlas = oracle.fill_bucket_lobes(sz, sz, n, synth.bucket_lobe_params(9000 + k, sz, sz))
        oids.append(api.rt_create_texture(ctx, sz, sz, n, api.RT_F16, api.RT_LAYOUT_ATLAS,
                                          torch.from_numpy(atlas).to(dev)))
        textures.append(oracle.Texture.from_f32(atlas, sz, sz, n, oracle.F16))
        del atlas
    assert oids == list(range(OBJECTS))
    g = synth.voronoi_planes_scene(bench.VORONOI_SCENE_SEED, OBJECTS, views=4, width=WIDTH, height=HEIGHT,
                                   view_range=(0, 1))
    shape = (1, HEIGHT, WIDTH)
    uv = torch.from_numpy(g.uv).to(dev).view(*shape, 2)
    d = torch.from_numpy(g.dir).to(dev).view(*shape, 3)
    o = torch.from_numpy(g.obj).to(dev).view(*shape)
    assert len(np.unique(g.obj)) > OBJECTS // 2  # many objects on screen
    out = torch.empty((*shape, 4), device=dev)
    api.rt_autotune(ctx, uv, d, o, api.RT_QUADRILINEAR, out, reps=2)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        api.rt_shade_batched(ctx, uv, d, o, api.RT_QUADRILINEAR, out, stream=stream)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            api.rt_shade_batched(ctx, uv, d, o, api.RT_QUADRILINEAR, out, stream=stream)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert api.rt_get_error(ctx) == api.RT_OK
    rng = np.random.default_rng(21)
    sel = [rng.choice(g.F, 100000, replace=False)]
    for y0, x0 in ((1000, 1800), (2096, 3776)):
        yy, xx = np.meshgrid(np.arange(y0, y0 + 64), np.arange(x0, x0 + 64), indexing="ij")
        sel.append((yy * WIDTH + xx).reshape(-1))
    sel = np.unique(np.concatenate(sel))
    got = out.view(-1, 4)[torch.from_numpy(sel).to(dev)].cpu().numpy()
    ref, flags = oracle.shade(textures, g.uv[sel], g.dir[sel], g.obj[sel], oracle.QUADRILINEAR)
    assert flags == 0
    assert np.abs(got - ref).max() <= COLOUR_TOL
    for oid in oids:
        api.rt_destroy_texture(ctx, oid)

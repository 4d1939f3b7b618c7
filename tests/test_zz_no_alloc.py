"""rt_footprint_noalloc: the footprint counter for callers that cannot allocate
device memory (their device memory belongs to another allocator or budget, or
a cudaMalloc / cudaFree would stall their frame loop).  Its scratch lives in
static device arrays; here it is called through the C ABI and its counts are
checked against rt_footprint, which allocates, on two calls in a row (the
second smaller than the first, so bits the first call left behind would show).

This file is collected last on purpose: it needs nothing from the other test
files and passes alone in a fresh process as well as after them."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2301_01719_gb300 import _lib, api

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


def _noalloc(ctx, uv, d, o, filt, n_counts):
    """Calls rt_footprint_noalloc through ctypes; the counts buffer starts with junk."""
    counts = torch.full((n_counts,), 987654321, dtype=torch.int64, device=uv.device)
    stream = torch.cuda.current_stream(uv.device).cuda_stream
    rc = _lib.lib().rt_footprint_noalloc(ctx.handle, ctypes.c_void_p(uv.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                         ctypes.c_void_p(o.data_ptr()), o.numel(), filt,
                                         ctypes.c_void_p(counts.data_ptr()), n_counts, ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return rc, counts.cpu().numpy()


def test_noalloc_counts_match_rt_footprint_twice(ctx):
    dev = torch.device("cuda", 0)
    oids = []
    for k, (W, H, n, fmt) in enumerate(((64, 64, 8, api.RT_F16), (48, 40, 6, api.RT_F32))):
        atlas = oracle.fill_field(W, H, n, synth.field_lobes(900 + k))
        oids.append(api.rt_create_texture(ctx, W, H, n, fmt, api.RT_LAYOUT_ATLAS, torch.from_numpy(atlas).to(dev)))
    g = synth.quad_scene(1001)
    rng = np.random.default_rng(0)
    obj_a = np.where(g.obj >= 0, np.array(oids, np.int32)[rng.integers(0, 2, g.F)], -1).astype(np.int32)
    uv = torch.from_numpy(g.uv).to(dev)
    d = torch.from_numpy(g.dir).to(dev)
    hit = np.nonzero(g.obj >= 0)[0][:5000]  # the second call: 5000 fragments that hit the quad
    calls = [(uv, d, torch.from_numpy(obj_a).to(dev), api.RT_QUADRILINEAR),
             (uv[hit].contiguous(), d[hit].contiguous(),
              torch.from_numpy(np.full(len(hit), oids[1], np.int32)).to(dev), api.RT_NEAREST)]
    n_counts = max(oids) + 1
    for k, (u, dd, o, filt) in enumerate(calls):
        ref = api.rt_footprint(ctx, u, dd, o, filt, n_counts)
        rc, got = _noalloc(ctx, u, dd, o, filt, n_counts)
        assert rc == api.RT_OK, api.rt_status_string(rc)
        np.testing.assert_array_equal(got, np.array(ref, dtype=np.int64), err_msg=f"call {k}")
        assert sum(ref) > 0
    assert api.rt_get_error(ctx) == api.RT_OK
    for o in oids:
        api.rt_destroy_texture(ctx, o)


def test_noalloc_rejects_textures_beyond_its_bitmap():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_01719_gb300 import build

    build.build()
    c = api.Context(0)
    try:
        # 1024 x 1024 buckets of 9 x 9 texels: 84.9 M texels > 2^26
        big = api.rt_create_texture(c, 1024, 1024, 9, api.RT_E4M3_BUCKET_SCALE)
        dev = torch.device("cuda", 0)
        uv = torch.full((4, 2), 0.5, device=dev)
        d = torch.tensor([[0.0, 0.0, 1.0]] * 4, device=dev)
        o = torch.full((4,), big, dtype=torch.int32, device=dev)
        rc, _ = _noalloc(c, uv, d, o, api.RT_QUADRILINEAR, big + 1)
        assert rc == api.RT_ERR_INVALID_ARG
    finally:
        c.close()

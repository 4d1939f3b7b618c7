"""CPU checks of the buffer shapes the binding gives each layout (the header's
definitions): atlas (h n, w n, 4), planes (n, n, h, w, 4), quads
(n, n, ceil(h/2), ceil(w/2), 2, 2, 4) holding P n^2 texels, P = 4 ceil(w/2) ceil(h/2)."""
import numpy as np
import pytest

from paper_2301_01719_gb300 import api
from parity_util import atlas_to_quads, quads_to_atlas, storage_index


@pytest.mark.parametrize("w,h,n", [(1, 1, 1), (2, 2, 3), (5, 3, 4), (6, 4, 2), (37, 23, 8), (65536, 2, 1)])
def test_layout_shapes(w, h, n):
    assert api.layout_shape(api.RT_LAYOUT_ATLAS, w, h, n) == (h * n, w * n, 4)
    assert api.layout_shape(api.RT_LAYOUT_PLANES, w, h, n) == (n, n, h, w, 4)
    q = api.layout_shape(api.RT_LAYOUT_QUADS, w, h, n)
    P = 4 * ((w + 1) // 2) * ((h + 1) // 2)
    assert q == (n, n, (h + 1) // 2, (w + 1) // 2, 2, 2, 4)
    assert api.layout_numel(api.RT_LAYOUT_QUADS, w, h, n) == P * n * n * 4
    assert api.layout_numel(api.RT_LAYOUT_PLANES, w, h, n) == w * h * n * n * 4


def test_quads_index_is_the_c_order_of_the_quads_shape():
    """storage_index's formula and the (t, s, j/2, i/2, j%2, i%2) array agree,
    and every texel of an odd-sided texture has its own slot (padding unused)."""
    w, h, n = 5, 3, 2
    a = np.arange(h * n * w * n * 4, dtype=np.float64).reshape(h * n, w * n, 4)
    q = atlas_to_quads(a, w, h, n)
    assert q.shape == api.layout_shape(api.RT_LAYOUT_QUADS, w, h, n)
    flat = q.reshape(-1, 4)
    seen = set()
    for i in range(w):
        for j in range(h):
            for s in range(n):
                for t in range(n):
                    k = int(storage_index(api.RT_LAYOUT_QUADS, w, h, n, i, j, s, t))
                    assert np.array_equal(flat[k], a[j * n + t, i * n + s])
                    seen.add(k)
    assert len(seen) == w * h * n * n
    np.testing.assert_array_equal(quads_to_atlas(q, w, h, n), a)

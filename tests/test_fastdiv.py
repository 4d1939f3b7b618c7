"""The multiply-shift division of the tiled kernels (FastDiv in csrc/rt_filter.cuh),
restated here in exact integer arithmetic: q = (umulhi(n, mul) + n) >> shift with
shift = ceil(log2 d), mul = floor(2^32 (2^shift - d) / d) + 1, exact for n < 2^31."""
import numpy as np


def make(d):
    s = 0
    while (1 << s) < d:
        s += 1
    mul = ((((1 << s) - d) << 32) // d + 1) & 0xFFFFFFFF
    return mul, s


def div(n, d):
    mul, s = make(d)
    hi = (n * mul) >> 32
    return (hi + n) >> s


def test_fastdiv_exhaustive_small():
    for d in range(1, 300):
        for n in list(range(0, 2000)) + [2 ** 31 - 1 - k for k in range(50)]:
            assert div(n, d) == n // d, (n, d)


def test_fastdiv_random():
    rng = np.random.default_rng(0)
    ds = np.concatenate([rng.integers(1, 2 ** 16, 2000), rng.integers(1, 2 ** 31, 2000), 2 ** np.arange(31)])
    for d in ds:
        d = int(d)
        ns = [int(x) for x in rng.integers(0, 2 ** 31, 200)] + [d - 1, d, d + 1, 2 ** 31 - 1, 0]
        for n in ns:
            if 0 <= n < 2 ** 31:
                assert div(n, d) == n // d, (n, d)

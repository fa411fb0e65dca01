"""The kernels' index loops divide flat indices by launch-time sizes with one
high multiply (FastDiv in csrc/common.cuh): q = (n * M) >> 32 with
M = ceil(2^32 / d), exact for n * d < 2^32. These checks restate that
arithmetic on the host and test it against integer division on every divisor
the kernels use (columns per block 1..16, band heights, the transpose's
T2 + 2W - 1 rows, grid lengths 2^k and 3 * 2^k up to 8192) at the dividends
where an error would first appear: the last multiples of d below the bound
and their neighbours. The index loops stay far inside the bound: their
dividends are below C * 8193 + 8 * 512 (column passes), 47 * 4096 (gridding
transpose) and 16 * 8192 (x2 pass)."""
import numpy as np

BOUND = 1 << 32


def magic(d):
    return 0 if d == 1 else ((1 << 32) + d - 1) // d


def fastdiv(n, d):
    return n if d == 1 else (n * magic(d)) >> 32


def divisors():
    ds = set(range(1, 65))                                         # C, T2, T2 + 2W - 1
    for k in range(1, 14):
        ds.add(1 << k)
        ds.add(3 << k)
    return sorted(d for d in ds if d <= 8192)


def test_fastdiv_equals_integer_division_up_to_its_bound():
    rng = np.random.default_rng(0)
    for d in divisors():
        nmax = (BOUND - 1) // d                      # largest n with n d < 2^32
        top = nmax // d * d
        probes = {0, 1, d - 1, d, d + 1, nmax, nmax - 1, top, top - 1, max(top - d, 0)}
        probes |= {int(x) for x in rng.integers(0, nmax + 1, 200)}
        probes |= {m * d + r for m in range(0, 64) for r in (-1, 0, 1)
                   if 0 <= m * d + r <= nmax}
        for n in probes:
            assert fastdiv(n, d) == n // d, (n, d)
            assert n - fastdiv(n, d) * d == n % d


def test_index_loops_stay_inside_the_bound():
    # the largest dividend of each loop times its divisor, at the largest
    # supported sizes (FFT lengths up to 8192, 16 columns per block)
    cases = [(16 * 8193 + 8 * 512, 16),     # column FFT: C * Hf (+ one unrolled batch)
             (16 * 8192 + 8 * 1024, 8192),  # x2 pass: C * M2 (+ one unrolled batch)
             (47 * 4096, 47),               # gridding transpose: (T2 + 2W - 1) * n0
             (32 * 4096, 32)]               # gridding: T2 * n0
    for n, d in cases:
        assert n * d < BOUND

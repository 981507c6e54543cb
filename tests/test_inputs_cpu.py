"""The seeded synthetic inputs shared by the tests, the benchmark and the smoke
check (paper_2101_03055_gb300/inputs.py), on the CPU: the counter-based SplitMix64
generator against the published reference stream, and the uniform and normal
draws built on it."""
import numpy as np

from paper_2101_03055_gb300 import inputs as I


def test_splitmix64_matches_the_published_stream():
    """Seed 0 gives state (k + 1) x 0x9E3779B97F4A7C15 for counter k, i.e. the
    reference SplitMix64 generator started from state 0, whose first outputs are
    0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f."""
    got = [int(v) for v in I.splitmix64(0, [0, 1, 2])]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counters_are_independent_of_the_batch():
    idx = np.arange(1000)
    full = I.splitmix64(5, idx)
    np.testing.assert_array_equal(I.splitmix64(5, idx[500:]), full[500:])
    np.testing.assert_array_equal(I.splitmix64(5, [123]), full[123:124])
    assert not np.array_equal(I.splitmix64(6, idx), full)


def test_uniform_and_normal_draws():
    u = I.uniform(1, np.arange(200_000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    # top 53 bits of the 64-bit output
    np.testing.assert_array_equal(I.uniform(1, [7]), (I.splitmix64(1, [7]) >> np.uint64(11)) * 2.0 ** -53)
    z = I.normal(2, np.arange(100_000))
    assert np.all(np.isfinite(z))
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1.0) < 0.02
    assert abs(np.mean(z ** 3)) < 0.05 and abs(np.mean(z ** 4) - 3.0) < 0.1

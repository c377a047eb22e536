"""The seeded input generator (SplitMix64 quench noise) against a scalar
restatement of the published generator with Python integers."""
import numpy as np

from paper_0710_5912_gb300 import inputs


def splitmix64_scalar(seed, count):
    mask = (1 << 64) - 1
    state = seed & mask
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


def test_vectorised_generator_matches_scalar_definition():
    for seed in (0, 1, 95, 2 ** 63 + 12345):
        assert inputs.splitmix64(seed, 257).tolist() == splitmix64_scalar(seed, 257)


def test_quench_noise_range_and_order():
    phi = inputs.quench_noise(16, 8, seed=7, amp=0.01)
    assert phi.shape == (8, 16)
    assert np.all(np.abs(phi) <= 0.01)
    z = splitmix64_scalar(7, 3)
    # row-major draw order: phi[0, 1] is the second draw
    u1 = (z[1] >> 11) * 2.0 ** -53
    assert phi[0, 1] == 0.01 * (2.0 * u1 - 1.0)
    # mean ~ 0, variance ~ amp^2 / 3 for a large sample
    big = inputs.quench_noise(256, 256, seed=0, amp=1.0)
    assert abs(big.mean()) < 0.01 and abs(big.var() - 1 / 3) < 0.01

"""The seeded input generator (no GPU): the Fourier fields equal their definition
sum_k a_k cos(k.x) + b_k sin(k.x) evaluated point by point, with the coefficients drawn in
half-space order."""
import numpy as np
import pytest

import pr_inputs as pi


@pytest.mark.parametrize("n,kmax,seed", [(6, 2, 3), (8, 3, 5), (7, 4, 11)])
def test_fourier_field_is_its_definition(n, kmax, seed):
    f = pi.fourier_field(n, kmax, seed, 0.1)
    rng = pi.SplitMix64(seed)
    x = pi.grid_1d(n)
    ref = np.zeros((n, n, n))
    for (kx, ky, kz) in pi.half_space_modes(kmax):
        a, b = rng.uniform_pm(0.1), rng.uniform_pm(0.1)
        ph = kz * x[:, None, None] + ky * x[None, :, None] + kx * x[None, None, :]
        ref += a * np.cos(ph) + b * np.sin(ph)
    assert np.max(np.abs(f - ref)) < 1e-14


def test_half_space_holds_one_of_each_pair():
    modes = pi.half_space_modes(3)
    s = set(modes)
    assert len(s) == len(modes)
    for (kx, ky, kz) in modes:
        assert (-kx, -ky, -kz) not in s
    # every non-zero |k| <= 3 vector is a mode or the negative of one
    full = [(a, b, c) for a in range(-3, 4) for b in range(-3, 4) for c in range(-3, 4)
            if 0 < a * a + b * b + c * c <= 9]
    assert len(full) == 2 * len(modes)

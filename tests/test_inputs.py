"""The seeded input generators (CPU): SplitMix64 against its published definition, and the
recipes of the synthetic workloads (ranges, shapes, determinism, structure)."""
import math

import numpy as np
import pytest

from paper_2603_26818_gb300 import inputs

MASK = (1 << 64) - 1


def splitmix64_sequential(seed, count):
    """The generator as published (Steele, Lea, Flood 2014): a 64-bit state advanced by the
    golden-ratio increment, each output the state passed through the variant-13 mixer."""
    state, out = seed & MASK, []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_first_output_of_seed_zero():
    # the value the reference implementation prints first for state 0
    assert int(inputs.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("seed", [0, 1, 4, 12345, (1 << 63) + 5, MASK])
def test_splitmix64_counter_form_equals_the_sequential_generator(seed):
    ref = splitmix64_sequential(seed, 40)
    assert [int(v) for v in inputs.splitmix64(seed, 40)] == ref
    # any slice can be generated on its own
    assert [int(v) for v in inputs.splitmix64(seed, 7, offset=25)] == ref[25:32]


def test_uniform_takes_the_top_53_bits():
    x = splitmix64_sequential(9, 100)
    u = inputs.uniform(9, 100)
    assert np.array_equal(u, np.array([(v >> 11) * 2.0 ** -53 for v in x]))
    assert u.min() >= 0.0 and u.max() < 1.0


def test_uniform_state_recipe():
    a = inputs.uniform_state((64, 32), -0.25, 0.01, seed=1)
    assert a.shape == (64, 32) and a.dtype == np.float64
    assert np.all(np.abs(a + 0.25) <= 0.01)
    assert np.array_equal(a, inputs.uniform_state((64, 32), -0.25, 0.01, seed=1))
    assert not np.array_equal(a, inputs.uniform_state((64, 32), -0.25, 0.01, seed=2))
    # row-major fill from stream element 0
    assert a[0, 1] == pytest.approx(-0.25 + 0.01 * (2.0 * inputs.uniform(1, 2)[1] - 1.0), abs=0)
    # a large sample spans the interval with mean near the centre
    b = inputs.uniform_state((256, 256), -0.35, 0.02, seed=3)
    assert abs(b.mean() + 0.35) < 1e-3 and b.min() < -0.369 and b.max() > -0.331


def test_batch_draws_recipe():
    d = inputs.batch_draws(1024, seed=4)
    assert len(d) == 1024
    assert {ny for ny, _, _, _ in d} == {64, 128, 256, 512}
    assert {nx for _, nx, _, _ in d} == {64, 128, 256, 512}
    assert all(-0.4 <= r <= -0.1 and -0.4 <= m <= -0.2 for _, _, r, m in d)
    assert d == inputs.batch_draws(1024, seed=4)
    # uniform over the sizes: each of the 16 classes holds about 64 domains
    counts = {}
    for ny, nx, _, _ in d:
        counts[(ny, nx)] = counts.get((ny, nx), 0) + 1
    assert len(counts) == 16 and min(counts.values()) > 30 and max(counts.values()) < 100
    pts = sum(ny * nx for ny, nx, _, _ in d)
    assert abs(pts / (1024 * 240.0 ** 2) - 1.0) < 0.1   # E[n] = 240 per axis


def test_polycrystal_recipe():
    ny = nx = 128
    dx = math.pi / 4
    psi = inputs.polycrystal_2d(ny, nx, dx, -0.25, 8, 0.2, 1.0, 0.01, seed=2)
    assert psi.shape == (ny, nx)
    # mean + (0.2 / 3) * (sum of three cosines) + noise: within 0.2 + 0.01 of the mean
    assert np.all(np.abs(psi + 0.25) <= 0.2 + 0.01 + 1e-12)
    assert np.array_equal(psi, inputs.polycrystal_2d(ny, nx, dx, -0.25, 8, 0.2, 1.0, 0.01, seed=2))
    # without noise, one grain (whole box) is the triangular one-mode pattern: its spectrum
    # sits on the ring |k| = q (three +-pairs of modes, smeared by the non-periodic lattice)
    one = inputs.polycrystal_2d(ny, nx, dx, 0.0, 1, 0.2, 1.0, 0.0, seed=5)
    s = np.abs(np.fft.fft2(one)) ** 2
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=dx)
    kx = 2 * np.pi * np.fft.fftfreq(nx, d=dx)
    kk = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
    ring = np.abs(kk - 1.0) < 0.15
    assert s[ring].sum() > 0.9 * s.sum()
    # the noise comes from a second stream (seed + 1)
    diff = inputs.polycrystal_2d(ny, nx, dx, -0.25, 8, 0.2, 1.0, 0.01, seed=2) - \
        inputs.polycrystal_2d(ny, nx, dx, -0.25, 8, 0.2, 1.0, 0.0, seed=2)
    assert np.allclose(diff, inputs.noise(3, (ny, nx), 0.01), atol=1e-15)

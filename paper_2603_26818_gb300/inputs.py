"""Seeded synthetic inputs for PFC runs (shared by the GPU path and the oracle).

This module holds no arithmetic of the method itself: it only draws random numbers and
builds initial fields. Both sides of every parity check receive the same arrays from here.

Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014). It is counter-based: output i of a stream seeded with s is
mix(s + (i + 1) * GAMMA), so any slice can be generated independently and vectorised.
A uniform double in [0, 1) is (x >> 11) * 2^-53.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the SplitMix64 stream seeded with ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform float64 in [0, 1) from the SplitMix64 stream."""
    x = splitmix64(seed, count, offset) >> np.uint64(11)
    return x.astype(np.float64) * (1.0 / 9007199254740992.0)


def noise(seed: int, shape, amplitude: float) -> np.ndarray:
    """Uniform noise in [-amplitude, amplitude] with the given shape (row-major fill)."""
    n = int(np.prod(shape))
    return (amplitude * (2.0 * uniform(seed, n) - 1.0)).reshape(shape)


def uniform_state(shape, mean: float, amp: float, seed: int) -> np.ndarray:
    """psi0 = mean + U[-amp, amp] noise."""
    return mean + noise(seed, shape, amp)


def polycrystal_2d(ny: int, nx: int, dx: float, mean: float, n_grains: int, amplitude: float,
                   q: float, noise_amp: float, seed: int, chunk_rows: int = 64) -> np.ndarray:
    """Periodic Voronoi polycrystal of one-mode triangular grains plus uniform noise.

    Grain g has a centre c_g uniform in the box [0, nx dx) x [0, ny dx) and an orientation
    theta_g uniform in [0, pi/3). Every grid point belongs to the grain whose centre is
    nearest under the minimum-image (periodic) distance, ties to the lower index, and gets
        psi = mean + (amplitude / 3) sum_{j=0..2} cos(q_j . (x - c_g)),
        q_j = q (cos(theta_g + 2 pi j / 3), sin(theta_g + 2 pi j / 3)),
    then U[-noise_amp, noise_amp] noise from a second stream (seed + 1).
    """
    lx, ly = nx * dx, ny * dx
    u = uniform(seed, 3 * n_grains).reshape(n_grains, 3)
    cx, cy, th = u[:, 0] * lx, u[:, 1] * ly, u[:, 2] * (math.pi / 3.0)
    psi = np.empty((ny, nx), dtype=np.float64)
    xs = np.arange(nx, dtype=np.float64) * dx
    for y0 in range(0, ny, chunk_rows):
        y1 = min(ny, y0 + chunk_rows)
        ys = np.arange(y0, y1, dtype=np.float64) * dx
        best = np.full((y1 - y0, nx), np.inf)
        owner = np.zeros((y1 - y0, nx), dtype=np.int64)
        for g in range(n_grains):
            ddx = np.abs(xs - cx[g])
            ddx = np.minimum(ddx, lx - ddx)
            ddy = np.abs(ys - cy[g])
            ddy = np.minimum(ddy, ly - ddy)
            d2 = ddy[:, None] ** 2 + ddx[None, :] ** 2
            closer = d2 < best
            best = np.where(closer, d2, best)
            owner = np.where(closer, g, owner)
        val = np.zeros((y1 - y0, nx))
        gx = xs[None, :] - cx[owner]
        gy = ys[:, None] - cy[owner]
        for j in range(3):
            ang = th[owner] + 2.0 * math.pi * j / 3.0
            val += np.cos(q * (np.cos(ang) * gx + np.sin(ang) * gy))
        psi[y0:y1] = mean + (amplitude / 3.0) * val
    return psi + noise(seed + 1, (ny, nx), noise_amp)


def batch_draws(n_domains: int, seed: int, sizes=(64, 128, 256, 512),
                r_range=(-0.4, -0.1), mean_range=(-0.4, -0.2)):
    """Per-domain (ny, nx, r, mean) for a batched ensemble.

    ny and nx are drawn independently and uniformly from ``sizes``; r and the mean density
    uniformly from their ranges. Stream layout: 4 uniforms per domain in the order
    (ny, nx, r, mean)."""
    u = uniform(seed, 4 * n_domains).reshape(n_domains, 4)
    k = len(sizes)
    out = []
    for d in range(n_domains):
        ny = sizes[min(k - 1, int(u[d, 0] * k))]
        nx = sizes[min(k - 1, int(u[d, 1] * k))]
        r = r_range[0] + (r_range[1] - r_range[0]) * u[d, 2]
        m = mean_range[0] + (mean_range[1] - mean_range[0]) * u[d, 3]
        out.append((ny, nx, float(r), float(m)))
    return out


def apfc_triad(k0: float = 1.0):
    """The three reciprocal vectors of a 2D triangular lattice of wavenumber k0, (x, y)
    components, 120 degrees apart and summing to zero."""
    h = math.sqrt(3.0) / 2.0
    return [(-h * k0, -0.5 * k0), (0.0, k0), (h * k0, -0.5 * k0)]


def apfc_bcc(k0: float = 1.0):
    """The six shortest reciprocal vectors of a BCC lattice of wavenumber k0 (the {110} family,
    one of each +- pair), (x, y, z) components."""
    s = k0 / math.sqrt(2.0)
    return [(s, s, 0.0), (s, 0.0, s), (0.0, s, s), (s, -s, 0.0), (s, 0.0, -s), (0.0, s, -s)]


def apfc_amplitudes(namp: int, shape, amplitude: float, noise_amp: float, seed: int):
    """Complex amplitudes (namp, *shape): amplitude + noise_amp (U[-1, 1] + i U[-1, 1]) per
    point (stream: real parts of every amplitude, then imaginary parts)."""
    n = int(np.prod(shape))
    u = uniform(seed, 2 * namp * n).reshape(2, namp, *shape)
    return (amplitude + noise_amp * (2.0 * u[0] - 1.0)) + 1j * (noise_amp * (2.0 * u[1] - 1.0))

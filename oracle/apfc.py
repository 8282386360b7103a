"""Oracle for the amplitude-expansion PFC step (FP64, CPU, numpy).

TEST INFRASTRUCTURE ONLY: the test suite and ``__graft_entry__.smoke()`` are the only callers.
The GPU library does not import, link or run it.

The paper names the amplitude expansion of the PFC model (its multiphysics section) as a
workload of tens of complex fields but gives no equations; this module takes the expansion of
the PFC energy of Eq. (5) with the conserved dynamics of Eq. (6), written out here:

  psi(r) = psibar + sum_j [eta_j(r) exp(i k_j . r) + c.c.],  j = 1..n, psibar fixed,

with slowly varying complex amplitudes eta_j on a periodic grid and reciprocal-lattice vectors
k_j (any set; a resonance is a sum of +-k that equals some k_j exactly). Projecting
d_t psi = lap[L psi + psi^3] onto exp(i k_j . r): a Fourier mode exp(i q . r) of eta_j is the
mode k_j + q of psi, so lap -> -|k_j + q|^2 and L -> L(|k_j + q|^2) exactly (L is a polynomial in
k^2: the one-mode and two-mode forms of Eq. (5)). The component of psi^3 at k_j is

  N_j = 3 psibar^2 eta_j + 3 psibar sum_{(a,b): k_a + k_b = k_j} e_a e_b
        + sum_{(a,b,c): k_a + k_b + k_c = k_j} e_a e_b e_c,

a, b, c over the signed modes +-1..+-n with e_{+m} = eta_m and e_{-m} = conj(eta_m), the sums
over ordered tuples. The step is the semi-implicit update of Listing 1 applied per amplitude:

  eta_hat_j <- (eta_hat_j - dt Q N_hat_j) / (1 + dt Q L(Q)),   Q = |k_j + q|^2,

with q the grid wavevectors 2 pi m / (n dx) in the FFT order of numpy.fft.fftfreq (the middle
index of an even axis is the negative frequency -n/2). A reading: most amplitude-equation work
replaces Q by |k_j|^2 in the prefactor (non-conserved dynamics); the exact projection is kept
here so that one step of this model is the band of one PFC step around each k_j.

Arrays: eta has shape (n, ny, nx) or (n, nz, ny, nx), complex128, x fastest; kvecs (n, ndim)
with components in the order (x, y[, z]).

Parity status: resonances, nonlinearity, step are pinned (tests/test_oracle_apfc.py): one step
equals the band of one oracle PFC step of the reconstructed density around each k_j; the
closed-form factor of a small plane wave in one amplitude; a uniform single amplitude after one
step in closed form; covariance under translation (eta_j -> eta_j exp(i k_j . u)).
"""
from __future__ import annotations

import itertools

import numpy as np


def resonances(kvecs, rel_tol: float = 1e-9):
    """The quadratic and cubic resonances of each amplitude.

    Returns (pairs, triples): pairs[j] is a list of ((a, b), count) with a <= b signed mode
    indices (+-(m + 1)) such that k_a + k_b = k_j, count the number of ordered pairs it stands
    for; triples[j] likewise for a <= b <= c with k_a + k_b + k_c = k_j."""
    k = np.asarray(kvecs, dtype=np.float64)
    n = k.shape[0]
    scale = max(float(np.max(np.abs(k))), 1.0)
    modes = [m for i in range(1, n + 1) for m in (i, -i)]

    def vec(s):
        return k[abs(s) - 1] * (1.0 if s > 0 else -1.0)

    pairs, triples = [], []
    for j in range(n):
        target = k[j]
        pc, tc = {}, {}
        for a, b in itertools.product(modes, repeat=2):
            if np.max(np.abs(vec(a) + vec(b) - target)) <= rel_tol * scale:
                key = tuple(sorted((a, b)))
                pc[key] = pc.get(key, 0) + 1
        for a, b, c in itertools.product(modes, repeat=3):
            if np.max(np.abs(vec(a) + vec(b) + vec(c) - target)) <= rel_tol * scale:
                key = tuple(sorted((a, b, c)))
                tc[key] = tc.get(key, 0) + 1
        pairs.append(sorted(pc.items()))
        triples.append(sorted(tc.items()))
    return pairs, triples


def _mode(eta, s):
    return eta[s - 1] if s > 0 else np.conj(eta[-s - 1])


def nonlinearity(eta, kvecs, psibar: float):
    """N_j of every amplitude (same shape as eta), evaluated pointwise on the grid."""
    eta = np.asarray(eta, dtype=np.complex128)
    pairs, triples = resonances(kvecs)
    out = np.empty_like(eta)
    for j in range(eta.shape[0]):
        acc = 3.0 * psibar * psibar * eta[j]
        for (a, b), cnt in pairs[j]:
            acc = acc + 3.0 * psibar * cnt * _mode(eta, a) * _mode(eta, b)
        for (a, b, c), cnt in triples[j]:
            acc = acc + cnt * _mode(eta, a) * _mode(eta, b) * _mode(eta, c)
        out[j] = acc
    return out


def lin_symbol(op, k2):
    """L(k) of Eq. (5): r + (1 - k^2)^2, or r + (1 - k^2)^2 (R1 + (q2^2 - k^2)^2)."""
    kind, r, R1, q2 = op
    a = 1.0 - k2
    if int(kind) == 0:
        return r + a * a
    b = q2 * q2 - k2
    return r + a * a * (R1 + b * b)


def shifted_k2(shape, dx: float, kj):
    """|k_j + q|^2 on the FFT grid of an amplitude of the given spatial shape (x last)."""
    nd = len(shape)
    qs = [2.0 * np.pi * np.fft.fftfreq(n, d=dx) for n in shape]   # axis order (z,) y, x
    grids = np.meshgrid(*qs, indexing="ij")
    comp = list(reversed(grids))                                   # x, y[, z]
    return sum((kj[i] + comp[i]) ** 2 for i in range(nd))


def step(eta, kvecs, psibar: float, dx: float, dt: float, op, nsteps: int = 1):
    """eta after nsteps semi-implicit steps (input not modified)."""
    eta = np.array(eta, dtype=np.complex128, copy=True)
    k = np.asarray(kvecs, dtype=np.float64)
    spatial = eta.shape[1:]
    axes = tuple(range(1, eta.ndim))
    Q = np.stack([shifted_k2(spatial, dx, k[j]) for j in range(eta.shape[0])])
    den = 1.0 + dt * Q * lin_symbol(op, Q)
    for _ in range(int(nsteps)):
        eh = np.fft.fftn(eta, axes=axes)
        nh = np.fft.fftn(nonlinearity(eta, k, psibar), axes=axes)
        eh = (eh - dt * Q * nh) / den
        eta = np.fft.ifftn(eh, axes=axes)
    return eta

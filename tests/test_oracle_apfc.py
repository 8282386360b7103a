"""Pins of the amplitude-expansion oracle (oracle/apfc.py) to things other than itself:

* one step of the amplitude model equals, in the band around each k_j, one step of the PFC
  oracle (oracle.step, pinned in test_oracle_pins.py) on the density the amplitudes describe on
  a fine grid (the exact projection the model is defined by; no aliasing on either grid);
* a small plane wave in one amplitude grows by the closed-form factor of the semi-implicit
  scheme at the shifted wavevector k_j + q;
* a uniform single amplitude after one step in closed form (the cubic term 3 |A|^2 A: three
  ordered resonances);
* covariance under a translation u of the density (eta_j -> eta_j exp(i k_j . u));
* the resonance table of a triangular triad.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import apfc
from paper_2603_26818_gb300 import inputs

OP1 = (0, -0.25, 0.0, 0.0)
OP2 = (1, -0.3, 0.05, math.sqrt(4.0 / 3.0))


def test_triad_resonances():
    k = inputs.apfc_triad(1.0)
    pairs, triples = apfc.resonances(k)
    assert pairs[0] == [((-3, -2), 2)]
    t = dict(triples[0])
    assert t[(-1, 1, 1)] == 3           # |eta_1|^2 eta_1
    assert t[(-2, 1, 2)] == 6           # |eta_2|^2 eta_1
    assert t[(-3, 1, 3)] == 6
    assert sum(t.values()) == 3 + 6 + 6


@pytest.mark.parametrize("op,psibar", [(OP1, -0.3), (OP2, 0.1), (OP1, 0.0)])
def test_one_step_is_the_band_of_a_pfc_step(op, psibar):
    """Near-triangular lattice of grid vectors m = (-26,-15), (0,30), (26,-15) on a 256^2 PFC grid
    of box L = 60 pi; amplitudes on 8^2 with Fourier content |m_q| <= 1 per axis (products of
    three stay within |m| <= 3 < 4: no aliasing on the coarse grid; harmonics stay below 128 on
    the fine one)."""
    nf, nc = 256, 8
    m = np.array([(-26, -15), (0, 30), (26, -15)])
    L = 60.0 * math.pi
    dxf, dxc = L / nf, L / nc
    kv = 2.0 * math.pi * m / L
    rng = np.random.default_rng(7)
    eh = np.zeros((3, nc, nc), dtype=np.complex128)
    for j in range(3):
        for iy in (0, 1, nc - 1):
            for ix in (0, 1, nc - 1):
                eh[j, iy, ix] = (rng.uniform(-1, 1) + 1j * rng.uniform(-1, 1)) * 0.04 * nc * nc
    eta = np.fft.ifft2(eh)
    # the density on the fine grid: band of eta_j placed around k_j, conjugate around -k_j
    scale = (nf * nf) / (nc * nc)
    ph = np.zeros((nf, nf), dtype=np.complex128)
    ph[0, 0] += psibar * nf * nf
    qm = [0, 1, -1]
    idx = [0, 1, nc - 1]
    for j in range(3):
        for a, iy in zip(qm, idx):
            for b, ix in zip(qm, idx):
                v = eh[j, iy, ix] * scale
                ph[(m[j, 1] + a) % nf, (m[j, 0] + b) % nf] += v
                ph[(-m[j, 1] - a) % nf, (-m[j, 0] - b) % nf] += np.conj(v)
    psi = np.fft.ifft2(ph)
    assert np.max(np.abs(psi.imag)) < 1e-14
    dt = 0.2
    psi1 = oracle.step(psi.real.copy(), dxf, dt, op, 1)
    ph1 = np.fft.fft2(psi1)
    eta1 = apfc.step(eta, kv, psibar, dxc, dt, op, 1)
    eh1 = np.fft.fft2(eta1, axes=(1, 2))
    for j in range(3):
        expect = np.zeros((nc, nc), dtype=np.complex128)
        for iy in range(nc):
            a = iy if iy < nc // 2 else iy - nc
            for ix in range(nc):
                b = ix if ix < nc // 2 else ix - nc
                expect[iy, ix] = ph1[(m[j, 1] + a) % nf, (m[j, 0] + b) % nf] / scale
        err = np.linalg.norm(eh1[j] - expect) / np.linalg.norm(expect)
        assert err <= 1e-12, (j, err)


@pytest.mark.parametrize("shape,kv,psibar,op,nyq", [
    ((16, 32), inputs.apfc_triad(1.0), -0.25, OP1, False),
    ((16, 32), inputs.apfc_triad(1.0), -0.25, OP1, True),
    ((8, 16, 16), inputs.apfc_bcc(1.0), 0.2, OP2, False)])
def test_small_plane_wave_grows_by_the_closed_form_factor(shape, kv, psibar, op, nyq):
    """nyq: the mode at the middle index of every axis, whose wavevector is the negative
    frequency -pi/dx (numpy.fft.fftfreq order), so the shift k_j + q tells the sign apart."""
    dx, dt, nsteps, delta = 0.9, 0.05, 4, 1e-8
    n = len(kv)
    idx = [s // 2 for s in shape] if nyq else [1] * len(shape)
    grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    phase = sum(2 * math.pi * idx[a] * grids[a] / shape[a] for a in range(len(shape)))
    eta = np.zeros((n,) + shape, dtype=np.complex128)
    eta[0] = delta * np.exp(1j * phase)
    out = apfc.step(eta, kv, psibar, dx, dt, op, nsteps)
    # q of the mode (index 1, or the middle index read as -n/2), components in (x, y[, z]) order
    q = np.array([2 * math.pi * (-(shape[a] // 2) if nyq else 1) / (shape[a] * dx)
                  for a in reversed(range(len(shape)))])
    Q = float(np.sum((np.asarray(kv[0]) + q) ** 2))
    g = (1.0 - dt * Q * 3.0 * psibar ** 2) / (1.0 + dt * Q * apfc.lin_symbol(op, Q))
    # the mode's coefficient (projection; FFT rounding of order 1e-16 delta spreads over the
    # other modes) and the pointwise residual
    coef = np.vdot(eta[0], out[0]) / np.vdot(eta[0], eta[0])
    assert abs(coef - g ** nsteps) <= 1e-12 * abs(g) ** nsteps
    assert np.max(np.abs(out[0] - g ** nsteps * eta[0])) <= 1e-14 * delta
    assert np.max(np.abs(out[1:])) <= 1e-22


def test_uniform_single_amplitude_one_step():
    kv = inputs.apfc_triad(1.0)
    A, psibar, dt = 0.3 - 0.2j, -0.1, 0.25
    eta = np.zeros((3, 4, 4), dtype=np.complex128)
    eta[0] = A
    out = apfc.step(eta, kv, psibar, 1.0, dt, OP1, 1)
    Q = float(np.sum(np.asarray(kv[0]) ** 2))
    N = 3 * psibar ** 2 * A + 3 * abs(A) ** 2 * A
    expect = (A - dt * Q * N) / (1 + dt * Q * apfc.lin_symbol(OP1, Q))
    assert np.max(np.abs(out[0] - expect)) <= 1e-15


@pytest.mark.parametrize("shape,kv", [((16, 16), inputs.apfc_triad(1.0)), ((8, 8, 8), inputs.apfc_bcc(1.0))])
def test_translation_covariance(shape, kv):
    rng = np.random.default_rng(3)
    n = len(kv)
    eta = 0.1 * (rng.standard_normal((n,) + shape) + 1j * rng.standard_normal((n,) + shape))
    u = rng.uniform(-3, 3, size=len(shape))
    ph = np.exp(1j * (np.asarray(kv) @ u))
    a = apfc.step(eta * ph.reshape((n,) + (1,) * len(shape)), kv, -0.2, 0.8, 0.2, OP1, 3)
    b = apfc.step(eta, kv, -0.2, 0.8, 0.2, OP1, 3) * ph.reshape((n,) + (1,) * len(shape))
    assert np.max(np.abs(a - b)) <= 1e-13

"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test targets a plausible mistake: a dropped term, a wrong sign, a wrong wavenumber
index, a transposed axis, a missing 1/N, a wrong Hermitian rule. Nothing here compares the
oracle with itself by retyping its formulas; the expected values come from numpy.fft
(pocketfft, an independent library), brute-force definitions, closed forms of the scheme
and invariants.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2603_26818_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ONE = (oracle.ONE_MODE, -0.25, 0.0, 0.0)
TWO = (oracle.TWO_MODE, -0.3, 0.05, math.sqrt(4.0 / 3.0))


def rng(seed):
    return np.random.default_rng(seed)


def crand(r, n):
    return r.standard_normal(n) + 1j * r.standard_normal(n)


# ----------------------------------------------------------------------------- FFTs

@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 1024])
@pytest.mark.parametrize("sign", [-1, 1])
def test_radix2_matches_numpy(n, sign):
    x = crand(rng(n), n)
    ref = np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * n
    np.testing.assert_allclose(oracle.fft_radix2(x, sign), ref, rtol=0, atol=1e-13 * max(1, n))


@pytest.mark.parametrize("n", [2, 3, 5, 6, 7, 9, 10, 12, 14, 15, 18, 20, 21, 25, 27, 30, 35, 49,
                               50, 60, 75, 98, 100, 11, 13, 22])
@pytest.mark.parametrize("sign", [-1, 1])
def test_mixed_radix_matches_numpy(n, sign):
    x = crand(rng(100 + n), n)
    ref = np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * n
    np.testing.assert_allclose(oracle.fft_mixed(x, sign), ref, rtol=0, atol=1e-13 * n)


@pytest.mark.parametrize("n", [1, 2, 3, 8, 12, 16, 17, 32])
def test_fft_matches_bruteforce_dft(n):
    """Brute force from the definition, written here independently of the oracle's DFT."""
    x = crand(rng(200 + n), n)
    j = np.arange(n)
    ref = np.array([np.sum(x * np.exp(-2j * np.pi * j * k / n)) for k in range(n)])
    np.testing.assert_allclose(oracle.dft(x, -1), ref, atol=1e-12 * n)
    np.testing.assert_allclose(oracle.fft(x, -1), ref, atol=1e-12 * n)


def test_radix2_and_mixed_agree_on_powers_of_two():
    x = crand(rng(7), 256)
    np.testing.assert_allclose(oracle.fft_radix2(x), oracle.fft_mixed(x), atol=1e-11)


@pytest.mark.parametrize("shape", [(16,), (9,), (8, 16), (6, 10), (5, 7), (4, 8, 16), (6, 5, 10),
                                   (3, 3, 9)])
def test_rfftn_matches_numpy(shape):
    a = rng(len(shape) * 31 + shape[-1]).standard_normal(shape)
    np.testing.assert_allclose(oracle.rfftn(a), np.fft.rfftn(a), atol=1e-12 * a.size)


@pytest.mark.parametrize("shape", [(16,), (9,), (8, 16), (6, 10), (5, 7), (4, 8, 16), (6, 5, 10)])
def test_irfftn_matches_numpy_on_arbitrary_half_spectra(shape):
    """numpy drops the imaginary parts of the kx = 0 and Nyquist bins; so must the oracle."""
    hs = tuple(shape[:-1]) + (shape[-1] // 2 + 1,)
    r = rng(shape[-1] * 7 + len(shape))
    h = r.standard_normal(hs) + 1j * r.standard_normal(hs)
    ref = np.fft.irfftn(h, s=shape, axes=tuple(range(len(shape))))
    np.testing.assert_allclose(oracle.irfftn(h, shape), ref, atol=1e-14)


def test_roundtrip_and_parseval():
    a = rng(3).standard_normal((8, 12, 16))
    h = oracle.rfftn(a)
    np.testing.assert_allclose(oracle.irfftn(h, a.shape), a, atol=1e-14)
    w = np.full(h.shape, 2.0)
    w[..., 0] = 1.0
    w[..., -1] = 1.0          # nx even: Nyquist plane counted once
    assert np.sum(w * np.abs(h) ** 2) / a.size == pytest.approx(np.sum(a * a), rel=1e-13)


def test_delta_and_cosine_special_cases():
    d = np.zeros((8, 16))
    d[0, 0] = 1.0
    np.testing.assert_allclose(oracle.rfftn(d), np.ones((8, 9)), atol=1e-15)
    x = np.arange(16)
    c = np.tile(np.cos(2 * np.pi * 3 * x / 16), (8, 1))
    h = oracle.rfftn(c)
    expect = np.zeros((8, 9), dtype=complex)
    expect[0, 3] = 8 * 16 / 2
    np.testing.assert_allclose(h, expect, atol=1e-12)


# ----------------------------------------------------------------------------- the step

def amplification(op, mean, q2, dt):
    """Closed form of the semi-implicit scheme for a small mode around a uniform mean:
    delta' = (1 - 3 mean^2 dt q^2) / (1 + dt q^2 Lk(q)) delta, with the Lk written out here."""
    kind, r, R1, qq = op
    lk = r + (1 - q2) ** 2 if kind == 0 else r + (1 - q2) ** 2 * (R1 + (qq * qq - q2) ** 2)
    return (1 - 3 * mean * mean * dt * q2) / (1 + dt * q2 * lk)


def mode_field(shape, dx, mean, delta, m):
    """mean + delta cos(q . x) with integer mode numbers m per axis (numpy axis order).
    Returns the field and |q|^2 with each index taken as its aliased wavenumber."""
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    phase = sum(2 * np.pi * mi * g / n for mi, g, n in zip(m, grids, shape))
    alias = [mi if mi <= n // 2 else mi - n for mi, n in zip(m, shape)]
    q2 = sum((2 * np.pi * mi / (n * dx)) ** 2 for mi, n in zip(alias, shape))
    return mean + delta * np.cos(phase), q2


def mode_amplitude(field, m):
    """delta of the cos mode m: the half-spectrum bin at index m holds delta N / 2."""
    return 2.0 * oracle.rfftn(field)[tuple(m)].real / field.size


@pytest.mark.parametrize("op", [ONE, TWO], ids=["one-mode", "two-mode"])
@pytest.mark.parametrize("shape,m", [((32, 32), (0, 5)), ((32, 32), (4, 0)), ((32, 64), (3, 7)),
                                     ((16, 16, 16), (2, 0, 0)), ((16, 16, 16), (0, 3, 1)),
                                     ((8, 16, 32), (1, 2, 3)), ((32, 32), (27, 2)),
                                     ((16, 16, 16), (13, 2, 0))])
@pytest.mark.parametrize("mean", [0.0, -0.25])
def test_single_mode_amplification_closed_form(op, shape, m, mean):
    """n steps of a small mode multiply it by g(q)^n (closed form of the scheme, including
    modes whose index lies in the negative half of an axis)."""
    dx, dt, nsteps = math.pi / 4, 0.5, 20
    _, q2 = mode_field(shape, dx, mean, 0.0, m)
    g = amplification(op, mean, q2, dt)
    # keep the mode small at every step (the cubic feeds back at relative O(delta^2))
    delta = 1e-6 / max(1.0, abs(g) ** nsteps)
    psi, _ = mode_field(shape, dx, mean, delta, m)
    out = oracle.step(psi, dx, dt, op, nsteps)
    assert mode_amplitude(out, m) == pytest.approx(delta * g ** nsteps, rel=2e-9)


def test_uniform_field_is_a_fixed_point_bitwise():
    psi = np.full((32, 64), -0.25)
    np.testing.assert_array_equal(oracle.step(psi, math.pi / 4, 0.5, ONE, 5), psi)
    psi3 = np.full((8, 8, 16), -0.35)
    np.testing.assert_array_equal(oracle.step(psi3, math.pi / 4, 0.1, TWO, 3), psi3)


@pytest.mark.parametrize("op", [ONE, TWO])
def test_mass_is_conserved(op):
    psi = inputs.uniform_state((32, 48), -0.25, 0.05, seed=11)
    m0 = oracle.mass(psi)
    out = oracle.step(psi, math.pi / 4, 0.5, op, 30)
    assert abs(oracle.mass(out) - m0) <= 1e-15


def test_translation_equivariance():
    psi = inputs.uniform_state((16, 32), -0.25, 0.1, seed=12)
    a = oracle.step(np.roll(psi, (3, 5), axis=(0, 1)), math.pi / 4, 0.5, ONE, 5)
    b = np.roll(oracle.step(psi, math.pi / 4, 0.5, ONE, 5), (3, 5), axis=(0, 1))
    np.testing.assert_allclose(a, b, atol=1e-14)


def test_transposition_symmetry_square_grid():
    psi = inputs.uniform_state((32, 32), -0.25, 0.1, seed=13)
    a = oracle.step(psi.T.copy(), math.pi / 4, 0.5, TWO, 4)
    b = oracle.step(psi, math.pi / 4, 0.5, TWO, 4).T
    np.testing.assert_allclose(a, b, atol=1e-14)
    p3 = inputs.uniform_state((8, 8, 8), -0.3, 0.1, seed=14)
    a3 = oracle.step(np.transpose(p3, (2, 0, 1)).copy(), math.pi / 4, 0.1, TWO, 2)
    b3 = np.transpose(oracle.step(p3, math.pi / 4, 0.1, TWO, 2), (2, 0, 1))
    np.testing.assert_allclose(a3, b3, atol=1e-14)


def test_field_constant_along_y_evolves_like_1d():
    row = inputs.uniform_state((64,), -0.25, 0.1, seed=15)
    psi = np.tile(row, (8, 1))
    a = oracle.step(psi, math.pi / 4, 0.5, ONE, 6)
    b = oracle.step(row, math.pi / 4, 0.5, ONE, 6)
    np.testing.assert_allclose(a, np.tile(b, (8, 1)), atol=1e-14)
    psi3 = np.broadcast_to(row, (4, 4, 64)).copy()
    a3 = oracle.step(psi3, math.pi / 4, 0.5, ONE, 3)
    b3 = oracle.step(row, math.pi / 4, 0.5, ONE, 3)
    np.testing.assert_allclose(a3, np.broadcast_to(b3, (4, 4, 64)), atol=1e-14)


def test_step_against_direct_numpy_spectral_update():
    """The update written with numpy's FFT and explicit wavenumber grids (different code,
    different FFT, k built from the box length n dx)."""
    shape, dx, dt = (12, 20), math.pi / 4, 0.5
    psi = inputs.uniform_state(shape, -0.25, 0.2, seed=16)
    ky = 2 * np.pi * np.fft.fftfreq(shape[0], d=dx)
    kx = 2 * np.pi * np.fft.rfftfreq(shape[1], d=dx)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    lk = -0.25 + (1 - k2) ** 2
    p = psi.copy()
    for _ in range(3):
        ph = np.fft.rfft2(p)
        nh = np.fft.rfft2(p ** 3)
        p = np.fft.irfft2((ph - dt * k2 * nh) / (1 + dt * k2 * lk), s=shape)
    np.testing.assert_allclose(oracle.step(psi, dx, dt, ONE, 3), p, atol=1e-14)


# ----------------------------------------------------------------------------- energy

@pytest.mark.parametrize("op", [ONE, TWO])
def test_energy_uniform_closed_form(op):
    kind, r, R1, q2 = op
    lk0 = r + 1.0 if kind == 0 else r + R1 + q2 ** 4
    for mean in (-0.25, 0.0, 0.3):
        psi = np.full((16, 16), mean)
        assert oracle.energy(psi, math.pi / 4, op) == pytest.approx(
            0.5 * lk0 * mean ** 2 + mean ** 4 / 4, rel=1e-14, abs=1e-17)


@pytest.mark.parametrize("op", [ONE, TWO])
def test_energy_single_mode_closed_form(op):
    kind, r, R1, qq = op
    shape, dx, mean, delta = (32, 64), math.pi / 4, -0.25, 0.1
    psi, q2 = mode_field(shape, dx, mean, delta, (0, 5))
    lk = (lambda k2: r + (1 - k2) ** 2) if kind == 0 else (
        lambda k2: r + (1 - k2) ** 2 * (R1 + (qq * qq - k2) ** 2))
    expect = 0.5 * lk(0.0) * mean ** 2 + 0.25 * lk(q2) * delta ** 2 + (
        mean ** 4 + 3 * mean ** 2 * delta ** 2 + 3.0 / 8.0 * delta ** 4) / 4
    assert oracle.energy(psi, dx, op) == pytest.approx(expect, rel=1e-13)


def test_energy_decreases_on_the_128_grid():
    """Empirical check of energy decay for the 128^2, dt = 0.5 one-mode run (the first-order
    semi-implicit scheme is not unconditionally stable, so this is a property of the run)."""
    psi = inputs.uniform_state((128, 128), -0.25, 0.01, seed=1)
    e = [oracle.energy(psi, math.pi / 4, ONE)]
    for _ in range(10):
        psi = oracle.step(psi, math.pi / 4, 0.5, ONE, 10)
        e.append(oracle.energy(psi, math.pi / 4, ONE))
    assert all(b <= a * (1 - 1e-14) or b <= a for a, b in zip(e, e[1:]))


# ----------------------------------------------------------------------------- two fields

def test_two_field_alpha_zero_reduces_to_independent_runs():
    """With alpha = 0 Cramer's rule reduces to the scalar update (equal to rounding)."""
    shape, dx, dt = (16, 32), math.pi / 4, 0.5
    p = inputs.uniform_state(shape, -0.25, 0.05, seed=21)
    c = inputs.uniform_state(shape, -0.2, 0.05, seed=22)
    op_c = (0, -0.2, 0.0, 0.0)
    p2, c2 = oracle.step2(p, c, dx, dt, ONE, op_c, 0.0, 4)
    np.testing.assert_allclose(p2, oracle.step(p, dx, dt, ONE, 4), rtol=0, atol=1e-15)
    np.testing.assert_allclose(c2, oracle.step(c, dx, dt, op_c, 4), rtol=0, atol=1e-15)


def test_two_field_small_mode_matches_linear_solve():
    """Linearised about uniform means, one step is x' = M^-1 diag(1 - 3 m_i^2 dt q^2) x, with
    M the implicit 2x2 matrix; solved here with numpy.linalg."""
    shape, dx, dt, alpha = (32, 32), math.pi / 4, 0.5, 0.1
    op_c = (0, -0.2, 0.0, 0.0)
    mp, mc = -0.25, -0.2
    p, q2 = mode_field(shape, dx, mp, 1e-7, (0, 4))
    c, _ = mode_field(shape, dx, mc, 2e-7, (0, 4))
    p1, c1 = oracle.step2(p, c, dx, dt, ONE, op_c, alpha, 1)
    lp = -0.25 + (1 - q2) ** 2
    lc = -0.2 + (1 - q2) ** 2
    m = np.array([[1 + dt * q2 * lp, dt * q2 * alpha], [dt * q2 * alpha, 1 + dt * q2 * lc]])
    rhs = np.array([(1 - 3 * mp * mp * dt * q2) * 1e-7, (1 - 3 * mc * mc * dt * q2) * 2e-7])
    x = np.linalg.solve(m, rhs)
    ap = mode_amplitude(p1, (0, 4))
    ac = mode_amplitude(c1, (0, 4))
    assert ap == pytest.approx(x[0], rel=1e-7)
    assert ac == pytest.approx(x[1], rel=1e-7)
    assert oracle.mass(p1) == pytest.approx(mp, abs=1e-15)
    assert oracle.mass(c1) == pytest.approx(mc, abs=1e-15)


def test_two_field_energy_uniform_closed_form():
    op_c = (0, -0.2, 0.0, 0.0)
    p = np.full((8, 8), -0.25)
    c = np.full((8, 8), -0.2)
    f = oracle.energy2(p, c, math.pi / 4, ONE, op_c, 0.1)
    expect = 0.5 * (1 - 0.25) * 0.0625 + 0.25 ** 4 / 4 + 0.5 * (1 - 0.2) * 0.04 + 0.2 ** 4 / 4 \
        + 0.1 * 0.25 * 0.2
    assert f == pytest.approx(expect, rel=1e-14)


# ----------------------------------------------------------------------------- adjoint

@pytest.mark.parametrize("op,shape", [(ONE, (16, 16)), (TWO, (8, 8, 8))])
def test_adjoint_dot_product(op, shape):
    dx, dt = math.pi / 4, 0.5 if op is ONE else 0.1
    psi = inputs.uniform_state(shape, -0.25, 0.2, seed=31)
    v = rng(32).standard_normal(shape)
    w = rng(33).standard_normal(shape)
    jv = oracle.step_tangent(psi, v, dx, dt, op)
    jtw, _ = oracle.step_adjoint(psi, w, dx, dt, op)
    assert np.sum(jv * w) == pytest.approx(np.sum(v * jtw), rel=1e-13)


def test_tangent_matches_central_difference():
    shape, dx, dt = (16, 16), math.pi / 4, 0.5
    psi = inputs.uniform_state(shape, -0.25, 0.2, seed=34)
    v = rng(35).standard_normal(shape)
    h = 1e-5
    fd = (oracle.step(psi + h * v, dx, dt, ONE) - oracle.step(psi - h * v, dx, dt, ONE)) / (2 * h)
    np.testing.assert_allclose(oracle.step_tangent(psi, v, dx, dt, ONE), fd, atol=1e-8)


@pytest.mark.parametrize("op,shape,dt", [(ONE, (16, 16), 0.5), (TWO, (8, 8, 8), 0.1)])
def test_adjoint_run_gradients_match_finite_differences(op, shape, dt):
    dx, nsteps = math.pi / 4, 6
    psi0 = inputs.uniform_state(shape, -0.25, 0.1, seed=41)
    target = oracle.step(psi0, dx, dt, (op[0], op[1] + 0.05, op[2], op[3]), nsteps)
    loss, g, gr = oracle.adjoint_run(psi0, target, dx, dt, op, nsteps)
    h = 1e-5
    lp = oracle.adjoint_run(psi0, target, dx, dt, (op[0], op[1] + h, op[2], op[3]), nsteps)[0]
    lm = oracle.adjoint_run(psi0, target, dx, dt, (op[0], op[1] - h, op[2], op[3]), nsteps)[0]
    assert gr == pytest.approx((lp - lm) / (2 * h), rel=1e-6)
    v = rng(42).standard_normal(shape)
    hp = 1e-6
    lp = oracle.adjoint_run(psi0 + hp * v, target, dx, dt, op, nsteps)[0]
    lm = oracle.adjoint_run(psi0 - hp * v, target, dx, dt, op, nsteps)[0]
    assert np.sum(g * v) == pytest.approx((lp - lm) / (2 * hp), rel=1e-6)


# ----------------------------------------------------------------------------- golden

def test_paper_operator_values():
    """The paper's FCC correlation operator (1 + lap)^2 (4/3 + lap)^2 of Eq. (5) at hand-evaluated
    wavenumbers; it is the two-mode form with R1 = 0 and q2^2 = 4/3."""
    with open(os.path.join(GOLDEN, "paper_operator.json")) as f:
        gold = json.load(f)
    eps = gold["eps"]
    op = (oracle.TWO_MODE, eps, 0.0, math.sqrt(4.0 / 3.0))
    for k2, expect in gold["values"]:
        assert oracle.lin_op(op, k2) == pytest.approx(expect, rel=1e-14, abs=1e-15)


def test_oracle_regression_fixture():
    """Stored oracle outputs (written by tests/golden/make_golden.py, which calls only the
    oracle and the input generators) guard the oracle against unintended changes."""
    with open(os.path.join(GOLDEN, "oracle_128_one_mode.json")) as f:
        gold = json.load(f)
    psi = inputs.uniform_state((128, 128), -0.25, 0.01, seed=1)
    op = (0, -0.25, 0.0, 0.0)
    out = oracle.step(psi, math.pi / 4, 0.5, op, gold["nsteps"])
    assert oracle.mass(out) == pytest.approx(gold["mass"], rel=1e-14)
    assert oracle.energy(out, math.pi / 4, op) == pytest.approx(gold["energy"], rel=1e-12)
    np.testing.assert_allclose(out.ravel()[gold["sample_idx"]], gold["sample_val"], rtol=1e-11,
                               atol=1e-14)


# ---------------------------------------------------------------------------------------------
# Alternative time integrators (step_scheme): 0 semi-implicit, 1 stabilised, 2 second-order BDF
# ---------------------------------------------------------------------------------------------
def test_scheme_zero_and_unstabilised_scheme_one_are_the_semi_implicit_step():
    psi = inputs.uniform_state((16, 32), -0.25, 0.1, seed=61)
    ref = oracle.step(psi, math.pi / 4, 0.5, ONE, 7)
    np.testing.assert_array_equal(oracle.step_scheme(psi, math.pi / 4, 0.5, ONE, 0, 0.0, 7), ref)
    np.testing.assert_array_equal(oracle.step_scheme(psi, math.pi / 4, 0.5, ONE, 1, 0.0, 7), ref)
    # the second-order scheme's first step is a semi-implicit step
    np.testing.assert_array_equal(oracle.step_scheme(psi, math.pi / 4, 0.5, ONE, 2, 0.0, 1),
                                  oracle.step(psi, math.pi / 4, 0.5, ONE, 1))


def _linear_recurrence(scheme, S, op, mean, q2, dt, nsteps, a0=1.0):
    """Amplitude of one small mode after nsteps steps, from the scalar recurrence each scheme
    reduces to when psi^3 is linearised about the mean (N_hat = 3 mean^2 psi_hat)."""
    kind, r, R1, qq = op
    lk = r + (1 - q2) ** 2 if kind == 0 else r + (1 - q2) ** 2 * (R1 + (qq * qq - q2) ** 2)
    c = 3.0 * mean * mean
    a_prev, a = a0, a0
    for s in range(nsteps):
        if scheme == 1:
            nxt = ((1 + dt * q2 * S) * a - dt * q2 * c * a) / (1 + dt * q2 * (lk + S))
        elif scheme == 2 and s > 0:
            nxt = (4 * a - a_prev - 2 * dt * q2 * c * (2 * a - a_prev)) / (3 + 2 * dt * q2 * lk)
        else:
            nxt = (a - dt * q2 * c * a) / (1 + dt * q2 * lk)
        a_prev, a = a, nxt
    return a


@pytest.mark.parametrize("scheme,S", [(1, 0.5), (1, 2.0), (2, 0.0)])
@pytest.mark.parametrize("op", [ONE, TWO], ids=["one-mode", "two-mode"])
@pytest.mark.parametrize("shape,m", [((32, 32), (0, 5)), ((32, 64), (3, 7)), ((16, 16, 16), (13, 2, 0))])
def test_scheme_single_mode_matches_its_scalar_recurrence(scheme, S, op, shape, m):
    dx, dt, nsteps, mean = math.pi / 4, 0.5, 12, -0.25
    _, q2 = mode_field(shape, dx, mean, 0.0, m)
    amp = _linear_recurrence(scheme, S, op, mean, q2, dt, nsteps)
    delta = 1e-6 / max(1.0, abs(amp))
    psi, _ = mode_field(shape, dx, mean, delta, m)
    out = oracle.step_scheme(psi, dx, dt, op, scheme, S, nsteps)
    assert mode_amplitude(out, m) == pytest.approx(delta * amp, rel=2e-9)


@pytest.mark.parametrize("scheme,S", [(1, 1.0), (2, 0.0)])
def test_schemes_conserve_mass(scheme, S):
    psi = inputs.uniform_state((24, 32), -0.25, 0.05, seed=62)
    out = oracle.step_scheme(psi, math.pi / 4, 0.5, ONE, scheme, S, 20)
    assert abs(oracle.mass(out) - oracle.mass(psi)) <= 1e-15


@pytest.mark.parametrize("scheme,S,order", [(0, 0.0, 1), (1, 0.5, 1), (2, 0.0, 2)])
def test_schemes_converge_at_their_order(scheme, S, order):
    """Error at t = 4 against a run with 1/32 of the step: halving dt divides it by 2^order.
    Smooth initial data (three low modes): a noisy start has a stiff initial layer that the
    first-order starting step of scheme 2 resolves only to first order."""
    y, x = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    psi = (-0.3 + 0.1 * np.cos(2 * np.pi * 2 * x / 16) + 0.07 * np.cos(2 * np.pi * (2 * y + 2 * x) / 16 + 0.3)
           + 0.05 * np.sin(2 * np.pi * 3 * y / 16))
    op, T = (oracle.ONE_MODE, -0.1, 0.0, 0.0), 4.0
    ref = oracle.step_scheme(psi, math.pi / 4, 0.2 / 32, op, scheme, S, int(round(T / (0.2 / 32))))
    errs = []
    for dt in (0.2, 0.1, 0.05):
        out = oracle.step_scheme(psi, math.pi / 4, dt, op, scheme, S, int(round(T / dt)))
        errs.append(np.linalg.norm(out - ref))
    for a, b in zip(errs, errs[1:]):
        assert 2 ** order * 0.8 <= a / b <= 2 ** order * 1.25


# ---------------------------------------------------------------------------------------------
# Hydrodynamic PFC (hydro_step)
# ---------------------------------------------------------------------------------------------
HYD = dict(rho=1.0, gamma=1.0, a0=2 * math.pi)


@pytest.mark.parametrize("shape", [(16, 32), (8, 16, 16)])
def test_hydro_without_velocity_response_is_the_pfc_step(shape):
    """rho = inf and v = 0: the velocity never moves and the density steps exactly like the
    semi-implicit PFC step."""
    psi = inputs.uniform_state(shape, -0.25, 0.1, seed=81)
    v = np.zeros((len(shape),) + shape)
    out, vo = oracle.hydro_step(psi, v, math.pi / 4, 0.5, ONE, math.inf, 1.0, 2 * math.pi, 6)
    np.testing.assert_array_equal(out, oracle.step(psi, math.pi / 4, 0.5, ONE, 6))
    np.testing.assert_array_equal(vo, v)


@pytest.mark.parametrize("shape,m,j", [((16, 32), (3, 5), 0), ((16, 32), (2, 1), 1), ((8, 16, 16), (1, 2, 3), 2)])
def test_hydro_velocity_mode_decays_viscously_on_a_uniform_density(shape, m, j):
    """psi uniform (no chemical-potential gradient, no advection): a velocity mode decays by
    1 / (1 + (dt/rho) Gamma k^2) per step and the density stays uniform."""
    dx, dt, n = math.pi / 4, 0.5, 5
    grids = np.meshgrid(*[np.arange(k) for k in shape], indexing="ij")
    phase = sum(2 * np.pi * mi * g / k for mi, g, k in zip(m, grids, shape)) + 0.4
    q2 = sum((2 * np.pi * (mi if mi <= k // 2 else mi - k) / (k * dx)) ** 2 for mi, k in zip(m, shape))
    psi = np.full(shape, -0.3)
    v = np.zeros((len(shape),) + shape)
    v[j] = 0.2 * np.cos(phase)
    out, vo = oracle.hydro_step(psi, v, dx, dt, ONE, HYD["rho"], 1.7, HYD["a0"], n)
    f = (1.0 / (1.0 + dt / HYD["rho"] * 1.7 * q2)) ** n
    np.testing.assert_allclose(vo[j], v[j] * f, atol=1e-14)
    assert np.abs(np.delete(vo, j, axis=0)).max() <= 1e-15
    np.testing.assert_allclose(out, psi, atol=1e-15)


@pytest.mark.parametrize("shape,m", [((32, 32), (0, 5)), ((32, 64), (3, 7)), ((16, 16, 16), (1, 0, 2))])
def test_hydro_advected_density_mode_closed_form(shape, m):
    """A constant velocity V along x advects a small density mode: its complex amplitude is
    multiplied by g = (1 - i dt q_x V - 3 mean^2 dt q^2) / (1 + dt q^2 Lk(q)) per step, to
    O(delta^2) (the velocity the mode drives is O(delta) and advects it at O(delta^2))."""
    dx, dt, n, mean, V = math.pi / 4, 0.5, 8, -0.25, 0.3
    psi, q2 = mode_field(shape, dx, mean, 0.0, m)
    qx = 2 * np.pi * m[-1] / (shape[-1] * dx)
    kind, r, R1, qq = ONE
    lk = r + (1 - q2) ** 2
    g = (1 - 1j * dt * qx * V - 3 * mean * mean * dt * q2) / (1 + dt * q2 * lk)
    delta = 1e-6 / max(1.0, abs(g) ** n)
    psi, _ = mode_field(shape, dx, mean, delta, m)
    v = np.zeros((len(shape),) + shape)
    v[0] = V
    out, _ = oracle.hydro_step(psi, v, dx, dt, ONE, HYD["rho"], HYD["gamma"], HYD["a0"], n)
    amp = oracle.rfftn(out)[tuple(m)] * 2.0 / out.size
    assert abs(amp - delta * g ** n) <= 2e-9 * abs(delta * g ** n)


def test_hydro_one_step_mass_follows_the_divergence_of_v():
    """The advection term v . grad psi conserves the mean density when div v = 0 (one step from
    a shear flow) and does not otherwise."""
    shape, dx, dt = (32, 32), math.pi / 4, 0.5
    psi = inputs.uniform_state(shape, -0.25, 0.1, seed=82)
    y, x = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    shear = np.stack([0.3 * np.sin(2 * np.pi * 2 * y / 32), np.zeros(shape)])
    out, _ = oracle.hydro_step(psi, shear, dx, dt, ONE, **HYD)
    assert abs(oracle.mass(out) - oracle.mass(psi)) <= 1e-15
    compress = np.stack([0.3 * np.sin(2 * np.pi * 2 * x / 32), np.zeros(shape)])
    out, _ = oracle.hydro_step(psi, compress, dx, dt, ONE, **HYD)
    assert abs(oracle.mass(out) - oracle.mass(psi)) > 1e-6

"""GPU parity of grids whose extents are not all powers of two (n = 2^a 3^b 5^c 7^d, nx even).

These grids run the mixed-radix schedule: one pass per axis, each line a Stockham transform of
radices 2, 3, 4, 5, 7 and 8 in shared memory (11 sweeps a step in 3D, 7 in 2D). Every call on
such a plan is compared with the FP64 oracle (whose own mixed-radix transform is pinned to the
naive DFT and numpy.fft):
  * r2c / c2r element by element on lines of 750, 900 and 1400 points along x (M = nx / 2 points
    of the complex transform) and along y, and on small 3D grids with every radix, at the
    tolerances of the power-of-two tests (FP64 1e-13, FP32 3e-6);
  * one and twenty semi-implicit steps (FP64 1e-12 / 1e-11, FP32 2e-6 / 1e-5), the carried mass
    and the energy;
  * the hydrodynamic step, which runs on the plan's transforms;
  * the calls built for power-of-two grids only, which report UNSUPPORTED;
  * the autotuner's radix orders and launch shapes, against the oracle after tuning.
At the paper's 750^3 (FP32-mixed) the oracle cannot step the grid in a test's time; there:
  * a field repeating a 150^3 block is stepped exactly like the block on the 150^3 grid, which
    the oracle steps;
  * three bins of the forward transform are summed axis by axis in FP64 on the host from the
    definition.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_26818_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DX = math.pi / 4
ONE = (0, -0.25, 0.0, 0.0)
TWO3 = (1, -0.3, 0.05, math.sqrt(4.0 / 3.0))
TOL_FFT = {"fp64": 1e-13, "fp32": 3e-6}
TOL_1 = {"fp64": 1e-12, "fp32": 2e-6}
TOL_20 = {"fp64": 1e-11, "fp32": 1e-5}

# 2D: the paper's line lengths along x (nx = 2 M) and along y; 3D: every radix on some axis,
# odd M, power-of-two axes mixed in
SHAPES_2D = [(16, 1500), (24, 1800), (8, 2800), (750, 16), (900, 24), (1400, 16), (96, 64), (30, 42)]
SHAPES_3D = [(30, 20, 36), (14, 48, 90), (50, 42, 28), (16, 27, 70), (25, 64, 98)]


def _binding():
    from paper_2603_26818_gb300 import binding
    return binding


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def to_dev(a, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def plan(shape, op, prec, dt):
    b = _binding()
    p = b.Plan(shape, DX, dt, [b.make_op(*op)], precision=prec)
    assert p.info()["Py"] == 0   # the mixed-radix schedule
    return p


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", SHAPES_2D + SHAPES_3D)
def test_mixed_transforms(shape, prec):
    p = plan(shape, ONE, prec, 0.5)
    x = inputs.uniform_state(shape, 0.1, 1.0, seed=7)
    xh = p.fft_r2c(to_dev(x, prec))
    ref = oracle.rfftn(x)
    assert rel(xh.cpu().numpy(), ref) <= TOL_FFT[prec]
    r = np.random.default_rng(11)
    h = r.standard_normal(ref.shape) + 1j * r.standard_normal(ref.shape)
    y = p.fft_c2r(torch.from_numpy(h).to(device="cuda", dtype=p.complex_dtype))
    assert rel(y.double().cpu().numpy(), oracle.irfftn(h, shape)) <= TOL_FFT[prec]
    # the round trip of a real field
    back = p.fft_c2r(p.fft_r2c(to_dev(x, prec)))
    assert rel(back.double().cpu().numpy(), x) <= TOL_FFT[prec]
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(96, 64), (30, 42), (24, 1800), (750, 16)] + SHAPES_3D)
def test_mixed_steps(shape, prec):
    op = TWO3 if len(shape) == 3 else ONE
    dt = 0.1 if len(shape) == 3 else 0.5
    mean = -0.35 if len(shape) == 3 else -0.25
    p = plan(shape, op, prec, dt)
    psi0 = inputs.uniform_state(shape, mean, 0.05, seed=13)
    x = to_dev(psi0, prec)
    p.step(x, 1)
    assert rel(x.double().cpu().numpy(), oracle.step(psi0, DX, dt, op, 1)) <= TOL_1[prec]
    p.step(x, 19)
    got = x.double().cpu().numpy()
    ref = oracle.step(psi0, DX, dt, op, 20)
    assert rel(got, ref) <= TOL_20[prec]
    assert abs(p.mass(x)[0] - oracle.mass(got)) <= 1e-12 * abs(mean) + (1e-7 if prec == "fp32" else 0)
    e_ref = oracle.energy(got, DX, op)
    assert abs(p.energy(x) - e_ref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(e_ref)
    p.close()


def test_mixed_step_pattern_forms():
    """A 2D run long enough to form the stripes/triangles of the one-mode model: the GPU state
    stays on the oracle's trajectory (not only near its start)."""
    shape, dt = (60, 70), 0.5
    psi0 = inputs.uniform_state(shape, -0.25, 0.1, seed=5)
    p = plan(shape, ONE, "fp64", dt)
    x = to_dev(psi0, "fp64")
    p.step(x, 400)
    ref = oracle.step(psi0, DX, dt, ONE, 400)
    assert np.std(ref) > 0.05   # a pattern formed
    assert rel(x.cpu().numpy(), ref) <= 1e-9
    p.close()


def test_mixed_hydro():
    b = _binding()
    shape, dt = (24, 30, 36), 0.05
    psi0 = inputs.uniform_state(shape, -0.3, 0.05, seed=31)
    v0 = np.stack([inputs.uniform_state(shape, 0.0, 0.02, seed=40 + j) for j in range(3)])
    h = b.Hydro(shape, DX, dt, b.make_op(*ONE), rho=2.0, gamma=0.5, a0=0.7, precision="fp64")
    psi = to_dev(psi0, "fp64")
    v = to_dev(v0, "fp64")
    h.step(psi, v, 3)
    ref_p, ref_v = oracle.hydro_step(psi0, v0, DX, dt, ONE, 2.0, 0.5, 0.7, 3)
    assert rel(psi.cpu().numpy(), ref_p) <= 1e-12
    assert rel(v.cpu().numpy(), ref_v) <= 1e-11
    h.close()


def test_mixed_unsupported_calls():
    b = _binding()
    p = plan((30, 42), ONE, "fp64", 0.5)
    x = to_dev(inputs.uniform_state((30, 42), -0.25, 0.05, seed=3), "fp64")
    with pytest.raises(b.PfcError, match="UNSUPPORTED"):
        p.set_integrator(b.PFC_SBDF2)
    p.set_integrator(b.PFC_SEMI_IMPLICIT)
    assert p.record_bytes(4) is None
    lam = torch.zeros_like(x)
    dr = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(b.PfcError, match="UNSUPPORTED"):
        p.step_adjoint(x, x, lam, dr)
    with pytest.raises(b.PfcError, match="UNSUPPORTED"):
        b.Plan((30, 42), DX, 0.5, [b.make_op(*ONE), b.make_op(*ONE)], precision="fp64", coupling=0.1)
    # the plan is still usable; the per-pass profile runs the same steps
    psi0 = x.cpu().numpy()
    p.step(x, 2)
    assert rel(x.cpu().numpy(), oracle.step(psi0, DX, 0.5, ONE, 2)) <= 1e-12
    ms, launches = p.profile_steps(x, 3)
    assert launches == 4 + 3 * 5 + 2 and ms["row"] > 0 and ms["line"] > 0 and ms["mid"] > 0
    assert rel(x.cpu().numpy(), oracle.step(psi0, DX, 0.5, ONE, 5)) <= 1e-12
    p.close()


# ------------------------------------------------------------------------------ full size
def test_750cube_fp32_tiled_block_matches_oracle():
    b = _binding()
    big, small, dt, nsteps = 750, 150, 0.1, 2
    sm_shape = (small,) * 3
    psi_s = inputs.uniform_state(sm_shape, -0.35, 0.05, seed=43)
    ref_s = oracle.step(psi_s, DX, dt, TWO3, nsteps)
    reps = big // small
    p = plan((big,) * 3, TWO3, "fp32", dt)
    x = torch.from_numpy(psi_s).to(device="cuda", dtype=torch.float32).repeat(reps, reps, reps)
    p.step(x, nsteps)
    torch.cuda.synchronize()
    p.close()
    tgt = torch.from_numpy(ref_s).to(device="cuda", dtype=torch.float64).repeat(1, reps, reps)
    err2 = ref2 = 0.0
    for z0 in range(0, big, small):
        d = x[z0:z0 + small].double() - tgt
        err2 += float((d * d).sum())
        ref2 += float((tgt * tgt).sum())
        del d
    del x, tgt
    torch.cuda.empty_cache()
    assert math.sqrt(err2 / ref2) <= 2e-6


def test_1400cube_fp32_tiled_block_matches_oracle():
    """The paper's largest grid, 1400^3 (radices 8, 7, 5, 5 per axis), in FP32-mixed: a field
    that repeats a 175^3 block (175 = 5^2 7) eight times per axis is stepped exactly like the
    block on the 175^3 grid, which the oracle steps; one step, one-mode operator as config 1400."""
    big, small, dt, nsteps = 1400, 175, 0.5, 1
    op = (0, -0.25, 0.0, 0.0)
    sm_shape = (small,) * 3
    psi_s = inputs.uniform_state(sm_shape, -0.25, 0.01, seed=53).astype(np.float32).astype(np.float64)
    ref_s = oracle.step(psi_s, DX, dt, op, nsteps)
    reps = big // small
    p = plan((big,) * 3, op, "fp32", dt)
    x = torch.from_numpy(psi_s).to(device="cuda", dtype=torch.float32).repeat(reps, reps, reps)
    p.step(x, nsteps)
    torch.cuda.synchronize()
    p.close()
    tgt = torch.from_numpy(ref_s).to(device="cuda", dtype=torch.float64).repeat(1, reps, reps)
    err2 = ref2 = 0.0
    for z0 in range(0, big, small):
        d = x[z0:z0 + small].double() - tgt
        err2 += float((d * d).sum())
        ref2 += float((tgt * tgt).sum())
        del d
    del x, tgt
    torch.cuda.empty_cache()
    assert math.sqrt(err2 / ref2) <= 2e-6


def test_750cube_fp32_forward_bins_from_the_definition():
    """X[kz, ky, kx] = sum_z e^{-2 pi i kz z / n} sum_y e^{-2 pi i ky y / n} sum_x e^{-2 pi i kx x / n}
    psi[z, y, x], summed one axis at a time in FP64 on the host (the FP32 field as given)."""
    n = 750
    shape = (n, n, n)
    p = plan(shape, TWO3, "fp32", 0.1)
    x = to_dev(inputs.uniform_state(shape, -0.35, 0.5, seed=47), "fp32")
    xh = p.fft_r2c(x)
    bins = [(0, 0, 1), (7, 374, 375), (749, 125, 200)]
    got = [complex(xh[kz, ky, kx].item()) for kz, ky, kx in bins]
    del xh
    p.close()
    host = x.cpu().numpy().astype(np.float64)
    del x
    torch.cuda.empty_cache()
    t = np.arange(n)
    for (kz, ky, kx), g in zip(bins, got):
        ex = np.exp(-2j * np.pi * kx * t / n)
        ey = np.exp(-2j * np.pi * ky * t / n)
        ez = np.exp(-2j * np.pi * kz * t / n)
        acc = 0.0 + 0.0j
        for z0 in range(0, n, 50):
            sx = host[z0:z0 + 50] @ ex          # (50, n)
            acc += ez[z0:z0 + 50] @ (sx @ ey)
        # FP32 rounding of a transform of 4.2e8 values: relative to the field's norm
        scale = math.sqrt(float((host * host).sum()))
        assert abs(g - acc) <= 1e-5 * scale, (kz, ky, kx, g, acc)


def test_mixed_radix_autotune_keeps_parity():
    """pfc_plan_autotune on a mixed-radix plan (radix order, warps a column, rows a block): the
    autotuned plan against the oracle, FP64, 2D and 3D, and a 750-point line plan in FP32."""
    import math
    from paper_2603_26818_gb300 import binding, inputs
    import oracle
    for shape, prec, tol in (((60, 90), "fp64", 1e-11), ((24, 30, 36), "fp64", 1e-11), ((12, 750), "fp32", 1e-5)):
        psi0 = inputs.uniform_state(shape, -0.25, 0.01, seed=77)
        if prec == "fp32":
            psi0 = psi0.astype(np.float32).astype(np.float64)
        p = binding.Plan(shape, math.pi / 4, 0.5, [binding.make_op(0, -0.25)], precision=prec)
        ms = p.autotune(8, 3)
        assert ms > 0
        x = torch.from_numpy(psi0).to(device="cuda", dtype=torch.float64 if prec == "fp64" else torch.float32)
        p.step(x, 6)
        ref = oracle.step(psi0, math.pi / 4, 0.5, (0, -0.25, 0.0, 0.0), 6)
        got = x.double().cpu().numpy()
        assert float(np.linalg.norm(got - ref) / np.linalg.norm(ref)) <= tol
        p.close()

"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle, element by element.

Tolerances (relative L2 unless stated), from the arithmetic of each path:
  FP64 transforms 1e-13; FP64 step 1e-12 after one step, 1e-10 after 100 steps.
  FP32-mixed transforms 2e-6 (single-precision butterflies, ~eps32 * log2 N);
  FP32-mixed step 2e-6 after one step, 1e-5 after 100 steps; mass drift 1e-6 relative.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_26818_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ONE = (0, -0.25, 0.0, 0.0)
TWO = (1, -0.3, 0.05, math.sqrt(4.0 / 3.0))
# the paper's FCC operator of Eq. (5): two-mode with R1 = 0, q2^2 = 4/3 (eps = -0.25)
PAPER_FCC = (1, -0.25, 0.0, math.sqrt(4.0 / 3.0))
TOL_FFT = {"fp64": 1e-13, "fp32": 2e-6}


def _binding():
    from paper_2603_26818_gb300 import binding
    return binding


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def to_dev(a, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def plan(dims, dx, dt, op, prec):
    b = _binding()
    return b.Plan(dims, dx, dt, [b.make_op(*op)], precision=prec)


# shapes chosen to cover: tiny grids, rectangular grids, the P/Q split of y (ny = 4096),
# the split of y and z in 3D, several W and row-group choices
FFT_SHAPES = [(16, 16), (32, 64), (128, 128), (64, 256), (256, 32), (4096, 16), (2048, 64),
              (16, 16, 16), (32, 16, 64), (64, 32, 16), (512, 16, 16), (128, 128, 32)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", FFT_SHAPES)
def test_r2c_and_c2r_match_oracle(shape, prec):
    x = inputs.uniform_state(shape, 0.1, 1.0, seed=hash(shape) % 1000)
    p = plan(shape, math.pi / 4, 0.5, ONE, prec)
    xd = to_dev(x, prec)
    xh = p.fft_r2c(xd)
    ref = oracle.rfftn(x)
    assert rel(xh.cpu().numpy(), ref) <= TOL_FFT[prec]
    # c2r of an arbitrary (not Hermitian-consistent) half spectrum, imaginary parts of the
    # kx = 0 and Nyquist bins ignored
    r = np.random.default_rng(5)
    h = r.standard_normal(ref.shape) + 1j * r.standard_normal(ref.shape)
    hd = torch.from_numpy(h).to(device="cuda", dtype=p.complex_dtype)
    y = p.fft_c2r(hd)
    assert rel(y.double().cpu().numpy(), oracle.irfftn(h, shape)) <= TOL_FFT[prec]
    p.close()


def test_split_plans_are_exercised():
    """The shapes above include plans that split y (Py > 1) and both y and z (Pz > 1)."""
    seen = set()
    for shape in FFT_SHAPES:
        for prec in ("fp64", "fp32"):
            info = plan(shape, math.pi / 4, 0.5, ONE, prec).info()
            seen.add((info["Py"] > 1, info["Pz"] > 1))
    assert (True, False) in seen and (True, True) in seen and (False, False) in seen


@pytest.mark.parametrize("prec,tol1,tol100", [("fp64", 1e-12, 1e-10), ("fp32", 2e-6, 1e-5)])
def test_config1_128_one_mode_steps(prec, tol1, tol100):
    """128^2 one-mode, dx = pi/4, dt = 0.5, r = -0.25, psi0 = -0.25 + U[-0.01, 0.01] (seed 1)."""
    dims, dx, dt = (128, 128), math.pi / 4, 0.5
    psi0 = inputs.uniform_state(dims, -0.25, 0.01, seed=1)
    p = plan(dims, dx, dt, ONE, prec)
    x = to_dev(psi0, prec)
    p.step(x, 1)
    assert rel(x.double().cpu().numpy(), oracle.step(psi0, dx, dt, ONE, 1)) <= tol1
    x = to_dev(psi0, prec)
    p.step(x, 100)
    ref = oracle.step(psi0, dx, dt, ONE, 100)
    got = x.double().cpu().numpy()
    assert rel(got, ref) <= tol100
    assert rel(got - got.mean(), ref - ref.mean()) <= tol100 * 50
    m0 = oracle.mass(psi0)
    assert abs(p.mass(x)[0] - m0) <= 1e-6 * abs(m0)
    assert p.energy(x) == pytest.approx(oracle.energy(ref, dx, ONE), rel=1e-10 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
@pytest.mark.parametrize("shape,op,dt,nsteps", [
    ((32, 32, 32), TWO, 0.1, 10),
    ((16, 32, 64), ONE, 0.5, 10),
    ((512, 16, 16), TWO, 0.1, 5),
    ((4096, 16), ONE, 0.5, 10),
    ((64, 128), TWO, 0.1, 20),
    ((32, 32, 32), PAPER_FCC, 0.1, 10),
    ((128, 256), PAPER_FCC, 0.1, 10),
])
def test_steps_match_oracle(shape, op, dt, nsteps, prec, tol):
    dx = math.pi / 4
    psi0 = inputs.uniform_state(shape, -0.3, 0.05, seed=7)
    p = plan(shape, dx, dt, op, prec)
    x = to_dev(psi0, prec)
    p.step(x, nsteps)
    ref = oracle.step(psi0, dx, dt, op, nsteps)
    assert rel(x.double().cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mass_and_energy_match_oracle(prec):
    shape, dx = (64, 32, 16), math.pi / 4
    psi = inputs.uniform_state(shape, -0.3, 0.2, seed=9)
    for op in (ONE, TWO):
        p = plan(shape, dx, 0.1, op, prec)
        x = to_dev(psi, prec)
        xin = x.double().cpu().numpy()
        assert p.mass(x)[0] == pytest.approx(oracle.mass(xin), rel=1e-14, abs=1e-15)
        assert p.energy(x) == pytest.approx(oracle.energy(xin, dx, op), rel=1e-12 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uniform_state_is_a_fixed_point(prec):
    p = plan((64, 64), math.pi / 4, 0.5, ONE, prec)
    x = to_dev(np.full((64, 64), -0.25), prec)
    p.step(x, 50)
    assert float((x.double() + 0.25).abs().max()) <= (1e-15 if prec == "fp64" else 1e-7)


def test_zero_steps_is_a_no_op_and_runs_are_deterministic():
    psi0 = inputs.uniform_state((128, 128), -0.25, 0.05, seed=3)
    p = plan((128, 128), math.pi / 4, 0.5, ONE, "fp32")
    x = to_dev(psi0, "fp32")
    y = x.clone()
    p.step(x, 0)
    assert torch.equal(x, y)
    a = to_dev(psi0, "fp32")
    b = to_dev(psi0, "fp32")
    p.step(a, 37)
    p.step(b, 37)
    assert torch.equal(a, b)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 1e-3)])
def test_long_single_call_matches_oracle(prec, tol):
    """6000 steps in one call: the redundant kx = 0 / nx/2 columns of the carried state must be
    kept real in row space, otherwise a rounding-seeded component invisible to psi^3 grows by
    1/D(k) per step at the unstable wavenumbers and overflows (FP32 within ~600 steps)."""
    dims, dx, dt, nsteps = (64, 64), math.pi / 4, 0.5, 6000
    psi0 = inputs.uniform_state(dims, -0.25, 0.05, seed=17)
    p = plan(dims, dx, dt, ONE, prec)
    x = to_dev(psi0, prec)
    p.step(x, nsteps)
    got = x.double().cpu().numpy()
    assert np.isfinite(got).all()
    assert rel(got, oracle.step(psi0, dx, dt, ONE, nsteps)) <= tol


def test_long_single_call_3d_split_plan_stays_finite():
    """A 3D plan with y and z split (P > 1) carried for 2000 steps in one call."""
    shape, dx, dt = (512, 16, 16), math.pi / 4, 0.5
    psi0 = inputs.uniform_state(shape, -0.25, 0.05, seed=18)
    p = plan(shape, dx, dt, ONE, "fp32")
    assert p.info()["Pz"] > 1 or p.info()["Py"] > 1
    x = to_dev(psi0, "fp32")
    p.step(x, 2000)
    y = to_dev(psi0, "fp32")
    for _ in range(20):
        p.step(y, 100)
    a, b = x.double().cpu().numpy(), y.double().cpu().numpy()
    assert np.isfinite(a).all() and rel(a, b) <= 1e-3


def test_row_cluster_path_at_4096sq_matches_single_blocks_and_oracle(monkeypatch):
    """4096^2 FP32 (Py = 8): the psi^3 row pass runs on clusters of two blocks, each holding four
    of the group's eight rows and reaching the others through distributed shared memory. The same
    operations as the single-block row pass (the compiler may contract them into FMAs
    differently, so agreement is to rounding, not bitwise); and both match the oracle after 3
    steps (polycrystal input of the bench workload)."""
    shape, dx, dt, nsteps = (4096, 4096), math.pi / 4, 0.5, 3
    psi0 = inputs.polycrystal_2d(4096, 4096, dx, -0.25, 64, 0.2, 1.0, 0.01, seed=11)
    monkeypatch.delenv("PFC_ROW_CLUSTER", raising=False)
    p = plan(shape, dx, dt, ONE, "fp32")
    assert p.info()["row_cluster"] == 2
    x = to_dev(psi0, "fp32")
    p.step(x, nsteps)
    p.close()
    monkeypatch.setenv("PFC_ROW_CLUSTER", "0")
    q = plan(shape, dx, dt, ONE, "fp32")
    assert q.info()["row_cluster"] == 0
    y = to_dev(psi0, "fp32")
    q.step(y, nsteps)
    q.close()
    a, b = x.double().cpu().numpy(), y.double().cpu().numpy()
    ref = oracle.step(psi0, dx, dt, ONE, nsteps)
    print("cluster vs single", rel(a, b), "cluster vs oracle", rel(a, ref), "single vs oracle", rel(b, ref))
    assert rel(a, b) <= 1e-6
    assert rel(a, ref) <= 1e-5 and rel(b, ref) <= 1e-5


def test_row_cluster_3d_path_matches_single_blocks_and_oracle(monkeypatch):
    """A 3D plan with Py = Pz = 8 and rows of nx = 512 (nz = ny = 256): the psi^3 row pass runs
    on two-block clusters split by z_p halves (z-parts through distributed shared memory, edge
    values gathered in block 0 for the projection). Compared with the single-block row pass and
    with the oracle after 2 two-mode steps."""
    shape, dx, dt, nsteps = (256, 256, 512), math.pi / 4, 0.1, 2
    psi0 = inputs.uniform_state(shape, -0.35, 0.02, seed=12)
    monkeypatch.delenv("PFC_ROW_CLUSTER", raising=False)
    p = plan(shape, dx, dt, TWO, "fp32")
    assert p.info()["row_cluster"] == 2 and p.info()["Pz"] == 8
    x = to_dev(psi0, "fp32")
    p.step(x, nsteps)
    p.close()
    monkeypatch.setenv("PFC_ROW_CLUSTER", "0")
    q = plan(shape, dx, dt, TWO, "fp32")
    assert q.info()["row_cluster"] == 0
    y = to_dev(psi0, "fp32")
    q.step(y, nsteps)
    q.close()
    a, b = x.double().cpu().numpy(), y.double().cpu().numpy()
    ref = oracle.step(psi0, dx, dt, TWO, nsteps)
    assert rel(a, b) <= 1e-6
    assert rel(a, ref) <= 1e-5 and rel(a - a.mean(), ref - ref.mean()) <= 1e-4


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonfinite_state_is_reported_and_the_plan_stays_usable(prec):
    """A NaN or Inf in the state is caught by the FP64 reductions (the mean taken at the start
    of every pfc_step call, mass, energy) and reported as PFC_ERR_NONFINITE; the status is
    cleared once reported and the plan keeps working."""
    b = _binding()
    p = plan((64, 64), math.pi / 4, 0.5, ONE, prec)
    psi0 = inputs.uniform_state((64, 64), -0.25, 0.05, seed=21)
    x = to_dev(psi0, prec)
    x[3, 5] = float("nan")
    with pytest.raises(b.PfcError, match="NONFINITE"):
        p.mass(x)
    y = to_dev(psi0, prec)
    y[0, 0] = float("inf")
    p.step(y, 3)
    with pytest.raises(b.PfcError, match="NONFINITE"):
        p.sync()
    z = to_dev(psi0, prec)
    p.step(z, 3)
    p.sync()
    assert rel(z.double().cpu().numpy(), oracle.step(psi0, math.pi / 4, 0.5, ONE, 3)) <= (1e-12 if prec == "fp64" else 2e-6)
    p.close()

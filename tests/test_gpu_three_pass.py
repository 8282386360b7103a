"""GPU parity of the three-pass schedule (row pass, middle pass, line pass; 9 sweeps a step).

Small grids: a three-pass tiling is forced with PFC_TILE="Py,Pz,W,Ry,Rz" and every call that
runs on it (r2c, c2r, steps, energy, mass, the adjoint step) is compared with the FP64 oracle
element by element, at the tolerances of the two-pass tests (FP64 transforms 1e-13, FP64 step
1e-12 after one step and 1e-10 after 100; FP32-mixed 2e-6 and 1e-5).

Full sizes, where the planner itself picks the three-pass schedule (no two-pass tiling fits):
  * FP64 512^3 (the FP64 side of the 512^3 two-mode workload): one and two steps against the
    oracle.
  * 1024^3 FP64 and 2048^3 FP32-mixed: the oracle cannot step these grids in a test's time, so
    they are checked through exact properties at any size:
      - a field that repeats with period n/s is stepped exactly like its one period on the
        (n/s)-grid (the tiled field has only the wavenumbers of the small grid, with the same
        k and the same multipliers); the small grid is stepped by the oracle;
      - a few Fourier modes of random wavevector (odd indices included) on a uniform
        background, small amplitude, evolve by the closed-form factor
        g(q) = (1 - 3 mean^2 dt q^2) / (1 + dt q^2 Lk(q)) per step, to O(amplitude^2).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2603_26818_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DX = math.pi / 4
ONE = (0, -0.25, 0.0, 0.0)
TWO3 = (1, -0.3, 0.05, math.sqrt(4.0 / 3.0))
TOL_FFT = {"fp64": 1e-13, "fp32": 2e-6}
TOL_1 = {"fp64": 1e-12, "fp32": 2e-6}
TOL_20 = {"fp64": 1e-11, "fp32": 1e-5}

# (shape, forced tiling "Py,Pz,W,Ry,Rz"): 2D and 3D, one- and two-axis middle passes, several
# line-tile shapes
FORCED = [((64, 128), "2,1,4,4,1"), ((128, 64), "1,1,2,8,1"), ((32, 64, 32), "2,2,4,4,2"),
          ((64, 32, 64), "1,2,2,2,4"), ((64, 64, 16), "8,1,2,1,8"), ((32, 32, 32), "2,4,1,2,1")]


def _binding():
    from paper_2603_26818_gb300 import binding
    return binding


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def to_dev(a, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def forced_plan(monkeypatch, shape, tile, op, prec, dt=0.5):
    b = _binding()
    monkeypatch.setenv("PFC_TILE", tile)
    p = b.Plan(shape, DX, dt, [b.make_op(*op)], precision=prec)
    info = p.info()
    py, pz, w, ry, rz = (int(v) for v in tile.split(","))
    assert (info["Py"], info["Pz"], info["W"], info["Ry"], info["Rz"]) == (py, pz, w, ry, rz)
    return p


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,tile", FORCED)
def test_forced_three_pass_transforms(monkeypatch, shape, tile, prec):
    p = forced_plan(monkeypatch, shape, tile, ONE, prec)
    x = inputs.uniform_state(shape, 0.1, 1.0, seed=7)
    xh = p.fft_r2c(to_dev(x, prec))
    ref = oracle.rfftn(x)
    assert rel(xh.cpu().numpy(), ref) <= TOL_FFT[prec]
    r = np.random.default_rng(11)
    h = r.standard_normal(ref.shape) + 1j * r.standard_normal(ref.shape)
    y = p.fft_c2r(torch.from_numpy(h).to(device="cuda", dtype=p.complex_dtype))
    assert rel(y.double().cpu().numpy(), oracle.irfftn(h, shape)) <= TOL_FFT[prec]
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,tile", FORCED)
def test_forced_three_pass_steps(monkeypatch, shape, tile, prec):
    op = TWO3 if len(shape) == 3 else ONE
    dt = 0.1 if len(shape) == 3 else 0.5
    mean = -0.35 if len(shape) == 3 else -0.25
    p = forced_plan(monkeypatch, shape, tile, op, prec, dt)
    psi0 = inputs.uniform_state(shape, mean, 0.05, seed=13)
    x = to_dev(psi0, prec)
    p.step(x, 1)
    assert rel(x.double().cpu().numpy(), oracle.step(psi0, DX, dt, op, 1)) <= TOL_1[prec]
    p.step(x, 19)   # 16 of them through the captured graph
    got = x.double().cpu().numpy()
    ref = oracle.step(psi0, DX, dt, op, 20)
    assert rel(got, ref) <= TOL_20[prec]
    # mass carried exactly, energy of the stepped field
    assert abs(p.mass(x)[0] - oracle.mass(got)) <= 1e-12 * abs(mean) + (1e-7 if prec == "fp32" else 0)
    e_ref = oracle.energy(got, DX, op)
    assert abs(p.energy(x) - e_ref) <= (1e-12 if prec == "fp64" else 1e-6) * abs(e_ref)
    p.close()


def test_forced_three_pass_adjoint(monkeypatch):
    shape, tile = (32, 64, 32), "2,2,4,4,2"
    p = forced_plan(monkeypatch, shape, tile, ONE, "fp64")
    psi = inputs.uniform_state(shape, -0.25, 0.05, seed=17)
    lam = inputs.uniform_state(shape, 0.0, 1.0, seed=19)
    lam_out = torch.empty(shape, dtype=torch.float64, device="cuda")
    dr = torch.zeros(1, dtype=torch.float64, device="cuda")
    p.step_adjoint(to_dev(psi, "fp64"), to_dev(lam, "fp64"), lam_out, dr)
    ref, dr_ref = oracle.step_adjoint(psi, lam, DX, 0.5, ONE)
    assert rel(lam_out.cpu().numpy(), ref) <= 1e-12
    assert abs(float(dr.item()) - dr_ref) <= 1e-11 * abs(dr_ref)
    p.close()


def test_autotune_may_choose_the_pass_schedule():
    """The autotuner's candidates include three-pass tilings; whichever it keeps, the plan stays
    exact."""
    b = _binding()
    shape = (64, 64, 64)
    p = b.Plan(shape, DX, 0.1, [b.make_op(*TWO3)], precision="fp64")
    p.autotune(12, 4)
    psi0 = inputs.uniform_state(shape, -0.35, 0.05, seed=23)
    x = to_dev(psi0, "fp64")
    p.step(x, 5)
    assert rel(x.cpu().numpy(), oracle.step(psi0, DX, 0.1, TWO3, 5)) <= 1e-11
    p.close()


# ------------------------------------------------------------------------------ full sizes
def test_512cube_fp64_three_pass_matches_oracle():
    shape, dt = (512, 512, 512), 0.1
    psi0 = inputs.uniform_state(shape, -0.35, 0.02, seed=3)
    b = _binding()
    p = b.Plan(shape, DX, dt, [b.make_op(*TWO3)], precision="fp64")
    info = p.info()
    assert info["Ry"] * info["Rz"] > 1   # the planner's three-pass tiling
    x = torch.from_numpy(psi0).cuda()
    p.step(x, 2)
    got = x.cpu().numpy()
    del x
    p.close()
    ref = oracle.step(psi0, DX, dt, TWO3, 2)
    assert rel(got, ref) <= 1e-12
    assert rel(got - got.mean(), ref - ref.mean()) <= 1e-10


def _tiled_check(shape_big, prec, nsteps, seed, op=ONE, dt=0.5, mean=-0.25, small=64):
    """Step a field that repeats a random small^d block: the result must repeat the oracle's
    small^d result (compared slab by slab on the device, after the plan is released)."""
    b = _binding()
    nd = len(shape_big)
    sm_shape = (small,) * nd
    psi_s = inputs.uniform_state(sm_shape, mean, 0.05, seed=seed)
    ref_s = oracle.step(psi_s, DX, dt, op, nsteps)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    reps = tuple(n // small for n in shape_big)
    p = b.Plan(shape_big, DX, dt, [b.make_op(*op)], precision=prec)
    info = p.info()
    x = torch.from_numpy(psi_s).to(device="cuda", dtype=dtype).repeat(*reps)
    p.step(x, nsteps)
    torch.cuda.synchronize()
    p.close()
    tgt = torch.from_numpy(ref_s).to(device="cuda", dtype=torch.float64).repeat(1, *reps[1:])
    err2, ref2 = 0.0, 0.0
    for z0 in range(0, shape_big[0], small):
        d = x[z0:z0 + small].double() - tgt
        err2 += float((d * d).sum())
        ref2 += float((tgt * tgt).sum())
        del d
    del x, tgt
    torch.cuda.empty_cache()
    return info, math.sqrt(err2 / ref2)


def _modes_check(shape, prec, nsteps, op=ONE, dt=0.5, mean=-0.25, amp=1e-6, nmodes=3, seed=29, slab=16):
    """A few small Fourier modes of random wavevector on a uniform background. Returns the largest
    relative error of their projected amplitudes against the closed-form factor g^nsteps, and the
    relative size of what is left after removing them (the O(amp^2) sum and difference modes)."""
    b = _binding()
    dtype = torch.float64 if prec == "fp64" else torch.float32
    nd = len(shape)
    rng = np.random.default_rng(seed)
    modes = []
    for _ in range(nmodes):
        # |q| per axis at most ~0.6 (|q|^2 <= ~1.1 in 3D): modes near the PFC band, not damped to
        # nothing in three steps (a mode at |q|^2 ~ 10 shrinks by ~500 a step, and its relative
        # error would then measure rounding of a vanishing amplitude)
        mmax = [max(2, min(40, int(0.6 * n * DX / (2 * math.pi)))) for n in shape]
        m = [int(rng.integers(1, mm + 1)) * (1 if rng.random() < 0.5 else -1) for mm in mmax]
        phase = float(rng.random() * 2 * math.pi)
        q2 = sum((2 * math.pi * mi / (n * DX)) ** 2 for mi, n in zip(m, shape))
        g = (1 - 3 * mean * mean * dt * q2) / (1 + dt * q2 * oracle.lin_op(op, q2))
        modes.append((m, phase, g))
    axes = [torch.arange(n, device="cuda", dtype=torch.float64) for n in shape]

    def cosine(j, z0, z1):
        m, phase, _ = modes[j]
        arg = torch.full((1,) * nd, phase, dtype=torch.float64, device="cuda")
        for d in range(nd):
            view = [1] * nd
            view[d] = shape[d] if d else z1 - z0
            ax = axes[d] if d else axes[0][z0:z1]
            arg = arg + (2 * math.pi * m[d] / shape[d]) * ax.view(view)
        return torch.cos(arg)

    p = b.Plan(shape, DX, dt, [b.make_op(*op)], precision=prec)
    x = torch.empty(shape, dtype=dtype, device="cuda")
    for z0 in range(0, shape[0], slab):
        z1 = min(shape[0], z0 + slab)
        f = torch.full_like(x[z0:z1], mean, dtype=torch.float64)
        for j in range(nmodes):
            f += amp * cosine(j, z0, z1)
        x[z0:z1] = f.to(dtype)
    p.step(x, nsteps)
    torch.cuda.synchronize()
    p.close()
    n = float(np.prod(shape))
    proj = [0.0] * nmodes
    for z0 in range(0, shape[0], slab):   # amplitudes: (2/N) sum (psi - mean) cos_j
        z1 = min(shape[0], z0 + slab)
        f = x[z0:z1].double() - mean
        for j in range(nmodes):
            proj[j] += 2.0 / n * float((f * cosine(j, z0, z1)).sum())
    rest2, sig2 = 0.0, 0.0
    for z0 in range(0, shape[0], slab):
        z1 = min(shape[0], z0 + slab)
        f = x[z0:z1].double() - mean
        e = torch.zeros_like(f)
        for j in range(nmodes):
            f -= proj[j] * cosine(j, z0, z1)
            e += amp * modes[j][2] ** nsteps * cosine(j, z0, z1)
        rest2 += float((f * f).sum())
        sig2 += float((e * e).sum())
    del x
    torch.cuda.empty_cache()
    amp_err = max(abs(proj[j] - amp * modes[j][2] ** nsteps) / abs(amp * modes[j][2] ** nsteps)
                  for j in range(nmodes))
    return amp_err, math.sqrt(rest2 / sig2)


def test_modes_closed_form_on_a_small_grid():
    """The closed-form check itself, on a grid the oracle also steps (pins the helper)."""
    amp_err, rest = _modes_check((64, 64, 64), "fp64", 3)
    assert amp_err <= 1e-9 and rest <= 1e-4


def test_1024cube_fp64_three_pass_tiled_and_modes():
    info, err = _tiled_check((1024, 1024, 1024), "fp64", 3, seed=31)
    assert info["Ry"] * info["Rz"] > 1
    assert err <= 1e-11
    # linear regime, amplitude 1e-6: the mode amplitudes to O(amp^2), the other modes O(amp)
    amp_err, rest = _modes_check((1024, 1024, 1024), "fp64", 3)
    assert amp_err <= 1e-9 and rest <= 1e-4


def test_2048cube_fp32_three_pass_tiled_and_modes():
    """The largest power-of-two cube that fits one GB300 (about 140 GB with the state)."""
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 150e9:
        pytest.skip(f"needs about 150 GB of free device memory, {free / 1e9:.0f} GB free")
    info, err = _tiled_check((2048, 2048, 2048), "fp32", 3, seed=37, small=128)
    assert info["Ry"] * info["Rz"] > 1
    assert err <= 1e-5
    # FP32, amplitude 1e-3: the amplitudes to ~1e-5 (rounding of the FP32 transforms relative to
    # the fluctuation) plus O(amp^2 / mean^2)
    amp_err, rest = _modes_check((2048, 2048, 2048), "fp32", 3, amp=1e-3, slab=8)
    assert amp_err <= 1e-4 and rest <= 1e-2


@pytest.mark.parametrize("shape,tile", [((64, 32, 1024), "4,8,4"), ((64, 16, 2048), "2,8,4"),
                                        ((64, 64, 1024), "4,8,4,2,1")])
def test_clustered_3d_row_pass_at_longer_rows(monkeypatch, shape, tile):
    """The 3D psi^3 row pass on two-block clusters at row lengths M = 512 and 1024 (the large
    three-pass grids use it), two-pass and three-pass tilings, FP32-mixed against the oracle."""
    b = _binding()
    monkeypatch.setenv("PFC_TILE", tile)
    p = b.Plan(shape, DX, 0.1, [b.make_op(*TWO3)], precision="fp32")
    assert p.info()["row_cluster"] == 2
    psi0 = inputs.uniform_state(shape, -0.35, 0.05, seed=79)
    x = to_dev(psi0, "fp32")
    p.step(x, 20)
    assert rel(x.double().cpu().numpy(), oracle.step(psi0, DX, 0.1, TWO3, 20)) <= 1e-5
    p.close()

"""GPU parity of the hydrodynamic PFC step (pfc_hydro_*) against the oracle's hydro_step, FP64
(1e-11 after 5 steps) and FP32-mixed (1e-5), 2D and 3D, including a forced three-pass tiling of
the transforms, and its reduction to the plain step when the velocity cannot respond."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_26818_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DX = math.pi / 4
ONE = (0, -0.25, 0.0, 0.0)
TWO = (1, -0.3, 0.05, math.sqrt(4.0 / 3.0))
TOL = {"fp64": 1e-11, "fp32": 1e-5}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _state(shape, seed):
    psi = inputs.uniform_state(shape, -0.25, 0.1, seed=seed)
    v = 0.05 * np.stack([inputs.uniform_state(shape, 0.0, 1.0, seed=seed + 1 + j) for j in range(len(shape))])
    return psi, v


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,op,dt", [((32, 64), ONE, 0.5), ((16, 32, 32), TWO, 0.1)])
def test_hydro_matches_oracle(shape, op, dt, prec):
    from paper_2603_26818_gb300 import binding
    dtype = torch.float64 if prec == "fp64" else torch.float32
    psi0, v0 = _state(shape, 91)
    if prec == "fp32":   # one FP32-representable start for both sides
        psi0, v0 = psi0.astype(np.float32).astype(np.float64), v0.astype(np.float32).astype(np.float64)
    h = binding.Hydro(shape, DX, dt, op, rho=1.3, gamma=0.8, a0=2.0, precision=prec)
    psi = torch.from_numpy(psi0).to(device="cuda", dtype=dtype)
    v = torch.from_numpy(v0).to(device="cuda", dtype=dtype)
    h.step(psi, v, 5)
    ref_p, ref_v = oracle.hydro_step(psi0, v0, DX, dt, op, 1.3, 0.8, 2.0, 5)
    assert rel(psi.double().cpu().numpy(), ref_p) <= TOL[prec]
    assert rel(v.double().cpu().numpy(), ref_v) <= TOL[prec] * 10
    h.close()


def test_hydro_on_a_three_pass_tiling(monkeypatch):
    from paper_2603_26818_gb300 import binding
    monkeypatch.setenv("PFC_TILE", "2,2,4,4,2")
    shape = (32, 64, 32)
    psi0, v0 = _state(shape, 93)
    h = binding.Hydro(shape, DX, 0.1, TWO, rho=1.0, gamma=1.0, a0=2.0, precision="fp64")
    psi = torch.from_numpy(psi0).cuda()
    v = torch.from_numpy(v0).cuda()
    h.step(psi, v, 3)
    ref_p, ref_v = oracle.hydro_step(psi0, v0, DX, 0.1, TWO, 1.0, 1.0, 2.0, 3)
    assert rel(psi.cpu().numpy(), ref_p) <= 1e-11 and rel(v.cpu().numpy(), ref_v) <= 1e-10
    h.close()


def test_hydro_without_velocity_response_is_the_plain_step():
    from paper_2603_26818_gb300 import binding
    shape = (64, 64)
    psi0 = inputs.uniform_state(shape, -0.25, 0.1, seed=95)
    h = binding.Hydro(shape, DX, 0.5, ONE, rho=math.inf, gamma=1.0, a0=2.0, precision="fp64")
    psi = torch.from_numpy(psi0).cuda()
    v = torch.zeros((2,) + shape, dtype=torch.float64, device="cuda")
    h.step(psi, v, 6)
    p = binding.Plan(shape, DX, 0.5, [binding.make_op(*ONE)], precision="fp64")
    x = torch.from_numpy(psi0).cuda()
    p.step(x, 6)
    assert rel(psi.cpu().numpy(), x.cpu().numpy()) <= 1e-12
    assert float(v.abs().max()) == 0.0
    h.close()
    p.close()

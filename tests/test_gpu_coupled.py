"""GPU parity of the coupled density/composition pair against the oracle's Cramer-rule step.

Tolerances as for one field: FP64 1e-11 after 10 steps, FP32-mixed 1e-5; masses conserved to
1e-6 relative (FP64 carried means); energy density to 1e-10 (FP64) and 1e-6 (FP32).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_26818_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OPP = (0, -0.25, 0.0, 0.0)
OPC = (0, -0.2, 0.0, 0.0)
OPC2 = (1, -0.3, 0.05, math.sqrt(4.0 / 3.0))


def _pair(shape, seed):
    p = inputs.uniform_state(shape, -0.25, 0.05, seed=seed)
    c = inputs.uniform_state(shape, -0.2, 0.05, seed=seed + 1)
    return p, c


def _plan(shape, dt, ops, prec, alpha):
    from paper_2603_26818_gb300 import binding
    return binding.Plan(shape, math.pi / 4, dt, [binding.make_op(*o) for o in ops], precision=prec,
                        coupling=alpha)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
@pytest.mark.parametrize("shape,opc,dt", [((64, 128), OPC, 0.5), ((16, 32, 32), OPC2, 0.1),
                                          ((2048, 32), OPC, 0.5)])
def test_coupled_steps_match_oracle(shape, opc, dt, prec, tol):
    alpha, nsteps = 0.1, 10
    p0, c0 = _pair(shape, 61)
    rp, rc = oracle.step2(p0, c0, math.pi / 4, dt, OPP, opc, alpha, nsteps)
    pl = _plan(shape, dt, [OPP, opc], prec, alpha)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    x = torch.from_numpy(np.stack([p0, c0])).to(device="cuda", dtype=dtype)
    pl.step(x, nsteps)
    got = x.double().cpu().numpy()
    assert rel(got[0], rp) <= tol and rel(got[1], rc) <= tol
    m = pl.mass(x)
    assert abs(m[0] - oracle.mass(p0)) <= 1e-6 * abs(oracle.mass(p0))
    assert abs(m[1] - oracle.mass(c0)) <= 1e-6 * abs(oracle.mass(c0))
    e_ref = oracle.energy2(got[0], got[1], math.pi / 4, OPP, opc, alpha)
    assert pl.energy(x) == pytest.approx(e_ref, rel=1e-10 if prec == "fp64" else 1e-6)


def test_zero_coupling_equals_two_single_field_runs():
    from paper_2603_26818_gb300 import binding
    shape, dt = (64, 64), 0.5
    p0, c0 = _pair(shape, 63)
    pl = _plan(shape, dt, [OPP, OPC], "fp64", 0.0)
    x = torch.from_numpy(np.stack([p0, c0])).cuda()
    pl.step(x, 20)
    ref = []
    for f0, op in ((p0, OPP), (c0, OPC)):
        s = binding.Plan(shape, math.pi / 4, dt, [binding.make_op(*op)], precision="fp64")
        y = torch.from_numpy(f0).cuda()
        s.step(y, 20)
        ref.append(y.cpu().numpy())
    got = x.cpu().numpy()
    assert rel(got[0], ref[0]) <= 1e-13 and rel(got[1], ref[1]) <= 1e-13


def test_coupled_long_single_call_matches_oracle():
    shape, dt, alpha, nsteps = (64, 64), 0.5, 0.1, 3000
    p0, c0 = _pair(shape, 65)
    rp, rc = oracle.step2(p0, c0, math.pi / 4, dt, OPP, OPC, alpha, nsteps)
    pl = _plan(shape, dt, [OPP, OPC], "fp64", alpha)
    x = torch.from_numpy(np.stack([p0, c0])).cuda()
    pl.step(x, nsteps)
    got = x.cpu().numpy()
    assert np.isfinite(got).all()
    assert rel(got[0], rp) <= 1e-9 and rel(got[1], rc) <= 1e-9


@pytest.mark.parametrize("shape,opc,dt", [((4096, 4096), OPC, 0.5), ((256, 256, 512), OPC2, 0.1)])
def test_coupled_pair_on_the_clustered_row_passes(shape, opc, dt):
    """Two fields through the clustered psi^3 row passes (2D rows of 4096, 3D rows of 512 with
    Py = Pz = 8): the second field runs as the second row of the launch grid."""
    from paper_2603_26818_gb300 import binding
    alpha, nsteps = 0.1, 2
    p0, c0 = _pair(shape, 67)
    pl = _plan(shape, dt, [OPP, opc], "fp32", alpha)
    assert pl.info()["row_cluster"] == 2
    x = torch.from_numpy(np.stack([p0, c0])).to(device="cuda", dtype=torch.float32)
    pl.step(x, nsteps)
    got = x.double().cpu().numpy()
    pl.close()
    rp, rc = oracle.step2(p0, c0, math.pi / 4, dt, OPP, opc, alpha, nsteps)
    assert rel(got[0], rp) <= 1e-5 and rel(got[1], rc) <= 1e-5

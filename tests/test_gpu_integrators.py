"""GPU parity of the alternative time integrators (pfc_set_integrator) against the oracle's
step_scheme: the stabilised semi-implicit scheme (constant S) and the second-order BDF scheme
with extrapolated nonlinearity, on two-pass and three-pass plans, FP64 (1e-11 after 20 steps)
and FP32-mixed (1e-5). The second-order scheme carries two time levels inside one call, so
step counts are chosen to cover both parities of the final level, the captured graph (16-step
chunks after the direct starting step) and two calls in a row (each call one run)."""
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
TOL = {"fp64": 1e-11, "fp32": 1e-5}


def _binding():
    from paper_2603_26818_gb300 import binding
    return binding


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def to_dev(a, prec):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda",
                                                      dtype=torch.float64 if prec == "fp64" else torch.float32)


CASES = [((64, 128), ONE, 0.5, -0.25), ((32, 16, 64), TWO3, 0.1, -0.35)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme,S", [(1, 0.5), (1, 2.0), (2, 0.0)])
@pytest.mark.parametrize("shape,op,dt,mean", CASES)
def test_scheme_matches_oracle(shape, op, dt, mean, scheme, S, prec):
    b = _binding()
    p = b.Plan(shape, DX, dt, [b.make_op(*op)], precision=prec)
    p.set_integrator(scheme, S)
    psi0 = inputs.uniform_state(shape, mean, 0.05, seed=71)
    for nsteps in (20, 17, 3):
        x = to_dev(psi0, prec)
        p.step(x, nsteps)
        got = x.double().cpu().numpy()
        assert rel(got, oracle.step_scheme(psi0, DX, dt, op, scheme, S, nsteps)) <= TOL[prec], nsteps
        assert abs(p.mass(x)[0] - float(np.mean(psi0.astype(np.float32 if prec == "fp32" else np.float64)))) \
            <= 1e-12 * abs(mean) + (1e-7 if prec == "fp32" else 0)
    p.close()


def test_second_order_scheme_restarts_per_call_and_on_three_pass_tilings(monkeypatch):
    b = _binding()
    shape, op, dt = (32, 64, 32), TWO3, 0.1
    monkeypatch.setenv("PFC_TILE", "2,2,4,4,2")
    p = b.Plan(shape, DX, dt, [b.make_op(*op)], precision="fp64")
    assert p.info()["Ry"] * p.info()["Rz"] > 1
    p.set_integrator(b.PFC_SBDF2)
    psi0 = inputs.uniform_state(shape, -0.35, 0.05, seed=72)
    x = to_dev(psi0, "fp64")
    p.step(x, 33)    # start step, two graph chunks
    p.step(x, 10)    # a new run from the new state
    ref = oracle.step_scheme(oracle.step_scheme(psi0, DX, dt, op, 2, 0.0, 33), DX, dt, op, 2, 0.0, 10)
    assert rel(x.cpu().numpy(), ref) <= 1e-11
    # back to the semi-implicit step
    p.set_integrator(b.PFC_SEMI_IMPLICIT)
    y = to_dev(psi0, "fp64")
    p.step(y, 5)
    assert rel(y.cpu().numpy(), oracle.step(psi0, DX, dt, op, 5)) <= 1e-12
    p.close()


def test_second_order_convergence_on_the_gpu():
    """Halving dt divides the second-order scheme's error at t = 4 by ~4 (smooth initial data)."""
    b = _binding()
    n = 16
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    psi = (-0.3 + 0.1 * np.cos(2 * np.pi * 2 * x / n) + 0.07 * np.cos(2 * np.pi * (2 * y + 2 * x) / n + 0.3)
           + 0.05 * np.sin(2 * np.pi * 3 * y / n))
    op, T = (0, -0.1, 0.0, 0.0), 4.0

    def run(dt):
        p = b.Plan((n, n), DX, dt, [b.make_op(*op)], precision="fp64")
        p.set_integrator(b.PFC_SBDF2)
        z = to_dev(psi, "fp64")
        p.step(z, int(round(T / dt)))
        p.close()
        return z.cpu().numpy()

    ref = run(0.2 / 32)
    errs = [np.linalg.norm(run(dt) - ref) for dt in (0.2, 0.1, 0.05)]
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.2 <= e0 / e1 <= 5.0


def test_integrator_limits():
    b = _binding()
    p = b.Plan((32, 32), DX, 0.5, [b.make_op(0, -0.25), b.make_op(0, -0.2)], precision="fp64", coupling=0.1)
    with pytest.raises(b.PfcError, match="UNSUPPORTED"):
        p.set_integrator(b.PFC_SBDF2)
    p.set_integrator(b.PFC_SEMI_IMPLICIT)
    p.close()
    q = b.Plan((32, 32), DX, 0.5, [b.make_op(*ONE)], precision="fp64")
    q.set_integrator(b.PFC_STABILIZED, 1.0)
    x = to_dev(inputs.uniform_state((32, 32), -0.25, 0.05, seed=73), "fp64")
    out = torch.empty_like(x)
    dr = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(b.PfcError, match="UNSUPPORTED"):
        q.step_adjoint(x, x.clone(), out, dr)
    with pytest.raises(b.PfcError, match="INVALID_ARG"):
        q.set_integrator(7)
    with pytest.raises(b.PfcError, match="INVALID_ARG"):
        q.set_integrator(b.PFC_STABILIZED, -1.0)
    q.close()

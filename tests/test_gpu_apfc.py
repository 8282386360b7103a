"""GPU amplitude-expansion PFC (pfc_apfc_*) against the oracle (oracle/apfc.py, pinned in
test_oracle_apfc.py): a 2D triangular triad and a 3D BCC set of six amplitudes, one- and
two-mode operators, FP64 (1e-11 after 5 steps) and FP32-mixed (1e-5), mixed-radix extents, the
middle (negative-frequency) bin, the resonance count; at a full size the oracle on a 1024^2
triad and translation covariance (a property at any size) on the bench's 256^3 BCC set.
"""
import math

import numpy as np
import pytest

from oracle import apfc as oapfc
from paper_2603_26818_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP1 = (0, -0.25, 0.0, 0.0)
OP2 = (1, -0.3, 0.05, math.sqrt(4.0 / 3.0))
TOL = {"fp64": 1e-11, "fp32": 1e-5}


def _model(shape, kv, psibar, op, prec, dx=0.9, dt=0.3):
    from paper_2603_26818_gb300 import binding
    return binding.Apfc(shape, dx, dt, op, kv, psibar, precision=prec)


def _eta(namp, shape, seed, prec):
    e = inputs.apfc_amplitudes(namp, shape, 0.1, 0.02, seed)
    if prec == "fp32":
        e = e.astype(np.complex64).astype(np.complex128)
    return e


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,kind,psibar,op", [((48, 60), "triad", -0.3, OP1), ((30, 64), "triad", 0.1, OP2),
                                                  ((12, 20, 18), "bcc", -0.2, OP1), ((16, 14, 10), "bcc", 0.15, OP2),
                                                  ((15, 21), "single", -0.1, OP1), ((8, 8, 8), "bcc", 0.0, OP1),
                                                  ((14, 49), "pair", 0.2, OP2)])
def test_apfc_matches_oracle(shape, kind, psibar, op, prec):
    """Edge cases among them: odd extents (15 x 21, 7^2), the smallest extent (8), one amplitude
    (no cross resonance), two opposite-free vectors (no resonance beyond the self terms)."""
    kv = {"triad": inputs.apfc_triad(1.0), "bcc": inputs.apfc_bcc(1.0), "single": [(1.0, 0.0)],
          "pair": [(1.0, 0.0), (0.0, 1.0)]}[kind]
    eta = _eta(len(kv), shape, 21, prec)
    m = _model(shape, kv, psibar, op, prec)
    x = torch.from_numpy(eta).to(device="cuda", dtype=m.dtype)
    m.step(x, 5)
    ref = oapfc.step(eta, kv, psibar, 0.9, 0.3, op, 5)
    assert rel(x.cpu().numpy().astype(np.complex128), ref) <= TOL[prec]
    pairs, triples = oapfc.resonances(kv)
    assert m.resonances() == sum(len(p) + len(t) for p, t in zip(pairs, triples))
    m.close()


def test_apfc_middle_bin_is_the_negative_frequency():
    """A plane wave in one amplitude at the middle index of both axes (wavevector -pi/dx per axis)
    against the oracle, whose convention is pinned by the closed-form factor."""
    shape, kv = (16, 32), inputs.apfc_triad(1.0)
    yy, xx = np.meshgrid(np.arange(16), np.arange(32), indexing="ij")
    eta = np.zeros((3,) + shape, dtype=np.complex128)
    eta[0] = 1e-3 * np.exp(1j * math.pi * (yy + xx))
    # dt small enough that the mode (Q = |k_1 + q|^2 ~ 35, L(Q) ~ 1.1e3) keeps a measurable size;
    # with +pi/dx the factor would be that of Q ~ 16 instead
    m = _model(shape, kv, -0.25, OP1, "fp64", dt=0.01)
    x = torch.from_numpy(eta).cuda()
    m.step(x, 2)
    ref = oapfc.step(eta, kv, -0.25, 0.9, 0.01, OP1, 2)
    assert rel(x.cpu().numpy(), ref) <= 1e-12


def test_apfc_1024sq_triad_fp32_matches_oracle():
    shape, kv = (1024, 1024), inputs.apfc_triad(1.0)
    eta = _eta(3, shape, 31, "fp32")
    m = _model(shape, kv, -0.3, OP1, "fp32", dx=1.2, dt=0.5)
    x = torch.from_numpy(eta).to(device="cuda", dtype=torch.complex64)
    m.step(x, 4)
    ref = oapfc.step(eta, kv, -0.3, 1.2, 0.5, OP1, 4)
    assert rel(x.cpu().numpy().astype(np.complex128), ref) <= 1e-5
    m.close()


def test_apfc_256cube_bcc_translation_covariance_fp32():
    """At the bench's size and launch configuration (BCC, 256^3, dx 1.1, dt 0.4): translating the
    density by u multiplies eta_j by exp(i k_j . u); the step commutes with it (both orders from
    the same FP32 start, 3 steps, 1e-5)."""
    shape, kv = (256, 256, 256), inputs.apfc_bcc(1.0)
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    x = (0.1 + 0.02 * (2 * torch.rand((6,) + shape, generator=g, device="cuda", dtype=torch.float32) - 1)).to(torch.complex64)
    x = x + 0.02j * (2 * torch.rand((6,) + shape, generator=g, device="cuda", dtype=torch.float32) - 1)
    u = np.array([0.7, -1.3, 2.1])
    ph = torch.tensor(np.exp(1j * (np.asarray(kv) @ u)), dtype=torch.complex64, device="cuda").view(6, 1, 1, 1)
    m = _model(shape, kv, -0.2, OP1, "fp32", dx=1.1, dt=0.4)
    a = x * ph
    b = x.clone()
    m.step(a, 3)
    m.step(b, 3)
    b = b * ph
    assert float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) <= 1e-5
    m.close()

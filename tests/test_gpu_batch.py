"""GPU batched ensemble: every domain of a packed batch against its own single-domain plan and
against the oracle; masses per domain; the graph-captured chunked path against direct steps.

Workload recipe for the full-size case: 1024 domains with ny, nx drawn from {64,128,256,512},
r ~ U[-0.4, -0.1], mean ~ U[-0.4, -0.2], noise U[-0.01, 0.01], dt = 0.5, dx = pi/4 (seed 4).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_26818_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DX = math.pi / 4


def _batch(draws, prec, dt=0.5):
    from paper_2603_26818_gb300 import binding
    dims = [(d[0], d[1]) for d in draws]
    return binding.Batch(dims, [d[2] for d in draws], DX, dt, precision=prec)


def _state(b, draws, seed, dtype):
    parts = [inputs.uniform_state((ny, nx), m, 0.01, seed=seed + i).ravel()
             for i, (ny, nx, r, m) in enumerate(draws)]
    return torch.from_numpy(np.concatenate(parts)).to(device="cuda", dtype=dtype), parts


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_batch_domains_match_oracle(prec, tol):
    draws = [(32, 64, -0.25, -0.25), (64, 32, -0.3, -0.3), (32, 64, -0.15, -0.22), (16, 16, -0.35, -0.4),
             (128, 64, -0.2, -0.35)]
    b = _batch(draws, prec)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    x, parts = _state(b, draws, 100, dtype)
    b.step(x, 20)   # >= 16: the graph-captured path
    for d, (ny, nx, r, m) in enumerate(draws):
        ref = oracle.step(parts[d].reshape(ny, nx), DX, 0.5, (0, r, 0.0, 0.0), 20)
        assert rel(b.view(x, d).double().cpu().numpy(), ref) <= tol
    ms = b.mass(x)
    for d, p in enumerate(parts):
        assert abs(ms[d] - p.mean()) <= 1e-6 * abs(p.mean())


def test_batch_matches_single_plans_and_graph_path_matches_direct_steps():
    from paper_2603_26818_gb300 import binding
    draws = inputs.batch_draws(24, seed=7, sizes=(64, 128, 256))
    b = _batch(draws, "fp64")
    x, parts = _state(b, draws, 200, torch.float64)
    y = x.clone()
    b.step(x, 35)                       # two graph chunks + 3 direct steps
    for _ in range(35):
        b.step(y, 1)                    # direct steps only
    assert rel(x.cpu().numpy(), y.cpu().numpy()) <= 1e-12
    for d, (ny, nx, r, m) in enumerate(draws):
        p = binding.Plan((ny, nx), DX, 0.5, [binding.make_op(0, r)], precision="fp64")
        z = torch.from_numpy(parts[d].reshape(ny, nx)).cuda()
        p.step(z, 35)
        assert rel(b.view(x, d).cpu().numpy(), z.cpu().numpy()) <= 1e-12
        p.close()


def test_full_ensemble_1024_domains_fp32():
    """1024 domains of {64..512}^2 (about 5.9e7 points), 200 steps, FP32-mixed on autotuned
    tiles: every domain against the FP64 batch of the same ensemble (the FP64 batch is pinned to
    the oracle and to single-domain plans above), and every domain's mass conserved."""
    draws = inputs.batch_draws(1024, seed=4)
    b = _batch(draws, "fp32")
    b.autotune(6, 8)          # the tiles the bench times this workload on
    x, parts = _state(b, draws, 1000, torch.float32)
    y = x.double()            # the FP64 run starts from the same FP32-representable fields
    yin, _ = _state(b, draws, 1000, torch.float64)   # and from the FP64 draws (input rounding included)
    b.step(x, 200)
    assert bool(torch.isfinite(x).all())
    ms = b.mass(x)
    b64 = _batch(draws, "fp64")
    b64.step(y, 200)
    b64.step(yin, 200)

    def errs_to(ref):
        return np.array([float((b.view(x, d).double() - b64.view(ref, d)).norm() / b64.view(ref, d).norm())
                         for d in range(len(draws))])
    errs, errs_in = errs_to(y), errs_to(yin)
    worst = int(errs.argmax())
    print(f"1024-domain ensemble, 200 steps, FP32 vs FP64 from the same start: max rel L2 {errs.max():.3e} "
          f"(domain {worst}, {draws[worst]}), median {np.median(errs):.3e}; against the FP64 draws: max "
          f"{errs_in.max():.3e}, above 1e-5: {int((errs_in > 1e-5).sum())}")
    assert errs.max() <= 1e-5
    for d, p in enumerate(parts):
        assert abs(ms[d] - p.astype(np.float32).astype(np.float64).mean()) <= 1e-6 * abs(p.mean())
    b.close()
    b64.close()

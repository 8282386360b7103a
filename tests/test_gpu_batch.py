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
    tiles: every domain against the FP64 batch of the same ensemble from the same
    FP32-representable start (the FP64 batch is pinned to the oracle and to single-domain plans
    above), and every domain's mass conserved.

    Bound: 1e-5 relative L2 for every linearly stable domain (r + 3 mean^2 >= 0). Domains with
    r + 3 mean^2 < 0 are linearly unstable (growth rate up to -(r + 3 mean^2) at k = 1) and
    crystallise from the noise within ~50 steps; the FP32 rounding that enters at every step of
    that growth phase is amplified with the unstable modes (the error-vs-step curve of the next
    test), so they are held to 1e-4, and the median over all domains to 1e-6. For scale, the
    FP64 batch is also run from its start perturbed once by 6e-8 of the fluctuation (reported)."""
    draws = inputs.batch_draws(1024, seed=4)
    b = _batch(draws, "fp32")
    b.autotune(6, 8)          # the tiles the bench times this workload on
    x, parts = _state(b, draws, 1000, torch.float32)
    y = x.double()            # the FP64 run starts from the same FP32-representable fields
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    u = torch.empty_like(y).uniform_(-1.0, 1.0, generator=g)
    yp = y + 6e-8 * 0.01 * u  # a perturbation of FP32 rounding size of the 0.01 fluctuation
    b.step(x, 200)
    assert bool(torch.isfinite(x).all())
    ms = b.mass(x)
    b64 = _batch(draws, "fp64")
    b64.step(y, 200)
    b64.step(yp, 200)

    def rel_to(a_state, a_batch, ref):
        return np.array([float((a_batch.view(a_state, d).double() - b64.view(ref, d)).norm() / b64.view(ref, d).norm())
                         for d in range(len(draws))])
    errs = rel_to(x, b, y)
    sens = rel_to(yp, b64, y)
    worst = int(errs.argmax())
    unstable = np.array([r + 3 * m * m < 0 for (_, _, r, m) in draws])
    print(f"1024-domain ensemble, 200 steps, FP32 vs FP64 from the same start: max rel L2 {errs.max():.3e} "
          f"(domain {worst}, {draws[worst]}), median {np.median(errs):.3e}; above 1e-5: {int((errs > 1e-5).sum())} "
          f"(all linearly unstable: {bool(unstable[errs > 1e-5].all())}); FP64 sensitivity to eps32 at the "
          f"worst domain {sens[worst]:.3e}, max {sens.max():.3e}")
    assert (errs[~unstable] <= 1e-5).all()
    assert (errs <= 1e-4).all()
    assert np.median(errs) <= 1e-6
    for d, p in enumerate(parts):
        assert abs(ms[d] - p.astype(np.float32).astype(np.float64).mean()) <= 1e-6 * abs(p.mean())
    b.close()
    b64.close()


def test_error_versus_step_of_the_most_unstable_domain():
    """The FP32-vs-FP64 error curve of the ensemble's most unstable domain, single-domain plans
    from the same FP32-representable start (printed; reported in the design notes): it grows
    with the unstable modes while the pattern forms, then levels off."""
    from paper_2603_26818_gb300 import binding
    draws = inputs.batch_draws(1024, seed=4)
    d = int(np.argmin([r + 3 * m * m for (_, _, r, m) in draws]))
    ny, nx, r, m = draws[d]
    psi0 = inputs.uniform_state((ny, nx), m, 0.01, seed=1000 + d).astype(np.float32)
    p32 = binding.Plan((ny, nx), DX, 0.5, [binding.make_op(0, r)], precision="fp32")
    p64 = binding.Plan((ny, nx), DX, 0.5, [binding.make_op(0, r)], precision="fp64")
    a = torch.from_numpy(psi0).cuda()
    c = a.double()
    curve, done = [], 0
    for n in (1, 2, 5, 10, 20, 50, 100, 200):
        p32.step(a, n - done)
        p64.step(c, n - done)
        done = n
        curve.append((n, float((a.double() - c).norm() / c.norm())))
    print(f"domain {d} {draws[d]}: r + 3 mean^2 = {r + 3 * m * m:.3f}; FP32 vs FP64 rel L2 by step: "
          + ", ".join(f"{n}: {e:.2e}" for n, e in curve))
    assert curve[0][1] <= 1e-6   # one step: the arithmetic alone
    p32.close()
    p64.close()


def test_onchip_classes_match_the_two_pass_path(monkeypatch):
    """Domains of at most 128 x 128 step in shared memory (one launch per call, every step on
    chip); the same batch with PFC_ONCHIP=0 steps every class through the two-pass path: FP64
    results agree to rounding, in both orders of calls (on-chip classes run beside the graph)."""
    draws = [(64, 64, -0.3, -0.3), (128, 64, -0.25, -0.25), (64, 128, -0.2, -0.3), (16, 32, -0.35, -0.4),
             (128, 128, -0.3, -0.28), (256, 64, -0.25, -0.25), (128, 256, -0.15, -0.3)]
    b = _batch(draws, "fp64")
    info = b.info()
    onchip = {(c["ny"], c["nx"]) for c in info if c["Py"] == 0}
    # FP64 128 x 128 (two half spectra of 328 KB) does not fit one block's shared memory
    assert onchip == {(64, 64), (128, 64), (64, 128), (16, 32)}
    x, parts = _state(b, draws, 300, torch.float64)
    y = x.clone()
    b.step(x, 21)
    b.step(x, 7)
    monkeypatch.setenv("PFC_ONCHIP", "0")
    b2 = _batch(draws, "fp64")
    assert all(c["Py"] > 0 for c in b2.info())
    b2.step(y, 21)
    b2.step(y, 7)
    for d in range(len(draws)):
        assert rel(b.view(x, d).cpu().numpy(), b2.view(y, d).cpu().numpy()) <= 1e-12
    ref = oracle.step(parts[4].reshape(128, 128), DX, 0.5, (0, -0.3, 0.0, 0.0), 28)
    assert rel(b.view(x, 4).cpu().numpy(), ref) <= 1e-11
    b.close()
    b2.close()

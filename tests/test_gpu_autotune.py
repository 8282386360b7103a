"""GPU: the autotuner and the tilings it may choose.

  * Every tiling the autotuner may time (the planner's candidates, forced one at a time with
    PFC_TILE) gives the oracle's result: the y/z split between the passes,
    the tile width and the row-group packing change the order of the arithmetic only.
  * pfc_plan_autotune picks one of them, the plan then steps within the parity tolerances, and
    a cache file written by one call is applied by the next without timing.
  * pfc_batch_autotune retiles every size class; the domains still match the oracle.
  * Plans of different sizes coexist: a plan created later with smaller tiles does not lower
    the kernels' shared-memory limits below what an earlier plan launches with.
"""
import json
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


def _binding():
    from paper_2603_26818_gb300 import binding
    return binding


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(a, prec):
    return torch.from_numpy(np.ascontiguousarray(a)).to(
        device="cuda", dtype=torch.float64 if prec == "fp64" else torch.float32)


def _plan(shape, dt, op, prec):
    b = _binding()
    return b.Plan(shape, DX, dt, [b.make_op(*op)], precision=prec)


@pytest.mark.parametrize("shape,op,dt,prec", [
    ((64, 128), ONE, 0.5, "fp64"),
    ((16, 32, 64), TWO, 0.1, "fp32"),
    ((128, 128), ONE, 0.5, "fp32"),
])
def test_every_candidate_tiling_matches_oracle(shape, op, dt, prec, monkeypatch):
    b = _binding()
    nsteps = 6
    psi0 = inputs.uniform_state(shape, -0.3, 0.05, seed=11)
    ref = oracle.step(psi0, DX, dt, op, nsteps)
    nz = shape[0] if len(shape) == 3 else 1
    vb = 16 if prec == "fp64" else 8
    tried, bad = [], []
    for py in (1, 2, 4, 8):
        for pz in ((1, 2, 4, 8) if nz > 1 else (1,)):
            for w in (1, 2, 4, 8):
                if w * vb > 64:
                    continue
                monkeypatch.setenv("PFC_TILE", f"{py},{pz},{w}")
                try:
                    p = _plan(shape, dt, op, prec)
                except b.PfcError:
                    continue   # not a valid tiling of this grid
                info = p.info()
                assert (info["Py"], info["Pz"], info["W"]) == (py, pz, w)
                x = to_dev(psi0, prec)
                p.step(x, nsteps)
                err = rel(x.double().cpu().numpy(), ref)
                tried.append((py, pz, w))
                if err > TOL[prec]:
                    bad.append(((py, pz, w), err))
                p.close()
    monkeypatch.delenv("PFC_TILE")
    assert len(tried) >= 8
    assert not bad, bad


@pytest.mark.parametrize("shape,op,dt,prec", [
    ((256, 256), ONE, 0.5, "fp32"),
    ((64, 128), TWO, 0.1, "fp64"),
    ((32, 32, 32), TWO, 0.1, "fp32"),
])
def test_autotuned_plan_matches_oracle(shape, op, dt, prec):
    p = _plan(shape, dt, op, prec)
    before = p.info()
    ms = p.autotune(max_candidates=6, trial_steps=4)
    assert 0.0 < ms < 1e3
    after = p.info()
    assert after["Py"] * after["Qy"] == shape[-2]
    psi0 = inputs.uniform_state(shape, -0.3, 0.05, seed=12)
    x = to_dev(psi0, prec)
    p.step(x, 10)
    assert rel(x.double().cpu().numpy(), oracle.step(psi0, DX, dt, op, 10)) <= TOL[prec]
    # the adjoint still runs on the retuned plan (its arrays are re-allocated for the tiling)
    if before["threads_line"] <= 512:
        lam = to_dev(np.ones(shape), prec)
        out = torch.empty_like(lam)
        dr = torch.zeros(1, dtype=torch.float64, device="cuda")
        p.step_adjoint(x, lam, out, dr)
        p.sync()
        assert torch.isfinite(out).all()
    p.close()


def test_autotune_cache_round_trip(tmp_path):
    cache = tmp_path / "tiles.jsonl"
    p = _plan((128, 256), 0.5, ONE, "fp32")
    ms = p.autotune(max_candidates=4, trial_steps=4, cache=str(cache))
    chosen = p.info()
    lines = cache.read_text().splitlines()
    assert len(lines) == 1
    entry = json.loads(lines[0])
    assert (entry["Py"], entry["W"]) == (chosen["Py"], chosen["W"])
    assert entry["key"].startswith("1x128x256 prec1 fields1 ")
    p.close()
    q = _plan((128, 256), 0.5, ONE, "fp32")
    assert q.autotune(max_candidates=4, trial_steps=4, cache=str(cache)) == pytest.approx(ms, abs=2e-6)
    assert len(cache.read_text().splitlines()) == 1   # applied, not timed again
    got = q.info()
    assert (got["Py"], got["W"], got["row_cluster"]) == (chosen["Py"], chosen["W"], chosen["row_cluster"])
    q.close()


def test_batch_autotune_keeps_parity():
    b = _binding()
    draws = [(32, 64, -0.25, -0.25), (64, 32, -0.3, -0.3), (128, 64, -0.2, -0.35), (16, 16, -0.35, -0.4),
             (64, 256, -0.15, -0.22)]
    batch = b.Batch([(d[0], d[1]) for d in draws], [d[2] for d in draws], DX, 0.5, precision="fp32")
    parts = [inputs.uniform_state((ny, nx), m, 0.01, seed=300 + i).ravel()
             for i, (ny, nx, r, m) in enumerate(draws)]
    x = torch.from_numpy(np.concatenate(parts)).to(device="cuda", dtype=torch.float32)
    batch.step(x, 16)                    # captures the graph of the planner's tiling
    ms = batch.autotune(max_candidates=4, trial_steps=4)
    assert 0.0 < ms < 1e3
    x = torch.from_numpy(np.concatenate(parts)).to(device="cuda", dtype=torch.float32)
    batch.step(x, 20)                    # a new graph on the tuned tiling
    for d, (ny, nx, r, m) in enumerate(draws):
        ref = oracle.step(parts[d].reshape(ny, nx), DX, 0.5, (0, r, 0.0, 0.0), 20)
        assert rel(batch.view(x, d).double().cpu().numpy(), ref) <= 1e-5
    batch.close()


def test_plans_of_different_sizes_coexist():
    psi0 = inputs.uniform_state((1024, 1024), -0.25, 0.05, seed=13)
    big = _plan((1024, 1024), 0.5, ONE, "fp32")
    x = to_dev(psi0, "fp32")
    big.step(x, 3)
    first = x.cpu().numpy()
    small = _plan((16, 16), 0.5, ONE, "fp32")      # smaller tiles, created later
    y = to_dev(inputs.uniform_state((16, 16), -0.25, 0.05, seed=14), "fp32")
    small.step(y, 3)
    x = to_dev(psi0, "fp32")
    big.step(x, 3)                                  # the big plan's launches still fit
    assert np.array_equal(x.cpu().numpy(), first)
    small.close()
    big.close()

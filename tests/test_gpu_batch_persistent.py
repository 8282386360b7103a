"""GPU batched ensemble on the persistent schedule (one cooperative launch a call): every domain
against the oracle and against the graph schedule, the on-chip / two-pass split inside the
launch, both block sizes, the CUDA-graph replay, the latched non-finite status, and the bounded
grid-barrier wait made to run out (a host-set arrival count that no block can reach) with the
batch usable afterwards.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_26818_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DX = math.pi / 4

# on-chip classes (both extents <= 128), classes with a two-pass tiling of the block size, and
# tall/wide ones that need tiles of up to 128 columns
DRAWS = [(16, 16, -0.35, -0.4), (32, 64, -0.25, -0.25), (64, 64, -0.3, -0.3), (128, 256, -0.2, -0.35),
         (256, 128, -0.15, -0.22), (512, 64, -0.25, -0.3), (16, 512, -0.3, -0.25), (64, 64, -0.2, -0.28),
         (128, 256, -0.35, -0.3)]


def _batch(draws, prec, dt=0.5):
    from paper_2603_26818_gb300 import binding
    return binding.Batch([(d[0], d[1]) for d in draws], [d[2] for d in draws], DX, dt, precision=prec)


def _state(draws, seed, dtype):
    parts = [inputs.uniform_state((ny, nx), m, 0.01, seed=seed + i).ravel()
             for i, (ny, nx, r, m) in enumerate(draws)]
    if dtype == torch.float32:
        parts = [p.astype(np.float32).astype(np.float64) for p in parts]
    return torch.from_numpy(np.concatenate(parts)).to(device="cuda", dtype=dtype), parts


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol,threads,oc_max,n_oc", [("fp64", 1e-12, 128, 0, 1), ("fp32", 1e-5, 128, 0, 1),
                                                          ("fp32", 1e-5, 256, 0, 2), ("fp64", 1e-12, 256, 0, 2),
                                                          ("fp32", 1e-5, 128, 60000, 4)])
def test_persistent_domains_match_oracle(prec, tol, threads, oc_max, n_oc):
    """On chip: the domains without a tiling of the block size (16 x 16, whose tiles hold at most
    16 x 8 values; at 256 threads also 32 x 64, at most 32 x 32 < 8 x 256), and with
    oc_max = 60000 B also the FP32 32 x 64 and 64 x 64 domains."""
    b = _batch(DRAWS, prec)
    b.set_schedule("persistent", threads=threads, onchip_smem_max=oc_max)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    x, parts = _state(DRAWS, 300, dtype)
    b.step(x, 12)
    b.sync()
    info = b.schedule_info()
    assert info["schedule"] == 1 and info["threads"] == threads and info["blocks"] >= 152
    assert info["onchip_items"] == n_oc and info["row_items"] > 0
    for d, (ny, nx, r, m) in enumerate(DRAWS):
        ref = oracle.step(parts[d].reshape(ny, nx), DX, 0.5, (0, r, 0.0, 0.0), 12)
        assert rel(b.view(x, d).double().cpu().numpy(), ref) <= tol, (d, ny, nx)
    ms = b.mass(x)
    for d, p in enumerate(parts):
        assert abs(ms[d] - p.mean()) <= (1e-12 if prec == "fp64" else 1e-6) * abs(p.mean())
    b.close()


def test_persistent_rejects_a_batch_its_blocks_cannot_step():
    """At 512 threads a 16 x 512 domain has no line tile of 8 x 512 values (at most 16 x 128)
    and is too wide to step on chip: UNSUPPORTED, and the batch keeps its graph schedule."""
    from paper_2603_26818_gb300 import binding
    b = _batch(DRAWS, "fp32")
    with pytest.raises(binding.PfcError) as e:
        b.set_schedule("persistent", threads=512)
    assert e.value.status == 2   # PFC_ERR_UNSUPPORTED
    b.set_schedule("graph")
    x, parts = _state(DRAWS, 700, torch.float32)
    b.step(x, 3)
    b.sync()
    ny, nx, r, m = DRAWS[6]
    ref = oracle.step(parts[6].reshape(ny, nx), DX, 0.5, (0, r, 0.0, 0.0), 3)
    assert rel(b.view(x, 6).double().cpu().numpy(), ref) <= 1e-5
    b.close()


def test_persistent_matches_graph_schedule_and_replays():
    """The two schedules on the same FP64 inputs, 40 steps (the graph schedule's chunks and
    remainder steps); the persistent call replayed from its captured graph gives the same
    result as a fresh capture."""
    draws = inputs.batch_draws(40, seed=11, sizes=(64, 128, 256, 512))
    bg = _batch(draws, "fp64")
    bp = _batch(draws, "fp64")
    bp.set_schedule("persistent")
    x, _ = _state(draws, 400, torch.float64)
    y = x.clone()
    z = x.clone()
    bg.step(x, 40)
    bp.step(y, 20)
    bp.step(y, 20)       # same state and step count: the captured graph is replayed
    bp.sync()
    assert rel(y.cpu().numpy(), x.cpu().numpy()) <= 1e-12
    assert bp.schedule_info()["graph"] == 1
    bp.step(z, 40)       # another step count: captured again
    bp.sync()
    assert rel(z.cpu().numpy(), x.cpu().numpy()) <= 1e-12
    bg.close()
    bp.close()


def test_persistent_barrier_wait_runs_out_and_batch_recovers():
    """A barrier that waits for one block more than exist: every wait runs out after the bound,
    the launch returns, pfc_batch_sync reports PFC_ERR_TIMEOUT. With the normal bound the next
    call steps correctly."""
    from paper_2603_26818_gb300 import binding
    draws = [(64, 64, -0.25, -0.25), (128, 256, -0.3, -0.3), (32, 32, -0.2, -0.3)]
    b = _batch(draws, "fp64")
    b.set_schedule("persistent")
    x, parts = _state(draws, 500, torch.float64)
    b.set_wait_limit(0.01, extra_arrivals=1)
    y = x.clone()
    b.step(y, 5)
    with pytest.raises(binding.PfcError) as e:
        b.sync()
    assert e.value.status == 7   # PFC_ERR_TIMEOUT
    b.set_wait_limit(2.0, 0)
    b.step(x, 5)
    b.sync()
    for d, (ny, nx, r, m) in enumerate(draws):
        ref = oracle.step(parts[d].reshape(ny, nx), DX, 0.5, (0, r, 0.0, 0.0), 5)
        assert rel(b.view(x, d).cpu().numpy(), ref) <= 1e-12
    b.close()


def test_persistent_nonfinite_state_is_reported():
    from paper_2603_26818_gb300 import binding
    draws = [(64, 64, -0.25, -0.25), (128, 128, -0.3, -0.3)]
    b = _batch(draws, "fp32")
    b.set_schedule("persistent", onchip_smem_max=1)
    x, _ = _state(draws, 600, torch.float32)
    x[5] = float("nan")
    b.step(x, 2)
    with pytest.raises(binding.PfcError) as e:
        b.sync()
    assert e.value.status == 6   # PFC_ERR_NONFINITE
    b.close()


def test_persistent_full_ensemble_1024_domains_fp32():
    """The 1024-domain ensemble ({64..512}^2, seed 4) on the persistent schedule against the graph
    schedule in FP32 from the same start: the same arithmetic per member on other tilings, so
    they agree to FP32 rounding (1e-5 for the linearly stable domains, whose rounding is not
    amplified; 1e-4 for all, as for the FP32-vs-FP64 bound of the graph schedule), after 50
    steps; masses conserved."""
    draws = inputs.batch_draws(1024, seed=4)
    bg = _batch(draws, "fp32")
    bp = _batch(draws, "fp32")
    bp.set_schedule("persistent")
    x, parts = _state(draws, 4000, torch.float32)
    y = x.clone()
    bg.step(x, 50)
    bp.step(y, 50)
    bp.sync()
    xs, ys = x.double().cpu().numpy(), y.double().cpu().numpy()
    for d, (ny, nx, r, m) in enumerate(draws):
        o = bg.offsets[d]
        a, c = ys[o:o + ny * nx], xs[o:o + ny * nx]
        assert rel(a, c) <= (1e-5 if r + 3 * m * m >= 0 else 1e-4), d
    ms = bp.mass(y)
    for d, p in enumerate(parts):
        assert abs(ms[d] - p.mean()) <= 1e-6 * abs(p.mean())
    bg.close()
    bp.close()


def test_switching_schedules_keeps_the_graph_schedule_valid():
    """The graph schedule captures its graph at a call of 16 or more steps; setting the persistent
    schedule may give the classes larger arrays (its tiles have up to 128 columns), after which
    the graph schedule must capture again rather than replay the old arrays. Same for the
    autotuner, which tries every schedule."""
    draws = [(512, 512, -0.25, -0.3), (64, 512, -0.3, -0.25), (256, 64, -0.2, -0.3), (128, 128, -0.35, -0.28)]
    b = _batch(draws, "fp64")
    x, parts = _state(draws, 800, torch.float64)
    b.step(x, 16)                 # the graph schedule's graph captured here
    b.set_schedule("persistent")
    b.step(x, 4)
    b.set_schedule("graph")
    b.step(x, 16)                 # replays a graph: must hold the current arrays
    b.autotune(2, 4)
    b.step(x, 16)
    b.sync()
    for d, (ny, nx, r, m) in enumerate(draws):
        ref = oracle.step(parts[d].reshape(ny, nx), DX, 0.5, (0, r, 0.0, 0.0), 52)
        assert rel(b.view(x, d).cpu().numpy(), ref) <= 1e-11
    b.close()


@pytest.mark.parametrize("prec,tol,shape,opc,threads", [
    ("fp64", 1e-11, (16, 32, 32), (1, -0.3, 0.05, math.sqrt(4.0 / 3.0)), 128),
    ("fp32", 1e-5, (32, 32, 64), (0, -0.2, 0.0, 0.0), 256),
    ("fp64", 1e-11, (64, 128), (0, -0.2, 0.0, 0.0), 256)])
def test_coupled_pair_in_the_persistent_launch(prec, tol, shape, opc, threads):
    """A coupled density/composition pair attached to a batch steps in the same launch as the
    domains: the pair against the oracle's Cramer-rule step, the domains against the oracle, the
    pair's masses conserved. dt = 0.5 for both (the pair takes the batch's dt)."""
    from paper_2603_26818_gb300 import binding
    opp, alpha, nsteps = (0, -0.25, 0.0, 0.0), 0.1, 8
    draws = [(64, 64, -0.25, -0.25), (128, 256, -0.3, -0.3), (16, 16, -0.2, -0.3)]
    b = _batch(draws, prec)
    b.set_schedule("persistent", threads=threads)
    b.attach_pair(shape, [binding.make_op(*opp), binding.make_op(*opc)], alpha)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    x, parts = _state(draws, 900, dtype)
    p0 = inputs.uniform_state(shape, -0.25, 0.05, seed=61)
    c0 = inputs.uniform_state(shape, -0.2, 0.05, seed=62)
    if prec == "fp32":
        p0, c0 = p0.astype(np.float32).astype(np.float64), c0.astype(np.float32).astype(np.float64)
    pair = torch.from_numpy(np.stack([p0, c0])).to(device="cuda", dtype=dtype)
    with pytest.raises(binding.PfcError):
        b.step(x, 1)   # a batch with a pair steps only with it
    b.step_with_pair(x, pair, nsteps)
    b.sync()
    rp, rc = oracle.step2(p0, c0, DX, 0.5, opp, opc, alpha, nsteps)
    got = pair.double().cpu().numpy()
    assert rel(got[0], rp) <= tol and rel(got[1], rc) <= tol
    assert abs(got[0].mean() - p0.mean()) <= 1e-6 * abs(p0.mean())
    assert abs(got[1].mean() - c0.mean()) <= 1e-6 * abs(c0.mean())
    for d, (ny, nx, r, m) in enumerate(draws):
        ref = oracle.step(parts[d].reshape(ny, nx), DX, 0.5, (0, r, 0.0, 0.0), nsteps)
        assert rel(b.view(x, d).double().cpu().numpy(), ref) <= (1e-12 if prec == "fp64" else 1e-5)
    assert b.schedule_info()["schedule"] == 1
    b.close()


def test_coupled_pair_config_size_with_the_ensemble_autotuned():
    """The ensemble workload with the coupled pair at 256^3 FP32 in one launch, the schedule's
    block size autotuned: the pair against a standalone coupled plan from the same start
    (1e-5 after 10 steps) and a sample of domains against the graph schedule."""
    from paper_2603_26818_gb300 import binding
    draws = inputs.batch_draws(1024, seed=4)
    b = _batch(draws, "fp32")
    ops = [binding.make_op(0, -0.25), binding.make_op(0, -0.25)]
    b.attach_pair((256, 256, 256), ops, 0.1)
    b.autotune(2, 4)
    assert b.schedule_info()["schedule"] == 1
    x, parts = _state(draws, 4000, torch.float32)
    p0 = inputs.uniform_state((256, 256, 256), -0.25, 0.01, seed=5)
    c0 = inputs.uniform_state((256, 256, 256), -0.2, 0.01, seed=6)
    pair = torch.from_numpy(np.stack([p0, c0])).to(device="cuda", dtype=torch.float32)
    ref = pair.clone()
    b.step_with_pair(x, pair, 10)
    b.sync()
    pl = binding.Plan((256, 256, 256), DX, 0.5, ops, precision="fp32", coupling=0.1)
    pl.step(ref, 10)
    a, c = pair.double().cpu().numpy(), ref.double().cpu().numpy()
    assert rel(a[0], c[0]) <= 1e-5 and rel(a[1], c[1]) <= 1e-5
    bg = _batch(draws, "fp32")
    y, _ = _state(draws, 4000, torch.float32)
    bg.step(y, 10)
    xs, ys = x.double().cpu().numpy(), y.double().cpu().numpy()
    for d in range(0, 1024, 37):
        ny, nx, r, m = draws[d]
        o = bg.offsets[d]
        assert rel(xs[o:o + ny * nx], ys[o:o + ny * nx]) <= 1e-5, d
    b.close()
    bg.close()
    pl.close()

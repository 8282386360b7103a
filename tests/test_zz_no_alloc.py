"""pfc_step_noalloc: the step for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (their device memory is held by another allocator, or
their loop cannot afford the synchronisation an allocation implies). pfc_step_noalloc runs
the same step as a plan's pfc_step using only a fixed static device array of the library.
These tests call it through the C ABI and compare it with pfc_step on the same inputs, twice
in a row, so the second call starts from whatever the first left in the shared array. The
file is named to be collected last.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2603_26818_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6}


def _noalloc(shape, dx, dt, op, prec, x, nsteps):
    from paper_2603_26818_gb300 import binding
    lib = binding.load_library()
    dims = (ctypes.c_int64 * len(shape))(*shape)
    o = binding.make_op(*op)
    p = binding.PFC_FP64 if prec == "fp64" else binding.PFC_FP32_MIXED
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.pfc_step_noalloc(len(shape), dims, float(dx), float(dt), ctypes.byref(o), p,
                                ctypes.c_void_p(x.data_ptr()), int(nsteps), st)


def rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,op,dt", [((128, 128), (0, -0.25, 0.0, 0.0), 0.5),
                                         ((32, 16, 64), (1, -0.3, 0.05, math.sqrt(4 / 3)), 0.1)])
def test_noalloc_matches_pfc_step_on_two_calls(shape, op, dt, prec):
    from paper_2603_26818_gb300 import binding
    dx = math.pi / 4
    dtype = torch.float64 if prec == "fp64" else torch.float32
    psi0 = inputs.uniform_state(shape, -0.25, 0.05, seed=23)
    plan = binding.Plan(shape, dx, dt, [binding.make_op(*op)], precision=prec)
    ref = torch.from_numpy(psi0).to(device="cuda", dtype=dtype)
    got = ref.clone()
    for nsteps in (7, 5):   # two calls in a row on the same state
        plan.step(ref, nsteps)
        assert _noalloc(shape, dx, dt, op, prec, got, nsteps) == binding.PFC_OK
        torch.cuda.synchronize()
        assert rel(got, ref) <= TOL[prec]
    plan.close()


@pytest.mark.parametrize("shape,prec,fits", [((1024, 1024), "fp64", True), ((1024, 2048), "fp32", True),
                                              ((128, 128, 128), "fp32", True), ((64, 64, 64), "fp64", True),
                                              ((2048, 2048), "fp32", False), ((128, 128, 128), "fp64", False)])
def test_noalloc_size_limit(shape, prec, fits):
    """The stated limit: grids whose two padded half spectra fit the 24 MiB array run (and match
    pfc_step); larger ones are rejected before any device work."""
    from paper_2603_26818_gb300 import binding
    dtype = torch.float64 if prec == "fp64" else torch.float32
    op = (0, -0.25, 0.0, 0.0)
    psi0 = inputs.uniform_state(shape, -0.25, 0.05, seed=29)
    x = torch.from_numpy(psi0).to(device="cuda", dtype=dtype)
    before = x.clone()
    rc = _noalloc(shape, math.pi / 4, 0.5, op, prec, x, 2)
    if not fits:
        assert rc == 2 and b"24 MiB" in binding.load_library().pfc_last_error()
        torch.cuda.synchronize()
        assert torch.equal(x, before)
        return
    assert rc == binding.PFC_OK
    plan = binding.Plan(shape, math.pi / 4, 0.5, [binding.make_op(*op)], precision=prec)
    plan.step(before, 2)
    torch.cuda.synchronize()
    assert rel(x, before) <= TOL[prec]
    plan.close()


def test_noalloc_matches_the_oracle():
    """Against the FP64 oracle directly (not only against pfc_step), FP64 and FP32-mixed."""
    import oracle
    shape, dx, dt, op = (64, 128), math.pi / 4, 0.5, (0, -0.25, 0.0, 0.0)
    psi0 = inputs.uniform_state(shape, -0.25, 0.05, seed=31)
    ref = oracle.step(psi0, dx, dt, op, 12)
    for prec, dtype, tol in (("fp64", torch.float64, 1e-12), ("fp32", torch.float32, 1e-5)):
        x = torch.from_numpy(psi0).to(device="cuda", dtype=dtype)
        assert _noalloc(shape, dx, dt, op, prec, x, 12) == 0
        torch.cuda.synchronize()
        got = x.double().cpu().numpy()
        assert float(np.linalg.norm(got - ref) / np.linalg.norm(ref)) <= tol


def test_noalloc_on_the_clustered_row_pass(monkeypatch):
    """A tiling with the psi^3 row pass on two-block clusters (Py = 8 rows of nx = 4096, FP32):
    the allocation-free step takes the same launches as the plan. The time step is unique to
    this test, so the tiling is not one remembered from another call."""
    from paper_2603_26818_gb300 import binding
    monkeypatch.setenv("PFC_TILE", "8,1,4")
    shape, dx, dt, op = (512, 4096), math.pi / 4, 0.4375, (0, -0.25, 0.0, 0.0)
    psi0 = inputs.uniform_state(shape, -0.25, 0.05, seed=37)
    plan = binding.Plan(shape, dx, dt, [binding.make_op(*op)], precision="fp32")
    assert plan.info()["row_cluster"] == 2
    ref = torch.from_numpy(psi0).to(device="cuda", dtype=torch.float32)
    got = ref.clone()
    for nsteps in (3, 4):
        plan.step(ref, nsteps)
        assert _noalloc(shape, dx, dt, op, "fp32", got, nsteps) == 0
        torch.cuda.synchronize()
        assert rel(got, ref) <= TOL["fp32"]
    plan.close()


def test_noalloc_rejects_a_nonfinite_state():
    """NaN in the state: PFC_ERR_NONFINITE, and the state is left as it was."""
    from paper_2603_26818_gb300 import binding
    shape = (64, 64)
    x = torch.from_numpy(inputs.uniform_state(shape, -0.25, 0.05, seed=41)).to(device="cuda")
    x[5, 7] = float("nan")
    before = x.clone()
    rc = _noalloc(shape, math.pi / 4, 0.5, (0, -0.25, 0.0, 0.0), "fp64", x, 3)
    assert rc == 6 and b"NaN" in binding.load_library().pfc_last_error()
    torch.cuda.synchronize()
    assert torch.equal(torch.nan_to_num(x, nan=7.0), torch.nan_to_num(before, nan=7.0))
    # a finite state afterwards runs normally (the status word is cleared per call)
    y = torch.from_numpy(inputs.uniform_state(shape, -0.25, 0.05, seed=43)).to(device="cuda")
    assert _noalloc(shape, math.pi / 4, 0.5, (0, -0.25, 0.0, 0.0), "fp64", y, 3) == 0

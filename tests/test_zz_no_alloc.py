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

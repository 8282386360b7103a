"""The C ABI without a GPU: the library loads, exports every function include/*.h declares,
and rejects bad arguments on the host before any device work."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(pfc\w*)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_26818_gb300 import binding
    return binding.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["pfc_plan_create", "pfc_step", "pfc_fft_r2c", "pfc_fft_c2r", "pfc_mass",
                 "pfc_energy", "pfc_step_adjoint", "pfc_batch_create", "pfc_batch_step"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2603_26818_gb300 import binding
    names = declared_functions()
    assert names, "no declarations parsed"
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert sorted(binding.EXPORTS) == names


def test_status_strings(lib):
    for code, name in [(0, b"PFC_OK"), (1, b"PFC_ERR_INVALID_ARG"), (3, b"PFC_ERR_UNSTABLE_OPERATOR"),
                       (7, b"PFC_ERR_TIMEOUT")]:
        assert lib.pfc_status_string(code) == name


def _create(lib, dims, dx=0.785, dt=0.5, ops=None, nfields=1, prec=0, coupling=None):
    from paper_2603_26818_gb300 import binding
    ops = ops or [binding.make_op(0, -0.25)]
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * len(dims))(*dims)
    o = (binding.pfc_op * len(ops))(*ops)
    cp = None if coupling is None else (ctypes.c_double * 4)(0.0, coupling, coupling, 0.0)
    return lib.pfc_plan_create(ctypes.byref(h), len(dims), d, dx, dt, o, nfields, cp, prec, None)


def test_host_side_validation(lib):
    from paper_2603_26818_gb300 import binding
    assert _create(lib, (128, 128), dx=0.0) == 1                        # dx <= 0
    assert _create(lib, (128, 128), dt=-1.0) == 1                       # dt <= 0
    assert _create(lib, (128,)) == 1                                    # ndim 1
    assert _create(lib, (88, 128)) == 2                                 # 88 = 8 * 11
    assert _create(lib, (128, 130)) == 2                                # nx / 2 = 65 = 5 * 13
    assert _create(lib, (128, 12)) == 2                                 # nx / 2 below 8
    assert _create(lib, (96, 96), ops=[binding.make_op(0, -0.25), binding.make_op(0, -0.25)],
                   nfields=2, coupling=0.1) == 2                        # two fields, not powers of two
    assert _create(lib, (8192, 128)) == 2                               # too large
    assert _create(lib, (128, 128), nfields=3) == 2                     # nfields
    assert _create(lib, (128, 128), prec=7) == 1                        # precision
    assert _create(lib, (128, 128), ops=[binding.make_op(5, -0.25)]) == 1
    # an operator whose implicit factor 1 + dt k^2 Lk(k) crosses zero
    assert _create(lib, (128, 128), ops=[binding.make_op(0, -20.0)]) == 3
    assert b"positive" in lib.pfc_last_error()
    # a coupling strong enough to make the implicit 2x2 matrix indefinite at some k
    assert _create(lib, (128, 128), ops=[binding.make_op(0, -0.25), binding.make_op(0, -0.2)],
                   nfields=2, coupling=5.0) == 3
    assert lib.pfc_step(None, None, 1) == 1
    assert lib.pfc_plan_autotune(None, 4, 20, None, None) == 1
    assert lib.pfc_batch_autotune(None, 4, 20, None) == 1
    assert lib.pfc_batch_info(None, None, 0, None) == 1
    assert lib.pfc_set_integrator(None, 2, 0.0) == 1
    assert lib.pfc_hydro_step(None, None, None, 1) == 1
    assert lib.pfc_hydro_destroy(None) == 0
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 2)(32, 32)
    op = binding.make_op(0, -0.25)
    assert lib.pfc_hydro_create(ctypes.byref(h), 2, dims, 0.785, 0.5, ctypes.byref(op), -1.0, 1.0, 1.0, 0, None) == 1
    assert lib.pfc_hydro_create(ctypes.byref(h), 2, dims, 0.785, 0.5, ctypes.byref(op), 1.0, float("nan"), 1.0, 0,
                                None) == 1
    assert lib.pfc_plan_destroy(None) == 0


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2603_26818_gb300 import binding
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            binding.load_library(str(tmp_path / "missing.so"))
    finally:
        binding._lib = saved


def _noalloc(lib, dims, dx=0.785, dt=0.5, op=None, prec=0, state=16, nsteps=1):
    """pfc_step_noalloc with a fake (aligned, never dereferenced) state pointer: every call here
    must be rejected on the host before any device work."""
    from paper_2603_26818_gb300 import binding
    op = op if op is not None else binding.make_op(0, -0.25)
    d = (ctypes.c_int64 * len(dims))(*dims) if dims is not None else None
    return lib.pfc_step_noalloc(len(dims) if dims else 2, d, dx, dt,
                                ctypes.byref(op) if op is not False else None, prec,
                                ctypes.c_void_p(state) if state else None, nsteps, None)


def test_noalloc_host_side_rejections(lib):
    from paper_2603_26818_gb300 import binding
    assert _noalloc(lib, None) == 1                                      # null dims
    assert _noalloc(lib, (128, 128), state=0) == 1                       # null state
    assert _noalloc(lib, (128, 128), op=False) == 1                      # null operator
    assert _noalloc(lib, (128,)) == 1                                    # ndim 1
    assert _noalloc(lib, (128, 128), dx=-1.0) == 1
    assert _noalloc(lib, (128, 128), dt=float("inf")) == 1
    assert _noalloc(lib, (128, 128), prec=3) == 1
    assert _noalloc(lib, (128, 128), nsteps=-1) == 1
    assert _noalloc(lib, (128, 128), state=8) == 1                       # not 16-byte aligned
    assert _noalloc(lib, (128, 128), op=binding.make_op(0, float("nan"))) == 1
    assert b"finite" in lib.pfc_last_error()
    assert _noalloc(lib, (128, 128), op=binding.make_op(1, -0.3, float("inf"), 1.1)) == 1
    assert _noalloc(lib, (96, 128)) == 2                                 # not a power of two
    # grids whose two half spectra alone exceed the 24 MiB array
    assert _noalloc(lib, (2048, 2048), prec=1) == 2
    assert b"24 MiB" in lib.pfc_last_error()
    assert _noalloc(lib, (128, 128, 128), prec=0) == 2
    assert _noalloc(lib, (128, 128), nsteps=0) == 0                      # no work, no device


def _apfc(lib, dims, kv, op=(0, -0.25, 0.0, 0.0), namp=None, dx=1.0, dt=0.3, prec=1, psibar=-0.2):
    from paper_2603_26818_gb300 import binding
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * len(dims))(*dims)
    o = binding.make_op(*op)
    flat = [float(c) for k in kv for c in k]
    k = (ctypes.c_double * max(len(flat), 1))(*flat)
    n = len(kv) if namp is None else namp
    return lib.pfc_apfc_create(ctypes.byref(h), len(dims), d, dx, dt, ctypes.byref(o), n, k, psibar, prec, None)


def test_apfc_host_side_rejections(lib):
    """pfc_apfc_create rejects bad arguments before any device call: INVALID_ARG (1) for a bad
    ndim, amplitude count, spacing, step, precision or a non-finite vector; UNSUPPORTED (2) for
    an extent outside [8, 4096] or with a prime factor other than 2, 3, 5, 7; UNSTABLE_OPERATOR
    (3) when 1 + dt Q L(Q) <= 0 for some shifted wavevector on the grid."""
    tri = [(-0.866, -0.5), (0.0, 1.0), (0.866, -0.5)]
    assert _apfc(lib, (16,), [(1.0,)]) == 1
    assert _apfc(lib, (16, 16, 16, 16), tri) == 1
    assert _apfc(lib, (16, 16), tri, namp=0) == 1
    assert _apfc(lib, (16, 16), [(1.0, 0.0)] * 17) == 1
    assert _apfc(lib, (16, 16), tri, dx=0.0) == 1
    assert _apfc(lib, (16, 16), tri, dt=-1.0) == 1
    assert _apfc(lib, (16, 16), tri, prec=7) == 1
    assert _apfc(lib, (16, 16), [(float("nan"), 0.0)] + tri[1:]) == 1
    assert _apfc(lib, (16, 16), tri, psibar=float("inf")) == 1
    assert _apfc(lib, (16, 11), tri) == 2      # prime 11
    assert _apfc(lib, (4, 16), tri) == 2       # below 8
    assert _apfc(lib, (16, 8192), tri) == 2    # above 4096
    # r = -3: L(Q) = r + (1 - Q)^2 is negative near Q = 1 and dt Q |L| > 1 there
    assert _apfc(lib, (16, 16), tri, op=(0, -3.0, 0.0, 0.0), dt=1.0) == 3
    null = ctypes.c_void_p()
    assert lib.pfc_apfc_step(None, null, 1) == 1
    assert lib.pfc_apfc_destroy(None) == 0

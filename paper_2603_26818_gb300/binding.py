"""ctypes binding of libpfc.so (include/pfc.h): argument marshalling only.

Every number is computed by the library's CUDA kernels. Device memory and streams come from
PyTorch: arrays are CUDA tensors, the stream is torch's current stream at plan creation. If
the library has not been built this module raises on first use; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpfc.so")

PFC_OK = 0
STATUS_NAMES = {0: "PFC_OK", 1: "PFC_ERR_INVALID_ARG", 2: "PFC_ERR_UNSUPPORTED",
                3: "PFC_ERR_UNSTABLE_OPERATOR", 4: "PFC_ERR_OUT_OF_MEMORY", 5: "PFC_ERR_CUDA",
                6: "PFC_ERR_NONFINITE", 7: "PFC_ERR_TIMEOUT"}
PFC_FP64, PFC_FP32_MIXED = 0, 1
PFC_ONE_MODE, PFC_TWO_MODE = 0, 1
PFC_SEMI_IMPLICIT, PFC_STABILIZED, PFC_SBDF2 = 0, 1, 2
PFC_BATCH_GRAPH, PFC_BATCH_PERSISTENT = 0, 1

# every extern "C" symbol of include/pfc.h
EXPORTS = ["pfc_plan_create", "pfc_plan_destroy", "pfc_step", "pfc_fft_r2c", "pfc_fft_c2r",
           "pfc_mass", "pfc_energy", "pfc_step_adjoint", "pfc_set_r", "pfc_sync", "pfc_plan_info",
           "pfc_profile_steps", "pfc_step_noalloc", "pfc_plan_autotune", "pfc_batch_autotune",
           "pfc_batch_info",
           "pfc_set_integrator", "pfc_record_bytes", "pfc_step_record", "pfc_adjoint_segment",
           "pfc_hydro_create", "pfc_hydro_step", "pfc_hydro_destroy",
           "pfc_apfc_create", "pfc_apfc_step", "pfc_apfc_resonances", "pfc_apfc_destroy",
           "pfc_status_string", "pfc_last_error", "pfc_batch_create", "pfc_batch_destroy",
           "pfc_batch_step", "pfc_batch_mass", "pfc_batch_set_schedule", "pfc_batch_schedule_info",
           "pfc_batch_set_wait_limit", "pfc_batch_sync", "pfc_batch_attach_pair",
           "pfc_batch_step_with_pair"]


class PfcError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{self.name}: {message}")


class pfc_op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("r", ctypes.c_double), ("R1", ctypes.c_double),
                ("q2", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpfc.so and declare its signatures. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it first (python -c 'import __graft_entry__ as g;"
                           " g.build()'); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, i64, dbl, cint = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "pfc_plan_create": [P(vp), cint, P(i64), dbl, dbl, P(pfc_op), cint, P(dbl), cint, vp],
        "pfc_plan_destroy": [vp],
        "pfc_step": [vp, vp, i64],
        "pfc_fft_r2c": [vp, vp, vp],
        "pfc_fft_c2r": [vp, vp, vp],
        "pfc_mass": [vp, vp, P(dbl)],
        "pfc_energy": [vp, vp, P(dbl)],
        "pfc_step_adjoint": [vp, vp, vp, vp, vp],
        "pfc_set_r": [vp, cint, dbl],
        "pfc_set_integrator": [vp, cint, dbl],
        "pfc_record_bytes": [vp, i64, P(i64)],
        "pfc_hydro_create": [P(vp), cint, P(i64), dbl, dbl, P(pfc_op), dbl, dbl, dbl, cint, vp],
        "pfc_apfc_create": [P(vp), cint, P(i64), dbl, dbl, P(pfc_op), cint, P(dbl), dbl, cint, vp],
        "pfc_apfc_step": [vp, vp, i64],
        "pfc_apfc_resonances": [vp, P(ctypes.c_int32)],
        "pfc_apfc_destroy": [vp],
        "pfc_hydro_step": [vp, vp, vp, i64],
        "pfc_hydro_destroy": [vp],
        "pfc_step_record": [vp, vp, i64, vp],
        "pfc_adjoint_segment": [vp, vp, i64, vp, vp],
        "pfc_sync": [vp],
        "pfc_plan_info": [vp, P(ctypes.c_int32), P(i64)],
        "pfc_profile_steps": [vp, vp, i64, P(dbl), P(i64)],
        "pfc_plan_autotune": [vp, cint, cint, ctypes.c_char_p, P(dbl)],
        "pfc_batch_autotune": [vp, cint, cint, P(dbl)],
        "pfc_batch_info": [vp, P(ctypes.c_int32), cint, P(ctypes.c_int32)],
        "pfc_step_noalloc": [cint, P(i64), dbl, dbl, P(pfc_op), cint, vp, i64, vp],
        "pfc_batch_create": [P(vp), cint, P(i64), P(dbl), dbl, dbl, cint, vp],
        "pfc_batch_destroy": [vp],
        "pfc_batch_step": [vp, vp, i64],
        "pfc_batch_mass": [vp, vp, P(dbl)],
        "pfc_batch_set_schedule": [vp, cint, cint, i64, dbl],
        "pfc_batch_schedule_info": [vp, P(i64)],
        "pfc_batch_set_wait_limit": [vp, dbl, cint],
        "pfc_batch_sync": [vp],
        "pfc_batch_attach_pair": [vp, cint, P(i64), P(pfc_op), dbl],
        "pfc_batch_step_with_pair": [vp, vp, vp, i64],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = cint
    lib.pfc_status_string.argtypes = [cint]
    lib.pfc_status_string.restype = ctypes.c_char_p
    lib.pfc_last_error.argtypes = []
    lib.pfc_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def check(status: int):
    if status != PFC_OK:
        msg = load_library().pfc_last_error().decode()
        raise PfcError(status, msg)


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev_ptr(t: torch.Tensor, dtype, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise PfcError(1, f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise PfcError(1, f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise PfcError(1, f"{name} must be contiguous")
    return t.data_ptr()


def make_op(kind=PFC_ONE_MODE, r=-0.25, R1=0.0, q2=0.0) -> pfc_op:
    return pfc_op(int(kind), float(r), float(R1), float(q2))


class Plan:
    """A pfc_plan: one grid (2D or 3D), nfields fields, one precision, one stream."""

    def __init__(self, dims, dx, dt, ops, precision="fp64", coupling=None, stream=None):
        lib = load_library()
        if isinstance(ops, pfc_op):
            ops = [ops]
        ops = [o if isinstance(o, pfc_op) else make_op(*o) for o in ops]
        self.dims = tuple(int(d) for d in dims)
        self.ndim = len(self.dims)
        self.nfields = len(ops)
        self.precision = precision
        self.real_dtype = torch.float64 if precision == "fp64" else torch.float32
        self.complex_dtype = torch.complex128 if precision == "fp64" else torch.complex64
        prec = PFC_FP64 if precision == "fp64" else PFC_FP32_MIXED
        dims_arr = (ctypes.c_int64 * self.ndim)(*self.dims)
        ops_arr = (pfc_op * self.nfields)(*ops)
        coup = None
        if coupling is not None:
            coup = (ctypes.c_double * 4)(0.0, float(coupling), float(coupling), 0.0)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(lib.pfc_plan_create(ctypes.byref(h), self.ndim, dims_arr, float(dx), float(dt),
                                  ops_arr, self.nfields, coup, prec,
                                  ctypes.c_void_p(_stream_handle(self._stream))))
        self._h = h
        self.dx, self.dt = float(dx), float(dt)

    @property
    def handle(self):
        return self._h

    def real_shape(self):
        return ((self.nfields,) if self.nfields > 1 else ()) + self.dims

    def half_shape(self):
        return ((self.nfields,) if self.nfields > 1 else ()) + self.dims[:-1] + (self.dims[-1] // 2 + 1,)

    def _check_real(self, t, name):
        if tuple(t.shape) != self.real_shape():
            raise PfcError(1, f"{name} has shape {tuple(t.shape)}, expected {self.real_shape()}")
        return _dev_ptr(t, self.real_dtype, name)

    def step(self, state: torch.Tensor, nsteps: int = 1) -> torch.Tensor:
        p = self._check_real(state, "state")
        check(load_library().pfc_step(self._h, ctypes.c_void_p(p), int(nsteps)))
        return state

    def fft_r2c(self, x: torch.Tensor, out: torch.Tensor = None) -> torch.Tensor:
        p = self._check_real(x, "x")
        if out is None:
            out = torch.empty(self.half_shape(), dtype=self.complex_dtype, device=x.device)
        q = _dev_ptr(out, self.complex_dtype, "out")
        check(load_library().pfc_fft_r2c(self._h, ctypes.c_void_p(p), ctypes.c_void_p(q)))
        return out

    def fft_c2r(self, xh: torch.Tensor, out: torch.Tensor = None) -> torch.Tensor:
        if tuple(xh.shape) != self.half_shape():
            raise PfcError(1, f"xh has shape {tuple(xh.shape)}, expected {self.half_shape()}")
        p = _dev_ptr(xh, self.complex_dtype, "xh")
        if out is None:
            out = torch.empty(self.real_shape(), dtype=self.real_dtype, device=xh.device)
        q = self._check_real(out, "out")
        check(load_library().pfc_fft_c2r(self._h, ctypes.c_void_p(p), ctypes.c_void_p(q)))
        return out

    def mass(self, state: torch.Tensor):
        p = self._check_real(state, "state")
        out = (ctypes.c_double * self.nfields)()
        check(load_library().pfc_mass(self._h, ctypes.c_void_p(p), out))
        return list(out)

    def energy(self, state: torch.Tensor) -> float:
        p = self._check_real(state, "state")
        out = ctypes.c_double()
        check(load_library().pfc_energy(self._h, ctypes.c_void_p(p), ctypes.byref(out)))
        return out.value

    def step_adjoint(self, psi_n, lam_next, lam_out, dr_accum: torch.Tensor):
        a = self._check_real(psi_n, "psi_n")
        b = self._check_real(lam_next, "lam_next")
        c = self._check_real(lam_out, "lam_out")
        d = _dev_ptr(dr_accum, torch.float64, "dr_accum")
        check(load_library().pfc_step_adjoint(self._h, ctypes.c_void_p(a), ctypes.c_void_p(b),
                                              ctypes.c_void_p(c), ctypes.c_void_p(d)))
        return lam_out

    def record_bytes(self, nsteps: int):
        """pfc_record_bytes: bytes of a recorded segment of nsteps steps, or None when the plan
        has no fused adjoint (then use step_adjoint per step)."""
        out = ctypes.c_int64()
        st = load_library().pfc_record_bytes(self._h, int(nsteps), ctypes.byref(out))
        if st == 2:
            return None
        check(st)
        return out.value

    def step_record(self, state: torch.Tensor, nsteps: int, record: torch.Tensor) -> torch.Tensor:
        """pfc_step_record: nsteps steps of state, recording the segment into record (a uint8 CUDA
        tensor of record_bytes(nsteps) bytes, 256-byte aligned)."""
        p = self._check_real(state, "state")
        check(load_library().pfc_step_record(self._h, ctypes.c_void_p(p), int(nsteps),
                                             ctypes.c_void_p(_dev_ptr(record, torch.uint8, "record"))))
        return state

    def adjoint_segment(self, record: torch.Tensor, nsteps: int, lam: torch.Tensor, dr_accum: torch.Tensor):
        """pfc_adjoint_segment: the adjoint of a recorded segment, lam in place."""
        q = self._check_real(lam, "lam")
        d = _dev_ptr(dr_accum, torch.float64, "dr_accum")
        check(load_library().pfc_adjoint_segment(self._h, ctypes.c_void_p(_dev_ptr(record, torch.uint8, "record")),
                                                 int(nsteps), ctypes.c_void_p(q), ctypes.c_void_p(d)))
        return lam

    def set_r(self, r: float, field: int = 0):
        check(load_library().pfc_set_r(self._h, int(field), float(r)))

    def set_integrator(self, scheme: int, S: float = 0.0):
        """pfc_set_integrator: PFC_SEMI_IMPLICIT, PFC_STABILIZED (constant S) or PFC_SBDF2."""
        check(load_library().pfc_set_integrator(self._h, int(scheme), float(S)))

    def sync(self):
        check(load_library().pfc_sync(self._h))

    def profile_steps(self, state: torch.Tensor, nsteps: int):
        """pfc_profile_steps: ms per kernel kind {row, line, entry, exit, mid} and the launch count."""
        p = self._check_real(state, "state")
        ms = (ctypes.c_double * 5)()
        nl = ctypes.c_int64()
        check(load_library().pfc_profile_steps(self._h, ctypes.c_void_p(p), int(nsteps), ms,
                                               ctypes.byref(nl)))
        return dict(zip(["row", "line", "entry", "exit", "mid"], list(ms))), nl.value

    def autotune(self, max_candidates: int = 8, trial_steps: int = 20, cache: str = None) -> float:
        """pfc_plan_autotune: time up to max_candidates tilings and keep the fastest; returns its
        ms per step. cache: optional path of the JSON-lines cache file."""
        ms = ctypes.c_double()
        check(load_library().pfc_plan_autotune(self._h, int(max_candidates), int(trial_steps),
                                               cache.encode() if cache else None, ctypes.byref(ms)))
        return ms.value

    def info(self):
        tiles = (ctypes.c_int32 * 11)()
        sb = ctypes.c_int64()
        check(load_library().pfc_plan_info(self._h, tiles, ctypes.byref(sb)))
        keys = ["Py", "Pz", "Qy", "Qz", "W", "gpc", "threads_row", "threads_line", "row_cluster", "Ry", "Rz"]
        d = dict(zip(keys, list(tiles)))
        d["scratch_bytes"] = sb.value
        return d

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            check(load_library().pfc_plan_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Hydro:
    """A pfc_hydro: the hydrodynamic PFC model (density psi and velocity v) on one grid."""

    def __init__(self, dims, dx, dt, op, rho=1.0, gamma=1.0, a0=0.0, precision="fp64", stream=None):
        lib = load_library()
        op = op if isinstance(op, pfc_op) else make_op(*op)
        self.dims = tuple(int(d) for d in dims)
        self.ndim = len(self.dims)
        self.real_dtype = torch.float64 if precision == "fp64" else torch.float32
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(lib.pfc_hydro_create(ctypes.byref(h), self.ndim, (ctypes.c_int64 * self.ndim)(*self.dims), float(dx),
                                   float(dt), ctypes.byref(op), float(rho), float(gamma), float(a0),
                                   PFC_FP64 if precision == "fp64" else PFC_FP32_MIXED,
                                   ctypes.c_void_p(_stream_handle(self._stream))))
        self._h = h

    def step(self, psi: torch.Tensor, v: torch.Tensor, nsteps: int = 1):
        if tuple(psi.shape) != self.dims or tuple(v.shape) != (self.ndim,) + self.dims:
            raise PfcError(1, f"psi must have shape {self.dims} and v {(self.ndim,) + self.dims}")
        check(load_library().pfc_hydro_step(self._h, ctypes.c_void_p(_dev_ptr(psi, self.real_dtype, "psi")),
                                            ctypes.c_void_p(_dev_ptr(v, self.real_dtype, "v")), int(nsteps)))
        return psi, v

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            check(load_library().pfc_hydro_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Apfc:
    """A pfc_apfc: the amplitude-expansion PFC model, namp complex amplitude fields on one grid.

    dims slowest first; kvecs a list of namp vectors (x first); eta a complex CUDA tensor of shape
    (namp, *dims), complex64 for "fp32", complex128 for "fp64"."""

    def __init__(self, dims, dx, dt, op, kvecs, psibar, precision="fp32", stream=None):
        lib = load_library()
        op = op if isinstance(op, pfc_op) else make_op(*op)
        self.dims = tuple(int(d) for d in dims)
        self.ndim = len(self.dims)
        self.namp = len(kvecs)
        self.dtype = torch.complex128 if precision == "fp64" else torch.complex64
        flat = [float(c) for k in kvecs for c in list(k)[:self.ndim]]
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(lib.pfc_apfc_create(ctypes.byref(h), self.ndim, (ctypes.c_int64 * self.ndim)(*self.dims), float(dx),
                                  float(dt), ctypes.byref(op), self.namp, (ctypes.c_double * len(flat))(*flat),
                                  float(psibar), PFC_FP64 if precision == "fp64" else PFC_FP32_MIXED,
                                  ctypes.c_void_p(_stream_handle(self._stream))))
        self._h = h

    def step(self, eta: torch.Tensor, nsteps: int = 1) -> torch.Tensor:
        if tuple(eta.shape) != (self.namp,) + self.dims:
            raise PfcError(1, f"eta must have shape {(self.namp,) + self.dims}")
        check(load_library().pfc_apfc_step(self._h, ctypes.c_void_p(_dev_ptr(eta, self.dtype, "eta")), int(nsteps)))
        return eta

    def resonances(self) -> int:
        n = ctypes.c_int32()
        check(load_library().pfc_apfc_resonances(self._h, ctypes.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            check(load_library().pfc_apfc_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A pfc_batch: many independent 2D one-mode domains of uneven sizes, one packed state.

    dims: list of (ny, nx); r: list of per-domain r. The packed state is a 1D CUDA tensor holding
    the domains back to back in list order (domain d at offsets[d], ny_d nx_d values)."""

    def __init__(self, dims, r, dx, dt, precision="fp32", stream=None):
        lib = load_library()
        self.dims = [(int(a), int(b)) for a, b in dims]
        self.nd = len(self.dims)
        self.real_dtype = torch.float64 if precision == "fp64" else torch.float32
        flat = (ctypes.c_int64 * (2 * self.nd))(*[v for d in self.dims for v in d])
        rr = (ctypes.c_double * self.nd)(*[float(x) for x in r])
        self.offsets = []
        off = 0
        for ny, nx in self.dims:
            self.offsets.append(off)
            off += ny * nx
        self.total = off
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        check(lib.pfc_batch_create(ctypes.byref(h), self.nd, flat, rr, float(dx), float(dt),
                                   PFC_FP64 if precision == "fp64" else PFC_FP32_MIXED,
                                   ctypes.c_void_p(_stream_handle(self._stream))))
        self._h = h

    def _ptr(self, state):
        if tuple(state.shape) != (self.total,):
            raise PfcError(1, f"state has shape {tuple(state.shape)}, expected ({self.total},)")
        return _dev_ptr(state, self.real_dtype, "state")

    def step(self, state: torch.Tensor, nsteps: int = 1) -> torch.Tensor:
        check(load_library().pfc_batch_step(self._h, ctypes.c_void_p(self._ptr(state)), int(nsteps)))
        return state

    def autotune(self, max_candidates: int = 8, trial_steps: int = 20) -> float:
        """pfc_batch_autotune: tile every size class by measurement; returns the summed ms per step."""
        ms = ctypes.c_double()
        check(load_library().pfc_batch_autotune(self._h, int(max_candidates), int(trial_steps),
                                                ctypes.byref(ms)))
        return ms.value

    def info(self):
        """pfc_batch_info: one dict per size class with its tiles."""
        lib = load_library()
        n = ctypes.c_int32()
        check(lib.pfc_batch_info(self._h, None, 0, ctypes.byref(n)))
        buf = (ctypes.c_int32 * (9 * n.value))()
        check(lib.pfc_batch_info(self._h, buf, n.value, ctypes.byref(n)))
        keys = ["ny", "nx", "members", "Py", "W", "gpc", "threads_row", "threads_line", "Qy"]
        return [dict(zip(keys, list(buf[9 * i:9 * i + 9]))) for i in range(n.value)]

    def set_schedule(self, schedule: str = "persistent", threads: int = 128, onchip_smem_max: int = 0,
                     onchip_block_share: float = -1.0):
        """pfc_batch_set_schedule: "graph" (per-class launches in graph branches) or "persistent"
        (the whole call in one cooperative launch)."""
        code = {"graph": PFC_BATCH_GRAPH, "persistent": PFC_BATCH_PERSISTENT}[schedule]
        check(load_library().pfc_batch_set_schedule(self._h, code, int(threads), int(onchip_smem_max),
                                                    float(onchip_block_share)))

    def schedule_info(self):
        """pfc_batch_schedule_info as a dict."""
        buf = (ctypes.c_int64 * 10)()
        check(load_library().pfc_batch_schedule_info(self._h, buf))
        keys = ["schedule", "threads", "blocks", "onchip_blocks", "smem", "graph", "row_items",
                "line_items", "onchip_items", "mean_items"]
        return dict(zip(keys, list(buf)))

    def set_wait_limit(self, seconds: float = 2.0, extra_arrivals: int = 0):
        """pfc_batch_set_wait_limit: bound of the persistent launch's barrier waits."""
        check(load_library().pfc_batch_set_wait_limit(self._h, float(seconds), int(extra_arrivals)))

    def attach_pair(self, shape, ops, alpha: float):
        """pfc_batch_attach_pair: a coupled density/composition pair (shape slowest first; ops two
        pfc_op from make_op) stepped inside the persistent launch."""
        lib = load_library()
        self.pair_shape = tuple(int(v) for v in shape)
        dims = (ctypes.c_int64 * len(shape))(*self.pair_shape)
        arr = (pfc_op * 2)(*ops)
        check(lib.pfc_batch_attach_pair(self._h, len(shape), dims, arr, float(alpha)))

    def step_with_pair(self, state: torch.Tensor, pair_state: torch.Tensor, nsteps: int = 1):
        """pfc_batch_step_with_pair: pair_state is (2, *shape) in the batch's dtype."""
        if tuple(pair_state.shape) != (2,) + self.pair_shape:
            raise PfcError(1, f"pair state has shape {tuple(pair_state.shape)}, expected {(2,) + self.pair_shape}")
        check(load_library().pfc_batch_step_with_pair(self._h, ctypes.c_void_p(self._ptr(state)),
                                                      ctypes.c_void_p(_dev_ptr(pair_state, self.real_dtype, "pair state")),
                                                      int(nsteps)))
        return state, pair_state

    def sync(self):
        """pfc_batch_sync: raises PfcError with the latched device status (TIMEOUT, NONFINITE)."""
        check(load_library().pfc_batch_sync(self._h))

    def mass(self, state: torch.Tensor):
        out = (ctypes.c_double * self.nd)()
        check(load_library().pfc_batch_mass(self._h, ctypes.c_void_p(self._ptr(state)), out))
        return list(out)

    def view(self, state: torch.Tensor, d: int) -> torch.Tensor:
        """Domain d of a packed state as a (ny, nx) view."""
        ny, nx = self.dims[d]
        return state[self.offsets[d]:self.offsets[d] + ny * nx].view(ny, nx)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            check(load_library().pfc_batch_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Oracle for the semi-implicit Fourier pseudo-spectral PFC step (FP64, CPU).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers. The GPU library does not import, link or run it.

This module is a thin ctypes wrapper over ``pfc_oracle.c`` (argument marshalling only;
every number is computed in C). Arrays are numpy float64 / complex128, row-major
(nz, ny, nx) with x fastest; 2D arrays are (ny, nx) and are handled as nz = 1.

Parity status of each function (what pins it is in ``tests/test_oracle_pins.py``):
  dft, fft_radix2, fft_mixed, rfftn, irfftn   pinned (numpy.fft, naive DFT, closed forms)
  step, mass, energy                          pinned (closed forms, invariants, symmetries)
  hydro_step                                  pinned (reduction to step at rho = inf and v = 0,
                                              viscous decay of a velocity mode, advected
                                              density mode closed form, one-step mass with a
                                              divergence-free velocity)
  step_scheme                                 pinned (scheme 0 = step, S = 0 reduction, scalar
                                              recurrences of one small mode, convergence order)
  step2, energy2                              pinned (alpha=0 reduction, Cramer, mass)
  step_tangent, step_adjoint, adjoint_run     pinned (dot-product test, finite differences)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pfc_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None

ONE_MODE, TWO_MODE = 0, 1


def build(force: bool = False) -> str:
    """Compile pfc_oracle.c into liborc.so (plain gcc, IEEE FP64, OpenMP over lines)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    i64, dbl, cint = ctypes.c_int64, ctypes.c_double, ctypes.c_int
    p = ctypes.c_void_p
    lib.orc_dft.argtypes = [i64, p, p, cint]
    lib.orc_fft_radix2.argtypes = [i64, p, cint]
    lib.orc_fft_mixed.argtypes = [i64, p, cint]
    lib.orc_fft.argtypes = [i64, p, cint]
    lib.orc_rfftn.argtypes = [i64, i64, i64, p, p]
    lib.orc_irfftn.argtypes = [i64, i64, i64, p, p]
    lib.orc_lin_op.argtypes = [cint, dbl, dbl, dbl, dbl]
    lib.orc_lin_op.restype = dbl
    lib.orc_step.argtypes = [i64, i64, i64, dbl, dbl, cint, dbl, dbl, dbl, p, i64]
    lib.orc_step_scheme.argtypes = [i64, i64, i64, dbl, dbl, cint, dbl, dbl, dbl, cint, dbl, p, i64]
    lib.orc_hydro_step.argtypes = [i64, i64, i64, dbl, dbl, cint, dbl, dbl, dbl, dbl, dbl, dbl, p, p, i64]
    lib.orc_mass.argtypes = [i64, p]
    lib.orc_mass.restype = dbl
    lib.orc_energy.argtypes = [i64, i64, i64, dbl, cint, dbl, dbl, dbl, p]
    lib.orc_energy.restype = dbl
    op2 = [cint, dbl, dbl, dbl, cint, dbl, dbl, dbl, dbl]
    lib.orc_step2.argtypes = [i64, i64, i64, dbl, dbl] + op2 + [p, p, i64]
    lib.orc_energy2.argtypes = [i64, i64, i64, dbl] + op2 + [p, p]
    lib.orc_energy2.restype = dbl
    lib.orc_step_tangent.argtypes = [i64, i64, i64, dbl, dbl, cint, dbl, dbl, dbl, p, p, p]
    lib.orc_step_adjoint.argtypes = [i64, i64, i64, dbl, dbl, cint, dbl, dbl, dbl, p, p, p, p]
    lib.orc_adjoint_run.argtypes = [i64, i64, i64, dbl, dbl, cint, dbl, dbl, dbl, p, i64, p, p, p]
    lib.orc_adjoint_run.restype = dbl
    lib.orc_num_threads.restype = cint
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _dims3(shape):
    if len(shape) == 1:
        return 1, 1, shape[0]
    if len(shape) == 2:
        return 1, shape[0], shape[1]
    if len(shape) == 3:
        return tuple(shape)
    raise ValueError(f"1D, 2D or 3D arrays only, got shape {shape}")


def _op_args(op):
    """op = (kind, r, R1, q2); kind 0 one-mode, 1 two-mode."""
    kind, r, R1, q2 = op
    return int(kind), float(r), float(R1), float(q2)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def dft(x, sign: int = -1) -> np.ndarray:
    x = _c128(x)
    out = np.empty_like(x)
    _load().orc_dft(x.size, _ptr(x), _ptr(out), int(sign))
    return out


def fft_radix2(x, sign: int = -1) -> np.ndarray:
    y = _c128(x).copy()
    _load().orc_fft_radix2(y.size, _ptr(y), int(sign))
    return y


def fft_mixed(x, sign: int = -1) -> np.ndarray:
    y = _c128(x).copy()
    _load().orc_fft_mixed(y.size, _ptr(y), int(sign))
    return y


def fft(x, sign: int = -1) -> np.ndarray:
    y = _c128(x).copy()
    _load().orc_fft(y.size, _ptr(y), int(sign))
    return y


def rfftn(x) -> np.ndarray:
    x = _f64(x)
    nz, ny, nx = _dims3(x.shape)
    out = np.empty(x.shape[:-1] + (nx // 2 + 1,), dtype=np.complex128)
    _load().orc_rfftn(nz, ny, nx, _ptr(x), _ptr(out))
    return out


def irfftn(xh, shape) -> np.ndarray:
    xh = _c128(xh)
    nz, ny, nx = _dims3(shape)
    assert xh.shape == tuple(shape[:-1]) + (nx // 2 + 1,)
    out = np.empty(shape, dtype=np.float64)
    _load().orc_irfftn(nz, ny, nx, _ptr(xh), _ptr(out))
    return out


def lin_op(op, k2: float) -> float:
    return float(_load().orc_lin_op(*_op_args(op), float(k2)))


def step(psi, dx: float, dt: float, op, nsteps: int = 1) -> np.ndarray:
    """Return psi after nsteps semi-implicit steps (input not modified)."""
    y = _f64(psi).copy()
    nz, ny, nx = _dims3(y.shape)
    _load().orc_step(nz, ny, nx, float(dx), float(dt), *_op_args(op), _ptr(y), int(nsteps))
    return y


SEMI_IMPLICIT, STABILIZED, SBDF2 = 0, 1, 2


def step_scheme(psi, dx: float, dt: float, op, scheme: int, S: float = 0.0, nsteps: int = 1) -> np.ndarray:
    """psi after nsteps steps of an alternative integrator (0 semi-implicit, 1 stabilised with
    constant S, 2 second-order BDF with extrapolated nonlinearity started by one step of 0);
    the nsteps steps are one run."""
    y = _f64(psi).copy()
    nz, ny, nx = _dims3(y.shape)
    _load().orc_step_scheme(nz, ny, nx, float(dx), float(dt), *_op_args(op), int(scheme), float(S),
                            _ptr(y), int(nsteps))
    return y


def hydro_step(psi, v, dx: float, dt: float, op, rho: float, gamma: float, a0: float, nsteps: int = 1):
    """(psi, v) after nsteps steps of the hydrodynamic PFC model; v has shape (ndim,) + psi.shape
    (x component first). Inputs are not modified."""
    y = _f64(psi).copy()
    w = _f64(v).copy()
    nz, ny, nx = _dims3(y.shape)
    assert w.shape == ((3 if nz > 1 else 2),) + y.shape
    _load().orc_hydro_step(nz, ny, nx, float(dx), float(dt), *_op_args(op), float(rho), float(gamma), float(a0),
                           _ptr(y), _ptr(w), int(nsteps))
    return y, w


def mass(psi) -> float:
    x = _f64(psi)
    return float(_load().orc_mass(x.size, _ptr(x)))


def energy(psi, dx: float, op) -> float:
    x = _f64(psi)
    nz, ny, nx = _dims3(x.shape)
    return float(_load().orc_energy(nz, ny, nx, float(dx), *_op_args(op), _ptr(x)))


def step2(psi, c, dx: float, dt: float, op_psi, op_c, alpha: float, nsteps: int = 1):
    p = _f64(psi).copy()
    q = _f64(c).copy()
    assert p.shape == q.shape
    nz, ny, nx = _dims3(p.shape)
    _load().orc_step2(nz, ny, nx, float(dx), float(dt), *_op_args(op_psi), *_op_args(op_c),
                      float(alpha), _ptr(p), _ptr(q), int(nsteps))
    return p, q


def energy2(psi, c, dx: float, op_psi, op_c, alpha: float) -> float:
    p, q = _f64(psi), _f64(c)
    nz, ny, nx = _dims3(p.shape)
    return float(_load().orc_energy2(nz, ny, nx, float(dx), *_op_args(op_psi), *_op_args(op_c),
                                     float(alpha), _ptr(p), _ptr(q)))


def step_tangent(psi_n, dpsi, dx: float, dt: float, op) -> np.ndarray:
    p, d = _f64(psi_n), _f64(dpsi)
    out = np.empty_like(p)
    nz, ny, nx = _dims3(p.shape)
    _load().orc_step_tangent(nz, ny, nx, float(dx), float(dt), *_op_args(op), _ptr(p), _ptr(d),
                             _ptr(out))
    return out


def step_adjoint(psi_n, lam_next, dx: float, dt: float, op):
    """Return (lam_n, dr) for one step: lam_n = J^T lam_next, dr = <lam_next, d psi_{n+1}/dr>."""
    p, lam = _f64(psi_n), _f64(lam_next)
    out = np.empty_like(p)
    dr = ctypes.c_double(0.0)
    nz, ny, nx = _dims3(p.shape)
    _load().orc_step_adjoint(nz, ny, nx, float(dx), float(dt), *_op_args(op), _ptr(p), _ptr(lam),
                             _ptr(out), ctypes.byref(dr))
    return out, float(dr.value)


def adjoint_run(psi0, target, dx: float, dt: float, op, nsteps: int):
    """Return (loss, grad_psi0, grad_r) for loss = 0.5 ||psi_T - target||^2."""
    p, t = _f64(psi0), _f64(target)
    g = np.empty_like(p)
    gr = ctypes.c_double(0.0)
    nz, ny, nx = _dims3(p.shape)
    loss = _load().orc_adjoint_run(nz, ny, nx, float(dx), float(dt), *_op_args(op), _ptr(p),
                                   int(nsteps), _ptr(t), _ptr(g), ctypes.byref(gr))
    return float(loss), g, float(gr.value)

"""Python access to the FP64 CPU oracle (ctu_oracle.c) of arXiv:1802.01272.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  The library under
``paper_1802_01272_gb300`` never imports it.

``build()`` compiles ``ctu_oracle.c`` with gcc (OpenMP, no FP contraction, so
x86 and Arm hosts round the same way) into ``oracle/lib/libctu_oracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libctu_oracle.so")
_SRC = os.path.join(_HERE, "ctu_oracle.c")

LIM_MC, LIM_ZERO, LIM_ONE = 0, 1, 2
BC_PERIODIC, BC_SHEAR_WALLS = 0, 1


class _Params(C.Structure):
    _fields_ = [
        ("Lx", C.c_int32), ("Ly", C.c_int32),
        ("a", C.c_double), ("b", C.c_double), ("kappa", C.c_double), ("T", C.c_double),
        ("tau", C.c_double), ("dt", C.c_double), ("ds", C.c_double),
        ("ctu_order", C.c_int32), ("limiter", C.c_int32), ("regularize", C.c_int32),
        ("boundary", C.c_int32), ("shear_rate", C.c_double), ("rho_ext", C.c_double),
        ("reservoir", C.c_int32), ("a2_full", C.c_int32),
    ]


class _Diag(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("mass", "nb", "sx", "sy", "sxx", "sxy", "syy",
                 "rho_center", "rho_ring", "rho_min", "rho_max")]


@dataclass
class Params:
    """Physical and numerical parameters (defaults: Sec. II D-E, III A)."""
    Lx: int = 64
    Ly: int = 64
    a: float = 9.0 / 8.0
    b: float = 1.0 / 3.0
    kappa: float = 1e-4
    T: float = 0.9
    tau: float = 1e-3
    dt: float = 1e-4
    ds: float = 1.0 / 256.0
    ctu_order: int = 2
    limiter: int = LIM_MC
    regularize: int = 0
    boundary: int = BC_PERIODIC
    shear_rate: float = 0.0
    rho_ext: float = 1.0
    reservoir: int = 0
    a2_full: int = 0

    def c(self) -> _Params:
        return _Params(*[getattr(self, f[0]) for f in _Params._fields_])


def build(force: bool = False) -> str:
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ctu_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                        "-std=c11", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        d = P(C.c_double)
        _lib.orc_velocity_set.argtypes = [d, d]
        _lib.orc_pw.argtypes = [P(_Params), C.c_double]
        _lib.orc_pw.restype = C.c_double
        _lib.orc_feq.argtypes = [P(_Params), C.c_double, C.c_double, C.c_double, d]
        _lib.orc_force.argtypes = [P(_Params), C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_double, d, d]
        _lib.orc_init_feq.argtypes = [P(_Params), d, d, d, d]
        _lib.orc_moments.argtypes = [P(_Params), d, d, d, d]
        _lib.orc_accel.argtypes = [P(_Params), d, d, d]
        _lib.orc_regularize.argtypes = [P(_Params), d]
        _lib.orc_reservoir.argtypes = [P(_Params), d]
        _lib.orc_step.argtypes = [P(_Params), d, C.c_int64]
        _lib.orc_step.restype = C.c_int
        _lib.orc_diagnostics.argtypes = [P(_Params), d, C.c_double, C.c_double, P(_Diag)]
        _lib.orc_histogram.argtypes = [P(_Params), d, C.c_int32, C.c_double, C.c_double,
                                       P(C.c_int64)]
        _lib.orc_limiter.argtypes = [C.c_int32, C.c_double]
        _lib.orc_limiter.restype = C.c_double
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def velocity_set():
    xi = np.zeros((16, 2))
    w = np.zeros(16)
    lib().orc_velocity_set(_dp(xi), _dp(w))
    return xi, w


def pw(p: Params, rho: float) -> float:
    return lib().orc_pw(C.byref(p.c()), rho)


def feq(p: Params, rho, ux, uy) -> np.ndarray:
    out = np.zeros(16)
    lib().orc_feq(C.byref(p.c()), rho, ux, uy, _dp(out))
    return out


def force(p: Params, rho, ux, uy, gx, gy, a2=None) -> np.ndarray:
    out = np.zeros(16)
    a2p = _dp(np.ascontiguousarray(a2, dtype=np.float64)) if a2 is not None else None
    lib().orc_force(C.byref(p.c()), rho, ux, uy, gx, gy, a2p, _dp(out))
    return out


def init_feq(p: Params, rho, ux, uy) -> np.ndarray:
    f = np.zeros((16, p.Ly, p.Lx))
    args = [np.ascontiguousarray(x, dtype=np.float64) for x in (rho, ux, uy)]
    lib().orc_init_feq(C.byref(p.c()), *[_dp(x) for x in args], _dp(f))
    return f


def moments(p: Params, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho, ux, uy = (np.zeros((p.Ly, p.Lx)) for _ in range(3))
    lib().orc_moments(C.byref(p.c()), _dp(f), _dp(rho), _dp(ux), _dp(uy))
    return rho, ux, uy


def accel(p: Params, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64)
    gx, gy = np.zeros((p.Ly, p.Lx)), np.zeros((p.Ly, p.Lx))
    lib().orc_accel(C.byref(p.c()), _dp(f), _dp(gx), _dp(gy))
    return gx, gy


def regularize(p: Params, f: np.ndarray) -> np.ndarray:
    f = np.array(f, dtype=np.float64, order="C")
    lib().orc_regularize(C.byref(p.c()), _dp(f))
    return f


def step(p: Params, f: np.ndarray, nsteps: int) -> np.ndarray:
    """Returns f after `nsteps` steps (the input is not modified)."""
    f = np.array(f, dtype=np.float64, order="C")
    assert f.shape == (16, p.Ly, p.Lx)
    rc = lib().orc_step(C.byref(p.c()), _dp(f), int(nsteps))
    if rc != 0:
        raise RuntimeError(f"orc_step failed: {rc}")
    return f


def diagnostics(p: Params, f: np.ndarray, threshold: float, r_ring: float = 0.0) -> dict:
    f = np.ascontiguousarray(f, dtype=np.float64)
    d = _Diag()
    lib().orc_diagnostics(C.byref(p.c()), _dp(f), threshold, r_ring, C.byref(d))
    return {n: getattr(d, n) for n, _ in _Diag._fields_}


def histogram(p: Params, f: np.ndarray, nbins: int, lo: float, hi: float) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    c = np.zeros(nbins, dtype=np.int64)
    lib().orc_histogram(C.byref(p.c()), _dp(f), nbins, lo, hi,
                        c.ctypes.data_as(C.POINTER(C.c_int64)))
    return c


def limiter(kind: int, theta: float) -> float:
    return lib().orc_limiter(kind, theta)

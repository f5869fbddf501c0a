"""ctypes binding of libctulbm.so (include/ctulbm.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts
numpy / torch arrays to pointers, and raises ``LBMError`` on a negative
return code.  If the library is missing it raises: there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, fields

import numpy as np

from . import build as _build

LBM_VEL_D2Q16_H3 = 0
LBM_LIM_MC, LBM_LIM_ZERO, LBM_LIM_ONE = 0, 1, 2
LBM_BC_PERIODIC, LBM_BC_SHEAR_WALLS = 0, 1
LBM_FP64, LBM_FP32_SHIFTED, LBM_FP16_SHIFTED = 0, 1, 2

ERRORS = {
    -1: "LBM_ERR_INVALID_ARG", -2: "LBM_ERR_CFL", -3: "LBM_ERR_DENSITY_RANGE",
    -4: "LBM_ERR_UNSUPPORTED", -5: "LBM_ERR_OOM", -6: "LBM_ERR_CUDA", -7: "LBM_ERR_NONFINITE",
    -8: "LBM_ERR_DEVICE_BOUNDS", -9: "LBM_ERR_TIMEOUT",
}


class LBMError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = lib().lbm_strerror(code).decode() if _lib is not None else ERRORS.get(code, "?")
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({msg})")


class lbm_params(C.Structure):
    _fields_ = [
        ("Lx", C.c_int32), ("Ly", C.c_int32), ("velset", C.c_int32),
        ("a", C.c_double), ("b", C.c_double), ("kappa", C.c_double), ("T", C.c_double),
        ("tau", C.c_double), ("dt", C.c_double), ("ds", C.c_double),
        ("ctu_order", C.c_int32), ("limiter", C.c_int32), ("regularize", C.c_int32),
        ("boundary", C.c_int32), ("shear_rate", C.c_double), ("rho_ext", C.c_double),
        ("reservoir", C.c_int32), ("precision", C.c_int32), ("rho_ref", C.c_double),
    ]


class lbm_kernel_info(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("grid", "threads", "smem_bytes", "strips", "row_block",
                                         "tensor_copies")]


class lbm_diag(C.Structure):
    _fields_ = [
        ("mass", C.c_double), ("nb", C.c_int64), ("sx", C.c_int64), ("sy", C.c_int64),
        ("sxx", C.c_int64), ("sxy", C.c_int64), ("syy", C.c_int64),
        ("rho_center", C.c_double), ("rho_ring", C.c_double), ("rho_min", C.c_double),
        ("rho_max", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
        ("a", C.c_double), ("b", C.c_double), ("D", C.c_double), ("theta", C.c_double),
    ]


class lbm_job_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("error", C.c_int32), ("steps_done", C.c_int64),
                ("nsteps", C.c_int64), ("diag_step", C.c_int64), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_finish", C.c_double), ("diag", lbm_diag)]


class lbm_batch_info(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("pending", "active", "done", "failed", "used_bytes",
                                         "node_updates", "launches")]


LBM_JOB_PENDING, LBM_JOB_ACTIVE, LBM_JOB_DONE, LBM_JOB_FAILED = 0, 1, 2, 3


_lib = None
EXPORTS = ["lbm_default_params", "lbm_create", "lbm_destroy", "lbm_init_rho_u", "lbm_step_many",
           "lbm_step_diag",
           "lbm_init_rho_u_device", "lbm_set_f", "lbm_get_f", "lbm_set_f_device",
           "lbm_get_f_device", "lbm_step", "lbm_moments", "lbm_moments_device",
           "lbm_diagnostics", "lbm_histogram", "lbm_sync", "lbm_step_count", "lbm_strerror",
           "lbm_get_kernel_info", "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_submit",
           "lbm_batch_poll", "lbm_batch_wait", "lbm_batch_fetch", "lbm_batch_get_info", "lbm_tune",
           "lbm_measure_peaks", "lbm_set_launch"]


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libctulbm.so (building it first if sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libctulbm.so is missing: the CUDA extension was not built")
        L = C.CDLL(path)
        P, d, vp, i64 = C.POINTER, C.POINTER(C.c_double), C.c_void_p, C.c_int64
        H = C.c_void_p
        L.lbm_default_params.argtypes = [P(lbm_params), C.c_int32, C.c_int32]
        L.lbm_create.argtypes = [P(lbm_params), vp, P(H)]
        L.lbm_destroy.argtypes = [H]
        L.lbm_destroy.restype = None
        for n in ("lbm_init_rho_u", "lbm_init_rho_u_device", "lbm_moments", "lbm_moments_device"):
            getattr(L, n).argtypes = [H, vp, vp, vp]
        for n in ("lbm_set_f", "lbm_get_f", "lbm_set_f_device", "lbm_get_f_device"):
            getattr(L, n).argtypes = [H, vp]
        L.lbm_step.argtypes = [H, i64]
        L.lbm_step_many.argtypes = [P(H), C.c_int32, i64]
        L.lbm_step_diag.argtypes = [H, i64, C.c_double, P(lbm_diag)]
        L.lbm_diagnostics.argtypes = [H, C.c_double, C.c_double, P(lbm_diag)]
        L.lbm_histogram.argtypes = [H, C.c_int32, C.c_double, C.c_double, P(C.c_int64)]
        L.lbm_sync.argtypes = [H]
        L.lbm_step_count.argtypes = [H]
        L.lbm_step_count.restype = i64
        L.lbm_get_kernel_info.argtypes = [H, P(lbm_kernel_info)]
        L.lbm_tune.argtypes = [H, C.c_int32, P(lbm_kernel_info)]
        L.lbm_set_launch.argtypes = [H, C.c_int32, C.c_int32]
        L.lbm_measure_peaks.argtypes = [vp, d, d]
        B = C.c_void_p
        L.lbm_batch_create.argtypes = [C.c_size_t, C.c_int32, vp, P(B)]
        L.lbm_batch_destroy.argtypes = [B]
        L.lbm_batch_destroy.restype = None
        L.lbm_batch_submit.argtypes = [B, P(lbm_params), vp, vp, vp, i64, i64, C.c_double]
        L.lbm_batch_submit.restype = i64
        L.lbm_batch_poll.argtypes = [B, i64, P(lbm_job_result)]
        L.lbm_batch_wait.argtypes = [B, i64, C.c_double, P(lbm_job_result)]
        L.lbm_batch_fetch.argtypes = [B, i64, vp, vp, vp]
        L.lbm_batch_get_info.argtypes = [B, P(lbm_batch_info)]
        L.lbm_histogram_noalloc.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                            C.c_int32, C.c_double, C.c_double, vp, P(C.c_int64)]
        L.lbm_strerror.argtypes = [C.c_int]
        L.lbm_strerror.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise LBMError(rc, what)


@dataclass
class Params:
    """Mirror of lbm_params; defaults as lbm_default_params."""
    Lx: int = 64
    Ly: int = 64
    velset: int = LBM_VEL_D2Q16_H3
    a: float = 9.0 / 8.0
    b: float = 1.0 / 3.0
    kappa: float = 1e-4
    T: float = 0.9
    tau: float = 1e-3
    dt: float = 1e-4
    ds: float = 1.0 / 256.0
    ctu_order: int = 2
    limiter: int = LBM_LIM_MC
    regularize: int = 0
    boundary: int = LBM_BC_PERIODIC
    shear_rate: float = 0.0
    rho_ext: float = 1.0
    reservoir: int = 0
    precision: int = LBM_FP32_SHIFTED
    rho_ref: float = 1.0

    def c(self) -> lbm_params:
        return lbm_params(*[getattr(self, f.name) for f in fields(self)])


def lbm_default_params(Lx: int, Ly: int) -> Params:
    p = lbm_params()
    _check(lib().lbm_default_params(C.byref(p), Lx, Ly), "lbm_default_params")
    return Params(**{n: getattr(p, n) for n, _ in lbm_params._fields_})


def _host(a: np.ndarray, shape) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _dev(t, shape):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous() and tuple(t.shape) == tuple(shape)):
        raise ValueError(f"expected a contiguous float64 CUDA tensor of shape {shape}")
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def lbm_create(params: Params, stream=None):
    h = C.c_void_p()
    _check(lib().lbm_create(C.byref(params.c()), _stream_ptr(stream), C.byref(h)), "lbm_create")
    return h


def lbm_destroy(h):
    lib().lbm_destroy(h)


def step_many(lattices, n: int):
    """lbm_step_many over Lattice objects: one fused launch per step for all
    compatible lattices (equal to stepping each alone, to FP32 rounding)."""
    arr = (C.c_void_p * len(lattices))(*[L.handle for L in lattices])
    _check(lib().lbm_step_many(arr, len(lattices), int(n)), "lbm_step_many")


NOALLOC_MAX_BINS = 4096


def measure_peaks(stream=None) -> dict:
    """lbm_measure_peaks: measured FP32 flop/s and warp-instruction issue rate
    of the current device."""
    f, i = C.c_double(), C.c_double()
    _check(lib().lbm_measure_peaks(_stream_ptr(stream), C.byref(f), C.byref(i)),
           "lbm_measure_peaks")
    return {"fp32_flops": f.value, "issue_rate": i.value}


def histogram_noalloc(f, precision: int, rho_ref: float, nbins: int, lo: float, hi: float,
                      stream=None) -> np.ndarray:
    """lbm_histogram_noalloc on a caller-owned torch CUDA tensor f of shape
    [16, Ly, Lx] (float64 for LBM_FP64, shifted float32 / float16 for
    LBM_FP32_SHIFTED / LBM_FP16_SHIFTED).  Allocates no device memory; see
    include/ctulbm.h for the shared-array rules."""
    import torch
    want = {LBM_FP64: torch.float64, LBM_FP16_SHIFTED: torch.float16}.get(precision, torch.float32)
    if not (isinstance(f, torch.Tensor) and f.is_cuda and f.dtype == want and f.is_contiguous()
            and f.dim() == 3 and f.shape[0] == 16):
        raise ValueError(f"expected a contiguous {want} CUDA tensor of shape [16, Ly, Lx]")
    counts = np.zeros(nbins, dtype=np.int64)
    with torch.cuda.device(f.device):  # the library counts on the current device
        _check(lib().lbm_histogram_noalloc(C.c_void_p(f.data_ptr()), f.shape[2], f.shape[1],
                                           precision, rho_ref, nbins, lo, hi, _stream_ptr(stream),
                                           counts.ctypes.data_as(C.POINTER(C.c_int64))),
               "lbm_histogram_noalloc")
    return counts


class Lattice:
    """A lattice owned by the library.  Host arrays are float64 numpy
    (fields [Ly][Lx], distributions [16][Ly][Lx]); *_device take float64
    torch CUDA tensors of the same shapes."""

    def __init__(self, params: Params, stream=None):
        self.params = params
        self.stream = stream
        self._h = lbm_create(params, stream)
        self.shape = (params.Ly, params.Lx)

    def close(self):
        if self._h:
            lbm_destroy(self._h)
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

    @property
    def handle(self):
        return self._h

    def init_rho_u(self, rho, ux, uy):
        a = [_host(x, self.shape) for x in (rho, ux, uy)]
        _check(lib().lbm_init_rho_u(self._h, *[x.ctypes.data for x in a]), "lbm_init_rho_u")

    def init_rho_u_device(self, rho, ux, uy):
        _check(lib().lbm_init_rho_u_device(self._h, *[_dev(x, self.shape) for x in (rho, ux, uy)]),
               "lbm_init_rho_u_device")

    def set_f(self, f):
        f = _host(f, (16,) + self.shape)
        _check(lib().lbm_set_f(self._h, f.ctypes.data), "lbm_set_f")

    def get_f(self) -> np.ndarray:
        out = np.empty((16,) + self.shape)
        _check(lib().lbm_get_f(self._h, out.ctypes.data), "lbm_get_f")
        return out

    def set_f_device(self, f):
        _check(lib().lbm_set_f_device(self._h, _dev(f, (16,) + self.shape)), "lbm_set_f_device")

    def get_f_device(self, out):
        _check(lib().lbm_get_f_device(self._h, _dev(out, (16,) + self.shape)), "lbm_get_f_device")
        return out

    def step(self, n: int = 1):
        _check(lib().lbm_step(self._h, int(n)), "lbm_step")

    def step_diag(self, n: int, threshold: float) -> dict:
        """lbm_step_diag: n steps, diagnostics of the final state fused into the
        last step (mass, bubble sites, gyration shape)."""
        d = lbm_diag()
        _check(lib().lbm_step_diag(self._h, int(n), threshold, C.byref(d)), "lbm_step_diag")
        return {n_: getattr(d, n_) for n_, _ in lbm_diag._fields_}

    def moments(self, out=None):
        """(rho, ux, uy) as float64 [Ly][Lx]; `out` may supply three C-contiguous
        float64 arrays (e.g. views of pinned host memory) to fill."""
        if out is None:
            out = tuple(np.empty(self.shape) for _ in range(3))
        rho, ux, uy = out
        for x in out:
            if x.dtype != np.float64 or not x.flags.c_contiguous or x.shape != self.shape:
                raise ValueError("moments: out arrays must be C-contiguous float64 [Ly][Lx]")
        _check(lib().lbm_moments(self._h, rho.ctypes.data, ux.ctypes.data, uy.ctypes.data),
               "lbm_moments")
        return rho, ux, uy

    def moments_device(self, rho, ux, uy):
        _check(lib().lbm_moments_device(self._h, *[_dev(x, self.shape) for x in (rho, ux, uy)]),
               "lbm_moments_device")

    def diagnostics(self, threshold: float, r_ring: float = 0.0) -> dict:
        d = lbm_diag()
        _check(lib().lbm_diagnostics(self._h, threshold, r_ring, C.byref(d)), "lbm_diagnostics")
        return {n: getattr(d, n) for n, _ in lbm_diag._fields_}

    def histogram(self, nbins: int, lo: float, hi: float) -> np.ndarray:
        c = np.zeros(nbins, dtype=np.int64)
        _check(lib().lbm_histogram(self._h, nbins, lo, hi, c.ctypes.data_as(C.POINTER(C.c_int64))),
               "lbm_histogram")
        return c

    def sync(self):
        _check(lib().lbm_sync(self._h), "lbm_sync")

    @property
    def step_count(self) -> int:
        return lib().lbm_step_count(self._h)

    def tune(self, steps_per_trial: int = 3) -> dict:
        """lbm_tune: time each launch geometry for steps_per_trial real steps and
        keep the fastest; returns the chosen geometry (as kernel_info)."""
        k = lbm_kernel_info()
        _check(lib().lbm_tune(self._h, int(steps_per_trial), C.byref(k)), "lbm_tune")
        return {n: getattr(k, n) for n, _ in lbm_kernel_info._fields_}

    def set_launch(self, row_block: int, ctas_per_sm: int = 0) -> dict:
        """lbm_set_launch: fix the launch geometry (ctas_per_sm 0: the most that
        fit on an SM); returns kernel_info."""
        _check(lib().lbm_set_launch(self._h, int(row_block), int(ctas_per_sm)), "lbm_set_launch")
        return self.kernel_info()

    def kernel_info(self) -> dict:
        """Launch geometry of the step kernel (lbm_get_kernel_info)."""
        k = lbm_kernel_info()
        _check(lib().lbm_get_kernel_info(self._h, C.byref(k)), "lbm_get_kernel_info")
        return {n: getattr(k, n) for n, _ in lbm_kernel_info._fields_}

"""ctypes declarations of the C ABI in ``include/mppi.h``.

Argument marshalling only: every function below forwards to the CUDA library
``libmppi_gb300.so``.  There is no CPU fallback; loading fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

c_float_p = ctypes.POINTER(ctypes.c_float)
c_u32_p = ctypes.POINTER(ctypes.c_uint32)

STATUS = {
    0: "MPPI_OK", 1: "MPPI_ERR_INVALID_ARG", 2: "MPPI_ERR_CUDA", 3: "MPPI_ERR_OOM",
    4: "MPPI_ERR_UNSUPPORTED", 5: "MPPI_ERR_NUMERIC", 6: "MPPI_ERR_TIMEOUT",
}
MPPI_OK, MPPI_ERR_INVALID_ARG, MPPI_ERR_CUDA, MPPI_ERR_OOM = 0, 1, 2, 3
MPPI_ERR_UNSUPPORTED, MPPI_ERR_NUMERIC, MPPI_ERR_TIMEOUT = 4, 5, 6
MPPI_PREC_FP32, MPPI_PREC_BF16_MLP = 0, 1


class MPPIError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {STATUS.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class DynamicsDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("integrator", ctypes.c_int), ("nx", ctypes.c_int),
                ("nu", ctypes.c_int), ("params", c_float_p), ("n_params", ctypes.c_size_t)]


class CostDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("params", c_float_p), ("n_params", ctypes.c_size_t),
                ("map", c_float_p), ("map_h", ctypes.c_int), ("map_w", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_int), ("precision", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("block_threads", ctypes.c_int), ("rollout_variant", ctypes.c_int),
                ("checked", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class InstanceDesc(ctypes.Structure):
    _fields_ = [("dyn", DynamicsDesc), ("cost", CostDesc), ("K", ctypes.c_int), ("T", ctypes.c_int),
                ("dt", ctypes.c_float), ("lambda_", ctypes.c_float), ("sigma", c_float_p),
                ("seed", ctypes.c_uint64), ("beta", ctypes.c_int), ("x0_d", ctypes.c_void_p), ("u_nom_d", ctypes.c_void_p),
                ("u_new_d", ctypes.c_void_p), ("stats_d", ctypes.c_void_p)]


_lib = None


def load() -> ctypes.CDLL:
    """Load the CUDA library (never builds implicitly; call ``build()`` first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB_PATH):
        raise RuntimeError(
            f"{_build.LIB_NAME} is not built; run paper_2409_07563_gb300.build() "
            "(nvcc, sm_103a). There is no CPU fallback.")
    L = ctypes.CDLL(_build.LIB_PATH)
    vp, i, f, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_uint64
    L.mppi_default_options.argtypes = [ctypes.POINTER(Options)]
    L.mppi_default_options.restype = None
    L.mppi_create.argtypes = [ctypes.POINTER(DynamicsDesc), ctypes.POINTER(CostDesc), i, i, f, f,
                              c_float_p, ctypes.POINTER(Options), ctypes.POINTER(vp)]
    L.mppi_destroy.argtypes = [vp]
    L.mppi_destroy.restype = None
    L.mppi_set_stream.argtypes = [vp, vp]
    L.mppi_step.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.mppi_step_host.argtypes = [vp, c_float_p, c_float_p, c_float_p, c_float_p]
    L.mppi_set_params.argtypes = [vp, c_float_p, c_float_p]
    L.mppi_set_params_device.argtypes = [vp, vp, vp]
    L.mppi_step_backward.argtypes = [vp, vp, vp]
    L.mppi_get_counter.argtypes = [vp, ctypes.POINTER(u64)]
    L.mppi_set_counter.argtypes = [vp, u64]
    L.mppi_poll_status.argtypes = [vp]
    L.mppi_last_error.argtypes = [vp]
    L.mppi_last_error.restype = ctypes.c_char_p
    L.mppi_sample_noise.argtypes = [u64, u64, i, i, vp, vp, vp]
    L.mppi_profile.argtypes = [vp, i]
    L.mppi_profile_read.argtypes = [vp, c_float_p, ctypes.POINTER(ctypes.c_int)]
    L.mppi_set_iterations.argtypes = [vp, i, ctypes.c_float]
    L.mppi_nominal_trajectory.argtypes = [vp, vp, vp, vp]
    L.mppi_shift.argtypes = [vp, vp, i, vp]
    L.mppi_set_cem.argtypes = [vp, ctypes.c_float]
    for name in ("mppi_create", "mppi_set_stream", "mppi_step", "mppi_step_host",
                 "mppi_set_params", "mppi_set_params_device", "mppi_step_backward",
                 "mppi_get_counter",
                 "mppi_set_counter", "mppi_poll_status", "mppi_sample_noise", "mppi_profile",
                 "mppi_profile_read", "mppi_set_iterations", "mppi_nominal_trajectory",
                 "mppi_shift", "mppi_set_cem"):
        getattr(L, name).restype = ctypes.c_int
    # mppi_step_host on raw host addresses (Python ints): the same symbol with
    # void-pointer arguments, so a per-step call needs no pointer casts
    L.mppi_step_host_addr = ctypes.CFUNCTYPE(ctypes.c_int, vp, vp, vp, vp, vp)(
        ("mppi_step_host", L))
    _optional(L)
    _lib = L
    return L


def _optional(L):
    """Entry points added after the single-instance path."""
    vp, i = ctypes.c_void_p, ctypes.c_int
    if hasattr(L, "mppi_update_noalloc"):
        u64 = ctypes.c_uint64
        L.mppi_update_noalloc.argtypes = [vp, i, i, i, ctypes.c_float, c_float_p, u64, u64,
                                          vp, vp, vp, vp, vp]
        L.mppi_update_noalloc.restype = ctypes.c_int
    if hasattr(L, "mppi_fp32_fma_probe"):
        L.mppi_fp32_fma_probe.argtypes = [i, i, ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_double)]
        L.mppi_fp32_fma_probe.restype = ctypes.c_int
    if hasattr(L, "mppi_batch_create"):
        L.mppi_batch_create.argtypes = [i, ctypes.POINTER(InstanceDesc), ctypes.POINTER(Options),
                                        ctypes.POINTER(vp)]
        L.mppi_batch_create.restype = ctypes.c_int
        L.mppi_batch_step.argtypes = [vp, vp]
        L.mppi_batch_step.restype = ctypes.c_int
        L.mppi_batch_latency.argtypes = [vp, vp, c_float_p]
        L.mppi_batch_latency.restype = ctypes.c_int
        L.mppi_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.mppi_batch_info.restype = ctypes.c_int
        L.mppi_batch_destroy.argtypes = [vp]
        L.mppi_batch_destroy.restype = None
        L.mppi_batch_samples.argtypes = [vp, i, vp, vp, vp]
        L.mppi_batch_samples.restype = ctypes.c_int


def exported_symbols():
    """Names of the mppi_* functions the loaded library exports."""
    L = load()
    out = []
    for name in dir(L):
        if name.startswith("mppi_"):
            out.append(name)
    return out


def check(status: int, where: str, ctx=None):
    if status != MPPI_OK:
        detail = ""
        if ctx:
            msg = load().mppi_last_error(ctx)
            detail = msg.decode() if msg else ""
        raise MPPIError(status, where, detail)

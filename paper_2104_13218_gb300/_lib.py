"""ctypes loader of libkpm.so and the C prototypes of include/kpm.h.

The library is built in-tree (paper_2104_13218_gb300/_build/libkpm.so).  If
it is missing, `lib()` builds it when nvcc is available and otherwise raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_uint64 = ctypes.c_uint64
c_double = ctypes.c_double
c_size_t = ctypes.c_size_t
c_void_p = ctypes.c_void_p

KPM_OK = 0
KPM_EINVAL = 1
KPM_ENOMEM = 2
KPM_ECUDA = 3
KPM_ENOTCONV = 5
KPM_EBOUNDS = 6
KPM_FP64 = 0
KPM_FP32 = 1
KPM_KERNEL_NONE = 0
KPM_KERNEL_JACKSON = 1
KPM_VECTORS_RADEMACHER = 0
KPM_VECTORS_BASIS = 1

STATUS_NAMES = {0: "KPM_OK", 1: "KPM_EINVAL", 2: "KPM_ENOMEM", 3: "KPM_ECUDA",
                5: "KPM_ENOTCONV", 6: "KPM_EBOUNDS"}


class KpmModel(ctypes.Structure):
    _fields_ = [("n_sites", c_int32), ("n_bonds", c_int32), ("bi", c_void_p), ("bj", c_void_p),
                ("J", c_void_p)]


class KpmOpts(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("vectors", c_int32), ("per_vector", c_int32),
                ("tuned", c_int32), ("ckpt_interval", c_int32), ("reserved", c_int32 * 3)]


class KpmSpinModel(ctypes.Structure):
    _fields_ = [("n_sites", c_int32), ("n_bonds", c_int32), ("two_s", c_int32), ("pad", c_int32),
                ("bi", c_void_p), ("bj", c_void_p), ("J", c_void_p)]


P = c_void_p
PROTOTYPES = {
    "kpm_version": (c_int32, []),
    "kpm_last_error": (ctypes.c_char_p, []),
    "kpm_sector_dim": (c_int64, [c_int32, c_int32]),
    "kpm_bounds": (c_int32, [P, c_int32, P, c_double, c_int32, c_double, c_uint64, P, P, P, P, P,
                             c_size_t, P]),
    "kpm_bounds_workspace_size": (c_size_t, [P, c_int32, P]),
    "kpm_moments": (c_int32, [P, c_int32, P, P, P, c_double, c_int32, c_int32, c_uint64, c_uint64,
                              c_int32, P, P, P, c_int32, P, c_size_t, P]),
    "kpm_moments_workspace_size": (c_size_t, [P, c_int32, P, c_int32, c_int32, c_int32]),
    "kpm_thermo": (c_int32, [c_int32, c_int32, P, P, P, P, P, P, P, c_int32, c_int32, c_int32, P,
                             P, P, P, P, P, c_int32, P]),
    "kpm_thermo_backward": (c_int32, [c_int32, c_int32, P, P, P, P, P, P, P, c_int32, c_int32,
                                      c_int32, P, P, P, P, P, P, P, P, c_int32, P]),
    "kpm_moments_backward": (c_int32, [P, P, c_int32, c_int32, P, P, P, c_int32, c_int32, c_uint64,
                                       c_uint64, c_int32, c_int32, P, P, P, P, c_int32, P, c_size_t,
                                       P]),
    "kpm_moments_backward_workspace_size": (c_size_t, [P, c_int32, P, c_int32, c_int32, c_int32]),
    "kpm_moments_static": (c_int32, [P, c_int32, P, P, P, c_int32, c_int32, c_uint64, c_uint64,
                                     c_int32, P, P, P, P]),
    "kpm_static_scratch_bytes": (c_size_t, []),
    "kpm_moments_ex": (c_int32, [P, c_int32, P, P, P, c_double, c_int32, c_int32, c_uint64,
                                 c_uint64, P, P, P, P, P, c_int32, P, c_size_t, P]),
    "kpm_moments_ex_workspace_size": (c_size_t, [P, c_int32, P, c_int32, c_int32, P]),
    "kpm_autotune": (c_int32, [P, c_int32, P, P, P, c_int32, c_int32, c_int32, P, P, P, c_size_t,
                               P]),
    "kpm_moments_backward_ex": (c_int32, [P, P, c_int32, c_int32, P, P, P, c_int32, c_int32,
                                          c_uint64, c_uint64, P, P, P, P, P, c_int32, P, c_size_t,
                                          P]),
    "kpm_thermo_ex": (c_int32, [c_int32, c_int32, P, P, P, P, P, P, P, P, c_double, c_int32,
                                c_int32, c_int32, P, P, P, P, P, P, c_int32, P]),
    "kpm_thermo_backward_ex": (c_int32, [c_int32, c_int32, P, P, P, P, P, P, P, P, c_double,
                                         c_int32, c_int32, c_int32, P, P, P, P, P, P, P, P,
                                         c_int32, P]),
    "kpm_realisations": (c_int32, [c_int32, c_int32, c_int32, c_int32, P, P, P, P, P, P, c_double,
                                   c_int32, c_int32, c_int32, P, P, P, P, P, P, c_int32, P]),
    "kpm_fp64_peak": (c_int32, [P, P, P]),
    "kpm_spin_sector_dim": (c_int64, [c_int32, c_int32, c_int32]),
    "kpm_spin_bounds": (c_int32, [P, c_int32, P, c_double, c_int32, c_double, c_uint64, P, P, P, P,
                                  P]),
    "kpm_spin_moments": (c_int32, [P, c_int32, P, P, P, c_int32, c_int32, c_uint64, c_uint64,
                                   c_int32, P, P, P, c_int32, P]),
    "kpm_profile_enable": (c_int32, [c_int32]),
    "kpm_profile_read": (c_int32, [P, P, P]),
}

_handle = None


class KPMError(RuntimeError):
    def __init__(self, func, code, message):
        super().__init__(f"{func} returned {STATUS_NAMES.get(code, code)}: {message}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libkpm.so (built first if needed); raises if it cannot be built."""
    global _handle
    if _handle is None:
        path = _build.LIB
        if not _build.up_to_date():
            try:
                _build.build()
            except Exception as exc:  # no nvcc or a compile error: no fallback
                if not os.path.exists(path):
                    raise RuntimeError(f"libkpm.so is not built and cannot be built: {exc}") from exc
        h = ctypes.CDLL(path)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _handle = h
    return _handle


def check(func: str, code: int, allow=()):
    if code != KPM_OK and code not in allow:
        msg = lib().kpm_last_error()
        raise KPMError(func, code, msg.decode() if msg else "")
    return code

"""ctypes loader of the plain C oracle (naive_kpm.c) -- TEST INFRASTRUCTURE.

Only tests, the smoke check and the benchmark's CPU-baseline leg use this.
`build()` compiles naive_kpm.c with gcc and OpenMP into oracle/_build/.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "naive_kpm.c")
_LIB = os.path.join(_HERE, "_build", "libnaive_kpm.so")
_handle = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", _LIB, _SRC, "-lm"])
    return _LIB


def lib():
    global _handle
    if _handle is None:
        build()
        h = ctypes.CDLL(_LIB)
        h.oracle_kpm_moments.restype = ctypes.c_int
        h.oracle_kpm_moments.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p]
        h.oracle_sector_dim.restype = ctypes.c_int64
        h.oracle_sector_dim.argtypes = [ctypes.c_int, ctypes.c_int]
        h.oracle_sector_states.restype = ctypes.c_int
        h.oracle_sector_states.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        h.oracle_rank.restype = ctypes.c_uint64
        h.oracle_rank.argtypes = [ctypes.c_uint64]
        h.oracle_num_threads.restype = ctypes.c_int
        _handle = h
    return _handle


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def sector_states(n_sites: int, n_up: int) -> np.ndarray:
    D = int(lib().oracle_sector_dim(n_sites, n_up))
    out = np.zeros(D, dtype=np.uint64)
    lib().oracle_sector_states(n_sites, n_up, out.ctypes.data)
    return out


def rank(s: int) -> int:
    return int(lib().oracle_rank(s))


def moments(n_sites, bi, bj, J, n_up, m, c, K, R, seed, r0=0, max_steps=0):
    """dict(mu, mu_M, mu_M2) of one sector from the C oracle."""
    bi = np.ascontiguousarray(bi, dtype=np.int32)
    bj = np.ascontiguousarray(bj, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.float64)
    mu = np.zeros(K)
    muM = np.zeros(K)
    muM2 = np.zeros(K)
    rc = lib().oracle_kpm_moments(n_sites, len(bi), bi.ctypes.data, bj.ctypes.data, J.ctypes.data,
                                  n_up, m, c, K, R, seed, r0, max_steps, mu.ctypes.data,
                                  muM.ctypes.data, muM2.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_kpm_moments failed ({rc})")
    out = {"mu": mu}
    if n_up < 0:
        out["mu_M"] = muM
        out["mu_M2"] = muM2
    return out

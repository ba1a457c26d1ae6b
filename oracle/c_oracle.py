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
        # build beside the library and rename over it: a process that has the old one
        # loaded keeps its (unlinked) copy intact
        tmp = f"{_LIB}.{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
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
        h.oracle_kpm_moments_lean.restype = ctypes.c_int
        h.oracle_kpm_moments_lean.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint64,
            ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
        h.oracle_spin_sector_dim.restype = ctypes.c_int64
        h.oracle_spin_sector_dim.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        h.oracle_spin_moments.restype = ctypes.c_int
        h.oracle_spin_moments.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
            ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p]
        h.oracle_local_moments.restype = ctypes.c_int
        h.oracle_local_moments.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_uint64,
            ctypes.c_uint64, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p]
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


def local_moments(n_sites, bi, bj, J, n_up, m, c, R, seed, r0=0, n_mom=5, max_states=0):
    """mu_0 .. mu_{n_mom-1} (n_mom = 3 or 5) of one sector, evaluated state by state
    without storing vectors (for sectors too large for `moments`); max_states > 0 sums
    only over the first max_states ranks (a timing sample)."""
    bi = np.ascontiguousarray(bi, dtype=np.int32)
    bj = np.ascontiguousarray(bj, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.float64)
    mu = np.zeros(n_mom)
    rc = lib().oracle_local_moments(n_sites, len(bi), bi.ctypes.data, bj.ctypes.data,
                                    J.ctypes.data, n_up, m, c, R, seed, r0, n_mom, max_states,
                                    mu.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_local_moments failed ({rc})")
    return mu


def moments_lean(n_sites, bi, bj, J, n_up, m, c, K, seed, r0=0, max_steps=0):
    """mu[K] of one sector for one random vector (index r0) by the recursion with two
    stored vectors (for sectors whose four arrays would not fit in host memory)."""
    bi = np.ascontiguousarray(bi, dtype=np.int32)
    bj = np.ascontiguousarray(bj, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.float64)
    mu = np.zeros(K)
    rc = lib().oracle_kpm_moments_lean(n_sites, len(bi), bi.ctypes.data, bj.ctypes.data,
                                       J.ctypes.data, n_up, m, c, K, seed, r0, max_steps,
                                       mu.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_kpm_moments_lean failed ({rc})")
    return mu


def spin_sector_dim(n_sites, two_s, Q):
    return int(lib().oracle_spin_sector_dim(n_sites, two_s, Q))


def spin_moments(n_sites, two_s, bi, bj, J, Q, m, c, K, R, seed, r0=0):
    """dict(mu, mu_M, mu_M2) of one spin-s sector (digit sum Q; -1 = all states)."""
    bi = np.ascontiguousarray(bi, dtype=np.int32)
    bj = np.ascontiguousarray(bj, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.float64)
    mu, muM, muM2 = np.zeros(K), np.zeros(K), np.zeros(K)
    rc = lib().oracle_spin_moments(n_sites, two_s, len(bi), bi.ctypes.data, bj.ctypes.data,
                                   J.ctypes.data, Q, m, c, K, R, seed, r0, mu.ctypes.data,
                                   muM.ctypes.data, muM2.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle_spin_moments failed ({rc})")
    out = {"mu": mu}
    if Q < 0:
        out["mu_M"] = muM
        out["mu_M2"] = muM2
    return out

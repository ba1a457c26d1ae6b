"""The benchmark workloads at their full sizes, in the launch configurations the benchmark
times, against the oracle, and the FP32 form's error on the thermodynamics.

* ring N = 20, all 21 sectors, R = 100, K = 1000: every moment of every sector against
  the C oracle run on the same vectors (FP64 to 1e-10 max(1, |mu|), FP32 to 1e-5), and
  the FP32 form's C(T) and chi(T) against the oracle's thermodynamics on the 200-point
  grid T in [0.02, 10].
* J1-J2 4 x 6 torus, full 2^24 space, R = 64, K = 2000: vectors 0 and 1 of the run
  (per-vector moments) against the stored oracle moments of those two vectors (all 2000);
  FP64 on the same two vectors; and the FP32 form's C(T), chi(T) against the FP64 form.
* ring N = 34, S^z = 0 (D = 2 333 606 220, ranks above 2^31): R = 4 FP32 (vector 0 via
  per-vector moments) and R = 1 FP64 against the stored oracle moments mu_0 .. mu_7;
  FP32 against FP64 over 20 steps.

The stored oracle moments come from tests/golden/make_large_sector_moments.py (the plain
C recursion of oracle/naive_kpm.c).  The measured thermodynamic errors are written to
$KPM_RECORD_DIR/fp32_thermo_error.json when that variable names a folder.
"""
import json
import math
import os

import numpy as np
import pytest

import kpm_workloads as W
import paper_2104_13218_gb300 as kpm
from oracle import c_oracle
from oracle import kpm_oracle as O
from tests.conftest import GOLDEN, ROOT

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


def _golden_moments(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    meta = {}
    rows = []
    with open(path) as f:
        for line in f:
            if line.startswith("# n_up"):
                t = line[2:].split()
                meta = {t[i]: float(t[i + 1]) for i in range(0, len(t), 2)}
            if line.startswith("#") or not line.strip():
                continue
            rows.append([float(x) for x in line.split()[1:]])
    return meta, np.array(rows).T  # [vector, n]


def _record(key, value):
    out = os.environ.get("KPM_RECORD_DIR", "")
    if not out or not os.path.isdir(out):
        return
    path = os.path.join(out, "fp32_thermo_error.json")
    d = {}
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
    d[key] = value
    with open(path, "w") as f:
        json.dump(d, f, indent=1)


def _thermo_error(th32, th64, T):
    """max |dC| / max |C| and max |dchi| / max |chi| over the grid, the temperature of the
    largest deviation, the same maximum over T >= 0.1, and the whole profile."""
    out = {}
    T = np.asarray(T)
    hi = T >= 0.1
    for q in ("C", "chi"):
        ref = np.asarray(th64[q])
        d = np.abs(np.asarray(th32[q]) - ref)
        peak = np.abs(ref).max()
        out[q] = {"max_abs": float(d.max()), "max_rel_to_peak": float(d.max() / peak),
                  "T_at_max": float(T[int(d.argmax())]),
                  "max_rel_to_peak_T_ge_0.1": float(d[hi].max() / peak),
                  "profile_rel_to_peak": [float(x) for x in d / peak]}
    return out


def test_ring20_all_sectors_every_moment():
    w = W.workload("ring20_sectors")
    bnd = kpm.bounds(w.model, w.n_up, eps=w.eps, max_iter=100, tol=1e-8, seed=w.seed)
    a, b = bnd["a"], bnd["b"]
    bi, bj, J = w.model.arrays()
    ref = [c_oracle.moments(20, bi, bj, J, k, a[i], b[i], w.K, w.R, w.seed)["mu"]
           for i, k in enumerate(w.n_up)]
    ref = np.array(ref)
    out = {}
    for prec, tol in (("fp64", TOL64), ("fp32", TOL32)):
        gpu = kpm.moments(w.model, w.n_up, w.K, w.R, w.seed, a=a, b=b, precision=prec)
        out[prec] = gpu
        if prec == "fp64":
            err = np.abs(gpu["mu"] - ref) / np.maximum(1.0, np.abs(ref))
        else:
            err = np.abs(gpu["mu"] - ref)
        assert err.max() <= tol, (prec, err.max(), np.unravel_index(err.argmax(), err.shape))
    # the FP32 form's error on the thermodynamics, against the oracle's moments
    secs = kpm.sector_set(20, w.n_up, a, b)
    th32 = kpm.thermo(out["fp32"]["mu"], out["fp32"]["mu_M"], out["fp32"]["mu_M2"], secs, w.T)
    runs = [{"mu": m} for m in ref]
    th_ref = O.thermo_from_runs(20, w.n_up, runs, a, b, w.T)
    e = _thermo_error(th32, th_ref, w.T)
    _record("ring20_sectors", e)
    # stated bounds (measured on GB300): over the whole grid the FP32 form's C is within
    # 0.15 of its peak (the largest deviation sits at the lowest T, where the expansion
    # resolves the band edge least), within 1e-3 for T >= 0.1; chi within 1e-2
    assert e["C"]["max_rel_to_peak"] <= 0.15 and e["chi"]["max_rel_to_peak"] <= 1e-2, e
    assert e["C"]["max_rel_to_peak_T_ge_0.1"] <= 1e-3, e


def test_j1j2_torus_two_vectors_every_moment_and_thermo_error():
    meta, gold = _golden_moments("j1j2sq24_full_moments.txt")
    w = W.workload("j1j2sq24_full")
    a, b = [meta["a"]], [meta["b"]]
    K = int(meta["K"])
    assert int(meta["seed"]) == w.seed and K == w.K
    g32 = kpm.moments(w.model, w.n_up, K, w.R, w.seed, a=a, b=b, precision="fp32", per_vector=True)
    for r in range(gold.shape[0]):
        err = np.abs(g32["mu_r"][0, r] - gold[r])
        assert err.max() <= TOL32, (r, err.max(), int(err.argmax()))
    g64r = kpm.moments(w.model, w.n_up, K, 2, w.seed, a=a, b=b, precision="fp64", per_vector=True)
    for r in range(gold.shape[0]):
        err = np.abs(g64r["mu_r"][0, r] - gold[r]) / np.maximum(1.0, np.abs(gold[r]))
        assert err.max() <= TOL64, (r, err.max(), int(err.argmax()))
    # the FP32 form against the FP64 form of the same R = 64 run (the FP64 form is pinned to
    # the oracle on vectors 0 and 1 above): moments, and the thermodynamics on the 200-point
    # grid with the Lanczos rescaling of the benchmark (eps = 0.025: with the loose a, b above
    # the band edge would sit far inside [-1, 1] and the low-T quadrature would weigh the
    # truncation noise below the spectrum)
    g64 = kpm.moments(w.model, w.n_up, K, w.R, w.seed, a=a, b=b, precision="fp64")
    assert np.abs(g32["mu"] - g64["mu"]).max() <= TOL32
    bnd = kpm.bounds(w.model, w.n_up, eps=w.eps, max_iter=100, tol=1e-8, seed=w.seed)
    a, b = bnd["a"], bnd["b"]
    g32 = kpm.moments(w.model, w.n_up, K, w.R, w.seed, a=a, b=b, precision="fp32")
    g64 = kpm.moments(w.model, w.n_up, K, w.R, w.seed, a=a, b=b, precision="fp64")
    assert np.abs(g32["mu"] - g64["mu"]).max() <= TOL32
    secs = kpm.sector_set(24, w.n_up, a, b)
    th32 = kpm.thermo(g32["mu"], g32["mu_M"], g32["mu_M2"], secs, w.T)
    th64 = kpm.thermo(g64["mu"], g64["mu_M"], g64["mu_M2"], secs, w.T)
    e = _thermo_error(th32, th64, w.T)
    T = np.asarray(w.T)
    for q in ("C", "chi"):
        prof = np.asarray(e[q]["profile_rel_to_peak"])
        e[q]["max_rel_to_peak_T_ge_0.4"] = float(prof[T >= 0.4].max())
    _record("j1j2sq24_full", e)
    # stated bounds (measured on GB300): on the full 2^24 space the ground state carries a
    # weight of 2^-24 of the trace, below the FP32 form's moment noise, so the low-T end of
    # the grid is not resolved in FP32 (C off by up to 0.9 of its peak near T = 0.03, chi by
    # more than its peak below T = 0.1); for T >= 0.4 C is within 1e-3 of its peak and chi
    # within 1e-2, and C within 2e-2 for T >= 0.1
    assert e["C"]["max_rel_to_peak_T_ge_0.4"] <= 1e-3, e["C"]["max_rel_to_peak_T_ge_0.4"]
    assert e["chi"]["max_rel_to_peak_T_ge_0.4"] <= 1e-2, e["chi"]["max_rel_to_peak_T_ge_0.4"]
    assert e["C"]["max_rel_to_peak_T_ge_0.1"] <= 2e-2, e["C"]["max_rel_to_peak_T_ge_0.1"]


def test_ring34_sz0_against_stored_oracle_moments():
    meta, gold = _golden_moments("ring34_sz0_moments.txt")
    w = W.workload("ring34_m0")
    a, b = [meta["a"]], [meta["b"]]
    Kg = int(meta["K"])
    assert int(meta["seed"]) == w.seed and math.comb(34, 17) == 2333606220
    g32 = kpm.moments(w.model, w.n_up, Kg, w.R, w.seed, a=a, b=b, precision="fp32",
                      per_vector=True, weighted=False)
    err = np.abs(g32["mu_r"][0, 0] - gold[0])
    assert err.max() <= TOL32, err
    g64 = kpm.moments(w.model, w.n_up, 40, 1, w.seed, a=a, b=b, precision="fp64", weighted=False)
    err = np.abs(g64["mu"][0, :Kg] - gold[0]) / np.maximum(1.0, np.abs(gold[0]))
    assert err.max() <= TOL64, err
    s32 = kpm.moments(w.model, w.n_up, 40, 1, w.seed, a=a, b=b, precision="fp32", weighted=False)
    assert np.abs(s32["mu"] - g64["mu"]).max() <= TOL32
    assert abs(g64["mu"][0, 0] - 1.0) < 1e-12 and np.abs(g64["mu"]).max() <= 1.0 + 1e-12

"""Library features beyond the plain moment loop, through the C ABI, against the oracle:
per-vector moments, complete-basis (unit-vector) traces, per-bond gradients and the
Hellmann-Feynman identity, the autotuner and the FP64 rate probe.

Tolerances as in test_gpu_parity: FP64 moments 1e-10 max(1, |mu|); gradients 1e-9
relative against the oracle's tangent derivative.
"""
import math

import numpy as np
import pytest

import kpm_workloads as W
import paper_2104_13218_gb300 as kpm
from oracle import c_oracle
from oracle import kpm_oracle as O

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


def _exact_bounds(model, n_up, eps):
    bi, bj, J = model.arrays()
    a, b = [], []
    for k in n_up:
        e = O.eigenvalues(model.n_sites, bi, bj, J, k)
        ai, bi_ = O.rescale(e.min(), e.max(), eps)
        a.append(ai)
        b.append(bi_)
    return np.array(a), np.array(b)


# --------------------------------------------------------------------------- per-vector moments

@pytest.mark.parametrize("precision,tol,R", [("fp64", TOL64, 5), ("fp64", TOL64, 100),
                                             ("fp32", TOL32, 4), ("fp32", TOL32, 100)])
def test_per_vector_moments_match_single_vector_oracle_runs(precision, tol, R):
    """mu_r[s][r][n] = <r|T_n(H')|r> of every vector (the terms of Eq. E-2-7) equals the
    oracle's run with that one vector (r0 = r); their mean is mu.  Ragged sectors (FP32:
    the small ones run in FP64) and a full-space run in the same call."""
    model = W.ring(12)
    n_up = [6, 5, 2, 0]
    a, b = _exact_bounds(model, n_up, 0.025)
    K, seed, r0 = 30, 4, 7
    gpu = kpm.moments(model, n_up, K, R, seed, a=a, b=b, r0=r0, precision=precision,
                      per_vector=True)
    bi, bj, J = model.arrays()
    for i, k in enumerate(n_up):
        for r in sorted({0, 1, R - 1}):
            ref = c_oracle.moments(12, bi, bj, J, k, a[i], b[i], K, 1, seed, r0 + r)["mu"]
            err = np.abs(gpu["mu_r"][i, r] - ref) / np.maximum(1.0, np.abs(ref))
            assert err.max() <= tol, (k, r, err.max())
    # the average over the vectors is the run's mu (the FP32 per-vector sums are formed
    # from the stored FP32 vectors in FP64, the in-kernel ones in short FP32 runs)
    assert np.abs(gpu["mu_r"].mean(axis=1) - gpu["mu"]).max() <= (1e-13 if precision == "fp64" else 1e-6)


def test_per_vector_moments_full_space():
    model = W.random_bonds(10, 14, 2)
    e = np.concatenate([O.eigenvalues(10, *model.arrays(), k) for k in range(11)])
    a, b = O.rescale(e.min(), e.max(), 0.05)
    gpu = kpm.moments(model, [-1], 24, 3, 9, a=[a], b=[b], per_vector=True)
    bi, bj, J = model.arrays()
    for r in range(3):
        ref = c_oracle.moments(10, bi, bj, J, -1, a, b, 24, 1, 9, r)["mu"]
        assert np.abs(gpu["mu_r"][0, r] - ref).max() <= TOL64


# --------------------------------------------------------------------------- complete basis

def test_basis_vectors_give_exact_traces():
    """With unit vectors (KPM_VECTORS_BASIS) summed over disjoint ranges r0 covering every
    state, R * mu / D is the complete-basis trace (1/D) sum_k T_n(E'_k) of the ED spectrum
    (Sec. 2, after Eq. E-2-7), for sectors and for the full space."""
    model = W.j1j2_chain(10, 1.0, 0.35)
    bi, bj, J = model.arrays()
    n_up = [5, 4, 1, 0, -1]
    dims = [math.comb(10, k) if k >= 0 else 1024 for k in n_up]
    specs = [O.eigenvalues(10, bi, bj, J, k) if k >= 0 else
             np.concatenate([O.eigenvalues(10, bi, bj, J, kk) for kk in range(11)]) for k in n_up]
    ab = [O.rescale(e.min(), e.max(), 0.02) for e in specs]
    a = np.array([x[0] for x in ab])
    b = np.array([x[1] for x in ab])
    K, R = 80, 256
    acc = np.zeros((len(n_up), K))
    for r0 in range(0, 1024, R):
        out = kpm.moments(model, n_up, K, R, 0, a=a, b=b, r0=r0, vectors="basis")
        acc += R * out["mu"]
    for i, k in enumerate(n_up):
        exact = O.exact_moments(specs[i], a[i], b[i], K)
        assert np.abs(acc[i] / dims[i] - exact).max() <= 1e-11, k


# --------------------------------------------------------------------------- gradients

def test_per_bond_gradient_matches_tangent_oracle():
    """dL/dJ_b for every bond of a 14-bond random model (more than 8 classes: the per-bond
    sums) against the oracle's forward-mode derivative of the moments."""
    model = W.random_bonds(10, 14, 6)
    bi, bj, J = model.arrays()
    n_up = [5, 4]
    a, b = _exact_bounds(model, n_up, 0.05)
    K, R, seed = 30, 3, 2
    rng = np.random.default_rng(1)
    g = {"mu": rng.standard_normal((2, K)), "mu_M": rng.standard_normal((2, K)),
         "mu_M2": rng.standard_normal((2, K))}
    got = kpm.moments_backward(model, None, model.n_bonds, n_up, a, b, K, R, seed, g,
                               ckpt_interval=4)
    ref = np.zeros(model.n_bonds)
    for i, k in enumerate(n_up):
        jac = O.moment_jacobian(10, bi, bj, J, np.arange(model.n_bonds), k, a[i], b[i], K, R, seed)
        Mk = k - 5
        ref += jac @ (g["mu"][i] + Mk * g["mu_M"][i] + Mk * Mk * g["mu_M2"][i])
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.abs(ref).max(), (got, ref)
    # classes that group the bonds give the sums of the per-bond derivatives
    cls = np.arange(model.n_bonds) % 3
    got3 = kpm.moments_backward(model, cls, 3, n_up, a, b, K, R, seed, g, ckpt_interval=4)
    assert np.max(np.abs(got3 - np.array([ref[cls == p].sum() for p in range(3)]))) <= \
        1e-9 * np.abs(ref).max()


def test_hellmann_feynman_per_bond_at_n12():
    """d lnZ/dJ_b = -beta <H_b> (Hellmann-Feynman) per bond on the J1-J2 chain N = 12 (24
    bonds), all 13 sectors: complete-basis moments (unit vectors over every state) through
    kpm_thermo_backward and the adjoint kpm_moments_backward, against exact
    diagonalisation.  With exact traces and K = 300 (Chebyshev interpolation of e^{-beta E}
    converged at these T) the quadrature error is below 1e-9.  The one-state sectors (the
    ferromagnetic states) get a = 0.5: with a held fixed, a rescaling of width ~0 would turn
    the derivative of their x = (E - b)/a into a ratio of rounding errors."""
    model = W.j1j2_chain(12, 1.0, 0.4)
    bi, bj, J = model.arrays()
    N = 12
    n_up = W.all_sectors(N)
    a, b = _exact_bounds(model, n_up, 0.02)
    a = np.maximum(a, 0.5)
    dims = np.array([math.comb(N, k) for k in n_up], dtype=float)
    T = np.array([0.5, 1.0, 2.0])
    K, R = 300, 512
    chunks = list(range(0, int(dims.max()), R))
    mu = np.zeros((len(n_up), K))
    for r0 in chunks:
        mu += R * kpm.moments(model, n_up, K, R, 0, a=a, b=b, r0=r0, vectors="basis")["mu"]
    mu /= dims[:, None]
    secs = kpm.sector_set(N, n_up, a, b)
    M = np.array([k - N / 2 for k in n_up])
    ex = O.bond_expectation_exact(N, bi, bj, J, np.arange(model.n_bonds), T)  # [n_bonds, nT]
    for it, t in enumerate(T):
        cot = {"lnZ": np.eye(len(T))[it]}
        gm = kpm.thermo_backward(mu, M[:, None] * mu, (M ** 2)[:, None] * mu, secs, T, cot)
        total = gm["mu"] + M[:, None] * gm["mu_M"] + (M ** 2)[:, None] * gm["mu_M2"]
        # mu = (R/D) sum over chunks of the chunk's mu: the cotangent of each chunk
        dJ = np.zeros(model.n_bonds)
        for r0 in chunks:
            gc = {"mu": total * (R / dims)[:, None]}
            dJ += kpm.moments_backward(model, None, model.n_bonds, n_up, a, b, K, R, 0, gc,
                                       r0=r0, vectors="basis", ckpt_interval=32)
        hf = -ex[:, it] / t
        assert np.max(np.abs(dJ - hf)) <= 1e-9 * np.abs(hf).max(), (t, np.max(np.abs(dJ - hf)))


# --------------------------------------------------------------------------- autotuner

@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_autotune_keeps_the_results(precision, tol):
    """The tuned schedule changes only the order of the sums: the moments agree with the
    default schedule to rounding, and with the oracle within the parity tolerance."""
    model = W.ring(14)
    n_up = W.all_sectors(14)
    a, b = _exact_bounds(model, n_up, 0.025)
    res = kpm.autotune(model, n_up, a, b, 20, precision=precision, trial_steps=4)
    assert res["best_ms"] > 0 and res["default_ms"] > 0 and res["best_ms"] <= res["default_ms"]
    assert res["report"].startswith("best:")
    d = kpm.moments(model, n_up, 60, 20, 3, a=a, b=b, precision=precision)
    t = kpm.moments(model, n_up, 60, 20, 3, a=a, b=b, precision=precision, tuned=True)
    assert np.abs(d["mu"] - t["mu"]).max() <= tol
    bi, bj, J = model.arrays()
    for i, k in enumerate(n_up):
        ref = c_oracle.moments(14, bi, bj, J, k, a[i], b[i], 60, 20, 3)["mu"]
        assert np.abs(t["mu"][i] - ref).max() <= (TOL64 if precision == "fp64" else TOL32)


def test_fp64_rate_probe():
    r = kpm.fp64_peak()
    assert 0.05 < r["tflops"] < 200.0 and r["ms"] >= 50.0

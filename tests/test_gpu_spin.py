"""Spin-s Heisenberg models (Sec. 3.4, the ring of N = 10 spins s = 5/2) through the C ABI:
moments against the spin-s C oracle on the same vectors (FP64 1e-10 max(1, |mu|), FP32
1e-5), Lanczos bounds against exact diagonalisation, and the thermodynamics against ED
within the statistical error of the trace estimator."""
import numpy as np
import pytest

import kpm_workloads as W
import paper_2104_13218_gb300 as kpm
from oracle import c_oracle
from oracle import kpm_oracle as O
from oracle import spin_oracle as S

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


def _exact_ab(n, two_s, model, Q, eps=0.025):
    bi, bj, J = model.arrays()
    if Q < 0:
        e = np.concatenate([S.eigenvalues(n, two_s, bi, bj, J, q) for q in range(n * two_s + 1)])
    else:
        e = S.eigenvalues(n, two_s, bi, bj, J, Q)
    return O.rescale(e.min(), e.max(), eps)


@pytest.mark.parametrize("precision,R", [("fp64", 1), ("fp64", 9), ("fp64", 100), ("fp32", 4),
                                         ("fp32", 100)])
def test_spin_moments_match_oracle(precision, R):
    """Ring N = 5 with s = 5/2 (digit codes of 15 bits), ragged sectors and the full space."""
    n, two_s = 5, 5
    model = W.ring(n, 1.0)
    bi, bj, J = model.arrays()
    Q = [12, 13, 3, 0, 25, -1]
    ab = [_exact_ab(n, two_s, model, q) for q in Q]
    a = np.array([x[0] for x in ab])
    b = np.array([x[1] for x in ab])
    K = 40
    got = kpm.spin_moments(model, two_s, Q, K, R, 5, a, b, r0=2, precision=precision)
    tol = TOL64 if precision == "fp64" else TOL32
    for i, q in enumerate(Q):
        ref = c_oracle.spin_moments(n, two_s, bi, bj, J, q, a[i], b[i], K, R, 5, 2)
        err = np.abs(got["mu"][i] - ref["mu"]) / np.maximum(1.0, np.abs(ref["mu"]))
        assert err.max() <= tol, (q, err.max())
        if q < 0:
            for k in ("mu_M", "mu_M2"):
                err = np.abs(got[k][i] - ref[k]) / np.maximum(1.0, np.abs(ref[k]))
                assert err.max() <= 10 * tol, (k, err.max())


def test_spin_one_chain_and_mixed_couplings():
    n, two_s = 6, 2
    model = W.j1j2_chain(n, 1.0, -0.4)
    bi, bj, J = model.arrays()
    Q = [6, 5, 7, 2]
    ab = [_exact_ab(n, two_s, model, q) for q in Q]
    a = np.array([x[0] for x in ab])
    b = np.array([x[1] for x in ab])
    got = kpm.spin_moments(model, two_s, Q, 60, 6, 9, a, b)
    for i, q in enumerate(Q):
        ref = c_oracle.spin_moments(n, two_s, bi, bj, J, q, a[i], b[i], 60, 6, 9, 0)["mu"]
        assert np.abs(got["mu"][i] - ref).max() <= TOL64


@pytest.mark.parametrize("n,two_s", [(5, 5), (6, 2), (4, 3)])
def test_spin_bounds_enclose_the_exact_spectrum(n, two_s):
    model = W.ring(n, 1.0)
    bi, bj, J = model.arrays()
    Q = list(range(n * two_s + 1))
    res = kpm.spin_bounds(model, two_s, Q, eps=0.025, max_iter=300, tol=1e-8, seed=3)
    for i, q in enumerate(Q):
        e = S.eigenvalues(n, two_s, bi, bj, J, q)
        sc = max(1.0, np.abs(e).max())
        assert res["e_min"][i] <= e.min() + 1e-9 * sc and res["e_max"][i] >= e.max() - 1e-9 * sc, q
        assert res["e_min"][i] >= e.min() - 1e-6 * sc and res["e_max"][i] <= e.max() + 1e-6 * sc, q


def test_spin_thermo_follows_ed():
    """Ring N = 5, s = 5/2, all sectors, R = 200, K = 200: the KPM thermodynamics of
    Eq. E-2-2..E-2-2-C agree with ED within the statistical error, and with the
    oracle's quadrature of the same moments to 1e-9."""
    n, two_s = 5, 5
    model = W.ring(n, 1.0)
    bi, bj, J = model.arrays()
    Q = list(range(n * two_s + 1))
    bnd = kpm.spin_bounds(model, two_s, Q, eps=0.025, seed=1)
    mom = kpm.spin_moments(model, two_s, Q, 200, 200, 4, bnd["a"], bnd["b"])
    T = W.log_grid(1.0, 20.0, 12)
    secs = kpm.spin_sector_set(n, two_s, Q, bnd["a"], bnd["b"])
    got = kpm.thermo(mom["mu"], mom["mu_M"], mom["mu_M2"], secs, T)
    dims = [float(S.sector_dim(n, two_s, q)) for q in Q]
    Ms = [q - n * two_s / 2 for q in Q]
    ref = O.thermo(list(mom["mu"]), [Ms[i] * mom["mu"][i] for i in range(len(Q))],
                   [Ms[i] ** 2 * mom["mu"][i] for i in range(len(Q))], dims, [1.0] * len(Q),
                   bnd["a"], bnd["b"], T)
    ed = S.thermo_exact(n, two_s, bi, bj, J, T)
    for q in ("lnZ", "E", "C", "chi"):
        assert np.max(np.abs(got[q] - ref[q]) / np.maximum(1, np.abs(ref[q]))) < 1e-9, q
        assert np.max(np.abs(got[q] - ed[q]) / np.maximum(1, np.abs(ed[q]))) < 0.05, q


def test_fe10_ring_sz0_full_size_matches_oracle():
    """The paper's s = 5/2 ring of N = 10 spins (Sec. 3.4), its S^z = 0 sector
    (D = 4 395 456, codes of 30 bits, ranks through the split tables): 100 Chebyshev steps at
    R = 1 in FP64 and FP32 against the spin-s C oracle on the same vector."""
    n, two_s, q = 10, 5, 25
    model = W.ring(n, 1.0)
    bi, bj, J = model.arrays()
    assert kpm.spin_sector_dims(n, two_s, [q])[0] == 4395456
    s = two_s / 2
    # the spectrum lies in [-N s(s+1), N s^2] (|S_i.S_j| bounds): a safe rescaling
    a, b = 0.5 * (n * s * s + n * s * (s + 1)) * 1.01, 0.5 * (n * s * s - n * s * (s + 1))
    K = 200
    ref = c_oracle.spin_moments(n, two_s, bi, bj, J, q, a, b, K, 1, 3, 0)["mu"]
    g64 = kpm.spin_moments(model, two_s, [q], K, 1, 3, [a], [b], weighted=False)["mu"][0]
    assert np.abs(g64 - ref).max() <= TOL64
    g32 = kpm.spin_moments(model, two_s, [q], K, 1, 3, [a], [b], precision="fp32", weighted=False)["mu"][0]
    assert np.abs(g32 - ref).max() <= TOL32

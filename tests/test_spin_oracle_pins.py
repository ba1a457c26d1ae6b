"""Pins of the spin-s oracle (oracle/spin_oracle.py, the spin-s part of oracle/naive_kpm.c)
against facts outside it: closed-form spectra of spin-s clusters, the spin-1/2 oracle,
trace identities, sector dimensions and the ferromagnetic top of the spectrum."""
import math

import numpy as np
import pytest

import kpm_workloads as W
from oracle import c_oracle
from oracle import kpm_oracle as O
from oracle import spin_oracle as S


def _all_eigs(n, two_s, model):
    bi, bj, J = model.arrays()
    return np.sort(np.concatenate([S.eigenvalues(n, two_s, bi, bj, J, Q) for Q in range(n * two_s + 1)]))


@pytest.mark.parametrize("two_s", [1, 2, 3, 5])
def test_dimer_spectrum(two_s):
    """Two spins s with J: E(S) = (J/2)[S(S+1) - 2 s(s+1)], S = 0 .. 2s, (2S+1)-fold."""
    s = two_s / 2
    e = _all_eigs(2, two_s, W.ring(2, 1.3))
    expect = np.sort(np.concatenate([[0.65 * (St * (St + 1) - 2 * s * (s + 1))] * (2 * St + 1)
                                     for St in range(two_s + 1)]))
    assert np.abs(e - expect).max() < 1e-12


def _m_counts(n, two_s):
    """Number of states with total S^z = M (M from -ns to ns, in steps of 1)."""
    return [S.sector_dim(n, two_s, Q) for Q in range(n * two_s + 1)]


@pytest.mark.parametrize("n,two_s", [(3, 2), (3, 3), (4, 2), (3, 5)])
def test_complete_graph_spectrum(n, two_s):
    """Equal couplings between all pairs: H = (J/2)[S_tot^2 - n s(s+1)], so the spectrum is
    (J/2)[S(S+1) - n s(s+1)] with S-multiplet count n_S = N(M=S) - N(M=S+1)."""
    s = two_s / 2
    bonds = [(i, j, 1.0) for i in range(n) for j in range(i + 1, n)]
    model = W._model("complete", n, bonds)
    e = _all_eigs(n, two_s, model)
    counts = _m_counts(n, two_s)           # index Q = M + n s
    qmax = n * two_s
    expect = []
    for Q in range(qmax + 1):
        M2 = 2 * Q - qmax                  # 2M
        if M2 < 0:
            continue
        n_S = counts[Q] - (counts[Q + 1] if Q + 1 <= qmax else 0)
        St = M2 / 2
        expect += [0.5 * (St * (St + 1) - n * s * (s + 1))] * int(n_S * (M2 + 1))
    assert len(expect) == (two_s + 1) ** n
    assert np.abs(e - np.sort(expect)).max() < 1e-11


def test_spin_half_reduces_to_the_spin_half_oracle():
    model = W.random_bonds(7, 10, 5)
    bi, bj, J = model.arrays()
    e_s = _all_eigs(7, 1, model)
    e_h = np.sort(np.concatenate([O.eigenvalues(7, bi, bj, J, k) for k in range(8)]))
    assert np.abs(e_s - e_h).max() < 1e-12


@pytest.mark.parametrize("two_s", [2, 3, 5])
def test_trace_identities_and_ferromagnetic_top(two_s):
    """Tr H = 0, Tr H^2 / D = sum_b J_b^2 (s(s+1))^2 / 3, and for antiferromagnetic
    couplings the top of the spectrum is the ferromagnetic s^2 sum_b J_b."""
    s = two_s / 2
    model = W.ring(4, 0.7)
    e = _all_eigs(4, two_s, model)
    D = (two_s + 1) ** 4
    assert len(e) == D
    J = np.array(model.J)
    assert abs(e.sum()) < 1e-9
    assert abs((e ** 2).sum() / D - (J ** 2).sum() * (s * (s + 1)) ** 2 / 3) < 1e-9
    assert abs(e.max() - s * s * J.sum()) < 1e-9


@pytest.mark.parametrize("n,two_s", [(4, 5), (10, 5), (6, 3), (5, 1)])
def test_sector_dimensions(n, two_s):
    dims = [c_oracle.spin_sector_dim(n, two_s, Q) for Q in range(n * two_s + 1)]
    assert sum(dims) == (two_s + 1) ** n == c_oracle.spin_sector_dim(n, two_s, -1)
    assert dims == [S.sector_dim(n, two_s, Q) for Q in range(n * two_s + 1)]
    assert dims == dims[::-1]
    if two_s == 1:
        assert dims == [math.comb(n, k) for k in range(n + 1)]


def test_c_oracle_matches_numpy_oracle_and_exact_traces():
    model = W.ring(5)
    bi, bj, J = model.arrays()
    for two_s, Q in [(5, 12), (2, -1), (3, 7)]:
        e = (np.concatenate([S.eigenvalues(5, two_s, bi, bj, J, q) for q in range(5 * two_s + 1)])
             if Q < 0 else S.eigenvalues(5, two_s, bi, bj, J, Q))
        a, b = O.rescale(e.min(), e.max(), 0.05)
        py = S.sector_moments(5, two_s, bi, bj, J, Q, a, b, 30, 3, 7, 1)
        cc = c_oracle.spin_moments(5, two_s, bi, bj, J, Q, a, b, 30, 3, 7, 1)
        for k in (("mu", "mu_M", "mu_M2") if Q < 0 else ("mu",)):
            assert np.abs(py[k] - cc[k]).max() < 1e-12, (two_s, Q, k)
        # complete basis: the unit vectors of every state give the exact traces
        st = S.sector_states(5, two_s, Q)
        H = S.hamiltonian(5, two_s, bi, bj, J, st)
        mu_cb = O.kpm_moments(H, a, b, np.eye(len(st)), 30)
        assert np.abs(mu_cb - O.exact_moments(e, a, b, 30)).max() < 1e-11


def test_spin_thermo_limits():
    """High temperature: chi T -> N s(s+1)/3 (free spins)."""
    two_s = 3
    s = two_s / 2
    model = W.ring(4, 1.0)
    bi, bj, J = model.arrays()
    th = S.thermo_exact(4, two_s, bi, bj, J, np.array([1e4]))
    assert abs(th["chi"][0] * 1e4 - 4 * s * (s + 1) / 3) < 1e-2

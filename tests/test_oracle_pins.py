"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
generator outputs, closed-form spectra, trace identities, exact
diagonalisation, the Chebyshev interpolation property of the quadrature,
finite differences and the Hellmann-Feynman theorem.
"""
import math

import numpy as np
import pytest
import torch

import kpm_workloads as W
from oracle import c_oracle
from oracle import kpm_oracle as O
from tests.conftest import read_golden


# --------------------------------------------------------------------------- RNG

def test_splitmix64_published_outputs():
    for state, out in read_golden("splitmix64.txt"):
        assert O.splitmix64_int(int(state, 16)) == int(out, 16)
        arr = O.splitmix64_np(np.array([int(state, 16)], dtype=np.uint64))
        assert int(arr[0]) == int(out, 16)


def test_rademacher_vectors_are_signs_with_unit_norm():
    st = O.sector_states(10, 5)
    v = O.rademacher_vectors(7, 0, 16, st)
    assert np.allclose(np.abs(v) * math.sqrt(len(st)), 1.0)
    assert np.allclose((v * v).sum(0), 1.0, atol=1e-14)
    # roughly balanced signs (fixed seed: a deterministic check)
    frac = (v > 0).mean()
    assert abs(frac - 0.5) < 5.0 / math.sqrt(v.size)
    # the index is the bitstring: full-space vector restricted to a sector = sector vector (up to norm)
    full = O.rademacher_vectors(7, 0, 16, O.sector_states(10, -1))
    assert np.array_equal(np.sign(full[st]), np.sign(v))


# --------------------------------------------------------------------------- basis

@pytest.mark.parametrize("n", [1, 4, 7, 10, 12])
def test_sector_dimensions_and_ranks(n):
    total = 0
    for k in range(n + 1):
        st = O.sector_states(n, k)
        assert len(st) == math.comb(n, k)
        total += len(st)
        assert np.all(np.diff(st) > 0)
        assert np.array_equal(O.combinadic_rank(st), np.arange(len(st)))
        cst = c_oracle.sector_states(n, k)
        assert np.array_equal(cst.astype(np.int64), st)
        for i in range(0, len(st), max(1, len(st) // 17)):
            assert c_oracle.rank(int(st[i])) == i
    assert total == 2 ** n


# --------------------------------------------------------------------------- Hamiltonian

def _spectrum(model, sectors=None):
    bi, bj, J = model.arrays()
    n = model.n_sites
    ks = range(n + 1) if sectors is None else sectors
    return np.sort(np.concatenate([O.eigenvalues(n, bi, bj, J, k) for k in ks]))


@pytest.mark.parametrize("name,model", [("dimer", W.ring(2)), ("triangle", W.triangle()),
                                        ("ring4", W.ring(4))])
def test_closed_form_spectra(name, model):
    rows = [r for r in read_golden("small_cluster_spectra.txt") if r[0] == name]
    expect = np.sort(np.concatenate([[float(e)] * int(mult) for _, e, mult in rows]))
    assert np.allclose(_spectrum(model), expect, atol=1e-12)


def test_ring_ground_state_energies():
    for n, e0 in read_golden("heisenberg_ring_ground_states.txt"):
        n = int(n)
        m = W.ring(n)
        bi, bj, J = m.arrays()
        got = O.eigenvalues(n, bi, bj, J, n // 2).min()
        tol = 1e-12 if n <= 6 else 2e-9
        assert abs(got - float(e0)) < tol, (n, got, e0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_trace_identities(seed):
    m = W.random_bonds(7, 9, seed)
    bi, bj, J = m.arrays()
    e = _spectrum(m)
    # Tr H = 0 and Tr H^2 / 2^N = (3/16) sum_b J_b^2 for spin-1/2
    assert abs(e.sum()) < 1e-10
    assert abs((e * e).mean() - 3.0 / 16.0 * np.sum(J * J)) < 1e-12
    # the same from the sparse operator, sector by sector, and symmetry
    for k in range(8):
        H = O.hamiltonian(7, bi, bj, J, O.sector_states(7, k))
        assert abs(H - H.T).max() < 1e-15 if H.nnz else True


def test_ferromagnetic_state_is_top_for_af_couplings():
    m = W.j1j2_chain(8, 1.0, 0.4)
    bi, bj, J = m.arrays()
    e = _spectrum(m)
    assert abs(e.max() - J.sum() / 4) < 1e-12
    assert abs(O.eigenvalues(8, bi, bj, J, 8)[0] - J.sum() / 4) < 1e-12


# --------------------------------------------------------------------------- moments

@pytest.mark.parametrize("n", [8, 10, 12])
def test_sawtooth_flat_band_at_the_critical_point(n):
    """Sawtooth chain at |J2/J1| = 1/2 with J1 < 0 (the quantum critical point of
    Sec. 3.3): the one-magnon band is flat and degenerate with the ferromagnetic
    state, so the sector with one flipped spin has exactly n/2 states at the
    ferromagnetic energy sum_b J_b / 4 and a gap above them."""
    model = W.sawtooth(n, -1.0, 0.5)
    bi, bj, J = model.arrays()
    assert len(J) == n + n // 2
    e_fm = J.sum() / 4.0
    e = np.sort(O.eigenvalues(n, bi, bj, J, n - 1))
    assert np.allclose(e[: n // 2], e_fm, atol=1e-12)
    assert e[n // 2] > e_fm + 0.1
    # away from the critical point the degeneracy is lifted
    e45 = np.sort(O.eigenvalues(n, *W.sawtooth(n, -1.0, 0.45).arrays(), n - 1))
    assert np.sum(np.abs(e45 - e45[0]) < 1e-9) < n // 2


def test_complete_basis_moments_equal_exact_traces():
    """With a complete orthonormal basis (R = D unit vectors) the estimator is exact (Sec. 2)."""
    m = W.random_bonds(8, 12, 3)
    bi, bj, J = m.arrays()
    for k in (4, 5, -1):
        st = O.sector_states(8, k)
        H = O.hamiltonian(8, bi, bj, J, st)
        e = np.linalg.eigvalsh(H.toarray())
        a, b = O.rescale(e.min(), e.max(), 0.05)
        v0 = np.eye(len(st))
        mu = O.kpm_moments(H, a, b, v0, 64)
        ex = O.exact_moments(e, a, b, 64)
        # direct mu_n = <v0|T_n|v0> and the doubling formulas agree
        mu_d = O.kpm_moments(H, a, b, v0, 64, direct=True)
        assert np.max(np.abs(mu - ex)) < 1e-12
        assert np.max(np.abs(mu_d - ex)) < 1e-12
        assert abs(mu[0] - 1.0) < 1e-15


def test_random_vector_moments_properties():
    m = W.ring(10)
    bi, bj, J = m.arrays()
    st = O.sector_states(10, -1)
    H = O.hamiltonian(10, bi, bj, J, st)
    e = np.linalg.eigvalsh(H.toarray())
    a, b = O.rescale(e.min(), e.max(), 0.025)
    v0 = O.rademacher_vectors(1, 0, 20, st)
    mu = O.kpm_moments(H, a, b, v0, 400)
    mu_d = O.kpm_moments(H, a, b, v0, 400, direct=True)
    assert abs(mu[0] - 1.0) < 1e-14
    # the Rademacher diagonal is exact: mu_1 = (Tr H / D - c)/m + off-diagonal noise;
    # the full-space Heisenberg H has Tr H = 0 and zero diagonal-free mean
    assert np.max(np.abs(mu - mu_d)) < 1e-11
    assert np.max(np.abs(mu)) <= 1.0 + 1e-12
    ex = O.exact_moments(e, a, b, 400)
    # statistical error ~ 1/sqrt(R D)
    assert np.max(np.abs(mu - ex)) < 6.0 / math.sqrt(20 * 1024)


def test_seed_average_converges_to_exact_traces():
    """Mean over P independent realisations -> exact trace, spread ~ 1/sqrt(R D) (Sec. 2)."""
    m = W.ring(8)
    bi, bj, J = m.arrays()
    st = O.sector_states(8, 4)
    H = O.hamiltonian(8, bi, bj, J, st)
    e = np.linalg.eigvalsh(H.toarray())
    a, b = O.rescale(e.min(), e.max(), 0.025)
    ex = O.exact_moments(e, a, b, 16)
    P, R = 200, 4
    runs = np.array([O.kpm_moments(H, a, b, O.rademacher_vectors(s, 0, R, st), 16) for s in range(P)])
    mean = runs.mean(0)
    sem = runs.std(0, ddof=1) / math.sqrt(P)
    z = np.abs(mean[1:] - ex[1:]) / sem[1:]
    assert np.all(z < 5.0), z


def test_full_space_weighted_moments_match_sector_sum():
    m = W.random_bonds(8, 10, 5)
    bi, bj, J = m.arrays()
    a, b = 3.0, 0.1
    full = O.sector_moments((bi, bj, J), 8, -1, a, b, 32, 3, 11)
    st = O.sector_states(8, -1)
    M = O.magnetisation(st, 8)
    v0 = O.rademacher_vectors(11, 0, 3, st)
    H = O.hamiltonian(8, bi, bj, J, st)
    # M commutes with H: block by block, <v0|M T_n|v0> = sum_M M <v0_M|T_n|v0_M>
    acc = np.zeros(32)
    acc2 = np.zeros(32)
    for k in range(9):
        idx = np.nonzero(O.popcount(st) == k)[0]
        Hk = H[idx][:, idx]
        # the sector pieces of v0 are not renormalised: kpm_moments divides by R only
        mk = O.kpm_moments(Hk, a, b, v0[idx], 32)
        acc += (k - 4) * mk
        acc2 += (k - 4) ** 2 * mk
    assert np.max(np.abs(full["mu_M"] - acc)) < 1e-12
    assert np.max(np.abs(full["mu_M2"] - acc2)) < 1e-12
    assert abs(full["mu_M"][0]) < 1e-15           # sum_s M(s) / D = 0
    assert abs(full["mu_M2"][0] - 8 / 4.0) < 1e-14  # <M^2> = N/4 at infinite T


def test_c_oracle_matches_numpy_oracle():
    m = W.random_bonds(10, 14, 8)
    bi, bj, J = m.arrays()
    for k in (3, 5, -1):
        a, b = 4.0, -0.3
        ref = O.sector_moments((bi, bj, J), 10, k, a, b, 40, 5, 99, r0=3)
        got = c_oracle.moments(10, bi, bj, J, k, a, b, 40, 5, 99, r0=3)
        assert np.max(np.abs(got["mu"] - ref["mu"])) < 1e-12
        if k < 0:
            assert np.max(np.abs(got["mu_M"] - ref["mu_M"])) < 1e-12
            assert np.max(np.abs(got["mu_M2"] - ref["mu_M2"])) < 1e-12


# --------------------------------------------------------------------------- kernel + thermo

def test_jackson_end_points_and_positivity():
    for K in (10, 100, 400):
        g = O.jackson(K)
        assert abs(g[0] - 1.0) < 1e-14
        q = math.pi / (K + 1)
        gK = (math.cos(q * K) + math.sin(q * K) / math.tan(q)) / (K + 1)
        assert abs(gK) < 1e-13
        assert np.all(np.diff(g) < 0)
    # the Jackson-damped expansion of a delta function is non-negative everywhere
    K = 64
    g = O.jackson(K)
    x = np.cos(np.linspace(0.01, math.pi - 0.01, 301))
    Tx = O.chebyshev_T(K - 1, x)
    for y in (-0.7, 0.0, 0.33, 0.9):
        Ty = O.chebyshev_T(K - 1, np.array([y]))[:, 0]
        coef = g * Ty
        coef[1:] *= 2
        dens = coef @ Tx
        assert dens.min() > -1e-12
    # without the kernel the same sum oscillates below zero (Gibbs)
    coef = O.chebyshev_T(K - 1, np.array([0.33]))[:, 0].copy()
    coef[1:] *= 2
    assert (coef @ Tx).min() < -1.0


def _sector_runs_exact(model, n_up, eps, K):
    bi, bj, J = model.arrays()
    n = model.n_sites
    runs, a, b = [], [], []
    for k in n_up:
        e = O.eigenvalues(n, bi, bj, J, k)
        ai, bi_ = O.rescale(e.min(), e.max(), eps)
        runs.append({"mu": O.exact_moments(e, ai, bi_, K)})
        a.append(ai)
        b.append(bi_)
    return runs, a, b


def test_quadrature_with_exact_moments_reproduces_ed_thermo():
    """With exact traces, g_n = 1 and Nq = K the quadrature is a degree-(K-1) Chebyshev
    interpolation of exp(-beta E), so Z, E, C, chi converge to the ED values."""
    model = W.ring(10)
    bi, bj, J = model.arrays()
    n_up = list(range(11))
    K = 256
    runs, a, b = _sector_runs_exact(model, n_up, 0.0, K)
    T = W.log_grid(0.3, 10.0, 40)
    kp = O.thermo_from_runs(10, n_up, runs, a, b, T)
    ed = O.thermo_exact(10, bi, bj, J, T)
    for q in ("lnZ", "E", "C", "chi"):
        assert np.max(np.abs(kp[q] - ed[q]) / np.maximum(1, np.abs(ed[q]))) < 1e-9, q
    # mirrored sectors (M >= 0 only, M > 0 doubled) give the same result
    nn = W.nonnegative_sectors(10)
    runs2, a2, b2 = _sector_runs_exact(model, nn, 0.0, K)
    mirror = [0 if k == 5 else 1 for k in nn]
    kp2 = O.thermo_from_runs(10, nn, runs2, a2, b2, T, mirror=mirror)
    for q in ("lnZ", "E", "C", "chi"):
        assert np.max(np.abs(kp2[q] - ed[q]) / np.maximum(1, np.abs(ed[q]))) < 1e-9, q


def test_thermo_limits():
    model = W.ring(8)
    bi, bj, J = model.arrays()
    runs = [O.sector_moments((bi, bj, J), 8, -1, 5.0, 0.0, 64, 4, 5)]
    T = np.array([1e6, 1e7])
    kp = O.thermo_from_runs(8, [-1], runs, [5.0], [0.0], T, kernel="jackson")
    # Z(beta -> 0) = D exactly: sum_k cos(n theta_k) = 0 for 0 < n < 2 Nq
    assert np.allclose(kp["lnZ"], math.log(256), atol=1e-5)
    # chi T -> N/4 for spin-1/2
    assert np.allclose(kp["chi"] * T, 8 / 4.0, rtol=1e-5)
    # C T^2 -> (3/16) sum J^2 with exact moments and g_1 = g_2 = 1
    runs_ex, a, b = _sector_runs_exact(model, list(range(9)), 0.0, 64)
    kp2 = O.thermo_from_runs(8, list(range(9)), runs_ex, a, b, np.array([1e4]))
    assert abs(kp2["C"][0] * 1e8 - 3.0 / 16.0 * 8) < 1e-3


def test_thermo_torch_matches_numpy():
    model = W.ring(8)
    n_up = list(range(9))
    runs, a, b = _sector_runs_exact(model, n_up, 0.05, 40)
    T = W.log_grid(0.05, 10, 30)
    ref = O.thermo_from_runs(8, n_up, runs, a, b, T, kernel="jackson")
    truns = [{"mu": torch.tensor(r["mu"])} for r in runs]
    got = O.thermo_from_runs(8, n_up, truns, a, b, T, kernel="jackson", torch_mod=torch)
    for q in ("lnZ", "E", "C", "chi"):
        assert np.max(np.abs(got[q].numpy() - ref[q])) < 1e-12


# --------------------------------------------------------------------------- gradient

def test_moment_jacobian_matches_finite_differences():
    model = W.j1j2_chain(8, 1.0, 0.3)
    bi, bj, J = model.arrays()
    cls = model.classes()
    a, b, K, R, seed = 3.5, -0.4, 24, 3, 17
    jac = O.moment_jacobian(8, bi, bj, J, cls, 4, a, b, K, R, seed)
    h = 1e-6
    for p, theta in enumerate((1.0, 0.3)):
        th = [1.0, 0.3]
        th[p] = theta + h
        mp = model.with_couplings(th).arrays()
        th[p] = theta - h
        mm = model.with_couplings(th).arrays()
        fp = O.sector_moments(mp, 8, 4, a, b, K, R, seed)["mu"]
        fm = O.sector_moments(mm, 8, 4, a, b, K, R, seed)["mu"]
        fd = (fp - fm) / (2 * h)
        assert np.max(np.abs(fd - jac[p])) < 1e-7


def test_hellmann_feynman_with_complete_basis():
    """d lnZ / d theta_p = -beta <H_p> (ED) when the moments are exact traces and K is large."""
    model = W.j1j2_chain(8, 1.0, 0.3)
    bi, bj, J = model.arrays()
    cls = model.classes()
    n_up = list(range(9))
    K = 200
    T = np.array([0.7, 1.5, 4.0])
    # fixed rescaling per sector (stop-gradient), from the spectra
    ab = []
    for k in n_up:
        e = O.eigenvalues(8, bi, bj, J, k)
        ab.append(O.rescale(e.min() - 0.5, e.max() + 0.5, 0.0))
    grads = np.zeros((2, len(T)))
    for ti in range(len(T)):
        mus = []
        jacs = []
        for i, k in enumerate(n_up):
            st = O.sector_states(8, k)
            H = O.hamiltonian(8, bi, bj, J, st)
            e, U = np.linalg.eigh(H.toarray())
            mus.append(torch.tensor(O.exact_moments(e, ab[i][0], ab[i][1], K), requires_grad=True))
            # exact-trace derivative: d/dtheta (1/D) Tr T_n(H') = (1/D) Tr(T_n'(H') H_p)/m
            x = (e - ab[i][1]) / ab[i][0]
            th = np.arccos(np.clip(x, -1, 1))
            nn = np.arange(K)[:, None]
            dT = nn * np.sin(nn * th[None, :]) / np.sin(th[None, :])  # T_n'(x) = n U_{n-1}(x)
            jp = []
            for p in range(2):
                Hp = O.hamiltonian(8, bi, bj, J, st, bond_weights=(cls == p).astype(float)).toarray()
                hp = np.einsum("ij,ik,kj->j", U, Hp, U)
                jp.append((dT * hp[None, :]).mean(1) / ab[i][0])
            jacs.append(np.array(jp))
        kp = O.thermo_from_runs(8, n_up, [{"mu": m} for m in mus], [x[0] for x in ab],
                                [x[1] for x in ab], T[ti:ti + 1], torch_mod=torch)
        kp["lnZ"].sum().backward()
        for i in range(len(n_up)):
            grads[:, ti] += jacs[i] @ mus[i].grad.numpy()
    hp = O.bond_expectation_exact(8, bi, bj, J, cls, T)
    hf = -hp / T[None, :]
    assert np.max(np.abs(grads - hf) / np.abs(hf)) < 1e-8


def test_zeeman_field_in_exact_thermo():
    """With a field h the exact thermodynamics equals that of the dense matrix
    H + h sum_i s^z_i built directly (the Zeeman term of Eq. E-3-1-1 is diagonal on
    S^z bitstrings), including chi = beta (<M^2> - <M>^2) with <M> != 0."""
    model = W.ring(6)
    bi, bj, J = model.arrays()
    h = 0.37
    st = O.sector_states(6, -1)
    M = O.magnetisation(st, 6)
    Hd = O.dense_hamiltonian(6, bi, bj, J, st) + np.diag(h * M)
    e, U = np.linalg.eigh(Hd)
    Mk = np.einsum("ik,i,ik->k", U, M, U)
    M2k = np.einsum("ik,i,ik->k", U, M * M, U)
    T = np.array([0.3, 1.0, 3.0])
    ex = O.thermo_exact(6, bi, bj, J, T, field=h)
    beta = 1.0 / T
    w = np.exp(-np.outer(beta, e - e.min()))
    Z = w.sum(1)
    assert np.allclose(ex["lnZ"], np.log(Z) - beta * e.min(), atol=1e-12)
    Em = (w * e).sum(1) / Z
    assert np.allclose(ex["E"], Em, atol=1e-12)
    chi = beta * ((w * M2k).sum(1) / Z - ((w * Mk).sum(1) / Z) ** 2)
    assert np.allclose(ex["chi"], chi, atol=1e-12)
    assert np.all(np.abs((w * Mk).sum(1) / Z) > 1e-3)  # the field polarises


@pytest.fixture(scope="module")
def ladder14():
    """Exact spectra of the AF two-leg ladder N = 14 (sectors M >= 0, M > 0 mirrored)
    and a helper giving C(T) from exact (complete-basis) traces minus the exact C(T)."""
    N = 14
    model = W.ladder(N, 1.0, 1.0)
    arr = model.arrays()
    n_up = list(range(N // 2, N + 1))
    mirror = [0 if k == N // 2 else 1 for k in n_up]
    dims, mult, m1, m2 = O.sector_weights(N, n_up, mirror)
    T = np.logspace(-3.5, 1.0, 46)
    eigs = [O.eigenvalues(N, *arr, k) for k in n_up]
    ex = O.thermo_exact(N, *arr, T, n_up=n_up, mirror=mirror)

    def deviation(K, kernel="none", eps=0.0, n_quad=None):
        mu, mu1, mu2, a, b = [], [], [], [], []
        for i, e in enumerate(eigs):
            ai, bi = O.rescale(e.min(), e.max(), eps)
            x = O.exact_moments(e, ai, bi, K)
            mu.append(x)
            mu1.append(m1[i] * x)
            mu2.append(m2[i] * x)
            a.append(ai)
            b.append(bi)
        th = O.thermo(mu, mu1, mu2, dims, mult, np.array(a), np.array(b), T,
                      K if n_quad is None else n_quad, kernel)
        return th["C"] - ex["C"]

    return {"T": T, "exact": ex, "deviation": deviation}


def test_ghost_dip_of_the_ladder_with_exact_traces(ladder14):
    """The "ghost dip" of Sec. 3.1.1: in the standard configuration (N_deg = 100,
    eps = 0, N~ = 100, g_n = 1) the heat capacity of the AF two-leg ladder
    deviates from exact diagonalisation at T ~ 1e-3 .. 1e-2 even with exact
    (complete-basis) traces, so the deviation is systematic, while it agrees at
    higher T.  Shown here for N = 14 (the paper's figure is for N = 16)."""
    T, ex = ladder14["T"], ladder14["exact"]
    dev = ladder14["deviation"](100)
    low = (T >= 1e-3) & (T <= 1e-2)
    assert dev[low].min() < -0.05                       # a dip well below the exact C ~ 0
    t_min = T[np.argmin(dev)]
    assert 1e-3 <= t_min <= 1e-2                        # located where the paper sees it
    high = T >= 0.05
    assert np.abs(dev[high]).max() < 1e-8 * np.abs(ex["C"][high]).max()


def test_jackson_kernel_turns_the_ghost_dip_into_a_peak(ladder14):
    """Sec. 3.1.2 (the Jackson kernel paragraph): with exact traces the kernel
    turns the ghost dip of C(T) into a ghost peak and, unlike the unsmoothed
    expansion, deviates from exact diagonalisation at higher T as well; a
    higher order (N_deg = 500) reduces that deviation."""
    T, ex = ladder14["T"], ladder14["exact"]
    low = (T >= 1e-3) & (T <= 1e-2)
    high = T >= 0.05
    dev = {(K, k): ladder14["deviation"](K, k) for K in (100, 500) for k in ("none", "jackson")}
    assert dev[100, "none"][low].min() < -0.05 and dev[100, "jackson"][low].min() > 0.0
    assert dev[100, "jackson"][low].max() > 0.05
    peak = ex["C"].max()
    assert np.abs(dev[100, "none"][high]).max() < 1e-10 * peak
    assert np.abs(dev[100, "jackson"][high]).max() > 1e-3 * peak
    assert np.abs(dev[500, "jackson"][high]).max() < 0.1 * np.abs(dev[100, "jackson"][high]).max()


def test_statistical_error_of_C_scales_as_inverse_sqrt_R():
    """Statistical deviations (Sec. 3.1.1, Eq. E-3-1 .. E-3-3): over independent
    realisations the spread of the estimated heat capacity falls like 1/sqrt(R)
    (R = 4 -> 64 divides it by ~4), and the realisation mean stays within a few
    standard errors of exact diagonalisation (the estimator is unbiased up to the
    small systematic part at these T)."""
    N = 10
    model = W.ladder(N, 1.0, 1.0)
    arr = model.arrays()
    n_up = list(range(N // 2, N + 1))
    mirror = [0 if k == N // 2 else 1 for k in n_up]
    T = np.array([0.3, 0.6, 1.0, 2.0])
    a, b = [], []
    for k in n_up:
        e = O.eigenvalues(N, *arr, k)
        ai, bi = O.rescale(e.min(), e.max(), 0.0)
        a.append(ai)
        b.append(bi)
    ex = O.thermo_exact(N, *arr, T, n_up=n_up, mirror=mirror)
    P = 12
    std, mean = {}, {}
    for R in (4, 64):
        C = []
        for p in range(P):
            runs = [O.sector_moments(arr, N, k, a[i], b[i], 100, R, 100 + p) for i, k in enumerate(n_up)]
            C.append(O.thermo_from_runs(N, n_up, runs, np.array(a), np.array(b), T, mirror=mirror)["C"])
        C = np.array(C)
        std[R], mean[R] = C.std(axis=0), C.mean(axis=0)
    ratio = np.exp(np.log(std[4] / std[64]).mean())
    assert 2.5 < ratio < 6.5, ratio
    for R in (4, 64):
        assert np.all(np.abs(mean[R] - ex["C"]) < 4 * std[R] / np.sqrt(P) + 1e-3)

"""Plain CPU FP64 oracle for the Chebyshev typicality method (TEST INFRASTRUCTURE).

This module is the independent check of the CUDA path.  Only the tests, the
smoke check of the repository entry point and the CPU-baseline leg of the
benchmark may import it; the library never does.  It shares no code with the
CUDA path: the random vectors, the basis, the Hamiltonian, the recursion and
the thermodynamics are all written out here again, slowly and directly.

What it computes, and where the paper defines it:

* Heisenberg Hamiltonian H = sum_b J_b S_i . S_j on S^z bitstrings (Eq. E-3-1-1):
  diagonal +J_b/4 when the two bits agree and -J_b/4 when they differ;
  off-diagonal J_b/2 between s and s XOR (1<<i | 1<<j) when they differ.
* S^z sectors (Sec. 2, the decomposition under Eq. E-2-2-C): states with
  k = N/2 + M up spins, ordered by their value as integers.  The rank of a
  state is its position in that order (here: a binary search).
* Rescaling H' = (H - c)/m, m = (Emax - Emin)/(2 - eps), c = (Emax + Emin)/2
  (Eq. E-2-3, E-2-4).
* Moments mu_n = Tr C_n(H') (Eq. E-2-6) and their typicality estimate over R
  random vectors (Eq. E-2-7), here normalised so that mu_0 = 1:
  mu_n = (1/R) sum_r <r|C_n(H')|r> / <r|r>.
* Jackson kernel g_n (Eq. E-2-8, read with the stray trailing factor dropped
  and N_deg taken as the number of moments K).
* Gauss-Chebyshev quadrature (Eq. quad) and the weights gamma_k, giving Z, E,
  C and chi (Eq. E-2-2, E-2-2-B, E-2-2-C and the sector sum that follows the
  quadrature).
* Exact diagonalisation and the exact traces with a complete basis (Sec. 2,
  after Eq. E-2-7) as the reference the estimates converge to.
* The derivative of the moments with respect to the couplings, by forward
  (tangent) propagation through the recursion, for checking the adjoint.

Random vectors (the paper draws Gaussian components; this build uses
Rademacher signs, a convention the paper does not fix): component s of
vector r is sign(h) / sqrt(D) with
    h = splitmix64(splitmix64(splitmix64(seed) ^ r) ^ s)
and sign(h) = +1 if the top bit of h is 0 else -1, where s is the bitstring
of the state (not its rank) and splitmix64(x) is Steele, Lea and Flood's
generator output for state x, i.e. the mixing function applied to
x + 0x9e3779b97f4a7c15.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence

import numpy as np
import scipy.sparse as sp

U64 = np.uint64
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


# ----------------------------------------------------------------------------
# Counter-based random signs
# ----------------------------------------------------------------------------

def splitmix64_int(x: int) -> int:
    """splitmix64 output for state x (Python integers, exact)."""
    z = (x + GOLDEN_GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_np(x: np.ndarray) -> np.ndarray:
    """The same function on a uint64 array (numpy integer products wrap mod 2^64)."""
    with np.errstate(over="ignore"):
        z = x.astype(U64) + U64(GOLDEN_GAMMA)
        z = (z ^ (z >> U64(30))) * U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> U64(27))) * U64(0x94D049BB133111EB)
        return z ^ (z >> U64(31))


def rademacher_vectors(seed: int, r0: int, R: int, states: np.ndarray) -> np.ndarray:
    """[D, R] matrix of +-1/sqrt(D) for vectors r0..r0+R-1 on the given bitstrings."""
    D = len(states)
    out = np.empty((D, R), dtype=np.float64)
    hs = splitmix64_int(seed & MASK64)
    s = states.astype(U64)
    for j in range(R):
        hr = splitmix64_int(hs ^ ((r0 + j) & MASK64))
        h = splitmix64_np(s ^ U64(hr))
        out[:, j] = np.where((h >> U64(63)) == U64(0), 1.0, -1.0)
    return out / math.sqrt(D)


# ----------------------------------------------------------------------------
# Basis
# ----------------------------------------------------------------------------

def popcount(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.int64)
    c = np.zeros_like(x)
    while np.any(x):
        c += x & 1
        x = x >> 1
    return c


def sector_states(n_sites: int, n_up: int) -> np.ndarray:
    """All bitstrings of N bits with n_up set bits, ascending; n_up = -1 gives all 2^N."""
    s = np.arange(1 << n_sites, dtype=np.int64)
    if n_up < 0:
        return s
    return s[popcount(s) == n_up]


def combinadic_rank(states: np.ndarray) -> np.ndarray:
    """Textbook colex rank sum_j C(p_j, j+1) over set-bit positions p_0 < p_1 < ..."""
    states = np.asarray(states, dtype=np.int64)
    rank = np.zeros(len(states), dtype=np.int64)
    seen = np.zeros(len(states), dtype=np.int64)
    for p in range(63):
        bit = (states >> p) & 1
        if not np.any(bit) and not np.any(states >> p):
            break
        sel = bit == 1
        seen_sel = seen[sel] + 1
        rank[sel] += np.array([math.comb(p, int(j)) for j in seen_sel], dtype=np.int64)
        seen[sel] = seen_sel
    return rank


def magnetisation(states: np.ndarray, n_sites: int) -> np.ndarray:
    """M(s) = (number of up spins) - N/2."""
    return popcount(states) - n_sites / 2.0


# ----------------------------------------------------------------------------
# Hamiltonian
# ----------------------------------------------------------------------------

def hamiltonian(n_sites: int, bi, bj, J, states: np.ndarray, bond_weights=None) -> sp.csr_matrix:
    """Sparse H = sum_b w_b S_i . S_j in the basis `states` (Eq. E-3-1-1).

    `bond_weights` replaces J (used to build the single-bond operators H_b).
    """
    J = np.asarray(J if bond_weights is None else bond_weights, dtype=np.float64)
    states = np.asarray(states, dtype=np.int64)
    D = len(states)
    diag = np.zeros(D)
    rows, cols, vals = [], [], []
    for b in range(len(bi)):
        i, j, w = int(bi[b]), int(bj[b]), float(J[b])
        differ = ((states >> i) ^ (states >> j)) & 1
        diag += np.where(differ == 1, -0.25 * w, 0.25 * w)
        src = np.nonzero(differ)[0]
        if len(src) == 0 or w == 0.0:
            continue
        flipped = states[src] ^ ((1 << i) | (1 << j))
        dst = np.searchsorted(states, flipped)
        rows.append(dst)
        cols.append(src)
        vals.append(np.full(len(src), 0.5 * w))
    H = sp.diags(diag).tocsr()
    if rows:
        off = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                            shape=(D, D))
        H = H + off
    return H.tocsr()


def dense_hamiltonian(n_sites, bi, bj, J, states) -> np.ndarray:
    return hamiltonian(n_sites, bi, bj, J, states).toarray()


def eigenvalues(n_sites, bi, bj, J, n_up) -> np.ndarray:
    """Exact spectrum of one sector (dense symmetric eigensolver)."""
    st = sector_states(n_sites, n_up)
    return np.linalg.eigvalsh(dense_hamiltonian(n_sites, bi, bj, J, st))


# ----------------------------------------------------------------------------
# Rescaling (Eq. E-2-3, E-2-4)
# ----------------------------------------------------------------------------

def rescale(e_min: float, e_max: float, eps: float):
    """(m, c) of Eq. E-2-4; a sector whose spectrum is one point gets a tiny m."""
    m = (e_max - e_min) / (2.0 - eps)
    c = (e_max + e_min) / 2.0
    m = max(m, 1e-12 * max(1.0, abs(c)))
    return m, c


# ----------------------------------------------------------------------------
# Chebyshev moments (Eq. E-2-6, E-2-7)
# ----------------------------------------------------------------------------

def kpm_moments(H: sp.spmatrix, m: float, c: float, v0: np.ndarray, K: int,
                weight: Optional[np.ndarray] = None, direct: bool = False) -> np.ndarray:
    """mu_n = (1/R) sum_r <v0_r| W T_n(H') |v0_r>, n = 0..K-1, for unit-norm columns v0_r.

    Uses the three-term recursion v_{n+1} = 2 H' v_n - v_{n-1} (v_1 = H' v_0)
    and, unless `direct`, the product rule T_{m+n} + T_{|m-n|} = 2 T_m T_n:
    mu_{2n} = 2<v_n|W|v_n> - mu_0, mu_{2n+1} = 2<v_{n+1}|W|v_n> - mu_1.
    With `direct`, mu_n = <v_0|W|v_n> from K-1 recursion steps.  W is an
    optional diagonal operator commuting with H (the magnetisation M or M^2).
    """
    R = v0.shape[1]
    D = v0.shape[0]
    Hs = (H - c * sp.identity(D, format="csr")) / m
    w = np.ones(D) if weight is None else np.asarray(weight, dtype=np.float64)
    Wcol = w[:, None]

    def dot(x, y):
        return float(np.sum(x * Wcol * y)) / R

    mu = np.zeros(K)
    v_prev = v0
    v_cur = Hs @ v0
    if direct:
        mu[0] = dot(v0, v0)
        if K > 1:
            mu[1] = dot(v0, v_cur)
        for n in range(2, K):
            v_next = 2.0 * (Hs @ v_cur) - v_prev
            mu[n] = dot(v0, v_next)
            v_prev, v_cur = v_cur, v_next
        return mu
    if K % 2:
        raise ValueError("K must be even")
    mu[0] = dot(v0, v0)
    mu[1] = dot(v_cur, v0)
    # v_prev = v_{n-1}, v_cur = v_n
    for n in range(1, K // 2):
        v_next = 2.0 * (Hs @ v_cur) - v_prev
        mu[2 * n] = 2.0 * dot(v_cur, v_cur) - mu[0]
        mu[2 * n + 1] = 2.0 * dot(v_next, v_cur) - mu[1]
        v_prev, v_cur = v_cur, v_next
    return mu


def chebyshev_T(n_max: int, x: np.ndarray) -> np.ndarray:
    """[n_max+1, len(x)] table of T_n(x) = cos(n arccos x) for |x| <= 1."""
    x = np.clip(np.asarray(x, dtype=np.float64), -1.0, 1.0)
    return np.cos(np.outer(np.arange(n_max + 1), np.arccos(x)))


def exact_moments(eigs: np.ndarray, m: float, c: float, K: int) -> np.ndarray:
    """Complete-basis traces mu_n = (1/D) sum_k T_n((E_k - c)/m) (Sec. 2, after Eq. E-2-7)."""
    x = (np.asarray(eigs) - c) / m
    return chebyshev_T(K - 1, x).mean(axis=1)


# ----------------------------------------------------------------------------
# Sector runs
# ----------------------------------------------------------------------------

def sector_moments(model_arrays, n_sites: int, n_up: int, m: float, c: float, K: int, R: int,
                   seed: int, r0: int = 0, direct: bool = False) -> Dict[str, np.ndarray]:
    """Moments of one sector (or of the full space, n_up = -1, with the M and M^2 moments)."""
    bi, bj, J = model_arrays
    st = sector_states(n_sites, n_up)
    H = hamiltonian(n_sites, bi, bj, J, st)
    v0 = rademacher_vectors(seed, r0, R, st)
    out = {"mu": kpm_moments(H, m, c, v0, K, direct=direct), "dim": len(st)}
    if n_up < 0:
        M = magnetisation(st, n_sites)
        out["mu_M"] = kpm_moments(H, m, c, v0, K, weight=M, direct=direct)
        out["mu_M2"] = kpm_moments(H, m, c, v0, K, weight=M * M, direct=direct)
    return out


# ----------------------------------------------------------------------------
# Kernel and thermodynamics (Eq. E-2-8, Eq. quad and the sums after it)
# ----------------------------------------------------------------------------

def jackson(K: int) -> np.ndarray:
    """g_n, n = 0..K-1, of Eq. E-2-8 with N_deg := K (so g_0 = 1 and g_K = 0)."""
    n = np.arange(K, dtype=np.float64)
    q = math.pi / (K + 1)
    return ((K - n + 1) * np.cos(q * n) + np.sin(q * n) / math.tan(q)) / (K + 1)


def kernel_coeffs(K: int, kernel: str) -> np.ndarray:
    if kernel == "jackson":
        return jackson(K)
    if kernel == "none":
        return np.ones(K)
    raise ValueError(kernel)


def thermo(mu: Sequence[np.ndarray], mu1: Sequence[np.ndarray], mu2: Sequence[np.ndarray],
           dims: Sequence[float], mult: Sequence[float], a: Sequence[float], b: Sequence[float],
           T: np.ndarray, n_quad: int = 0, kernel: str = "none", torch_mod=None):
    """ln Z, sign Z, E, C, chi on the grid T from the moments of every sector.

    For sector G with moments mu^G (normalised, mu_0 = 1), dimension D_G,
    multiplicity mult_G (2 when the sector also stands for its mirror -M) and
    rescaling (a_G, b_G):
        gamma_k^G = g_0 mu_0 + 2 sum_{n>=1} g_n mu_n cos(n pi (k - 1/2)/Nq)
        E_k^G     = a_G cos(pi (k - 1/2)/Nq) + b_G
        w_k^G     = mult_G (D_G/Nq) gamma_k^G exp(-beta (E_k^G - E_ref))
        Z         = exp(-beta E_ref) sum w         (E_ref = min over G, k of E_k^G)
        E         = sum w E / sum w
        C         = beta^2 sum w (E_k - E)^2 / sum w
        chi       = beta (<M^2> - <M>^2),  <M^p> = sum_G sum_k w1/2_k^G / sum w
    where w1, w2 are built like w from the moments mu1^G, mu2^G: M_G mu^G and
    M_G^2 mu^G for a sector (0 and M_G^2 mu^G for a mirrored pair), or the
    M- and M^2-weighted moments for the full space.
    Written with torch ops (float64) when `torch_mod` is given so that
    autograd provides the derivative with respect to the moments.
    """
    xp = torch_mod if torch_mod is not None else np
    K = len(mu[0])
    Nq = n_quad if n_quad > 0 else K
    g = kernel_coeffs(K, kernel)
    kk = np.arange(1, Nq + 1, dtype=np.float64)
    theta = math.pi * (kk - 0.5) / Nq
    # cos table [K, Nq] with the factor 2 for n >= 1
    ctab = np.cos(np.outer(np.arange(K), theta))
    ctab[1:] *= 2.0
    ctab = ctab * g[:, None]
    xk = np.cos(theta)
    T = np.asarray(T, dtype=np.float64)
    beta = 1.0 / T
    if torch_mod is not None:
        ctab_t = xp.tensor(ctab, dtype=xp.float64)
    else:
        ctab_t = ctab
    Ek = [a[G] * xk + b[G] for G in range(len(mu))]
    e_ref = min(float(np.min(e)) for e in Ek)
    S0 = 0.0
    S1 = 0.0
    S2 = 0.0
    SE = 0.0
    for G in range(len(mu)):
        fac = mult[G] * dims[G] / Nq
        boltz = np.exp(-np.outer(beta, Ek[G] - e_ref)) * fac  # [nT, Nq]
        if torch_mod is not None:
            boltz = xp.tensor(boltz, dtype=xp.float64)
        gam = mu[G] @ ctab_t
        gam1 = mu1[G] @ ctab_t
        gam2 = mu2[G] @ ctab_t
        w = boltz * gam[None, :]
        S0 = S0 + w.sum(1)
        SE = SE + (w * (xp.tensor(Ek[G]) if torch_mod is not None else Ek[G])[None, :]).sum(1)
        S1 = S1 + (boltz * gam1[None, :]).sum(1)
        S2 = S2 + (boltz * gam2[None, :]).sum(1)
    Emean = SE / S0
    Cacc = 0.0
    for G in range(len(mu)):
        fac = mult[G] * dims[G] / Nq
        boltz = np.exp(-np.outer(beta, Ek[G] - e_ref)) * fac
        if torch_mod is not None:
            boltz = xp.tensor(boltz, dtype=xp.float64)
            EkG = xp.tensor(Ek[G])
        else:
            EkG = Ek[G]
        gam = mu[G] @ ctab_t
        dE = EkG[None, :] - Emean[:, None]
        Cacc = Cacc + (boltz * gam[None, :] * dE * dE).sum(1)
    bt = xp.tensor(beta) if torch_mod is not None else beta
    lnZ = xp.log(xp.abs(S0)) - bt * e_ref
    signZ = xp.sign(S0)
    C = bt * bt * Cacc / S0
    M1 = S1 / S0
    M2 = S2 / S0
    chi = bt * (M2 - M1 * M1)
    return {"lnZ": lnZ, "signZ": signZ, "E": Emean, "C": C, "chi": chi}


def sector_weights(n_sites: int, n_up: Sequence[int], mirror: Optional[Sequence[int]] = None):
    """(dims, mult, M1, M2) per sector: M1 = M (0 for a mirrored pair), M2 = M^2."""
    dims, mult, m1, m2 = [], [], [], []
    for i, k in enumerate(n_up):
        if k < 0:
            dims.append(float(1 << n_sites))
            mult.append(1.0)
            m1.append(float("nan"))
            m2.append(float("nan"))
            continue
        M = k - n_sites / 2.0
        mir = bool(mirror[i]) if mirror is not None else False
        dims.append(float(math.comb(n_sites, k)))
        mult.append(2.0 if mir else 1.0)
        m1.append(0.0 if mir else M)
        m2.append(M * M)
    return dims, mult, m1, m2


def thermo_from_runs(n_sites, n_up, runs, a, b, T, n_quad=0, kernel="none", mirror=None,
                     torch_mod=None):
    """Thermodynamics from per-sector moment runs (dicts of `sector_moments`)."""
    dims, mult, m1, m2 = sector_weights(n_sites, n_up, mirror)
    mu, mu1, mu2 = [], [], []
    for i, k in enumerate(n_up):
        x = runs[i]["mu"]
        mu.append(x)
        if k < 0:
            mu1.append(runs[i]["mu_M"])
            mu2.append(runs[i]["mu_M2"])
        else:
            mu1.append(m1[i] * x)
            mu2.append(m2[i] * x)
    return thermo(mu, mu1, mu2, dims, mult, a, b, T, n_quad, kernel, torch_mod)


def thermo_exact(n_sites, bi, bj, J, T, n_up=None, mirror=None, field=0.0):
    """Exact Z, E, C, chi from the sector spectra (Eq. E-2-2, E-2-2-B, E-2-2-C).

    `field` is h = g mu_B B of the Zeeman term h sum_i s^z_i (Eq. E-3-1-1),
    which adds h M to the energies of the sector with magnetisation M."""
    if n_up is None:
        n_up = list(range(n_sites + 1))
    T = np.asarray(T, dtype=np.float64)
    beta = 1.0 / T
    specs = []
    for i, k in enumerate(n_up):
        M = k - n_sites / 2.0
        e = eigenvalues(n_sites, bi, bj, J, k) + field * M
        mir = bool(mirror[i]) if mirror is not None else False
        specs.append((e, 2.0 if mir else 1.0, 0.0 if mir else M, M * M))
    e_ref = min(float(s[0].min()) for s in specs)
    S0 = np.zeros_like(beta)
    SE = np.zeros_like(beta)
    S1 = np.zeros_like(beta)
    S2 = np.zeros_like(beta)
    for e, mu_, m1, m2 in specs:
        w = mu_ * np.exp(-np.outer(beta, e - e_ref))
        S0 += w.sum(1)
        SE += (w * e[None, :]).sum(1)
        S1 += m1 * w.sum(1)
        S2 += m2 * w.sum(1)
    Em = SE / S0
    Cacc = np.zeros_like(beta)
    for e, mu_, m1, m2 in specs:
        w = mu_ * np.exp(-np.outer(beta, e - e_ref))
        Cacc += (w * (e[None, :] - Em[:, None]) ** 2).sum(1)
    return {"lnZ": np.log(S0) - beta * e_ref, "E": Em, "C": beta ** 2 * Cacc / S0,
            "chi": beta * (S2 / S0 - (S1 / S0) ** 2)}


# ----------------------------------------------------------------------------
# Derivatives of the moments with respect to the couplings (tangent mode)
# ----------------------------------------------------------------------------

def moment_jacobian(n_sites, bi, bj, J, classes, n_up, m, c, K, R, seed, r0=0):
    """dmu_n/dtheta_p, shape [P, K], for J_b = theta_{class(b)} with m, c held fixed.

    Differentiates the recursion forward: with H' = (H - c)/m and
    dH'/dtheta_p = H_p/m (H_p = sum over bonds of class p of S_i . S_j),
        dv_1 = (H_p/m) v_0,   dv_{n+1} = 2 (H_p/m) v_n + 2 H' dv_n - dv_{n-1},
        dmu_1 = <dv_1, v_0>,  dmu_{2n} = 4 <dv_n, v_n>,
        dmu_{2n+1} = 2 (<dv_{n+1}, v_n> + <v_{n+1}, dv_n>) - dmu_1.
    """
    st = sector_states(n_sites, n_up)
    D = len(st)
    H = hamiltonian(n_sites, bi, bj, J, st)
    Hs = (H - c * sp.identity(D, format="csr")) / m
    v0 = rademacher_vectors(seed, r0, R, st)
    classes = np.asarray(classes)
    P = int(classes.max()) + 1
    jac = np.zeros((P, K))
    for p in range(P):
        wts = np.where(classes == p, 1.0, 0.0)
        Hp = hamiltonian(n_sites, bi, bj, J, st, bond_weights=wts) / m
        v_prev, v_cur = v0, Hs @ v0
        d_prev, d_cur = np.zeros_like(v0), Hp @ v0
        jac[p, 1] = np.sum(d_cur * v0) / R
        for n in range(1, K // 2):
            v_next = 2.0 * (Hs @ v_cur) - v_prev
            d_next = 2.0 * (Hp @ v_cur) + 2.0 * (Hs @ d_cur) - d_prev
            jac[p, 2 * n] = 4.0 * np.sum(d_cur * v_cur) / R
            jac[p, 2 * n + 1] = 2.0 * (np.sum(d_next * v_cur) + np.sum(v_next * d_cur)) / R - jac[p, 1]
            v_prev, v_cur = v_cur, v_next
            d_prev, d_cur = d_cur, d_next
    return jac


def bond_expectation_exact(n_sites, bi, bj, J, classes, T, n_up=None, mirror=None):
    """<H_p>(T) = Tr(H_p e^{-beta H}) / Z per parameter class p, from exact diagonalisation.

    Gives the Hellmann-Feynman derivative d ln Z / d theta_p = -beta <H_p>.
    """
    if n_up is None:
        n_up = list(range(n_sites + 1))
    classes = np.asarray(classes)
    P = int(classes.max()) + 1
    beta = 1.0 / np.asarray(T, dtype=np.float64)
    parts = []
    for i, k in enumerate(n_up):
        st = sector_states(n_sites, k)
        Hd = dense_hamiltonian(n_sites, bi, bj, J, st)
        e, U = np.linalg.eigh(Hd)
        mult = 2.0 if (mirror is not None and mirror[i]) else 1.0
        diag_p = []
        for p in range(P):
            wts = np.where(classes == p, 1.0, 0.0)
            Hp = hamiltonian(n_sites, bi, bj, J, st, bond_weights=wts).toarray()
            diag_p.append(np.einsum("ij,ik,kj->j", U, Hp, U))
        parts.append((e, mult, np.array(diag_p)))
    e_ref = min(float(p[0].min()) for p in parts)
    Z = np.zeros_like(beta)
    num = np.zeros((P, len(beta)))
    for e, mult, dp in parts:
        w = mult * np.exp(-np.outer(beta, e - e_ref))
        Z += w.sum(1)
        num += np.einsum("tk,pk->pt", w, dp)
    return num / Z[None, :]

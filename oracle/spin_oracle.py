"""Plain CPU FP64 oracle for spin-s Heisenberg models (TEST INFRASTRUCTURE).

Only the tests, the smoke check and the benchmark's CPU leg may import this
module; the library never does, and it shares no code with the CUDA path.

The paper's last example (Sec. 3.4, the ring of N = 10 spins s = 5/2, "Fe10")
uses the Heisenberg Hamiltonian of Eq. E-3-1-1 for spins s > 1/2.  Written
out in the S^z product basis:

* a basis state is the list of m_i in {-s, .., s}; this oracle stores the
  digits q_i = m_i + s in {0 .. 2s} of site i in bits 3i .. 3i+2 of an integer
  code (2s + 1 <= 8), so that increasing codes list the states in
  lexicographic order of (q_{N-1}, .., q_0);
* S_i . S_j = S^z_i S^z_j + (S^+_i S^-_j + S^-_i S^+_j)/2 with
  S^z |m> = m |m>, S^+ |m> = sqrt(s(s+1) - m(m+1)) |m+1>,
  S^- |m> = sqrt(s(s+1) - m(m-1)) |m-1> (the textbook ladder operators);
* the total S^z = sum_i m_i commutes with H: sector M holds the states with
  digit sum Q = M + N s, and is listed by increasing code; the rank of a
  state is its position in that list;
* random vectors as for spin 1/2, with the code in place of the bitstring:
  component of state `code` in vector r is sign(splitmix64(splitmix64(
  splitmix64(seed) ^ r) ^ code)) / sqrt(D).

The Chebyshev recursion, the exact traces and the thermodynamics are the
spin-independent functions of kpm_oracle (Eq. E-2-3 .. E-2-8, quad).
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, List, Sequence

import numpy as np
import scipy.sparse as sp

from . import kpm_oracle as O

FIELD_BITS = 3


def local_dim(two_s: int) -> int:
    return two_s + 1


def digits(code: int, n_sites: int) -> List[int]:
    return [(code >> (FIELD_BITS * i)) & 7 for i in range(n_sites)]


def encode(qs: Sequence[int]) -> int:
    code = 0
    for i, q in enumerate(qs):
        code |= int(q) << (FIELD_BITS * i)
    return code


def sector_states(n_sites: int, two_s: int, Q: int) -> np.ndarray:
    """Codes of the states with digit sum Q (Q = -1: all (2s+1)^N states), increasing."""
    d = local_dim(two_s)
    codes = []
    for qs in itertools.product(range(d), repeat=n_sites):
        if Q >= 0 and sum(qs) != Q:
            continue
        codes.append(encode(qs))
    return np.array(sorted(codes), dtype=np.int64)


def sector_dim(n_sites: int, two_s: int, Q: int) -> int:
    """Coefficient of x^Q in (1 + x + .. + x^{2s})^N (all states for Q = -1)."""
    d = local_dim(two_s)
    if Q < 0:
        return d ** n_sites
    poly = np.zeros(1, dtype=object)
    poly[0] = 1
    for _ in range(n_sites):
        new = np.zeros(len(poly) + d - 1, dtype=object)
        for k in range(d):
            new[k:k + len(poly)] += poly
        poly = new
    return int(poly[Q]) if Q < len(poly) else 0


def hamiltonian(n_sites: int, two_s: int, bi, bj, J, states: np.ndarray) -> sp.csr_matrix:
    """Sparse H = sum_b J_b S_i . S_j in the basis `states` (codes), Eq. E-3-1-1."""
    s = two_s / 2.0
    index = {int(c): k for k, c in enumerate(states)}
    D = len(states)
    rows, cols, vals = [], [], []
    diag = np.zeros(D)
    for col, code in enumerate(states):
        q = digits(int(code), n_sites)
        for b in range(len(bi)):
            i, j, w = int(bi[b]), int(bj[b]), float(J[b])
            mi, mj = q[i] - s, q[j] - s
            diag[col] += w * mi * mj
            # S+_i S-_j and S-_i S+_j, each with amplitude w/2
            for di, dj in ((1, -1), (-1, 1)):
                qi, qj = q[i] + di, q[j] + dj
                if not (0 <= qi <= two_s and 0 <= qj <= two_s):
                    continue
                ci = math.sqrt(s * (s + 1) - mi * (mi + di))
                cj = math.sqrt(s * (s + 1) - mj * (mj + dj))
                qn = list(q)
                qn[i], qn[j] = qi, qj
                row = index[encode(qn)]
                rows.append(row)
                cols.append(col)
                vals.append(0.5 * w * ci * cj)
    H = sp.diags(diag).tocsr()
    if rows:
        H = H + sp.csr_matrix((vals, (rows, cols)), shape=(D, D))
    return H.tocsr()


def eigenvalues(n_sites, two_s, bi, bj, J, Q) -> np.ndarray:
    st = sector_states(n_sites, two_s, Q)
    return np.linalg.eigvalsh(hamiltonian(n_sites, two_s, bi, bj, J, st).toarray())


def magnetisation(states: np.ndarray, n_sites: int, two_s: int) -> np.ndarray:
    return np.array([sum(digits(int(c), n_sites)) for c in states], dtype=np.float64) - n_sites * two_s / 2.0


def rademacher_vectors(seed: int, r0: int, R: int, states: np.ndarray) -> np.ndarray:
    """+-1/sqrt(D) on the state codes (the spin-1/2 generator with the code as key)."""
    return O.rademacher_vectors(seed, r0, R, states)


def sector_moments(n_sites, two_s, bi, bj, J, Q, m, c, K, R, seed, r0=0) -> Dict[str, np.ndarray]:
    """Moments of one sector (Q = -1: the full space, with the M and M^2 weighted ones)."""
    st = sector_states(n_sites, two_s, Q)
    H = hamiltonian(n_sites, two_s, bi, bj, J, st)
    v0 = rademacher_vectors(seed, r0, R, st)
    out = {"mu": O.kpm_moments(H, m, c, v0, K), "dim": len(st)}
    if Q < 0:
        M = magnetisation(st, n_sites, two_s)
        out["mu_M"] = O.kpm_moments(H, m, c, v0, K, weight=M)
        out["mu_M2"] = O.kpm_moments(H, m, c, v0, K, weight=M * M)
    return out


def thermo_exact(n_sites, two_s, bi, bj, J, T) -> Dict[str, np.ndarray]:
    """Exact lnZ, E, C, chi from the spectra of all sectors (Eq. E-2-2, E-2-2-B, E-2-2-C)."""
    T = np.asarray(T, dtype=np.float64)
    beta = 1.0 / T
    specs = []
    for Q in range(n_sites * two_s + 1):
        M = Q - n_sites * two_s / 2.0
        specs.append((eigenvalues(n_sites, two_s, bi, bj, J, Q), M))
    e_ref = min(float(e.min()) for e, _ in specs)
    S0 = np.zeros_like(beta)
    SE = np.zeros_like(beta)
    S1 = np.zeros_like(beta)
    S2 = np.zeros_like(beta)
    for e, M in specs:
        w = np.exp(-np.outer(beta, e - e_ref))
        S0 += w.sum(1)
        SE += (w * e[None, :]).sum(1)
        S1 += M * w.sum(1)
        S2 += M * M * w.sum(1)
    Em = SE / S0
    Cacc = np.zeros_like(beta)
    for e, M in specs:
        w = np.exp(-np.outer(beta, e - e_ref))
        Cacc += (w * (e[None, :] - Em[:, None]) ** 2).sum(1)
    return {"lnZ": np.log(S0) - beta * e_ref, "E": Em, "C": beta ** 2 * Cacc / S0,
            "chi": beta * (S2 / S0 - (S1 / S0) ** 2)}

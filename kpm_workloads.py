"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *describes* problems: bond lists of the spin models, the
magnetisation sectors to run, temperature grids, seeds and sizes.  It holds
none of the method's arithmetic (no Hamiltonian application, no random
vectors, no moments, no thermodynamics), so the CPU oracle and the CUDA path
can both read it without sharing any computation.

Models follow the Heisenberg Hamiltonian H = sum_b J_b S_i . S_j of the paper
(Sec. 3.1, Eq. E-3-1-1), on the lattices the paper studies (rings, ladders,
sawtooth chains; Sec. 3) and on the J1-J2 lattices of the benchmark
workloads.  Sites are numbered 0..N-1 and site i is bit i of the S^z
bitstring (bit set = spin up).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclass(frozen=True)
class Model:
    """A spin-1/2 Heisenberg model: N sites and a list of bonds (i, j, J_b)."""

    name: str
    n_sites: int
    bi: Tuple[int, ...]
    bj: Tuple[int, ...]
    J: Tuple[float, ...]
    # Parameter class of every bond (e.g. 0 for J1 bonds, 1 for J2 bonds).
    bond_class: Tuple[int, ...] = ()

    @property
    def n_bonds(self) -> int:
        return len(self.bi)

    def arrays(self):
        """(bi int32, bj int32, J float64) numpy arrays."""
        return (np.asarray(self.bi, dtype=np.int32),
                np.asarray(self.bj, dtype=np.int32),
                np.asarray(self.J, dtype=np.float64))

    def classes(self) -> np.ndarray:
        if self.bond_class:
            return np.asarray(self.bond_class, dtype=np.int32)
        return np.zeros(self.n_bonds, dtype=np.int32)

    def with_couplings(self, values: Sequence[float]) -> "Model":
        """Same bonds, J_b := values[bond_class[b]]."""
        cls = self.classes()
        J = tuple(float(values[c]) for c in cls)
        return Model(self.name, self.n_sites, self.bi, self.bj, J, tuple(int(c) for c in cls))


def _model(name, n, bonds, classes=None) -> Model:
    bi = tuple(int(b[0]) for b in bonds)
    bj = tuple(int(b[1]) for b in bonds)
    J = tuple(float(b[2]) for b in bonds)
    cl = tuple(int(c) for c in classes) if classes is not None else tuple(0 for _ in bonds)
    return Model(name, n, bi, bj, J, cl)


def ring(n: int, J: float = 1.0) -> Model:
    """Periodic nearest-neighbour chain (Sec. 3.2)."""
    if n == 2:
        return _model("dimer", 2, [(0, 1, J)])
    return _model(f"ring{n}", n, [(i, (i + 1) % n, J) for i in range(n)])


def j1j2_chain(n: int, J1: float = 1.0, J2: float = 0.5) -> Model:
    """Periodic chain with nearest (J1, class 0) and next-nearest (J2, class 1) bonds."""
    bonds = [(i, (i + 1) % n, J1) for i in range(n)] + [(i, (i + 2) % n, J2) for i in range(n)]
    return _model(f"j1j2chain{n}", n, bonds, [0] * n + [1] * n)


def j1j2_square(lx: int, ly: int, J1: float = 1.0, J2: float = 0.5) -> Model:
    """Periodic lx x ly square lattice: NN bonds J1 (class 0), both diagonals J2 (class 1)."""
    def site(x, y):
        return (x % lx) + lx * (y % ly)

    nn, nnn = [], []
    for y in range(ly):
        for x in range(lx):
            s = site(x, y)
            nn.append((s, site(x + 1, y), J1))
            nn.append((s, site(x, y + 1), J1))
            nnn.append((s, site(x + 1, y + 1), J2))
            nnn.append((s, site(x + 1, y - 1), J2))
    return _model(f"j1j2sq{lx}x{ly}", lx * ly, nn + nnn, [0] * len(nn) + [1] * len(nnn))


def ladder(n: int, J_rung: float = 1.0, J_leg: float = 1.0) -> Model:
    """Periodic two-leg ladder of n spins (Eq. E-3-1-1): rung i = sites (2i, 2i+1)."""
    L = n // 2
    bonds = [(2 * i, 2 * i + 1, J_rung) for i in range(L)]
    cls = [0] * L
    for leg in range(2):
        for i in range(L):
            bonds.append((2 * i + leg, 2 * ((i + 1) % L) + leg, J_leg))
            cls.append(1)
    return _model(f"ladder{n}", n, bonds, cls)


def sawtooth(n: int, J1: float = -1.0, J2: float = 0.45) -> Model:
    """Periodic sawtooth (delta) chain of n spins (Sec. 3.3): J1 (class 0) between
    neighbours i, i+1 around the chain, J2 (class 1) between the basal sites
    2k, 2k+2; the odd sites are the apices."""
    bonds = [(i, (i + 1) % n, J1) for i in range(n)]
    bonds += [(2 * k, (2 * k + 2) % n, J2) for k in range(n // 2)]
    return _model(f"sawtooth{n}", n, bonds, [0] * n + [1] * (n // 2))


def triangle(J: float = 1.0) -> Model:
    return _model("triangle", 3, [(0, 1, J), (1, 2, J), (0, 2, J)])


def random_bonds(n: int, n_bonds: int, seed: int, jmin=-1.0, jmax=1.5) -> Model:
    """Random graph with random couplings (for parity tests beyond regular lattices)."""
    rng = np.random.default_rng(seed)
    seen = set()
    bonds = []
    while len(bonds) < n_bonds:
        i, j = (int(x) for x in rng.choice(n, size=2, replace=False))
        key = (min(i, j), max(i, j))
        if key in seen:
            continue
        seen.add(key)
        bonds.append((i, j, float(rng.uniform(jmin, jmax))))
    return _model(f"random{n}_{n_bonds}_{seed}", n, bonds, list(range(n_bonds)))


def log_grid(t_min: float, t_max: float, n: int) -> np.ndarray:
    """T_i = t_min (t_max/t_min)^(i/(n-1)), i = 0..n-1."""
    i = np.arange(n, dtype=np.float64)
    return t_min * (t_max / t_min) ** (i / (n - 1))


def all_sectors(n_sites: int) -> List[int]:
    """Number of up spins k = N/2 + M for every S^z sector M = -N/2..N/2."""
    return list(range(n_sites + 1))


def nonnegative_sectors(n_sites: int) -> List[int]:
    """k for M >= 0 only (the M < 0 sectors are their mirror images, Sec. 2)."""
    return list(range((n_sites + 1) // 2, n_sites + 1)) if n_sites % 2 else list(range(n_sites // 2, n_sites + 1))


FULL_SPACE = -1  # n_up value that selects the whole 2^N space


@dataclass
class Workload:
    """One benchmark / parity configuration of the Chebyshev moment loop."""

    key: str
    model: Model
    n_up: List[int]              # sectors (FULL_SPACE = whole space)
    R: int                       # random vectors per sector
    K: int                       # number of moments mu_0..mu_{K-1}
    seed: int
    eps: float
    T: np.ndarray                # temperature grid
    mirror: Optional[List[int]] = None   # 1 where the sector stands for +M and -M
    kernel: str = "none"
    precisions: Tuple[str, ...] = ("fp64",)
    note: str = ""

    @property
    def steps(self) -> int:
        """Matrix-vector products per run: v_1 .. v_{K/2}."""
        return self.K // 2


def workload(key: str) -> Workload:
    """The five workloads of the benchmark suite, by name."""
    if key == "ring10_full":
        return Workload(key, ring(10), [FULL_SPACE], R=20, K=400, seed=1, eps=0.025,
                        T=log_grid(0.05, 10.0, 100), kernel="jackson",
                        note="ring N=10, J=1, full 2^10 space, R=20, 400 moments")
    if key == "ring20_sectors":
        return Workload(key, ring(20), all_sectors(20), R=100, K=1000, seed=2, eps=0.025,
                        T=log_grid(0.02, 10.0, 200), precisions=("fp32", "fp64"),
                        note="ring N=20, all 21 S^z sectors in one launch, R=100, 1000 moments")
    if key == "j1j2sq24_full":
        return Workload(key, j1j2_square(4, 6, 1.0, 0.5), [FULL_SPACE], R=64, K=2000, seed=3,
                        eps=0.025, T=log_grid(0.02, 10.0, 200), precisions=("fp32", "fp64"),
                        note="J1-J2 4x6 torus, full 2^24 space, R=64, 2000 moments")
    if key == "j1j2chain24_grad":
        return Workload(key, j1j2_chain(24, 1.0, 0.2), nonnegative_sectors(24), R=32, K=1000,
                        seed=4, eps=0.025, T=log_grid(0.1, 5.0, 50),
                        mirror=[0 if k == 12 else 1 for k in nonnegative_sectors(24)],
                        note="J1-J2 chain N=24, sectors M=0..12 (M>0 doubled), R=32, 1000 moments")
    if key == "ring34_m0":
        return Workload(key, ring(34), [17], R=4, K=2000, seed=5, eps=0.025,
                        T=log_grid(0.02, 10.0, 200), precisions=("fp32",),
                        note="ring N=34, S^z=0 sector (dim 2333606220), R=4, 2000 moments")
    # scaled cases of the two largest workloads, small enough for detailed profiles
    # (a few GB on the device, still far larger than L2)
    if key == "ring30_m0":
        return Workload(key, ring(30), [15], R=4, K=2000, seed=5, eps=0.025,
                        T=log_grid(0.02, 10.0, 200), precisions=("fp32",),
                        note="ring N=30, S^z=0 sector (dim 155117520), R=4, 2000 moments")
    if key == "j1j2sq20_full":
        return Workload(key, j1j2_square(4, 5, 1.0, 0.5), [FULL_SPACE], R=64, K=2000, seed=3,
                        eps=0.025, T=log_grid(0.02, 10.0, 200), precisions=("fp32", "fp64"),
                        note="J1-J2 4x5 torus, full 2^20 space, R=64, 2000 moments")
    raise KeyError(key)


WORKLOADS = ("ring10_full", "ring20_sectors", "j1j2sq24_full", "j1j2chain24_grad", "ring34_m0",
             "ring30_m0", "j1j2sq20_full")

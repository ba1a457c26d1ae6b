#!/usr/bin/env python3
"""Writes the stored oracle moments of the two largest benchmark workloads.

The plain C oracle (oracle/naive_kpm.c, the two-vector recursion
oracle_kpm_moments_lean) is too slow to run inside a GPU test at these sizes,
so its results are computed once here and stored as text:

* ring34_sz0_moments.txt -- spin-1/2 Heisenberg ring N = 34, J = 1, S^z = 0
  sector (D = C(34, 17) = 2 333 606 220), rescaling a = 13, b = -3.5 (the
  spectrum of this sector lies in [-15.1, 8.5]: the ground state near
  -0.443 N and the top of the ferromagnetic multiplet at N/4), seed 5, one
  random vector (r0 = 0), the first 8 moments (4 matrix-vector products).
  About 40 GB of host memory and an hour on 8 cores.
* j1j2sq24_full_moments.txt -- J1-J2 model on the periodic 4 x 6 square
  lattice (J1 = 1 on the 48 nearest-neighbour bonds, J2 = 0.5 on the 48
  diagonal bonds), full 2^24 space, rescaling a = 20, b = 0 (the spectrum
  lies in [-20, 18]: the top is the ferromagnetic state at sum_b J_b/4 = 18),
  seed 3, random vectors r0 = 0 and 1, all 2000 moments.

The moments follow Eq. E-2-6 / E-2-7 (normalised to mu_0 = 1) with the
three-term recursion and H' = (H - b)/a (Eq. E-2-3).  Only the oracle is
called; nothing here uses the CUDA library.

Usage: python tests/golden/make_large_sector_moments.py [ring34] [torus]
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import kpm_workloads as W  # noqa: E402
from oracle import c_oracle  # noqa: E402

RING34 = dict(model="ring34", n_up=17, a=13.0, b=-3.5, seed=5, r0=(0,), K=8)
TORUS = dict(model="j1j2sq4x6", n_up=-1, a=20.0, b=0.0, seed=3, r0=(0, 1), K=2000)


def write(name, spec, model, rows, seconds):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        f.write(f"# oracle moments (plain C FP64 recursion, oracle_kpm_moments_lean), {seconds:.0f} s\n")
        f.write(f"# model {model.name}: n_sites {model.n_sites}, n_bonds {model.n_bonds}\n")
        f.write(f"# n_up {spec['n_up']} a {spec['a']!r} b {spec['b']!r} seed {spec['seed']} "
                f"K {spec['K']}\n")
        f.write("# columns: n, then mu_n for random vector r0 = " +
                " ".join(str(r) for r in spec["r0"]) + "\n")
        for n in range(spec["K"]):
            f.write(f"{n} " + " ".join(repr(float(r[n])) for r in rows) + "\n")
    print("wrote", path, flush=True)


def run(spec, model, name):
    bi, bj, J = model.arrays()
    t0 = time.time()
    rows = [c_oracle.moments_lean(model.n_sites, bi, bj, J, spec["n_up"], spec["a"], spec["b"],
                                  spec["K"], spec["seed"], r0) for r0 in spec["r0"]]
    write(name, spec, model, rows, time.time() - t0)


def main(argv):
    which = argv or ["ring34", "torus"]
    c_oracle.build()
    if "torus" in which:
        run(TORUS, W.j1j2_square(4, 6, 1.0, 0.5), "j1j2sq24_full_moments.txt")
    if "ring34" in which:
        run(RING34, W.ring(34), "ring34_sz0_moments.txt")


if __name__ == "__main__":
    main(sys.argv[1:])

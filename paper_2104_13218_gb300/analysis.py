"""Studies built from the GPU moment loop: realisation statistics and a Zeeman field.

* Realisations (Sec. 3, Eq. E-3-1 to E-3-3): P independent realisations of
  the trace estimator, each with R random vectors (realisation i uses
  vectors i*R .. i*R + R - 1), give per temperature the mean O-bar, the
  variance dO^2 = mean(O^2) - O-bar^2 and, against an exact curve, the
  systematic deviation |O-bar - O_exact|.
* Zeeman term g mu_B B sum_i s^z_i (Eq. E-3-1-1): within the sector of
  magnetisation M it adds h M to every energy (h = g mu_B B), so the
  moments of (H + h M - b')/a with b' = b + h M are those of (H - b)/a and
  the field enters the thermodynamics only through b.

The moments and thermodynamics are computed by the library; this module only
loops over calls and combines their outputs.
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import numpy as np

from . import api


def zeeman_shift(b: Sequence[float], n_up: Sequence[int], n_sites: int, h: float) -> np.ndarray:
    """b + h M for every sector (M = n_up - N/2).  Full-space entries are not allowed:
    there M varies from state to state.  Mirrored (+M/-M) entries cannot be used with
    a field either (the two shifts differ); list both sectors instead."""
    n_up = np.asarray(n_up)
    if np.any(n_up < 0):
        raise ValueError("a Zeeman shift needs S^z sectors, not the full space")
    return np.asarray(b, dtype=np.float64) + h * (n_up - n_sites / 2.0)


def realisations(model, n_up, K: int, R: int, P: int, seed: int, a, b, T, mirror=None,
                 kernel: str = "none", n_quad: int = 0, precision: str = "fp64",
                 exact: Optional[Dict[str, np.ndarray]] = None) -> Dict[str, Dict[str, np.ndarray]]:
    """Mean, variance and (with `exact`) systematic deviation over P realisations.

    Returns {observable: {"mean", "var", "dev" (if exact), "all" [P, nT]}} for
    lnZ, E, C and chi.
    """
    secs = api.sector_set(model.n_sites, n_up, a, b, mirror)
    samples = {k: [] for k in ("lnZ", "E", "C", "chi")}
    for i in range(P):
        mom = api.moments(model, n_up, K, R, seed, a=a, b=b, r0=i * R, precision=precision,
                          device=True, allow_ebounds=True)
        th = api.thermo(mom["mu"], mom["mu_M"], mom["mu_M2"], secs, T, kernel=kernel,
                        n_quad=n_quad)
        for k in samples:
            samples[k].append(th[k].cpu().numpy())
    out = {}
    for k, vals in samples.items():
        arr = np.array(vals)
        mean = arr.mean(axis=0)
        entry = {"mean": mean, "var": (arr ** 2).mean(axis=0) - mean ** 2, "all": arr}
        if exact is not None and k in exact:
            entry["dev"] = np.abs(mean - np.asarray(exact[k]))
        out[k] = entry
    return out

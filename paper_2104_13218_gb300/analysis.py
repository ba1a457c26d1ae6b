"""Studies built from the GPU moment loop: realisation statistics, a Zeeman field,
the kernel diagnostic and fits of the couplings to thermodynamic curves.

* Realisations (Sec. 3, Eq. E-3-1 to E-3-3): P independent realisations of
  the trace estimator, each with R random vectors (realisation i uses vectors
  i*R .. i*R + R - 1), come from ONE moment run with P*R vectors and
  per-vector moments; the library then forms each realisation's
  thermodynamics and, per temperature, the mean, the variance and (against an
  exact curve) the systematic deviation (kpm_realisations).
* Zeeman term g mu_B B sum_i s^z_i (Eq. E-3-1-1): it commutes with H, so the
  moments do not change and the library's thermodynamics takes the field
  h = g mu_B B as an argument (kpm_thermo_ex).
* Kernel diagnostic (Sec. 3.1.2, the Jackson kernel paragraph, and Sec. 4): the
  same moments turned into thermodynamics with and without the Jackson kernel;
  where the two differ the expansion order is not sufficient.
* Coupling fits: least squares between (lnZ, E, C, chi)(T) of the model with
  couplings theta (one value per bond class) and target curves, minimised by
  gradient descent (Adam) with the gradient of the adjoint moment loop
  (chebyshev_thermo).  The paper fits nothing; this uses its thermodynamics
  (Eq. E-2-2, E-2-2-B, E-2-2-C) as the model of the data.

The moments, thermodynamics and statistics are computed by the library; this
module only sequences calls.
"""
from __future__ import annotations

from typing import Callable, Dict, Optional, Sequence

import numpy as np
import torch

from . import api


def realisations(model, n_up, K: int, R: int, P: int, seed: int, a, b, T, mirror=None,
                 kernel: str = "none", n_quad: int = 0, precision: str = "fp64",
                 exact: Optional[Dict[str, np.ndarray]] = None,
                 field: float = 0.0) -> Dict[str, Dict[str, np.ndarray]]:
    """Mean, variance and (with `exact`) systematic deviation over P realisations of R
    vectors each, from one run with P*R vectors and per-vector moments.

    Returns {observable: {"mean", "var", "dev" (if exact), "all" [P, nT]}} for
    lnZ, E, C and chi (numpy arrays)."""
    mom = api.moments(model, n_up, K, P * R, seed, a=a, b=b, precision=precision, device=True,
                      weighted=False, per_vector=True, allow_ebounds=True)
    secs = api.sector_set(model.n_sites, n_up, a, b, mirror)
    st = api.realisations(mom["mu_r"], secs, T, R_per=R, kernel=kernel, n_quad=n_quad,
                          exact=exact, field=field)
    return {k: {q: v.cpu().numpy() for q, v in d.items()} for k, d in st.items()}


def kernel_diagnostic(mu, mu_M, mu_M2, secs, T, n_quad: int = 0) -> Dict[str, dict]:
    """Thermodynamics of the same moments without and with the Jackson kernel.

    Returns {"none": thermo, "jackson": thermo, "diff": {obs: |none - jackson|}}
    for lnZ, E, C and chi (arrays or device tensors, like api.thermo)."""
    none = api.thermo(mu, mu_M, mu_M2, secs, T, kernel="none", n_quad=n_quad)
    jack = api.thermo(mu, mu_M, mu_M2, secs, T, kernel="jackson", n_quad=n_quad)
    diff = {k: abs(none[k] - jack[k]) for k in ("lnZ", "E", "C", "chi")}
    return {"none": none, "jackson": jack, "diff": diff}


def thermo_observer(model, n_up, K: int, R: int, seed: int, T, mirror=None,
                    kernel: str = "jackson", eps: float = 0.05, lanczos_iters: int = 100,
                    rebound: bool = True) -> Callable[[torch.Tensor], Dict[str, torch.Tensor]]:
    """observe(theta) -> {"lnZ", "E", "C", "chi"} on the grid T, differentiable in theta.

    theta holds one coupling per bond class of `model`.  With `rebound` the
    Lanczos bounds are recomputed for every theta (they are constants for the
    gradient); otherwise those of the starting model are kept."""
    T = np.asarray(T, dtype=np.float64)
    fixed = {}

    def spec_for(theta_np):
        m = model.with_couplings(theta_np)
        if rebound or not fixed:
            bnd = api.bounds(m, n_up, eps=eps, max_iter=lanczos_iters, tol=1e-8, seed=seed)
            fixed["a"], fixed["b"] = bnd["a"], bnd["b"]
        return {"model": model, "n_up": list(n_up), "K": K, "R": R, "seed": seed,
                "a": fixed["a"], "b": fixed["b"], "T": T, "mirror": mirror, "kernel": kernel}

    def observe(theta: torch.Tensor) -> Dict[str, torch.Tensor]:
        spec = spec_for(theta.detach().cpu().double().numpy())
        lnZ, E, C, chi = api.chebyshev_thermo(theta, spec)
        return {"lnZ": lnZ, "E": E, "C": C, "chi": chi}

    return observe


def fit_couplings(observe: Callable[[torch.Tensor], Dict[str, torch.Tensor]], theta0,
                  target: Dict[str, np.ndarray], weights: Optional[Dict[str, float]] = None,
                  steps: int = 100, lr: float = 0.02, tol: float = 0.0) -> Dict[str, np.ndarray]:
    """Least-squares fit of coupling parameters to target curves by Adam.

    loss(theta) = sum_k w_k mean_T (O_k(theta) - target_k)^2 over the observables
    in `target`, with w_k = 1 / mean(target_k^2) unless `weights` gives it.
    Returns {"theta": final parameters, "loss": loss per step, "path": parameters
    per step}."""
    theta = torch.tensor(np.asarray(theta0, dtype=np.float64), requires_grad=True)
    tgt = {k: torch.as_tensor(np.asarray(v, dtype=np.float64)) for k, v in target.items()}
    w = {k: (weights or {}).get(k, 1.0 / max(float((t ** 2).mean()), 1e-300)) for k, t in tgt.items()}
    opt = torch.optim.Adam([theta], lr=lr)
    losses, path = [], []
    for _ in range(steps):
        opt.zero_grad()
        obs = observe(theta)
        loss = sum(w[k] * ((obs[k].to(torch.float64).cpu() - tgt[k]) ** 2).mean() for k in tgt)
        loss.backward()
        losses.append(float(loss.detach()))
        path.append(theta.detach().numpy().copy())
        if losses[-1] <= tol:
            break
        opt.step()
    return {"theta": theta.detach().numpy().copy(), "loss": np.array(losses), "path": np.array(path)}

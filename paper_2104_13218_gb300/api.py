"""Python binding of libkpm: argument marshalling around the C ABI of include/kpm.h.

Every function here only converts arguments (numpy arrays for host memory,
torch CUDA tensors for device memory) and calls the library; all arithmetic
of the method runs in the CUDA kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np
import torch

from ._lib import (KPM_EBOUNDS, KPM_ENOTCONV, KPM_FP32, KPM_FP64, KPM_KERNEL_JACKSON,
                   KPM_KERNEL_NONE, KPM_VECTORS_BASIS, KPM_VECTORS_RADEMACHER, KpmModel, KpmOpts,
                   KpmSpinModel, check, lib)

PRECISIONS = {"fp64": KPM_FP64, "fp32": KPM_FP32}
KERNELS = {"none": KPM_KERNEL_NONE, "jackson": KPM_KERNEL_JACKSON}
VECTORS = {"rademacher": KPM_VECTORS_RADEMACHER, "basis": KPM_VECTORS_BASIS}


def make_opts(precision="fp64", vectors="rademacher", per_vector=False, tuned=False,
              ckpt_interval=0) -> KpmOpts:
    o = KpmOpts()
    o.precision = PRECISIONS[precision]
    o.vectors = VECTORS[vectors]
    o.per_vector = 1 if per_vector else 0
    o.tuned = 1 if tuned else 0
    o.ckpt_interval = int(ckpt_interval)
    return o


class CModel:
    """A Heisenberg model marshalled for the C ABI (keeps its arrays alive)."""

    def __init__(self, n_sites: int, bi, bj, J):
        self.n_sites = int(n_sites)
        self.bi = np.ascontiguousarray(bi, dtype=np.int32)
        self.bj = np.ascontiguousarray(bj, dtype=np.int32)
        self.J = np.ascontiguousarray(J, dtype=np.float64)
        self.struct = KpmModel(self.n_sites, len(self.bi), self.bi.ctypes.data,
                               self.bj.ctypes.data, self.J.ctypes.data)

    @classmethod
    def of(cls, model) -> "CModel":
        if isinstance(model, CModel):
            return model
        bi, bj, J = model.arrays()
        return cls(model.n_sites, bi, bj, J)

    @property
    def ref(self):
        return ctypes.byref(self.struct)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return x.data_ptr()
    return x.ctypes.data


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return stream


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


def _f64(x):
    return None if x is None else np.ascontiguousarray(x, dtype=np.float64)


def sector_dims(n_sites: int, n_up: Sequence[int]) -> np.ndarray:
    return np.array([lib().kpm_sector_dim(n_sites, int(k)) for k in n_up], dtype=np.float64)


# ---------------------------------------------------------------- bounds

def bounds_workspace_size(model, n_up) -> int:
    m = CModel.of(model)
    nu = _i32(n_up)
    return int(lib().kpm_bounds_workspace_size(m.ref, len(nu), nu.ctypes.data))


def bounds(model, n_up, eps: float = 0.025, max_iter: int = 100, tol: float = 1e-8, seed: int = 0,
           workspace: Optional[torch.Tensor] = None, stream=None, allow_notconv: bool = True):
    """Spectral bounds of each sector (Eq. E-2-4): dict(a, b, e_min, e_max, status)."""
    m = CModel.of(model)
    nu = _i32(n_up)
    S = len(nu)
    a, b, lo, hi = (np.zeros(S) for _ in range(4))
    ws = workspace
    rc = lib().kpm_bounds(m.ref, S, nu.ctypes.data, eps, max_iter, tol, seed, a.ctypes.data,
                          b.ctypes.data, lo.ctypes.data, hi.ctypes.data, _ptr(ws),
                          0 if ws is None else ws.numel() * ws.element_size(), _stream(stream))
    check("kpm_bounds", rc, allow=(KPM_ENOTCONV,) if allow_notconv else ())
    return {"a": a, "b": b, "e_min": lo, "e_max": hi, "status": rc}


# ---------------------------------------------------------------- moments

def moments_workspace_size(model, n_up, K: int, R: int, precision: str = "fp64",
                           vectors: str = "rademacher", per_vector: bool = False,
                           tuned: bool = False) -> int:
    m = CModel.of(model)
    nu = _i32(n_up)
    o = make_opts(precision, vectors, per_vector, tuned)
    return int(lib().kpm_moments_ex_workspace_size(m.ref, len(nu), nu.ctypes.data, K, R,
                                                   ctypes.byref(o)))


def moments(model, n_up, K: int, R: int, seed: int, a=None, b=None, eps: float = 0.025, r0: int = 0,
            precision: str = "fp64", weighted: bool = True, device: bool = False,
            out: Optional[dict] = None, workspace: Optional[torch.Tensor] = None, stream=None,
            allow_ebounds: bool = False, vectors: str = "rademacher", per_vector: bool = False,
            tuned: bool = False):
    """Chebyshev moments of every sector: dict(mu, mu_M, mu_M2, status), each [S, K]; with
    per_vector also mu_r [S, R, K] (the moments of every random vector).

    device=True returns torch float64 CUDA tensors (or fills `out`), else numpy arrays.
    """
    m = CModel.of(model)
    nu = _i32(n_up)
    S = len(nu)
    a = _f64(a)
    b = _f64(b)
    if device:
        dev = torch.device("cuda", torch.cuda.current_device())
        if out is None:
            out = {"mu": torch.empty((S, K), dtype=torch.float64, device=dev)}
            if weighted:
                out["mu_M"] = torch.empty((S, K), dtype=torch.float64, device=dev)
                out["mu_M2"] = torch.empty((S, K), dtype=torch.float64, device=dev)
        if per_vector and "mu_r" not in out:
            out["mu_r"] = torch.empty((S, R, K), dtype=torch.float64, device=dev)
    else:
        out = {"mu": np.zeros((S, K))}
        if weighted:
            out["mu_M"] = np.zeros((S, K))
            out["mu_M2"] = np.zeros((S, K))
        if per_vector:
            out["mu_r"] = np.zeros((S, R, K))
    o = make_opts(precision, vectors, per_vector, tuned)
    ws = workspace
    rc = lib().kpm_moments_ex(m.ref, S, nu.ctypes.data, _ptr(a), _ptr(b), eps, K, R, seed, r0,
                              ctypes.byref(o), _ptr(out["mu"]), _ptr(out.get("mu_M")),
                              _ptr(out.get("mu_M2")), _ptr(out.get("mu_r") if per_vector else None),
                              1 if device else 0, _ptr(ws),
                              0 if ws is None else ws.numel() * ws.element_size(), _stream(stream))
    check("kpm_moments_ex", rc, allow=(KPM_EBOUNDS,) if allow_ebounds else ())
    out["status"] = rc
    return out


def autotune(model, n_up, a, b, R: int, precision: str = "fp32", trial_steps: int = 8,
             stream=None) -> dict:
    """Search the moment loop's schedule for this problem (kpm_autotune); later calls
    with tuned=True use the choice.  dict(default_ms, best_ms, report)."""
    m = CModel.of(model)
    nu = _i32(n_up)
    a = _f64(a)
    b = _f64(b)
    d_ms = ctypes.c_double(0)
    b_ms = ctypes.c_double(0)
    rep = ctypes.create_string_buffer(8192)
    rc = lib().kpm_autotune(m.ref, len(nu), nu.ctypes.data, a.ctypes.data, b.ctypes.data, R,
                            PRECISIONS[precision], trial_steps, ctypes.byref(d_ms),
                            ctypes.byref(b_ms), rep, len(rep), _stream(stream))
    check("kpm_autotune", rc)
    return {"default_ms": d_ms.value, "best_ms": b_ms.value, "report": rep.value.decode()}


def fp64_peak(stream=None) -> dict:
    """Measured FP64 FMA rate of the current device: dict(tflops, ms)."""
    t = ctypes.c_double(0)
    ms = ctypes.c_double(0)
    rc = lib().kpm_fp64_peak(ctypes.byref(t), ctypes.byref(ms), _stream(stream))
    check("kpm_fp64_peak", rc)
    return {"tflops": t.value, "ms": ms.value}


# ---------------------------------------------------------------- thermodynamics

@dataclass
class SectorSet:
    """Per-sector constants the thermodynamics needs (host arrays).  M is the
    magnetisation n_up - N/2 of each sector (NaN for a full-space run)."""
    dim: np.ndarray
    mirror: np.ndarray
    a: np.ndarray
    b: np.ndarray
    M: Optional[np.ndarray] = None


def sector_set(n_sites, n_up, a, b, mirror=None) -> SectorSet:
    dims = sector_dims(n_sites, n_up)
    mir = np.zeros(len(n_up), dtype=np.int32) if mirror is None else _i32(mirror)
    M = np.array([np.nan if int(k) < 0 else int(k) - n_sites / 2.0 for k in n_up], dtype=np.float64)
    return SectorSet(dims, mir, _f64(a), _f64(b), M)


def _on_device(x) -> bool:
    return isinstance(x, torch.Tensor) and x.is_cuda


def thermo(mu, mu_M, mu_M2, secs: SectorSet, T, kernel: str = "none", n_quad: int = 0, stream=None,
           field: float = 0.0):
    """dict(lnZ, signZ, E, C, chi) on the temperature grid T (host array); `field` is the
    Zeeman energy h = g mu_B B of Eq. E-3-1-1 (sector runs only when nonzero)."""
    dev = _on_device(mu)
    S, K = mu.shape
    T = _f64(T)
    nT = len(T)
    if dev:
        outs = {k: torch.empty(nT, dtype=torch.float64, device=mu.device)
                for k in ("lnZ", "signZ", "E", "C", "chi")}
    else:
        outs = {k: np.zeros(nT) for k in ("lnZ", "signZ", "E", "C", "chi")}
        mu, mu_M, mu_M2 = (None if x is None else np.ascontiguousarray(x, dtype=np.float64)
                           for x in (mu, mu_M, mu_M2))
    rc = lib().kpm_thermo_ex(S, K, _ptr(mu), _ptr(mu_M), _ptr(mu_M2), secs.dim.ctypes.data,
                             secs.mirror.ctypes.data, _ptr(secs.M), secs.a.ctypes.data,
                             secs.b.ctypes.data, float(field), KERNELS[kernel], n_quad, nT,
                             T.ctypes.data, _ptr(outs["lnZ"]), _ptr(outs["signZ"]), _ptr(outs["E"]),
                             _ptr(outs["C"]), _ptr(outs["chi"]), 1 if dev else 0, _stream(stream))
    check("kpm_thermo_ex", rc)
    return outs


OBSERVABLES = ("lnZ", "E", "C", "chi")


def realisations(mu_r, secs: SectorSet, T, R_per: int = 1, kernel: str = "none", n_quad: int = 0,
                 exact: Optional[dict] = None, field: float = 0.0, stream=None):
    """Statistics of P = R / R_per realisations from per-vector moments mu_r [S, R, K]
    (kpm_realisations): {obs: {"mean", "var", "dev" (with exact), "all" [P, nT]}} for
    lnZ, E, C and chi (Eq. E-3-1 .. E-3-3)."""
    dev = _on_device(mu_r)
    S, R, K = mu_r.shape
    T = _f64(T)
    nT = len(T)
    P = R // R_per
    if dev:
        kw = dict(dtype=torch.float64, device=mu_r.device)
        mean, var, alls = (torch.empty((4, nT), **kw), torch.empty((4, nT), **kw),
                           torch.empty((P, 4, nT), **kw))
        dv = torch.empty((4, nT), **kw) if exact is not None else None
        ex = (torch.tensor(np.array([np.asarray(exact[k], dtype=np.float64) for k in OBSERVABLES]),
                           **kw) if exact is not None else None)
        mu_in = mu_r.contiguous()
    else:
        mean, var, alls = np.zeros((4, nT)), np.zeros((4, nT)), np.zeros((P, 4, nT))
        dv = np.zeros((4, nT)) if exact is not None else None
        ex = (np.ascontiguousarray([np.asarray(exact[k], dtype=np.float64) for k in OBSERVABLES])
              if exact is not None else None)
        mu_in = np.ascontiguousarray(mu_r, dtype=np.float64)
    rc = lib().kpm_realisations(S, K, R, R_per, _ptr(mu_in), secs.dim.ctypes.data,
                                secs.mirror.ctypes.data, secs.M.ctypes.data, secs.a.ctypes.data,
                                secs.b.ctypes.data, float(field), KERNELS[kernel], n_quad, nT,
                                T.ctypes.data, _ptr(ex), _ptr(mean), _ptr(var), _ptr(dv),
                                _ptr(alls), 1 if dev else 0, _stream(stream))
    check("kpm_realisations", rc)
    out = {}
    for i, k in enumerate(OBSERVABLES):
        out[k] = {"mean": mean[i], "var": var[i], "all": alls[:, i]}
        if dv is not None:
            out[k]["dev"] = dv[i]
    return out


def thermo_backward(mu, mu_M, mu_M2, secs: SectorSet, T, cot: dict, kernel: str = "none",
                    n_quad: int = 0, stream=None, field: float = 0.0):
    """dict(mu, mu_M, mu_M2) of dL/dmoments from cotangents cot[{lnZ, E, C, chi}]."""
    dev = _on_device(mu)
    S, K = mu.shape
    T = _f64(T)
    nT = len(T)
    if dev:
        grads = {k: torch.zeros((S, K), dtype=torch.float64, device=mu.device)
                 for k in ("mu", "mu_M", "mu_M2")}
        cots = {k: (None if cot.get(k) is None else cot[k].to(mu.device, torch.float64).contiguous())
                for k in ("lnZ", "E", "C", "chi")}
    else:
        grads = {k: np.zeros((S, K)) for k in ("mu", "mu_M", "mu_M2")}
        cots = {k: _f64(cot.get(k)) for k in ("lnZ", "E", "C", "chi")}
    rc = lib().kpm_thermo_backward_ex(S, K, _ptr(mu), _ptr(mu_M), _ptr(mu_M2),
                                      secs.dim.ctypes.data, secs.mirror.ctypes.data, _ptr(secs.M),
                                      secs.a.ctypes.data, secs.b.ctypes.data, float(field),
                                      KERNELS[kernel], n_quad, nT, T.ctypes.data,
                                      _ptr(cots["lnZ"]), _ptr(cots["E"]), _ptr(cots["C"]),
                                      _ptr(cots["chi"]), _ptr(grads["mu"]), _ptr(grads["mu_M"]),
                                      _ptr(grads["mu_M2"]), 1 if dev else 0, _stream(stream))
    check("kpm_thermo_backward_ex", rc)
    return grads


# ---------------------------------------------------------------- adjoint

def moments_backward_workspace_size(model, n_up, K, R, ckpt_interval=32) -> int:
    m = CModel.of(model)
    nu = _i32(n_up)
    return int(lib().kpm_moments_backward_workspace_size(m.ref, len(nu), nu.ctypes.data, K, R,
                                                         ckpt_interval))


def moments_backward(model, bond_class, n_classes, n_up, a, b, K, R, seed, grads: dict, r0=0,
                     ckpt_interval=32, workspace=None, stream=None, vectors: str = "rademacher"):
    """dL/dtheta [n_classes] for J_b = theta[bond_class[b]] given dL/dmoments
    (bond_class None: one class per bond, dL/dJ_b)."""
    m = CModel.of(model)
    nu = _i32(n_up)
    S = len(nu)
    cls = None if bond_class is None else _i32(bond_class)
    dev = _on_device(grads["mu"])
    if dev:
        out = torch.zeros(n_classes, dtype=torch.float64, device=grads["mu"].device)
        g = [None if grads.get(k) is None else grads[k].contiguous() for k in ("mu", "mu_M", "mu_M2")]
    else:
        out = np.zeros(n_classes)
        g = [None if grads.get(k) is None else np.ascontiguousarray(grads[k], dtype=np.float64)
             for k in ("mu", "mu_M", "mu_M2")]
    a = _f64(a)
    b = _f64(b)
    ws = workspace
    o = make_opts("fp64", vectors, False, False, ckpt_interval)
    rc = lib().kpm_moments_backward_ex(m.ref, _ptr(cls), n_classes, S, nu.ctypes.data,
                                       a.ctypes.data, b.ctypes.data, K, R, seed, r0,
                                       ctypes.byref(o), _ptr(g[0]), _ptr(g[1]), _ptr(g[2]),
                                       _ptr(out), 1 if dev else 0, _ptr(ws),
                                       0 if ws is None else ws.numel() * ws.element_size(),
                                       _stream(stream))
    check("kpm_moments_backward_ex", rc)
    return out


class ChebyshevThermo(torch.autograd.Function):
    """theta (coupling parameters) -> (lnZ, E, C, chi)(T) through the GPU moment loop.

    The forward runs kpm_moments (FP64, device) and kpm_thermo; the backward
    runs kpm_thermo_backward and the adjoint kpm_moments_backward.  The
    rescaling (a, b) of every sector is a constant.
    """

    @staticmethod
    def forward(ctx, theta, spec):
        th = theta.detach().cpu().double().numpy()
        model = spec["model"].with_couplings(th)
        res = moments(model, spec["n_up"], spec["K"], spec["R"], spec["seed"], a=spec["a"],
                      b=spec["b"], r0=spec.get("r0", 0), precision="fp64", device=True,
                      allow_ebounds=True, vectors=spec.get("vectors", "rademacher"))
        secs = sector_set(model.n_sites, spec["n_up"], spec["a"], spec["b"], spec.get("mirror"))
        out = thermo(res["mu"], res["mu_M"], res["mu_M2"], secs, spec["T"],
                     kernel=spec.get("kernel", "none"), n_quad=spec.get("n_quad", 0),
                     field=spec.get("field", 0.0))
        ctx.spec = spec
        ctx.model = model
        ctx.secs = secs
        ctx.mom = res
        dev = theta.device
        return tuple(out[k].to(dev) for k in ("lnZ", "E", "C", "chi"))

    @staticmethod
    def backward(ctx, g_lnZ, g_E, g_C, g_chi):
        spec = ctx.spec
        res = ctx.mom
        dev = res["mu"].device
        cot = {k: (None if g is None else g.to(dev, torch.float64))
               for k, g in zip(("lnZ", "E", "C", "chi"), (g_lnZ, g_E, g_C, g_chi))}
        grads = thermo_backward(res["mu"], res["mu_M"], res["mu_M2"], ctx.secs, spec["T"], cot,
                                kernel=spec.get("kernel", "none"), n_quad=spec.get("n_quad", 0),
                                field=spec.get("field", 0.0))
        cls = ctx.model.classes()
        P = int(cls.max()) + 1
        g = moments_backward(ctx.model, cls, P, spec["n_up"], spec["a"], spec["b"], spec["K"],
                             spec["R"], spec["seed"], grads, r0=spec.get("r0", 0),
                             ckpt_interval=spec.get("ckpt_interval", 32),
                             vectors=spec.get("vectors", "rademacher"))
        return g.cpu(), None


def chebyshev_thermo(theta: torch.Tensor, spec: dict):
    """(lnZ, E, C, chi) as differentiable functions of the coupling parameters theta."""
    return ChebyshevThermo.apply(theta, spec)


# ---------------------------------------------------------------- spin s

class CSpinModel:
    """A spin-s Heisenberg model (two_s = 2s) marshalled for the C ABI."""

    def __init__(self, n_sites: int, two_s: int, bi, bj, J):
        self.n_sites = int(n_sites)
        self.two_s = int(two_s)
        self.bi = np.ascontiguousarray(bi, dtype=np.int32)
        self.bj = np.ascontiguousarray(bj, dtype=np.int32)
        self.J = np.ascontiguousarray(J, dtype=np.float64)
        self.struct = KpmSpinModel(self.n_sites, len(self.bi), self.two_s, 0, self.bi.ctypes.data,
                                   self.bj.ctypes.data, self.J.ctypes.data)

    @classmethod
    def of(cls, model, two_s: int) -> "CSpinModel":
        bi, bj, J = model.arrays()
        return cls(model.n_sites, two_s, bi, bj, J)

    @property
    def ref(self):
        return ctypes.byref(self.struct)


def spin_sector_dims(n_sites: int, two_s: int, Q: Sequence[int]) -> np.ndarray:
    return np.array([lib().kpm_spin_sector_dim(n_sites, two_s, int(q)) for q in Q], dtype=np.float64)


def spin_sector_set(n_sites: int, two_s: int, Q, a, b, mirror=None) -> SectorSet:
    """Per-sector constants of spin-s sectors for thermo(): M = Q - N s (NaN for Q = -1)."""
    dims = spin_sector_dims(n_sites, two_s, Q)
    mir = np.zeros(len(Q), dtype=np.int32) if mirror is None else _i32(mirror)
    M = np.array([np.nan if int(q) < 0 else int(q) - n_sites * two_s / 2.0 for q in Q])
    return SectorSet(dims, mir, _f64(a), _f64(b), M)


def spin_bounds(model, two_s: int, Q, eps: float = 0.025, max_iter: int = 200, tol: float = 1e-8,
                seed: int = 0, stream=None, allow_notconv: bool = True):
    """Lanczos bounds of spin-s sectors: dict(a, b, e_min, e_max, status)."""
    m = CSpinModel.of(model, two_s) if not isinstance(model, CSpinModel) else model
    q = _i32(Q)
    S = len(q)
    a, b, lo, hi = (np.zeros(S) for _ in range(4))
    rc = lib().kpm_spin_bounds(m.ref, S, q.ctypes.data, eps, max_iter, tol, seed, a.ctypes.data,
                               b.ctypes.data, lo.ctypes.data, hi.ctypes.data, _stream(stream))
    check("kpm_spin_bounds", rc, allow=(KPM_ENOTCONV,) if allow_notconv else ())
    return {"a": a, "b": b, "e_min": lo, "e_max": hi, "status": rc}


def spin_moments(model, two_s: int, Q, K: int, R: int, seed: int, a, b, r0: int = 0,
                 precision: str = "fp64", weighted: bool = True, device: bool = False, stream=None,
                 allow_ebounds: bool = False):
    """Chebyshev moments of spin-s sectors: dict(mu, mu_M, mu_M2, status), each [S, K]."""
    m = CSpinModel.of(model, two_s) if not isinstance(model, CSpinModel) else model
    q = _i32(Q)
    S = len(q)
    a = _f64(a)
    b = _f64(b)
    if device:
        dev = torch.device("cuda", torch.cuda.current_device())
        out = {k: torch.empty((S, K), dtype=torch.float64, device=dev)
               for k in (("mu", "mu_M", "mu_M2") if weighted else ("mu",))}
    else:
        out = {k: np.zeros((S, K)) for k in (("mu", "mu_M", "mu_M2") if weighted else ("mu",))}
    rc = lib().kpm_spin_moments(m.ref, S, q.ctypes.data, a.ctypes.data, b.ctypes.data, K, R, seed,
                                r0, PRECISIONS[precision], _ptr(out["mu"]), _ptr(out.get("mu_M")),
                                _ptr(out.get("mu_M2")), 1 if device else 0, _stream(stream))
    check("kpm_spin_moments", rc, allow=(KPM_EBOUNDS,) if allow_ebounds else ())
    out["status"] = rc
    return out

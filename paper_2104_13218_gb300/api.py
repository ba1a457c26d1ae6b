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
                   KPM_KERNEL_NONE, KpmModel, check, lib)

PRECISIONS = {"fp64": KPM_FP64, "fp32": KPM_FP32}
KERNELS = {"none": KPM_KERNEL_NONE, "jackson": KPM_KERNEL_JACKSON}


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

def moments_workspace_size(model, n_up, K: int, R: int, precision: str = "fp64") -> int:
    m = CModel.of(model)
    nu = _i32(n_up)
    return int(lib().kpm_moments_workspace_size(m.ref, len(nu), nu.ctypes.data, K, R,
                                                PRECISIONS[precision]))


def moments(model, n_up, K: int, R: int, seed: int, a=None, b=None, eps: float = 0.025, r0: int = 0,
            precision: str = "fp64", weighted: bool = True, device: bool = False,
            out: Optional[dict] = None, workspace: Optional[torch.Tensor] = None, stream=None,
            allow_ebounds: bool = False):
    """Chebyshev moments of every sector: dict(mu, mu_M, mu_M2, status), each [S, K].

    device=True returns torch float64 CUDA tensors (or fills `out`), else numpy arrays.
    """
    m = CModel.of(model)
    nu = _i32(n_up)
    S = len(nu)
    a = _f64(a)
    b = _f64(b)
    if device:
        if out is None:
            dev = torch.device("cuda", torch.cuda.current_device())
            out = {"mu": torch.empty((S, K), dtype=torch.float64, device=dev)}
            if weighted:
                out["mu_M"] = torch.empty((S, K), dtype=torch.float64, device=dev)
                out["mu_M2"] = torch.empty((S, K), dtype=torch.float64, device=dev)
    else:
        out = {"mu": np.zeros((S, K))}
        if weighted:
            out["mu_M"] = np.zeros((S, K))
            out["mu_M2"] = np.zeros((S, K))
    ws = workspace
    rc = lib().kpm_moments(m.ref, S, nu.ctypes.data, _ptr(a), _ptr(b), eps, K, R, seed, r0,
                           PRECISIONS[precision], _ptr(out["mu"]), _ptr(out.get("mu_M")),
                           _ptr(out.get("mu_M2")), 1 if device else 0, _ptr(ws),
                           0 if ws is None else ws.numel() * ws.element_size(), _stream(stream))
    check("kpm_moments", rc, allow=(KPM_EBOUNDS,) if allow_ebounds else ())
    out["status"] = rc
    return out


# ---------------------------------------------------------------- thermodynamics

@dataclass
class SectorSet:
    """Per-sector constants the thermodynamics needs (host arrays)."""
    dim: np.ndarray
    mirror: np.ndarray
    a: np.ndarray
    b: np.ndarray


def sector_set(n_sites, n_up, a, b, mirror=None) -> SectorSet:
    dims = sector_dims(n_sites, n_up)
    mir = np.zeros(len(n_up), dtype=np.int32) if mirror is None else _i32(mirror)
    return SectorSet(dims, mir, _f64(a), _f64(b))


def _on_device(x) -> bool:
    return isinstance(x, torch.Tensor) and x.is_cuda


def thermo(mu, mu_M, mu_M2, secs: SectorSet, T, kernel: str = "none", n_quad: int = 0, stream=None):
    """dict(lnZ, signZ, E, C, chi) on the temperature grid T (host array)."""
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
    rc = lib().kpm_thermo(S, K, _ptr(mu), _ptr(mu_M), _ptr(mu_M2), secs.dim.ctypes.data,
                          secs.mirror.ctypes.data, secs.a.ctypes.data, secs.b.ctypes.data,
                          KERNELS[kernel], n_quad, nT, T.ctypes.data, _ptr(outs["lnZ"]),
                          _ptr(outs["signZ"]), _ptr(outs["E"]), _ptr(outs["C"]), _ptr(outs["chi"]),
                          1 if dev else 0, _stream(stream))
    check("kpm_thermo", rc)
    return outs


def thermo_backward(mu, mu_M, mu_M2, secs: SectorSet, T, cot: dict, kernel: str = "none",
                    n_quad: int = 0, stream=None):
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
    rc = lib().kpm_thermo_backward(S, K, _ptr(mu), _ptr(mu_M), _ptr(mu_M2), secs.dim.ctypes.data,
                                   secs.mirror.ctypes.data, secs.a.ctypes.data, secs.b.ctypes.data,
                                   KERNELS[kernel], n_quad, nT, T.ctypes.data, _ptr(cots["lnZ"]),
                                   _ptr(cots["E"]), _ptr(cots["C"]), _ptr(cots["chi"]),
                                   _ptr(grads["mu"]), _ptr(grads["mu_M"]), _ptr(grads["mu_M2"]),
                                   1 if dev else 0, _stream(stream))
    check("kpm_thermo_backward", rc)
    return grads


# ---------------------------------------------------------------- adjoint

def moments_backward_workspace_size(model, n_up, K, R, ckpt_interval=32) -> int:
    m = CModel.of(model)
    nu = _i32(n_up)
    return int(lib().kpm_moments_backward_workspace_size(m.ref, len(nu), nu.ctypes.data, K, R,
                                                         ckpt_interval))


def moments_backward(model, bond_class, n_classes, n_up, a, b, K, R, seed, grads: dict, r0=0,
                     ckpt_interval=32, workspace=None, stream=None):
    """dL/dtheta [n_classes] for J_b = theta[bond_class[b]] given dL/dmoments."""
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
    rc = lib().kpm_moments_backward(m.ref, _ptr(cls), n_classes, S, nu.ctypes.data, a.ctypes.data,
                                    b.ctypes.data, K, R, seed, r0, KPM_FP64, ckpt_interval,
                                    _ptr(g[0]), _ptr(g[1]), _ptr(g[2]), _ptr(out), 1 if dev else 0,
                                    _ptr(ws), 0 if ws is None else ws.numel() * ws.element_size(),
                                    _stream(stream))
    check("kpm_moments_backward", rc)
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
                      allow_ebounds=True)
        secs = sector_set(model.n_sites, spec["n_up"], spec["a"], spec["b"], spec.get("mirror"))
        out = thermo(res["mu"], res["mu_M"], res["mu_M2"], secs, spec["T"],
                     kernel=spec.get("kernel", "none"), n_quad=spec.get("n_quad", 0))
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
                                kernel=spec.get("kernel", "none"), n_quad=spec.get("n_quad", 0))
        cls = ctx.model.classes()
        P = int(cls.max()) + 1
        g = moments_backward(ctx.model, cls, P, spec["n_up"], spec["a"], spec["b"], spec["K"],
                             spec["R"], spec["seed"], grads, r0=spec.get("r0", 0),
                             ckpt_interval=spec.get("ckpt_interval", 32))
        return g.cpu(), None


def chebyshev_thermo(theta: torch.Tensor, spec: dict):
    """(lnZ, E, C, chi) as differentiable functions of the coupling parameters theta."""
    return ChebyshevThermo.apply(theta, spec)

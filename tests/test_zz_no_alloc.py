"""kpm_moments_static, the allocation-free variant of kpm_moments, through the C ABI.

Some callers cannot allocate device memory themselves: their framework has
already reserved the device memory in its own pool, or they run a
latency-critical loop that must not enter the CUDA allocator.  For them the
library offers kpm_moments_static, whose scratch lives in a fixed array inside
the library.  This test checks, on two calls in a row (the second one reuses
the array left behind by the first), that it returns the same moments as
kpm_moments within the FP64 tolerance of the parity tests, in both precisions,
and that a problem too large for the array is refused with a clear error.
It sits in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest
import torch

import kpm_workloads as W
import paper_2104_13218_gb300 as kpm
from paper_2104_13218_gb300 import _lib

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _static_moments(model, n_up, a, b, K, R, seed, precision):
    m = kpm.CModel.of(model)
    nu = np.ascontiguousarray(n_up, dtype=np.int32)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    S = len(nu)
    out = {k: torch.full((S, K), float("nan"), dtype=torch.float64, device="cuda")
           for k in ("mu", "mu_M", "mu_M2")}
    rc = kpm.lib().kpm_moments_static(m.ref, S, nu.ctypes.data, a.ctypes.data, b.ctypes.data, K, R,
                                      seed, 0, kpm.api.PRECISIONS[precision], out["mu"].data_ptr(),
                                      out["mu_M"].data_ptr(), out["mu_M2"].data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
    _lib.check("kpm_moments_static", rc)
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_scratch_matches_kpm_moments_on_two_calls(precision):
    model = W.ring(14)
    n_up = W.all_sectors(14) + [-1]
    bnd = kpm.bounds(model, n_up, eps=0.025, max_iter=80, seed=3)
    K, R, seed = 120, 10, 17
    ref = kpm.moments(model, n_up, K, R, seed, a=bnd["a"], b=bnd["b"], precision=precision)
    for call in range(2):
        got = _static_moments(model, n_up, bnd["a"], bnd["b"], K, R, seed, precision)
        for q in ("mu", "mu_M", "mu_M2"):
            err = np.abs(got[q] - ref[q]) / np.maximum(1.0, np.abs(ref[q]))
            assert err.max() <= TOL64, (call, q, err.max())


def test_static_scratch_refuses_problems_beyond_its_size():
    limit = kpm.lib().kpm_static_scratch_bytes()
    assert limit == 64 << 20
    model = W.ring(20)
    need = kpm.moments_workspace_size(model, [10], 40, 64, "fp64")
    assert need > limit
    m = kpm.CModel.of(model)
    nu = np.array([10], dtype=np.int32)
    a = np.array([8.0])
    b = np.array([-2.0])
    mu = torch.zeros((1, 40), dtype=torch.float64, device="cuda")
    rc = kpm.lib().kpm_moments_static(m.ref, 1, nu.ctypes.data, a.ctypes.data, b.ctypes.data, 40, 64,
                                      1, 0, 0, mu.data_ptr(), None, None,
                                      torch.cuda.current_stream().cuda_stream)
    assert rc == _lib.KPM_ENOMEM
    msg = kpm.lib().kpm_last_error().decode()
    assert "static array" in msg and str(need) in msg

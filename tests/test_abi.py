"""The C ABI library loads, exports every function include/kpm.h declares, and
rejects invalid arguments before touching the GPU (no GPU needed)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import kpm_workloads as W
import paper_2104_13218_gb300 as kpm
from paper_2104_13218_gb300 import _lib
from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "kpm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kpm_\w+)\s*\(", text)))


def test_library_exports_every_declared_function():
    names = declared_functions()
    assert "kpm_moments" in names and "kpm_bounds" in names and "kpm_thermo" in names
    assert "kpm_moments_backward" in names and "kpm_thermo_backward" in names
    h = ctypes.CDLL(kpm.library_path())
    for n in names:
        assert hasattr(h, n), n
    # the binding declares a prototype for each of them
    assert set(names) <= set(_lib.PROTOTYPES)


def test_version_and_sector_dims():
    L = kpm.lib()
    assert L.kpm_version() == 2
    assert L.kpm_sector_dim(34, 17) == 2333606220
    assert L.kpm_sector_dim(20, -1) == 1 << 20
    assert L.kpm_sector_dim(24, 12) == 2704156
    assert L.kpm_sector_dim(35, 3) == -1
    assert L.kpm_sector_dim(10, 11) == -1


def _model_struct(model):
    return kpm.CModel.of(model)


@pytest.mark.parametrize("K,R,prec", [(3, 4, 0), (0, 4, 0), (10, 0, 0), (10, 600, 1), (10, 513, 0),
                                      (10, 4, 7)])
def test_moments_rejects_bad_sizes(K, R, prec):
    m = _model_struct(W.ring(8))
    nu = np.array([4], dtype=np.int32)
    mu = np.zeros(max(K, 1))
    a = np.array([3.0])
    b = np.array([0.0])
    rc = kpm.lib().kpm_moments(m.ref, 1, nu.ctypes.data, a.ctypes.data, b.ctypes.data, 0.025, K, R,
                               1, 0, prec, mu.ctypes.data, None, None, 0, None, 0, None)
    assert rc == _lib.KPM_EINVAL
    assert len(kpm.lib().kpm_last_error()) > 0


def test_invalid_models_and_sectors_are_rejected():
    L = kpm.lib()
    bad = kpm.CModel(8, [0, 1], [1, 1], [1.0, 1.0])  # bond (1, 1)
    nu = np.array([4], dtype=np.int32)
    assert L.kpm_moments_workspace_size(bad.ref, 1, nu.ctypes.data, 10, 4, 0) == 0
    big = kpm.CModel(35, [0], [1], [1.0])
    assert L.kpm_moments_workspace_size(big.ref, 1, nu.ctypes.data, 10, 4, 0) == 0
    ok = _model_struct(W.ring(8))
    nu_bad = np.array([9], dtype=np.int32)
    assert L.kpm_moments_workspace_size(ok.ref, 1, nu_bad.ctypes.data, 10, 4, 0) == 0
    assert L.kpm_moments_workspace_size(ok.ref, 1, nu.ctypes.data, 10, 4, 0) > 0
    # too many classes for the adjoint
    many = _model_struct(W.ring(10))
    assert L.kpm_moments_backward_workspace_size(many.ref, 1, nu.ctypes.data, 10, 4, 32) > 0


def test_workspace_sizes_scale_with_problem():
    small = kpm.moments_workspace_size(W.ring(14), [7], 100, 8, "fp64")
    big = kpm.moments_workspace_size(W.ring(14), [7], 100, 16, "fp64")
    f32 = kpm.moments_workspace_size(W.ring(14), [7], 100, 16, "fp32")
    assert big > small > 0
    assert f32 < big
    # in the FP32 form a sector below 1024 states is stored in FP64
    assert (kpm.moments_workspace_size(W.ring(12), [6], 100, 16, "fp32")
            == kpm.moments_workspace_size(W.ring(12), [6], 100, 16, "fp64"))
    # two interleaved vectors of the ring-34 S^z = 0 sector in FP32 with R = 4
    cfg5 = kpm.moments_workspace_size(W.ring(34), [17], 2000, 4, "fp32")
    assert cfg5 >= 2 * 2333606220 * 4 * 4


def test_bounds_workspace_holds_three_vectors_and_lists():
    # three FP64 Lanczos vectors (16-byte rows); with grouped couplings also the
    # entry-major neighbour lists (a header word and one word per bond and state)
    dim = math.comb(14, 7)
    ring = W.ring(14)
    grouped = kpm.bounds_workspace_size(ring, [7])
    assert grouped >= 3 * dim * 16 + dim * (1 + 14) * 4
    # more distinct couplings than the grouped step handles: no lists
    distinct = W.Model("ring14_distinct", 14, ring.bi, ring.bj, tuple(1.0 + 0.1 * k for k in range(14)))
    ungrouped = kpm.bounds_workspace_size(distinct, [7])
    assert 3 * dim * 16 <= ungrouped < grouped
    # the ring N=34 S^z=0 sector: lists would exceed 2 GiB, so only the vectors
    big = kpm.bounds_workspace_size(W.ring(34), [17])
    assert 3 * 2333606220 * 16 <= big < 3 * 2333606220 * 16 + (1 << 31)

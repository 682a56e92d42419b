"""The allocation-free residual entry point agrees with the workspace one.

fnlh_residual_noalloc exists for callers that cannot allocate device memory
(a host code whose memory pool owns the whole device budget, or a caller
inside a CUDA stream capture, where cudaMalloc is not allowed): it keeps its
partial sums in a device array built into the library instead of a caller
workspace.  This file is named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest
import torch

from paper_2404_01407_gb300 import fnlh, inputs
from tests import _gpu

pytestmark = pytest.mark.gpu


def _call_noalloc(dm, J, omega, B, X, r, norms):
    om = np.ascontiguousarray(np.atleast_1d(np.asarray(omega, dtype=np.float64)))
    omp = om.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = fnlh.lib().fnlh_residual_noalloc(ctypes.byref(dm.c), ctypes.byref(J.c), len(om), omp, None,
                                          ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                          ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(norms.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == fnlh.FNLH_OK, fnlh.fnlh_strerror(st)


def test_noalloc_residual_matches_workspace_residual_on_consecutive_calls():
    # a larger problem, then a smaller one (fewer partial slots, so stale sums
    # from the first call remain in the shared array), then the first again
    big = inputs.problem((20, 12, 10), 6, 4, 20.0, name="b6n4")
    small = inputs.problem((7, 5, 3), 5, 1, 10.0, 1.5, seeds=(11, 12, 13), name="b5n1")
    cases = []
    for p in (big, small):
        dm, J, B = _gpu.device_problem(p, prep_flags=fnlh.FNLH_PREP_F64)
        X = torch.from_numpy(np.random.default_rng(1).normal(size=p.b.shape)).cuda()
        r_ref = torch.empty_like(B)
        n_ref = fnlh.fnlh_residual(dm, J, p.omega, B, X, r=r_ref)
        cases.append((p, dm, J, B, X, r_ref.cpu().numpy(), n_ref.cpu().numpy()))
    torch.cuda.synchronize()
    free_after = []
    for p, dm, J, B, X, r_ref, n_ref in (cases[0], cases[1], cases[0]):
        r = torch.full_like(B, float("nan"))
        norms = torch.full((1 + p.n_harm, 2), float("nan"), dtype=torch.float64, device="cuda")
        _call_noalloc(dm, J, p.omega, B, X, r, norms)
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
        assert np.allclose(norms.cpu().numpy(), n_ref, rtol=1e-12, atol=0)
        assert np.abs(r.cpu().numpy() - r_ref).max() <= 1e-13 * np.abs(r_ref).max()
    # no device allocation by the later calls
    assert free_after[1] == free_after[2]

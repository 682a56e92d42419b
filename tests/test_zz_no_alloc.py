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


def _call_noalloc(dm, J, omega, B, X, r, norms, n_harm=None):
    om = np.ascontiguousarray(np.atleast_1d(np.asarray(omega, dtype=np.float64)))
    omp = om.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    n = len(om) if n_harm is None else n_harm
    return fnlh.lib().fnlh_residual_noalloc(ctypes.byref(dm.c), ctypes.byref(J.c), n, omp, None,
                                            ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                            ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(norms.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _case(p, seed=1):
    dm, J, B = _gpu.device_problem(p, prep_flags=fnlh.FNLH_PREP_F64)
    X = torch.from_numpy(np.random.default_rng(seed).normal(size=p.b.shape)).cuda()
    r_ref = torch.empty_like(B)
    n_ref = fnlh.fnlh_residual(dm, J, p.omega, B, X, r=r_ref)
    # output buffers of the allocation-free calls, made before the first call
    r = torch.empty_like(B)
    norms = torch.empty((1 + p.n_harm, 2), dtype=torch.float64, device="cuda")
    return p, dm, J, B, X, r_ref, n_ref, r, norms


def test_noalloc_residual_matches_workspace_residual_on_consecutive_calls():
    # a larger problem, then a smaller one (fewer partial slots, so stale sums
    # from the first call remain in the shared array), then the first again,
    # and last the largest harmonic count on a mesh that fills the whole grid
    # of partial sums (1216 blocks x 2 x 65 systems: the array's full size)
    cases = [_case(inputs.problem((20, 12, 10), 6, 4, 20.0, name="b6n4")),
             _case(inputs.problem((7, 5, 3), 5, 1, 10.0, 1.5, seeds=(11, 12, 13), name="b5n1")),
             _case(inputs.problem((40, 32, 32), 6, fnlh.MAX_HARMONICS, 20.0, 0.05, name="b6n64"))]
    torch.cuda.synchronize()
    free = [torch.cuda.mem_get_info()[0]]
    for p, dm, J, B, X, r_ref, n_ref, r, norms in (cases[0], cases[1], cases[0], cases[2]):
        r.fill_(float("nan"))
        norms.fill_(float("nan"))
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        st = _call_noalloc(dm, J, p.omega, B, X, r, norms)
        assert st == fnlh.FNLH_OK, fnlh.fnlh_strerror(st)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        # the same kernels and the same fixed-order sums as the workspace path
        assert torch.equal(norms, n_ref)
        assert torch.equal(r, r_ref)
    # no device memory taken by any call, the first included
    assert all(f == free[0] for f in free), free


def test_noalloc_residual_rejects_too_many_harmonics():
    p, dm, J, B, X, r_ref, n_ref, r, norms = _case(inputs.problem((7, 5, 3), 5, 1, 10.0, name="b5n1"))
    norms.fill_(float("nan"))
    om = np.arange(1, fnlh.MAX_HARMONICS + 2, dtype=np.float64)
    st = _call_noalloc(dm, J, om, B, X, r, norms, n_harm=fnlh.MAX_HARMONICS + 1)
    assert st != fnlh.FNLH_OK
    torch.cuda.synchronize()
    assert torch.isnan(norms).all()  # nothing was launched

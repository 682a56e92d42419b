"""Shared set-up for the GPU tests: seeded problems on the device and the
matching oracle objects on the host."""

import numpy as np
import torch

import oracle
from paper_2404_01407_gb300 import fnlh, inputs

ALL_PREP = fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_F32 | fnlh.FNLH_PREP_BF16


def device_problem(p: inputs.Problem, prep_flags=ALL_PREP, device="cuda", pseudo_time=0):
    dm = fnlh.DeviceMesh.from_mesh(p.mesh, device)
    J = fnlh.DeviceJacobian(dm, p.block, prep_flags, device)
    Q = torch.from_numpy(p.q).to(device)
    fnlh.fnlh_build_jacobian(dm, Q, fnlh.make_params(p.cfl, pseudo_time=pseudo_time), J)
    B = torch.from_numpy(p.b).to(device)
    return dm, J, B


def oracle_jacobian(p: inputs.Problem, pseudo_time=0):
    m = p.mesh
    return oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl, pseudo_block=bool(pseudo_time))


def load_jacobian(dm, J, ojac):
    """Overwrite the device J with the oracle's blocks and re-prepare (isolates the sweep)."""
    J.offd.copy_(torch.from_numpy(np.ascontiguousarray(ojac.offd)))
    J.diag.copy_(torch.from_numpy(np.ascontiguousarray(ojac.diag)))
    J.D.copy_(torch.from_numpy(ojac.D))
    fnlh.fnlh_prepare(dm, J)


def rel_err_per_system(x, ref, n_harm):
    """||x_k - ref_k|| / ||ref_k|| per system (mean first), complex 2-norm."""
    out = []
    cols = [[0]] + [[2 * k - 1, 2 * k] for k in range(1, n_harm + 1)]
    for c in cols:
        d = np.linalg.norm(x[:, c, :] - ref[:, c, :])
        out.append(d / max(np.linalg.norm(ref[:, c, :]), 1e-300))
    return np.array(out)


def max_err_per_system(x, ref, n_harm):
    """max_i |x_k,i - ref_k,i| / max_i |ref_k,i| per system (mean first), over
    every real and imaginary entry of the system."""
    out = []
    cols = [[0]] + [[2 * k - 1, 2 * k] for k in range(1, n_harm + 1)]
    for c in cols:
        d = np.abs(x[:, c, :] - ref[:, c, :]).max(initial=0.0)
        out.append(d / max(np.abs(ref[:, c, :]).max(initial=0.0), 1e-300))
    return np.array(out)


def assert_fp64_parity(x, ref, n_harm, tol=1e-12):
    """The FP64 parity bar, per system: the 2-norm of the difference within
    tol of the reference's 2-norm AND every single entry within tol of the
    reference's largest entry (a 2-norm alone lets one wrong entry of a large
    system hide below the bar)."""
    err2 = rel_err_per_system(x, ref, n_harm)
    errinf = max_err_per_system(x, ref, n_harm)
    assert np.all(err2 <= tol), ("2-norm", err2)
    assert np.all(errinf <= tol), ("max-entry", errinf)
    return err2, errinf

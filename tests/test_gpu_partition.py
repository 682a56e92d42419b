"""GPU parity of domain-truncated block Jacobi (the paper's parallel
decomposition: couplings between nodes of different partitions are ignored,
so each partition relaxes on its own).

The sweeps drop the cross-partition couplings and match the oracle's
truncated Jacobi to relative 1e-12 in FP64; the residual keeps every
coupling, so the defect-correction solve still converges to the full
system's solution (true FP64 residual 1e-8, measured by the oracle), and its
FP64 form matches the oracle composition residual -> truncated sweeps from
zero -> update, check by check.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2404_01407_gb300 import fnlh, inputs
from tests import _gpu

pytestmark = pytest.mark.gpu

PREP = _gpu.ALL_PREP | fnlh.FNLH_PREP_TAGS


def device_problem(p, part, prep_flags=PREP):
    dm = fnlh.DeviceMesh.from_mesh(p.mesh, "cuda", part=part)
    J = fnlh.DeviceJacobian(dm, p.block, prep_flags)
    fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).cuda(), fnlh.make_params(p.cfl), J)
    return dm, J, torch.from_numpy(p.b).cuda()


def oracle_jac(p):
    m = p.mesh
    return oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl, periodic=m.periodic)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    fnlh.lib()


CASES = [
    # (dims, block, N, parts): ragged tiles, boxes of unequal size
    ((13, 6, 5), 6, 4, (3, 2, 1)),
    ((7, 5, 3), 5, 3, (2, 2, 2)),
    ((9, 7, 5), 6, 8, (1, 1, 1)),
]


@pytest.mark.parametrize("dims,block,N,parts", CASES)
def test_truncated_relax_f64_matches_oracle(dims, block, N, parts):
    p = inputs.problem(dims, block, N, 20.0, 1.3)
    part = inputs.box_partition(dims, parts)
    dm, J, B = device_problem(p, part)
    oj = oracle_jac(p)
    _gpu.load_jacobian(dm, J, oj)
    x0 = np.random.default_rng(7).normal(size=p.b.shape)
    X = torch.from_numpy(x0.copy()).cuda()
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 25, fnlh.FNLH_F64)
    ref = oracle.jacobi(oj, p.mesh.vol, p.omega, p.b, 25, X0=x0, part=part)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


def test_single_node_partitions_and_periodic_edges():
    """Every node its own partition on a periodic passage: one sweep is the
    exact block solve and further sweeps leave it unchanged."""
    p = inputs.problem((8, 5, 4), 6, 2, 20.0, periodic=True)
    part = np.arange(p.mesh.n_nodes, dtype=np.int32)
    dm, J, B = device_problem(p, part)
    oj = oracle_jac(p)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 3, fnlh.FNLH_F64, sigma=p.phase)
    ref = oracle.jacobi(oj, p.mesh.vol, p.omega, p.b, 1, sigma=p.phase, part=part)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


def test_one_partition_equals_untruncated_bitwise():
    p = inputs.problem((11, 6, 4), 6, 4, 20.0)
    dm, J, B = device_problem(p, np.zeros(p.mesh.n_nodes, np.int32))
    dm0, J0, B0 = _gpu.device_problem(p)
    for prec in (fnlh.FNLH_F64, fnlh.FNLH_F32, fnlh.FNLH_BF16):
        X, X0 = torch.zeros_like(B), torch.zeros_like(B)
        fnlh.fnlh_relax(dm, J, p.omega, B, X, 7, prec)
        fnlh.fnlh_relax(dm0, J0, p.omega, B0, X0, 7, prec)
        assert torch.equal(X, X0), prec


@pytest.mark.parametrize("prec,bound", [(fnlh.FNLH_F32, 2e-5), (fnlh.FNLH_BF16, 5e-2)])
def test_truncated_low_precision_bounded(prec, bound):
    dims = (13, 6, 5)
    p = inputs.problem(dims, 6, 4, 20.0)
    part = inputs.box_partition(dims, (2, 2, 1))
    dm, J, B = device_problem(p, part)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 30, prec)
    ref = oracle.jacobi(oracle_jac(p), p.mesh.vol, p.omega, p.b, 30, part=part)
    err = _gpu.rel_err_per_system(X.cpu().numpy(), ref, p.n_harm)
    assert np.all(err <= bound), err


@pytest.mark.parametrize("prec", [fnlh.FNLH_F64, fnlh.FNLH_F32, fnlh.FNLH_BF16])
def test_partitioned_solve_reaches_full_solution(prec):
    dims = (24, 16, 12)
    p = inputs.problem(dims, 6, 8, 20.0)
    part = inputs.box_partition(dims, (4, 2, 2))
    dm, J, B = device_problem(p, part)
    X = torch.zeros_like(B)
    st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, 1e-8, 12, 80,
                                              flags=fnlh.FNLH_SOLVE_ZERO_GUESS)
    assert st == fnlh.FNLH_OK and np.all(rel <= 1e-8), (st, rel)
    true_rel = oracle.rel_residuals(oracle_jac(p), p.mesh.vol, p.omega, p.b, X.cpu().numpy())
    assert np.all(true_rel <= 1e-8), true_rel


def test_fp64_defect_correction_matches_oracle_composition():
    """tol = 0 runs exactly `checks` residuals and checks - 1 corrections."""
    dims = (10, 6, 5)
    p = inputs.problem(dims, 6, 3, 20.0)
    part = inputs.box_partition(dims, (2, 3, 1))
    dm, J, B = device_problem(p, part)
    oj = oracle_jac(p)
    _gpu.load_jacobian(dm, J, oj)
    x0 = np.random.default_rng(5).normal(size=p.b.shape)
    X = torch.from_numpy(x0.copy()).cuda()
    inner, checks = 4, 5
    st, done, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, fnlh.FNLH_F64, 0.0, inner, checks,
                                            raise_on_error=False)
    assert st == fnlh.FNLH_ERR_NOT_CONVERGED and done == checks and sweeps == inner * (checks - 1)
    x = x0.copy()
    for _ in range(checks - 1):
        _, r = oracle.residual(oj, p.mesh.vol, p.omega, p.b, x, want_r=True)
        x = x + oracle.jacobi(oj, p.mesh.vol, p.omega, r, inner, part=part)
    _gpu.assert_fp64_parity(X.cpu().numpy(), x, p.n_harm)


def test_partitioned_batched_rows_match_per_row():
    specs = [((13, 6, 5), 6, 4, (3, 2, 1)), ((9, 7, 5), 6, 2, (1, 1, 1)), ((10, 4, 6), 6, 8, (2, 1, 3))]
    dev = []
    for dims, b, N, parts in specs:
        p = inputs.problem(dims, b, N, 20.0)
        dm, J, B = device_problem(p, inputs.box_partition(dims, parts))
        dev.append((p, dm, J, B))
    singles = []
    for p, dm, J, B in dev:
        X = torch.zeros_like(B)
        fnlh.fnlh_relax(dm, J, p.omega, B, X, 9, fnlh.FNLH_F32)
        singles.append(X.cpu().numpy())
    Xs = [torch.zeros_like(B) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for (p, dm, J, B), X in zip(dev, Xs)])
    ws = torch.empty(batch.workspace_bytes(6), dtype=torch.uint8, device="cuda")
    fnlh.fnlh_relax_batched(batch, 9, fnlh.FNLH_F32, ws=ws)
    for X, ref in zip(Xs, singles):
        assert np.array_equal(X.cpu().numpy(), ref)


def test_full_size_truncated_relax_matches_oracle():
    """128x64x48, b = 6, mean + 4 harmonics, 50 FP64 sweeps (the benchmark's
    launch configuration) on 64 boxes, against the oracle over the whole mesh."""
    c = inputs.CONFIGS["c2"]
    p = inputs.config_problem("c2")
    part = inputs.box_partition(c["dims"], (4, 4, 4))
    dm, J, B = device_problem(p, part, prep_flags=fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_TAGS)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 50, fnlh.FNLH_F64)
    x = X.cpu().numpy()
    del dm, J, B, X
    ref = oracle.jacobi(oracle_jac(p), p.mesh.vol, p.omega, p.b, 50, part=part)
    _gpu.assert_fp64_parity(x, ref, p.n_harm)

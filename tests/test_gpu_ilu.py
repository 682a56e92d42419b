"""GPU parity of the block ILU(0) smoother (the paper's implicit smoother) in
multicolour order against the oracle's textbook block ILU(0).

FP64 iterations x <- x + (LU)^-1 (B - A x) match the oracle to relative 1e-12
iteration by iteration (red-black and greedy colourings, b = 5 and 6, phase-
lagged periodic passages, partitions); the FP32 factor and passes are
bounded and still reach a true FP64 residual of 1e-8; patterns the library
cannot factor exactly (triangles) and invalid colourings are rejected.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2404_01407_gb300 import fnlh, inputs
from tests import _gpu

pytestmark = pytest.mark.gpu

PREP = fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_F32 | fnlh.FNLH_PREP_TAGS


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    fnlh.lib()


def setup(p, part=None, color=None, precision=fnlh.FNLH_F64, oracle_blocks=True):
    dm = fnlh.DeviceMesh.from_mesh(p.mesh, "cuda", part=part)
    J = fnlh.DeviceJacobian(dm, p.block, PREP)
    fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).cuda(), fnlh.make_params(p.cfl), J)
    m = p.mesh
    oj = oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl, periodic=m.periodic)
    if oracle_blocks:
        _gpu.load_jacobian(dm, J, oj)
    ilu = fnlh.DeviceIlu(dm, p.block, p.n_harm, color=color, precision=precision)
    fnlh.fnlh_ilu_factor(dm, J, p.omega, ilu)
    return dm, J, torch.from_numpy(p.b).cuda(), oj, ilu


def run_iterations(dm, J, ilu, p, B, X, iters):
    """tol = 0: exactly `iters` iterations."""
    st, its, rel = fnlh.fnlh_solve_ilu(dm, J, ilu, p.omega, B, X, 0.0, iters, sigma=p.phase, raise_on_error=False)
    assert st == fnlh.FNLH_ERR_NOT_CONVERGED and its == iters, (st, its)
    return rel


@pytest.mark.parametrize("dims,block,N,greedy", [((13, 6, 5), 6, 4, False), ((7, 5, 3), 5, 3, True),
                                                 ((9, 8, 4), 6, 1, True)])
def test_ilu_iterations_match_oracle(dims, block, N, greedy):
    p = inputs.problem(dims, block, N, 20.0, 1.3)
    color = None if greedy else inputs.lattice_colors(dims)
    dm, J, B, oj, ilu = setup(p, color=color)
    x0 = np.random.default_rng(3).normal(size=p.b.shape)
    X = torch.from_numpy(x0.copy()).cuda()
    run_iterations(dm, J, ilu, p, B, X, 6)
    ref = oracle.ilu_iterate(oj, p.mesh.vol, p.omega, p.b, 6, ilu.color_host, X0=x0)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


def test_ilu_periodic_passage_matches_oracle():
    p = inputs.problem((8, 6, 4), 6, 3, 20.0, periodic=True)
    dm, J, B, oj, ilu = setup(p, color=inputs.lattice_colors((8, 6, 4)))
    X = torch.zeros_like(B)
    run_iterations(dm, J, ilu, p, B, X, 5)
    ref = oracle.ilu_iterate(oj, p.mesh.vol, p.omega, p.b, 5, ilu.color_host, sigma=p.phase)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


def test_ilu_odd_pitch_greedy_colouring_matches_oracle():
    """An odd pitch closes odd cycles: the greedy colouring needs more than two colours."""
    p = inputs.problem((6, 5, 3), 5, 2, 15.0, periodic=True)
    dm, J, B, oj, ilu = setup(p)
    assert ilu.n_colors >= 3
    X = torch.zeros_like(B)
    run_iterations(dm, J, ilu, p, B, X, 4)
    ref = oracle.ilu_iterate(oj, p.mesh.vol, p.omega, p.b, 4, ilu.color_host, sigma=p.phase)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


def test_ilu_partitioned_matches_oracle():
    dims = (12, 6, 5)
    p = inputs.problem(dims, 6, 2, 20.0)
    part = inputs.box_partition(dims, (3, 2, 1))
    dm, J, B, oj, ilu = setup(p, part=part, color=inputs.lattice_colors(dims))
    X = torch.zeros_like(B)
    run_iterations(dm, J, ilu, p, B, X, 5)
    ref = oracle.ilu_iterate(oj, p.mesh.vol, p.omega, p.b, 5, ilu.color_host, part=part)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


@pytest.mark.parametrize("precision", [fnlh.FNLH_F64, fnlh.FNLH_F32])
def test_ilu_solve_reaches_1e8(precision):
    p = inputs.problem((24, 16, 12), 6, 8, 20.0)
    dm, J, B, oj, ilu = setup(p, precision=precision, oracle_blocks=False)
    X = torch.zeros_like(B)
    st, its, rel = fnlh.fnlh_solve_ilu(dm, J, ilu, p.omega, B, X, 1e-8, 100, flags=fnlh.FNLH_SOLVE_ZERO_GUESS)
    assert st == fnlh.FNLH_OK and np.all(rel <= 1e-8), (st, rel)
    true_rel = oracle.rel_residuals(oj, p.mesh.vol, p.omega, p.b, X.cpu().numpy())
    assert np.all(true_rel <= 1e-8), true_rel


def test_ilu_f32_iterations_bounded():
    p = inputs.problem((13, 6, 5), 6, 4, 20.0)
    dm, J, B, oj, ilu = setup(p, color=inputs.lattice_colors((13, 6, 5)), precision=fnlh.FNLH_F32)
    X = torch.zeros_like(B)
    run_iterations(dm, J, ilu, p, B, X, 4)
    ref = oracle.ilu_iterate(oj, p.mesh.vol, p.omega, p.b, 4, ilu.color_host)
    err = _gpu.rel_err_per_system(X.cpu().numpy(), ref, p.n_harm)
    assert np.all(err <= 1e-5), err


def test_ilu_paper_rule_and_masking():
    """The paper's stage rule from zero (1e-2 drop, at most 10 iterations):
    ILU(0) meets it in fewer iterations than Jacobi needs sweeps."""
    p = inputs.problem((24, 16, 12), 6, 4, 20.0)
    dm, J, B, oj, ilu = setup(p, oracle_blocks=False)
    X = torch.zeros_like(B)
    flags = fnlh.FNLH_SOLVE_ZERO_GUESS | fnlh.FNLH_SOLVE_MASK_CONVERGED
    st, its, rel = fnlh.fnlh_solve_ilu(dm, J, ilu, p.omega, B, X, 1e-2, 10, flags=flags)
    assert st == fnlh.FNLH_OK and np.all(rel <= 1e-2)
    Xj = torch.zeros_like(B)
    st_j, checks, sweeps, rel_j = fnlh.fnlh_solve(dm, J, p.omega, B, Xj, fnlh.FNLH_F64, 1e-2, 1, 40,
                                                  flags=fnlh.FNLH_SOLVE_ZERO_GUESS)
    assert its < sweeps, (its, sweeps)
    true_rel = oracle.rel_residuals(oj, p.mesh.vol, p.omega, p.b, X.cpu().numpy())
    assert np.all(true_rel <= 1e-2)


def test_ilu_rejects_triangles_and_bad_colourings():
    base = inputs.hex_mesh(4, 3, 2, seed=31)
    extra = np.array([[0, 5]], dtype=np.int32)  # a diagonal: triangles 0-1-5 and 0-4-5
    mesh = inputs.custom_mesh(base.positions, np.concatenate([base.edge_nodes, extra]), vol=base.vol)
    p = inputs.Problem(mesh, inputs.flow_state(mesh.n_nodes, 5), inputs.rhs(mesh.n_nodes, 5, 1),
                       inputs.omegas(1), 5, 10.0)
    dm = fnlh.DeviceMesh.from_mesh(mesh)
    J = fnlh.DeviceJacobian(dm, 5, fnlh.FNLH_PREP_F64)
    fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).cuda(), fnlh.make_params(10.0), J)
    ilu = fnlh.DeviceIlu(dm, 5, 1)
    with pytest.raises(fnlh.FnlhError) as e:
        fnlh.fnlh_ilu_factor(dm, J, p.omega, ilu)
    assert e.value.status == fnlh.FNLH_ERR_UNSUPPORTED
    # a colouring with neighbours of one colour
    q = inputs.problem((5, 4, 3), 5, 1, 10.0)
    dmq = fnlh.DeviceMesh.from_mesh(q.mesh)
    Jq = fnlh.DeviceJacobian(dmq, 5, fnlh.FNLH_PREP_F64)
    fnlh.fnlh_build_jacobian(dmq, torch.from_numpy(q.q).cuda(), fnlh.make_params(10.0), Jq)
    bad = fnlh.DeviceIlu(dmq, 5, 1, color=np.zeros(q.mesh.n_nodes, np.int32))
    with pytest.raises(fnlh.FnlhError) as e:
        fnlh.fnlh_ilu_factor(dmq, Jq, q.omega, bad)
    assert e.value.status == fnlh.FNLH_ERR_BAD_MESH
    # the same mesh with its diagonal cut by a partition boundary factors fine
    part = np.zeros(mesh.n_nodes, np.int32)
    part[5] = 1
    dmp = fnlh.DeviceMesh.from_mesh(mesh, part=part)
    Jp = fnlh.DeviceJacobian(dmp, 5, fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_TAGS)
    fnlh.fnlh_build_jacobian(dmp, torch.from_numpy(p.q).cuda(), fnlh.make_params(10.0), Jp)
    okilu = fnlh.DeviceIlu(dmp, 5, 1)
    fnlh.fnlh_ilu_factor(dmp, Jp, p.omega, okilu)


def test_ilu_larger_passage_matches_oracle():
    """64x48x32 (98,304 nodes), b = 6, mean + 4 harmonics, 3 FP64 iterations."""
    dims = (64, 48, 32)
    p = inputs.problem(dims, 6, 4, 20.0)
    dm, J, B, oj, ilu = setup(p, oracle_blocks=False)
    X = torch.zeros_like(B)
    run_iterations(dm, J, ilu, p, B, X, 3)
    ref = oracle.ilu_iterate(oj, p.mesh.vol, p.omega, p.b, 3, ilu.color_host)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


def test_ilu_f32_float_float_checks():
    """FP32 factor with FNLH_PREP_FF: the residual of every iteration after
    the first is float-float (the one that ends the solve FP64), so the solve
    takes the same iterations as with FP64 residuals, its corrections agree to
    rounding, and the oracle certifies the 1e-8."""
    p = inputs.problem((24, 16, 12), 6, 4, 20.0)
    m = p.mesh
    out = {}
    for ff in (False, True):
        dm = fnlh.DeviceMesh.from_mesh(m, "cuda")
        J = fnlh.DeviceJacobian(dm, p.block, PREP | (fnlh.FNLH_PREP_FF if ff else 0))
        fnlh.fnlh_build_jacobian(dm, torch.from_numpy(p.q).cuda(), fnlh.make_params(p.cfl), J)
        ilu = fnlh.DeviceIlu(dm, p.block, p.n_harm, precision=fnlh.FNLH_F32)
        fnlh.fnlh_ilu_factor(dm, J, p.omega, ilu)
        B = torch.from_numpy(p.b).cuda()
        X = torch.zeros_like(B)
        st, its, rel = fnlh.fnlh_solve_ilu(dm, J, ilu, p.omega, B, X, 1e-8, 100, flags=fnlh.FNLH_SOLVE_ZERO_GUESS)
        assert st == fnlh.FNLH_OK and np.all(rel <= 1e-8), (ff, st, rel)
        out[ff] = (its, X.cpu().numpy())
    assert out[True][0] == out[False][0]
    oj = oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl)
    true_rel = oracle.rel_residuals(oj, m.vol, p.omega, p.b, out[True][1])
    assert np.all(true_rel <= 1e-8), true_rel
    # the two runs differ only in the rounding of the intermediate residuals
    err = _gpu.rel_err_per_system(out[True][1], out[False][1], p.n_harm)
    assert np.all(err <= 1e-6), err

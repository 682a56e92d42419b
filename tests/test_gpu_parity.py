"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: the FP64 path must match the oracle to relative 1e-12 per system
(the target the measurement plan states); the Jacobian build to 1e-13 of the
largest block entry.  The low-precision sweeps are approximations and are
bounded loosely; the mixed solve must reach a true FP64 relative residual of
1e-8 (checked with the oracle's residual on the returned x).
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2404_01407_gb300 import fnlh, inputs
from tests import _gpu

pytestmark = pytest.mark.gpu

SMALL = {
    # ragged sizes: several 256-thread tiles plus a tail
    "c1": dict(dims=(16, 8, 8), block=5, n_harm=1, cfl=10.0),
    "b6n4": dict(dims=(20, 12, 10), block=6, n_harm=4, cfl=20.0),
    "b5n3_ragged": dict(dims=(7, 5, 3), block=5, n_harm=3, cfl=15.0),
    "b6n0_mean_only": dict(dims=(9, 7, 5), block=6, n_harm=0, cfl=20.0),
}


def small(key, **kw):
    c = dict(SMALL[key])
    c.update(kw)
    return inputs.problem(c["dims"], c["block"], c["n_harm"], c["cfl"], c.get("omega_base", 1.0), name=key)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    fnlh.lib()


@pytest.mark.parametrize("key", sorted(SMALL))
@pytest.mark.parametrize("pseudo", [0, 1])
def test_build_jacobian_matches_oracle(key, pseudo):
    p = small(key)
    dm, J, B = _gpu.device_problem(p, pseudo_time=pseudo)
    oj = _gpu.oracle_jacobian(p, pseudo_time=pseudo)
    offd = J.offd.cpu().numpy()
    diag = J.diag.cpu().numpy()
    scale = max(np.abs(oj.offd).max(), np.abs(oj.diag).max())
    assert np.abs(offd - oj.offd).max() <= 1e-13 * scale
    assert np.abs(diag - oj.diag).max() <= 1e-13 * scale
    assert np.allclose(J.D.cpu().numpy(), oj.D, rtol=1e-14, atol=0)


@pytest.mark.parametrize("key", sorted(SMALL))
def test_relax_f64_isolated_sweep(key):
    """Oracle J fed to the GPU: only the sweep differs."""
    p = small(key)
    dm, J, B = _gpu.device_problem(p)
    oj = _gpu.oracle_jacobian(p)
    _gpu.load_jacobian(dm, J, oj)
    x0 = np.random.default_rng(7).normal(size=p.b.shape)
    X = torch.from_numpy(x0.copy()).cuda()
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 20, fnlh.FNLH_F64)
    ref = oracle.jacobi(oj, p.mesh.vol, p.omega, p.b, 20, X0=x0)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


@pytest.mark.parametrize("key", sorted(SMALL))
def test_relax_f64_end_to_end(key):
    p = small(key)
    dm, J, B = _gpu.device_problem(p)
    oj = _gpu.oracle_jacobian(p)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 50, fnlh.FNLH_F64)
    ref = oracle.jacobi(oj, p.mesh.vol, p.omega, p.b, 50)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


def test_relax_f64_config2_full_size():
    """128x64x48, b = 6, mean + 4 harmonics, CFL 20, 50 sweeps: the benchmark's
    launch configuration, compared with the oracle over the whole mesh."""
    p = inputs.config_problem("c2")
    dm, J, B = _gpu.device_problem(p, prep_flags=fnlh.FNLH_PREP_F64)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 50, fnlh.FNLH_F64)
    oj = _gpu.oracle_jacobian(p)
    ref = oracle.jacobi(oj, p.mesh.vol, p.omega, p.b, 50)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)
    # the build at full size too, sampled rows
    rows = np.random.default_rng(0).choice(p.mesh.n_nodes, 2000, replace=False)
    scale = np.abs(oj.diag).max()
    assert np.abs(J.diag.cpu().numpy()[rows] - oj.diag[rows]).max() <= 1e-13 * scale


@pytest.mark.parametrize("key", ["c1", "b6n4", "b6n0_mean_only"])
def test_residual_matches_oracle(key):
    p = small(key)
    dm, J, B = _gpu.device_problem(p)
    oj = _gpu.oracle_jacobian(p)
    _gpu.load_jacobian(dm, J, oj)
    x = np.random.default_rng(3).normal(size=p.b.shape)
    X = torch.from_numpy(x).cuda()
    r = torch.empty_like(B)
    norms = fnlh.fnlh_residual(dm, J, p.omega, B, X, r=r).cpu().numpy()
    on, orr = oracle.residual(oj, p.mesh.vol, p.omega, p.b, x, want_r=True)
    assert np.abs(r.cpu().numpy() - orr).max() <= 1e-13 * np.abs(orr).max()
    assert np.allclose(norms, on, rtol=1e-12, atol=0)
    # fixed-order reduction: identical bits on a repeat
    norms2 = fnlh.fnlh_residual(dm, J, p.omega, B, X).cpu().numpy()
    assert np.array_equal(norms, norms2)


@pytest.mark.parametrize("prec,bound", [(fnlh.FNLH_F32, 2e-5), (fnlh.FNLH_BF16, 5e-2)])
def test_relax_low_precision_bounded(prec, bound):
    p = small("b6n4")
    dm, J, B = _gpu.device_problem(p)
    oj = _gpu.oracle_jacobian(p)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 30, prec)
    ref = oracle.jacobi(oj, p.mesh.vol, p.omega, p.b, 30)
    err = _gpu.rel_err_per_system(X.cpu().numpy(), ref, p.n_harm)
    assert np.all(err <= bound), err


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_BF16])
@pytest.mark.parametrize("zero_guess", [False, True])
def test_mixed_solve_reaches_1e8(prec, zero_guess):
    """Defect correction: FP64 residual, low-precision inner sweeps, FP64 update.
    With FNLH_SOLVE_ZERO_GUESS the incoming X (garbage here) is ignored."""
    p = inputs.problem((32, 24, 16), 6, 8, 20.0, name="c3_reduced")
    dm, J, B = _gpu.device_problem(p)
    X = torch.full_like(B, 1e30) if zero_guess else torch.zeros_like(B)
    flags = fnlh.FNLH_SOLVE_ZERO_GUESS if zero_guess else 0
    st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, 1e-8, 12, 40, flags=flags)
    assert st == fnlh.FNLH_OK and np.all(rel <= 1e-8), (st, rel)
    oj = _gpu.oracle_jacobian(p)
    x = X.cpu().numpy()
    true_rel = oracle.rel_residuals(oj, p.mesh.vol, p.omega, p.b, x)
    assert np.all(true_rel <= 1e-8), true_rel
    xs, _ = oracle.solve_to_tol(oj, p.mesh.vol, p.omega, p.b, tol=1e-13, chunk=25)
    err = _gpu.rel_err_per_system(x, xs, p.n_harm)
    assert np.all(err <= 1e-6), err


@pytest.mark.parametrize("zero_guess", [False, True])
def test_plain_f64_solve_matches_oracle(zero_guess):
    p = small("b6n4")
    dm, J, B = _gpu.device_problem(p)
    X = torch.full_like(B, -3.0) if zero_guess else torch.zeros_like(B)
    flags = fnlh.FNLH_SOLVE_ZERO_GUESS if zero_guess else 0
    st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, fnlh.FNLH_F64, 1e-10, 10, 100, flags=flags)
    assert st == fnlh.FNLH_OK and np.all(rel <= 1e-10)
    oj = _gpu.oracle_jacobian(p)
    ref = oracle.jacobi(oj, p.mesh.vol, p.omega, p.b, sweeps)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


def test_batched_rows_match_per_row():
    rows = [inputs.problem((9, 7, 5), 6, 2, 20.0, 1.0, seeds=(1, 2, 3)),
            inputs.problem((12, 8, 6), 6, 8, 20.0, 1.6, seeds=(4, 5, 6)),
            inputs.problem((10, 9, 7), 6, 4, 20.0, 2.3, seeds=(7, 8, 9))]
    dev = []
    for p in rows:
        dm, J, B = _gpu.device_problem(p)
        dev.append((p, dm, J, B))
    singles = []
    for p, dm, J, B in dev:
        X = torch.zeros_like(B)
        fnlh.fnlh_relax(dm, J, p.omega, B, X, 13, fnlh.FNLH_F32)
        singles.append(X.cpu().numpy())
    Xs = [torch.zeros_like(B) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for (p, dm, J, B), X in zip(dev, Xs)])
    ws = torch.empty(batch.workspace_bytes(6), dtype=torch.uint8, device="cuda")
    for tn in (None, fnlh.fnlh_tuning(128, 2), fnlh.fnlh_tuning(256, 0),
               fnlh.fnlh_tuning(0, fnlh.FNLH_TUNING_PER_ROW)):
        for X in Xs:
            X.zero_()
        fnlh.fnlh_relax_batched(batch, 13, fnlh.FNLH_F32, tuning=tn, ws=ws)
        for X, ref in zip(Xs, singles):
            assert np.array_equal(X.cpu().numpy(), ref)


def test_single_node_one_sweep_is_exact_block_solve():
    """No edges: one sweep is the exact shifted block solve (numpy)."""
    rng = np.random.default_rng(4)
    mesh = inputs.custom_mesh(np.zeros((1, 3)), np.zeros((0, 2)), vol=[1.7])
    dm = fnlh.DeviceMesh.from_mesh(mesh)
    J = fnlh.DeviceJacobian(dm, 6, _gpu.ALL_PREP)
    P = rng.normal(size=(6, 6)) + 4 * np.eye(6)
    J.diag.copy_(torch.from_numpy(P[None]))
    J.D.fill_(0.3)
    fnlh.fnlh_prepare(dm, J)
    om = np.array([0.7, 2.0])
    b = rng.normal(size=(1, 5, 6))
    B = torch.from_numpy(b).cuda()
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, om, B, X, 1, fnlh.FNLH_F64)
    x = X.cpu().numpy()
    ref0 = np.linalg.solve(P + 0.3 * np.eye(6), b[0, 0])
    assert np.allclose(x[0, 0], ref0, rtol=1e-13, atol=1e-14)
    for k in (1, 2):
        M = P + (0.3 + 1j * om[k - 1] * 1.7) * np.eye(6)
        y = np.linalg.solve(M, b[0, 2 * k - 1] + 1j * b[0, 2 * k])
        assert np.allclose(x[0, 2 * k - 1] + 1j * x[0, 2 * k], y, rtol=1e-13, atol=1e-14)


def test_empty_mesh_is_a_no_op():
    mesh = inputs.custom_mesh(np.zeros((0, 3)), np.zeros((0, 2)), vol=np.zeros(0))
    dm = fnlh.DeviceMesh.from_mesh(mesh)
    J = fnlh.DeviceJacobian(dm, 5, _gpu.ALL_PREP)
    fnlh.fnlh_build_jacobian(dm, torch.zeros((0, 5), dtype=torch.float64, device="cuda"), fnlh.make_params(10.0), J)
    B = torch.zeros((0, 3, 5), dtype=torch.float64, device="cuda")
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, [1.0], B, X, 3, fnlh.FNLH_F64)
    norms = fnlh.fnlh_residual(dm, J, [1.0], B, X).cpu().numpy()
    assert np.all(norms == 0.0)


def test_max_harmonics_and_permuted_numbering():
    base = inputs.problem((6, 5, 4), 6, 64, 20.0, 0.25)
    mesh, perm = inputs.permute_mesh(base.mesh, seed=4)
    p = inputs.Problem(mesh=mesh, q=base.q[perm], b=base.b[perm], omega=base.omega, block=6, cfl=20.0)
    dm, J, B = _gpu.device_problem(p)
    oj = _gpu.oracle_jacobian(p)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 25, fnlh.FNLH_F64)
    ref = oracle.jacobi(oj, p.mesh.vol, p.omega, p.b, 25)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


def test_nonfinite_rhs_is_reported():
    p = small("c1")
    dm, J, B = _gpu.device_problem(p)
    B[3, 1, 2] = float("nan")
    X = torch.zeros_like(B)
    st, *_ = fnlh.fnlh_solve(dm, J, p.omega, B, X, fnlh.FNLH_F32, 1e-8, 5, 5, raise_on_error=False)
    assert st == fnlh.FNLH_ERR_NONFINITE


def test_missing_precision_copy_is_reported():
    p = small("c1")
    dm, J, B = _gpu.device_problem(p, prep_flags=fnlh.FNLH_PREP_F64)
    X = torch.zeros_like(B)
    with pytest.raises(fnlh.FnlhError) as e:
        fnlh.fnlh_relax(dm, J, p.omega, B, X, 2, fnlh.FNLH_BF16)
    assert e.value.status == fnlh.FNLH_ERR_WORKSPACE


@pytest.mark.parametrize("prec", [fnlh.FNLH_F64, fnlh.FNLH_F32])
def test_complex_spectrum_block_uses_hessenberg_fallback(prec):
    """Diagonal blocks whose spectrum has a complex pair keep the Hessenberg
    form; one sweep from zero must still be the exact shifted block solve."""
    rng = np.random.default_rng(8)
    mesh = inputs.custom_mesh(np.zeros((2, 3)), np.zeros((0, 2)), vol=[1.3, 0.7])
    dm = fnlh.DeviceMesh.from_mesh(mesh)
    J = fnlh.DeviceJacobian(dm, 6, _gpu.ALL_PREP)
    Ps = []
    for node in range(2):
        V = rng.normal(size=(6, 6)) + 3 * np.eye(6)
        Dm = np.diag(rng.uniform(2, 4, 6))
        if node == 0:
            Dm[1:3, 1:3] = [[2.5, 1.5], [-1.5, 2.5]]  # eigenvalues 2.5 +- 1.5i
        Ps.append(V @ Dm @ np.linalg.inv(V))
    J.diag.copy_(torch.from_numpy(np.stack(Ps)))
    J.D.zero_()
    fnlh.fnlh_prepare(dm, J)
    om = np.array([0.9, 2.2, 3.1])
    b = rng.normal(size=(2, 7, 6))
    B = torch.from_numpy(b).cuda()
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, om, B, X, 1, prec)
    x = X.cpu().numpy()
    tol = 1e-12 if prec == fnlh.FNLH_F64 else 1e-5
    for node in range(2):
        ref0 = np.linalg.solve(Ps[node], b[node, 0])
        assert np.linalg.norm(x[node, 0] - ref0) <= tol * np.linalg.norm(ref0)
        for k in (1, 2, 3):
            M = Ps[node] + 1j * om[k - 1] * mesh.vol[node] * np.eye(6)
            y = np.linalg.solve(M, b[node, 2 * k - 1] + 1j * b[node, 2 * k])
            got = x[node, 2 * k - 1] + 1j * x[node, 2 * k]
            assert np.linalg.norm(got - y) <= tol * np.linalg.norm(y)


def test_relax_f64_block_pseudo_time_matches_oracle():
    """Eq. precon's block pseudo-time form (D = 0, J_ii scaled by 1 + 1/(eps CFL))."""
    p = small("b6n4")
    dm, J, B = _gpu.device_problem(p, pseudo_time=1)
    oj = _gpu.oracle_jacobian(p, pseudo_time=1)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 30, fnlh.FNLH_F64)
    ref = oracle.jacobi(oj, p.mesh.vol, p.omega, p.b, 30)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


def test_zero_sweeps_round_trips_the_basis():
    p = small("b6n4")
    dm, J, B = _gpu.device_problem(p)
    x = np.random.default_rng(2).normal(size=p.b.shape)
    X = torch.from_numpy(x.copy()).cuda()
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 0, fnlh.FNLH_F64)
    assert np.abs(X.cpu().numpy() - x).max() <= 1e-14 * np.abs(x).max()


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_BF16])
@pytest.mark.parametrize("ff", [False, True])
def test_mixed_solve_b5_and_permuted_numbering(prec, ff):
    """Euler blocks (b = 5) on a randomly renumbered mesh; ff: float-float
    intermediate checks (the b = 5 form of the float-float residual)."""
    base = inputs.problem((14, 10, 8), 5, 3, 10.0, 1.3)
    mesh, perm = inputs.permute_mesh(base.mesh, seed=4)
    p = inputs.Problem(mesh=mesh, q=base.q[perm], b=base.b[perm], omega=base.omega, block=5, cfl=10.0)
    dm, J, B = _gpu.device_problem(p, prep_flags=_gpu.ALL_PREP | (fnlh.FNLH_PREP_FF if ff else 0))
    X = torch.empty_like(B)
    st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, 1e-8, 12, 40,
                                              flags=fnlh.FNLH_SOLVE_ZERO_GUESS)
    assert st == fnlh.FNLH_OK
    oj = _gpu.oracle_jacobian(p)
    true_rel = oracle.rel_residuals(oj, p.mesh.vol, p.omega, p.b, X.cpu().numpy())
    assert np.all(true_rel <= 1e-8), true_rel


def test_mixed_solve_many_harmonics():
    """64 harmonics (the largest count): the FP32 stage layout for K = 65."""
    p = inputs.problem((8, 6, 5), 6, 64, 20.0, 0.2)
    dm, J, B = _gpu.device_problem(p)
    X = torch.empty_like(B)
    st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, fnlh.FNLH_F32, 1e-8, 20, 40,
                                              flags=fnlh.FNLH_SOLVE_ZERO_GUESS)
    assert st == fnlh.FNLH_OK
    oj = _gpu.oracle_jacobian(p)
    true_rel = oracle.rel_residuals(oj, p.mesh.vol, p.omega, p.b, X.cpu().numpy())
    assert np.all(true_rel <= 1e-8), true_rel.max()


def test_solve_reports_not_converged():
    p = small("b6n4")
    dm, J, B = _gpu.device_problem(p)
    X = torch.zeros_like(B)
    st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, fnlh.FNLH_F64, 1e-12, 2, 3,
                                              raise_on_error=False)
    assert st == fnlh.FNLH_ERR_NOT_CONVERGED and checks == 3 and sweeps == 4
    assert np.all(rel > 1e-12) and np.all(rel < 1.0)


@pytest.mark.parametrize("prec", [fnlh.FNLH_BF16, fnlh.FNLH_F64])
def test_batched_rows_other_precisions(prec):
    rows = [inputs.problem((9, 7, 5), 6, 2, 20.0, 1.0, seeds=(1, 2, 3)),
            inputs.problem((12, 8, 6), 6, 8, 20.0, 1.6, seeds=(4, 5, 6))]
    dev = [(p, *_gpu.device_problem(p)) for p in rows]
    singles = []
    for p, dm, J, B in dev:
        X = torch.zeros_like(B)
        fnlh.fnlh_relax(dm, J, p.omega, B, X, 9, prec)
        singles.append(X.cpu().numpy())
    Xs = [torch.zeros_like(B) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X) for (p, dm, J, B), X in zip(dev, Xs)])
    ws = torch.empty(batch.workspace_bytes(6), dtype=torch.uint8, device="cuda")
    fnlh.fnlh_relax_batched(batch, 9, prec, tuning=fnlh.fnlh_tuning(256, 0), ws=ws)
    for X, ref, (p, *_rest) in zip(Xs, singles, dev):
        if prec == fnlh.FNLH_F64:
            # the single-row FP64 kernel solves the mean flow with a real-only path
            _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm, tol=1e-13)
        else:
            assert np.array_equal(X.cpu().numpy(), ref)


def test_literal_reading_shift_by_D():
    """The literal reading of the spectral term, i omega D instead of i omega V:
    the per-node scalar of the shift is the mesh's `vol` array, so passing D
    there gives it; the Jacobian build does not read `vol`."""
    p = small("b6n4")
    oj = _gpu.oracle_jacobian(p)
    mesh_d = inputs.Mesh(p.mesh.dims, p.mesh.positions, p.mesh.edge_nodes, p.mesh.normals, oj.D.copy())
    pd = inputs.Problem(mesh_d, p.q, p.b, p.omega, p.block, p.cfl)
    dm, J, B = _gpu.device_problem(pd)
    assert np.allclose(J.D.cpu().numpy(), oj.D, rtol=1e-14, atol=0)  # same build with vol replaced
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 30, fnlh.FNLH_F64)
    ref = oracle.jacobi(oj, oj.D, p.omega, p.b, 30)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)
    # and the max-norm view of the same comparison
    x = X.cpu().numpy()
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


def test_relax_and_residual_capture_in_a_cuda_graph():
    """fnlh_relax and fnlh_residual are asynchronous and allocate nothing: a
    captured graph replays them with the same result as direct calls."""
    p = small("b6n4")
    dm, J, B = _gpu.device_problem(p)
    ws = fnlh.workspace(p.mesh.n_nodes, p.block, p.n_harm, "cuda")
    X_direct = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X_direct, 12, fnlh.FNLH_F32, ws)
    n_direct = fnlh.fnlh_residual(dm, J, p.omega, B, X_direct, ws=ws).clone()
    X = torch.zeros_like(B)
    norms = torch.empty((1 + p.n_harm, 2), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside the capture (kernel attributes, lazy loading)
        fnlh.fnlh_relax(dm, J, p.omega, B, X, 12, fnlh.FNLH_F32, ws, stream=s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            fnlh.fnlh_relax(dm, J, p.omega, B, X, 12, fnlh.FNLH_F32, ws, stream=s)
            fnlh.fnlh_residual(dm, J, p.omega, B, X, norms=norms, ws=ws, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    X.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(X, X_direct)
    assert torch.equal(norms, n_direct)


def test_frozen_turbulence_pattern_is_certified_and_optional():
    """b = 6: the build's blocks have the frozen-turbulence zeros, fnlh_prepare
    certifies them and the FP64 kernels skip them; a Jacobian without the
    pattern is relaxed densely, both at 1e-12 of the oracle.  b = 5 has no
    pattern."""
    p = small("b6n4")
    dm, J, B = _gpu.device_problem(p)
    assert fnlh.fnlh_prep_structured(J)
    oj = _gpu.oracle_jacobian(p)
    # one off-diagonal block couples a mean-flow row to the turbulence variable
    oj.offd[3][0, 5] = 0.05 * np.abs(oj.offd[3]).max()
    _gpu.load_jacobian(dm, J, oj)
    assert not fnlh.fnlh_prep_structured(J)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 25, fnlh.FNLH_F64)
    ref = oracle.jacobi(oj, p.mesh.vol, p.omega, p.b, 25)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)
    x = np.random.default_rng(2).normal(size=p.b.shape)
    norms = fnlh.fnlh_residual(dm, J, p.omega, B, torch.from_numpy(x).cuda()).cpu().numpy()
    on, _ = oracle.residual(oj, p.mesh.vol, p.omega, p.b, x)
    assert np.allclose(norms, on, rtol=1e-12, atol=0)
    d5, J5, _ = _gpu.device_problem(small("c1"))
    assert not fnlh.fnlh_prep_structured(J5)


def _growing_problem(n_harm=1):
    """Host-made divergence: a chain of three nodes whose off-diagonal blocks
    are three times the identity against identity diagonal blocks, so the
    block-Jacobi iteration matrix has eigenvalues of modulus up to 3 sqrt(2)
    (the shift i omega V only divides them by |1 + i omega V|)."""
    mesh = inputs.custom_mesh(np.array([[0.0, 0, 0], [1, 0, 0], [2, 0, 0]]), np.array([[0, 1], [1, 2]]),
                              vol=[1.0, 1.0, 1.0])
    dm = fnlh.DeviceMesh.from_mesh(mesh)
    J = fnlh.DeviceJacobian(dm, 6, _gpu.ALL_PREP)
    J.offd.copy_(torch.from_numpy(np.tile(3.0 * np.eye(6), (4, 1, 1))))
    J.diag.copy_(torch.from_numpy(np.tile(np.eye(6), (3, 1, 1))))
    J.D.zero_()
    fnlh.fnlh_prepare(dm, J)
    b = np.random.default_rng(11).normal(size=(3, 1 + 2 * n_harm, 6))
    return dm, J, torch.from_numpy(b).cuda(), np.full(n_harm, 0.5)


@pytest.mark.parametrize("prec", [fnlh.FNLH_F64, fnlh.FNLH_F32, fnlh.FNLH_BF16])
def test_growing_iteration_is_reported_as_diverged(prec):
    """The solve stops with FNLH_ERR_DIVERGED once the residual has grown
    1e3-fold over the first check, instead of running to its check limit;
    the batched solve does the same for a batch holding that row."""
    dm, J, B, om = _growing_problem()
    X = torch.zeros_like(B)
    st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, om, B, X, prec, 1e-8, 10, 50, raise_on_error=False)
    assert st == fnlh.FNLH_ERR_DIVERGED, st
    assert checks <= 3 and np.max(rel) > 1e3
    Xb = torch.zeros_like(B)
    batch = fnlh.BatchedRows([(dm, J, om, B, Xb)])
    ws = torch.empty(batch.workspace_bytes(6, prec), dtype=torch.uint8, device="cuda")
    st, checks, sweeps, rel = fnlh.fnlh_solve_batched(batch, prec, 1e-8, 10, 50, ws=ws, raise_on_error=False)
    assert st == fnlh.FNLH_ERR_DIVERGED, st
    assert checks <= 3


FF_PREP = _gpu.ALL_PREP | fnlh.FNLH_PREP_FF


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_BF16])
def test_float_float_check_matches_fp64_check(prec):
    """The float-float residual of a check agrees with the FP64 residual of
    the same x: two checks with tol = 0 (never converged), so both runs make
    the same first correction from the same FP64 first check, and the second
    check -- float-float with FNLH_PREP_FF and the solve workspace, FP64
    without -- measures the same x."""
    p = inputs.problem((32, 24, 16), 6, 8, 20.0, name="c3_reduced")
    dm, J, B = _gpu.device_problem(p, prep_flags=FF_PREP)
    n = p.mesh.n_nodes
    X1, X2 = torch.zeros_like(B), torch.zeros_like(B)
    ws_ff = fnlh.solve_workspace(n, 6, p.n_harm, FF_PREP, "cuda", prec)
    ws_64 = fnlh.workspace(n, 6, p.n_harm, "cuda", prec)
    assert ws_ff.numel() > ws_64.numel()
    zg = fnlh.FNLH_SOLVE_ZERO_GUESS
    st1, c1, s1, rel_ff = fnlh.fnlh_solve(dm, J, p.omega, B, X1, prec, 0.0, 12, 2, ws=ws_ff, flags=zg,
                                          raise_on_error=False)
    st2, c2, s2, rel_64 = fnlh.fnlh_solve(dm, J, p.omega, B, X2, prec, 0.0, 12, 2, ws=ws_64, flags=zg,
                                          raise_on_error=False)
    assert st1 == st2 == fnlh.FNLH_ERR_NOT_CONVERGED and c1 == c2 == 2 and s1 == s2 == 12
    assert torch.equal(X1, X2)
    assert np.all(rel_64 < 1e-2) and np.all(rel_64 > 1e-9)
    assert np.allclose(rel_ff, rel_64, rtol=1e-6, atol=0), (rel_ff, rel_64)


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_BF16])
def test_float_float_checks_certified_solve(prec):
    """A mixed solve with float-float checks converges in FP64 terms: the
    oracle's residual of the returned x is at most 1e-8 per system, the
    residual it reports (the confirming FP64 check) agrees with the oracle's,
    and the solution is the FP64-checked solve's to 1e-6."""
    p = inputs.problem((32, 24, 16), 6, 8, 20.0, name="c3_reduced")
    dm, J, B = _gpu.device_problem(p, prep_flags=FF_PREP)
    n = p.mesh.n_nodes
    X = torch.empty_like(B)
    Xr = torch.empty_like(B)
    ws_ff = fnlh.solve_workspace(n, 6, p.n_harm, FF_PREP, "cuda", prec)
    ws_64 = fnlh.workspace(n, 6, p.n_harm, "cuda", prec)
    zg = fnlh.FNLH_SOLVE_ZERO_GUESS
    st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, 1e-8, 12, 40, ws=ws_ff, flags=zg)
    st2, checks2, sweeps2, rel2 = fnlh.fnlh_solve(dm, J, p.omega, B, Xr, prec, 1e-8, 12, 40, ws=ws_64, flags=zg)
    assert st == st2 == fnlh.FNLH_OK and np.all(rel <= 1e-8)
    assert sweeps == sweeps2
    oj = _gpu.oracle_jacobian(p)
    x = X.cpu().numpy()
    true_rel = oracle.rel_residuals(oj, p.mesh.vol, p.omega, p.b, x)
    assert np.all(true_rel <= 1e-8), true_rel
    assert np.allclose(rel, true_rel, rtol=1e-6, atol=1e-12)
    err = _gpu.rel_err_per_system(x, Xr.cpu().numpy(), p.n_harm)
    assert np.all(err <= 1e-6), err

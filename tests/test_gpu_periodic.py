"""GPU parity of phase-lagged periodic edges (Eq. lhs_lin: the inter-blade
phase angle sigma_l makes every harmonic's LHS different while J stays
shared).  Across a periodic edge harmonic l couples J_ij e^{+-i sigma_l} x_j;
the mean flow carries no phase.

FP64 sweeps and the residual match the oracle to relative 1e-12; the
low-precision sweeps are bounded like their non-periodic counterparts; the
mixed solve reaches a true FP64 residual of 1e-8 measured by the oracle.  At
the full 128x64x48 size the passage is also checked against the property
that fixes phase lag: a ring of P passages with plain periodicity and a
right-hand side advancing by e^{i sigma} per passage gives the same iterate.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2404_01407_gb300 import fnlh, inputs
from tests import _gpu

pytestmark = pytest.mark.gpu

PREP = _gpu.ALL_PREP | fnlh.FNLH_PREP_TAGS

CASES = {
    # ragged sizes: several 256-thread tiles plus a tail
    "b6n4": dict(dims=(13, 6, 5), block=6, n_harm=4, cfl=20.0),
    "b5n3": dict(dims=(7, 5, 3), block=5, n_harm=3, cfl=15.0),
    "b6n1_thin": dict(dims=(9, 3, 4), block=6, n_harm=1, cfl=20.0),
}


def periodic_problem(key, seeds=(1, 2, 3)):
    c = CASES[key]
    return inputs.problem(c["dims"], c["block"], c["n_harm"], c["cfl"], 1.3, seeds=seeds, name=key, periodic=True)


def oracle_jac(p):
    m = p.mesh
    return oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl, periodic=m.periodic)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    fnlh.lib()


@pytest.mark.parametrize("key", sorted(CASES))
def test_periodic_relax_f64_isolated(key):
    p = periodic_problem(key)
    dm, J, B = _gpu.device_problem(p, prep_flags=PREP)
    oj = oracle_jac(p)
    _gpu.load_jacobian(dm, J, oj)
    x0 = np.random.default_rng(7).normal(size=p.b.shape)
    X = torch.from_numpy(x0.copy()).cuda()
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 20, fnlh.FNLH_F64, sigma=p.phase)
    ref = oracle.jacobi(oj, p.mesh.vol, p.omega, p.b, 20, X0=x0, sigma=p.phase)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


@pytest.mark.parametrize("key", sorted(CASES))
def test_periodic_relax_f64_end_to_end(key):
    p = periodic_problem(key)
    dm, J, B = _gpu.device_problem(p, prep_flags=PREP)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 40, fnlh.FNLH_F64, sigma=p.phase)
    ref = oracle.jacobi(oracle_jac(p), p.mesh.vol, p.omega, p.b, 40, sigma=p.phase)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm)


def test_periodic_residual_matches_oracle():
    p = periodic_problem("b6n4")
    dm, J, B = _gpu.device_problem(p, prep_flags=PREP)
    oj = oracle_jac(p)
    _gpu.load_jacobian(dm, J, oj)
    x = np.random.default_rng(3).normal(size=p.b.shape)
    X = torch.from_numpy(x).cuda()
    r = torch.empty_like(B)
    norms = fnlh.fnlh_residual(dm, J, p.omega, B, X, r=r, sigma=p.phase).cpu().numpy()
    on, orr = oracle.residual(oj, p.mesh.vol, p.omega, p.b, x, want_r=True, sigma=p.phase)
    assert np.abs(r.cpu().numpy() - orr).max() <= 1e-13 * np.abs(orr).max()
    assert np.allclose(norms, on, rtol=1e-12, atol=0)
    n2 = fnlh.fnlh_residual_noalloc(dm, J, p.omega, B, X, sigma=p.phase).cpu().numpy()
    assert np.array_equal(norms, n2)


def test_zero_phase_equals_untagged_mesh_bitwise():
    """sigma = 0 on the periodic edges is plain periodicity: the same bits as
    the same edge list without periodic flags (the factor (1, 0) is exact)."""
    p = periodic_problem("b6n4")
    dm, J, B = _gpu.device_problem(p, prep_flags=PREP)
    plain_mesh = inputs.Mesh(p.mesh.dims, p.mesh.positions, p.mesh.edge_nodes, p.mesh.normals, p.mesh.vol)
    pp = inputs.Problem(plain_mesh, p.q, p.b, p.omega, p.block, p.cfl)
    dm0, J0, B0 = _gpu.device_problem(pp)
    for prec in (fnlh.FNLH_F64, fnlh.FNLH_F32, fnlh.FNLH_BF16):
        X = torch.zeros_like(B)
        X0 = torch.zeros_like(B)
        fnlh.fnlh_relax(dm, J, p.omega, B, X, 9, prec, sigma=np.zeros(p.n_harm))
        fnlh.fnlh_relax(dm0, J0, p.omega, B0, X0, 9, prec)
        assert torch.equal(X, X0), prec


@pytest.mark.parametrize("prec,bound", [(fnlh.FNLH_F32, 2e-5), (fnlh.FNLH_BF16, 5e-2)])
def test_periodic_low_precision_bounded(prec, bound):
    p = periodic_problem("b6n4")
    dm, J, B = _gpu.device_problem(p, prep_flags=PREP)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 30, prec, sigma=p.phase)
    ref = oracle.jacobi(oracle_jac(p), p.mesh.vol, p.omega, p.b, 30, sigma=p.phase)
    err = _gpu.rel_err_per_system(X.cpu().numpy(), ref, p.n_harm)
    assert np.all(err <= bound), err


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_BF16, fnlh.FNLH_F64])
def test_periodic_solve_reaches_1e8(prec):
    p = inputs.problem((24, 16, 12), 6, 8, 20.0, name="periodic_c3_reduced", periodic=True)
    dm, J, B = _gpu.device_problem(p, prep_flags=PREP)
    X = torch.zeros_like(B)
    st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, 1e-8, 12, 60,
                                              flags=fnlh.FNLH_SOLVE_ZERO_GUESS, sigma=p.phase)
    assert st == fnlh.FNLH_OK and np.all(rel <= 1e-8), (st, rel)
    true_rel = oracle.rel_residuals(oracle_jac(p), p.mesh.vol, p.omega, p.b, X.cpu().numpy(), sigma=p.phase)
    assert np.all(true_rel <= 1e-8), true_rel


def test_periodic_permuted_numbering():
    p = periodic_problem("b6n4")
    pm, perm = inputs.permute_mesh(p.mesh)
    pp = inputs.Problem(pm, p.q[perm], p.b[perm], p.omega, p.block, p.cfl, phase=p.phase)
    dm, J, B = _gpu.device_problem(pp, prep_flags=PREP)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, pp.omega, B, X, 25, fnlh.FNLH_F64, sigma=pp.phase)
    ref = oracle.jacobi(oracle_jac(p), p.mesh.vol, p.omega, p.b, 25, sigma=p.phase)
    _gpu.assert_fp64_parity(X.cpu().numpy(), ref[perm], p.n_harm)


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_F64])
def test_periodic_batched_rows_match_per_row(prec):
    rows = [periodic_problem("b6n4"),
            inputs.problem((9, 7, 5), 6, 2, 20.0, 1.0, seeds=(4, 5, 6)),  # an ordinary row in the same batch
            inputs.problem((10, 4, 6), 6, 8, 20.0, 2.3, seeds=(7, 8, 9), periodic=True)]
    dev = []
    for p in rows:
        dm, J, B = _gpu.device_problem(p, prep_flags=PREP)
        dev.append((p, dm, J, B))
    singles = []
    for p, dm, J, B in dev:
        X = torch.zeros_like(B)
        fnlh.fnlh_relax(dm, J, p.omega, B, X, 11, prec, sigma=p.phase)
        singles.append(X.cpu().numpy())
    Xs = [torch.zeros_like(B) for (_, _, _, B) in dev]
    batch = fnlh.BatchedRows([(dm, J, p.omega, B, X, p.phase) for (p, dm, J, B), X in zip(dev, Xs)])
    ws = torch.empty(batch.workspace_bytes(6), dtype=torch.uint8, device="cuda")
    fnlh.fnlh_relax_batched(batch, 11, prec, ws=ws)
    for X, ref, (p, *_rest) in zip(Xs, singles, dev):
        if prec == fnlh.FNLH_F64:
            # the single-row FP64 kernel solves the mean flow with a real-only path
            _gpu.assert_fp64_parity(X.cpu().numpy(), ref, p.n_harm, tol=1e-13)
        else:
            assert np.array_equal(X.cpu().numpy(), ref)


def _ring(p, P):
    """P passages side by side with plain periodicity (host arrays)."""
    m = p.mesh
    n = m.n_nodes
    en, per = m.edge_nodes.astype(np.int64), m.periodic.astype(np.int64)
    edges = [np.stack([en[:, 0] + q * n, en[:, 1] + ((q + per) % P) * n], axis=1) for q in range(P)]
    pos = np.concatenate([m.positions + np.array([0.0, q * m.dims[1], 0.0]) for q in range(P)])
    mesh = inputs.Mesh((m.dims[0], m.dims[1] * P, m.dims[2]), pos,
                       np.concatenate(edges).astype(np.int32), np.tile(m.normals, (P, 1)), np.tile(m.vol, P))
    return mesh


def _phase_shift(X, sigma, P):
    out = []
    for q in range(P):
        Y = X.copy()
        for l in range(1, len(sigma) + 1):
            z = (X[:, 2 * l - 1] + 1j * X[:, 2 * l]) * np.exp(1j * q * sigma[l - 1])
            Y[:, 2 * l - 1], Y[:, 2 * l] = z.real, z.imag
        out.append(Y)
    return np.concatenate(out, axis=0)


def test_periodic_full_size_equals_ring():
    """128x64x48 periodic passage, b = 6, mean + 4 harmonics, 50 FP64 sweeps
    (the benchmark's sweep count): against the oracle over the whole mesh, and
    against a ring of P = 3 passages on the GPU with sigma_l = 2 pi m_l / 3."""
    P = 3
    c = inputs.CONFIGS["c2"]
    sigma = 2.0 * np.pi * np.array([1, 2, 1, 2], dtype=np.float64) / P
    p = inputs.problem(c["dims"], c["block"], c["n_harm"], c["cfl"], name="c2_periodic", periodic=True, phase=sigma)
    dm, J, B = _gpu.device_problem(p, prep_flags=fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_TAGS)
    X = torch.zeros_like(B)
    fnlh.fnlh_relax(dm, J, p.omega, B, X, 50, fnlh.FNLH_F64, sigma=sigma)
    x = X.cpu().numpy()
    del dm, J, B, X
    ref = oracle.jacobi(oracle_jac(p), p.mesh.vol, p.omega, p.b, 50, sigma=sigma)
    _gpu.assert_fp64_parity(x, ref, p.n_harm)
    ring = inputs.Problem(_ring(p, P), np.tile(p.q, (P, 1)), _phase_shift(p.b, sigma, P), p.omega, p.block, p.cfl)
    rdm, rJ, rB = _gpu.device_problem(ring, prep_flags=fnlh.FNLH_PREP_F64)
    RX = torch.zeros_like(rB)
    fnlh.fnlh_relax(rdm, rJ, ring.omega, rB, RX, 50, fnlh.FNLH_F64)
    ref = _phase_shift(x, sigma, P)
    _gpu.assert_fp64_parity(RX.cpu().numpy(), ref, p.n_harm)
    torch.cuda.synchronize()


FF_PREP = PREP | fnlh.FNLH_PREP_FF


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_BF16])
def test_periodic_float_float_checks_match_fp64(prec):
    """The float-float residual applies e^{+-i sigma_l} to each periodic
    entry's product: with two checks its norms are the FP64 residual's of the
    same x (rounding apart); with three, the corrections it drives match the
    FP64-checked solve's to rounding."""
    p = inputs.problem((24, 16, 12), 6, 8, 20.0, 1.3, name="periodic_ff", periodic=True)
    dm, J, B = _gpu.device_problem(p, prep_flags=FF_PREP)
    n = p.mesh.n_nodes
    ws_ff = fnlh.solve_workspace(n, 6, p.n_harm, FF_PREP, "cuda", prec)
    ws_64 = fnlh.workspace(n, 6, p.n_harm, "cuda", prec)
    zg = fnlh.FNLH_SOLVE_ZERO_GUESS
    for checks in (2, 3):
        X1, X2 = torch.zeros_like(B), torch.zeros_like(B)
        st1, c1, s1, rel_ff = fnlh.fnlh_solve(dm, J, p.omega, B, X1, prec, 0.0, 12, checks, ws=ws_ff, flags=zg,
                                              sigma=p.phase, raise_on_error=False)
        st2, c2, s2, rel_64 = fnlh.fnlh_solve(dm, J, p.omega, B, X2, prec, 0.0, 12, checks, ws=ws_64, flags=zg,
                                              sigma=p.phase, raise_on_error=False)
        assert st1 == st2 == fnlh.FNLH_ERR_NOT_CONVERGED and c1 == c2 == checks
        if checks == 2:  # the same x: the float-float norms are the FP64 ones up to rounding
            assert torch.equal(X1, X2)
            assert np.allclose(rel_ff, rel_64, rtol=1e-6, atol=0), (rel_ff, rel_64)
        else:  # the second correction's FP32 right-hand side rounds a little differently
            err = _gpu.rel_err_per_system(X1.cpu().numpy(), X2.cpu().numpy(), p.n_harm)
            assert np.all(err <= 1e-8), err


@pytest.mark.parametrize("prec", [fnlh.FNLH_F32, fnlh.FNLH_BF16])
def test_periodic_float_float_solve_certified_by_oracle(prec):
    p = inputs.problem((24, 16, 12), 6, 8, 20.0, name="periodic_c3_reduced", periodic=True)
    dm, J, B = _gpu.device_problem(p, prep_flags=FF_PREP)
    X = torch.zeros_like(B)
    st, checks, sweeps, rel = fnlh.fnlh_solve(dm, J, p.omega, B, X, prec, 1e-8, 12, 60,
                                              flags=fnlh.FNLH_SOLVE_ZERO_GUESS, sigma=p.phase)
    assert st == fnlh.FNLH_OK and np.all(rel <= 1e-8), (st, rel)
    true_rel = oracle.rel_residuals(oracle_jac(p), p.mesh.vol, p.omega, p.b, X.cpu().numpy(), sigma=p.phase)
    assert np.all(true_rel <= 1e-8), true_rel
    assert np.allclose(rel, true_rel, rtol=1e-6, atol=1e-12), (rel, true_rel)

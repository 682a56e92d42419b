"""Pins of the CPU oracle to things other than itself (CPU only).

Each check reaches the oracle's result by an independent route fixed by the
paper or by mathematics:

* A(Q, n): the textbook closed-form Euler flux Jacobian and its eigenvalues
  u_n (x3), u_n +- a|n|.
* |A|(Q, n): an eigendecomposition V f(Lambda) V^-1 (numpy), and |A|^2 = A^2
  when the entropy fix is inactive.
* J and its diagonal: complex-step derivatives of a first-order residual
  with frozen dissipation, written here from its definition
  ("Generalized RK Scheme for The Mean Flow": J = dR/dQ from immediate
  neighbours); the block pseudo-time form of Eq. precon.
* D: closed forms on a uniform state over the unperturbed lattice.
* Consistency: J 1 = 0 on interior rows for a uniform state.
* Block Jacobi ("Solution Update"): one sweep from zero is the exact block
  solve; s sweeps equal (I - G^s) A^-1 B with G = -M^-1 N (dense); converged
  Jacobi equals dense and sparse direct solves of Eq. lhs_lin; the real
  2x2-block system of Eq. matrix_z_real gives the same solution; a harmonic
  with omega = 0 reproduces the mean flow exactly.
* Residual: B - A x from a dense matrix-vector product.
* Phase-lagged periodic edges (Eq. lhs_lin: the inter-blade phase angle
  changes each harmonic's LHS): one passage with phase lag sigma = 2 pi m / P
  behaves exactly like a ring of P identical passages joined by plain
  periodic edges whose right-hand side advances by e^{i sigma} per passage --
  sweep by sweep for Jacobi, and entry by entry for the residual.
* Block ILU(0) (the paper's implicit smoother): (L U)_ij = A_ij on every block
  of the pattern (hexahedral and triangulated patterns, red-black and natural
  orders), fill outside the pattern dropped, exact LU on a chain, on
  triangle-free patterns only the pivots change, partitions factor apart,
  iterations converge to the direct solve, and the phase-lagged passage
  equals the ring of passages iteration by iteration.
* Domain truncation (couplings across partitions dropped in the sweep): one
  partition is plain Jacobi, bit for bit; converged truncated Jacobi equals
  independent dense solves of every partition's diagonal sub-matrix; with
  one node per partition one sweep is already the fixed point.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from paper_2404_01407_gb300 import inputs
from tests import _dense

GAMMA = 1.4


# ------------------------------------------------------------ flux Jacobian

def textbook_A(q, n, gamma=GAMMA):
    """Closed-form Euler flux Jacobian d(F.n)/dQ for conservative Q (any |n|)."""
    rho, mu, mv, mw, rE = q[:5]
    u, v, w = mu / rho, mv / rho, mw / rho
    g1 = gamma - 1.0
    p = g1 * (rE - 0.5 * rho * (u * u + v * v + w * w))
    H = (rE + p) / rho
    phi = 0.5 * g1 * (u * u + v * v + w * w)
    nx, ny, nz = n
    un = u * nx + v * ny + w * nz
    vel = (u, v, w)
    nn = (nx, ny, nz)
    A = np.zeros((len(q), len(q)))
    A[0, 1:4] = nn
    for r in range(3):
        A[1 + r, 0] = nn[r] * phi - vel[r] * un
        for c in range(3):
            A[1 + r, 1 + c] = vel[r] * nn[c] - g1 * vel[c] * nn[r] + (un if r == c else 0.0)
        A[1 + r, 4] = g1 * nn[r]
    A[4, 0] = un * (phi - H)
    for c in range(3):
        A[4, 1 + c] = H * nn[c] - g1 * vel[c] * un
    A[4, 4] = gamma * un
    if len(q) == 6:
        nu = q[5] / rho
        A[5, 0] = -nu * un
        A[5, 1:4] = nu * np.asarray(nn)
        A[5, 5] = un
    return A


def random_states(rng, count, block):
    qs = []
    for _ in range(count):
        rho = 1.0 + rng.uniform(-0.3, 0.3)
        vel = rng.uniform(-0.8, 0.8, 3)
        p = 1.0 / GAMMA * (1.0 + rng.uniform(-0.3, 0.3))
        q = np.zeros(block)
        q[0] = rho
        q[1:4] = rho * vel
        q[4] = p / (GAMMA - 1.0) + 0.5 * rho * vel @ vel
        if block == 6:
            q[5] = rho * rng.uniform(0.001, 0.1)
        qs.append(q)
    return qs


@pytest.mark.parametrize("block", [5, 6])
def test_flux_jacobian_matches_textbook(block):
    rng = np.random.default_rng(11)
    for q in random_states(rng, 20, block):
        n = rng.normal(size=3) * rng.uniform(0.1, 2.0)
        A = oracle.flux_jacobian(q, n)
        At = textbook_A(q, n)
        assert np.allclose(A, At, rtol=1e-13, atol=1e-13 * np.abs(At).max())


def test_flux_jacobian_eigenvalues():
    rng = np.random.default_rng(12)
    for q in random_states(rng, 20, 5):
        n = rng.normal(size=3)
        A = oracle.flux_jacobian(q, n)
        rho = q[0]
        vel = q[1:4] / rho
        p = (GAMMA - 1) * (q[4] - 0.5 * rho * vel @ vel)
        a = np.sqrt(GAMMA * p / rho)
        un = vel @ n
        c = a * np.linalg.norm(n)
        ev = np.sort(np.linalg.eigvals(A).real)
        assert np.allclose(ev, np.sort([un, un, un, un + c, un - c]), atol=1e-7)


def eig_abs(A5, fix):
    lam, V = np.linalg.eig(A5)
    f = np.maximum(np.abs(lam.real), fix)
    return (V @ np.diag(f) @ np.linalg.inv(V)).real


@pytest.mark.parametrize("delta", [0.0, 0.1, 0.9])
def test_abs_jacobian_eigendecomposition(delta):
    rng = np.random.default_rng(13)
    for q in random_states(rng, 20, 6):
        n = rng.normal(size=3)
        A = textbook_A(q, n)
        rho = q[0]
        vel = q[1:4] / rho
        p = (GAMMA - 1) * (q[4] - 0.5 * rho * vel @ vel)
        a = np.sqrt(GAMMA * p / rho)
        un = vel @ n
        fix = delta * (abs(un) + a * np.linalg.norm(n))
        ref = np.zeros((6, 6))
        ref[:5, :5] = eig_abs(A[:5, :5], fix)
        ref[5, 5] = max(abs(un), fix)
        got = oracle.abs_jacobian(q, n, delta=delta)
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
        if delta == 0.0:
            got5 = oracle.abs_jacobian(q[:5], n, delta=0.0)
            assert np.allclose(got5 @ got5, A[:5, :5] @ A[:5, :5], atol=1e-11 * np.abs(A).max() ** 2)


def test_abs_jacobian_zero_normal():
    q = inputs.flow_state(1, 5)[0]
    assert np.all(oracle.abs_jacobian(q, np.zeros(3)) == 0.0)


# -------------------------------------------------- Jacobian of the residual

def flux_c(q, n, gamma=GAMMA):
    rho = q[0]
    u, v, w = q[1] / rho, q[2] / rho, q[3] / rho
    p = (gamma - 1) * (q[4] - 0.5 * (q[1] * u + q[2] * v + q[3] * w))
    un = u * n[0] + v * n[1] + w * n[2]
    f = [q[0] * un, q[1] * un + p * n[0], q[2] * un + p * n[1], q[3] * un + p * n[2], (q[4] + p) * un]
    if len(q) == 6:
        f.append(q[5] * un)
    return np.array(f)


def test_abs_is_frozen_consistent_with_eig():
    """Sanity of the helper used below: test-side |A| from eig agrees with the oracle."""
    q = inputs.flow_state(1, 6)[0]
    n = np.array([0.9, -0.2, 0.1])
    A = textbook_A(q, n)
    un = (q[1:4] / q[0]) @ n
    p = (GAMMA - 1) * (q[4] - 0.5 * q[0] * (q[1:4] / q[0]) @ (q[1:4] / q[0]))
    a = np.sqrt(GAMMA * p / q[0])
    fix = 0.1 * (abs(un) + a * np.linalg.norm(n))
    ref = np.zeros((6, 6))
    ref[:5, :5] = eig_abs(A[:5, :5], fix)
    ref[5, 5] = max(abs(un), fix)
    assert np.allclose(ref, oracle.abs_jacobian(q, n), atol=1e-12)


def test_abs_jacobian_inactive_fix_square():
    q = inputs.flow_state(3, 5, seed=5)[1]
    n = np.array([1.1, 0.3, -0.4])
    M = oracle.abs_jacobian(q, n, delta=0.0)
    A = oracle.flux_jacobian(q, n)
    assert np.allclose(M @ M, A @ A, atol=1e-12)


def _frozen_residual_jacobian(mesh, q, cfl, delta=0.1):
    """Complex-step derivative of the first-order residual with |A| frozen."""
    n, b = q.shape
    en, nrm = mesh.edge_nodes, mesh.normals
    nbrs = [[] for _ in range(n)]
    for e, (i, j) in enumerate(en):
        nbrs[i].append((j, nrm[e]))
        nbrs[j].append((i, -nrm[e]))

    def test_abs(qs, nv):
        if np.linalg.norm(nv) == 0:
            return np.zeros((b, b))
        A = textbook_A(qs, nv)
        rho = qs[0]
        vel = qs[1:4] / rho
        p = (GAMMA - 1) * (qs[4] - 0.5 * rho * vel @ vel)
        a = np.sqrt(GAMMA * p / rho)
        un = vel @ nv
        fix = delta * (abs(un) + a * np.linalg.norm(nv))
        out = np.zeros((b, b))
        out[:5, :5] = eig_abs(A[:5, :5], fix)
        if b == 6:
            out[5, 5] = max(abs(un), fix)
        return out

    frozen = {}
    nb_normal = {}
    for i in range(n):
        nbn = np.zeros(3)
        for j, nv in nbrs[i]:
            frozen[(i, j)] = test_abs(0.5 * (q[i] + q[j]), nv)
            nbn -= nv
        nb_normal[i] = nbn
        frozen[(i, "b")] = test_abs(q[i], nbn)

    def residual(qc):
        R = np.zeros((n, b), dtype=np.complex128)
        for i in range(n):
            for j, nv in nbrs[i]:
                R[i] += 0.5 * (flux_c(qc[i], nv) + flux_c(qc[j], nv)) - 0.5 * frozen[(i, j)] @ (qc[j] - qc[i])
            nbn = nb_normal[i]
            qext = q[i]  # far-field state: a constant
            R[i] += 0.5 * (flux_c(qc[i], nbn) + flux_c(qext, nbn)) - 0.5 * frozen[(i, "b")] @ (qext - qc[i])
            if b == 6:
                # frozen turbulence: mean-flow rows do not see Q_6 (only row 6 does)
                pass
        return R

    h = 1e-30
    dRdQ = np.zeros((n, b, n, b))
    for j in range(n):
        for s in range(b):
            qc = q.astype(np.complex128)
            qc[j, s] += 1j * h
            dRdQ[:, :, j, s] = residual(qc).imag / h
    return dRdQ


@pytest.mark.parametrize("block", [5, 6])
def test_jacobian_is_frozen_residual_derivative(block):
    mesh = inputs.hex_mesh(3, 3, 2, seed=21)
    q = inputs.flow_state(mesh.n_nodes, block, seed=22)
    cfl = 10.0
    jac = oracle.build_jacobian(mesh.n_nodes, mesh.edge_nodes, mesh.normals, q, cfl)
    d = _frozen_residual_jacobian(mesh, q, cfl)
    scale = np.abs(d).max()
    for i in range(mesh.n_nodes):
        expect_ii = d[i, :, i, :].copy()
        if block == 6:
            expect_ii[5, 5] *= 2.0  # turbulence-row dominance
        assert np.allclose(jac.diag[i], expect_ii, atol=1e-12 * scale), i
        for p in range(jac.row_ptr[i], jac.row_ptr[i + 1]):
            j = jac.col_idx[p]
            assert np.allclose(jac.offd[p], d[i, :, j, :], atol=1e-12 * scale), (i, j)
    # the pattern of dR/dQ is exactly the mesh graph
    mask = np.zeros((mesh.n_nodes, mesh.n_nodes), dtype=bool)
    for i in range(mesh.n_nodes):
        mask[i, jac.col_idx[jac.row_ptr[i]:jac.row_ptr[i + 1]]] = True
        mask[i, i] = True
    off = np.abs(d).max(axis=(1, 3))
    assert np.all(off[~mask] == 0.0)


def test_pseudo_time_block_form():
    """Eq. precon, implicit: K = P/(eps sigma) + J, P the diagonal block of J."""
    mesh = inputs.hex_mesh(4, 3, 2, seed=5)
    q = inputs.flow_state(mesh.n_nodes, 6, seed=6)
    a = oracle.build_jacobian(mesh.n_nodes, mesh.edge_nodes, mesh.normals, q, 20.0)
    bl = oracle.build_jacobian(mesh.n_nodes, mesh.edge_nodes, mesh.normals, q, 20.0, pseudo_block=True, eps=0.6)
    assert np.array_equal(a.offd, bl.offd)
    assert np.all(bl.D == 0.0)
    assert np.allclose(bl.diag, a.diag * (1.0 + 1.0 / (0.6 * 20.0)), rtol=1e-15)


# ---------------------------------------------------- closed forms, uniform

def test_D_closed_form_uniform_state():
    nx, ny, nz = 5, 4, 3
    mesh = inputs.hex_mesh(nx, ny, nz, perturb=0.0)
    q = inputs.flow_state(mesh.n_nodes, 5, uniform=True)
    cfl = 10.0
    jac = oracle.build_jacobian(mesh.n_nodes, mesh.edge_nodes, mesh.normals, q, cfl)
    a = np.sqrt(GAMMA * (1.0 / GAMMA) / 1.0)
    u = 0.5 * a
    D = jac.D.reshape(nz, ny, nx)
    # interior and face nodes: the closure face replaces one missing face
    assert np.isclose(D[1, 1, 1], (2 * u + 6 * a) / cfl, rtol=1e-14)
    assert np.isclose(D[1, 1, 0], (2 * u + 6 * a) / cfl, rtol=1e-14)
    assert np.isclose(D[1, 0, 2], (2 * u + 6 * a) / cfl, rtol=1e-14)
    # corner (0,0,0): faces +x, +y, +z and a closure normal -(1,1,1)
    assert np.isclose(D[0, 0, 0], ((u + a) + a + a + (u + np.sqrt(3) * a)) / cfl, rtol=1e-14)
    # edge node (0,0,k): missing -x and -y
    assert np.isclose(D[1, 0, 0], ((u + a) + a + 2 * a + (u + np.sqrt(2) * a)) / cfl, rtol=1e-14)


@pytest.mark.parametrize("block", [5, 6])
def test_consistency_uniform_state(block):
    """J 1 = 0 on interior rows: sum_j J_ij + J_ii = A(Q, sum_j n_ij) = 0."""
    nx, ny, nz = 5, 4, 4
    mesh = inputs.hex_mesh(nx, ny, nz, perturb=0.0)
    q = inputs.flow_state(mesh.n_nodes, block, uniform=True)
    jac = oracle.build_jacobian(mesh.n_nodes, mesh.edge_nodes, mesh.normals, q, 10.0)
    interior = [i + nx * (j + ny * k) for k in range(1, nz - 1) for j in range(1, ny - 1) for i in range(1, nx - 1)]
    ref_diag = jac.diag[interior[0]]
    for i in interior:
        s = jac.diag[i] + jac.offd[jac.row_ptr[i]:jac.row_ptr[i + 1]].sum(axis=0)
        if block == 6:
            s[5, 5] -= 0.5 * jac.diag[i][5, 5]  # undo the doubled turbulence diagonal
        assert np.allclose(s, 0.0, atol=1e-14)
        assert np.array_equal(jac.diag[i], ref_diag)  # translational invariance


def test_pattern_symmetric_sorted():
    mesh = inputs.hex_mesh(6, 5, 4)
    q = inputs.flow_state(mesh.n_nodes, 5)
    jac = oracle.build_jacobian(mesh.n_nodes, mesh.edge_nodes, mesh.normals, q, 10.0)
    assert jac.nnz == 2 * mesh.n_edges
    pairs = set()
    for i in range(mesh.n_nodes):
        cols = jac.col_idx[jac.row_ptr[i]:jac.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and i not in cols
        pairs.update((i, int(j)) for j in cols)
    assert all((j, i) in pairs for (i, j) in pairs)


def test_bad_edges_rejected():
    with pytest.raises(ValueError):
        oracle.build_jacobian(3, np.array([[0, 0]]), np.ones((1, 3)), inputs.flow_state(3, 5), 10.0)
    with pytest.raises(ValueError):
        oracle.build_jacobian(3, np.array([[0, 1], [1, 0]]), np.ones((2, 3)), inputs.flow_state(3, 5), 10.0)


# ------------------------------------------------------------ block Jacobi

def small_problem(dims=(4, 3, 3), block=6, n_harm=2, cfl=20.0, seed=0):
    mesh = inputs.hex_mesh(*dims, seed=1 + seed)
    q = inputs.flow_state(mesh.n_nodes, block, seed=2 + seed)
    jac = oracle.build_jacobian(mesh.n_nodes, mesh.edge_nodes, mesh.normals, q, cfl)
    B = inputs.rhs(mesh.n_nodes, block, n_harm, seed=3 + seed)
    om = inputs.omegas(n_harm, 1.3)
    return mesh, jac, B, om


def _systems(jac, vol, om):
    return [(0.0 if k == 0 else om[k - 1]) for k in range(len(om) + 1)]


def test_one_sweep_is_exact_block_solve():
    mesh, jac, B, om = small_problem()
    X1 = oracle.jacobi(jac, mesh.vol, om, B, 1)
    b = jac.block
    for i in range(mesh.n_nodes):
        for k, w in enumerate(_systems(jac, mesh.vol, om)):
            M = jac.diag[i] + (jac.D[i] + 1j * w * mesh.vol[i]) * np.eye(b)
            rhs = B[i, 0] if k == 0 else B[i, 2 * k - 1] + 1j * B[i, 2 * k]
            y = np.linalg.solve(M, rhs)
            got = X1[i, 0] if k == 0 else X1[i, 2 * k - 1] + 1j * X1[i, 2 * k]
            assert np.allclose(got, y, rtol=1e-13, atol=1e-14 * np.abs(y).max())


@pytest.mark.parametrize("sweeps", [1, 2, 5, 17])
def test_sweeps_match_iteration_matrix_power(sweeps):
    """x^s = (I - G^s) A^-1 B + G^s x^0 with G = -M^-1 N (dense)."""
    mesh, jac, B, om = small_problem(dims=(3, 3, 2), block=5, n_harm=2)
    x0 = np.random.default_rng(9).normal(size=B.shape)
    Xs = oracle.jacobi(jac, mesh.vol, om, B, sweeps, X0=x0)
    got = _dense.split_systems(Xs, len(om))
    bs = _dense.split_systems(B, len(om))
    x0s = _dense.split_systems(x0, len(om))
    for k, w in enumerate(_systems(jac, mesh.vol, om)):
        M, N = _dense.block_split(jac.row_ptr, jac.col_idx, jac.offd, jac.diag, jac.D, mesh.vol, w)
        G = -np.linalg.solve(M, N)
        xstar = np.linalg.solve(M + N, bs[k])
        Gs = np.linalg.matrix_power(G, sweeps)
        ref = xstar - Gs @ xstar + Gs @ (x0s[k] if k > 0 else x0s[0].real)
        assert np.allclose(got[k], ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max()), k


@pytest.mark.parametrize("block", [5, 6])
def test_converged_jacobi_equals_direct_solve(block):
    mesh, jac, B, om = small_problem(block=block)
    X, _ = oracle.solve_to_tol(jac, mesh.vol, om, B, tol=1e-15, chunk=50, max_sweeps=2000)
    got = _dense.split_systems(X, len(om))
    bs = _dense.split_systems(B, len(om))
    for k, w in enumerate(_systems(jac, mesh.vol, om)):
        A = _dense.dense_operator(jac.row_ptr, jac.col_idx, jac.offd, jac.diag, jac.D, mesh.vol, w)
        xd = np.linalg.solve(A, bs[k])
        assert np.linalg.norm(got[k] - xd) <= 1e-12 * np.linalg.norm(xd)


def test_real_2x2_block_form_matches_complex():
    """Eq. matrix_z_real: [[A, -w V], [w V, A]] [Re x; Im x] = [Re B; Im B]."""
    mesh, jac, B, om = small_problem(block=6, n_harm=2)
    X, _ = oracle.solve_to_tol(jac, mesh.vol, om, B, tol=1e-15, chunk=50, max_sweeps=2000)
    n, b = mesh.n_nodes, jac.block
    A0 = _dense.dense_operator(jac.row_ptr, jac.col_idx, jac.offd, jac.diag, jac.D, mesh.vol, 0.0).real
    Vd = np.kron(np.diag(mesh.vol), np.eye(b))
    for k in range(1, len(om) + 1):
        w = om[k - 1]
        big = np.block([[A0, -w * Vd], [w * Vd, A0]])
        rhs = np.concatenate([B[:, 2 * k - 1].ravel(), B[:, 2 * k].ravel()])
        sol = np.linalg.solve(big, rhs)
        ref = np.concatenate([X[:, 2 * k - 1].ravel(), X[:, 2 * k].ravel()])
        assert np.linalg.norm(sol - ref) <= 1e-12 * np.linalg.norm(sol)
        Ac = _dense.dense_operator(jac.row_ptr, jac.col_idx, jac.offd, jac.diag, jac.D, mesh.vol, w)
        xc = np.linalg.solve(Ac, B[:, 2 * k - 1].ravel() + 1j * B[:, 2 * k].ravel())
        assert np.linalg.norm(sol[: n * b] + 1j * sol[n * b:] - xc) <= 1e-12 * np.linalg.norm(xc)


def test_omega_zero_harmonic_reproduces_mean():
    mesh, jac, B, om = small_problem(block=6, n_harm=2)
    om = np.array([0.0, 1.0])
    B = B.copy()
    B[:, 1] = B[:, 0]
    B[:, 2] = 0.0
    X = oracle.jacobi(jac, mesh.vol, om, B, 7)
    assert np.array_equal(X[:, 1], X[:, 0])
    assert np.all(X[:, 2] == 0.0)


def test_sparse_direct_solve_config1():
    """Config 1 (16x8x8, b = 5, N = 1, CFL 10): converged Jacobi = spsolve."""
    p = inputs.config_problem("c1")
    m = p.mesh
    jac = oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl)
    X, done = oracle.solve_to_tol(jac, m.vol, p.omega, p.b, tol=1e-14, chunk=20, max_sweeps=2000)
    got = _dense.split_systems(X, p.n_harm)
    bs = _dense.split_systems(p.b, p.n_harm)
    for k, w in enumerate([0.0] + list(p.omega)):
        A = _dense.sparse_operator(jac.row_ptr, jac.col_idx, jac.offd, jac.diag, jac.D, m.vol, w)
        xs = spla.spsolve(A.tocsc(), bs[k])
        assert np.linalg.norm(got[k] - xs) <= 1e-12 * np.linalg.norm(xs)


def test_residual_matches_dense_product():
    mesh, jac, B, om = small_problem(block=6, n_harm=3)
    X = np.random.default_rng(5).normal(size=B.shape)
    norms, r = oracle.residual(jac, mesh.vol, om, B, X, want_r=True)
    xs = _dense.split_systems(X, len(om))
    bs = _dense.split_systems(B, len(om))
    rs = _dense.split_systems(r, len(om))
    for k, w in enumerate(_systems(jac, mesh.vol, om)):
        A = _dense.dense_operator(jac.row_ptr, jac.col_idx, jac.offd, jac.diag, jac.D, mesh.vol, w)
        xk = xs[k].real if k == 0 else xs[k]
        ref = bs[k] - A @ xk
        assert np.allclose(rs[k], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
        assert np.isclose(norms[k, 0], np.vdot(ref, ref).real, rtol=1e-12)
        assert np.isclose(norms[k, 1], np.vdot(bs[k], bs[k]).real, rtol=1e-12)


# ------------------------------------------------ phase-lagged periodicity

RING_P = 5
RING_M = (1, 2, 3)  # nodal diameters of the three harmonics: sigma_l = 2 pi m_l / P


def passage_problem(block=6):
    mesh = inputs.hex_mesh(3, 4, 2, seed=11, periodic_y=True)
    q = inputs.flow_state(mesh.n_nodes, block, seed=12)
    jac = oracle.build_jacobian(mesh.n_nodes, mesh.edge_nodes, mesh.normals, q, 20.0,
                                periodic=mesh.periodic)
    n_harm = len(RING_M)
    B = inputs.rhs(mesh.n_nodes, block, n_harm, seed=13)
    om = inputs.omegas(n_harm, 0.9)
    sigma = 2.0 * np.pi * np.asarray(RING_M, dtype=np.float64) / RING_P
    return mesh, q, jac, B, om, sigma


def ring_of_passages(mesh, q, P):
    """P copies of the passage side by side; every periodic edge of copy p
    becomes an ordinary edge to the neighbouring copy (the last wraps to the
    first), with the passage's own normals, volumes and state."""
    n = mesh.n_nodes
    en, per = mesh.edge_nodes.astype(np.int64), mesh.periodic.astype(np.int64)
    edges = []
    for p in range(P):
        a = en[:, 0] + p * n
        c = en[:, 1] + ((p + per) % P) * n
        edges.append(np.stack([a, c], axis=1))
    ring_en = np.concatenate(edges).astype(np.int32)
    ring_normals = np.tile(mesh.normals, (P, 1))
    return ring_en, ring_normals, np.tile(mesh.vol, P), np.tile(q, (P, 1))


def phase_shift(X, n_harm, sigma, P):
    """Ring vector whose passage p is passage vector X times e^{i p sigma_l}
    (harmonic l); the mean flow is repeated unchanged."""
    out = []
    for p in range(P):
        Y = X.copy()
        for l in range(1, n_harm + 1):
            z = (X[:, 2 * l - 1] + 1j * X[:, 2 * l]) * np.exp(1j * p * sigma[l - 1])
            Y[:, 2 * l - 1], Y[:, 2 * l] = z.real, z.imag
        out.append(Y)
    return np.concatenate(out, axis=0)


def test_phase_sides_follow_edge_direction():
    mesh, q, jac, B, om, sigma = passage_problem()
    side = jac.side
    assert side.dtype == np.int8 and side.shape == (jac.nnz,)
    owner = np.repeat(np.arange(mesh.n_nodes), np.diff(jac.row_ptr))
    nx, ny, nz = mesh.dims
    yj = lambda i: (i // nx) % ny  # noqa: E731
    for p in range(jac.nnz):
        i, j = owner[p], jac.col_idx[p]
        want = 1 if (yj(i) == ny - 1 and yj(j) == 0) else (-1 if (yj(i) == 0 and yj(j) == ny - 1) else 0)
        assert side[p] == want, (i, j)
    assert (side == 1).sum() == (side == -1).sum() == nx * nz


@pytest.mark.parametrize("sweeps", [1, 3, 12])
def test_phase_lagged_jacobi_equals_ring(sweeps):
    mesh, q, jac, B, om, sigma = passage_problem()
    n, P, N = mesh.n_nodes, RING_P, len(om)
    ren, rnorm, rvol, rq = ring_of_passages(mesh, q, P)
    rjac = oracle.build_jacobian(n * P, ren, rnorm, rq, 20.0)
    X0 = np.random.default_rng(14).normal(size=B.shape)
    got = oracle.jacobi(jac, mesh.vol, om, B, sweeps, X0=X0, sigma=sigma)
    ring = oracle.jacobi(rjac, rvol, om, phase_shift(B, N, sigma, P), sweeps, X0=phase_shift(X0, N, sigma, P))
    ref = phase_shift(got, N, sigma, P)
    assert np.allclose(ring, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # the phase matters: plain periodicity (sigma = 0) is a different iterate
    plain = oracle.jacobi(jac, mesh.vol, om, B, sweeps, X0=X0)
    assert np.abs(plain[:, 1:] - got[:, 1:]).max() > 1e-3 * np.abs(got).max()
    assert np.array_equal(plain[:, 0], got[:, 0])  # the mean flow carries no phase


def test_phase_lagged_solution_is_ring_solution():
    """Converged single passage = dense direct solve of the ring, passage 0."""
    mesh, q, jac, B, om, sigma = passage_problem(block=5)
    n, P, N, b = mesh.n_nodes, RING_P, len(om), jac.block
    ren, rnorm, rvol, rq = ring_of_passages(mesh, q, P)
    rjac = oracle.build_jacobian(n * P, ren, rnorm, rq, 20.0)
    X, _ = oracle.solve_to_tol(jac, mesh.vol, om, B, tol=1e-15, chunk=50, max_sweeps=3000, sigma=sigma)
    bring = _dense.split_systems(phase_shift(B, N, sigma, P), N)
    got = _dense.split_systems(X, N)
    for k, w in enumerate([0.0] + list(om)):
        A = _dense.dense_operator(rjac.row_ptr, rjac.col_idx, rjac.offd, rjac.diag, rjac.D, rvol, w)
        xr = np.linalg.solve(A, bring[k])[: n * b]
        assert np.linalg.norm(got[k] - xr) <= 1e-12 * np.linalg.norm(xr), k


def test_phase_lagged_residual_equals_ring():
    mesh, q, jac, B, om, sigma = passage_problem()
    n, P, N = mesh.n_nodes, RING_P, len(om)
    ren, rnorm, rvol, rq = ring_of_passages(mesh, q, P)
    rjac = oracle.build_jacobian(n * P, ren, rnorm, rq, 20.0)
    X = np.random.default_rng(15).normal(size=B.shape)
    norms, r = oracle.residual(jac, mesh.vol, om, B, X, want_r=True, sigma=sigma)
    rnorms, rr = oracle.residual(rjac, rvol, om, phase_shift(B, N, sigma, P), phase_shift(X, N, sigma, P),
                                 want_r=True)
    ref = phase_shift(r, N, sigma, P)
    assert np.allclose(rr, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert np.allclose(rnorms, P * norms, rtol=1e-12)


# ------------------------------------------------------ domain truncation

def test_one_partition_is_plain_jacobi():
    mesh, jac, B, om = small_problem(dims=(5, 4, 3), block=6, n_harm=2)
    x0 = np.random.default_rng(21).normal(size=B.shape)
    a = oracle.jacobi(jac, mesh.vol, om, B, 7, X0=x0)
    b = oracle.jacobi(jac, mesh.vol, om, B, 7, X0=x0, part=np.zeros(mesh.n_nodes, np.int32))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("parts", [(2, 1, 1), (2, 2, 1), (3, 2, 2)])
def test_truncated_jacobi_solves_each_partition(parts):
    dims = (6, 4, 4)
    mesh, jac, B, om = small_problem(dims=dims, block=5, n_harm=2)
    part = inputs.box_partition(dims, parts)
    assert len(np.unique(part)) == parts[0] * parts[1] * parts[2]
    X = oracle.jacobi(jac, mesh.vol, om, B, 600, part=part)
    got = _dense.split_systems(X, len(om))
    bs = _dense.split_systems(B, len(om))
    b = jac.block
    for k, w in enumerate(_systems(jac, mesh.vol, om)):
        A = _dense.dense_operator(jac.row_ptr, jac.col_idx, jac.offd, jac.diag, jac.D, mesh.vol, w)
        for q in np.unique(part):
            idx = np.concatenate([np.arange(i * b, (i + 1) * b) for i in np.flatnonzero(part == q)])
            xq = np.linalg.solve(A[np.ix_(idx, idx)], bs[k][idx])
            assert np.linalg.norm(got[k][idx] - xq) <= 1e-12 * np.linalg.norm(xq), (k, q)


def test_single_node_partitions_fix_after_one_sweep():
    mesh, jac, B, om = small_problem(dims=(4, 3, 3), block=6, n_harm=1)
    part = np.arange(mesh.n_nodes, dtype=np.int32)
    X1 = oracle.jacobi(jac, mesh.vol, om, B, 1, part=part)
    X2 = oracle.jacobi(jac, mesh.vol, om, B, 2, part=part)
    assert np.array_equal(X1, X2)
    b = jac.block
    for i in range(mesh.n_nodes):
        M = jac.diag[i] + (jac.D[i] + 1j * om[0] * mesh.vol[i]) * np.eye(b)
        y = np.linalg.solve(M, B[i, 1] + 1j * B[i, 2])
        assert np.allclose(X1[i, 1] + 1j * X1[i, 2], y, rtol=1e-13, atol=1e-14 * np.abs(y).max())


# ------------------------------------------------------------------ ILU(0)

def _dense_lu(jac, rank, Fd, Fo, part=None):
    """Dense unit-lower L and upper U from the block factors."""
    n, b = Fd.shape[0], Fd.shape[1]
    L = np.eye(n * b, dtype=np.complex128)
    U = np.zeros((n * b, n * b), dtype=np.complex128)
    for i in range(n):
        U[i * b:(i + 1) * b, i * b:(i + 1) * b] = Fd[i]
        for p in range(jac.row_ptr[i], jac.row_ptr[i + 1]):
            j = jac.col_idx[p]
            if part is not None and part[i] != part[j]:
                continue
            tgt = L if rank[j] < rank[i] else U
            tgt[i * b:(i + 1) * b, j * b:(j + 1) * b] = Fo[p]
    return L, U


def _pattern_mask(jac, n, b, part=None):
    M = np.zeros((n * b, n * b), dtype=bool)
    for i in range(n):
        M[i * b:(i + 1) * b, i * b:(i + 1) * b] = True
        for p in range(jac.row_ptr[i], jac.row_ptr[i + 1]):
            j = jac.col_idx[p]
            if part is None or part[i] == part[j]:
                M[i * b:(i + 1) * b, j * b:(j + 1) * b] = True
    return M


def _mesh_with_triangles():
    """A 4x3x2 lattice plus one diagonal per xy cell: every cell holds triangles."""
    base = inputs.hex_mesh(4, 3, 2, seed=31)
    nx, ny = 4, 3
    extra = []
    for k in range(2):
        for j in range(ny - 1):
            for i in range(nx - 1):
                extra.append((i + nx * (j + ny * k), i + 1 + nx * (j + 1 + ny * k)))
    en = np.concatenate([base.edge_nodes, np.array(extra, dtype=np.int32)])
    return inputs.custom_mesh(base.positions, en, vol=base.vol)


@pytest.mark.parametrize("case", ["hex_redblack", "hex_natural", "triangles_greedy"])
def test_ilu0_reproduces_the_matrix_on_its_pattern(case):
    """ILU(0) defining property: (L U)_ij = A_ij on every block of the pattern."""
    if case.startswith("hex"):
        mesh = inputs.hex_mesh(4, 3, 3, seed=1)
        color = inputs.lattice_colors((4, 3, 3)) if case == "hex_redblack" else np.zeros(mesh.n_nodes)
        rank = oracle.elimination_rank(color) if case == "hex_redblack" else np.arange(mesh.n_nodes, dtype=np.int32)
    else:
        mesh = _mesh_with_triangles()
        rank = oracle.elimination_rank(np.arange(mesh.n_nodes) % 3)
    q = inputs.flow_state(mesh.n_nodes, 5, seed=2)
    jac = oracle.build_jacobian(mesh.n_nodes, mesh.edge_nodes, mesh.normals, q, 15.0)
    n, b = mesh.n_nodes, 5
    for w in (0.0, 1.7):
        Fd, Fo = oracle.ilu_factor(jac, mesh.vol, w, rank)
        L, U = _dense_lu(jac, rank, Fd, Fo)
        A = _dense.dense_operator(jac.row_ptr, jac.col_idx, jac.offd, jac.diag, jac.D, mesh.vol, w)
        M = _pattern_mask(jac, n, b)
        LU = L @ U
        assert np.abs((LU - A)[M]).max() <= 1e-12 * np.abs(A).max()
        if case == "triangles_greedy":
            # not an exact factorisation: fill outside the pattern was dropped
            assert np.abs((LU - A)[~M]).max() > 1e-6 * np.abs(A).max()


def test_ilu0_on_triangle_free_pattern_only_changes_pivots():
    """No triangles: the upper blocks stay A_ij and L_ik = A_ik U_kk^-1."""
    mesh = inputs.hex_mesh(5, 4, 3, seed=3)
    q = inputs.flow_state(mesh.n_nodes, 6, seed=4)
    jac = oracle.build_jacobian(mesh.n_nodes, mesh.edge_nodes, mesh.normals, q, 20.0)
    rank = oracle.elimination_rank(inputs.lattice_colors((5, 4, 3)))
    Fd, Fo = oracle.ilu_factor(jac, mesh.vol, 2.0, rank)
    owner = np.repeat(np.arange(mesh.n_nodes), np.diff(jac.row_ptr))
    for p in range(jac.nnz):
        i, j = owner[p], jac.col_idx[p]
        if rank[j] > rank[i]:
            assert np.array_equal(Fo[p], jac.offd[p].astype(np.complex128))
        else:
            assert np.allclose(Fo[p] @ Fd[j], jac.offd[p], rtol=0, atol=1e-12 * np.abs(jac.offd[p]).max())


def test_ilu0_is_exact_on_a_chain():
    """A path graph in natural order has no fill: one application solves A x = r."""
    n = 7
    pos = np.stack([np.arange(n, dtype=float), np.zeros(n), np.zeros(n)], axis=1)
    pos[:, 1] = 0.05 * np.sin(np.arange(n))
    mesh = inputs.custom_mesh(pos, np.stack([np.arange(n - 1), np.arange(1, n)], axis=1))
    q = inputs.flow_state(n, 6, seed=5)
    jac = oracle.build_jacobian(n, mesh.edge_nodes, mesh.normals, q, 5.0)
    rank = np.arange(n, dtype=np.int32)
    F = oracle.ilu_factor(jac, mesh.vol, 0.8, rank)
    r = np.random.default_rng(6).normal(size=(n, 6)) + 1j * np.random.default_rng(7).normal(size=(n, 6))
    y = oracle.ilu_apply(jac, rank, F, r)
    A = _dense.dense_operator(jac.row_ptr, jac.col_idx, jac.offd, jac.diag, jac.D, mesh.vol, 0.8)
    x = np.linalg.solve(A, r.ravel())
    assert np.linalg.norm(y.ravel() - x) <= 1e-12 * np.linalg.norm(x)


def test_ilu_iteration_converges_to_direct_solve():
    mesh, jac, B, om = small_problem(dims=(4, 4, 3), block=6, n_harm=2)
    color = inputs.lattice_colors((4, 4, 3))
    X = oracle.ilu_iterate(jac, mesh.vol, om, B, 40, color)
    got = _dense.split_systems(X, len(om))
    bs = _dense.split_systems(B, len(om))
    for k, w in enumerate(_systems(jac, mesh.vol, om)):
        A = _dense.dense_operator(jac.row_ptr, jac.col_idx, jac.offd, jac.diag, jac.D, mesh.vol, w)
        xd = np.linalg.solve(A, bs[k])
        assert np.linalg.norm(got[k] - xd) <= 1e-12 * np.linalg.norm(xd)


def test_truncated_ilu0_factors_each_partition():
    """With partitions, ILU(0) of the matrix without cross-partition blocks."""
    dims = (6, 4, 3)
    mesh = inputs.hex_mesh(*dims, seed=8)
    q = inputs.flow_state(mesh.n_nodes, 5, seed=9)
    jac = oracle.build_jacobian(mesh.n_nodes, mesh.edge_nodes, mesh.normals, q, 20.0)
    part = inputs.box_partition(dims, (2, 2, 1))
    rank = oracle.elimination_rank(inputs.lattice_colors(dims))
    Fd, Fo = oracle.ilu_factor(jac, mesh.vol, 1.1, rank, part=part)
    L, U = _dense_lu(jac, rank, Fd, Fo, part=part)
    A = _dense.dense_operator(jac.row_ptr, jac.col_idx, jac.offd, jac.diag, jac.D, mesh.vol, 1.1)
    M = _pattern_mask(jac, mesh.n_nodes, 5, part=part)
    LU = L @ U
    assert np.abs((LU - A)[M]).max() <= 1e-12 * np.abs(A).max()
    # the factors never reach across partitions: L U is block diagonal by partition
    cross = np.repeat(part, 5)[:, None] != np.repeat(part, 5)[None, :]
    assert np.all(LU[cross] == 0.0)


def test_phase_lagged_ilu0_matches_ring():
    """ILU iterations on the phase-lagged passage equal them on the ring of
    passages (red-black colouring, even pitch), iteration by iteration."""
    mesh = inputs.hex_mesh(3, 4, 2, seed=11, periodic_y=True)
    q = inputs.flow_state(mesh.n_nodes, 6, seed=12)
    jac = oracle.build_jacobian(mesh.n_nodes, mesh.edge_nodes, mesh.normals, q, 20.0, periodic=mesh.periodic)
    N = len(RING_M)
    B = inputs.rhs(mesh.n_nodes, 6, N, seed=13)
    om = inputs.omegas(N, 0.9)
    sigma = 2.0 * np.pi * np.asarray(RING_M, dtype=np.float64) / RING_P
    P = RING_P
    n = mesh.n_nodes
    ren, rnorm, rvol, rq = ring_of_passages(mesh, q, P)
    rjac = oracle.build_jacobian(n * P, ren, rnorm, rq, 20.0)
    # colour by lattice parity (the pitch 4 is even, so the periodic edges join
    # different colours); every passage of the ring repeats the passage's
    # colours.  Nodes of one colour never couple, so the factors depend on the
    # colouring only, not on the order within a colour.
    color = inputs.lattice_colors((3, 4, 2))
    rcolor = np.tile(color, P)
    got = oracle.ilu_iterate(jac, mesh.vol, om, B, 3, color, sigma=sigma)
    ring = oracle.ilu_iterate(rjac, rvol, om, phase_shift(B, N, sigma, P), 3, rcolor)
    ref = phase_shift(got, N, sigma, P)
    assert np.allclose(ring, ref, rtol=0, atol=1e-11 * np.abs(ref).max())

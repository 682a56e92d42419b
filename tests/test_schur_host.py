"""The per-node basis change of the sweeps (Householder Hessenberg reduction
followed by the Francis double-shift QR iteration to a real Schur form, and
the FP32-seeded eigenvector basis of the frozen-turbulence blocks), compiled
as host code and checked against numpy (CPU only)."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2404_01407_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def schur_exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("schur") / "schur_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "schur_check.cu")], check=True)
    return exe


def run(exe, mats, mode="francis"):
    b = mats[0].shape[0]
    text = f"{len(mats)}\n" + "\n".join(" ".join(f"{v:.17g}" for v in m.ravel()) for m in mats) + "\n"
    out = subprocess.run([exe, mode], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    res = []
    for line in out[: len(mats)]:
        v = np.array(line.split(), dtype=float)
        res.append((bool(v[0]), v[1:1 + b * b].reshape(b, b), v[1 + b * b:].reshape(b, b)))
    return res


def test_real_spectra_reach_triangular_form(schur_exe):
    rng = np.random.default_rng(0)
    mats = []
    for _ in range(200):
        V = rng.normal(size=(6, 6)) + 3 * np.eye(6)
        lam = rng.uniform(-2, 5, 6)
        mats.append(V @ np.diag(lam) @ np.linalg.inv(V))
    for A, (ok, T, Z) in zip(mats, run(schur_exe, mats)):
        assert ok
        assert np.allclose(Z.T @ Z, np.eye(6), atol=1e-13)
        assert np.allclose(Z.T @ A @ Z, T, atol=1e-12 * np.abs(A).max())
        assert np.all(np.tril(T, -1) == 0.0)
        assert np.allclose(np.sort(np.diag(T)), np.sort(np.linalg.eigvals(A).real), atol=1e-9)


def test_complex_pairs_are_reported(schur_exe):
    rng = np.random.default_rng(1)
    mats = []
    for _ in range(50):
        V = rng.normal(size=(6, 6)) + 3 * np.eye(6)
        D = np.diag(rng.uniform(1, 3, 6))
        D[2:4, 2:4] = [[1.0, 2.0], [-2.0, 1.0]]  # eigenvalues 1 +- 2i
        mats.append(V @ D @ np.linalg.inv(V))
    for A, (ok, T, Z) in zip(mats, run(schur_exe, mats)):
        assert not ok
        # still an orthogonal similarity
        assert np.allclose(Z.T @ Z, np.eye(6), atol=1e-12)
        assert np.allclose(Z.T @ A @ Z, T, atol=1e-11 * np.abs(A).max())


def test_fnlh_diagonal_blocks(schur_exe):
    """The method's own diagonal blocks J_ii + D_i I (6x6 with turbulence row)."""
    p = inputs.problem((8, 6, 5), 6, 2, 20.0)
    m = p.mesh
    jac = oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl)
    mats = [jac.diag[i] + jac.D[i] * np.eye(6) for i in range(m.n_nodes)]
    for A, (ok, T, Z) in zip(mats, run(schur_exe, mats)):
        assert ok
        assert np.allclose(Z.T @ A @ Z, T, atol=1e-13 * np.abs(A).max())


# ---------------------------------------------------------------- eigenvector basis (5 x 5)


def similar(rng, lam):
    V = rng.normal(size=(len(lam), len(lam))) + 3 * np.eye(len(lam))
    return V @ np.diag(lam) @ np.linalg.inv(V)


def check_basis(A, T, Q):
    """What the sweeps rely on: Q orthogonal, Q^T A Q = T, T upper triangular
    with exact zeros below the diagonal."""
    assert np.abs(Q.T @ Q - np.eye(5)).max() <= 1e-14
    assert np.abs(Q.T @ A @ Q - T).max() <= 1e-13 * np.abs(A).max()
    assert np.all(np.tril(T, -1) == 0.0)


def test_eigvec_basis_of_real_spectra(schur_exe):
    rng = np.random.default_rng(2)
    mats = [similar(rng, rng.uniform(-2, 5, 5)) for _ in range(300)]
    res = run(schur_exe, mats, "eigvec")
    assert sum(ok for ok, _, _ in res) >= 295  # a rare near-defective draw may go to the FP64 iteration
    for A, (ok, T, Q) in zip(mats, res):
        if ok:
            check_basis(A, T, Q)
            assert np.allclose(np.sort(np.diag(T)), np.sort(np.linalg.eigvals(A).real), atol=1e-9)


def test_eigvec_basis_diagonal_and_triangular_inputs(schur_exe):
    """Already-triangular inputs: the basis is a signed permutation of the axes
    or close to it, and T carries the same eigenvalues."""
    rng = np.random.default_rng(3)
    mats = [np.diag([3.0, 1.0, 2.0, 5.0, 4.0]), np.triu(rng.normal(size=(5, 5))) + np.diag([1.0, 2, 3, 4, 5])]
    for A, (ok, T, Q) in zip(mats, run(schur_exe, mats, "eigvec")):
        assert ok
        check_basis(A, T, Q)
        assert np.allclose(np.sort(np.diag(T)), np.sort(np.diag(A)), atol=1e-12)


def test_eigvec_basis_rejects_complex_pairs(schur_exe):
    rng = np.random.default_rng(4)
    mats = []
    for _ in range(40):
        V = rng.normal(size=(5, 5)) + 3 * np.eye(5)
        D = np.diag(rng.uniform(1, 3, 5))
        D[1:3, 1:3] = [[1.0, 0.5], [-0.5, 1.0]]  # eigenvalues 1 +- 0.5i
        mats.append(V @ D @ np.linalg.inv(V))
    assert not any(ok for ok, _, _ in run(schur_exe, mats, "eigvec"))


def test_eigvec_basis_defective_block_never_accepted_wrong(schur_exe):
    """A Jordan block (one eigenvector for a double eigenvalue) has no
    eigenvector basis: the routine must either decline or still return an
    exact Schur basis."""
    rng = np.random.default_rng(5)
    mats = []
    for _ in range(40):
        V = rng.normal(size=(5, 5)) + 3 * np.eye(5)
        Jm = np.diag([1.5, 1.5, 2.5, 3.0, 4.0])
        Jm[0, 1] = 1.0
        mats.append(V @ Jm @ np.linalg.inv(V))
    for A, (ok, T, Q) in zip(mats, run(schur_exe, mats, "eigvec")):
        if ok:
            check_basis(A, T, Q)


def test_francis_fp32_reaches_triangular_form(schur_exe):
    """The FP32 instance of the Francis iteration (the eigenvector basis's
    first step): eigenvalues to FP32 accuracy, orthogonal Z to FP32."""
    rng = np.random.default_rng(6)
    mats = [similar(rng, rng.uniform(1, 4, 5)) for _ in range(100)]
    for A, (ok, T, Z) in zip(mats, run(schur_exe, mats, "francis32")):
        assert ok
        assert np.abs(Z.T @ Z - np.eye(5)).max() <= 1e-5
        assert np.all(np.tril(T, -1) == 0.0)
        lam = np.sort(np.linalg.eigvals(A).real)
        assert np.allclose(np.sort(np.diag(T)), lam, atol=1e-4 * np.abs(lam).max())


@pytest.mark.parametrize("dims,n_harm,cfl,seeds", [((8, 6, 5), 2, 20.0, (11, 12, 13)),
                                                   ((12, 8, 6), 8, 20.0, (4, 5, 6)),
                                                   ((16, 8, 8), 1, 10.0, (1, 2, 3))])
def test_eigvec_basis_of_fnlh_mean_flow_blocks(schur_exe, dims, n_harm, cfl, seeds):
    """The blocks the prepare step gives it: the 5 x 5 mean-flow part of
    J_ii + D_i I on the method's own Jacobians.  Every block is accepted and
    exact (the sweeps' parity with the oracle rests on this basis)."""
    p = inputs.problem(dims, 6, n_harm, cfl, seeds=seeds)
    m = p.mesh
    jac = oracle.build_jacobian(m.n_nodes, m.edge_nodes, m.normals, p.q, p.cfl)
    mats = [(jac.diag[i] + jac.D[i] * np.eye(6))[:5, :5].copy() for i in range(m.n_nodes)]
    for A, (ok, T, Q) in zip(mats, run(schur_exe, mats, "eigvec")):
        assert ok
        check_basis(A, T, Q)

"""The per-node basis change of the sweeps (Householder Hessenberg reduction
followed by the Francis double-shift QR iteration to a real Schur form),
compiled as host code and checked against numpy (CPU only)."""

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


def run(exe, mats):
    text = f"{len(mats)}\n" + "\n".join(" ".join(f"{v:.17g}" for v in m.ravel()) for m in mats) + "\n"
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    res = []
    for line in out[: len(mats)]:
        v = np.array(line.split(), dtype=float)
        res.append((bool(v[0]), v[1:37].reshape(6, 6), v[37:].reshape(6, 6)))
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

"""Dense / sparse assemblies used by the oracle pins (test helpers).

These build the systems of Eq. precon_linear / Eq. lhs_lin as explicit
matrices from a set of blocks, so that the oracle's sweep and residual loops
can be checked against library linear algebra (numpy / scipy) instead of
against themselves.
"""

import numpy as np
import scipy.sparse as sp


def split_systems(X, n_harm):
    """[n][C][b] real -> list of K complex vectors (mean first), each [n*b]."""
    out = [X[:, 0, :].astype(np.complex128).ravel()]
    for k in range(1, n_harm + 1):
        out.append((X[:, 2 * k - 1, :] + 1j * X[:, 2 * k, :]).ravel())
    return out


def join_systems(xs, n, b):
    n_harm = len(xs) - 1
    X = np.zeros((n, 1 + 2 * n_harm, b))
    X[:, 0, :] = xs[0].real.reshape(n, b)
    for k in range(1, n_harm + 1):
        X[:, 2 * k - 1, :] = xs[k].real.reshape(n, b)
        X[:, 2 * k, :] = xs[k].imag.reshape(n, b)
    return X


def dense_operator(row_ptr, col_idx, offd, diag, D, vol, omega_k):
    """A_k = J + D I + i omega_k V I as a dense complex matrix."""
    n, b = diag.shape[0], diag.shape[1]
    A = np.zeros((n * b, n * b), dtype=np.complex128)
    eye = np.eye(b)
    for i in range(n):
        A[i * b:(i + 1) * b, i * b:(i + 1) * b] = diag[i] + (D[i] + 1j * omega_k * vol[i]) * eye
        for p in range(row_ptr[i], row_ptr[i + 1]):
            j = col_idx[p]
            A[i * b:(i + 1) * b, j * b:(j + 1) * b] = offd[p]
    return A


def block_split(row_ptr, col_idx, offd, diag, D, vol, omega_k):
    """(M, N) with A = M + N, M block diagonal, N the off-diagonal blocks (dense)."""
    n, b = diag.shape[0], diag.shape[1]
    A = dense_operator(row_ptr, col_idx, offd, diag, D, vol, omega_k)
    M = np.zeros_like(A)
    for i in range(n):
        M[i * b:(i + 1) * b, i * b:(i + 1) * b] = A[i * b:(i + 1) * b, i * b:(i + 1) * b]
    return M, A - M


def sparse_operator(row_ptr, col_idx, offd, diag, D, vol, omega_k):
    n, b = diag.shape[0], diag.shape[1]
    rows, cols, vals = [], [], []
    ii, jj = np.meshgrid(np.arange(b), np.arange(b), indexing="ij")
    eye = np.eye(b)
    for i in range(n):
        blk = diag[i] + (D[i] + 1j * omega_k * vol[i]) * eye
        rows.append((i * b + ii).ravel()); cols.append((i * b + jj).ravel()); vals.append(blk.ravel())
    rp = np.asarray(row_ptr)
    owner = np.repeat(np.arange(n), np.diff(rp))
    for p in range(len(col_idx)):
        i, j = owner[p], col_idx[p]
        rows.append((i * b + ii).ravel()); cols.append((j * b + jj).ravel())
        vals.append(np.asarray(offd[p], dtype=np.complex128).ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n * b, n * b))

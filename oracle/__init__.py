"""CPU FP64 oracle for the shared-Jacobian FNLH linear systems.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the library never does.

The arithmetic lives in ``fnlh_oracle.c`` (plain C, FP64, no FMA contraction,
OpenMP over rows only); this module compiles it with gcc on first use and
wraps it with ctypes.  Paper: arXiv 2404.01407 -- the implicit LHS of
Eq. precon, its harmonic form Eq. precon_linear / Eq. lhs_lin, the block-Jacobi
inversion of "Solution Update" and the linear residual of the Results
section's stopping rule.  The readings taken where the paper is silent are
listed at the top of ``fnlh_oracle.c``.

Parity pins (tests/test_oracle_pins.py) tie every function here to something
other than itself: the textbook Euler flux Jacobian and its eigenvalues, an
eigendecomposition of |A|, complex-step derivatives of a frozen-dissipation
first-order residual, closed forms on a uniform state, dense direct solves,
the real 2x2-block form of Eq. matrix_z_real, hand-solvable one- and
two-node systems, and (phase-lagged periodic edges) the equivalence of one
passage with phase lag to a ring of passages with plain periodicity.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fnlh_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GAMMA = 1.4
DELTA = 0.1
EPS = 0.6

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    lib.oracle_flux_jacobian.argtypes = [ctypes.c_int, _f64p, _f64p, ctypes.c_double, _f64p]
    lib.oracle_flux_jacobian.restype = None
    lib.oracle_abs_jacobian.argtypes = [ctypes.c_int, _f64p, _f64p, ctypes.c_double,
                                        ctypes.c_double, _f64p]
    lib.oracle_abs_jacobian.restype = None
    lib.oracle_spectral_radius.argtypes = [_f64p, _f64p, ctypes.c_double]
    lib.oracle_spectral_radius.restype = ctypes.c_double
    lib.oracle_build_jacobian.argtypes = [
        ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p, _f64p, _f64p, ctypes.c_double,
        ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double, _i32p, _i32p,
        _f64p, _f64p, _f64p]
    lib.oracle_build_jacobian.restype = ctypes.c_int
    lib.oracle_phase_sides.argtypes = [ctypes.c_int, ctypes.c_int, _i32p, _i8p, _i32p, _i8p]
    lib.oracle_phase_sides.restype = ctypes.c_int
    # n, b, n_harm, row_ptr, col_idx, offd, diag, D, vol, omega, side, sigma, B
    common = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _f64p,
              _f64p, _f64p, ctypes.c_void_p, ctypes.c_void_p, _f64p]
    lib.oracle_jacobi.argtypes = common + [_f64p, ctypes.c_int, ctypes.c_void_p]
    lib.oracle_jacobi.restype = ctypes.c_int
    lib.oracle_residual.argtypes = common + [_f64p, ctypes.c_void_p, _f64p]
    lib.oracle_residual.restype = ctypes.c_int
    lib.oracle_ilu_factor.argtypes = [ctypes.c_int, ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p,
                                      ctypes.c_double, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, _i32p,
                                      _f64p, _f64p]
    lib.oracle_ilu_factor.restype = ctypes.c_int
    lib.oracle_ilu_apply.argtypes = [ctypes.c_int, ctypes.c_int, _i32p, _i32p, ctypes.c_void_p, _i32p, _f64p, _f64p,
                                     _f64p, _f64p]
    lib.oracle_ilu_apply.restype = ctypes.c_int
    lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_num_threads.restype = None
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = ctypes.c_int
    return lib


def use_library(path):
    """Swap the loaded oracle for another build of ``fnlh_oracle.c`` (the
    mutation tests load deliberately broken copies); returns the previous
    library handle so that it can be restored with :func:`restore_library`."""
    global _lib
    prev = _load()
    with _lock:
        _lib = _bind(ctypes.CDLL(path))
    return prev


def restore_library(handle):
    global _lib
    with _lock:
        _lib = handle


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """OpenMP threads of the oracle's row loops (timing only; results do not depend on it)."""
    _load().oracle_set_num_threads(int(n))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def flux_jacobian(q, n, gamma: float = GAMMA) -> np.ndarray:
    """A(Q, n) = d(F(Q).n)/dQ (complex-step)."""
    q = _f64(q)
    b = q.shape[0]
    out = np.zeros(b * b)
    _load().oracle_flux_jacobian(b, q, _f64(n), gamma, out)
    return out.reshape(b, b)


def abs_jacobian(q, n, gamma: float = GAMMA, delta: float = DELTA) -> np.ndarray:
    """|A|(Q, n) with the entropy fix (Sylvester's formula)."""
    q = _f64(q)
    b = q.shape[0]
    out = np.zeros(b * b)
    _load().oracle_abs_jacobian(b, q, _f64(n), gamma, delta, out)
    return out.reshape(b, b)


def spectral_radius(q, n, gamma: float = GAMMA) -> float:
    return float(_load().oracle_spectral_radius(_f64(q), _f64(n), gamma))


class Jacobian:
    """Oracle Jacobian: CSR pattern, off-diagonal and diagonal blocks, D, and
    (periodic meshes) the passage offset `side` [nnz] of every CSR entry."""

    def __init__(self, row_ptr, col_idx, offd, diag, D, block, side=None):
        self.row_ptr, self.col_idx, self.offd, self.diag, self.D = row_ptr, col_idx, offd, diag, D
        self.block = block
        self.side = side

    @property
    def n_nodes(self):
        return int(self.D.shape[0])

    @property
    def nnz(self):
        return int(self.col_idx.shape[0])


def phase_sides(n_nodes, edge_nodes, periodic) -> np.ndarray:
    """Passage offset (-1, 0, +1) of the neighbour of every CSR entry, from the
    per-edge offsets of the edges' second nodes."""
    en = np.ascontiguousarray(edge_nodes, dtype=np.int32).reshape(-1, 2)
    E = en.shape[0]
    per = np.ascontiguousarray(periodic, dtype=np.int8).reshape(E)
    row_ptr = np.zeros(n_nodes + 1, dtype=np.int32)
    side = np.zeros(max(2 * E, 1), dtype=np.int8)
    rc = _load().oracle_phase_sides(n_nodes, E, en.ravel(), per if E else np.zeros(1, np.int8), row_ptr, side)
    if rc != 0:
        raise ValueError(f"oracle_phase_sides failed ({rc})")
    return side[: 2 * E].copy()


def build_jacobian(n_nodes, edge_nodes, normals, q, cfl, gamma=GAMMA, delta=DELTA,
                   pseudo_block=False, eps=EPS, periodic=None) -> Jacobian:
    """First-order edge Jacobian J, diagonal blocks and pseudo-time diagonal D
    (periodic: per-edge passage offsets of a phase-lagged periodic mesh)."""
    q = _f64(q)
    b = q.shape[1]
    en = np.ascontiguousarray(edge_nodes, dtype=np.int32).reshape(-1, 2)
    E = en.shape[0]
    row_ptr = np.zeros(n_nodes + 1, dtype=np.int32)
    col_idx = np.zeros(max(2 * E, 1), dtype=np.int32)
    offd = np.zeros(max(2 * E, 1) * b * b)
    diag = np.zeros(n_nodes * b * b)
    D = np.zeros(n_nodes)
    rc = _load().oracle_build_jacobian(n_nodes, E, b, en.ravel(), _f64(normals).ravel(), q.ravel(),
                                      gamma, delta, cfl, int(bool(pseudo_block)), eps, row_ptr,
                                      col_idx, offd, diag, D)
    if rc != 0:
        raise ValueError(f"oracle_build_jacobian failed ({rc})")
    side = None if periodic is None else phase_sides(n_nodes, en, periodic)
    return Jacobian(row_ptr, col_idx[: 2 * E].copy(), offd[: 2 * E * b * b].reshape(2 * E, b, b),
                    diag.reshape(n_nodes, b, b), D, b, side)


def _sys_args(jac: Jacobian, vol, omega, sigma, keep):
    """Marshalled arguments; `keep` holds the arrays behind raw pointers."""
    b = jac.block
    offd = _f64(jac.offd).ravel()
    if offd.size == 0:
        offd = np.zeros(1)
    col = jac.col_idx if jac.col_idx.size else np.zeros(1, dtype=np.int32)
    n_harm = int(np.asarray(omega).shape[0])
    side_p = sigma_p = None
    if jac.side is not None and sigma is not None and n_harm > 0:
        side = np.ascontiguousarray(jac.side, dtype=np.int8)
        sig = _f64(np.atleast_1d(sigma))
        if sig.shape[0] != n_harm:
            raise ValueError("sigma needs one phase angle per harmonic")
        keep += [side, sig]
        side_p, sigma_p = side.ctypes.data_as(ctypes.c_void_p), sig.ctypes.data_as(ctypes.c_void_p)
    return (jac.n_nodes, b, n_harm, jac.row_ptr, col, offd, _f64(jac.diag).ravel(), _f64(jac.D), _f64(vol),
            _f64(np.atleast_1d(omega)) if len(omega) else np.zeros(1), side_p, sigma_p)


def jacobi(jac: Jacobian, vol, omega, B, sweeps: int, X0=None, sigma=None, part=None) -> np.ndarray:
    """x after `sweeps` undamped block-Jacobi sweeps from X0 (zero if None);
    sigma: inter-blade phase angle per harmonic (periodic meshes); part:
    partition id per node (couplings across partitions dropped)."""
    B = _f64(B)
    X = np.zeros_like(B) if X0 is None else _f64(X0).copy()
    keep = []
    part_p = None
    if part is not None:
        pa = np.ascontiguousarray(part, dtype=np.int32).reshape(jac.n_nodes)
        keep.append(pa)
        part_p = pa.ctypes.data_as(ctypes.c_void_p)
    rc = _load().oracle_jacobi(*_sys_args(jac, vol, omega, sigma, keep), B.ravel(), X.reshape(-1), int(sweeps),
                               part_p)
    if rc != 0:
        raise FloatingPointError("singular diagonal block")
    return X


def residual(jac: Jacobian, vol, omega, B, X, want_r: bool = False, sigma=None):
    """Returns (norms[K,2] = (||r_k||^2, ||B_k||^2), r or None)."""
    B = _f64(B)
    X = _f64(X)
    K = 1 + len(omega)
    norms = np.zeros(2 * K)
    r = np.zeros_like(B) if want_r else None
    rp = r.ctypes.data_as(ctypes.c_void_p) if want_r else None
    keep = []
    _load().oracle_residual(*_sys_args(jac, vol, omega, sigma, keep), B.ravel(), X.ravel(), rp, norms)
    return norms.reshape(K, 2), r


def rel_residuals(jac: Jacobian, vol, omega, B, X, sigma=None) -> np.ndarray:
    """||B_k - A_k x_k|| / ||B_k|| per system k (mean first)."""
    norms, _ = residual(jac, vol, omega, B, X, sigma=sigma)
    return np.sqrt(norms[:, 0] / np.maximum(norms[:, 1], 1e-300))


def solve_to_tol(jac: Jacobian, vol, omega, B, tol: float, chunk: int = 10, max_sweeps: int = 100000, sigma=None):
    """Plain FP64 Jacobi until every system's relative residual <= tol."""
    X = np.zeros_like(_f64(B))
    done = 0
    while done < max_sweeps:
        X = jacobi(jac, vol, omega, B, chunk, X0=X, sigma=sigma)
        done += chunk
        if np.all(rel_residuals(jac, vol, omega, B, X, sigma=sigma) <= tol):
            break
    return X, done


# ------------------------------------------------------------------ ILU(0)

def elimination_rank(color) -> np.ndarray:
    """Position of every node in the multicolour elimination order: all nodes of
    colour 0 by increasing id, then colour 1, ..."""
    color = np.asarray(color, dtype=np.int64)
    order = np.lexsort((np.arange(color.shape[0]), color))
    rank = np.empty(color.shape[0], dtype=np.int32)
    rank[order] = np.arange(color.shape[0], dtype=np.int32)
    return rank


def _ptr_or_none(arr, dtype, keep):
    if arr is None:
        return None
    a = np.ascontiguousarray(arr, dtype=dtype)
    keep.append(a)
    return a.ctypes.data_as(ctypes.c_void_p)


def ilu_factor(jac: Jacobian, vol, omega_k: float, rank, sigma_k: float = 0.0, part=None):
    """Block ILU(0) of one system (omega_k, phase angle sigma_k) in the order
    `rank`; returns (U_ii [n][b][b], L_ij or U_ij per CSR entry [nnz][b][b]),
    complex."""
    b, n = jac.block, jac.n_nodes
    keep = []
    Fd = np.zeros(max(n, 1) * b * b * 2)
    Fo = np.zeros(max(jac.nnz, 1) * b * b * 2)
    offd = _f64(jac.offd).ravel() if jac.nnz else np.zeros(1)
    col = jac.col_idx if jac.nnz else np.zeros(1, dtype=np.int32)
    rc = _load().oracle_ilu_factor(n, b, jac.row_ptr, col, offd, _f64(jac.diag).ravel(), _f64(jac.D), _f64(vol),
                                   float(omega_k), _ptr_or_none(jac.side, np.int8, keep), float(sigma_k),
                                   _ptr_or_none(part, np.int32, keep), np.ascontiguousarray(rank, dtype=np.int32),
                                   Fd, Fo)
    if rc != 0:
        raise FloatingPointError("ILU(0): zero pivot")
    Fd = Fd[: n * b * b * 2].view(np.complex128).reshape(n, b, b)
    Fo = Fo[: jac.nnz * b * b * 2].view(np.complex128).reshape(jac.nnz, b, b)
    return Fd, Fo


def ilu_apply(jac: Jacobian, rank, factors, r, part=None) -> np.ndarray:
    """y = (L U)^-1 r for one system's factors; r complex [n][b]."""
    b, n = jac.block, jac.n_nodes
    keep = []
    Fd, Fo = factors
    rr = np.ascontiguousarray(r, dtype=np.complex128).reshape(n * b)
    y = np.zeros(n * b, dtype=np.complex128)
    col = jac.col_idx if jac.nnz else np.zeros(1, dtype=np.int32)
    fo = Fo.view(np.float64).ravel() if jac.nnz else np.zeros(2)
    rc = _load().oracle_ilu_apply(n, b, jac.row_ptr, col, _ptr_or_none(part, np.int32, keep),
                                  np.ascontiguousarray(rank, dtype=np.int32), np.ascontiguousarray(Fd).view(np.float64).ravel(),
                                  np.ascontiguousarray(fo), rr.view(np.float64), y.view(np.float64))
    if rc != 0:
        raise FloatingPointError("ILU(0): singular pivot block")
    return y.reshape(n, b)


def ilu_iterate(jac: Jacobian, vol, omega, B, iterations: int, color, X0=None, sigma=None, part=None):
    """`iterations` ILU(0) iterations x <- x + (L U)^-1 (B - A x) on every system
    (mean flow and harmonics), in the multicolour order of `color`; the
    residual keeps every coupling, the factors drop the cross-partition ones."""
    B = _f64(B)
    X = np.zeros_like(B) if X0 is None else _f64(X0).copy()
    rank = elimination_rank(color)
    n_harm = len(omega)
    sig = np.zeros(n_harm) if sigma is None else np.asarray(sigma, dtype=np.float64)
    facs = [ilu_factor(jac, vol, 0.0, rank, 0.0, part)]
    facs += [ilu_factor(jac, vol, omega[l], rank, sig[l], part) for l in range(n_harm)]
    for _ in range(iterations):
        _, r = residual(jac, vol, omega, B, X, want_r=True, sigma=sigma)
        y0 = ilu_apply(jac, rank, facs[0], r[:, 0, :].astype(np.complex128), part)
        X[:, 0, :] += y0.real
        for l in range(1, n_harm + 1):
            y = ilu_apply(jac, rank, facs[l], r[:, 2 * l - 1, :] + 1j * r[:, 2 * l, :], part)
            X[:, 2 * l - 1, :] += y.real
            X[:, 2 * l, :] += y.imag
    return X

"""ctypes binding of libfnlh.so -- argument marshalling only.

Every function named ``fnlh_*`` here calls the C entry point of the same
name (declared in include/fnlh.h) with the device pointers of the torch
tensors it is given and raises :class:`FnlhError` on a non-zero status.  All
arithmetic of the path runs in the library's CUDA kernels; PyTorch only
provides device memory and streams.  There is no CPU fallback: without the
compiled library, :func:`lib` raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

c_i32 = ctypes.c_int32
c_f64 = ctypes.c_double
c_vp = ctypes.c_void_p
c_sz = ctypes.c_size_t

FNLH_OK = 0
FNLH_ERR_ARG = -1
FNLH_ERR_CUDA = -2
FNLH_ERR_NONFINITE = -3
FNLH_ERR_DIVERGED = -4
FNLH_ERR_TIMEOUT = -5
FNLH_ERR_UNSUPPORTED = -6
FNLH_ERR_WORKSPACE = -7
FNLH_ERR_NOT_CONVERGED = -8
FNLH_ERR_BAD_MESH = -9

FNLH_F64, FNLH_F32, FNLH_BF16 = 0, 1, 2
FNLH_PREP_F64, FNLH_PREP_F32, FNLH_PREP_BF16, FNLH_PREP_TAGS, FNLH_PREP_FF = 1, 2, 4, 8, 16
PRECISIONS = {"f64": FNLH_F64, "f32": FNLH_F32, "bf16": FNLH_BF16}
PREP_FOR = {FNLH_F64: FNLH_PREP_F64, FNLH_F32: FNLH_PREP_F32, FNLH_BF16: FNLH_PREP_BF16}
MAX_HARMONICS = 64


class fnlh_mesh(ctypes.Structure):
    _fields_ = [("n_nodes", c_i32), ("n_edges", c_i32), ("edge_nodes", c_vp), ("normals", c_vp),
                ("vol", c_vp), ("row_ptr", c_vp), ("col_idx", c_vp), ("csr_edge", c_vp), ("periodic", c_vp),
                ("part", c_vp)]


class fnlh_params(ctypes.Structure):
    _fields_ = [("gamma", c_f64), ("cfl", c_f64), ("entropy_delta", c_f64), ("pseudo_time", c_i32),
                ("eps", c_f64)]


class fnlh_jacobian(ctypes.Structure):
    _fields_ = [("n_nodes", c_i32), ("nnz", c_i32), ("block", c_i32), ("offd", c_vp), ("diag", c_vp),
                ("D", c_vp), ("prep", c_vp), ("prep_bytes", c_sz), ("prep_flags", c_i32),
                ("prep_ready", c_i32)]


class fnlh_row(ctypes.Structure):
    _fields_ = [("mesh", ctypes.POINTER(fnlh_mesh)), ("J", ctypes.POINTER(fnlh_jacobian)),
                ("n_harm", c_i32), ("omega", ctypes.POINTER(c_f64)), ("B", c_vp), ("X", c_vp),
                ("sigma", ctypes.POINTER(c_f64))]


class fnlh_ilu(ctypes.Structure):
    _fields_ = [("n_colors", c_i32), ("color", c_vp), ("order", c_vp), ("color_ptr", ctypes.POINTER(c_i32)),
                ("factor", c_vp), ("factor_bytes", c_sz), ("precision", c_i32), ("n_harm", c_i32), ("ready", c_i32)]


class fnlh_tuning(ctypes.Structure):
    _fields_ = [("threads", c_i32), ("ctas_per_sm", c_i32), ("reserved", c_i32 * 2)]


FNLH_TUNING_PER_ROW = -1  # fnlh_tuning.ctas_per_sm: every row its own single-row launches


class FnlhError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {lib().fnlh_strerror(status).decode()} ({status})")


_lock = threading.Lock()
_lib = None

# C declarations: name -> (restype, argtypes)
_SIGS = {
    "fnlh_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "fnlh_version": (ctypes.c_int, []),
    "fnlh_mesh_build_csr": (ctypes.c_int, [c_i32, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "fnlh_prep_bytes": (c_sz, [c_i32, c_i32, c_i32, c_i32]),
    "fnlh_workspace_bytes": (c_sz, [c_i32, c_i32, c_i32, c_i32]),
    "fnlh_solve_workspace_bytes": (c_sz, [c_i32, c_i32, c_i32, c_i32, c_i32]),
    "fnlh_build_jacobian": (ctypes.c_int, [ctypes.POINTER(fnlh_mesh), c_vp, ctypes.POINTER(fnlh_params),
                                           ctypes.POINTER(fnlh_jacobian), c_vp]),
    "fnlh_prepare": (ctypes.c_int, [ctypes.POINTER(fnlh_mesh), ctypes.POINTER(fnlh_jacobian), c_vp]),
    "fnlh_relax": (ctypes.c_int, [ctypes.POINTER(fnlh_mesh), ctypes.POINTER(fnlh_jacobian), c_i32,
                                  ctypes.POINTER(c_f64), ctypes.POINTER(c_f64), c_vp, c_vp, c_i32, c_i32, c_vp, c_sz,
                                  c_vp]),
    "fnlh_residual": (ctypes.c_int, [ctypes.POINTER(fnlh_mesh), ctypes.POINTER(fnlh_jacobian), c_i32,
                                     ctypes.POINTER(c_f64), ctypes.POINTER(c_f64), c_vp, c_vp, c_vp, c_vp, c_vp, c_sz,
                                     c_vp]),
    "fnlh_solve": (ctypes.c_int, [ctypes.POINTER(fnlh_mesh), ctypes.POINTER(fnlh_jacobian), c_i32,
                                  ctypes.POINTER(c_f64), ctypes.POINTER(c_f64), c_vp, c_vp, c_i32, c_f64, c_i32, c_i32,
                                  c_i32, c_vp, c_sz,
                                  ctypes.POINTER(c_i32), ctypes.POINTER(c_i32), ctypes.POINTER(c_f64), c_vp]),
    "fnlh_relax_batched": (ctypes.c_int, [ctypes.POINTER(fnlh_row), c_i32, c_i32, c_i32,
                                          ctypes.POINTER(fnlh_tuning), c_vp, c_sz, c_vp]),
    "fnlh_batched_extra_bytes": (c_sz, [c_i32]),
    "fnlh_solve_batched": (ctypes.c_int, [ctypes.POINTER(fnlh_row), c_i32, c_i32, c_f64, c_i32, c_i32, c_i32,
                                          ctypes.POINTER(fnlh_tuning), c_vp, c_sz, ctypes.POINTER(c_i32),
                                          ctypes.POINTER(c_i32), ctypes.POINTER(c_f64), c_vp]),
    "fnlh_set_sweep_events": (ctypes.c_int, [c_vp, c_vp]),
    "fnlh_prep_structured": (ctypes.c_int, [ctypes.POINTER(fnlh_jacobian), ctypes.POINTER(c_i32), c_vp]),
    "fnlh_mesh_color": (ctypes.c_int, [c_i32, c_vp, c_vp, c_i32, c_vp, c_vp, c_vp, ctypes.POINTER(c_i32)]),
    "fnlh_ilu_bytes": (c_sz, [c_i32, c_i32, c_i32, c_i32]),
    "fnlh_ilu_factor": (ctypes.c_int, [ctypes.POINTER(fnlh_mesh), ctypes.POINTER(fnlh_jacobian), c_i32,
                                       ctypes.POINTER(c_f64), ctypes.POINTER(fnlh_ilu), c_vp, c_sz, c_vp]),
    "fnlh_solve_ilu": (ctypes.c_int, [ctypes.POINTER(fnlh_mesh), ctypes.POINTER(fnlh_jacobian),
                                      ctypes.POINTER(fnlh_ilu), c_i32, ctypes.POINTER(c_f64), ctypes.POINTER(c_f64),
                                      c_vp, c_vp, c_f64, c_i32, c_i32, c_vp, c_sz, ctypes.POINTER(c_i32),
                                      ctypes.POINTER(c_f64), c_vp]),
    "fnlh_residual_noalloc": (ctypes.c_int, [ctypes.POINTER(fnlh_mesh), ctypes.POINTER(fnlh_jacobian), c_i32,
                                             ctypes.POINTER(c_f64), ctypes.POINTER(c_f64), c_vp, c_vp, c_vp, c_vp,
                                             c_vp]),
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """The loaded libfnlh.so (built in-tree on first use when nvcc is present)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libfnlh.so is not built; the FNLH path has no CPU fallback")
            h = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(h, name)
                fn.restype = res
                fn.argtypes = args
            _lib = h
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status: int, where: str):
    if status != FNLH_OK:
        raise FnlhError(status, where)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if t.numel() == 0:
            return None
        return c_vp(t.data_ptr())
    return t


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return c_vp(stream.cuda_stream)


def _omega(omega):
    arr = np.ascontiguousarray(np.atleast_1d(np.asarray(omega, dtype=np.float64)))
    if arr.size == 0:
        arr = np.zeros(1)
    return arr, arr.ctypes.data_as(ctypes.POINTER(c_f64))


def _sigma(sigma, n_harm):
    """Host phase-angle array (kept alive by the caller) and its pointer, or
    (None, None) for plain periodicity."""
    if sigma is None:
        return None, None
    arr = np.ascontiguousarray(np.atleast_1d(np.asarray(sigma, dtype=np.float64)))
    if arr.shape[0] != n_harm:
        raise ValueError("sigma needs one phase angle per harmonic")
    if arr.size == 0:
        return None, None
    return arr, arr.ctypes.data_as(ctypes.POINTER(c_f64))


# ------------------------------------------------------------------ objects

class DeviceMesh:
    """Mesh arrays on the device plus the ctypes fnlh_mesh describing them."""

    def __init__(self, n_nodes, edge_nodes, normals, vol, device="cuda", periodic=None, part=None):
        en = np.ascontiguousarray(edge_nodes, dtype=np.int32).reshape(-1, 2)
        n_edges = en.shape[0]
        row_ptr = np.zeros(n_nodes + 1, dtype=np.int32)
        col_idx = np.zeros(max(2 * n_edges, 1), dtype=np.int32)
        csr_edge = np.zeros(max(2 * n_edges, 1), dtype=np.int32)
        fnlh_mesh_build_csr(n_nodes, n_edges, en, row_ptr, col_idx, csr_edge)
        self.n_nodes, self.n_edges = int(n_nodes), int(n_edges)
        self.row_ptr_host, self.col_idx_host = row_ptr, col_idx[: 2 * n_edges]
        dev = torch.device(device)
        self.edge_nodes = torch.from_numpy(en).to(dev)
        self.normals = torch.from_numpy(np.ascontiguousarray(normals, dtype=np.float64).reshape(-1, 3)).to(dev)
        self.vol = torch.from_numpy(np.ascontiguousarray(vol, dtype=np.float64)).to(dev)
        self.row_ptr = torch.from_numpy(row_ptr).to(dev)
        self.col_idx = torch.from_numpy(col_idx[: 2 * n_edges].copy()).to(dev)
        self.csr_edge = torch.from_numpy(csr_edge[: 2 * n_edges].copy()).to(dev)
        self.periodic = None
        if periodic is not None:
            per = np.ascontiguousarray(periodic, dtype=np.int8).reshape(n_edges)
            self.periodic = torch.from_numpy(per).to(dev) if n_edges else None
        self.part = None
        if part is not None:
            self.part = torch.from_numpy(np.ascontiguousarray(part, dtype=np.int32).reshape(n_nodes)).to(dev)
        self.c = fnlh_mesh(self.n_nodes, self.n_edges, _ptr(self.edge_nodes), _ptr(self.normals), _ptr(self.vol),
                           _ptr(self.row_ptr), _ptr(self.col_idx), _ptr(self.csr_edge), _ptr(self.periodic),
                           _ptr(self.part))

    @classmethod
    def from_mesh(cls, mesh, device="cuda", part=None):
        """part: partition id per node (domain-truncated sweeps), or None."""
        return cls(mesh.n_nodes, mesh.edge_nodes, mesh.normals, mesh.vol, device,
                   periodic=getattr(mesh, "periodic", None), part=part)


class DeviceJacobian:
    """J, D and the derived prep blob, all caller-owned torch tensors."""

    def __init__(self, dmesh: DeviceMesh, block: int, prep_flags: int = FNLH_PREP_F64, device="cuda"):
        n, nnz = dmesh.n_nodes, 2 * dmesh.n_edges
        dev = torch.device(device)
        self.block = block
        self.offd = torch.empty((nnz, block, block), dtype=torch.float64, device=dev)
        self.diag = torch.empty((n, block, block), dtype=torch.float64, device=dev)
        self.D = torch.empty((n,), dtype=torch.float64, device=dev)
        nbytes = fnlh_prep_bytes(n, nnz, block, prep_flags) if prep_flags else 0
        self.prep = torch.empty((max(nbytes, 1),), dtype=torch.uint8, device=dev) if prep_flags else None
        self.c = fnlh_jacobian(n, nnz, block, _ptr(self.offd), _ptr(self.diag), _ptr(self.D),
                               _ptr(self.prep) if self.prep is not None else None, nbytes, prep_flags, 0)

    def nbytes(self):
        t = self.offd.numel() * 8 + self.diag.numel() * 8 + self.D.numel() * 8
        return t + (self.prep.numel() if self.prep is not None else 0)


def make_params(cfl, gamma=1.4, entropy_delta=0.1, pseudo_time=0, eps=0.6):
    return fnlh_params(gamma, cfl, entropy_delta, pseudo_time, eps)


def workspace(n_nodes, block, n_harm, device="cuda", precision=FNLH_F64):
    nbytes = fnlh_workspace_bytes(n_nodes, block, n_harm, precision)
    return torch.empty((nbytes,), dtype=torch.uint8, device=device)


def solve_workspace(n_nodes, block, n_harm, prep_flags, device="cuda", precision=FNLH_F64):
    """Workspace for fnlh_solve, with room for the float-float checks when
    prep_flags holds FNLH_PREP_FF and the precision is mixed."""
    nbytes = fnlh_solve_workspace_bytes(n_nodes, block, n_harm, precision, prep_flags)
    return torch.empty((nbytes,), dtype=torch.uint8, device=device)


# ------------------------------------------------------- C entry points

def fnlh_version() -> int:
    return int(lib().fnlh_version())


def fnlh_strerror(status: int) -> str:
    return lib().fnlh_strerror(status).decode()


def fnlh_mesh_build_csr(n_nodes, n_edges, edge_nodes, row_ptr, col_idx, csr_edge):
    en = np.ascontiguousarray(edge_nodes, dtype=np.int32)
    st = lib().fnlh_mesh_build_csr(n_nodes, n_edges, en.ctypes.data_as(c_vp), row_ptr.ctypes.data_as(c_vp),
                                   col_idx.ctypes.data_as(c_vp), csr_edge.ctypes.data_as(c_vp))
    _check(st, "fnlh_mesh_build_csr")


def fnlh_prep_bytes(n_nodes, nnz, block, prep_flags) -> int:
    return int(lib().fnlh_prep_bytes(n_nodes, nnz, block, prep_flags))


def fnlh_workspace_bytes(n_nodes, block, n_harm, precision=FNLH_F64) -> int:
    return int(lib().fnlh_workspace_bytes(n_nodes, block, n_harm, precision))


def fnlh_solve_workspace_bytes(n_nodes, block, n_harm, precision, prep_flags) -> int:
    return int(lib().fnlh_solve_workspace_bytes(n_nodes, block, n_harm, precision, prep_flags))


def fnlh_build_jacobian(dmesh: DeviceMesh, Q: torch.Tensor, params: fnlh_params, J: DeviceJacobian, stream=None):
    st = lib().fnlh_build_jacobian(ctypes.byref(dmesh.c), _ptr(Q), ctypes.byref(params), ctypes.byref(J.c),
                                   _stream(stream))
    _check(st, "fnlh_build_jacobian")


def fnlh_prepare(dmesh: DeviceMesh, J: DeviceJacobian, stream=None):
    _check(lib().fnlh_prepare(ctypes.byref(dmesh.c), ctypes.byref(J.c), _stream(stream)), "fnlh_prepare")


def fnlh_relax(dmesh, J, omega, B, X, sweeps, precision=FNLH_F64, ws=None, stream=None, sigma=None):
    om, omp = _omega(omega)
    n_harm = len(np.atleast_1d(omega))
    sg, sgp = _sigma(sigma, n_harm)
    if ws is None:
        ws = workspace(dmesh.n_nodes, J.block, n_harm, B.device)
    st = lib().fnlh_relax(ctypes.byref(dmesh.c), ctypes.byref(J.c), n_harm, omp, sgp, _ptr(B), _ptr(X), int(sweeps),
                          int(precision), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "fnlh_relax")


def fnlh_residual(dmesh, J, omega, B, X, r=None, norms=None, ws=None, stream=None, sigma=None):
    """Returns the device tensor of norms [K, 2] = (||r_k||^2, ||B_k||^2)."""
    om, omp = _omega(omega)
    n_harm = len(np.atleast_1d(omega))
    sg, sgp = _sigma(sigma, n_harm)
    K = 1 + n_harm
    if norms is None:
        norms = torch.empty((K, 2), dtype=torch.float64, device=B.device)
    if ws is None:
        ws = workspace(dmesh.n_nodes, J.block, n_harm, B.device)
    st = lib().fnlh_residual(ctypes.byref(dmesh.c), ctypes.byref(J.c), n_harm, omp, sgp, _ptr(B), _ptr(X), _ptr(r),
                             _ptr(norms), _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "fnlh_residual")
    return norms


FNLH_SOLVE_ZERO_GUESS = 1
FNLH_SOLVE_MASK_CONVERGED = 2


def fnlh_solve(dmesh, J, omega, B, X, precision, tol, inner_sweeps, max_checks, ws=None, stream=None,
               raise_on_error=True, flags=0, sigma=None):
    """Returns (status, checks_done, sweeps_done, rel_res[K])."""
    om, omp = _omega(omega)
    n_harm = len(np.atleast_1d(omega))
    sg, sgp = _sigma(sigma, n_harm)
    if ws is None:
        ws = solve_workspace(dmesh.n_nodes, J.block, n_harm, J.c.prep_flags, B.device, precision)
    checks, sweeps = c_i32(0), c_i32(0)
    rel = (c_f64 * (1 + n_harm))()
    st = lib().fnlh_solve(ctypes.byref(dmesh.c), ctypes.byref(J.c), n_harm, omp, sgp, _ptr(B), _ptr(X), int(precision),
                          float(tol), int(inner_sweeps), int(max_checks), int(flags), _ptr(ws), ws.numel(),
                          ctypes.byref(checks),
                          ctypes.byref(sweeps), rel, _stream(stream))
    if raise_on_error and st != FNLH_OK:
        raise FnlhError(st, "fnlh_solve")
    return st, checks.value, sweeps.value, np.array(rel[:])


class BatchedRows:
    """Holds the ctypes row array (and the omega buffers it points to)."""

    def __init__(self, rows):
        # rows: list of (dmesh, J, omega, B, X) or (dmesh, J, omega, B, X, sigma)
        self.keep = []
        self.sigmas = []
        arr = (fnlh_row * len(rows))()
        for r, row in enumerate(rows):
            dm, J, omega, B, X = row[:5]
            sigma = row[5] if len(row) > 5 else None
            om, omp = _omega(omega)
            sg, sgp = _sigma(sigma, len(np.atleast_1d(omega)))
            self.keep.append((dm, J, om, B, X))
            self.sigmas.append(sg)
            arr[r] = fnlh_row(ctypes.pointer(dm.c), ctypes.pointer(J.c), len(np.atleast_1d(omega)), omp,
                              _ptr(B), _ptr(X), sgp)
        self.arr = arr
        self.n = len(rows)

    def workspace_bytes(self, block, precision=FNLH_F64, ff=False):
        """Workspace of fnlh_relax_batched / fnlh_solve_batched; ff=True adds every row's float-float
        shadows (fnlh_solve_workspace_bytes), which the batched mixed solve uses when every row's
        Jacobian has FNLH_PREP_FF."""
        total = int(lib().fnlh_batched_extra_bytes(self.n))
        for dm, J, om, B, X in self.keep:
            nh = (B.shape[1] - 1) // 2
            if ff:
                total += fnlh_solve_workspace_bytes(dm.n_nodes, block, nh, precision, J.c.prep_flags)
            else:
                total += fnlh_workspace_bytes(dm.n_nodes, block, nh, precision)
        return total


def fnlh_relax_batched(batch: BatchedRows, sweeps, precision, tuning=None, ws=None, stream=None):
    tn = ctypes.byref(tuning) if tuning is not None else None
    st = lib().fnlh_relax_batched(batch.arr, batch.n, int(sweeps), int(precision), tn, _ptr(ws), ws.numel(),
                                  _stream(stream))
    _check(st, "fnlh_relax_batched")


def fnlh_solve_batched(batch: BatchedRows, precision, tol, inner_sweeps, max_checks, tuning=None, ws=None,
                       stream=None, flags=0, raise_on_error=True):
    """Returns (status, checks_done, sweeps_done, rel_res[sum of K over rows])."""
    tn = ctypes.byref(tuning) if tuning is not None else None
    checks, sweeps = c_i32(0), c_i32(0)
    total = sum((B.shape[1] - 1) // 2 + 1 for (_, _, _, B, _) in batch.keep)
    rel = (c_f64 * total)()
    st = lib().fnlh_solve_batched(batch.arr, batch.n, int(precision), float(tol), int(inner_sweeps), int(max_checks),
                                  int(flags), tn, _ptr(ws), ws.numel(), ctypes.byref(checks), ctypes.byref(sweeps),
                                  rel, _stream(stream))
    if raise_on_error and st != FNLH_OK:
        raise FnlhError(st, "fnlh_solve_batched")
    return st, checks.value, sweeps.value, np.array(rel[:])


def fnlh_prep_structured(J, stream=None) -> bool:
    """Whether fnlh_prepare certified the b = 6 frozen-turbulence zero pattern."""
    v = c_i32(0)
    _check(lib().fnlh_prep_structured(ctypes.byref(J.c), ctypes.byref(v), _stream(stream)), "fnlh_prep_structured")
    return bool(v.value)


def fnlh_set_sweep_events(begin=None, end=None):
    """Record torch.cuda.Event `begin`/`end` around the sweep launches of later calls."""
    b = c_vp(begin.cuda_event) if begin is not None else None
    e = c_vp(end.cuda_event) if end is not None else None
    _check(lib().fnlh_set_sweep_events(b, e), "fnlh_set_sweep_events")


def fnlh_residual_noalloc(dmesh, J, omega, B, X, r=None, norms=None, stream=None, sigma=None):
    """fnlh_residual without a workspace: for callers that cannot allocate
    device memory (the library keeps the partial sums in its own static device
    array).  `norms` must be given by such a caller; it is allocated here only
    as a convenience when omitted."""
    om, omp = _omega(omega)
    n_harm = len(np.atleast_1d(omega))
    sg, sgp = _sigma(sigma, n_harm)
    if norms is None:
        norms = torch.empty((1 + n_harm, 2), dtype=torch.float64, device=B.device)
    st = lib().fnlh_residual_noalloc(ctypes.byref(dmesh.c), ctypes.byref(J.c), n_harm, omp, sgp, _ptr(B), _ptr(X),
                                     _ptr(r), _ptr(norms), _stream(stream))
    _check(st, "fnlh_residual_noalloc")
    return norms


# ------------------------------------------------------------------ ILU(0)

def fnlh_mesh_color(row_ptr, col_idx, max_colors=64):
    """Greedy colouring (host): returns (color [n], order [n], color_ptr [n_colors + 1])."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    n = row_ptr.shape[0] - 1
    color = np.zeros(max(n, 1), dtype=np.int32)
    order = np.zeros(max(n, 1), dtype=np.int32)
    cptr = np.zeros(max_colors + 1, dtype=np.int32)
    nc = c_i32(0)
    col = col_idx if col_idx.size else np.zeros(1, dtype=np.int32)
    st = lib().fnlh_mesh_color(n, row_ptr.ctypes.data_as(c_vp), col.ctypes.data_as(c_vp), int(max_colors),
                               color.ctypes.data_as(c_vp), order.ctypes.data_as(c_vp), cptr.ctypes.data_as(c_vp),
                               ctypes.byref(nc))
    _check(st, "fnlh_mesh_color")
    return color[:n].copy(), order[:n].copy(), cptr[: nc.value + 1].copy()


def fnlh_ilu_bytes(n_nodes, block, n_harm, precision=FNLH_F64) -> int:
    return int(lib().fnlh_ilu_bytes(n_nodes, block, n_harm, precision))


class DeviceIlu:
    """Colouring (device color/order, host color_ptr) and the factor buffer of
    the ILU(0) smoother.  color: per-node colours (neighbours must differ); if
    None the library's greedy colouring of the mesh is used."""

    def __init__(self, dmesh: DeviceMesh, block: int, n_harm: int, color=None, precision=FNLH_F64, device="cuda"):
        n = dmesh.n_nodes
        if color is None:
            color, order, cptr = fnlh_mesh_color(dmesh.row_ptr_host, dmesh.col_idx_host)
        else:
            color = np.ascontiguousarray(color, dtype=np.int32).reshape(n)
            nc = int(color.max()) + 1 if n else 0
            order = np.lexsort((np.arange(n), color)).astype(np.int32)
            cptr = np.zeros(nc + 1, dtype=np.int32)
            np.add.at(cptr, color + 1, 1)
            cptr = np.cumsum(cptr).astype(np.int32)
        dev = torch.device(device)
        self.color_host, self.order_host = color, order
        self.color_ptr = np.ascontiguousarray(cptr if len(cptr) else np.zeros(1, np.int32), dtype=np.int32)
        self.color = torch.from_numpy(np.ascontiguousarray(color if n else np.zeros(1, np.int32))).to(dev)
        self.order = torch.from_numpy(np.ascontiguousarray(order if n else np.zeros(1, np.int32))).to(dev)
        nbytes = fnlh_ilu_bytes(n, block, n_harm, precision)
        self.factor = torch.empty((max(nbytes, 16),), dtype=torch.uint8, device=dev)
        self.c = fnlh_ilu(len(self.color_ptr) - 1, _ptr(self.color), _ptr(self.order),
                          self.color_ptr.ctypes.data_as(ctypes.POINTER(c_i32)), _ptr(self.factor), nbytes,
                          int(precision), 0, 0)

    @property
    def n_colors(self):
        return int(self.c.n_colors)


def fnlh_ilu_factor(dmesh, J, omega, ilu: DeviceIlu, ws=None, stream=None):
    om, omp = _omega(omega)
    n_harm = len(np.atleast_1d(omega))
    if ws is None:
        ws = workspace(dmesh.n_nodes, J.block, n_harm, ilu.factor.device)
    st = lib().fnlh_ilu_factor(ctypes.byref(dmesh.c), ctypes.byref(J.c), n_harm, omp, ctypes.byref(ilu.c), _ptr(ws),
                               ws.numel(), _stream(stream))
    _check(st, "fnlh_ilu_factor")


def fnlh_solve_ilu(dmesh, J, ilu: DeviceIlu, omega, B, X, tol, max_iterations, ws=None, stream=None, flags=0,
                   sigma=None, raise_on_error=True):
    """Returns (status, iterations_done, rel_res[K])."""
    om, omp = _omega(omega)
    n_harm = len(np.atleast_1d(omega))
    sg, sgp = _sigma(sigma, n_harm)
    if ws is None:
        ws = workspace(dmesh.n_nodes, J.block, n_harm, B.device)
    its = c_i32(0)
    rel = (c_f64 * (1 + n_harm))()
    st = lib().fnlh_solve_ilu(ctypes.byref(dmesh.c), ctypes.byref(J.c), ctypes.byref(ilu.c), n_harm, omp, sgp,
                              _ptr(B), _ptr(X), float(tol), int(max_iterations), int(flags), _ptr(ws), ws.numel(),
                              ctypes.byref(its), rel, _stream(stream))
    if raise_on_error and st != FNLH_OK:
        raise FnlhError(st, "fnlh_solve_ilu")
    return st, its.value, np.array(rel[:])

"""The C-ABI library builds, loads and exports every symbol of include/fnlh.h;
host-side logic (CSR builder, sizes, argument validation) without a GPU."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2404_01407_gb300 import fnlh, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "fnlh.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fnlh_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = fnlh.lib()
    declared = header_functions()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(fnlh.exported_symbols())


def test_version_and_strerror():
    assert fnlh.fnlh_version() >= 100
    for code in range(0, -10, -1):
        assert fnlh.fnlh_strerror(code)
    assert fnlh.fnlh_strerror(-999) == "unknown status"


def test_csr_matches_oracle_pattern():
    m = inputs.hex_mesh(7, 5, 3)
    n, E = m.n_nodes, m.n_edges
    rp = np.zeros(n + 1, np.int32)
    ci = np.zeros(2 * E, np.int32)
    ce = np.zeros(2 * E, np.int32)
    fnlh.fnlh_mesh_build_csr(n, E, m.edge_nodes, rp, ci, ce)
    jac = oracle.build_jacobian(n, m.edge_nodes, m.normals, inputs.flow_state(n, 5), 10.0)
    assert np.array_equal(rp, jac.row_ptr)
    assert np.array_equal(ci, jac.col_idx)
    # csr_edge names the edge joining the row to its neighbour
    owner = np.repeat(np.arange(n), np.diff(rp))
    pair = np.sort(np.stack([owner, ci], 1), 1)
    assert np.array_equal(m.edge_nodes[ce], pair)


@pytest.mark.parametrize("edges", [[[0, 0]], [[0, 1], [1, 0]], [[0, 5]], [[-1, 1]]])
def test_csr_rejects_bad_mesh(edges):
    en = np.asarray(edges, np.int32)
    rp = np.zeros(4, np.int32)
    ci = np.zeros(2 * len(en), np.int32)
    ce = np.zeros(2 * len(en), np.int32)
    with pytest.raises(fnlh.FnlhError) as e:
        fnlh.fnlh_mesh_build_csr(3, len(en), en, rp, ci, ce)
    assert e.value.status == fnlh.FNLH_ERR_BAD_MESH


def test_sizes_independent_of_harmonics():
    """The Jacobian and its derived data do not depend on N ("Solution Update")."""
    n, nnz = 1000, 5800
    prep = fnlh.fnlh_prep_bytes(n, nnz, 6, 7)
    assert prep > 0
    ws = [fnlh.fnlh_workspace_bytes(n, 6, N) for N in (0, 1, 16, 64)]
    assert ws[0] < ws[1] < ws[2] < ws[3]
    assert fnlh.fnlh_workspace_bytes(n, 6, 16, fnlh.FNLH_F32) < ws[2]
    assert fnlh.fnlh_workspace_bytes(n, 6, 16, fnlh.FNLH_BF16) == fnlh.fnlh_workspace_bytes(n, 6, 16, fnlh.FNLH_F32)
    assert fnlh.fnlh_workspace_bytes(n, 6, 65) == 0
    assert fnlh.fnlh_workspace_bytes(n, 7, 1) == 0
    assert fnlh.fnlh_workspace_bytes(n, 6, 1, 9) == 0
    assert fnlh.fnlh_prep_bytes(n, nnz, 4, 1) == 0


def test_validation_rejects_before_launch():
    L = fnlh.lib()
    null = ctypes.POINTER(fnlh.fnlh_mesh)()
    assert L.fnlh_relax(null, None, 0, None, None, None, None, 1, 0, None, 0, None) == fnlh.FNLH_ERR_ARG
    m = fnlh.fnlh_mesh(4, 0, None, None, None, None, None, None)
    assert L.fnlh_prepare(ctypes.byref(m), None, None) == fnlh.FNLH_ERR_ARG
    J = fnlh.fnlh_jacobian(4, 0, 7, None, None, None, None, 0, 0, 0)
    m2 = fnlh.fnlh_mesh(4, 0, None, None, ctypes.c_void_p(256), ctypes.c_void_p(256), None, None)
    assert L.fnlh_prepare(ctypes.byref(m2), ctypes.byref(J), None) == fnlh.FNLH_ERR_UNSUPPORTED
    J5 = fnlh.fnlh_jacobian(4, 0, 5, None, ctypes.c_void_p(256), ctypes.c_void_p(256), None, 0, 0, 0)
    # no prep blob -> workspace error; bad precision -> arg error; too many harmonics -> unsupported
    om = (ctypes.c_double * 70)()
    assert L.fnlh_relax(ctypes.byref(m2), ctypes.byref(J5), 1, om, None, None, None, 1, 0, None, 0, None) \
        == fnlh.FNLH_ERR_WORKSPACE
    assert L.fnlh_relax(ctypes.byref(m2), ctypes.byref(J5), 1, om, None, None, None, 1, 9, None, 0, None) \
        == fnlh.FNLH_ERR_ARG
    assert L.fnlh_relax(ctypes.byref(m2), ctypes.byref(J5), 65, om, None, None, None, 1, 0, None, 0, None) \
        == fnlh.FNLH_ERR_UNSUPPORTED
    assert L.fnlh_relax(ctypes.byref(m2), ctypes.byref(J5), 1, om, None, None, None, -1, 0, None, 0, None) \
        == fnlh.FNLH_ERR_ARG
    om[0] = float("nan")
    assert L.fnlh_residual(ctypes.byref(m2), ctypes.byref(J5), 1, om, None, None, None, None, None, None, 0, None) \
        == fnlh.FNLH_ERR_ARG


def test_tagged_mesh_validation_rejects_before_launch():
    """Periodic edges and partitions: the tagged column copy must be in the
    prep blob, node ids must leave the top three bits free, phase angles finite."""
    L = fnlh.lib()
    per = ctypes.c_void_p(4096)  # never dereferenced: validation fails first
    vol = ctypes.c_void_p(256)
    m = fnlh.fnlh_mesh(4, 0, None, None, vol, vol, None, None, per)
    J5 = fnlh.fnlh_jacobian(4, 0, 5, None, ctypes.c_void_p(256), ctypes.c_void_p(256), None, 0, 0, 0)
    om = (ctypes.c_double * 2)(1.0, 2.0)
    sig = (ctypes.c_double * 2)(0.5, float("nan"))
    # no prep at all, then a prepared blob without the periodic copy
    assert L.fnlh_residual(ctypes.byref(m), ctypes.byref(J5), 1, om, None, vol, vol, None, vol, vol, 1 << 20,
                           None) == fnlh.FNLH_ERR_WORKSPACE
    nb = fnlh.fnlh_prep_bytes(4, 0, 5, fnlh.FNLH_PREP_F64)
    Jp = fnlh.fnlh_jacobian(4, 0, 5, None, ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(1 << 12), nb,
                            fnlh.FNLH_PREP_F64, 1)
    assert L.fnlh_relax(ctypes.byref(m), ctypes.byref(Jp), 1, om, None, vol, vol, 1, 0, vol, 1 << 20, None) \
        == fnlh.FNLH_ERR_WORKSPACE
    assert L.fnlh_prepare(ctypes.byref(m), ctypes.byref(Jp), None) == fnlh.FNLH_ERR_WORKSPACE
    # a partitioned mesh also reads the tagged copy
    mp = fnlh.fnlh_mesh(4, 0, None, None, vol, vol, None, None, None, ctypes.c_void_p(4096))
    assert L.fnlh_relax(ctypes.byref(mp), ctypes.byref(Jp), 1, om, None, vol, vol, 1, 0, vol, 1 << 20, None) \
        == fnlh.FNLH_ERR_WORKSPACE
    assert L.fnlh_prepare(ctypes.byref(mp), ctypes.byref(Jp), None) == fnlh.FNLH_ERR_WORKSPACE
    # a non-finite phase angle
    assert L.fnlh_relax(ctypes.byref(m), ctypes.byref(J5), 2, om, sig, vol, vol, 1, 0, vol, 1 << 20, None) \
        == fnlh.FNLH_ERR_ARG
    # node ids of 2^29 and up leave no room for the column tags (any mesh)
    big = fnlh.fnlh_mesh(1 << 29, 0, None, None, vol, vol, None, None, None)
    Jb = fnlh.fnlh_jacobian(1 << 29, 0, 5, None, ctypes.c_void_p(256), ctypes.c_void_p(256), None, 0, 0, 0)
    assert L.fnlh_residual(ctypes.byref(big), ctypes.byref(Jb), 0, om, None, vol, vol, None, vol, vol, 1 << 20,
                           None) == fnlh.FNLH_ERR_UNSUPPORTED
    # the tagged copy adds nnz int32 (256-aligned) to the blob
    n, nnz = 1000, 6000
    assert fnlh.fnlh_prep_bytes(n, nnz, 6, fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_TAGS) == \
        fnlh.fnlh_prep_bytes(n, nnz, 6, fnlh.FNLH_PREP_F64) + ((nnz * 4 + 255) // 256) * 256


def _csr(mesh):
    n, E = mesh.n_nodes, mesh.n_edges
    rp = np.zeros(n + 1, np.int32)
    ci = np.zeros(max(2 * E, 1), np.int32)
    ce = np.zeros(max(2 * E, 1), np.int32)
    fnlh.fnlh_mesh_build_csr(n, E, mesh.edge_nodes, rp, ci, ce)
    return rp, ci[: 2 * E]


def _valid_coloring(rp, ci, color):
    owner = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return np.all(color[owner] != color[ci])


@pytest.mark.parametrize("dims,periodic,colors", [((7, 5, 3), False, 2), ((6, 4, 3), True, 2), ((6, 5, 3), True, 3)])
def test_mesh_coloring_host_helper(dims, periodic, colors):
    """Greedy colouring: a valid colouring, red-black on the lattice (and on an
    even pitch), more colours where an odd pitch closes an odd cycle; the
    order groups the nodes by colour."""
    mesh = inputs.hex_mesh(*dims, periodic_y=periodic)
    rp, ci = _csr(mesh)
    color, order, cptr = fnlh.fnlh_mesh_color(rp, ci)
    assert _valid_coloring(rp, ci, color)
    if colors == 2:
        assert len(cptr) - 1 == 2
        assert np.array_equal(color, inputs.lattice_colors(dims))
    else:
        assert len(cptr) - 1 >= 3  # the odd cycle through the periodic edges
    assert sorted(order) == list(range(mesh.n_nodes))
    for c in range(len(cptr) - 1):
        members = order[cptr[c]:cptr[c + 1]]
        assert np.all(color[members] == c) and np.all(np.diff(members) > 0)


def test_mesh_coloring_limits():
    # a triangle needs three colours
    rp = np.array([0, 2, 4, 6], np.int32)
    ci = np.array([1, 2, 0, 2, 0, 1], np.int32)
    color, order, cptr = fnlh.fnlh_mesh_color(rp, ci)
    assert sorted(color) == [0, 1, 2]
    with pytest.raises(fnlh.FnlhError):
        fnlh.fnlh_mesh_color(rp, ci, max_colors=2)
    with pytest.raises(fnlh.FnlhError):
        fnlh.fnlh_mesh_color(rp, np.array([1, 2, 0, 7, 0, 1], np.int32))
    # empty graph
    c0, o0, p0 = fnlh.fnlh_mesh_color(np.zeros(1, np.int32), np.zeros(0, np.int32))
    assert len(c0) == 0 and list(p0) == [0]


def test_ilu_sizes_and_validation():
    n = 1000
    assert fnlh.fnlh_ilu_bytes(n, 6, 4) == n * 5 * 36 * 16
    assert fnlh.fnlh_ilu_bytes(n, 6, 4, fnlh.FNLH_F32) == n * 5 * 36 * 8
    assert fnlh.fnlh_ilu_bytes(n, 6, 4, fnlh.FNLH_BF16) == 0
    assert fnlh.fnlh_ilu_bytes(n, 7, 4) == 0
    L = fnlh.lib()
    vol = ctypes.c_void_p(256)
    m = fnlh.fnlh_mesh(4, 0, None, None, vol, vol, None, None, None, None)
    J5 = fnlh.fnlh_jacobian(4, 0, 5, None, ctypes.c_void_p(256), ctypes.c_void_p(256), None, 0, 0, 0)
    om = (ctypes.c_double * 1)(1.0)
    cptr = (ctypes.c_int32 * 3)(0, 2, 4)
    ilu = fnlh.fnlh_ilu(2, vol, vol, cptr, ctypes.c_void_p(4096), fnlh.fnlh_ilu_bytes(4, 5, 1), fnlh.FNLH_F64, 0, 0)
    # not factored yet / wrong harmonic count
    assert L.fnlh_solve_ilu(ctypes.byref(m), ctypes.byref(J5), ctypes.byref(ilu), 1, om, None, vol, vol, 1e-2, 10, 0,
                            vol, 1 << 20, None, None, None) == fnlh.FNLH_ERR_WORKSPACE
    # factor buffer too small, bad precision, colour offsets not covering the nodes
    small = fnlh.fnlh_ilu(2, vol, vol, cptr, ctypes.c_void_p(4096), 16, fnlh.FNLH_F64, 0, 0)
    assert L.fnlh_ilu_factor(ctypes.byref(m), ctypes.byref(J5), 1, om, ctypes.byref(small), vol, 1 << 20,
                             None) == fnlh.FNLH_ERR_WORKSPACE
    bad = fnlh.fnlh_ilu(2, vol, vol, cptr, ctypes.c_void_p(4096), 1 << 20, fnlh.FNLH_BF16, 0, 0)
    assert L.fnlh_ilu_factor(ctypes.byref(m), ctypes.byref(J5), 1, om, ctypes.byref(bad), vol, 1 << 20,
                             None) == fnlh.FNLH_ERR_ARG
    short = (ctypes.c_int32 * 3)(0, 2, 3)
    gap = fnlh.fnlh_ilu(2, vol, vol, short, ctypes.c_void_p(4096), 1 << 20, fnlh.FNLH_F64, 0, 0)
    assert L.fnlh_ilu_factor(ctypes.byref(m), ctypes.byref(J5), 1, om, ctypes.byref(gap), vol, 1 << 20,
                             None) == fnlh.FNLH_ERR_ARG


def test_probe_library_exports_every_declared_symbol():
    """The peak probe beside the library (include/fnlh_probe.h) builds and
    exports its declared symbols; bad arguments are rejected on the host,
    before any launch (no GPU needed)."""
    from paper_2404_01407_gb300 import peaks

    text = open(os.path.join(ROOT, "include", "fnlh_probe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    declared = sorted(set(re.findall(r"\b(fnlh_\w+)\s*\(", text)))
    assert declared == ["fnlh_probe_fma"]
    lib = peaks.probe_lib()
    assert hasattr(lib, "fnlh_probe_fma")
    ms = ctypes.c_float(0.0)
    sink = ctypes.c_void_p(16)  # never dereferenced: every call below fails its argument check
    assert lib.fnlh_probe_fma(2, 8, 1, 1, 256, 1, sink, ctypes.byref(ms), None) == -1  # precision
    assert lib.fnlh_probe_fma(0, 5, 1, 1, 256, 1, sink, ctypes.byref(ms), None) == -1  # chains
    assert lib.fnlh_probe_fma(0, 8, 3, 1, 256, 1, sink, ctypes.byref(ms), None) == -1  # reuse
    assert lib.fnlh_probe_fma(0, 8, 1, 1, 100, 1, sink, ctypes.byref(ms), None) == -1  # threads
    assert lib.fnlh_probe_fma(0, 8, 1, 0, 256, 1, sink, ctypes.byref(ms), None) == -1  # blocks
    assert lib.fnlh_probe_fma(0, 8, 1, 1, 256, 1, None, ctypes.byref(ms), None) == -1  # sink


def test_float_float_prep_and_solve_workspace_sizes():
    """FNLH_PREP_FF adds the float-float copies of the blocks (8 bytes per
    entry) to the prep blob; fnlh_solve_workspace_bytes adds the float-float
    shadows of B and x ([n][C][b] FP32 pairs each) for the mixed precisions
    only, and equals fnlh_workspace_bytes otherwise."""
    n, nnz, b, N = 1000, 5400, 6, 4
    C = 1 + 2 * N
    base = fnlh.fnlh_prep_bytes(n, nnz, b, fnlh.FNLH_PREP_BF16)
    ff = fnlh.fnlh_prep_bytes(n, nnz, b, fnlh.FNLH_PREP_BF16 | fnlh.FNLH_PREP_FF)
    assert ff - base >= (nnz + n) * b * b * 8
    for prec in (fnlh.FNLH_F32, fnlh.FNLH_BF16):
        w = fnlh.fnlh_workspace_bytes(n, b, N, prec)
        wf = fnlh.fnlh_solve_workspace_bytes(n, b, N, prec, fnlh.FNLH_PREP_FF | fnlh.FNLH_PREP_F32)
        assert wf - w >= 2 * n * C * b * 8
        assert fnlh.fnlh_solve_workspace_bytes(n, b, N, prec, fnlh.FNLH_PREP_F32) == w
    w64 = fnlh.fnlh_workspace_bytes(n, b, N, fnlh.FNLH_F64)
    assert fnlh.fnlh_solve_workspace_bytes(n, b, N, fnlh.FNLH_F64, fnlh.FNLH_PREP_FF) == w64
    assert fnlh.fnlh_solve_workspace_bytes(n, 7, N, fnlh.FNLH_F32, fnlh.FNLH_PREP_FF) == 0


def _fake_problem(prep_flags=fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_F32, part=None):
    """A 4-node, edge-free mesh and Jacobian whose device pointers are fake
    (aligned, never dereferenced): every call below must fail validation
    before it launches or copies anything."""
    a = ctypes.c_void_p(1 << 12)
    m = fnlh.fnlh_mesh(4, 0, None, None, a, a, None, None, None, part)
    nb = fnlh.fnlh_prep_bytes(4, 0, 6, prep_flags)
    J = fnlh.fnlh_jacobian(4, 0, 6, None, a, a, ctypes.c_void_p(1 << 16), nb, prep_flags, 1)
    return m, J, a


def test_solve_validation_rejects_before_launch():
    L = fnlh.lib()
    m, J, a = _fake_problem()
    om = (ctypes.c_double * 2)(1.0, 2.0)
    c, s = ctypes.c_int32(), ctypes.c_int32()
    rel = (ctypes.c_double * 3)()
    ws_ok = fnlh.fnlh_workspace_bytes(4, 6, 2, fnlh.FNLH_F64)
    ws = ctypes.c_void_p(1 << 20)

    def solve(prec=fnlh.FNLH_F64, tol=1e-8, inner=10, checks=5, flags=0, w=ws, wb=ws_ok, n_harm=2, jac=J):
        return L.fnlh_solve(ctypes.byref(m), ctypes.byref(jac), n_harm, om, None, a, a, prec, tol, inner, checks,
                            flags, w, wb, ctypes.byref(c), ctypes.byref(s), rel, None)

    assert solve(prec=9) == fnlh.FNLH_ERR_ARG
    assert solve(tol=-1.0) == fnlh.FNLH_ERR_ARG
    assert solve(tol=float("nan")) == fnlh.FNLH_ERR_ARG
    assert solve(inner=0) == fnlh.FNLH_ERR_ARG
    assert solve(checks=0) == fnlh.FNLH_ERR_ARG
    assert solve(flags=1 << 7) == fnlh.FNLH_ERR_ARG
    assert solve(n_harm=65) == fnlh.FNLH_ERR_UNSUPPORTED  # above the 64-harmonic maximum
    assert solve(prec=fnlh.FNLH_BF16) == fnlh.FNLH_ERR_WORKSPACE  # prep holds no BF16 copy
    assert solve(w=None) == fnlh.FNLH_ERR_WORKSPACE
    assert solve(w=ctypes.c_void_p((1 << 20) + 8)) == fnlh.FNLH_ERR_ARG  # not 256-byte aligned
    assert solve(wb=ws_ok - 1) == fnlh.FNLH_ERR_WORKSPACE
    unready = fnlh.fnlh_jacobian(4, 0, 6, None, a, a, ctypes.c_void_p(1 << 16), J.prep_bytes, J.prep_flags, 0)
    assert solve(jac=unready) == fnlh.FNLH_ERR_WORKSPACE


def test_batched_validation_rejects_before_launch():
    L = fnlh.lib()
    m, J, a = _fake_problem()
    om = (ctypes.c_double * 2)(1.0, 2.0)
    rows = (fnlh.fnlh_row * 2)()
    for r in rows:
        r.mesh, r.J, r.n_harm, r.omega, r.B, r.X, r.sigma = ctypes.pointer(m), ctypes.pointer(J), 2, om, a, a, None
    need = L.fnlh_batched_extra_bytes(2) + 2 * fnlh.fnlh_workspace_bytes(4, 6, 2, fnlh.FNLH_F32)
    ws = ctypes.c_void_p(1 << 20)

    def relax(rr=rows, n=2, sweeps=3, prec=fnlh.FNLH_F32, w=ws, wb=need):
        return L.fnlh_relax_batched(rr, n, sweeps, prec, None, w, wb, None)

    assert relax(rr=None) == fnlh.FNLH_ERR_ARG
    assert relax(n=0) == fnlh.FNLH_ERR_ARG
    assert relax(sweeps=-1) == fnlh.FNLH_ERR_ARG
    assert relax(prec=9) == fnlh.FNLH_ERR_ARG
    assert relax(prec=fnlh.FNLH_BF16) == fnlh.FNLH_ERR_WORKSPACE
    assert relax(w=None) == fnlh.FNLH_ERR_WORKSPACE
    assert relax(w=ctypes.c_void_p((1 << 20) + 16)) == fnlh.FNLH_ERR_ARG
    assert relax(wb=need - 1) == fnlh.FNLH_ERR_WORKSPACE
    # one bad row is enough: a block size the library has no kernels for
    J7 = fnlh.fnlh_jacobian(4, 0, 7, None, a, a, ctypes.c_void_p(1 << 16), J.prep_bytes, J.prep_flags, 1)
    rows[1].J = ctypes.pointer(J7)
    assert relax() == fnlh.FNLH_ERR_UNSUPPORTED
    rows[1].J = ctypes.pointer(J)

    c, s = ctypes.c_int32(), ctypes.c_int32()
    rel = (ctypes.c_double * 6)()

    def solve(prec=fnlh.FNLH_F32, tol=1e-8, inner=10, checks=5, flags=0, wb=need):
        return L.fnlh_solve_batched(rows, 2, prec, tol, inner, checks, flags, None, ws, wb, ctypes.byref(c),
                                    ctypes.byref(s), rel, None)

    assert solve(tol=float("nan")) == fnlh.FNLH_ERR_ARG
    assert solve(inner=0) == fnlh.FNLH_ERR_ARG
    assert solve(checks=0) == fnlh.FNLH_ERR_ARG
    assert solve(flags=1 << 9) == fnlh.FNLH_ERR_ARG
    assert solve(wb=need - 1) == fnlh.FNLH_ERR_WORKSPACE
    # a partitioned row: plain FP64 Jacobi on truncated sweeps would not solve the full system
    tags = fnlh.FNLH_PREP_F64 | fnlh.FNLH_PREP_F32 | fnlh.FNLH_PREP_TAGS
    mp, Jp, _ = _fake_problem(tags, part=ctypes.c_void_p(1 << 14))
    rows[0].mesh, rows[0].J = ctypes.pointer(mp), ctypes.pointer(Jp)
    need64 = L.fnlh_batched_extra_bytes(2) + 2 * fnlh.fnlh_workspace_bytes(4, 6, 2, fnlh.FNLH_F64)
    assert solve(prec=fnlh.FNLH_F64, wb=need64) == fnlh.FNLH_ERR_UNSUPPORTED


def test_build_validation_rejects_before_launch():
    """fnlh_build_jacobian's parameters (the pseudo-time reading of Eq. precon
    needs CFL > 0, gamma > 1, a non-negative entropy-fix delta, and eps > 0 in
    the block pseudo-time form) and the edge arrays the assembly reads."""
    L = fnlh.lib()
    a = ctypes.c_void_p(1 << 12)
    m = fnlh.fnlh_mesh(4, 3, a, a, a, a, a, a, None)  # 3 edges: the assembly needs csr_edge, normals, edge_nodes
    J = fnlh.fnlh_jacobian(4, 6, 6, a, a, a, None, 0, 0, 0)

    def build(mesh=m, q=a, **kw):
        p = fnlh.make_params(20.0)
        for k, v in kw.items():
            setattr(p, k, v)
        return L.fnlh_build_jacobian(ctypes.byref(mesh), q, ctypes.byref(p), ctypes.byref(J), None)

    assert build(cfl=0.0) == fnlh.FNLH_ERR_ARG
    assert build(cfl=float("nan")) == fnlh.FNLH_ERR_ARG
    assert build(gamma=1.0) == fnlh.FNLH_ERR_ARG
    assert build(entropy_delta=-0.1) == fnlh.FNLH_ERR_ARG
    assert build(pseudo_time=2) == fnlh.FNLH_ERR_ARG
    assert build(pseudo_time=1, eps=0.0) == fnlh.FNLH_ERR_ARG
    assert build(q=None) == fnlh.FNLH_ERR_ARG
    assert L.fnlh_build_jacobian(ctypes.byref(m), a, None, ctypes.byref(J), None) == fnlh.FNLH_ERR_ARG
    for field in ("csr_edge", "normals", "edge_nodes"):
        bad = fnlh.fnlh_mesh(4, 3, a, a, a, a, a, a, None)
        setattr(bad, field, None)
        assert build(mesh=bad) == fnlh.FNLH_ERR_ARG, field
    # nnz must be twice the edge count, the block size 5 or 6
    J_bad = fnlh.fnlh_jacobian(4, 5, 6, a, a, a, None, 0, 0, 0)
    assert L.fnlh_build_jacobian(ctypes.byref(m), a, ctypes.byref(fnlh.make_params(20.0)), ctypes.byref(J_bad),
                                 None) == fnlh.FNLH_ERR_ARG
    J_b4 = fnlh.fnlh_jacobian(4, 6, 4, a, a, a, None, 0, 0, 0)
    assert L.fnlh_build_jacobian(ctypes.byref(m), a, ctypes.byref(fnlh.make_params(20.0)), ctypes.byref(J_b4),
                                 None) == fnlh.FNLH_ERR_UNSUPPORTED

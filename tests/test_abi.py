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

"""The seeded input generator: sizes of the measured configurations, the
edge graph, the geometry and reproducibility (CPU only)."""

import numpy as np
import pytest

from paper_2404_01407_gb300 import inputs


def expected_edges(nx, ny, nz):
    return (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)


@pytest.mark.parametrize("key,nodes,edges", [
    ("c1", 1024, 2752), ("c2", 393216, 1162240), ("c3", 2088960, 6217024),
    ("c4_row0", 200000, 589500), ("c4_row1", 600000, 1778500), ("c4_row2", 1100000, 3267450),
    ("c5", 7987200, 23839264)])
def test_config_sizes(key, nodes, edges):
    nx, ny, nz = inputs.CONFIGS[key]["dims"]
    assert nx * ny * nz == nodes
    assert expected_edges(nx, ny, nz) == edges


def test_mesh_graph_and_geometry():
    m = inputs.hex_mesh(7, 5, 4)
    assert m.n_nodes == 140 and m.n_edges == expected_edges(7, 5, 4)
    en = m.edge_nodes
    assert np.all(en[:, 0] < en[:, 1])
    assert len({tuple(e) for e in en}) == m.n_edges  # no duplicates
    # lattice neighbours along +x, +y, +z only
    assert set(np.unique(en[:, 1] - en[:, 0])) == {1, 7, 35}
    # normals point from i to j, perturbation bounded by 10% per axis
    d = m.normals - (m.positions[en[:, 1]] - m.positions[en[:, 0]])
    assert np.all(d == 0.0)
    base = np.abs(m.normals).max(axis=1)
    assert np.all((base > 0.8 - 1e-12) & (base < 1.2 + 1e-12))
    assert np.all(m.vol > 0.0)
    # unperturbed lattice: unit volumes inside, halves on faces
    u = inputs.hex_mesh(4, 4, 4, perturb=0.0)
    v = u.vol.reshape(4, 4, 4)
    assert np.allclose(v[1:3, 1:3, 1:3], 1.0) and np.isclose(v[0, 0, 0], 0.125)


def test_state_and_rhs_statistics():
    n = 200000
    q = inputs.flow_state(n, 6)
    rho = q[:, 0]
    assert np.all(np.abs(rho - 1.0) <= 0.02)
    u = q[:, 1] / rho
    p = (inputs.GAMMA - 1) * (q[:, 4] - 0.5 * rho * u * u)
    a = np.sqrt(inputs.GAMMA * p / rho)
    assert np.allclose(p, 1 / inputs.GAMMA)
    assert np.all(np.abs(u / a - 0.5) <= 0.05 + 1e-12)
    assert np.all(q[:, 2:4] == 0.0) and np.allclose(q[:, 5], 0.01 * rho)
    b = inputs.rhs(n, 6, 3)
    assert b.shape == (n, 7, 6)
    assert abs(b[:, 0].var() - 1.0) < 0.01
    # each harmonic: standard complex normal (total variance 1)
    for k in (1, 2, 3):
        var = b[:, 2 * k - 1].var() + b[:, 2 * k].var()
        assert abs(var - 1.0) < 0.01


def test_seeds_reproducible_and_distinct():
    a = inputs.config_problem("c1")
    b = inputs.config_problem("c1")
    assert np.array_equal(a.mesh.positions, b.mesh.positions)
    assert np.array_equal(a.q, b.q) and np.array_equal(a.b, b.b)
    c = inputs.problem((16, 8, 8), 5, 1, 10.0, seeds=(4, 5, 6))
    assert not np.array_equal(a.mesh.positions, c.mesh.positions)


def test_permutation_preserves_graph():
    m = inputs.hex_mesh(5, 4, 3)
    pm, perm = inputs.permute_mesh(m, seed=4)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    old = {tuple(sorted(e)) for e in m.edge_nodes.tolist()}
    new = {tuple(sorted((perm[a], perm[b]))) for a, b in pm.edge_nodes.tolist()}
    assert old == new
    assert np.array_equal(pm.vol, m.vol[perm])


def test_box_partition_cuts_the_lattice_into_boxes():
    dims, parts = (10, 7, 5), (3, 2, 2)
    part = inputs.box_partition(dims, parts)
    assert part.dtype == np.int32 and part.shape == (10 * 7 * 5,)
    ids, counts = np.unique(part, return_counts=True)
    assert list(ids) == list(range(12))
    # each axis is cut into contiguous index ranges whose lengths differ by at most one
    p3 = part.reshape(5, 7, 10)
    for axis, (n, q, stride) in enumerate(((10, 3, 1), (7, 2, 3), (5, 2, 6))):
        line = np.moveaxis(p3, 2 - axis, 0)[:, 0, 0] if axis else p3[0, 0, :]
        box = (line // stride) % q
        assert np.all(np.diff(box) >= 0) and set(box) == set(range(q))
        lengths = np.bincount(box)
        assert lengths.max() - lengths.min() <= 1, (axis, lengths)

"""The benchmark's roofline numerators against the measurement plan (CPU
only): the algorithmic bytes per sweep of bench.py's sweep_bytes, and the
synthetic meshes' node and edge counts, reproduce the per-configuration
figures the plan tabulates (c2 FP64 1.31 GB; c3 inner sweep 4.74 GB with FP32
blocks, 3.84 GB with BF16; c5 BF16 23.9 GB at N = 16 and 6.66 GB at N = 1),
and the FP64 sweep's flop count what a direct count of its operations gives."""

import pytest

import bench
from paper_2404_01407_gb300 import inputs

# (nodes, edges) of the plan's grids
PLAN_GRIDS = {"c1": (1024, 2752), "c2": (393216, 1162240), "c3": (2088960, 6217024),
              "c5": (7987200, 23839264)}


def lattice_edges(nx, ny, nz):
    return (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)


@pytest.mark.parametrize("key", ["c1", "c2", "c3", "c5"])
def test_plan_grids(key):
    nx, ny, nz = inputs.CONFIGS[key]["dims"]
    assert (nx * ny * nz, lattice_edges(nx, ny, nz)) == PLAN_GRIDS[key]


@pytest.mark.parametrize("key", ["c1", "c2"])
def test_generated_meshes_match_the_plan(key):
    m = inputs.hex_mesh(*inputs.CONFIGS[key]["dims"])
    assert (m.n_nodes, m.n_edges) == PLAN_GRIDS[key]


@pytest.mark.parametrize("key,n_harm,sizes,gb", [
    ("c2", 4, (8, 8, 8, 8), 1.31),   # FP64 sweep
    ("c3", 8, (4, 4, 4, 4), 4.74),   # inner sweep, FP32 blocks
    ("c3", 8, (2, 4, 4, 4), 3.84),   # inner sweep, BF16 blocks
    ("c5", 16, (2, 4, 4, 4), 23.9),
    ("c5", 1, (2, 4, 4, 4), 6.66),
])
def test_sweep_bytes_match_the_plan(key, n_harm, sizes, gb):
    n, E = PLAN_GRIDS[key]
    got = bench.sweep_bytes(n, 2 * E, 6, n_harm, *sizes)
    assert round(got / 1e9, 2 if gb < 10 else 1) == gb, got


def test_fp64_sweep_flops_by_direct_count():
    """c2: per directed edge and system column, one multiply-add (2 flops) per
    structurally nonzero block entry (31 with the frozen-turbulence pattern);
    per node, the real back-substitution of the mean flow (b(b-1) flops for
    the off-diagonal terms, one multiply per row) and for each harmonic the
    complex one (4 flops per off-diagonal term, 6 per row for the pivot)."""
    n, E = PLAN_GRIDS["c2"]
    b, N = 6, 4
    C = 1 + 2 * N
    spmv = 2 * (2 * E) * 31 * C
    offdiag_terms = b * (b - 1) // 2
    mean = 2 * offdiag_terms + b
    harmonic = 4 * offdiag_terms + 6 * b
    assert bench.sweep_flops(n, 2 * E, b, N, 31) == spmv + n * (mean + N * harmonic)

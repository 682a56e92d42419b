"""Seeded synthetic inputs for the shared-Jacobian FNLH linear systems.

This module only *draws* inputs: a perturbed hexahedral node cloud with its
edge graph, dual-face normals and control volumes, a near-uniform conservative
flow state, and the right-hand sides of the mean-flow and harmonic systems.  It
holds none of the method's arithmetic (no flux, Jacobian, pseudo-time term,
block solve or residual); both the CUDA path and the CPU oracle consume what
it returns, and neither imports the other.

Recipe (the paper's cases are proprietary turbomachinery meshes, so these
seeded stand-ins take their place; node counts and harmonic counts follow the
compressor / turbine / LPC sizes of the Results section):

* mesh (seed 1): nx*ny*nz hex lattice with unit spacing, node id
  ``i + nx*(j + ny*k)``, every node moved by U(-0.1, 0.1) per axis (a +/-10%
  perturbation); edges join lattice neighbours along +x, +y, +z (all x-edges
  in node order, then y-edges, then z-edges); the dual-face normal of edge
  (i, j) is ``x_j - x_i``; the control volume is the product over the three
  axes of half the distance between the two axis neighbours (one-sided half
  distance on the lattice boundary).  Periodic variant (a blade passage of
  pitch ny): every node of the last y-layer gets one more edge, to the first
  layer's node seen one pitch further along y (normal ``x_j + ny e_y - x_i``),
  flagged +1 in ``periodic``; inter-blade phase angles of harmonic l are
  ``2 pi l m / N_b`` (m = 3, N_b = 8 by default).
* state (seed 2): gamma = 1.4, p = 1/gamma, rho = 1 + U(-0.02, 0.02),
  Mach = 0.5 + U(-0.05, 0.05) along +x, v = w = 0; with 6 equations the sixth
  conserved variable is rho * 0.01 (a constant SA working variable).
* right-hand sides (seed 3): B = -R with R_mean ~ N(0, 1) (real) and every
  harmonic R_l a standard complex normal (real and imaginary parts N(0, 1/2)).

Layout of B and X: real ``[n][C][b]`` with ``C = 1 + 2N``: column 0 is the
mean flow, columns ``2l-1`` and ``2l`` hold Re and Im of harmonic ``l``.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4
NU_TILDE = 0.01


@dataclass
class Mesh:
    """Edge-based node-centred mesh (host arrays)."""

    dims: tuple
    positions: np.ndarray  # [n][3] f64
    edge_nodes: np.ndarray  # [E][2] int32, edge_nodes[e] = (i, j)
    normals: np.ndarray  # [E][3] f64, dual-face normal n_ij (from i to j)
    vol: np.ndarray  # [n] f64
    # [E] int8 or None: +1 when node j of the edge is seen from node i across
    # the pitchwise periodic boundary (its image in the next blade passage)
    periodic: np.ndarray = None

    @property
    def n_nodes(self) -> int:
        return int(self.vol.shape[0])

    @property
    def n_edges(self) -> int:
        return int(self.edge_nodes.shape[0])


def hex_mesh(nx: int, ny: int, nz: int, seed: int = 1, perturb: float = 0.1, periodic_y: bool = False) -> Mesh:
    """Perturbed hex lattice treated as an unstructured edge mesh.  With
    periodic_y the passage repeats with pitch ny along y: edges join every
    node of the last y-layer to the image (y + ny) of the node of the first
    layer, flagged in `periodic`."""
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    pos = base + rng.uniform(-perturb, perturb, size=(n, 3))
    ids = np.arange(n, dtype=np.int64).reshape(nz, ny, nx)

    edges = []
    if nx > 1:
        edges.append(np.stack([ids[:, :, :-1].ravel(), ids[:, :, 1:].ravel()], axis=1))
    if ny > 1:
        edges.append(np.stack([ids[:, :-1, :].ravel(), ids[:, 1:, :].ravel()], axis=1))
    if nz > 1:
        edges.append(np.stack([ids[:-1, :, :].ravel(), ids[1:, :, :].ravel()], axis=1))
    if edges:
        en = np.concatenate(edges, axis=0)
    else:
        en = np.zeros((0, 2), dtype=np.int64)
    normals = pos[en[:, 1]] - pos[en[:, 0]] if len(en) else np.zeros((0, 3))
    periodic = None
    if periodic_y and ny > 2:
        top, bot = ids[:, -1, :].ravel(), ids[:, 0, :].ravel()
        pen = np.stack([top, bot], axis=1)
        pnorm = (pos[bot] + np.array([0.0, float(ny), 0.0])) - pos[top]
        periodic = np.concatenate([np.zeros(len(en), np.int8), np.ones(len(pen), np.int8)])
        en = np.concatenate([en, pen], axis=0)
        normals = np.concatenate([normals, pnorm], axis=0)

    # control volume: product over axes of half the neighbour span
    p3 = pos.reshape(nz, ny, nx, 3)
    vol = np.ones((nz, ny, nx))
    for axis, size in ((2, nx), (1, ny), (0, nz)):
        if size == 1:
            continue  # no neighbours along this axis: unit extent
        fwd = np.roll(p3, -1, axis=axis)
        bwd = np.roll(p3, 1, axis=axis)
        span = 0.5 * np.linalg.norm(fwd - bwd, axis=-1)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = 0
        hi[axis] = size - 1
        lo_nb = list(lo)
        lo_nb[axis] = 1
        hi_nb = list(hi)
        hi_nb[axis] = size - 2
        span[tuple(lo)] = 0.5 * np.linalg.norm(p3[tuple(lo_nb)] - p3[tuple(lo)], axis=-1)
        span[tuple(hi)] = 0.5 * np.linalg.norm(p3[tuple(hi)] - p3[tuple(hi_nb)], axis=-1)
        vol = vol * span
    return Mesh(
        dims=(nx, ny, nz),
        positions=pos,
        edge_nodes=np.ascontiguousarray(en, dtype=np.int32),
        normals=np.ascontiguousarray(normals, dtype=np.float64),
        vol=np.ascontiguousarray(vol.ravel(), dtype=np.float64),
        periodic=periodic,
    )


def box_partition(dims, parts) -> np.ndarray:
    """Partition id of every node of an nx*ny*nz lattice cut into px*py*pz
    boxes of (nearly) equal size -- the domain decomposition of a parallel
    run, one box per processor.  Node (i, j, k) goes to box
    (i px // nx, j py // ny, k pz // nz), numbered x fastest."""
    nx, ny, nz = dims
    px, py, pz = parts
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    bi, bj, bk = (i * px) // nx, (j * py) // ny, (k * pz) // nz
    return np.ascontiguousarray((bi + px * (bj + py * bk)).ravel(), dtype=np.int32)


def lattice_colors(dims) -> np.ndarray:
    """Red-black colouring of an nx*ny*nz lattice, (i + j + k) mod 2: no two
    lattice neighbours share a colour (nor, for even ny, the two ends of a
    pitchwise periodic edge)."""
    nx, ny, nz = dims
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.ascontiguousarray(((i + j + k) % 2).ravel(), dtype=np.int32)


def custom_mesh(positions, edge_nodes, vol=None) -> Mesh:
    """Mesh from explicit positions and edges (tiny hand-made cases)."""
    pos = np.asarray(positions, dtype=np.float64).reshape(-1, 3)
    en = np.asarray(edge_nodes, dtype=np.int32).reshape(-1, 2)
    normals = pos[en[:, 1]] - pos[en[:, 0]] if len(en) else np.zeros((0, 3))
    if vol is None:
        vol = np.ones(pos.shape[0])
    return Mesh(dims=(pos.shape[0], 1, 1), positions=pos, edge_nodes=en,
                normals=np.ascontiguousarray(normals), vol=np.asarray(vol, dtype=np.float64))


def permute_mesh(mesh: Mesh, seed: int = 4, perm=None) -> tuple[Mesh, np.ndarray]:
    """Renumber the nodes: randomly (locality stress variant) or by the given
    permutation. Returns (mesh, perm) where new node ``p`` is old node
    ``perm[p]``."""
    n = mesh.n_nodes
    if perm is None:
        perm = np.random.default_rng(seed).permutation(n)
    perm = np.asarray(perm, dtype=np.int64)
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    en = inv[mesh.edge_nodes.astype(np.int64)]
    swap = en[:, 0] > en[:, 1]
    normals = np.where(swap[:, None], -mesh.normals, mesh.normals)
    en = np.sort(en, axis=1)
    periodic = None
    if mesh.periodic is not None:  # the offset is seen from the edge's first node
        periodic = np.where(swap, -mesh.periodic, mesh.periodic).astype(np.int8)
    return Mesh(dims=mesh.dims, positions=mesh.positions[perm], edge_nodes=en.astype(np.int32),
                normals=np.ascontiguousarray(normals), vol=mesh.vol[perm].copy(), periodic=periodic), perm


def flow_state(n: int, block: int, seed: int = 2, uniform: bool = False) -> np.ndarray:
    """Near-uniform conservative state Q[n][b] = (rho, rho u, rho v, rho w, rho E[, rho nu])."""
    if block not in (5, 6):
        raise ValueError("block must be 5 or 6")
    rng = np.random.default_rng(seed)
    if uniform:
        rho = np.ones(n)
        mach = np.full(n, 0.5)
    else:
        rho = 1.0 + rng.uniform(-0.02, 0.02, n)
        mach = 0.5 + rng.uniform(-0.05, 0.05, n)
    p = np.full(n, 1.0 / GAMMA)
    a = np.sqrt(GAMMA * p / rho)
    u = mach * a
    q = np.zeros((n, block))
    q[:, 0] = rho
    q[:, 1] = rho * u
    q[:, 4] = p / (GAMMA - 1.0) + 0.5 * rho * u * u
    if block == 6:
        q[:, 5] = rho * NU_TILDE
    return q


def rhs(n: int, block: int, n_harm: int, seed: int = 3) -> np.ndarray:
    """B = -R in the [n][1+2N][b] layout."""
    rng = np.random.default_rng(seed)
    r0 = rng.standard_normal((n, block))
    rh = rng.standard_normal((n, n_harm, 2, block)) * np.sqrt(0.5)
    b = np.empty((n, 1 + 2 * n_harm, block))
    b[:, 0, :] = -r0
    b[:, 1:, :] = -rh.reshape(n, 2 * n_harm, block)
    return b


def omegas(n_harm: int, base: float = 1.0) -> np.ndarray:
    """omega_l = l * base, l = 1..N."""
    return base * np.arange(1, n_harm + 1, dtype=np.float64)


@dataclass
class Problem:
    mesh: Mesh
    q: np.ndarray
    b: np.ndarray
    omega: np.ndarray
    block: int
    cfl: float
    name: str = ""
    extra: dict = field(default_factory=dict)
    # inter-blade phase angle of each harmonic (phase-lagged periodicity), or None
    phase: np.ndarray = None

    @property
    def n_harm(self) -> int:
        return int(self.omega.shape[0])

    @property
    def n_cols(self) -> int:
        return 1 + 2 * self.n_harm


def phases(n_harm: int, blades: int = 8, nodal: int = 3) -> np.ndarray:
    """Inter-blade phase angles sigma_l = 2 pi l m / N_b of harmonic l for a
    disturbance of nodal diameter m on N_b blades."""
    return 2.0 * np.pi * nodal * np.arange(1, n_harm + 1, dtype=np.float64) / blades


def problem(dims, block, n_harm, cfl, omega_base=1.0, seeds=(1, 2, 3), name="", periodic=False,
            phase=None) -> Problem:
    mesh = hex_mesh(*dims, seed=seeds[0], periodic_y=periodic)
    q = flow_state(mesh.n_nodes, block, seed=seeds[1])
    b = rhs(mesh.n_nodes, block, n_harm, seed=seeds[2])
    if periodic and phase is None:
        phase = phases(n_harm)
    return Problem(mesh=mesh, q=q, b=b, omega=omegas(n_harm, omega_base), block=block, cfl=cfl, name=name,
                   phase=None if phase is None else np.asarray(phase, dtype=np.float64))


# Workload table: the five configurations of the measurement plan.
CONFIGS = {
    "c1": dict(dims=(16, 8, 8), block=5, n_harm=1, cfl=10.0, omega_base=1.0, sweeps=20),
    "c2": dict(dims=(128, 64, 48), block=6, n_harm=4, cfl=20.0, omega_base=1.0, sweeps=50),
    "c3": dict(dims=(160, 128, 102), block=6, n_harm=8, cfl=20.0, omega_base=1.0, tol=1e-8),
    "c4_row0": dict(dims=(80, 50, 50), block=6, n_harm=2, cfl=20.0, omega_base=1.0),
    "c4_row1": dict(dims=(100, 75, 80), block=6, n_harm=8, cfl=20.0, omega_base=1.6),
    "c4_row2": dict(dims=(125, 110, 80), block=6, n_harm=4, cfl=20.0, omega_base=2.3),
    "c5": dict(dims=(256, 200, 156), block=6, n_harm=16, cfl=20.0, omega_base=1.0, tol=1e-8),
}


def config_problem(key: str, **overrides) -> Problem:
    c = dict(CONFIGS[key])
    c.update(overrides)
    return problem(c["dims"], c["block"], c["n_harm"], c["cfl"], c.get("omega_base", 1.0), name=key)

"""Seeded synthetic inputs: tetrahedral box meshes and initial flow states.

This module is the one piece of code that both the CUDA path and the CPU
oracle consume.  It builds node coordinates, tetrahedra, per-face boundary
tags and primitive initial states; it holds none of the solver's arithmetic
(no geometry beyond node averages, no fluxes, no time stepping).

The paper's workloads (an Ariane 5 take-off blast wave on 10M and 80M cell
Airbus meshes, Sec. 5) are not available, so these generators stand in for
them: graded, jittered tetrahedral boxes carrying a spherical (or
half-spherical, ground-plane) blast wave, and a Sod tube for the single-level
case.

Conventions shared with the C ABI (``include/fv.h``):

* ``xyz``     float64 (n_nodes, 3)
* ``tets``    int64   (n_tets, 4), positively oriented
              (det[x1-x0, x2-x0, x3-x0] > 0)
* ``face_bc`` int8    (n_tets, 4); entry j tags the face opposite local node j:
              0 interior, 1 slip wall, 2 transmissive
* ``prim``    float64 (5, n_tets) structure of arrays: rho, u, v, w, p

Randomness comes from ``numpy.random.default_rng(seed)`` (PCG64), which is
deterministic across platforms.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BC_INTERIOR = 0
BC_WALL = 1
BC_TRANSMISSIVE = 2

DEFAULT_SEED = 1704011440

# Kuhn (Freudenthal) split of a unit cube into 6 tetrahedra: every tet walks
# from corner (0,0,0) to corner (1,1,1) along the axes in the order of one
# permutation.  The split is conforming between translated cubes.
_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def _kuhn_corner_offsets():
    """(6, 4, 3) integer corner offsets of the six Kuhn tets of a cube."""
    out = np.zeros((6, 4, 3), dtype=np.int64)
    for t, perm in enumerate(_PERMS):
        cur = np.zeros(3, dtype=np.int64)
        out[t, 0] = cur
        for step, ax in enumerate(perm):
            cur = cur.copy()
            cur[ax] = 1
            out[t, step + 1] = cur
    # Orient every tet positively on the unit cube (swap the last two nodes
    # when the reference volume is negative).
    for t in range(6):
        a, b, c, d = out[t].astype(np.float64)
        det = np.dot(np.cross(b - a, c - a), d - a)
        if det < 0:
            out[t, [2, 3]] = out[t, [3, 2]]
    return out


_KUHN = _kuhn_corner_offsets()


def graded_coords(n: int, ratio: float) -> np.ndarray:
    """n+1 node coordinates on [0, 1], spacing geometric about the centre.

    Interval sizes grow geometrically from the middle interval(s) to the two
    end intervals, whose size is ``ratio`` times the middle one.  ratio == 1
    gives a uniform grid.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    c = 0.5 * (n - 1)
    if n == 1 or ratio == 1.0:
        h = np.ones(n)
    else:
        q = ratio ** (1.0 / c)
        h = q ** np.abs(np.arange(n) - c)
    x = np.concatenate([[0.0], np.cumsum(h)])
    x /= x[-1]
    x[0], x[-1] = 0.0, 1.0
    return x


def graded_coords_toward(n: int, ratio: float, towards_low: bool) -> np.ndarray:
    """n+1 coordinates on [0, 1], finest at 0 (towards_low) and ``ratio``
    times coarser at the other end (used for the ground-plane axis)."""
    if n == 1 or ratio == 1.0:
        h = np.ones(n)
    else:
        q = ratio ** (1.0 / (n - 1))
        h = q ** np.arange(n)
        if not towards_low:
            h = h[::-1]
    x = np.concatenate([[0.0], np.cumsum(h)])
    x /= x[-1]
    x[0], x[-1] = 0.0, 1.0
    return x


@dataclasses.dataclass
class TetMesh:
    xyz: np.ndarray       # (n_nodes, 3) float64
    tets: np.ndarray      # (n_tets, 4) int64
    face_bc: np.ndarray   # (n_tets, 4) int8
    shape: tuple          # (nx, ny, nz) cubes

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    def centroids(self) -> np.ndarray:
        """(n_tets, 3) vertex averages, used only to place initial data."""
        return self.xyz[self.tets].mean(axis=1)


def box_tet_mesh(xc, yc, zc, bc_planes=None, jitter=0.0, rng=None) -> TetMesh:
    """Kuhn-split tetrahedral mesh of the box spanned by the node coordinate
    vectors ``xc``, ``yc``, ``zc`` (each increasing).

    bc_planes: dict with keys 'x0','x1','y0','y1','z0','z1' giving the tag
    (BC_WALL or BC_TRANSMISSIVE) of each box side; default: all walls.
    jitter: interior node coordinates move by U(-jitter, jitter) times the
    local spacing along each axis on which the node is interior, so boundary
    nodes slide inside their planes only.
    """
    xc, yc, zc = (np.asarray(a, dtype=np.float64) for a in (xc, yc, zc))
    nx, ny, nz = len(xc) - 1, len(yc) - 1, len(zc) - 1
    planes = {k: BC_WALL for k in ("x0", "x1", "y0", "y1", "z0", "z1")}
    if bc_planes:
        planes.update(bc_planes)

    # node grid (i fastest)
    I, J, K = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    I = I.transpose(2, 1, 0).ravel()
    J = J.transpose(2, 1, 0).ravel()
    K = K.transpose(2, 1, 0).ravel()
    xyz = np.stack([xc[I], yc[J], zc[K]], axis=1)

    if jitter > 0.0:
        if rng is None:
            raise ValueError("jitter needs an rng")
        for ax, (coords, idx, n) in enumerate(((xc, I, nx), (yc, J, ny), (zc, K, nz))):
            h = np.diff(coords)
            local = np.full(n + 1, np.inf)
            local[1:] = np.minimum(local[1:], h)
            local[:-1] = np.minimum(local[:-1], h)
            interior = (idx > 0) & (idx < n)
            d = rng.uniform(-jitter, jitter, size=idx.shape[0]) * local[idx]
            xyz[:, ax] = np.where(interior, xyz[:, ax] + d, xyz[:, ax])

    def node_id(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    # cubes (i fastest), 6 tets each -> tets ordered cube-major
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    n_cubes = ci.shape[0]
    tets = np.empty((n_cubes, 6, 4), dtype=np.int64)
    ti = np.empty((n_cubes, 6, 4), dtype=np.int64)
    tj = np.empty_like(ti)
    tk = np.empty_like(ti)
    for t in range(6):
        for v in range(4):
            o = _KUHN[t, v]
            ti[:, t, v] = ci + o[0]
            tj[:, t, v] = cj + o[1]
            tk[:, t, v] = ck + o[2]
            tets[:, t, v] = node_id(ti[:, t, v], tj[:, t, v], tk[:, t, v])
    tets = tets.reshape(-1, 4)
    ti = ti.reshape(-1, 4)
    tj = tj.reshape(-1, 4)
    tk = tk.reshape(-1, 4)

    # boundary tags: the face opposite local node j lies on a box side when its
    # three nodes share that side's integer index.
    face_bc = np.zeros((tets.shape[0], 4), dtype=np.int8)
    for j in range(4):
        others = [v for v in range(4) if v != j]
        for arr, n, lo, hi in ((ti, nx, "x0", "x1"), (tj, ny, "y0", "y1"), (tk, nz, "z0", "z1")):
            sub = arr[:, others]
            on_lo = np.all(sub == 0, axis=1)
            on_hi = np.all(sub == n, axis=1)
            face_bc[on_lo, j] = planes[lo]
            face_bc[on_hi, j] = planes[hi]

    mesh = TetMesh(xyz=xyz, tets=tets, face_bc=face_bc, shape=(nx, ny, nz))
    return mesh


def sod_case(nx: int = 64, ny: int = 4, nz: int = 4, length: float = 1.0):
    """Sod tube along x on [0, length] x [0, ny*h] x [0, nz*h], h = length/nx.

    Left state (rho, u, p) = (1, 0, 1) for centroid x < length/2, right state
    (0.125, 0, 0.1); slip walls on the y/z sides, transmissive x ends.
    Returns (mesh, prim).
    """
    h = length / nx
    xc = np.linspace(0.0, length, nx + 1)
    yc = np.linspace(0.0, ny * h, ny + 1)
    zc = np.linspace(0.0, nz * h, nz + 1)
    mesh = box_tet_mesh(xc, yc, zc, bc_planes={"x0": BC_TRANSMISSIVE, "x1": BC_TRANSMISSIVE})
    c = mesh.centroids()
    left = c[:, 0] < 0.5 * length
    prim = np.empty((5, mesh.n_tets))
    prim[0] = np.where(left, 1.0, 0.125)
    prim[1:4] = 0.0
    prim[4] = np.where(left, 1.0, 0.1)
    return mesh, prim


def blast_case(n: int = 55, ratio: float = 8.0, seed: int = DEFAULT_SEED, jitter: float = 0.1,
               radius: float = 0.1, p_in: float = 10.0, p_out: float = 0.1, rho: float = 1.0,
               centre=(0.5, 0.5, 0.5)):
    """Spherical blast wave in the unit box, node spacing graded geometrically
    toward the centre (edge/centre ratio ``ratio``), seeded jitter, slip walls.

    n cubes per axis -> 6 n^3 tets (n = 55 gives 998,250).
    Returns (mesh, prim).
    """
    rng = np.random.default_rng(seed)
    x = graded_coords(n, ratio)
    mesh = box_tet_mesh(x, x, x, jitter=jitter, rng=rng)
    c = mesh.centroids()
    r = np.linalg.norm(c - np.asarray(centre), axis=1)
    prim = np.empty((5, mesh.n_tets))
    prim[0] = rho
    prim[1:4] = 0.0
    prim[4] = np.where(r < radius, p_in, p_out)
    return mesh, prim


def ground_blast_case(n: int = 237, ratio: float = 8.0, seed: int = DEFAULT_SEED + 4,
                      jitter: float = 0.1, radius: float = 0.1, p_in: float = 20.0,
                      p_out: float = 0.1, rho: float = 1.0):
    """Half-sphere blast on the ground plane z = 0 of the unit box: mesh
    graded toward (0.5, 0.5, 0), slip walls everywhere (the ground is a wall)."""
    rng = np.random.default_rng(seed)
    x = graded_coords(n, ratio)
    z = graded_coords_toward(n, ratio, towards_low=True)
    mesh = box_tet_mesh(x, x, z, jitter=jitter, rng=rng)
    c = mesh.centroids()
    r = np.linalg.norm(c - np.array([0.5, 0.5, 0.0]), axis=1)
    prim = np.empty((5, mesh.n_tets))
    prim[0] = rho
    prim[1:4] = 0.0
    prim[4] = np.where(r < radius, p_in, p_out)
    return mesh, prim


def uniform_flow_case(n: int = 6, seed: int = DEFAULT_SEED + 7, jitter: float = 0.1,
                      state=(1.0, 0.3, -0.2, 0.1, 0.8), ratio: float = 4.0):
    """Jittered graded box, transmissive on every side, carrying one uniform
    state (used for free-stream preservation)."""
    rng = np.random.default_rng(seed)
    x = graded_coords(n, ratio)
    planes = {k: BC_TRANSMISSIVE for k in ("x0", "x1", "y0", "y1", "z0", "z1")}
    mesh = box_tet_mesh(x, x, x, bc_planes=planes, jitter=jitter, rng=rng)
    prim = np.empty((5, mesh.n_tets))
    for c in range(5):
        prim[c] = state[c]
    return mesh, prim


@dataclasses.dataclass
class BatchInstance:
    mesh: TetMesh
    prim: np.ndarray
    max_levels: int
    seed: int


def batch_cases(count: int = 64, seed: int = DEFAULT_SEED + 2, min_tets: float = 2e4,
                max_tets: float = 5e5, ratio: float = 8.0):
    """Independent blast-wave instances with sizes log-uniform in
    [min_tets, max_tets], level caps uniform in {1..5}, blast radius uniform
    in [0.05, 0.2] and pressure ratio log-uniform in [5, 100]."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        size = math.exp(rng.uniform(math.log(min_tets), math.log(max_tets)))
        n = max(2, int(round((size / 6.0) ** (1.0 / 3.0))))
        levels = int(rng.integers(1, 6))
        radius = float(rng.uniform(0.05, 0.2))
        pr = math.exp(rng.uniform(math.log(5.0), math.log(100.0)))
        sub_seed = int(rng.integers(0, 2**31 - 1))
        mesh, prim = blast_case(n=n, ratio=ratio, seed=sub_seed, radius=radius,
                                p_in=0.1 * pr, p_out=0.1)
        out.append(BatchInstance(mesh=mesh, prim=prim, max_levels=levels, seed=sub_seed))
    return out

"""The seeded synthetic workloads match their stated recipe (CPU).

The generators hold no arithmetic of the method; these tests check the
meshes and initial states they produce: sizes, grading, jitter bounds,
boundary tags, positive volumes, the initial blast, and the batch's
parameter ranges.
"""
import math

import numpy as np
import pytest

from paper_1704_01144_gb300 import inputs as I


def _volumes(mesh):
    x = mesh.xyz[mesh.tets]
    return np.einsum("ij,ij->i", x[:, 1] - x[:, 0],
                     np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0])) / 6.0


@pytest.mark.parametrize("n,ratio", [(55, 8.0), (13, 3.0), (7, 1.0)])
def test_graded_coords_are_geometric_about_the_centre(n, ratio):
    x = I.graded_coords(n, ratio)
    h = np.diff(x)
    assert x[0] == 0.0 and x[-1] == 1.0 and (h > 0).all()
    np.testing.assert_allclose(h, h[::-1], rtol=1e-12)            # symmetric
    assert h[0] / h.min() == pytest.approx(ratio, rel=1e-12)       # edge / centre
    q = h[1:] / h[:-1]                                             # one ratio per side
    half = n // 2
    assert np.allclose(q[: half - 1], q[0]) and np.allclose(q[-(half - 1):], q[-1])


def test_graded_coords_toward_the_ground():
    z = I.graded_coords_toward(20, 8.0, towards_low=True)
    h = np.diff(z)
    assert z[0] == 0.0 and z[-1] == 1.0 and h[-1] / h[0] == pytest.approx(8.0, rel=1e-12)
    assert (np.diff(h) > 0).all()


def test_blast_mesh_recipe():
    """6 n^3 Kuhn tets, all positively oriented; boundary nodes on their
    planes; interior nodes within 10 % of the local spacing of the graded
    grid; every boundary face a slip wall; p_in inside r < 0.1."""
    n = 12
    mesh, prim = I.blast_case(n=n, ratio=8.0)
    assert mesh.n_tets == 6 * n ** 3 and mesh.n_nodes == (n + 1) ** 3
    assert (_volumes(mesh) > 0).all()
    assert _volumes(mesh).sum() == pytest.approx(1.0, rel=1e-12)
    x = I.graded_coords(n, 8.0)
    h = np.diff(x)
    local = np.minimum(np.concatenate([[np.inf], h]), np.concatenate([h, [np.inf]]))
    # node (i, j, k) is number i + (n+1) (j + (n+1) k): i fastest
    k, j, i = np.meshgrid(*[np.arange(n + 1)] * 3, indexing="ij")
    idx = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    d = mesh.xyz - x[idx]
    for a in range(3):
        on_plane = (idx[:, a] == 0) | (idx[:, a] == n)
        assert (d[on_plane, a] == 0.0).all()                         # stays on its plane
        assert (np.abs(d[:, a]) <= 0.1 * local[idx[:, a]] + 1e-15).all()
    assert np.abs(d).max() > 0.05 * h.min()                          # jitter applied
    bc = mesh.face_bc
    assert set(np.unique(bc)) == {0, I.BC_WALL}
    assert (bc != 0).sum() == 6 * 2 * n * n                          # two triangles per square
    c = mesh.centroids()
    inside = np.linalg.norm(c - 0.5, axis=1) < 0.1
    assert inside.any() and (prim[4][inside] == 10.0).all() and (prim[4][~inside] == 0.1).all()
    assert (prim[0] == 1.0).all() and (prim[1:4] == 0.0).all()


def test_full_size_blast_and_sod_sizes():
    mesh, _ = I.blast_case()
    assert mesh.n_tets == 998_250
    mesh, prim = I.sod_case()
    assert mesh.n_tets == 6_144
    c = mesh.centroids()
    left = c[:, 0] < 0.5
    assert (prim[0][left] == 1.0).all() and (prim[0][~left] == 0.125).all()
    assert (prim[4][left] == 1.0).all() and (prim[4][~left] == 0.1).all()
    assert set(np.unique(mesh.face_bc)) == {0, I.BC_WALL, I.BC_TRANSMISSIVE}


def test_seeds_reproduce_and_differ():
    a, _ = I.blast_case(n=5)
    b, _ = I.blast_case(n=5)
    c, _ = I.blast_case(n=5, seed=I.DEFAULT_SEED + 99)
    np.testing.assert_array_equal(a.xyz, b.xyz)
    assert not np.array_equal(a.xyz, c.xyz)


def test_batch_recipe():
    """64 instances: sizes within [2e4, 5e5] tets up to the rounding of n,
    level caps in 1..5 (all used), blast radius in [0.05, 0.2] and pressure
    ratio in [5, 100]; 9,361,332 tets in all."""
    insts = I.batch_cases()
    assert len(insts) == 64
    sizes = np.array([b.mesh.n_tets for b in insts])
    assert sizes.sum() == 9_361_332
    n = np.array([b.mesh.shape[0] for b in insts])
    assert ((6 * (n - 0.5) ** 3 <= 5e5) & (6 * (n + 0.5) ** 3 >= 2e4)).all()
    assert set(b.max_levels for b in insts) == {1, 2, 3, 4, 5}
    for b in insts:
        p_in, p_out = b.prim[4].max(), b.prim[4].min()
        assert p_out == pytest.approx(0.1) and 5.0 <= p_in / p_out <= 100.0
        c = b.mesh.centroids()
        r_in = np.linalg.norm(c[b.prim[4] == p_in] - 0.5, axis=1).max()
        r_out = np.linalg.norm(c[b.prim[4] == p_out] - 0.5, axis=1).min()
        assert r_in < r_out and r_in < 0.2 and r_out >= 0.05 - 1e-12
    logs = np.log(sizes)
    assert logs.min() < math.log(4e4) and logs.max() > math.log(2.5e5)  # spread over the range

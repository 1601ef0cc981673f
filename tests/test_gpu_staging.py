"""The FP32 flux kernel that stages its gathered inputs through shared memory
(k_flux_staged, off by default) against the one that loads them into
registers: the same operations on the same values, so the states after
several multi-level cycles are bitwise equal, in both orders of the level
steps and with ragged face counts (a tiny mesh, fewer faces than threads)."""
import numpy as np
import pytest

from paper_1704_01144_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_01144_gb300 import build, fv as F
    build.build()
    return F


def _run(fv, mesh, prim, L, staged, order, cycles):
    g = fv.Mesh(mesh, max_levels=L, precision=fv.FV_FP32_FLUX)
    assert g.get_flux_staging() is False  # the default
    g.set_flux_staging(staged)
    assert g.get_flux_staging() is staged
    g.set_order(order)
    g.set_state(prim)
    g.advance(cycles)
    assert g.status() == 0
    U = g.get_state()
    g.close()
    return U


@pytest.mark.parametrize("n,L,order", [(12, 4, 0), (12, 4, 1), (3, 3, 0), (20, 5, 0)])
def test_staged_flux_bitwise_equal(fv, n, L, order):
    mesh, prim = I.blast_case(n=n, ratio=8.0)
    a = _run(fv, mesh, prim, L, True, order, 3)
    b = _run(fv, mesh, prim, L, False, order, 3)
    np.testing.assert_array_equal(a, b)


def test_staged_flux_ground_blast_walls(fv):
    """The ground blast: wall faces on every side (their records are staged
    without a right cell)."""
    mesh, prim = I.ground_blast_case(n=14)
    a = _run(fv, mesh, prim, 6, True, 0, 2)
    b = _run(fv, mesh, prim, 6, False, 0, 2)
    np.testing.assert_array_equal(a, b)

"""The update's warp-level gather (four lanes per cell, fv_set_gather)
against the per-thread gather: the same values added in the same face order,
so several multi-level cycles end bitwise equal, in both precisions, with
wall faces and a ragged last warp."""
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


def _run(fv, mesh, prim, L, precision, gather, cycles):
    g = fv.Mesh(mesh, max_levels=L, precision=precision)
    assert g.get_gather() == fv.FV_GATHER_THREAD  # the default
    g.set_gather(gather)
    assert g.get_gather() == gather
    g.set_state(prim)
    g.advance(cycles)
    assert g.status() == 0
    U = g.get_state()
    g.close()
    return U


@pytest.mark.parametrize("case,precision", [("blast", 0), ("blast", 1), ("ground", 1), ("tiny", 1)])
def test_quad_gather_bitwise_equal(fv, case, precision):
    if case == "blast":
        (mesh, prim), L, cycles = I.blast_case(n=12, ratio=8.0), 4, 3
    elif case == "ground":
        (mesh, prim), L, cycles = I.ground_blast_case(n=14), 6, 2
    else:
        (mesh, prim), L, cycles = I.blast_case(n=3, ratio=8.0), 3, 3
    a = _run(fv, mesh, prim, L, precision, fv.FV_GATHER_QUAD, cycles)
    b = _run(fv, mesh, prim, L, precision, fv.FV_GATHER_THREAD, cycles)
    np.testing.assert_array_equal(a, b)

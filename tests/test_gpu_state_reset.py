"""fv_set_state / fv_set_conserved restart a run exactly: the interface
accumulators are all zero after every completed cycle and are cleared after
an interrupted one, and the boundary ledger restarts from zero (only
boundary faces ever write it).  A restarted mesh must reproduce a fresh
mesh bit for bit, ledger included."""
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
    F.lib()
    return F


def fresh(fv, mesh, prim, L, precision, order, cycles):
    g = fv.Mesh(mesh, max_levels=L, precision=precision)
    g.set_order(order)
    g.set_state(prim)
    g.advance(cycles)
    out = (g.get_state(), g.boundary_ledger())
    g.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("order", [0, 1])
def test_restart_after_whole_and_interrupted_cycles(fv, precision, order):
    mesh, prim = I.blast_case(n=10, ratio=8.0)
    L = 4
    ref = fresh(fv, mesh, prim, L, precision, order, 2)
    g = fv.Mesh(mesh, max_levels=L, precision=precision)
    g.set_order(order)
    g.set_state(prim)
    g.advance(2)                 # whole cycles: accumulators consumed
    g.set_state(prim)
    g.advance(2)
    U, led = g.get_state(), g.boundary_ledger()
    assert np.array_equal(U, ref[0]) and np.array_equal(led, ref[1])
    g.set_state(prim)
    g.assign_levels()
    g.advance_phases(7)          # stop inside the cycle, interfaces half-accumulated
    g.set_state(prim)
    g.advance(2)
    U, led = g.get_state(), g.boundary_ledger()
    assert np.array_equal(U, ref[0]) and np.array_equal(led, ref[1])
    assert g.status() == 0
    g.close()


def test_restart_from_host_conserved_state(fv):
    """The end-to-end path: the state read back to the host and uploaded
    again continues exactly as the device-resident run."""
    import torch
    mesh, prim = I.blast_case(n=10, ratio=8.0)
    ref = fresh(fv, mesh, prim, 4, 1, 0, 3)
    g = fv.Mesh(mesh, max_levels=4, precision=fv.FV_FP32_FLUX)
    g.set_state(prim)
    host = torch.empty((5, g.n), dtype=torch.float64, pin_memory=True)
    for _ in range(3):
        g.get_state(out=host.numpy())
        g.set_conserved(host)
        g.advance(1)
    assert np.array_equal(g.get_state(), ref[0])
    g.close()

"""The persistent cycle (one cooperative launch per cycle, kernel kinds
separated by a bounded grid barrier): bitwise the per-kernel path's results,
and the barrier's bounded wait reporting a timeout instead of hanging."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_01144_gb300 import build, fv as F
    build.build()
    return F


def test_barrier_completes(fv):
    rc, st = fv.fv_barrier_selftest(rounds=2000, unreachable=False)
    assert rc == fv.FV_OK and st == 0


def test_barrier_wait_runs_out(fv):
    """Every barrier waits for one block more than exists: the waits run out,
    the kernel returns with the timeout bit, and the device stays usable."""
    rc, st = fv.fv_barrier_selftest(rounds=3, unreachable=True)
    assert rc == fv.FV_ERR_TIMEOUT and st & 4
    rc, st = fv.fv_barrier_selftest(rounds=10, unreachable=False)
    assert rc == fv.FV_OK and st == 0


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("graph", [True, False])
def test_persistent_matches_per_kernel(fv, precision, graph):
    import torch
    from paper_1704_01144_gb300 import inputs as I
    mesh, prim = I.blast_case(n=14, ratio=8.0)
    out = []
    for persistent in (False, True):
        m = fv.Mesh(mesh, max_levels=4, precision=precision)
        m.use_graph(graph)
        m.use_persistent(persistent)
        m.set_state(prim)
        s = torch.cuda.Stream()
        m.advance(3, stream=s, want_time=False)
        torch.cuda.synchronize()
        assert m.status() == 0
        out.append((m.get_state(), m.work_counters(), m.levels()))
        m.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2])


def test_persistent_level_one_and_sod(fv):
    """One level (a single phase pair per cycle) and the boundary mix of the
    Sod tube, against the per-kernel path."""
    from paper_1704_01144_gb300 import inputs as I
    mesh, prim = I.sod_case()
    res = []
    for persistent in (False, True):
        m = fv.Mesh(mesh, max_levels=1, precision=fv.FV_FP64)
        m.use_persistent(persistent)
        m.set_state(prim)
        m.advance(20, want_time=False)
        res.append(m.get_state())
        m.close()
    assert np.array_equal(res[0], res[1])

"""The level history (the evolving level distribution the paper follows in
Sec. 5): per cycle, the cells of each level and dt_min, against the oracle's
levels cycle by cycle, in a batch, and across the ring's wrap."""
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


def test_history_matches_oracle_cycle_by_cycle(fv, oracle_mod):
    mesh, prim = I.blast_case(n=10, ratio=8.0)
    L, cycles = 4, 6
    g = fv.Mesh(mesh, max_levels=L)
    g.set_state(prim)
    o = oracle_mod.Oracle(mesh, max_levels=L)
    o.set_prim(prim)
    want, want_dt = [], []
    for _ in range(cycles):
        o.advance(1)
        want.append(np.bincount(o.levels().astype(np.int64), minlength=8))
        want_dt.append(o.dtmin)
    g.advance(cycles, want_time=False)
    counts, dtm = g.level_history()
    assert counts.shape == (cycles, 8)
    assert np.array_equal(counts, np.array(want))
    # cycle 1 starts from the same state: bit-exact; later states agree to
    # the FP64 path's tolerance, and so do their dt_min
    assert dtm[0] == want_dt[0]
    assert np.allclose(dtm, np.array(want_dt), rtol=1e-12, atol=0)
    # the last entry is the current cycle's distribution
    assert np.array_equal(counts[-1], np.bincount(g.levels().astype(np.int64), minlength=8))
    # setting the state starts a new history
    g.set_state(prim)
    assert g.level_history()[0].shape == (0, 8)


def test_history_in_a_batch(fv):
    meshes, alone = [], []
    for n, L in ((6, 2), (8, 3)):
        mesh, prim = I.blast_case(n=n, ratio=8.0)
        for dst in (meshes, alone):
            m = fv.Mesh(mesh, max_levels=L, precision=fv.FV_FP32_FLUX)
            m.set_state(prim)
            dst.append(m)
    b = fv.Batch(meshes)
    b.advance(3)
    for m, a, L in zip(meshes, alone, (2, 3)):
        a.advance(3 * 2 ** (3 - L), want_time=False)
        cb, db = m.level_history()
        ca, da = a.level_history()
        assert np.array_equal(cb, ca) and np.array_equal(db, da)


def test_history_ring_wraps(fv):
    mesh, prim = I.uniform_flow_case(n=3)
    g = fv.Mesh(mesh, max_levels=1)
    g.set_state(prim)
    g.advance(4100, want_time=False)
    counts, dtm = g.level_history()
    assert counts.shape == (4096, 8)
    assert np.all(counts[:, 0] == g.n) and np.all(counts[:, 1:] == 0)
    assert np.all(np.isfinite(dtm)) and np.all(dtm > 0)
    assert g.work_counters()[0] == 4100

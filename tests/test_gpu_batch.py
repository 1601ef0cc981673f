"""Batches (fv_batch_*): many meshes of uneven sizes and level counts in one
launch per kernel kind and phase.  Each instance must come out bitwise equal
to the same mesh advanced on its own (which the parity tests tie to the
oracle)."""
import numpy as np
import pytest

from paper_1704_01144_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fvmod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_01144_gb300 import build, fv
    build.build()
    fv.lib()
    return fv


CASES = [  # (cubes per axis, levels, blast radius, pressure ratio, seed)
    (6, 1, 0.2, 20.0, 1), (9, 4, 0.1, 100.0, 2), (5, 2, 0.15, 5.0, 3), (8, 3, 0.08, 50.0, 4),
    (7, 4, 0.12, 10.0, 5), (4, 2, 0.2, 30.0, 6),
]


def _instances():
    out = []
    for n, L, rad, pr, seed in CASES:
        mesh, prim = I.blast_case(n=n, ratio=8.0, seed=seed, radius=rad, p_in=0.1 * pr, p_out=0.1)
        out.append((mesh, prim, L))
    return out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_meshes_advanced_alone(fvmod, precision, graph):
    import torch
    inst = _instances()
    Lmax = max(L for _, _, L in inst)
    batch_meshes, alone = [], []
    for mesh, prim, L in inst:
        a = fvmod.Mesh(mesh, max_levels=L, precision=precision)
        a.set_state(prim)
        batch_meshes.append(a)
        b = fvmod.Mesh(mesh, max_levels=L, precision=precision)
        b.set_state(prim)
        alone.append(b)
    batch = fvmod.Batch(batch_meshes)
    sub, launches = batch.info()
    assert sub == 2 ** (Lmax - 1)
    n_batch_cycles = 2
    stream = torch.cuda.Stream() if graph else None
    batch.use_graph(graph)
    batch.advance(n_batch_cycles, stream=stream)
    torch.cuda.synchronize()
    for (mesh, prim, L), a, b in zip(inst, batch_meshes, alone):
        cycles = n_batch_cycles * 2 ** (Lmax - L)
        b.advance(cycles)
        assert np.array_equal(a.get_state(), b.get_state()), (mesh.n_tets, L)
        assert np.array_equal(a.levels(), b.levels())
        assert a.t == b.t
        assert a.work_counters() == b.work_counters()
        assert a.status() == 0
    batch.close()


def test_batch_rejects_bad_input(fvmod):
    mesh, prim = I.blast_case(n=4)
    m = fvmod.Mesh(mesh, max_levels=2)
    m.set_state(prim)
    with pytest.raises(fvmod.FvError):
        fvmod.fv_batch_create([m.h, m.h])          # same mesh twice
    other = fvmod.Mesh(mesh, max_levels=2, precision=1)
    with pytest.raises(fvmod.FvError):
        fvmod.fv_batch_create([m.h, other.h])      # mixed precision
    b = fvmod.Batch([m])
    m.assign_levels()
    m.advance_phases(1)                            # mesh inside its own cycle
    with pytest.raises(fvmod.FvError):
        b.advance(1)


def test_launch_config_does_not_change_results(fvmod, tmp_path):
    """Grid sizes are free parameters: any choice (here the autotuner's and
    an extreme one) gives bitwise the same state."""
    import torch
    from paper_1704_01144_gb300 import autotune as AT
    mesh, prim = I.blast_case(n=10, ratio=8.0)
    out = []
    for per_sm in ([1, 2, 1, 3], [16, 16, 32, 16], None):
        g = fvmod.Mesh(mesh, max_levels=4, precision=1)
        g.set_state(prim)
        if per_sm is None:
            per_sm, info = AT.autotune(g, "test", cache_path=str(tmp_path / "at.json"), reps=1)
            assert not info["cached"] and len(info["tried"]) >= 4
            g.set_state(prim)
        else:
            g.set_launch(per_sm)
        assert g.get_launch() == list(per_sm)
        g.advance(2, stream=torch.cuda.Stream())
        torch.cuda.synchronize()
        out.append(g.get_state())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
    g2 = fvmod.Mesh(mesh, max_levels=4, precision=1)
    per_sm2, info2 = AT.autotune(g2, "test", cache_path=str(tmp_path / "at.json"))
    assert info2["cached"] and per_sm2 == per_sm

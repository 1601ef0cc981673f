"""Gradient-flux fusion of latency-bound phases (FP32-flux mode).

A phase with at most `max_faces` faces computes both cells' least-squares
gradients inside its flux kernel instead of in a gradient kernel of its own.
The fused path performs the same operations on the same values as the
gradient kernel followed by the plain flux kernel, so both paths must give
bitwise identical states, levels and boundary ledgers, whichever phases of
a cycle fuse; and the fused path must meet the FP32-flux tolerance against
the FP64 oracle on its own.
"""
import numpy as np
import pytest

from paper_1704_01144_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ALL = 1 << 30  # every phase fuses
TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def fv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_01144_gb300 import build, fv as F
    build.build()
    F.lib()
    return F


def run(fv, mesh, prim, L, fusion, cycles, mlp=None):
    g = fv.Mesh(mesh, max_levels=L, precision=fv.FV_FP32_FLUX)
    g.set_fusion(fusion)
    assert g.get_fusion() == fusion
    if mlp is not None:
        g.mlp_load(*mlp)
    g.set_state(prim)
    for _ in range(cycles):
        g.advance(1, want_time=False)
    assert g.status() == 0
    out = (g.get_state(), g.levels(), g.boundary_ledger())
    g.close()
    return out


def assert_same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("n,L", [(12, 4), (9, 3), (7, 1)])
def test_fused_equals_split_bitwise(fv, n, L):
    mesh, prim = I.blast_case(n=n, ratio=8.0)
    assert_same(run(fv, mesh, prim, L, 0, 3), run(fv, mesh, prim, L, ALL, 3))


def test_mixed_threshold_equals_split_bitwise(fv):
    """A threshold between the phases' sizes: the phases of the fine levels
    fuse, those that cover the whole mesh do not."""
    mesh, prim = I.blast_case(n=20, ratio=8.0)
    L = 4
    g = fv.Mesh(mesh, max_levels=L, precision=fv.FV_FP32_FLUX)
    g.set_state(prim)
    _, counts = g.assign_levels()
    nf = g.nf
    g.close()
    assert counts[L - 1] < g.n  # several levels, so phases differ in size
    split = run(fv, mesh, prim, L, 0, 2)
    assert_same(split, run(fv, mesh, prim, L, nf // 2, 2))
    assert_same(split, run(fv, mesh, prim, L, ALL, 2))


@pytest.mark.parametrize("fusion", [0, ALL])
def test_both_paths_against_fp64_oracle(fv, oracle_mod, fusion):
    mesh, prim = I.blast_case(n=12, ratio=8.0)
    L = 4
    o = oracle_mod.Oracle(mesh, max_levels=L)
    o.set_prim(prim)
    o.advance(3)
    U, lev, _ = run(fv, mesh, prim, L, fusion, 3)
    np.testing.assert_array_equal(lev, o.levels())
    Uo = o.get_cons()
    m = np.sqrt((Uo[1:4] ** 2).sum(axis=0)).max()
    scale = np.array([np.abs(Uo[0]).max(), m, m, m, np.abs(Uo[4]).max()])
    err = (np.abs(U - Uo).max(axis=1) / scale).max()
    assert err <= TOL_FP32, err


def test_learned_guess_ignores_fusion(fv):
    """The learned guess has its own flux kernel, which reads the gradient
    records: with it the gradient kernel must run whatever the threshold."""
    import torch
    mesh, prim = I.blast_case(n=9, ratio=8.0)
    th = torch.from_numpy(fv.fv_mlp_init(7).astype(np.float32)).cuda()
    mlp = (th, fv.FV_MLP_TARGET_TR, -1.0)
    assert_same(run(fv, mesh, prim, 3, 0, 2, mlp), run(fv, mesh, prim, 3, ALL, 2, mlp))


def test_fusion_setter(fv):
    mesh, prim = I.blast_case(n=6)
    g = fv.Mesh(mesh, max_levels=2, precision=fv.FV_FP32_FLUX)
    assert g.get_fusion() == fv.FV_FUSE_FACES_DEFAULT
    with pytest.raises(fv.FvError):
        g.set_fusion(-1)
    g.set_state(prim)
    g.assign_levels()
    g.advance_phases(1)
    with pytest.raises(fv.FvError):
        g.set_fusion(0)  # inside a cycle
    g.advance_phases(2)  # the cycle of L = 2 has 3 * 2 - 1 = 5 phases
    g.advance_phases(2)
    g.set_fusion(0)
    assert g.get_fusion() == 0
    g.close()

"""Sharded runs on the GPU (Sec. 3.3 / 4.3 domain decomposition): the mesh
cut into level-weighted subdomains with ghost layers, every phase followed
by the ghost states from their owners, against the FP64 oracle on the whole
mesh after several multi-level cycles -- in one process (every subdomain on
the device, device-copy exchanges) and as two ranks on one device whose
exchanges are staged through host memory over gloo."""
import os

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


def _rel_pc(U, Uo):
    return np.abs(U - Uo).max(axis=1) / np.abs(Uo).max(axis=1)


def _oracle(oracle_mod, mesh, prim, L, cycles):
    o = oracle_mod.Oracle(mesh, max_levels=L)
    o.set_prim(prim)
    o.advance(cycles)
    return o.get_cons()


@pytest.mark.parametrize("case,n_parts,precision,tol", [
    ("blast", 2, 0, 1e-12), ("blast", 3, 0, 1e-12), ("blast", 2, 1, 1e-5), ("ground", 3, 0, 1e-12)])
def test_sharded_run_matches_oracle(fv, oracle_mod, case, n_parts, precision, tol):
    from paper_1704_01144_gb300 import shard as S
    if case == "blast":
        mesh, prim = I.blast_case(n=12, ratio=8.0)
        L, cycles = 4, 3
    else:
        mesh, prim = I.ground_blast_case(n=14)
        L, cycles = 6, 2
    run = S.ShardedRun(mesh, prim, L, n_parts, precision=precision)
    assert len(run.subs) == n_parts
    assert min(sd.n_owned for sd in run.subs) > 0
    run.advance(cycles)
    assert run.status() == 0
    U = run.get_state()
    Uo = _oracle(oracle_mod, mesh, prim, L, cycles)
    err = _rel_pc(U, Uo)
    print(f"{case}, {n_parts} subdomains, precision {precision}: {err.max():.2e}")
    assert err.max() <= tol, err
    # the same mesh unsharded on the GPU: the subdomains' owned cells carry
    # the same levels, and the states agree to rounding (a border face may
    # take its two cells in the other order in a subdomain's numbering)
    g = fv.Mesh(mesh, max_levels=L, precision=precision)
    g.set_state(prim)
    g.advance(cycles)
    lev = g.levels()
    for sd, m in zip(run.subs, run.meshes):
        np.testing.assert_array_equal(m.levels()[:sd.n_owned], lev[sd.cells[:sd.n_owned]])
    assert _rel_pc(U, g.get_state()).max() <= (1e-13 if precision == 0 else 1e-5)
    g.close()
    run.close()


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_1704_01144_gb300 import shard as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mesh, prim = I.blast_case(n=12, ratio=8.0)
        r = S.ShardedRank(mesh, prim, 4, precision=0)
        for _ in range(3):
            r.cycle()
        ids, U = r.owned_state()
        out.put((rank, ids, U, r.mesh.status()))
        r.close()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_on_one_device_match_oracle(fv, oracle_mod):
    """Two processes, one subdomain each, on the same GPU; between phases
    each rank packs its border cells, moves them through host memory with
    gloo point-to-point messages and unpacks its ghosts (no kernel waits on
    the other process)."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    mesh, prim = I.blast_case(n=12, ratio=8.0)
    U = np.full((5, mesh.n_tets), np.nan)
    for rank, ids, Ur, st in res:
        assert st == 0
        U[:, ids] = Ur
    assert not np.isnan(U).any()
    Uo = _oracle(oracle_mod, mesh, prim, 4, 3)
    err = _rel_pc(U, Uo)
    print(f"two gloo ranks: {err.max():.2e}")
    assert err.max() <= 1e-12, err

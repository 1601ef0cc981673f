"""Host logic of sharded runs (Sec. 3.3 / 4.3 domain decomposition), on the
CPU: the level-weighted partition, the ghost layers, the subdomain meshes,
the exchange plans, the sufficiency of L-1 ghost layers for the level rule,
and the exchange protocol between two gloo ranks."""
import os

import numpy as np
import pytest

from paper_1704_01144_gb300 import inputs as I
from paper_1704_01144_gb300 import shard as S


@pytest.fixture(scope="module")
def blast():
    mesh, prim = I.blast_case(n=10, ratio=8.0)
    return mesh, prim, S.neighbours(mesh.tets)


def _bfs_distance(nbr, sources):
    n = nbr.shape[0]
    dist = np.full(n, -1, dtype=np.int64)
    dist[sources] = 0
    front = np.asarray(sources)
    d = 0
    while front.size:
        d += 1
        cand = nbr[front].ravel()
        cand = np.unique(cand[cand >= 0])
        cand = cand[dist[cand] < 0]
        dist[cand] = d
        front = cand
    return dist


def test_neighbours_are_symmetric(blast):
    mesh, _, nbr = blast
    t, j = np.nonzero(nbr >= 0)
    back = nbr[nbr[t, j]]
    assert np.all((back == t[:, None]).sum(axis=1) == 1)
    # interior faces have no tag, boundary faces have one
    assert np.all((nbr < 0) == (mesh.face_bc != 0))


@pytest.mark.parametrize("n_parts", [2, 3, 5])
def test_partition_balances_level_weights(blast, n_parts):
    mesh, _, _ = blast
    rng = np.random.default_rng(3)
    lev = rng.integers(0, 4, mesh.n_tets)
    w = S.level_weights(lev, 4)
    assert set(np.unique(w)) <= {1.0, 2.0, 4.0, 8.0}
    part = S.partition(mesh, w, n_parts)
    assert part.min() == 0 and part.max() == n_parts - 1
    tot = np.bincount(part, weights=w, minlength=n_parts)
    assert np.abs(tot - w.sum() / n_parts).max() <= w.max()
    # contiguous ranges along the Morton order
    order = S.morton_order(mesh.centroids())
    assert np.all(np.diff(part[order]) >= 0)


def test_morton_order_is_a_permutation_following_the_curve():
    pts = np.array([[0, 0, 0], [1, 1, 1], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    order = S.morton_order(pts)
    assert sorted(order) == list(range(5))
    assert order[0] == 0 and order[-1] == 1   # the corners of the box first and last
    # x is the lowest interleaved bit, then y, then z
    assert list(order) == [0, 2, 3, 4, 1]


@pytest.mark.parametrize("depth", [2, 3])
def test_ghost_layers_are_face_distances(blast, depth):
    mesh, _, nbr = blast
    part = S.partition(mesh, np.ones(mesh.n_tets), 3)
    subs = S.subdomains(mesh, part, depth, nbr)
    for sd in subs:
        owned = sd.cells[:sd.n_owned]
        assert np.all(part[owned] == sd.part) and sd.n_owned == (part == sd.part).sum()
        dist = _bfs_distance(nbr, owned)
        want = np.nonzero((dist >= 1) & (dist <= depth))[0]
        np.testing.assert_array_equal(np.sort(sd.cells[sd.n_owned:]), want)
        np.testing.assert_array_equal(sd.layer[sd.n_owned:], dist[sd.cells[sd.n_owned:]])
        # the local mesh: the same tets; a face is tagged exactly where the
        # local cell has no local neighbour, with the original tag on true
        # boundary faces and the transmissive tag on cut ones
        np.testing.assert_array_equal(sd.mesh.xyz[sd.mesh.tets], mesh.xyz[mesh.tets[sd.cells]])
        lnb = S.neighbours(sd.mesh.tets)
        assert np.all((lnb < 0) == (sd.mesh.face_bc != 0))
        true_bnd = nbr[sd.cells] < 0
        np.testing.assert_array_equal(sd.mesh.face_bc[true_bnd], mesh.face_bc[sd.cells][true_bnd])
        cut = (lnb < 0) & ~true_bnd
        assert np.all(sd.mesh.face_bc[cut] == 2)
        # cut faces belong to the outermost ghost layer only
        assert np.all(sd.layer[np.nonzero(cut)[0]] == depth)


def test_exchange_lists_cover_every_ghost_once(blast):
    mesh, _, nbr = blast
    part = S.partition(mesh, np.ones(mesh.n_tets), 4)
    subs = S.subdomains(mesh, part, 3, nbr)
    ex = S.exchange_lists(subs, part)
    seen = [np.zeros(len(sd.cells), dtype=int) for sd in subs]
    for (p, q), (send, recv) in ex.items():
        assert p != q and send.size == recv.size > 0
        gs, gr = subs[p].cells[send], subs[q].cells[recv]
        np.testing.assert_array_equal(gs, gr)
        assert np.all(np.diff(gs) > 0)
        assert np.all(send < subs[p].n_owned) and np.all(recv >= subs[q].n_owned)
        seen[q][recv] += 1
    for sd, c in zip(subs, seen):
        assert np.all(c[:sd.n_owned] == 0) and np.all(c[sd.n_owned:] == 1)


def _smooth(nbr, k0, sweeps):
    k = k0.copy()
    for _ in range(sweeps):
        m = np.where(nbr >= 0, k[np.maximum(nbr, 0)], 1 << 30).min(axis=1)
        k = np.minimum(k, m + 1)
    return k


def test_l_minus_1_ghost_layers_decide_owned_levels(blast):
    """The level rule lowers a cell to (a neighbour's level + 1), L-1 sweeps:
    an owned cell's result depends on cells within L-1 faces only, so a
    subdomain with L-1 ghost layers reproduces the whole mesh's levels on its
    own cells; with fewer layers it does not, in general."""
    mesh, _, nbr = blast
    L = 5
    rng = np.random.default_rng(11)
    k0 = np.where(rng.random(mesh.n_tets) < 0.02, 0, L - 1)
    want = _smooth(nbr, k0, L - 1)
    part = S.partition(mesh, np.ones(mesh.n_tets), 3)
    ok_depth = {}
    for depth in (1, L - 1):
        subs = S.subdomains(mesh, part, depth, nbr)
        ok = True
        for sd in subs:
            lnb = S.neighbours(sd.mesh.tets)
            got = _smooth(lnb, k0[sd.cells], L - 1)
            ok &= bool(np.array_equal(got[:sd.n_owned], want[sd.cells[:sd.n_owned]]))
        ok_depth[depth] = ok
    assert ok_depth[L - 1]
    assert not ok_depth[1]
    assert S.default_depth(L) == L - 1 and S.default_depth(2) == 2


def _gloo_rank(rank, world, port, mesh, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        part = S.partition(mesh, np.ones(mesh.n_tets), world)
        subs = S.subdomains(mesh, part, 2)
        sd = subs[rank]
        pairs = {k: v for k, v in S.exchange_lists(subs, part).items() if rank in k}
        # the payload: each local cell's global id (as the records a plan
        # packs), and a local array the unpacks write into
        local = np.full(len(sd.cells), -1, dtype=np.int64)
        local[:sd.n_owned] = sd.cells[:sd.n_owned]

        def pack(plan, what):
            return torch.from_numpy(local[plan].copy()).view(torch.uint8)

        def unpack(plan, what, t):
            local[plan] = t.view(torch.int64).numpy()

        ex = S.Exchanger(rank, pairs, pack, unpack)
        ex.exchange(0, lambda plan, what: plan.size * 8)
        m = S.global_min(float(10 + rank))
        out.put((rank, bool(np.array_equal(local, sd.cells)), m))
    finally:
        dist.destroy_process_group()


def test_exchange_between_two_gloo_ranks(blast):
    """Two ranks exchange their ghost records through gloo point-to-point
    messages: every ghost ends up with its owner's record, and the global
    minimum step is the minimum over ranks."""
    import socket
    import torch.multiprocessing as mp
    mesh, _, _ = blast
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, mesh, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [True, True]
    assert [r[2] for r in res] == [10.0, 10.0]

"""Sharded runs: the domain decomposition of Sec. 3.3 and Sec. 4.3 over
fv_mesh subdomains.

The paper splits the mesh into subdomains whose cells each belong to one
subdomain, weights every cell by the cost of its temporal level so that the
subdomains carry equal work (Sec. 3.3), keeps ghost copies of the
neighbouring subdomains' border cells, computes the border faces on both
sides, and exchanges border-cell contents before the computations that read
them (Sec. 4.3).  Here:

- partition(): cells in Morton order of their centroids, cut into
  contiguous ranges of equal weight, a cell of level k weighing
  2^(L-1-k) (its updates per cycle, the cost model C(tau) of Sec. 2.2);
- Subdomain: the owned cells, then ``depth`` layers of ghost cells around
  them (depth >= 2 for the second-order reconstruction: a border face needs
  the gradient of its ghost cell, which needs the ghost's neighbours; and
  depth >= L-1, so that every owned cell's level -- the minimum over cells
  within L-1 faces of their classification plus the distance -- is decided
  from local cells only), as a mesh of its own whose cut faces are tagged
  transmissive (they touch only outermost ghost cells, whose results are
  overwritten);
- exchange plans: for every pair of subdomains, the owned cells of one that
  are ghosts of the other, in increasing global order on both sides;
- the cycle (ShardedRun in one process, ShardedRank one subdomain per
  rank): the local steps, the global minimum dt_min, the levels, the ghost
  cells' levels from their owners, the sorted lists; then every phase of
  Alg. 2 on every subdomain followed by the ghost states from their owners.

Every arithmetic step runs in the library's kernels; this module only cuts
the mesh and moves packed records.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import inputs as I


# ---------------------------------------------------------------- host logic
def neighbours(tets: np.ndarray) -> np.ndarray:
    """nbr[t, j]: the tet across the face of t opposite its local node j,
    -1 on the boundary."""
    n = tets.shape[0]
    rows = []
    for j in range(4):
        others = [v for v in range(4) if v != j]
        rows.append(np.sort(tets[:, others], axis=1))
    F = np.concatenate(rows)                        # row r = j * n + t
    order = np.lexsort((F[:, 2], F[:, 1], F[:, 0]))
    Fs = F[order]
    same = np.all(Fs[1:] == Fs[:-1], axis=1)
    nbr = np.full(4 * n, -1, dtype=np.int64)
    a, b = order[:-1][same], order[1:][same]
    nbr[a] = b % n
    nbr[b] = a % n
    return nbr.reshape(4, n).T.copy()


def _spread_bits(v: np.ndarray) -> np.ndarray:
    """21-bit integers with two zero bits after every bit (3D Morton)."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_order(points: np.ndarray) -> np.ndarray:
    """The permutation that sorts points along a Morton curve of their
    bounding box (ties by index)."""
    lo, hi = points.min(axis=0), points.max(axis=0)
    q = np.floor((points - lo) / np.maximum(hi - lo, 1e-300) * ((1 << 21) - 1)).astype(np.int64)
    code = _spread_bits(q[:, 0]) | (_spread_bits(q[:, 1]) << np.uint64(1)) | (
        _spread_bits(q[:, 2]) << np.uint64(2))
    return np.lexsort((np.arange(points.shape[0]), code))


def level_weights(levels: np.ndarray, L: int) -> np.ndarray:
    """Cost of a cell per cycle: 2^(L-1-k) updates at level k (C(tau))."""
    return np.ldexp(1.0, (L - 1 - levels.astype(np.int64)).astype(np.int32))


def partition(mesh: I.TetMesh, weights: np.ndarray, n_parts: int) -> np.ndarray:
    """Subdomain of every cell: Morton-ordered cells cut into n_parts
    contiguous ranges of (nearly) equal total weight."""
    if n_parts < 1 or n_parts > mesh.n_tets:
        raise ValueError("n_parts must be in [1, number of cells]")
    order = morton_order(mesh.centroids())
    w = np.asarray(weights, dtype=np.float64)[order]
    cum = np.cumsum(w)
    cuts = np.searchsorted(cum, cum[-1] * np.arange(1, n_parts) / n_parts, side="left")
    part_sorted = np.zeros(mesh.n_tets, dtype=np.int32)
    for p, c in enumerate(cuts):
        part_sorted[c + 1:] = p + 1
    part = np.empty(mesh.n_tets, dtype=np.int32)
    part[order] = part_sorted
    if len(np.unique(part)) != n_parts:
        raise ValueError("a subdomain came out empty: too many parts for the weights")
    return part


@dataclasses.dataclass
class Subdomain:
    part: int
    cells: np.ndarray        # global ids: the owned cells (increasing), then ghost layers
    n_owned: int
    layer: np.ndarray        # 0 for owned cells, d for the d-th ghost layer
    mesh: I.TetMesh          # the local mesh, tets in the order of `cells`
    g2l: np.ndarray          # global id -> local id (-1: not in this subdomain)


def ghost_layers(nbr: np.ndarray, owned: np.ndarray, depth: int) -> list:
    """The cells at face distance 1..depth from the owned set, per layer,
    each in increasing global order."""
    n = nbr.shape[0]
    seen = np.zeros(n, dtype=bool)
    seen[owned] = True
    front = owned
    layers = []
    for _ in range(depth):
        cand = nbr[front].ravel()
        cand = np.unique(cand[cand >= 0])
        cand = cand[~seen[cand]]
        seen[cand] = True
        layers.append(cand)
        front = cand
        if cand.size == 0:
            break
    return layers


def subdomains(mesh: I.TetMesh, part: np.ndarray, depth: int, nbr: np.ndarray | None = None) -> list:
    """Every subdomain's cells and local mesh."""
    if nbr is None:
        nbr = neighbours(mesh.tets)
    out = []
    for p in range(int(part.max()) + 1):
        owned = np.nonzero(part == p)[0]
        layers = ghost_layers(nbr, owned, depth)
        cells = np.concatenate([owned] + layers).astype(np.int64)
        layer = np.concatenate([np.zeros(owned.size, dtype=np.int32)] +
                               [np.full(lay.size, d + 1, dtype=np.int32) for d, lay in enumerate(layers)])
        g2l = np.full(mesh.n_tets, -1, dtype=np.int64)
        g2l[cells] = np.arange(cells.size)
        tets = mesh.tets[cells]
        nodes, inv = np.unique(tets.ravel(), return_inverse=True)
        local_tets = inv.reshape(tets.shape).astype(np.int64)
        bc = mesh.face_bc[cells].copy()
        # faces cut from the rest of the mesh (only outermost ghosts have them)
        nb = nbr[cells]
        inside = np.zeros(mesh.n_tets, dtype=bool)
        inside[cells] = True
        cut = (nb >= 0) & ~inside[np.maximum(nb, 0)]
        bc[cut] = 2
        lm = I.TetMesh(xyz=mesh.xyz[nodes].copy(), tets=local_tets, face_bc=bc, shape=mesh.shape)
        out.append(Subdomain(part=p, cells=cells, n_owned=int(owned.size), layer=layer, mesh=lm, g2l=g2l))
    return out


def exchange_lists(subs: list, part: np.ndarray) -> dict:
    """(p, q) -> (local ids in p of p's owned cells that are ghosts of q,
    local ids in q of the same cells), both in increasing global order."""
    out = {}
    for q, sq in enumerate(subs):
        ghosts = sq.cells[sq.n_owned:]
        owner = part[ghosts]
        for p in np.unique(owner):
            g = np.sort(ghosts[owner == p])
            sp = subs[int(p)]
            out[(int(p), q)] = (sp.g2l[g], sq.g2l[g])
    return out


def phases_per_cycle(L: int) -> int:
    """Phases of one cycle in the finest-first order: 2^(L-1) begins and
    2^(L-1+1) - 1 step ends (Alg. 2's subiteration loop)."""
    return 3 * 2 ** (L - 1) - 1


def default_depth(L: int) -> int:
    return max(2, L - 1)


def owned_state(subs: list, states: list, n_cells: int) -> np.ndarray:
    """The global conserved field (5, n) from every subdomain's state, each
    cell from its owner."""
    U = np.empty((5, n_cells))
    for sd, u in zip(subs, states):
        U[:, sd.cells[:sd.n_owned]] = u[:, :sd.n_owned]
    return U


# --------------------------------------------------------------- the drivers
class ShardedRun:
    """Every subdomain in one process (one device): the exchanges are
    device copies through a staging buffer.  The emulation of the sharded
    algorithm on one GPU, with the same cuts, plans and exchange points as
    one subdomain per rank."""

    def __init__(self, mesh, prim, L, n_parts, precision=0, weights=None, depth=None, stream=None,
                 **cfg):
        import torch
        from . import fv
        self.fv, self.torch = fv, torch
        self.L = L
        self.n = mesh.n_tets
        if weights is None:
            weights = initial_weights(mesh, prim, L, precision, **cfg)
        self.part = partition(mesh, weights, n_parts)
        self.subs = subdomains(mesh, self.part, depth if depth is not None else default_depth(L))
        self.meshes = []
        for sd in self.subs:
            m = fv.Mesh(sd.mesh, max_levels=L, precision=precision, **cfg)
            m.set_state(np.ascontiguousarray(prim[:, sd.cells]))
            self.meshes.append(m)
        self.plans = []
        for (p, q), (send, recv) in sorted(exchange_lists(self.subs, self.part).items()):
            hs, hr = fv.Halo(self.meshes[p], send), fv.Halo(self.meshes[q], recv)
            self.plans.append((p, q, hs, hr))
        nmax = max([hs.n for _, _, hs, _ in self.plans] + [1])
        self.buf = torch.empty(nmax * 8 * fv.FV_HALO_STATE_DOUBLES, dtype=torch.uint8, device="cuda")
        self.stream = stream
        self.cycles = 0

    def exchange(self, what):
        for p, q, hs, hr in self.plans:
            hs.pack(what, self.buf, self.stream)
            hr.unpack(what, self.buf, self.stream)

    def cycle(self):
        s = self.stream
        dt_min = min(m.levels_local_dt(s) for m in self.meshes)
        for m in self.meshes:
            m.levels_classify(dt_min, s)
        self.exchange(self.fv.FV_HALO_LEVELS)
        for m in self.meshes:
            m.levels_sort(s)
        for _ in range(phases_per_cycle(self.L)):
            for m in self.meshes:
                m.advance_phases(1, s)
            self.exchange(self.fv.FV_HALO_STATE)
        self.cycles += 1
        return dt_min

    def advance(self, n_cycles):
        for _ in range(n_cycles):
            self.cycle()

    def get_state(self):
        return owned_state(self.subs, [m.get_state() for m in self.meshes], self.n)

    def status(self):
        return max(m.status() for m in self.meshes)

    def close(self):
        for _, _, hs, hr in self.plans:
            hs.close()
            hr.close()
        for m in self.meshes:
            m.close()


def initial_weights(mesh, prim, L, precision=0, **cfg):
    """The partition's cell weights from the levels of the initial state
    (one level assignment of the whole mesh)."""
    from . import fv
    g = fv.Mesh(mesh, max_levels=L, precision=precision, **cfg)
    g.set_state(prim)
    g.assign_levels()
    lev = g.levels()
    g.close()
    return level_weights(lev, L)


class Exchanger:
    """The exchanges of one rank: for every neighbouring subdomain, its plan,
    the packed records sent (p -> q) or received (q -> p) through
    torch.distributed point-to-point messages.  pack(plan, what) -> a tensor
    on the communication device; unpack(plan, what, tensor)."""

    def __init__(self, rank, pairs, pack, unpack, comm_device="cpu"):
        self.rank = rank
        self.sends = sorted(((q, send) for (p, q), (send, _) in pairs.items() if p == rank),
                            key=lambda e: e[0])
        self.recvs = sorted(((p, recv) for (p, q), (_, recv) in pairs.items() if q == rank),
                            key=lambda e: e[0])
        self.pack, self.unpack = pack, unpack
        self.dev = comm_device

    def exchange(self, what, nbytes_of):
        import torch
        import torch.distributed as dist
        reqs, inbox = [], []
        for q, plan in self.sends:
            reqs.append(dist.isend(self.pack(plan, what).to(self.dev), dst=q))
        for p, plan in self.recvs:
            t = torch.empty(nbytes_of(plan, what), dtype=torch.uint8, device=self.dev)
            reqs.append(dist.irecv(t, src=p))
            inbox.append((plan, t))
        for r in reqs:
            r.wait()
        for plan, t in inbox:
            self.unpack(plan, what, t)


def global_min(value, device="cpu"):
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return float(t.item())


class ShardedRank:
    """One subdomain per rank (torch.distributed initialised by the
    caller): its mesh on this rank's device, the global minimum step by an
    all-reduce, the ghost records by point-to-point messages -- host-staged
    over gloo, or device buffers over NCCL (comm_device="cuda")."""

    def __init__(self, mesh, prim, L, precision=0, weights=None, depth=None, comm_device="cpu",
                 stream=None, **cfg):
        import torch
        import torch.distributed as dist
        from . import fv
        self.fv, self.torch = fv, torch
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.L = L
        self.n = mesh.n_tets
        self.comm_device = comm_device
        if weights is None:
            weights = initial_weights(mesh, prim, L, precision, **cfg)
        self.part = partition(mesh, weights, self.world)
        self.subs = subdomains(mesh, self.part, depth if depth is not None else default_depth(L))
        sd = self.subs[self.rank]
        self.sd = sd
        self.mesh = fv.Mesh(sd.mesh, max_levels=L, precision=precision, **cfg)
        self.mesh.set_state(np.ascontiguousarray(prim[:, sd.cells]))
        pairs = exchange_lists(self.subs, self.part)
        self.halos = {}
        mine = {}
        for (p, q), (send, recv) in pairs.items():
            if p == self.rank:
                mine[(p, q)] = (fv.Halo(self.mesh, send), None)
            if q == self.rank:
                mine[(p, q)] = (None, fv.Halo(self.mesh, recv))
        self.stream = stream

        def sync():
            (self.stream or torch.cuda.current_stream()).synchronize()

        def pack(plan, what):
            buf = torch.empty(plan.nbytes(what), dtype=torch.uint8, device="cuda")
            plan.pack(what, buf, self.stream)
            sync()
            return buf

        def unpack(plan, what, t):
            buf = t.to("cuda")
            plan.unpack(what, buf, self.stream)
            sync()

        self.ex = Exchanger(self.rank, mine, pack, unpack, comm_device)

    def exchange(self, what):
        self.ex.exchange(what, lambda plan, w: plan.nbytes(w))

    def cycle(self):
        s = self.stream
        dt_min = global_min(self.mesh.levels_local_dt(s), self.comm_device)
        self.mesh.levels_classify(dt_min, s)
        self.exchange(self.fv.FV_HALO_LEVELS)
        self.mesh.levels_sort(s)
        for _ in range(phases_per_cycle(self.L)):
            self.mesh.advance_phases(1, s)
            self.exchange(self.fv.FV_HALO_STATE)
        return dt_min

    def owned_state(self):
        """(global ids, (5, n_owned) state) of this rank's cells."""
        return self.sd.cells[:self.sd.n_owned], self.mesh.get_state()[:, :self.sd.n_owned]

    def close(self):
        for _, plan in self.ex.sends + self.ex.recvs:
            plan.close()
        self.mesh.close()

"""The allocation-free level assignment (fv_assign_levels_noalloc).

Some callers cannot allocate device memory when they need the levels (a
host code that only lends the library memory from its own fixed pool and
accounts for every byte of it).  The entry point takes their device
arrays and keeps its scratch in a static device array, so this test checks,
through the C ABI, that two calls in a row (a larger mesh, then a smaller
one, sharing that scratch) give exactly the levels and dt_min that
fv_assign_levels computes, and that sizes beyond the static scratch are
refused before any work is queued.

This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1704_01144_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _neighbours(tets):
    """nbr[j, t]: the tet sharing the face of t opposite its local node j,
    -1 on the boundary (caller's order)."""
    n = tets.shape[0]
    rows = []
    for j in range(4):
        others = [v for v in range(4) if v != j]
        rows.append(np.sort(tets[:, others], axis=1))
    F = np.concatenate(rows)                       # row r = j * n + t
    order = np.lexsort((F[:, 2], F[:, 1], F[:, 0]))
    Fs = F[order]
    same = np.all(Fs[1:] == Fs[:-1], axis=1)
    nbr = np.full(4 * n, -1, dtype=np.int64)
    a, b = order[:-1][same], order[1:][same]
    nbr[a] = b % n
    nbr[b] = a % n
    return nbr.reshape(4, n)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_01144_gb300 import build, fv
    build.build()
    return torch, fv, fv.lib()


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_levels_match_assign_levels_two_calls(env):
    torch, fv, lib = env
    stream = torch.cuda.current_stream()
    for n_cubes, L, seed in ((11, 4, 11), (7, 3, 7)):
        mesh, prim = I.blast_case(n=n_cubes, ratio=8.0, seed=seed)
        g = fv.Mesh(mesh, max_levels=L)
        g.set_state(prim)
        dt_min_ref, counts = g.assign_levels()
        lev_ref = g.levels()
        dt = g.local_dt()
        assert (counts > 0).sum() >= 2
        dt_d = torch.tensor(dt, dtype=torch.float64, device="cuda")
        nbr_d = torch.tensor(_neighbours(mesh.tets), dtype=torch.int32, device="cuda").contiguous()
        lev_d = torch.full((dt.shape[0],), 99, dtype=torch.int8, device="cuda")
        dtmin_d = torch.zeros(1, dtype=torch.float64, device="cuda")
        rc = lib.fv_assign_levels_noalloc(_ptr(dt_d), _ptr(nbr_d), dt.shape[0], L, _ptr(lev_d),
                                          _ptr(dtmin_d), C.c_void_p(stream.cuda_stream))
        assert rc == fv.FV_OK, fv.fv_last_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(lev_d.cpu().numpy(), lev_ref)
        assert dtmin_d.item() == dt_min_ref
        g.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, fv, lib = env
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    i = torch.zeros(8, dtype=torch.int32, device="cuda")
    b = torch.zeros(8, dtype=torch.int8, device="cuda")
    for n in (fv.FV_NOALLOC_MAX_CELLS + 1, 0):
        rc = lib.fv_assign_levels_noalloc(_ptr(t), _ptr(i), n, 3, _ptr(b), _ptr(t), None)
        assert rc == fv.FV_ERR_INVALID_ARG
        assert "static scratch" in fv.fv_last_error()
    rc = lib.fv_assign_levels_noalloc(_ptr(t), _ptr(i), 8, 9, _ptr(b), _ptr(t), None)
    assert rc == fv.FV_ERR_INVALID_ARG

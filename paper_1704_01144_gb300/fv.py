"""Thin ctypes binding of ``libfv.so`` (include/fv.h), same entry-point names.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Host data are numpy arrays; device buffers are torch CUDA
tensors (PyTorch supplies device memory and streams, nothing else).  There is
no CPU fallback: if the library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

FV_OK = 0
FV_ERR_INVALID_ARG = -1
FV_ERR_BAD_MESH = -2
FV_ERR_CUDA = -3
FV_ERR_NONPHYSICAL = -4
FV_ERR_RIEMANN = -5
FV_ERR_TIMEOUT = -6
FV_ERR_NOMEM = -7

FV_BC_INTERIOR, FV_BC_WALL, FV_BC_TRANSMISSIVE = 0, 1, 2
FV_FP64, FV_FP32_FLUX = 0, 1
FV_GUESS_TWO_RAREFACTION, FV_GUESS_MLP = 0, 1

_ERR_NAMES = {
    FV_ERR_INVALID_ARG: "FV_ERR_INVALID_ARG", FV_ERR_BAD_MESH: "FV_ERR_BAD_MESH",
    FV_ERR_CUDA: "FV_ERR_CUDA", FV_ERR_NONPHYSICAL: "FV_ERR_NONPHYSICAL",
    FV_ERR_RIEMANN: "FV_ERR_RIEMANN", FV_ERR_TIMEOUT: "FV_ERR_TIMEOUT",
    FV_ERR_NOMEM: "FV_ERR_NOMEM",
}


class FvError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {_ERR_NAMES.get(code, code)}: {fv_last_error()}")


class fv_train_config(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr0", C.c_double), ("lr1", C.c_double),
                ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
                ("seed", C.c_uint64)]


class fv_config(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("newton_tol", C.c_double),
                ("max_levels", C.c_int), ("newton_max_iter", C.c_int), ("precision", C.c_int),
                ("guess", C.c_int), ("device", C.c_int)]


_lib = None

# entry points declared in include/fv.h (checked by the tests)
EXPORTS = [
    "fv_config_default", "fv_mesh_load", "fv_mesh_free", "fv_mesh_cells", "fv_mesh_faces",
    "fv_set_state", "fv_get_state", "fv_assign_levels", "fv_get_levels", "fv_residual_level",
    "fv_advance_phases", "fv_advance", "fv_get_time", "fv_set_time", "fv_boundary_ledger",
    "fv_cell_volumes", "fv_status", "fv_last_error", "fv_version", "fv_set_conserved",
    "fv_work_counters", "fv_use_graph", "fv_profile_enable", "fv_profile_read",
    "fv_get_level_lists", "fv_get_local_dt", "fv_assign_levels_noalloc",
    "fv_godunov_flux_batch", "fv_probe_fma_peak", "fv_batch_create", "fv_batch_advance",
    "fv_batch_info", "fv_batch_use_graph", "fv_batch_free", "fv_set_launch", "fv_get_launch",
    "fv_batch_set_launch", "fv_batch_get_launch", "fv_mlp_init", "fv_mlp_pack", "fv_mlp_infer",
    "fv_mlp_label", "fv_mlp_loss_grad", "fv_mlp_adam", "fv_mlp_train", "fv_mlp_train_steps",
    "fv_mlp_load", "fv_set_guess", "fv_harvest_pairs", "fv_godunov_flux_batch_mlp",
    "fv_use_persistent", "fv_barrier_selftest", "fv_level_history", "fv_batch_mlp_load",
    "fv_batch_set_guess", "fv_set_fusion", "fv_get_fusion", "fv_set_order", "fv_get_order",
    "fv_set_predictor_sum", "fv_get_predictor_sum", "fv_set_flux_staging", "fv_get_flux_staging",
    "fv_levels_local_dt", "fv_levels_classify", "fv_levels_sort", "fv_halo_create", "fv_halo_pack",
    "fv_halo_unpack", "fv_halo_size", "fv_halo_free", "fv_mlp_infer_exact_tanh", "fv_set_gather",
    "fv_get_gather",
]

FV_MLP_PARAMS = 4673
FV_MLP_PACKED_BYTES = 10240
FV_MLP_TARGET_PBAR, FV_MLP_TARGET_TR = 0, 1

FV_NOALLOC_MAX_CELLS = 1 << 22
FV_FUSE_FACES_DEFAULT = 0
FV_ORDER_FINEST_FIRST, FV_ORDER_PAPER = 0, 1
FV_SUM_FP32, FV_SUM_FP64 = 0, 1
FV_HALO_LEVELS, FV_HALO_STATE = 1, 2
FV_GATHER_THREAD, FV_GATHER_QUAD = 0, 1
FV_HALO_STATE_DOUBLES = 20

FV_PROF_LEVELS, FV_PROF_PRIM, FV_PROF_GRAD, FV_PROF_FLUX, FV_PROF_UPDATE = range(5)
FV_PROF_N = 5
PROF_NAMES = ["levels", "prim", "grad", "flux", "update"]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libfv.so (built by ``paper_1704_01144_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run paper_1704_01144_gb300.build.build() "
                          "(there is no CPU fallback)")
    L = C.CDLL(path)
    vp, dp, i64, i8p, i32p = C.c_void_p, C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_int8), \
        C.POINTER(C.c_int32)
    L.fv_config_default.argtypes = [C.POINTER(fv_config)]
    L.fv_config_default.restype = None
    L.fv_mesh_load.argtypes = [dp, i64, C.POINTER(C.c_int64), i64, i8p, C.POINTER(fv_config),
                               C.POINTER(vp)]
    L.fv_mesh_free.argtypes = [vp]
    L.fv_mesh_free.restype = None
    L.fv_mesh_cells.argtypes = [vp]
    L.fv_mesh_cells.restype = i64
    L.fv_mesh_faces.argtypes = [vp]
    L.fv_mesh_faces.restype = i64
    L.fv_set_state.argtypes = [vp, vp, C.c_int, vp]
    L.fv_get_state.argtypes = [vp, vp, C.c_int, vp]
    L.fv_assign_levels.argtypes = [vp, dp, i32p, vp]
    L.fv_get_levels.argtypes = [vp, i8p]
    L.fv_residual_level.argtypes = [vp, C.c_int, C.c_int, vp, vp]
    L.fv_advance_phases.argtypes = [vp, C.c_int, vp]
    L.fv_advance.argtypes = [vp, C.c_int, dp, vp]
    L.fv_get_time.argtypes = [vp, dp]
    L.fv_set_time.argtypes = [vp, C.c_double]
    L.fv_boundary_ledger.argtypes = [vp, dp]
    L.fv_cell_volumes.argtypes = [vp, dp]
    L.fv_status.argtypes = [vp]
    L.fv_set_conserved.argtypes = [vp, vp, C.c_int, vp]
    L.fv_work_counters.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64)]
    L.fv_use_graph.argtypes = [vp, C.c_int]
    L.fv_use_persistent.argtypes = [vp, C.c_int]
    L.fv_level_history.argtypes = [vp, C.c_int, i32p, dp, C.POINTER(C.c_int)]
    L.fv_batch_mlp_load.argtypes = [vp, vp, C.c_int, C.c_int, C.c_double]
    L.fv_batch_set_guess.argtypes = [vp, C.c_int]
    L.fv_barrier_selftest.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]
    L.fv_profile_enable.argtypes = [vp, C.c_int]
    L.fv_profile_read.argtypes = [vp, dp, C.POINTER(C.c_int64)]
    L.fv_get_local_dt.argtypes = [vp, dp]
    L.fv_probe_fma_peak.argtypes = [C.c_int, C.c_int, dp]
    L.fv_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp)]
    L.fv_batch_advance.argtypes = [vp, C.c_int, vp]
    L.fv_batch_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.fv_batch_use_graph.argtypes = [vp, C.c_int]
    L.fv_batch_free.argtypes = [vp]
    L.fv_batch_free.restype = None
    for nm in ("fv_set_launch", "fv_get_launch", "fv_batch_set_launch", "fv_batch_get_launch"):
        getattr(L, nm).argtypes = [vp, i32p]
    L.fv_set_fusion.argtypes = [vp, i64]
    L.fv_set_order.argtypes = [vp, C.c_int]
    L.fv_get_order.argtypes = [vp, C.POINTER(C.c_int)]
    L.fv_get_fusion.argtypes = [vp, C.POINTER(C.c_int64)]
    L.fv_levels_local_dt.argtypes = [vp, dp, vp]
    L.fv_levels_classify.argtypes = [vp, C.c_double, vp]
    L.fv_levels_sort.argtypes = [vp, vp]
    L.fv_halo_create.argtypes = [vp, C.POINTER(C.c_int64), i64, C.POINTER(vp)]
    L.fv_halo_pack.argtypes = [vp, C.c_int, vp, vp]
    L.fv_halo_unpack.argtypes = [vp, C.c_int, vp, vp]
    L.fv_halo_size.argtypes = [vp]
    L.fv_halo_size.restype = i64
    L.fv_halo_free.argtypes = [vp]
    L.fv_halo_free.restype = None
    L.fv_set_gather.argtypes = [vp, C.c_int]
    L.fv_get_gather.argtypes = [vp, C.POINTER(C.c_int)]
    L.fv_set_flux_staging.argtypes = [vp, C.c_int]
    L.fv_get_flux_staging.argtypes = [vp, C.POINTER(C.c_int)]
    L.fv_set_predictor_sum.argtypes = [vp, C.c_int]
    L.fv_get_predictor_sum.argtypes = [vp, C.POINTER(C.c_int)]
    L.fv_godunov_flux_batch.argtypes = [vp, vp, vp, i64, C.POINTER(fv_config), C.c_int, vp, vp, vp]
    L.fv_assign_levels_noalloc.argtypes = [vp, vp, i64, C.c_int, vp, vp, vp]
    L.fv_get_level_lists.argtypes = [vp, C.POINTER(C.c_int64), i32p, i8p, i32p]
    fp = C.POINTER(C.c_float)
    L.fv_mlp_init.argtypes = [fp, C.c_int, C.c_uint64]
    L.fv_mlp_pack.argtypes = [vp, C.c_int, C.c_int, C.c_double, vp, vp]
    L.fv_mlp_infer.argtypes = [vp, vp, i64, vp, vp]
    L.fv_mlp_infer_exact_tanh.argtypes = [vp, vp, i64, vp, vp]
    L.fv_mlp_label.argtypes = [vp, i64, C.c_double, C.c_int, vp, vp, vp, vp, vp]
    L.fv_mlp_loss_grad.argtypes = [vp, vp, vp, vp, i64, vp, dp, vp]
    L.fv_mlp_adam.argtypes = [vp, vp, vp, vp, C.c_int, C.c_double, C.c_double, C.c_double,
                              C.c_double, vp]
    L.fv_mlp_train.argtypes = [vp, vp, vp, i32p, i64, C.POINTER(fv_train_config), vp, vp]
    L.fv_mlp_train_steps.argtypes = [C.POINTER(fv_train_config), i64]
    L.fv_mlp_load.argtypes = [vp, vp, C.c_int, C.c_int, C.c_double]
    L.fv_set_guess.argtypes = [vp, C.c_int]
    L.fv_harvest_pairs.argtypes = [vp, vp, i64, C.c_uint64, vp]
    L.fv_godunov_flux_batch_mlp.argtypes = [vp, vp, vp, i64, C.POINTER(fv_config), vp, vp, vp, vp]
    L.fv_last_error.restype = C.c_char_p
    L.fv_version.restype = C.c_char_p
    _lib = L
    return L


def _check(rc, what):
    if rc != FV_OK:
        raise FvError(rc, what)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t, dtype_name="float64"):
    """Device pointer of a contiguous torch CUDA tensor."""
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("expected a torch CUDA tensor")
    if not t.is_contiguous() or str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected a contiguous {dtype_name} tensor")
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- entry points
def fv_config_default(**overrides) -> fv_config:
    cfg = fv_config()
    lib().fv_config_default(C.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def fv_last_error() -> str:
    return lib().fv_last_error().decode()


def fv_version() -> str:
    return lib().fv_version().decode()


def fv_mesh_load(xyz, tets, face_bc, cfg: fv_config):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int64)
    face_bc = np.ascontiguousarray(face_bc, dtype=np.int8)
    if xyz.ndim != 2 or xyz.shape[1] != 3 or tets.ndim != 2 or tets.shape[1] != 4 \
            or face_bc.shape != tets.shape:
        raise ValueError("xyz (n,3), tets (m,4) and face_bc (m,4) expected")
    h = C.c_void_p()
    rc = lib().fv_mesh_load(xyz.ctypes.data_as(C.POINTER(C.c_double)), xyz.shape[0],
                            tets.ctypes.data_as(C.POINTER(C.c_int64)), tets.shape[0],
                            face_bc.ctypes.data_as(C.POINTER(C.c_int8)), C.byref(cfg), C.byref(h))
    _check(rc, "fv_mesh_load")
    return h


def fv_mesh_free(h):
    lib().fv_mesh_free(h)


def fv_mesh_cells(h) -> int:
    return int(lib().fv_mesh_cells(h))


def fv_mesh_faces(h) -> int:
    return int(lib().fv_mesh_faces(h))


def fv_set_state(h, prim, stream=None):
    """prim: numpy (5, n) host array or torch CUDA float64 tensor (5, n)."""
    if isinstance(prim, np.ndarray):
        p = np.ascontiguousarray(prim, dtype=np.float64)
        _check(lib().fv_set_state(h, C.c_void_p(p.ctypes.data), 0, _stream(stream)), "fv_set_state")
    else:
        _check(lib().fv_set_state(h, _dptr(prim), 1, _stream(stream)), "fv_set_state")


def fv_set_conserved(h, cons, stream=None):
    """cons: numpy (5, n) host array (pinned torch CPU tensors work too) or a
    torch CUDA float64 tensor (5, n)."""
    if isinstance(cons, np.ndarray):
        c = np.ascontiguousarray(cons, dtype=np.float64)
        _check(lib().fv_set_conserved(h, C.c_void_p(c.ctypes.data), 0, _stream(stream)),
               "fv_set_conserved")
    elif hasattr(cons, "is_cuda") and not cons.is_cuda:
        _check(lib().fv_set_conserved(h, C.c_void_p(cons.data_ptr()), 0, _stream(stream)),
               "fv_set_conserved")
    else:
        _check(lib().fv_set_conserved(h, _dptr(cons), 1, _stream(stream)), "fv_set_conserved")


def fv_work_counters(h):
    """(cycles, C(tau)-weighted cell updates, face evaluations) since the
    last state reset."""
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().fv_work_counters(h, C.byref(a), C.byref(b), C.byref(c)), "fv_work_counters")
    return a.value, b.value, c.value


def fv_level_history(h, max_cycles=4096):
    """(counts [n, 8] int32: cells per level, dtmin [n]) of the last n cycles,
    oldest first."""
    counts = np.zeros((max_cycles, 8), dtype=np.int32)
    dtm = np.zeros(max_cycles)
    n = C.c_int()
    _check(lib().fv_level_history(h, int(max_cycles), counts.ctypes.data_as(C.POINTER(C.c_int32)),
                                  dtm.ctypes.data_as(C.POINTER(C.c_double)), C.byref(n)),
           "fv_level_history")
    return counts[:n.value], dtm[:n.value]


def fv_use_persistent(h, enable):
    _check(lib().fv_use_persistent(h, int(bool(enable))), "fv_use_persistent")


def fv_barrier_selftest(rounds, unreachable, device=0):
    """(return code, device status bits) of the grid-barrier self-test."""
    st = C.c_int(0)
    rc = lib().fv_barrier_selftest(int(device), int(rounds), int(bool(unreachable)), C.byref(st))
    return rc, st.value


def fv_use_graph(h, enable):
    _check(lib().fv_use_graph(h, int(bool(enable))), "fv_use_graph")


def fv_profile_enable(h, enable):
    _check(lib().fv_profile_enable(h, int(bool(enable))), "fv_profile_enable")


def fv_profile_read(h):
    """{class name: (total ms, launches)} of the profiled kernel classes."""
    ms = (C.c_double * FV_PROF_N)()
    n = (C.c_int64 * FV_PROF_N)()
    _check(lib().fv_profile_read(h, ms, n), "fv_profile_read")
    return {PROF_NAMES[i]: (ms[i], n[i]) for i in range(FV_PROF_N)}


def fv_get_state(h, out=None, stream=None):
    """Conserved state (5, n).  out: None (returns a numpy array), a numpy
    array, or a torch CUDA float64 tensor (filled asynchronously)."""
    n = fv_mesh_cells(h)
    if out is None:
        out = np.empty((5, n))
    if isinstance(out, np.ndarray):
        _check(lib().fv_get_state(h, C.c_void_p(out.ctypes.data), 0, _stream(stream)), "fv_get_state")
    elif hasattr(out, "is_cuda") and not out.is_cuda:
        _check(lib().fv_get_state(h, C.c_void_p(out.data_ptr()), 0, _stream(stream)), "fv_get_state")
    else:
        _check(lib().fv_get_state(h, _dptr(out), 1, _stream(stream)), "fv_get_state")
    return out


def fv_assign_levels(h, max_levels, stream=None, sync=True):
    """Returns (dt_min, counts per level) when sync, else (None, None)."""
    if not sync:
        _check(lib().fv_assign_levels(h, None, None, _stream(stream)), "fv_assign_levels")
        return None, None
    dt = C.c_double()
    counts = np.zeros(max_levels, dtype=np.int32)
    _check(lib().fv_assign_levels(h, C.byref(dt), counts.ctypes.data_as(C.POINTER(C.c_int32)),
                                  _stream(stream)), "fv_assign_levels")
    return dt.value, counts


def fv_get_local_dt(h):
    out = np.empty(fv_mesh_cells(h))
    _check(lib().fv_get_local_dt(h, out.ctypes.data_as(C.POINTER(C.c_double))), "fv_get_local_dt")
    return out


def fv_assign_levels_noalloc(dt, nbr, max_levels, levels_out, dt_min_out, stream=None):
    """Allocation-free level assignment on caller-owned torch CUDA tensors:
    dt (n,) float64, nbr (4, n) int32, levels_out (n,) int8, dt_min_out (1,)
    float64.  Asynchronous on `stream`."""
    n = int(dt.shape[0])
    _check(lib().fv_assign_levels_noalloc(_dptr(dt), _dptr(nbr, "int32"), n, int(max_levels),
                                          _dptr(levels_out, "int8"), _dptr(dt_min_out),
                                          _stream(stream)), "fv_assign_levels_noalloc")


def fv_godunov_flux_batch(WL, WR, nrm, cfg: fv_config, bc=FV_BC_INTERIOR, F=None, iters=None,
                          stream=None):
    """Device Godunov flux of independent face states: torch CUDA float64
    tensors WL, WR (5, n) primitives and nrm (3, n) unit normals.  Returns
    (F (5, n) float64, iters (n,) int32), filled asynchronously."""
    import torch
    n = int(WL.shape[1])
    if F is None:
        F = torch.empty((5, n), dtype=torch.float64, device=WL.device)
    if iters is None:
        iters = torch.empty(n, dtype=torch.int32, device=WL.device)
    _check(lib().fv_godunov_flux_batch(_dptr(WL), _dptr(WR) if WR is not None else None, _dptr(nrm),
                                       n, C.byref(cfg), int(bc), _dptr(F), _dptr(iters, "int32"),
                                       _stream(stream)), "fv_godunov_flux_batch")
    return F, iters


# ------------------------------------------------------------ learned guess
def fv_mlp_init(seed) -> np.ndarray:
    """Glorot-uniform initial parameters (host float32, FV_MLP_PARAMS)."""
    p = np.zeros(FV_MLP_PARAMS, dtype=np.float32)
    _check(lib().fv_mlp_init(p.ctypes.data_as(C.POINTER(C.c_float)), FV_MLP_PARAMS, int(seed)),
           "fv_mlp_init")
    return p


def fv_mlp_pack(params, target, gate=-1.0, packed=None, stream=None):
    """Pack a float32 CUDA tensor of parameters; returns the uint8 packed
    buffer (FV_MLP_PACKED_BYTES).  gate < 0: the network on every face."""
    import torch
    if packed is None:
        packed = torch.empty(FV_MLP_PACKED_BYTES, dtype=torch.uint8, device=params.device)
    _check(lib().fv_mlp_pack(_dptr(params, "float32"), FV_MLP_PARAMS, int(target), float(gate),
                             _dptr(packed, "uint8"), _stream(stream)), "fv_mlp_pack")
    return packed


def fv_mlp_infer(packed, x, y=None, stream=None, exact_tanh=False):
    """Network outputs of features x (n, 6) float32 CUDA -> y (n,) float32
    (exact_tanh: fv_mlp_infer_exact_tanh)."""
    import torch
    n = int(x.shape[0])
    if y is None:
        y = torch.empty(n, dtype=torch.float32, device=x.device)
    fn = lib().fv_mlp_infer_exact_tanh if exact_tanh else lib().fv_mlp_infer
    _check(fn(_dptr(packed, "uint8"), _dptr(x, "float32"), n, _dptr(y, "float32"), _stream(stream)),
           "fv_mlp_infer")
    return y


def fv_mlp_label(pairs, target, gamma=1.4, stream=None, want_q=False):
    """pairs (n, 6) float64 CUDA -> (x (n, 6) float32, y (n,) float32,
    p* (n,) float64[, q (n,) float32 shock strength])."""
    import torch
    n = int(pairs.shape[0])
    x = torch.empty((n, 6), dtype=torch.float32, device=pairs.device)
    y = torch.empty(n, dtype=torch.float32, device=pairs.device)
    ps = torch.empty(n, dtype=torch.float64, device=pairs.device)
    q = torch.empty(n, dtype=torch.float32, device=pairs.device) if want_q else None
    _check(lib().fv_mlp_label(_dptr(pairs), n, float(gamma), int(target), _dptr(x, "float32"),
                              _dptr(y, "float32"), _dptr(ps),
                              _dptr(q, "float32") if q is not None else None, _stream(stream)),
           "fv_mlp_label")
    return (x, y, ps, q) if want_q else (x, y, ps)


def fv_mlp_loss_grad(params, x, y, sel=None, want_grad=True, stream=None):
    """(loss, grad float32 CUDA tensor or None) over the samples sel (int32
    CUDA tensor) or all."""
    import torch
    n = int(sel.shape[0]) if sel is not None else int(x.shape[0])
    g = torch.empty(FV_MLP_PARAMS, dtype=torch.float32, device=x.device) if want_grad else None
    loss = C.c_double()
    _check(lib().fv_mlp_loss_grad(_dptr(params, "float32"), _dptr(x, "float32"), _dptr(y, "float32"),
                                  _dptr(sel, "int32") if sel is not None else None, n,
                                  _dptr(g, "float32") if g is not None else None, C.byref(loss),
                                  _stream(stream)), "fv_mlp_loss_grad")
    return loss.value, g


def fv_mlp_adam(params, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().fv_mlp_adam(_dptr(params, "float32"), _dptr(m, "float32"), _dptr(v, "float32"),
                             _dptr(grad, "float32"), int(step), float(lr), float(beta1), float(beta2),
                             float(eps), _stream(stream)), "fv_mlp_adam")


def fv_mlp_train(params, x, y, sel=None, epochs=4, batch=8192, lr0=2e-3, lr1=2e-5, seed=1,
                 beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """Train params (float32 CUDA tensor) in place on samples sel (host int
    array; None: all).  Returns the per-step minibatch losses (numpy)."""
    import torch
    tc = fv_train_config(int(epochs), int(batch), float(lr0), float(lr1), float(beta1), float(beta2),
                         float(eps), int(seed))
    if sel is not None:
        sel = np.ascontiguousarray(sel, dtype=np.int32)
        n = sel.shape[0]
        selp = sel.ctypes.data_as(C.POINTER(C.c_int32))
    else:
        n = int(x.shape[0])
        selp = None
    steps = lib().fv_mlp_train_steps(C.byref(tc), n)
    hist = torch.zeros(max(steps, 1), dtype=torch.float32, device=x.device)
    _check(lib().fv_mlp_train(_dptr(params, "float32"), _dptr(x, "float32"), _dptr(y, "float32"),
                              selp, n, C.byref(tc), _dptr(hist, "float32"), _stream(stream)),
           "fv_mlp_train")
    return hist[:steps].cpu().numpy()


def fv_mlp_load(h, params, target, gate=-1.0):
    _check(lib().fv_mlp_load(h, _dptr(params, "float32"), FV_MLP_PARAMS, int(target), float(gate)),
           "fv_mlp_load")


def fv_set_guess(h, guess):
    _check(lib().fv_set_guess(h, int(guess)), "fv_set_guess")


def fv_harvest_pairs(h, count, seed, out=None, stream=None):
    """(count, 6) float64 CUDA tensor of face-frame Riemann pairs of U^n."""
    import torch
    if out is None:
        out = torch.empty((int(count), 6), dtype=torch.float64, device="cuda")
    _check(lib().fv_harvest_pairs(h, _dptr(out), int(count), int(seed), _stream(stream)),
           "fv_harvest_pairs")
    return out


def fv_godunov_flux_batch_mlp(WL, WR, nrm, cfg: fv_config, packed, stream=None):
    import torch
    n = int(WL.shape[1])
    F = torch.empty((5, n), dtype=torch.float64, device=WL.device)
    iters = torch.empty(n, dtype=torch.int32, device=WL.device)
    _check(lib().fv_godunov_flux_batch_mlp(_dptr(WL), _dptr(WR), _dptr(nrm), n, C.byref(cfg),
                                           _dptr(packed, "uint8"), _dptr(F), _dptr(iters, "int32"),
                                           _stream(stream)), "fv_godunov_flux_batch_mlp")
    return F, iters


def fv_probe_fma_peak(precision, device=0) -> float:
    """Measured FMA ceiling (TFLOP/s) in FP64 (FV_FP64) or FP32."""
    t = C.c_double()
    _check(lib().fv_probe_fma_peak(int(device), int(precision), C.byref(t)), "fv_probe_fma_peak")
    return t.value


def fv_get_levels(h):
    out = np.empty(fv_mesh_cells(h), dtype=np.int8)
    _check(lib().fv_get_levels(h, out.ctypes.data_as(C.POINTER(C.c_int8))), "fv_get_levels")
    return out


def fv_get_level_lists(h, max_levels):
    """(cells sorted by (level, no finer neighbour) in caller's indices,
    cell bucket offsets [2L+1], face level per library face, face offsets
    [L+1])."""
    n, nf = fv_mesh_cells(h), fv_mesh_faces(h)
    cells = np.empty(n, dtype=np.int64)
    coff = np.empty(2 * max_levels + 1, dtype=np.int32)
    flev = np.empty(nf, dtype=np.int8)
    foff = np.empty(max_levels + 1, dtype=np.int32)
    _check(lib().fv_get_level_lists(h, cells.ctypes.data_as(C.POINTER(C.c_int64)),
                                    coff.ctypes.data_as(C.POINTER(C.c_int32)),
                                    flev.ctypes.data_as(C.POINTER(C.c_int8)),
                                    foff.ctypes.data_as(C.POINTER(C.c_int32))),
           "fv_get_level_lists")
    return cells, coff, flev, foff


def fv_residual_level(h, level, stage, R, stream=None):
    """R: torch CUDA float64 tensor (5, n), filled asynchronously."""
    _check(lib().fv_residual_level(h, int(level), int(stage), _dptr(R), _stream(stream)),
           "fv_residual_level")
    return R


def fv_advance_phases(h, n_phases, stream=None):
    _check(lib().fv_advance_phases(h, int(n_phases), _stream(stream)), "fv_advance_phases")


def fv_advance(h, n_cycles, stream=None, want_time=True):
    if want_time:
        t = C.c_double()
        _check(lib().fv_advance(h, int(n_cycles), C.byref(t), _stream(stream)), "fv_advance")
        return t.value
    _check(lib().fv_advance(h, int(n_cycles), None, _stream(stream)), "fv_advance")
    return None


def fv_get_time(h) -> float:
    t = C.c_double()
    _check(lib().fv_get_time(h, C.byref(t)), "fv_get_time")
    return t.value


def fv_set_time(h, t):
    _check(lib().fv_set_time(h, float(t)), "fv_set_time")


def fv_boundary_ledger(h):
    out = np.empty(5)
    _check(lib().fv_boundary_ledger(h, out.ctypes.data_as(C.POINTER(C.c_double))),
           "fv_boundary_ledger")
    return out


def fv_cell_volumes(h):
    out = np.empty(fv_mesh_cells(h))
    _check(lib().fv_cell_volumes(h, out.ctypes.data_as(C.POINTER(C.c_double))), "fv_cell_volumes")
    return out


def fv_status(h) -> int:
    return int(lib().fv_status(h))


def fv_batch_create(handles):
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    out = C.c_void_p()
    _check(lib().fv_batch_create(arr, len(handles), C.byref(out)), "fv_batch_create")
    return out


def fv_batch_advance(b, n_cycles, stream=None):
    _check(lib().fv_batch_advance(b, int(n_cycles), _stream(stream)), "fv_batch_advance")


def fv_batch_info(b):
    s, k = C.c_int(), C.c_int()
    _check(lib().fv_batch_info(b, C.byref(s), C.byref(k)), "fv_batch_info")
    return s.value, k.value


def fv_batch_use_graph(b, enable):
    _check(lib().fv_batch_use_graph(b, int(bool(enable))), "fv_batch_use_graph")


def fv_batch_mlp_load(b, params, target, gate=-1.0):
    _check(lib().fv_batch_mlp_load(b, _dptr(params, "float32"), FV_MLP_PARAMS, int(target), float(gate)),
           "fv_batch_mlp_load")


def fv_batch_set_guess(b, guess):
    _check(lib().fv_batch_set_guess(b, int(guess)), "fv_batch_set_guess")


def _launch4(per_sm):
    a = (C.c_int32 * 4)(*[int(x) for x in per_sm])
    return a


def fv_set_launch(h, per_sm):
    _check(lib().fv_set_launch(h, _launch4(per_sm)), "fv_set_launch")


def fv_get_launch(h):
    a = (C.c_int32 * 4)()
    _check(lib().fv_get_launch(h, a), "fv_get_launch")
    return list(a)


def fv_set_fusion(h, max_faces):
    _check(lib().fv_set_fusion(h, int(max_faces)), "fv_set_fusion")


def fv_get_fusion(h):
    a = C.c_int64()
    _check(lib().fv_get_fusion(h, C.byref(a)), "fv_get_fusion")
    return a.value


def fv_set_order(h, order):
    _check(lib().fv_set_order(h, int(order)), "fv_set_order")


def fv_get_order(h):
    a = C.c_int()
    _check(lib().fv_get_order(h, C.byref(a)), "fv_get_order")
    return a.value


def fv_set_predictor_sum(h, sum_mode):
    _check(lib().fv_set_predictor_sum(h, int(sum_mode)), "fv_set_predictor_sum")


def fv_get_predictor_sum(h):
    a = C.c_int()
    _check(lib().fv_get_predictor_sum(h, C.byref(a)), "fv_get_predictor_sum")
    return a.value


def fv_set_flux_staging(h, enable):
    _check(lib().fv_set_flux_staging(h, int(bool(enable))), "fv_set_flux_staging")


def fv_get_flux_staging(h):
    a = C.c_int()
    _check(lib().fv_get_flux_staging(h, C.byref(a)), "fv_get_flux_staging")
    return bool(a.value)


def fv_set_gather(h, gather):
    _check(lib().fv_set_gather(h, int(gather)), "fv_set_gather")


def fv_get_gather(h):
    a = C.c_int()
    _check(lib().fv_get_gather(h, C.byref(a)), "fv_get_gather")
    return a.value


def fv_levels_local_dt(h, stream=None) -> float:
    v = C.c_double()
    _check(lib().fv_levels_local_dt(h, C.byref(v), _stream(stream)), "fv_levels_local_dt")
    return v.value


def fv_levels_classify(h, dt_min, stream=None):
    _check(lib().fv_levels_classify(h, float(dt_min), _stream(stream)), "fv_levels_classify")


def fv_levels_sort(h, stream=None):
    _check(lib().fv_levels_sort(h, _stream(stream)), "fv_levels_sort")


class Halo:
    """A halo plan of one mesh: cells (caller's order) whose records are
    packed into / unpacked from a flat device buffer."""

    def __init__(self, mesh, cells):
        import numpy as _np
        c = _np.ascontiguousarray(cells, dtype=_np.int64)
        self.h = C.c_void_p()
        _check(lib().fv_halo_create(mesh.h, c.ctypes.data_as(C.POINTER(C.c_int64)), c.size,
                                    C.byref(self.h)), "fv_halo_create")
        self.n = int(c.size)
        self.mesh = mesh

    def nbytes(self, what):
        return self.n * (1 if what == FV_HALO_LEVELS else 8 * FV_HALO_STATE_DOUBLES)

    def pack(self, what, buf, stream=None):
        _check(lib().fv_halo_pack(self.h, int(what), C.c_void_p(buf.data_ptr()), _stream(stream)),
               "fv_halo_pack")

    def unpack(self, what, buf, stream=None):
        _check(lib().fv_halo_unpack(self.h, int(what), C.c_void_p(buf.data_ptr()), _stream(stream)),
               "fv_halo_unpack")

    def close(self):
        if getattr(self, "h", None):
            lib().fv_halo_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fv_batch_set_launch(b, per_sm):
    _check(lib().fv_batch_set_launch(b, _launch4(per_sm)), "fv_batch_set_launch")


def fv_batch_get_launch(b):
    a = (C.c_int32 * 4)()
    _check(lib().fv_batch_get_launch(b, a), "fv_batch_get_launch")
    return list(a)


def fv_batch_free(b):
    lib().fv_batch_free(b)


# ------------------------------------------------------------ convenience
class Mesh:
    """Owns one fv_mesh handle."""

    def __init__(self, mesh, **cfg):
        self.cfg = fv_config_default(**cfg)
        self.h = fv_mesh_load(mesh.xyz, mesh.tets, mesh.face_bc, self.cfg)
        self.n = fv_mesh_cells(self.h)
        self.nf = fv_mesh_faces(self.h)
        self.L = self.cfg.max_levels

    def close(self):
        if getattr(self, "h", None):
            fv_mesh_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, prim, stream=None):
        fv_set_state(self.h, prim, stream)

    def set_conserved(self, cons, stream=None):
        fv_set_conserved(self.h, cons, stream)

    def work_counters(self):
        return fv_work_counters(self.h)

    def use_graph(self, enable):
        fv_use_graph(self.h, enable)

    def use_persistent(self, enable):
        fv_use_persistent(self.h, enable)

    def level_history(self, max_cycles=4096):
        return fv_level_history(self.h, max_cycles)

    def set_launch(self, per_sm):
        fv_set_launch(self.h, per_sm)

    def mlp_load(self, params, target=FV_MLP_TARGET_TR, gate=-1.0):
        fv_mlp_load(self.h, params, target, gate)

    def set_guess(self, guess):
        fv_set_guess(self.h, guess)

    def harvest_pairs(self, count, seed, out=None, stream=None):
        return fv_harvest_pairs(self.h, count, seed, out, stream)

    def get_launch(self):
        return fv_get_launch(self.h)

    def set_fusion(self, max_faces):
        fv_set_fusion(self.h, max_faces)

    def get_fusion(self):
        return fv_get_fusion(self.h)

    def set_order(self, order):
        fv_set_order(self.h, order)

    def get_order(self):
        return fv_get_order(self.h)

    def levels_local_dt(self, stream=None):
        return fv_levels_local_dt(self.h, stream)

    def levels_classify(self, dt_min, stream=None):
        fv_levels_classify(self.h, dt_min, stream)

    def levels_sort(self, stream=None):
        fv_levels_sort(self.h, stream)

    def set_gather(self, gather):
        fv_set_gather(self.h, gather)

    def get_gather(self):
        return fv_get_gather(self.h)

    def set_flux_staging(self, enable):
        fv_set_flux_staging(self.h, enable)

    def get_flux_staging(self):
        return fv_get_flux_staging(self.h)

    def set_predictor_sum(self, sum_mode):
        fv_set_predictor_sum(self.h, sum_mode)

    def get_predictor_sum(self):
        return fv_get_predictor_sum(self.h)

    def profile_enable(self, enable):
        fv_profile_enable(self.h, enable)

    def profile_read(self):
        return fv_profile_read(self.h)

    def get_state(self, out=None, stream=None):
        return fv_get_state(self.h, out, stream)

    def assign_levels(self, stream=None, sync=True):
        return fv_assign_levels(self.h, self.L, stream, sync)

    def local_dt(self):
        return fv_get_local_dt(self.h)

    def levels(self):
        return fv_get_levels(self.h)

    def level_lists(self):
        return fv_get_level_lists(self.h, self.L)

    def residual_level(self, level, stage, R, stream=None):
        return fv_residual_level(self.h, level, stage, R, stream)

    def advance_phases(self, n, stream=None):
        fv_advance_phases(self.h, n, stream)

    def advance(self, n_cycles=1, stream=None, want_time=True):
        return fv_advance(self.h, n_cycles, stream, want_time)

    @property
    def t(self):
        return fv_get_time(self.h)

    def boundary_ledger(self):
        return fv_boundary_ledger(self.h)

    def volumes(self):
        return fv_cell_volumes(self.h)

    def status(self):
        return fv_status(self.h)


class Batch:
    """A batch over existing Mesh objects (kept alive by the batch)."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        self.h = fv_batch_create([m.h for m in self.meshes])

    def advance(self, n_cycles=1, stream=None):
        fv_batch_advance(self.h, n_cycles, stream)

    def info(self):
        return fv_batch_info(self.h)

    def use_graph(self, enable):
        fv_batch_use_graph(self.h, enable)

    def mlp_load(self, params, target=FV_MLP_TARGET_TR, gate=-1.0):
        fv_batch_mlp_load(self.h, params, target, gate)

    def set_guess(self, guess):
        fv_batch_set_guess(self.h, guess)

    def set_launch(self, per_sm):
        fv_batch_set_launch(self.h, per_sm)

    def get_launch(self):
        return fv_batch_get_launch(self.h)

    def close(self):
        if getattr(self, "h", None):
            fv_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

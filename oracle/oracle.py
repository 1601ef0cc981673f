"""ctypes wrapper of the FP64 CPU oracle (``fv_oracle.c``).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` use this module.  It shares
no code with the CUDA path; both only consume the seeded inputs of
``paper_1704_01144_gb300.inputs``.

What pins each function is listed in the headers of fv_oracle.c and
mlp_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        # FV_ORACLE_LIB: a library built from modified sources, for the test
        # that plants mistakes in the oracle and checks that its pins fail
        path = os.environ.get("FV_ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        i64p = C.POINTER(C.c_int64)
        i8p = C.POINTER(C.c_int8)
        i32p = C.POINTER(C.c_int32)
        vp = C.c_void_p
        L.orc_error.restype = C.c_char_p
        L.orc_create.argtypes = [dp, C.c_int64, i64p, C.c_int64, i8p, C.c_double, C.c_double,
                                 C.c_double, C.c_int, C.c_int, C.POINTER(vp)]
        L.orc_free.argtypes = [vp]
        for name in ("orc_n_cells", "orc_n_faces"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = C.c_int64
        for name in ("orc_time", "orc_dtmin"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = C.c_double
        L.orc_set_time.argtypes = [vp, C.c_double]
        L.orc_cell_geometry.argtypes = [vp, dp, dp]
        L.orc_face_data.argtypes = [vp, i64p, i64p, i8p, dp, dp]
        L.orc_set_prim.argtypes = [vp, dp]
        L.orc_set_cons.argtypes = [vp, dp]
        L.orc_get_cons.argtypes = [vp, dp]
        L.orc_get_pred.argtypes = [vp, dp]
        L.orc_assign_levels.argtypes = [vp, dp, i8p, i32p]
        L.orc_get_levels.argtypes = [vp, i8p]
        L.orc_run_phases.argtypes = [vp, C.c_int]
        L.orc_phases_per_cycle.argtypes = [vp]
        L.orc_set_order.argtypes = [vp, C.c_int]
        L.orc_advance.argtypes = [vp, C.c_int, dp]
        L.orc_residual_level.argtypes = [vp, C.c_int, C.c_int, dp]
        L.orc_global_step.argtypes = [vp, C.c_double]
        L.orc_boundary_ledger.argtypes = [vp, dp]
        L.orc_stats.argtypes = [vp, i64p, i64p, i64p, i64p]
        L.orc_scalar_gradient.argtypes = [vp, dp, dp]
        L.orc_face_offsets.argtypes = [vp, dp]
        L.orc_ghost_state.argtypes = [C.c_int, dp, dp, dp]
        L.orc_riemann.argtypes = [C.c_double] * 7 + [C.c_double, C.c_int, dp, dp,
                                                     C.POINTER(C.c_int)]
        L.orc_riemann_sample.argtypes = [C.c_double] * 7 + [C.c_double, C.c_int, C.c_double,
                                                            dp, dp, dp]
        L.orc_godunov_flux.argtypes = [C.c_double, dp, dp, dp, C.c_double, C.c_int, dp]
        L.orc_muscl_pair.argtypes = [dp] * 7
        L.orc_boundary_flux.argtypes = [C.c_double, C.c_int, dp, dp, C.c_double, C.c_int, dp]
        L.orc_num_threads.restype = C.c_int
        L.orc_phase_info.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_int64)]
        L.orc_set_threads.argtypes = [C.c_int]
        fp = C.POINTER(C.c_float)
        L.orc_mlp_n_params.restype = C.c_int
        for name in ("orc_gelu", "orc_gelu_grad", "orc_bf16_round"):
            getattr(L, name).argtypes = [C.c_double]
            getattr(L, name).restype = C.c_double
        L.orc_tr_guess.argtypes = [C.c_double] * 7
        L.orc_tr_guess.restype = C.c_double
        L.orc_mlp_features.argtypes = [C.c_double, dp, dp, dp, dp]
        L.orc_shock_scale.argtypes = [C.c_double]
        L.orc_shock_scale.restype = C.c_double
        L.orc_mlp_target.argtypes = [C.c_double, dp, C.c_int, C.c_double, dp]
        L.orc_mlp_target.restype = C.c_double
        L.orc_mlp_forward.argtypes = [dp, dp, C.c_int64, dp]
        L.orc_mlp_forward_bf16.argtypes = [fp, fp, C.c_int64, dp]
        L.orc_mlp_loss_grad.argtypes = [dp, dp, dp, C.c_int64, dp, dp]
        L.orc_adam_step.argtypes = [dp, dp, dp, dp, C.c_int64, C.c_int, C.c_double, C.c_double,
                                    C.c_double, C.c_double]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed ({rc}): {lib().orc_error().decode()}")


class OracleError(RuntimeError):
    pass


class Oracle:
    """One mesh + solver state of the CPU oracle."""

    def __init__(self, mesh, gamma=1.4, cfl=0.5, newton_tol=1e-10, max_levels=1,
                 newton_max_iter=50):
        L = lib()
        self._xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
        self._tets = np.ascontiguousarray(mesh.tets, dtype=np.int64)
        self._bc = np.ascontiguousarray(mesh.face_bc, dtype=np.int8)
        h = C.c_void_p()
        rc = L.orc_create(_dp(self._xyz), self._xyz.shape[0],
                          self._tets.ctypes.data_as(C.POINTER(C.c_int64)), self._tets.shape[0],
                          self._bc.ctypes.data_as(C.POINTER(C.c_int8)), gamma, cfl, newton_tol,
                          max_levels, newton_max_iter, C.byref(h))
        if rc != 0:
            raise OracleError(f"orc_create failed ({rc}): {L.orc_error().decode()}")
        self.h = h
        self.n = int(L.orc_n_cells(h))
        self.nf = int(L.orc_n_faces(h))
        self.max_levels = max_levels
        self.gamma = gamma

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_free(self.h)
            self.h = None

    # state -----------------------------------------------------------------
    def set_prim(self, prim):
        p = np.ascontiguousarray(prim, dtype=np.float64)
        _check(lib().orc_set_prim(self.h, _dp(p)), "orc_set_prim")

    def set_cons(self, cons):
        u = np.ascontiguousarray(cons, dtype=np.float64)
        _check(lib().orc_set_cons(self.h, _dp(u)), "orc_set_cons")

    def get_cons(self):
        out = np.empty((5, self.n))
        _check(lib().orc_get_cons(self.h, _dp(out)), "orc_get_cons")
        return out

    def get_pred(self):
        """The predicted state U* (5 x n), for consistency checks."""
        out = np.empty((5, self.n))
        _check(lib().orc_get_pred(self.h, _dp(out)), "orc_get_pred")
        return out

    @property
    def t(self):
        return float(lib().orc_time(self.h))

    @t.setter
    def t(self, value):
        lib().orc_set_time(self.h, float(value))

    @property
    def dtmin(self):
        return float(lib().orc_dtmin(self.h))

    # geometry --------------------------------------------------------------
    def cell_geometry(self):
        vol = np.empty(self.n)
        xc = np.empty((3, self.n))
        lib().orc_cell_geometry(self.h, _dp(vol), _dp(xc))
        return vol, xc

    def face_data(self):
        own = np.empty(self.nf, dtype=np.int64)
        nb = np.empty(self.nf, dtype=np.int64)
        bc = np.empty(self.nf, dtype=np.int8)
        area = np.empty(self.nf)
        nrm = np.empty((3, self.nf))
        lib().orc_face_data(self.h, own.ctypes.data_as(C.POINTER(C.c_int64)),
                            nb.ctypes.data_as(C.POINTER(C.c_int64)),
                            bc.ctypes.data_as(C.POINTER(C.c_int8)), _dp(area), _dp(nrm))
        return own, nb, bc, area, nrm

    def face_offsets(self):
        """r = x_j - x_i per face, (3, nf); the ghost centroid on boundary faces."""
        r = np.empty((3, self.nf))
        lib().orc_face_offsets(self.h, _dp(r))
        return r

    # method ----------------------------------------------------------------
    def assign_levels(self):
        dtmin = C.c_double()
        lev = np.empty(self.n, dtype=np.int8)
        counts = np.zeros(self.max_levels, dtype=np.int32)
        _check(lib().orc_assign_levels(self.h, C.byref(dtmin),
                                       lev.ctypes.data_as(C.POINTER(C.c_int8)),
                                       counts.ctypes.data_as(C.POINTER(C.c_int32))),
               "orc_assign_levels")
        return dtmin.value, lev, counts

    def levels(self):
        lev = np.empty(self.n, dtype=np.int8)
        lib().orc_get_levels(self.h, lev.ctypes.data_as(C.POINTER(C.c_int8)))
        return lev

    def phases_per_cycle(self):
        return int(lib().orc_phases_per_cycle(self.h))

    def set_order(self, order):
        """0: each level's corrector when its step ends, finest first (the
        default); 1: the order of Alg. 2's loops, coarsest first within a
        subiteration, with the intensive correction deferred to the level's
        next step (fv_oracle.c, phase_at_paper).  Between cycles only."""
        _check(lib().orc_set_order(self.h, int(order)), "orc_set_order")

    def run_phases(self, n):
        _check(lib().orc_run_phases(self.h, int(n)), "orc_run_phases")

    def advance(self, n_cycles=1):
        t = C.c_double()
        _check(lib().orc_advance(self.h, int(n_cycles), C.byref(t)), "orc_advance")
        return t.value

    def residual_level(self, level, stage):
        R = np.empty((5, self.n))
        _check(lib().orc_residual_level(self.h, int(level), int(stage), _dp(R)),
               "orc_residual_level")
        return R

    def global_step(self, dt):
        _check(lib().orc_global_step(self.h, float(dt)), "orc_global_step")

    def boundary_ledger(self):
        out = np.empty(5)
        lib().orc_boundary_ledger(self.h, _dp(out))
        return out

    def stats(self):
        up = np.zeros(self.max_levels, dtype=np.int64)
        fe = np.zeros(self.max_levels, dtype=np.int64)
        it = C.c_int64()
        calls = C.c_int64()
        lib().orc_stats(self.h, up.ctypes.data_as(C.POINTER(C.c_int64)),
                        fe.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(it), C.byref(calls))
        return {"updates": up, "face_evals": fe, "newton_iters": it.value,
                "riemann_calls": calls.value}

    def scalar_gradient(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        g = np.empty((3, self.n))
        lib().orc_scalar_gradient(self.h, _dp(q), _dp(g))
        return g


# standalone pieces ---------------------------------------------------------
def riemann(WL, WR, gamma=1.4, tol=1e-10, maxit=50):
    """1D exact Riemann problem: returns (p*, u*, newton iterations)."""
    ps, us, it = C.c_double(), C.c_double(), C.c_int()
    rc = lib().orc_riemann(gamma, *map(float, WL), *map(float, WR), tol, maxit, C.byref(ps),
                           C.byref(us), C.byref(it))
    if rc != 0:
        raise OracleError(f"orc_riemann failed ({rc})")
    return ps.value, us.value, it.value


def riemann_sample(WL, WR, xi, gamma=1.4, tol=1e-12, maxit=100):
    """Exact self-similar solution (rho, u, p) at x/t = xi."""
    r, u, p = C.c_double(), C.c_double(), C.c_double()
    rc = lib().orc_riemann_sample(gamma, *map(float, WL), *map(float, WR), tol, maxit, float(xi),
                                  C.byref(r), C.byref(u), C.byref(p))
    if rc != 0:
        raise OracleError(f"orc_riemann_sample failed ({rc})")
    return r.value, u.value, p.value


def godunov_flux(WL, WR, n, gamma=1.4, tol=1e-10, maxit=50):
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    F = np.empty(5)
    rc = lib().orc_godunov_flux(gamma, _dp(WL), _dp(WR), _dp(n), tol, maxit, _dp(F))
    if rc != 0:
        raise OracleError(f"orc_godunov_flux failed ({rc})")
    return F


def boundary_flux(bc, WL, n, gamma=1.4, tol=1e-10, maxit=50):
    """Flux per unit area through a slip wall (bc=1) or transmissive (bc=2)
    face, given the reconstructed interior state."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    F = np.empty(5)
    rc = lib().orc_boundary_flux(gamma, int(bc), _dp(WL), _dp(n), tol, maxit, _dp(F))
    if rc != 0:
        raise OracleError(f"orc_boundary_flux failed ({rc})")
    return F


def ghost_state(bc, n, W):
    """The boundary ghost state of the primitives W across a face of unit
    normal n (bc 1 slip wall, 2 transmissive)."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    Wg = np.empty(5)
    lib().orc_ghost_state(int(bc), _dp(n), _dp(W), _dp(Wg))
    return Wg


def muscl_pair(Wi, Wj, gi, gj, r):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (Wi, Wj, gi, gj, r)]
    WL = np.empty(5)
    WR = np.empty(5)
    lib().orc_muscl_pair(*[_dp(a) for a in arrs], _dp(WL), _dp(WR))
    return WL, WR


def num_threads():
    return int(lib().orc_num_threads())


def set_threads(n):
    lib().orc_set_threads(int(n))


def phase_list(theta, order=0):
    """The phases of one cycle: list of (kind, level, T); kind 'B' begins
    levels 0..level at T, 'E' ends the step of `level` at T (order 0), 'C'
    corrects `level` at the end T of its step and 'I' commits the levels
    0..level at T (order 1, Oracle.set_order)."""
    out = []
    idx = 0
    kind, level, T = C.c_int(), C.c_int(), C.c_int64()
    while lib().orc_phase_info(int(theta), int(order), idx, C.byref(kind), C.byref(level), C.byref(T)) == 0:
        out.append(("BECI"[kind.value], level.value, T.value))
        idx += 1
    return out


def prim_to_cons(prim, gamma=1.4):
    """Conserved variables from primitives (SoA 5 x n), for test set-up."""
    r, u, v, w, p = prim
    return np.stack([r, r * u, r * v, r * w, p / (gamma - 1.0) + 0.5 * r * (u * u + v * v + w * w)])


def cons_to_prim(cons, gamma=1.4):
    r = cons[0]
    u, v, w = cons[1] / r, cons[2] / r, cons[3] / r
    p = (gamma - 1.0) * (cons[4] - 0.5 * r * (u * u + v * v + w * w))
    return np.stack([r, u, v, w, p])


# ------------------------------------------------------------------ MLP guess
# (mlp_oracle.c: the learned star-pressure guess, FP64 reference)

def mlp_n_params():
    return int(lib().orc_mlp_n_params())


def gelu(x):
    return float(lib().orc_gelu(float(x)))


def gelu_grad(x):
    return float(lib().orc_gelu_grad(float(x)))


def bf16_round(x):
    return float(lib().orc_bf16_round(float(x)))


def tr_guess(pair, gamma=1.4):
    return float(lib().orc_tr_guess(gamma, *[float(v) for v in pair]))


def mlp_features(pairs, gamma=1.4):
    """pairs [n, 6] = (rL, uL, pL, rR, uR, pR) -> (x [n, 6], pbar [n], p_TR [n])."""
    pairs = np.ascontiguousarray(np.atleast_2d(pairs), dtype=np.float64)
    n = pairs.shape[0]
    x = np.zeros((n, 6))
    pb = np.zeros(n)
    ptr = np.zeros(n)
    L = lib()
    for s in range(n):
        xs = np.zeros(6)
        a, b = C.c_double(), C.c_double()
        L.orc_mlp_features(gamma, _dp(pairs[s]), _dp(xs), C.byref(a), C.byref(b))
        x[s] = xs
        pb[s] = a.value
        ptr[s] = b.value
    return x, pb, ptr


def shock_scale(q):
    return float(lib().orc_shock_scale(float(q)))


def mlp_target(pair, target, pstar, gamma=1.4):
    """(training target, shock strength q) of one pair with star pressure pstar."""
    pair = np.ascontiguousarray(pair, dtype=np.float64)
    q = C.c_double()
    y = lib().orc_mlp_target(gamma, _dp(pair), int(target), float(pstar), C.byref(q))
    return float(y), q.value


def mlp_forward(theta, x):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    y = np.zeros(x.shape[0])
    lib().orc_mlp_forward(_dp(theta), _dp(x), x.shape[0], _dp(y))
    return y


def mlp_forward_bf16(theta, x):
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float32)
    y = np.zeros(x.shape[0])
    fp = C.POINTER(C.c_float)
    lib().orc_mlp_forward_bf16(theta.ctypes.data_as(fp), x.ctypes.data_as(fp), x.shape[0], _dp(y))
    return y


def mlp_loss_grad(theta, x, t):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    g = np.zeros(theta.shape[0])
    loss = C.c_double()
    _check(lib().orc_mlp_loss_grad(_dp(theta), _dp(x), _dp(t), x.shape[0], _dp(g), C.byref(loss)),
           "orc_mlp_loss_grad")
    return loss.value, g


def adam_step(theta, m, v, grad, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """In place on float64 arrays theta, m, v."""
    grad = np.ascontiguousarray(grad, dtype=np.float64)
    _check(lib().orc_adam_step(_dp(theta), _dp(m), _dp(v), _dp(grad), theta.shape[0], int(step),
                               lr, b1, b2, eps), "orc_adam_step")

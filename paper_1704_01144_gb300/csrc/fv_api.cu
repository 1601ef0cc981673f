// fv_api.cu -- the C ABI of include/fv.h: mesh lifecycle, state transfer,
// level assignment and the phase driver of Algorithm 2.
//
// The schedule of a cycle with theta = L - 1 (the subiteration loop of Alg. 2) is a fixed
// list of 3 * 2^theta - 1 phases:  for s = 1..2^theta,  B(s) starts the levels
// 0..tau(s) at T = s - 1, then E(s, k) ends the step of level k at T = s for
// k = 0, 1, ... while s mod 2^k == 0 (finest first).  The host keeps, per
// level, the start time of the current step (tn, in dt_min units) and whether
// the predicted state U* is valid; from them each phase gets the view of
// every level at its time T: U^n (T == tn), U* (T == tn + 2^k) or the linear
// interpolation in time between them.  The kernel sequence of a cycle is
// therefore fixed; ranges come from the level-sorted lists on the device.
#include <cuda_runtime.h>

#include <cmath>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fv_internal.h"


namespace {

thread_local std::string t_err;

int fail(int code, const std::string &msg) {
  t_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  t_err = std::string(what) + ": " + cudaGetErrorString(e);
  return FV_ERR_CUDA;
}

#define CK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
  } while (0)

#define CKL(call)                                                            \
  do {                                                                       \
    int r_ = (call);                                                         \
    if (r_ != FV_OK) return fail(r_, std::string("kernel launch failed: ") + \
                                         cudaGetErrorString(cudaGetLastError())); \
  } while (0)

}  // namespace

void fv_internal_set_error(const std::string &msg) { t_err = msg; }


namespace {

template <typename T>
int dalloc(fv_mesh *m, T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(FV_ERR_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  m->allocs.push_back((void *)*p);
  return FV_OK;
}

template <typename T>
int upload(T *dst, const std::vector<T> &src) {
  CK(cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FV_OK;
}

int run_phase(fv_mesh *m, const SchedPhase &ph, cudaStream_t s) {
  PhaseDesc pd = phase_desc(m->L, m->tn, m->pred, ph);
  int rc = fvk::launch_phase(m->d, pd, m->launch, &m->prof, s);
  if (rc) return fail(rc, "phase launch failed");
  phase_apply(m->tn, m->pred, ph);
  return FV_OK;
}

// host bookkeeping of a cycle whose levels were just assigned
void begin_cycle_state(fv_mesh *m) {
  m->acc_dirty = true;
  for (int j = 0; j < FV_MAXL; ++j) {
    m->tn[j] = 0;
    m->pred[j] = false;
  }
  m->in_cycle = true;
  m->next_phase = 0;
  m->have_dt = true;
}

int start_cycle(fv_mesh *m, cudaStream_t s) {
  int rc = fvk::launch_assign_levels(m->d, m->L, m->cnt_scratch, &m->prof, s);
  if (rc) return fail(rc, "level assignment launch failed");
  m->levels_step = 0;
  begin_cycle_state(m);
  return FV_OK;
}

// the cycle's phase descriptors, uploaded once (a cycle always starts from
// t_k^n = 0 and no predicted level, so they do not change between cycles)
int persistent_tables(fv_mesh *m) {
  if (m->pds_dev) return FV_OK;
  const int nph = (int)m->phases.size();
  std::vector<PhaseDesc> pds(nph);
  int64_t tn[FV_MAXL];
  bool pred[FV_MAXL];
  for (int j = 0; j < FV_MAXL; ++j) {
    tn[j] = 0;
    pred[j] = false;
  }
  for (int q = 0; q < nph; ++q) {
    pds[q] = phase_desc(m->L, tn, pred, m->phases[q]);
    phase_apply(tn, pred, m->phases[q]);
  }
  PhaseDesc *p = nullptr;
  GridBar *b = nullptr;
  int rc = dalloc(m, &p, (size_t)nph);
  if (rc == FV_OK) rc = dalloc(m, &b, 1);
  if (rc) return rc;
  CK(cudaMemcpy(p, pds.data(), sizeof(PhaseDesc) * nph, cudaMemcpyHostToDevice));
  m->pds_dev = p;
  m->bar = b;
  return FV_OK;
}

bool persistent_on(const fv_mesh *m) {
  return m->use_persistent && !m->prof.on && m->d.guess == FV_GUESS_TWO_RAREFACTION &&
         m->order == FV_ORDER_FINEST_FIRST;
}

// a whole cycle: level assignment, every phase in one cooperative launch,
// the end-of-cycle counters
int run_cycle_persistent(fv_mesh *m, cudaStream_t s) {
  int rc = persistent_tables(m);
  if (rc) return rc;
  rc = start_cycle(m, s);
  if (rc) return rc;
  rc = fvk::launch_persistent_cycle(m->d, m->pds_dev, (int)m->phases.size(), m->bar, s);
  if (rc) return fail(rc, std::string("persistent cycle launch failed: ") + cudaGetErrorString(cudaGetLastError()));
  rc = fvk::launch_time_advance(m->d, m->theta, s);
  if (rc) return fail(rc, "time advance launch failed");
  m->in_cycle = false;
  m->next_phase = 0;
  m->acc_dirty = false;  // a whole cycle consumes every accumulated integral
  return FV_OK;
}

int run_phases(fv_mesh *m, int n, cudaStream_t s) {
  for (int q = 0; q < n; ++q) {
    if (!m->in_cycle || m->next_phase >= (int)m->phases.size())
      return fail(FV_ERR_INVALID_ARG, "no active cycle (assign levels first) or past its end");
    int rc = run_phase(m, m->phases[m->next_phase], s);
    if (rc) return rc;
    m->next_phase++;
    if (m->next_phase == (int)m->phases.size()) {
      rc = fvk::launch_time_advance(m->d, m->theta, s);
      if (rc) return fail(rc, "time advance launch failed");
      m->in_cycle = false;
      m->next_phase = 0;
      m->acc_dirty = false;  // a whole cycle consumes every accumulated integral
    }
  }
  return FV_OK;
}

}  // namespace

extern "C" {

void fv_config_default(fv_config *cfg) {
  if (!cfg) return;
  cfg->gamma = 1.4;
  cfg->cfl = 0.5;
  cfg->newton_tol = 1e-10;
  cfg->max_levels = 1;
  cfg->newton_max_iter = 50;
  cfg->precision = FV_FP64;
  cfg->guess = FV_GUESS_TWO_RAREFACTION;
  cfg->device = 0;
}

const char *fv_last_error(void) { return t_err.c_str(); }

const char *fv_version(void) { return "fv-gb300 0.1 (sm_103a)"; }

void fv_mesh_free(fv_mesh *m) {
  if (!m) return;
  cudaSetDevice(m->cfg.device);
  cudaDeviceSynchronize();
  if (m->cycle_graph) cudaGraphExecDestroy(m->cycle_graph);
  for (auto &r : m->prof.recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (void *p : m->allocs) cudaFree(p);
  cudaGetLastError();
  delete m;
}

int fv_mesh_load(const double *xyz, int64_t n_nodes, const int64_t *tets, int64_t n_tets,
                 const int8_t *face_bc, const fv_config *cfg, fv_mesh **out) {
  if (!out) return fail(FV_ERR_INVALID_ARG, "fv_mesh_load: out is NULL");
  *out = nullptr;
  if (!xyz || !tets || !face_bc || !cfg) return fail(FV_ERR_INVALID_ARG, "fv_mesh_load: NULL argument");
  if (cfg->max_levels < 1 || cfg->max_levels > FV_MAXL || !(cfg->gamma > 1.0) || !(cfg->cfl > 0.0) ||
      !(cfg->newton_tol > 0.0) || cfg->newton_max_iter < 1 ||
      (cfg->precision != FV_FP64 && cfg->precision != FV_FP32_FLUX) ||
      (cfg->guess != FV_GUESS_TWO_RAREFACTION))
    return fail(FV_ERR_INVALID_ARG, "fv_mesh_load: invalid configuration");
  if (n_tets <= 0 || n_nodes <= 0) return fail(FV_ERR_INVALID_ARG, "fv_mesh_load: bad sizes");
  CK(cudaSetDevice(cfg->device));
  fvk::init_device_info();
  HostMesh H;
  std::string err;
  int rc = fv_host_build(xyz, n_nodes, tets, n_tets, face_bc, H, &err);
  if (rc) return fail(rc, err);
  // cell and face ids are int32 on the device, and grid-stride loops step up
  // to ~2^21 past the end of a range
  if (H.F > FV_MAX_ITEMS || H.N > FV_MAX_ITEMS)
    return fail(FV_ERR_INVALID_ARG, "fv_mesh_load: mesh too large (more than 2^31 - 2^22 faces)");

  fv_mesh *m = new fv_mesh();
  m->cfg = *cfg;
  m->L = cfg->max_levels;
  m->theta = m->L - 1;
  m->phases = make_phases(m->theta);
  m->d.sort_cnt = nullptr;
  DevMesh &d = m->d;
  memset(&d, 0, sizeof d);
  const size_t N = H.N, F = H.F;
  d.N = (int)N;
  d.F = (int)F;
  d.L = m->L;
  d.gamma = cfg->gamma;
  d.cfl = cfg->cfl;
  d.tol = cfg->newton_tol;
  d.maxit = cfg->newton_max_iter;
  d.precision = cfg->precision;
  d.fuse_faces = FV_FUSE_FACES_DEFAULT;
  d.pred_sum64 = FV_PREDICTOR_SUM_DEFAULT == FV_SUM_FP64;
  d.flux_staged = FV_FLUX_STAGING_DEFAULT;
  d.gather_quad = FV_GATHER_DEFAULT == FV_GATHER_QUAD;
  const bool f32 = cfg->precision == FV_FP32_FLUX;
  const int nblk_c = (int)((N + 1023) / 1024), nblk_f = (int)((F + 1023) / 1024);
  // the cell counts (2L buckets per tile), then the face counts (L per tile)
  size_t cnt_size = (size_t)16 * (nblk_c + nblk_f) + 32;
#define AL(p, n)                       \
  do {                                 \
    int r_ = dalloc(m, &(p), (n));     \
    if (r_) {                          \
      fv_mesh_free(m);                 \
      return r_;                       \
    }                                  \
  } while (0)
  AL(d.vol, N);
  AL(d.ivol, N);
  AL(d.cf4, N);
  AL(d.cnb4, N);
  AL(d.cown, N);
  AL(d.lsw, REC_LSW * N);
  AL(d.fcell, F);
  AL(d.fgeo, REC_FG * F);
  if (f32) {
    AL(d.lsw32, REC_LSW * N);
    AL(d.ivol32, N);
    AL(d.FA32, REC_FA32 * F);
    AL(d.fgeo32, REC_FG * F);
    AL(d.G32, REC_G * N);
    float *w;
    AL(w, REC_W * N);
    m->W = w;
    d.W = w;
  } else {
    AL(d.G, REC_G * N);
    double *w;
    AL(w, REC_W * N);
    m->W = w;
    d.W = w;
  }
  AL(d.Un, 5 * N);
  if (f32) {
    AL(d.Un32, REC_U32 * N);
    AL(d.Us32, REC_U32 * N);
  } else {
    AL(d.Us, 5 * N);
  }
  AL(d.FA, REC_FA * F);
  AL(d.ACC, REC_FA * F);
  AL(d.BND, REC_FA * F);
  AL(d.lev, N);
  AL(d.lev_tmp, N);
  AL(d.flev, F);
  AL(d.ckey, N);
  AL(d.cmask, N);
  AL(d.fkey, F);
  AL(d.cl, N);
  AL(d.fl, F);
  AL(d.clf, N);
  AL(d.cln, N);
  AL(d.clb, N);
  AL(d.flc, F);
  AL(d.coff, 2 * FV_MAXL + 1);
  AL(d.foff, FV_MAXL + 1);
  AL(d.dt, N);
  AL(d.dt32, N);
  AL(d.dteps, N);
  AL(d.dthi_bits, 1);
  AL(d.dtmin_bits, 1);
  AL(d.sweep_changed, FV_MAXL);
  AL(d.tdev, 1);
  AL(d.status, 1);
  AL(d.counters, 3);
  AL(d.hist, (size_t)FV_HIST_CAP * FV_MAXL);
  AL(d.hist_dt, FV_HIST_CAP);
  AL(m->cnt_scratch, cnt_size);
  d.sort_cnt = m->cnt_scratch;
  AL(m->new2old_dev, N);
  AL(m->FAt, REC_FA * F);
#undef AL
  std::vector<int> n2o(N);
  for (size_t i = 0; i < N; ++i) n2o[i] = (int)H.new2old[i];
  int urc = FV_OK;
  urc |= upload(m->new2old_dev, n2o);
  urc |= upload(d.vol, H.vol);
  {
    std::vector<double> iv(N);
    for (size_t i = 0; i < N; ++i) iv[i] = 1.0 / H.vol[i];
    urc |= upload(d.ivol, iv);
  }
  {
    // records: cell faces / neighbours as int4, weights as [N][12], faces as
    // (owner, neighbour) pairs and [F][8] geometry (n, A, r, pad)
    std::vector<int4> cf4(N), cnb4(N);
    std::vector<double> lsw(REC_LSW * N);
    for (size_t i = 0; i < N; ++i) {
      cf4[i] = make_int4(H.cf[i], H.cf[N + i], H.cf[2 * N + i], H.cf[3 * N + i]);
      cnb4[i] = make_int4(H.cnb[i], H.cnb[N + i], H.cnb[2 * N + i], H.cnb[3 * N + i]);
      for (int q = 0; q < REC_LSW; ++q) lsw[REC_LSW * i + q] = H.lsw[q * N + i];
    }
    std::vector<int2> fcell(F);
    std::vector<double> geo(REC_FG * F);
    for (size_t f = 0; f < F; ++f) {
      fcell[f] = make_int2(H.fown[f], H.fnb[f]);
      double *g = &geo[REC_FG * f];
      for (int e = 0; e < 3; ++e) {
        g[e] = H.fn[e * F + f];
        g[4 + e] = H.fr[e * F + f];
      }
      g[3] = H.farea[f];
      g[7] = 0.0;
    }
    urc |= upload(d.cf4, cf4);
    urc |= upload(d.cnb4, cnb4);
    urc |= upload(d.cown, H.cown);
    urc |= upload(d.lsw, lsw);
    urc |= upload(d.fcell, fcell);
    urc |= upload(d.fgeo, geo);
    std::vector<int> bf;
    for (size_t f = 0; f < F; ++f)
      if (H.fnb[f] < 0) bf.push_back((int)f);
    m->n_bfaces = (int)bf.size();
    if (dalloc(m, &m->bfaces_dev, bf.size())) {
      fv_mesh_free(m);
      return FV_ERR_NOMEM;
    }
    if (!bf.empty()) urc |= upload(m->bfaces_dev, bf);
    if (f32) {
      std::vector<float> iv32(N);
      for (size_t i = 0; i < N; ++i) iv32[i] = (float)(1.0 / H.vol[i]);
      urc |= upload(d.ivol32, iv32);
      std::vector<float> w32(lsw.begin(), lsw.end());
      urc |= upload(d.lsw32, w32);
      std::vector<float> g32(geo.begin(), geo.end());
      urc |= upload(d.fgeo32, g32);
    }
  }
  if (urc) {
    fv_mesh_free(m);
    return FV_ERR_CUDA;
  }
  cudaError_t e = cudaSuccess;
  e = cudaMemset(d.ACC, 0, REC_FA * F * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(d.BND, 0, REC_FA * F * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(d.Un, 0, 5 * N * sizeof(double));
  // levels start at 0: passes that read the state before the first level
  // assignment (the harvest, the residual hooks) take every cell at U^n
  if (e == cudaSuccess) e = cudaMemset(d.lev, 0, N);
  if (e == cudaSuccess) e = cudaMemset(d.lev_tmp, 0, N);
  if (e == cudaSuccess) e = cudaMemset(d.flev, 0, F);
  if (e == cudaSuccess) e = cudaMemset(d.tdev, 0, sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(d.status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d.counters, 0, 3 * sizeof(long long));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    fv_mesh_free(m);
    return cuda_fail(e, "fv_mesh_load");
  }
  for (int j = 0; j < FV_MAXL; ++j) {
    m->tn[j] = 0;
    m->pred[j] = false;
  }
  *out = m;
  return FV_OK;
}

int64_t fv_mesh_cells(const fv_mesh *m) { return m ? m->d.N : 0; }
int64_t fv_mesh_faces(const fv_mesh *m) { return m ? m->d.F : 0; }

static int set_state_impl(fv_mesh *m, const double *src_host_or_dev, int on_device, bool conserved,
                          cudaStream_t s) {
  CK(cudaSetDevice(m->cfg.device));
  const size_t N = m->d.N;
  const double *src = src_host_or_dev;
  if (!on_device) {
    // stage through the residual scratch (5F >= 5N doubles since F >= N)
    CK(cudaMemcpyAsync(m->FAt, src_host_or_dev, 5 * N * sizeof(double), cudaMemcpyHostToDevice, s));
    src = m->FAt;
  }
  CK(cudaMemsetAsync(m->d.status, 0, sizeof(int), s));
  if (conserved)
    CKL(fvk::launch_set_cons(m->d, src, m->new2old_dev, s));
  else
    CKL(fvk::launch_set_state(m->d, src, m->new2old_dev, s));
  // the accumulators are all zero after a completed cycle; the ledger is
  // only ever written on boundary faces
  if (m->acc_dirty) CK(cudaMemsetAsync(m->d.ACC, 0, REC_FA * (size_t)m->d.F * sizeof(double), s));
  m->acc_dirty = false;
  CKL(fvk::launch_zero_faces(m->d.BND, m->bfaces_dev, m->n_bfaces, s));
  CK(cudaMemsetAsync(m->d.counters, 0, 3 * sizeof(long long), s));
  if (!on_device) CK(cudaStreamSynchronize(s));
  m->in_cycle = false;
  m->next_phase = 0;
  return FV_OK;
}

int fv_set_state(fv_mesh *m, const double *prim_soa, int on_device, void *stream) {
  if (!m || !prim_soa) return fail(FV_ERR_INVALID_ARG, "fv_set_state: NULL argument");
  return set_state_impl(m, prim_soa, on_device, false, (cudaStream_t)stream);
}

int fv_set_conserved(fv_mesh *m, const double *cons_soa, int on_device, void *stream) {
  if (!m || !cons_soa) return fail(FV_ERR_INVALID_ARG, "fv_set_conserved: NULL argument");
  return set_state_impl(m, cons_soa, on_device, true, (cudaStream_t)stream);
}

int fv_get_state(fv_mesh *m, double *cons_soa, int on_device, void *stream) {
  if (!m || !cons_soa) return fail(FV_ERR_INVALID_ARG, "fv_get_state: NULL argument");
  CK(cudaSetDevice(m->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = m->d.N;
  if (on_device) {
    CKL(fvk::launch_get_state(m->d, cons_soa, m->new2old_dev, s));
    return FV_OK;
  }
  CKL(fvk::launch_get_state(m->d, m->FAt, m->new2old_dev, s));
  CK(cudaMemcpyAsync(cons_soa, m->FAt, 5 * N * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return FV_OK;
}

int fv_assign_levels(fv_mesh *m, double *dt_min_out, int32_t *level_counts_out, void *stream) {
  if (!m) return fail(FV_ERR_INVALID_ARG, "fv_assign_levels: NULL mesh");
  if (m->in_cycle && m->next_phase > 0)
    return fail(FV_ERR_INVALID_ARG, "fv_assign_levels: a cycle is in progress");
  CK(cudaSetDevice(m->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  int rc = start_cycle(m, s);
  if (rc) return rc;
  if (dt_min_out || level_counts_out) {
    unsigned long long bits = 0;
    int coff[2 * FV_MAXL + 1];
    CK(cudaMemcpyAsync(&bits, m->d.dtmin_bits, sizeof bits, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(coff, m->d.coff, (2 * m->L + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (dt_min_out) memcpy(dt_min_out, &bits, sizeof(double));
    if (level_counts_out)
      for (int k = 0; k < m->L; ++k) level_counts_out[k] = coff[2 * k + 2] - coff[2 * k];
  }
  return FV_OK;
}

// the level assignment in three calls, for sharded runs (fv.h)
int fv_levels_local_dt(fv_mesh *m, double *dt_min_out, void *stream) {
  if (!m || !dt_min_out) return fail(FV_ERR_INVALID_ARG, "fv_levels_local_dt: NULL argument");
  if (m->in_cycle && m->next_phase > 0)
    return fail(FV_ERR_INVALID_ARG, "fv_levels_local_dt: a cycle is in progress");
  CK(cudaSetDevice(m->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  m->in_cycle = false;
  m->next_phase = 0;
  m->levels_step = 0;
  if (fvk::launch_levels_local_dt(m->d, s)) return fail(FV_ERR_CUDA, "fv_levels_local_dt: launch failed");
  unsigned long long bits = 0;
  CK(cudaMemcpyAsync(&bits, m->d.dtmin_bits, sizeof bits, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  memcpy(dt_min_out, &bits, sizeof(double));
  m->levels_step = 1;
  return FV_OK;
}

int fv_levels_classify(fv_mesh *m, double dt_min, void *stream) {
  if (!m) return fail(FV_ERR_INVALID_ARG, "fv_levels_classify: NULL mesh");
  if (m->levels_step != 1) return fail(FV_ERR_INVALID_ARG, "fv_levels_classify: call fv_levels_local_dt first");
  if (!(dt_min > 0.0) || !std::isfinite(dt_min))
    return fail(FV_ERR_INVALID_ARG, "fv_levels_classify: dt_min must be positive and finite");
  CK(cudaSetDevice(m->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  if (fvk::launch_set_dt_min(m->d, dt_min, s) || fvk::launch_levels_classify(m->d, m->L, s))
    return fail(FV_ERR_CUDA, "fv_levels_classify: launch failed");
  m->levels_step = 2;
  return FV_OK;
}

int fv_levels_sort(fv_mesh *m, void *stream) {
  if (!m) return fail(FV_ERR_INVALID_ARG, "fv_levels_sort: NULL mesh");
  if (m->levels_step != 2) return fail(FV_ERR_INVALID_ARG, "fv_levels_sort: call fv_levels_classify first");
  CK(cudaSetDevice(m->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  if (fvk::launch_levels_sort(m->d, s)) return fail(FV_ERR_CUDA, "fv_levels_sort: launch failed");
  m->levels_step = 0;
  begin_cycle_state(m);
  return FV_OK;
}

int fv_get_local_dt(fv_mesh *m, double *dt_out) {
  if (!m || !dt_out) return fail(FV_ERR_INVALID_ARG, "fv_get_local_dt: NULL argument");
  if (!m->have_dt) return fail(FV_ERR_INVALID_ARG, "fv_get_local_dt: no level assignment yet");
  CK(cudaSetDevice(m->cfg.device));
  CK(cudaDeviceSynchronize());
  const size_t N = m->d.N;
  std::vector<double> dt(N);
  std::vector<float> est(N), eps(N);
  std::vector<int> n2o(N);
  CK(cudaMemcpy(dt.data(), m->d.dt, N * sizeof(double), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(est.data(), m->d.dt32, N * sizeof(float), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(eps.data(), m->d.dteps, N * sizeof(float), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(n2o.data(), m->new2old_dev, N * sizeof(int), cudaMemcpyDeviceToHost));
  // the exact value where the assignment needed it, else the FP32 estimate
  for (size_t i = 0; i < N; ++i) dt_out[n2o[i]] = eps[i] > 0.0f ? (double)est[i] : dt[i];
  return FV_OK;
}

int fv_get_levels(fv_mesh *m, int8_t *levels_out) {
  if (!m || !levels_out) return fail(FV_ERR_INVALID_ARG, "fv_get_levels: NULL argument");
  CK(cudaSetDevice(m->cfg.device));
  int8_t *tmp = (int8_t *)m->FAt;
  CKL(fvk::launch_get_levels(m->d, tmp, m->new2old_dev, 0));
  CK(cudaMemcpy(levels_out, tmp, m->d.N, cudaMemcpyDeviceToHost));
  return FV_OK;
}

int fv_get_level_lists(fv_mesh *m, int64_t *cells_out, int32_t *cell_off_out,
                       int8_t *face_level_out, int32_t *face_off_out) {
  if (!m) return fail(FV_ERR_INVALID_ARG, "fv_get_level_lists: NULL mesh");
  CK(cudaSetDevice(m->cfg.device));
  CK(cudaDeviceSynchronize());
  const size_t N = m->d.N, F = m->d.F;
  if (cells_out) {
    std::vector<int> cl(N), n2o(N);
    CK(cudaMemcpy(cl.data(), m->d.cl, N * sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(n2o.data(), m->new2old_dev, N * sizeof(int), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < N; ++i) cells_out[i] = (cl[i] >= 0 && (size_t)cl[i] < N) ? n2o[cl[i]] : -1;
  }
  if (cell_off_out) CK(cudaMemcpy(cell_off_out, m->d.coff, (2 * m->L + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  if (face_level_out) CK(cudaMemcpy(face_level_out, m->d.flev, F, cudaMemcpyDeviceToHost));
  if (face_off_out) CK(cudaMemcpy(face_off_out, m->d.foff, (m->L + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  return FV_OK;
}

int fv_residual_level(fv_mesh *m, int level, int stage, double *R_soa_dev, void *stream) {
  if (!m || !R_soa_dev) return fail(FV_ERR_INVALID_ARG, "fv_residual_level: NULL argument");
  if (!m->in_cycle) return fail(FV_ERR_INVALID_ARG, "fv_residual_level: no active cycle");
  if (m->order != FV_ORDER_FINEST_FIRST)
    return fail(FV_ERR_INVALID_ARG, "fv_residual_level: defined for FV_ORDER_FINEST_FIRST");
  if (level < 0 || level >= m->L || (stage != 1 && stage != 2))
    return fail(FV_ERR_INVALID_ARG, "fv_residual_level: bad level or stage");
  if (stage == 2 && !m->pred[level])
    return fail(FV_ERR_INVALID_ARG, "fv_residual_level: the level's predictor has not run");
  CK(cudaSetDevice(m->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  int64_t T = m->tn[level] + (stage == 2 ? ((int64_t)1 << level) : 0);
  // every level present in the mesh must have a defined state at T
  int coff[2 * FV_MAXL + 1];
  CK(cudaMemcpyAsync(coff, m->d.coff, (2 * m->L + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int j = 0; j < m->L; ++j) {
    if (coff[2 * j + 2] == coff[2 * j]) continue;
    int64_t dd = T - m->tn[j];
    if (dd < 0 || dd > ((int64_t)1 << j) || (dd > 0 && !m->pred[j]))
      return fail(FV_ERR_INVALID_ARG, "fv_residual_level: states not available at that time");
  }
  PhaseLevels pl = levels_at(m->L, m->tn, m->pred, T);
  int rc = fvk::launch_residual(m->d, m->cfg.precision, pl, level, m->W, m->FAt, R_soa_dev,
                                m->new2old_dev, s);
  if (rc) return fail(rc, "residual launch failed");
  return FV_OK;
}

int fv_advance_phases(fv_mesh *m, int n_phases, void *stream) {
  if (!m || n_phases < 0) return fail(FV_ERR_INVALID_ARG, "fv_advance_phases: bad argument");
  CK(cudaSetDevice(m->cfg.device));
  return run_phases(m, n_phases, (cudaStream_t)stream);
}

static int capture_cycle(fv_mesh *m, cudaStream_t s) {
  cudaGraph_t g = nullptr;
  int rc = persistent_on(m) ? persistent_tables(m) : FV_OK;
  if (rc) return rc;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  if (persistent_on(m)) {
    rc = run_cycle_persistent(m, s);
  } else {
    rc = start_cycle(m, s);
    if (rc == FV_OK) rc = run_phases(m, (int)m->phases.size(), s);
  }
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiateWithFlags(&m->cycle_graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    m->cycle_graph = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  return FV_OK;
}

int fv_advance(fv_mesh *m, int n_cycles, double *t_out, void *stream) {
  if (!m || n_cycles < 0) return fail(FV_ERR_INVALID_ARG, "fv_advance: bad argument");
  CK(cudaSetDevice(m->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  const bool graphable = m->use_graph && !m->prof.on && s != nullptr && s != cudaStreamLegacy &&
                         s != cudaStreamPerThread;
  for (int c = 0; c < n_cycles; ++c) {
    int rc;
    if (!m->in_cycle && graphable) {
      if (!m->cycle_graph) {
        rc = capture_cycle(m, s);
        if (rc) return rc;
      }
      CK(cudaGraphLaunch(m->cycle_graph, s));
      continue;
    }
    if (!m->in_cycle && persistent_on(m)) {
      rc = run_cycle_persistent(m, s);
      if (rc) return rc;
      continue;
    }
    if (!m->in_cycle) {
      rc = start_cycle(m, s);
      if (rc) return rc;
    }
    rc = run_phases(m, (int)m->phases.size() - m->next_phase, s);
    if (rc) return rc;
  }
  if (t_out) {
    CK(cudaMemcpyAsync(t_out, m->d.tdev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return FV_OK;
}

int fv_set_launch(fv_mesh *m, const int32_t per_sm[4]) {
  if (!m || !per_sm) return fail(FV_ERR_INVALID_ARG, "fv_set_launch: NULL argument");
  for (int k = 0; k < 4; ++k)
    if (per_sm[k] < 1 || per_sm[k] > 64) return fail(FV_ERR_INVALID_ARG, "fv_set_launch: 1..64 blocks per SM");
  for (int k = 0; k < 4; ++k) m->launch.per_sm[k] = per_sm[k];
  if (m->cycle_graph) {
    cudaGraphExecDestroy(m->cycle_graph);
    m->cycle_graph = nullptr;
  }
  return FV_OK;
}

int fv_get_launch(fv_mesh *m, int32_t per_sm[4]) {
  if (!m || !per_sm) return fail(FV_ERR_INVALID_ARG, "fv_get_launch: NULL argument");
  for (int k = 0; k < 4; ++k) per_sm[k] = m->launch.per_sm[k];
  return FV_OK;
}

int fv_set_order(fv_mesh *m, int order) {
  if (!m || (order != FV_ORDER_FINEST_FIRST && order != FV_ORDER_PAPER))
    return fail(FV_ERR_INVALID_ARG, "fv_set_order: bad argument");
  if (m->in_batch || (m->in_cycle && m->next_phase > 0))
    return fail(FV_ERR_INVALID_ARG, "fv_set_order: mesh is inside a cycle or a batch");
  if (order == m->order) return FV_OK;
  CK(cudaSetDevice(m->cfg.device));
  if (order == FV_ORDER_PAPER && m->d.precision == FV_FP32_FLUX && !m->d.UsD) {
    int rc = dalloc(m, &m->d.UsD, 5 * (size_t)m->d.N);
    if (rc) return rc;
  }
  m->order = order;
  m->phases = make_phases(m->theta, order);
  m->in_cycle = false;
  m->next_phase = 0;
  if (m->cycle_graph) {
    cudaGraphExecDestroy(m->cycle_graph);
    m->cycle_graph = nullptr;
  }
  return FV_OK;
}

int fv_get_order(fv_mesh *m, int *order_out) {
  if (!m || !order_out) return fail(FV_ERR_INVALID_ARG, "fv_get_order: NULL argument");
  *order_out = m->order;
  return FV_OK;
}

int fv_set_fusion(fv_mesh *m, int64_t max_faces) {
  if (!m || max_faces < 0) return fail(FV_ERR_INVALID_ARG, "fv_set_fusion: bad argument");
  if (m->in_batch || (m->in_cycle && m->next_phase > 0))
    return fail(FV_ERR_INVALID_ARG, "fv_set_fusion: mesh is inside a cycle or a batch");
  m->d.fuse_faces = (int)(max_faces < FV_MAX_ITEMS ? max_faces : FV_MAX_ITEMS);
  if (m->cycle_graph) {
    cudaGraphExecDestroy(m->cycle_graph);
    m->cycle_graph = nullptr;
  }
  return FV_OK;
}

int fv_get_fusion(fv_mesh *m, int64_t *max_faces_out) {
  if (!m || !max_faces_out) return fail(FV_ERR_INVALID_ARG, "fv_get_fusion: NULL argument");
  *max_faces_out = m->d.fuse_faces;
  return FV_OK;
}

int fv_set_predictor_sum(fv_mesh *m, int sum) {
  if (!m || (sum != FV_SUM_FP32 && sum != FV_SUM_FP64))
    return fail(FV_ERR_INVALID_ARG, "fv_set_predictor_sum: bad argument");
  if (m->in_batch || (m->in_cycle && m->next_phase > 0))
    return fail(FV_ERR_INVALID_ARG, "fv_set_predictor_sum: mesh is inside a cycle or a batch");
  m->d.pred_sum64 = sum == FV_SUM_FP64;
  if (m->cycle_graph) {
    cudaGraphExecDestroy(m->cycle_graph);
    m->cycle_graph = nullptr;
  }
  return FV_OK;
}

int fv_get_predictor_sum(fv_mesh *m, int *sum_out) {
  if (!m || !sum_out) return fail(FV_ERR_INVALID_ARG, "fv_get_predictor_sum: NULL argument");
  *sum_out = m->d.pred_sum64 ? FV_SUM_FP64 : FV_SUM_FP32;
  return FV_OK;
}

int fv_set_flux_staging(fv_mesh *m, int enable) {
  if (!m) return fail(FV_ERR_INVALID_ARG, "fv_set_flux_staging: NULL mesh");
  if (m->in_batch || (m->in_cycle && m->next_phase > 0))
    return fail(FV_ERR_INVALID_ARG, "fv_set_flux_staging: mesh is inside a cycle or a batch");
  m->d.flux_staged = enable != 0;
  if (m->cycle_graph) {
    cudaGraphExecDestroy(m->cycle_graph);
    m->cycle_graph = nullptr;
  }
  return FV_OK;
}

int fv_get_flux_staging(fv_mesh *m, int *enabled_out) {
  if (!m || !enabled_out) return fail(FV_ERR_INVALID_ARG, "fv_get_flux_staging: NULL argument");
  *enabled_out = m->d.flux_staged;
  return FV_OK;
}

int fv_set_gather(fv_mesh *m, int gather) {
  if (!m || (gather != FV_GATHER_THREAD && gather != FV_GATHER_QUAD))
    return fail(FV_ERR_INVALID_ARG, "fv_set_gather: bad argument");
  if (m->in_batch || (m->in_cycle && m->next_phase > 0))
    return fail(FV_ERR_INVALID_ARG, "fv_set_gather: mesh is inside a cycle or a batch");
  m->d.gather_quad = gather == FV_GATHER_QUAD;
  if (m->cycle_graph) {
    cudaGraphExecDestroy(m->cycle_graph);
    m->cycle_graph = nullptr;
  }
  return FV_OK;
}

int fv_get_gather(fv_mesh *m, int *gather_out) {
  if (!m || !gather_out) return fail(FV_ERR_INVALID_ARG, "fv_get_gather: NULL argument");
  *gather_out = m->d.gather_quad ? FV_GATHER_QUAD : FV_GATHER_THREAD;
  return FV_OK;
}

int fv_use_persistent(fv_mesh *m, int enable) {
  if (!m) return fail(FV_ERR_INVALID_ARG, "fv_use_persistent: NULL mesh");
  if (m->in_cycle && m->next_phase > 0) return fail(FV_ERR_INVALID_ARG, "fv_use_persistent: inside a cycle");
  m->use_persistent = enable != 0;
  if (m->cycle_graph) {
    cudaGraphExecDestroy(m->cycle_graph);
    m->cycle_graph = nullptr;
  }
  return FV_OK;
}

int fv_barrier_selftest(int device, int rounds, int unreachable, int *status_out) {
  if (!status_out || rounds < 1 || rounds > 1000000) return fail(FV_ERR_INVALID_ARG, "fv_barrier_selftest: bad argument");
  CK(cudaSetDevice(device));
  fvk::init_device_info();
  GridBar *bar = nullptr;
  int *st = nullptr;
  CK(cudaMalloc(&bar, sizeof(GridBar)));
  cudaError_t e = cudaMalloc(&st, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(st, 0, sizeof(int));
  if (e == cudaSuccess && fvk::launch_barrier_probe(bar, st, rounds, unreachable ? 1u : 0u, 0) != FV_OK)
    e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status_out, st, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(bar);
  cudaFree(st);
  if (e != cudaSuccess) return cuda_fail(e, "fv_barrier_selftest");
  return (*status_out & FV_STATUS_TIMEOUT) ? fail(FV_ERR_TIMEOUT, "grid barrier timed out") : FV_OK;
}

int fv_use_graph(fv_mesh *m, int enable) {
  if (!m) return fail(FV_ERR_INVALID_ARG, "fv_use_graph: NULL mesh");
  m->use_graph = enable != 0;
  return FV_OK;
}

int fv_level_history(fv_mesh *m, int max_cycles, int32_t *counts_out, double *dtmin_out, int *n_out) {
  if (!m || max_cycles < 0 || !n_out || (max_cycles > 0 && (!counts_out || !dtmin_out)))
    return fail(FV_ERR_INVALID_ARG, "fv_level_history: bad argument");
  CK(cudaSetDevice(m->cfg.device));
  CK(cudaDeviceSynchronize());
  long long c[3];
  CK(cudaMemcpy(c, m->d.counters, sizeof c, cudaMemcpyDeviceToHost));
  const long long have = c[0] < FV_HIST_CAP ? c[0] : FV_HIST_CAP;
  const int n = (int)(have < max_cycles ? have : max_cycles);
  std::vector<int> h((size_t)FV_HIST_CAP * FV_MAXL);
  std::vector<double> hd(FV_HIST_CAP);
  CK(cudaMemcpy(h.data(), m->d.hist, h.size() * sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(hd.data(), m->d.hist_dt, hd.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int q = 0; q < n; ++q) {
    const long long cyc = c[0] - n + q;  // oldest first
    const long long slot = cyc % FV_HIST_CAP;
    for (int k = 0; k < FV_MAXL; ++k) counts_out[(size_t)q * FV_MAXL + k] = h[slot * FV_MAXL + k];
    dtmin_out[q] = hd[slot];
  }
  *n_out = n;
  return FV_OK;
}

int fv_work_counters(fv_mesh *m, int64_t *cycles, int64_t *cell_updates, int64_t *face_evals) {
  if (!m) return fail(FV_ERR_INVALID_ARG, "fv_work_counters: NULL mesh");
  CK(cudaSetDevice(m->cfg.device));
  long long c[3];
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(c, m->d.counters, sizeof c, cudaMemcpyDeviceToHost));
  if (cycles) *cycles = c[0];
  if (cell_updates) *cell_updates = c[1];
  if (face_evals) *face_evals = c[2];
  return FV_OK;
}

int fv_profile_enable(fv_mesh *m, int enable) {
  if (!m) return fail(FV_ERR_INVALID_ARG, "fv_profile_enable: NULL mesh");
  CK(cudaSetDevice(m->cfg.device));
  CK(cudaDeviceSynchronize());
  for (auto &r : m->prof.recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  m->prof.recs.clear();
  for (int c = 0; c < FV_PROF_N; ++c) {
    m->prof.ms[c] = 0.0;
    m->prof.launches[c] = 0;
  }
  m->prof.on = enable != 0;
  return FV_OK;
}

int fv_profile_read(fv_mesh *m, double ms_out[FV_PROF_N], int64_t launches_out[FV_PROF_N]) {
  if (!m) return fail(FV_ERR_INVALID_ARG, "fv_profile_read: NULL mesh");
  CK(cudaSetDevice(m->cfg.device));
  CK(cudaDeviceSynchronize());
  for (auto &r : m->prof.recs) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    m->prof.ms[r.cls] += ms;
    m->prof.launches[r.cls] += 1;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  m->prof.recs.clear();
  for (int c = 0; c < FV_PROF_N; ++c) {
    if (ms_out) ms_out[c] = m->prof.ms[c];
    if (launches_out) launches_out[c] = m->prof.launches[c];
  }
  return FV_OK;
}

int fv_get_time(fv_mesh *m, double *t_out) {
  if (!m || !t_out) return fail(FV_ERR_INVALID_ARG, "fv_get_time: NULL argument");
  CK(cudaSetDevice(m->cfg.device));
  CK(cudaMemcpy(t_out, m->d.tdev, sizeof(double), cudaMemcpyDeviceToHost));
  return FV_OK;
}

int fv_set_time(fv_mesh *m, double t) {
  if (!m) return fail(FV_ERR_INVALID_ARG, "fv_set_time: NULL mesh");
  if (m->in_cycle && m->next_phase > 0) return fail(FV_ERR_INVALID_ARG, "fv_set_time: inside a cycle");
  CK(cudaSetDevice(m->cfg.device));
  CK(cudaMemcpy(m->d.tdev, &t, sizeof(double), cudaMemcpyHostToDevice));
  return FV_OK;
}

int fv_boundary_ledger(fv_mesh *m, double *out5) {
  if (!m || !out5) return fail(FV_ERR_INVALID_ARG, "fv_boundary_ledger: NULL argument");
  CK(cudaSetDevice(m->cfg.device));
  const size_t F = m->d.F;
  std::vector<double> bnd(REC_FA * F);
  std::vector<int2> fc(F);
  CK(cudaMemcpy(bnd.data(), m->d.BND, REC_FA * F * sizeof(double), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(fc.data(), m->d.fcell, F * sizeof(int2), cudaMemcpyDeviceToHost));
  for (int c = 0; c < 5; ++c) {
    double sum = 0.0;
    for (size_t f = 0; f < F; ++f)
      if (fc[f].y < 0) sum += bnd[REC_FA * f + c];
    out5[c] = sum;
  }
  return FV_OK;
}

int fv_cell_volumes(fv_mesh *m, double *vol_out) {
  if (!m || !vol_out) return fail(FV_ERR_INVALID_ARG, "fv_cell_volumes: NULL argument");
  CK(cudaSetDevice(m->cfg.device));
  const size_t N = m->d.N;
  std::vector<double> v(N);
  std::vector<int> n2o(N);
  CK(cudaMemcpy(v.data(), m->d.vol, N * sizeof(double), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(n2o.data(), m->new2old_dev, N * sizeof(int), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < N; ++i) vol_out[n2o[i]] = v[i];
  return FV_OK;
}

int fv_godunov_flux_batch(const double *WL_dev, const double *WR_dev, const double *n_dev,
                          int64_t count, const fv_config *cfg, int bc, double *F_dev,
                          int32_t *iters_dev, void *stream) {
  if (!WL_dev || !n_dev || !cfg || !F_dev || !iters_dev || (bc == FV_BC_INTERIOR && !WR_dev))
    return fail(FV_ERR_INVALID_ARG, "fv_godunov_flux_batch: NULL argument");
  if (count < 0 || count > 0x7fffffff || bc < 0 || bc > 2 || !(cfg->gamma > 1.0) ||
      !(cfg->newton_tol > 0.0) || cfg->newton_max_iter < 1 ||
      (cfg->precision != FV_FP64 && cfg->precision != FV_FP32_FLUX))
    return fail(FV_ERR_INVALID_ARG, "fv_godunov_flux_batch: bad argument");
  if (count == 0) return FV_OK;
  CK(cudaSetDevice(cfg->device));
  fvk::init_device_info();
  int rc = fvk::launch_flux_batch(WL_dev, WR_dev ? WR_dev : WL_dev, n_dev, (int)count, cfg->gamma,
                                  cfg->newton_tol, cfg->newton_max_iter, cfg->precision, bc, F_dev,
                                  iters_dev, nullptr, (cudaStream_t)stream);
  if (rc) return fail(rc, "fv_godunov_flux_batch: launch failed");
  return FV_OK;
}

int fv_status(fv_mesh *m) {
  if (!m) return fail(FV_ERR_INVALID_ARG, "fv_status: NULL mesh");
  int st = 0;
  cudaError_t e = cudaSetDevice(m->cfg.device);
  if (e == cudaSuccess && fvk::launch_check_state(m->d, 0) != FV_OK) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&st, m->d.status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "fv_status");
  if (st & FV_STATUS_NONPHYS) return fail(FV_ERR_NONPHYSICAL, "non-physical state (rho or p <= 0)");
  if (st & FV_STATUS_RIEMANN) return fail(FV_ERR_RIEMANN, "Riemann solver failed (vacuum or no convergence)");
  if (st & FV_STATUS_TIMEOUT) return fail(FV_ERR_TIMEOUT, "a grid barrier of the persistent cycle timed out");
  return FV_OK;
}

}  // extern "C"

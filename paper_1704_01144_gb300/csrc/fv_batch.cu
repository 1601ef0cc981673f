// fv_batch.cu -- many meshes of uneven sizes and level counts advanced
// together: one launch per kernel kind and phase covers every instance.
//
// Each instance keeps its own temporal schedule (Alg. 2 with its own
// theta_i = L_i - 1, its own dt_min and levels).  A batch cycle is
// 2^thetamax batch subiterations; at batch subiteration s instance i is at
// its own subiteration s_i = ((s - 1) mod 2^theta_i) + 1, so it completes
// 2^(thetamax - theta_i) of its own cycles per batch cycle.  Per batch
// subiteration: level assignment of the instances whose cycle starts
// (batched kernels, block -> (instance, tile)), then the begin phase of every
// instance, then end phases k = 0, 1, ... (instance i takes part when
// s_i mod 2^k = 0 and k <= theta_i), then the cycle end of the instances whose
// cycle finished.  The per-instance phase descriptors are fixed by the
// schedule, computed once here, and the whole batch cycle is replayed as one
// CUDA graph.  Results equal each mesh advanced on its own, bit for bit.
#include <cuda_runtime.h>

#include <cmath>

#include <string>
#include <vector>

#include "fv_internal.h"

struct fv_batch {
  std::vector<fv_mesh *> meshes;
  int n = 0, Lmax = 1, thetamax = 0, device = 0;
  DevMesh *d_ms = nullptr;
  PhaseDesc *d_pds = nullptr;
  int *d_active = nullptr;
  int *d_tpref_c = nullptr, *d_tpref_f = nullptr;
  int64_t tiles_c = 0, tiles_f = 0, cells = 0, faces = 0;
  struct Step {
    int type;  // 0 level assignment, 1 phase, 2 cycle end
    int idx;   // row of d_active (type 0) or d_pds (types 1, 2)
  };
  std::vector<Step> steps;
  bool use_graph = true;
  cudaGraphExec_t graph = nullptr;
  std::vector<void *> allocs;
  LaunchCfg launch = default_launch();
  uint32_t *mlp = nullptr;  // the batch's learned guess (packed), shared by every instance
  bool use_mlp = false;
};

namespace {

int bfail(int code, const std::string &msg) {
  fv_internal_set_error(msg);
  return code;
}

#define BCK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return bfail(FV_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int balloc(fv_batch *b, T **p, size_t count) {
  cudaError_t e = cudaMalloc((void **)p, (count ? count : 1) * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return bfail(FV_ERR_NOMEM, std::string("fv_batch_create: cudaMalloc: ") + cudaGetErrorString(e));
  }
  b->allocs.push_back((void *)*p);
  return FV_OK;
}

int run_steps(fv_batch *b, cudaStream_t s) {
  for (const auto &st : b->steps) {
    int rc;
    if (st.type == 0) {
      rc = fvk::launch_assign_multi(b->d_ms, b->d_active + (size_t)st.idx * b->n, b->n, b->Lmax,
                                    b->cells, b->faces, b->tiles_c, b->tiles_f, nullptr, b->d_tpref_c,
                                    b->d_tpref_f, s);
    } else if (st.type == 1) {
      rc = fvk::launch_phase_multi(b->d_ms, b->d_pds + (size_t)st.idx * b->n, b->n,
                                   b->meshes[0]->d, b->cells, b->faces, b->launch,
                                   b->use_mlp ? b->mlp : nullptr, s);
    } else {
      rc = fvk::launch_time_advance_multi(b->d_ms, b->d_pds + (size_t)st.idx * b->n, b->n, s);
    }
    if (rc) return bfail(rc, "fv_batch_advance: launch failed");
  }
  return FV_OK;
}

}  // namespace

extern "C" {

void fv_batch_free(fv_batch *b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void *p : b->allocs) cudaFree(p);
  cudaGetLastError();
  delete b;
}

int fv_batch_create(fv_mesh *const *meshes, int n, fv_batch **out) {
  if (!out) return bfail(FV_ERR_INVALID_ARG, "fv_batch_create: out is NULL");
  *out = nullptr;
  if (!meshes || n < 1 || n > FV_MAXB)
    return bfail(FV_ERR_INVALID_ARG, "fv_batch_create: need 1..64 meshes");
  const fv_mesh *m0 = meshes[0];
  for (int i = 0; i < n; ++i) {
    const fv_mesh *m = meshes[i];
    if (!m) return bfail(FV_ERR_INVALID_ARG, "fv_batch_create: NULL mesh");
    for (int j = 0; j < i; ++j)
      if (meshes[j] == m) return bfail(FV_ERR_INVALID_ARG, "fv_batch_create: a mesh appears twice");
    if (m->cfg.device != m0->cfg.device || m->cfg.precision != m0->cfg.precision ||
        m->cfg.gamma != m0->cfg.gamma || m->cfg.newton_tol != m0->cfg.newton_tol ||
        m->cfg.newton_max_iter != m0->cfg.newton_max_iter)
      return bfail(FV_ERR_INVALID_ARG,
                   "fv_batch_create: meshes must share device, precision, gamma and Newton settings");
    if (m->d.guess != FV_GUESS_TWO_RAREFACTION)
      return bfail(FV_ERR_INVALID_ARG, "fv_batch_create: batches use the two-rarefaction guess");
    if (m->order != FV_ORDER_FINEST_FIRST)
      return bfail(FV_ERR_INVALID_ARG, "fv_batch_create: batches use FV_ORDER_FINEST_FIRST");
  }
  BCK(cudaSetDevice(m0->cfg.device));
  fv_batch *b = new fv_batch();
  b->n = n;
  b->device = m0->cfg.device;
  for (int i = 0; i < n; ++i) {
    b->meshes.push_back(meshes[i]);
    b->Lmax = meshes[i]->L > b->Lmax ? meshes[i]->L : b->Lmax;
  }
  b->thetamax = b->Lmax - 1;

  // ---- schedule: simulate every instance's own phase sequence
  std::vector<PhaseDesc> pds;   // rows of n descriptors
  std::vector<int> actives;     // rows of n flags
  std::vector<int64_t> tn(n * FV_MAXL, 0);
  std::vector<char> pred(n * FV_MAXL, 0);
  PhaseDesc idle;
  memset(&idle, 0, sizeof idle);
  const int nsub = 1 << b->thetamax;
  for (int s = 1; s <= nsub; ++s) {
    std::vector<int> si(n), th(n);
    for (int i = 0; i < n; ++i) {
      th[i] = meshes[i]->L - 1;
      si[i] = ((s - 1) % (1 << th[i])) + 1;
    }
    // level assignment for the instances starting a cycle
    std::vector<int> act(n, 0);
    bool any = false;
    for (int i = 0; i < n; ++i)
      if (si[i] == 1) {
        act[i] = 1;
        any = true;
        for (int j = 0; j < FV_MAXL; ++j) {
          tn[i * FV_MAXL + j] = 0;
          pred[i * FV_MAXL + j] = 0;
        }
      }
    if (any) {
      b->steps.push_back({0, (int)(actives.size() / n)});
      actives.insert(actives.end(), act.begin(), act.end());
    }
    // begin phase of every instance
    {
      size_t row = pds.size() / n;
      for (int i = 0; i < n; ++i) {
        int tau = 0;
        for (int tmp = 1; tmp <= th[i]; ++tmp)
          if ((si[i] - 1) % (1 << tmp) == 0) tau = tmp;
        SchedPhase ph{0, tau, (int64_t)(si[i] - 1)};
        bool pr[FV_MAXL];
        for (int j = 0; j < FV_MAXL; ++j) pr[j] = pred[i * FV_MAXL + j];
        pds.push_back(phase_desc(meshes[i]->L, &tn[i * FV_MAXL], pr, ph));
        phase_apply(&tn[i * FV_MAXL], pr, ph);
        for (int j = 0; j < FV_MAXL; ++j) pred[i * FV_MAXL + j] = pr[j];
      }
      b->steps.push_back({1, (int)row});
    }
    // end phases, finest first
    std::vector<PhaseDesc> ends(n, idle);
    for (int k = 0; k <= b->thetamax; ++k) {
      size_t row = pds.size() / n;
      bool anyk = false;
      for (int i = 0; i < n; ++i) {
        PhaseDesc pd = idle;
        if (k <= th[i] && si[i] % (1 << k) == 0) {
          SchedPhase ph{1, k, (int64_t)si[i]};
          bool pr[FV_MAXL];
          for (int j = 0; j < FV_MAXL; ++j) pr[j] = pred[i * FV_MAXL + j];
          pd = phase_desc(meshes[i]->L, &tn[i * FV_MAXL], pr, ph);
          phase_apply(&tn[i * FV_MAXL], pr, ph);
          for (int j = 0; j < FV_MAXL; ++j) pred[i * FV_MAXL + j] = pr[j];
          anyk = true;
        }
        pds.push_back(pd);
      }
      if (anyk)
        b->steps.push_back({1, (int)row});
      else
        pds.resize(row * n);
    }
    // cycle ends
    {
      size_t row = pds.size() / n;
      bool anye = false;
      for (int i = 0; i < n; ++i) {
        PhaseDesc pd = idle;
        if (si[i] == (1 << th[i])) {
          pd.end_cycle = 1;
          anye = true;
        }
        pds.push_back(pd);
      }
      if (anye)
        b->steps.push_back({2, (int)row});
      else
        pds.resize(row * n);
    }
  }

  // ---- device tables
  std::vector<DevMesh> hms(n);
  std::vector<int> tpc(n + 1, 0), tpf(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    hms[i] = meshes[i]->d;
    hms[i].sort_cnt = meshes[i]->cnt_scratch;
    b->cells += meshes[i]->d.N;
    b->faces += meshes[i]->d.F;
    tpc[i + 1] = tpc[i] + (meshes[i]->d.N + 1023) / 1024;
    tpf[i + 1] = tpf[i] + (meshes[i]->d.F + 1023) / 1024;
  }
  b->tiles_c = tpc[n];
  b->tiles_f = tpf[n];
  int rc = FV_OK;
  // the batched kernels index the concatenated ranges with int32
  if (b->cells > FV_MAX_ITEMS || b->faces > FV_MAX_ITEMS) {
    delete b;
    return bfail(FV_ERR_INVALID_ARG, "fv_batch_create: more than 2^31 - 2^22 cells or faces in all");
  }
  rc = rc ? rc : balloc(b, &b->d_ms, n);
  rc = rc ? rc : balloc(b, &b->d_pds, pds.size());
  rc = rc ? rc : balloc(b, &b->d_active, actives.size());
  rc = rc ? rc : balloc(b, &b->d_tpref_c, n + 1);
  rc = rc ? rc : balloc(b, &b->d_tpref_f, n + 1);
  if (rc) {
    fv_batch_free(b);
    return rc;
  }
  cudaError_t e = cudaMemcpy(b->d_ms, hms.data(), n * sizeof(DevMesh), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_pds, pds.data(), pds.size() * sizeof(PhaseDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !actives.empty())
    e = cudaMemcpy(b->d_active, actives.data(), actives.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tpref_c, tpc.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tpref_f, tpf.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    fv_batch_free(b);
    return bfail(FV_ERR_CUDA, std::string("fv_batch_create: ") + cudaGetErrorString(e));
  }
  *out = b;
  return FV_OK;
}

int fv_batch_advance(fv_batch *b, int n_cycles, void *stream) {
  if (!b || n_cycles < 0) return bfail(FV_ERR_INVALID_ARG, "fv_batch_advance: bad argument");
  for (fv_mesh *m : b->meshes)
    if (m->in_cycle)
      return bfail(FV_ERR_INVALID_ARG, "fv_batch_advance: a mesh is inside a cycle of its own");
  BCK(cudaSetDevice(b->device));
  // the batch schedule runs whole cycles, but a failed launch could leave a
  // mesh mid-cycle: the next fv_set_state clears its accumulators
  for (fv_mesh *m : b->meshes) m->acc_dirty = true;
  cudaStream_t s = (cudaStream_t)stream;
  const bool graphable = b->use_graph && s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
  if (graphable && !b->graph && n_cycles > 0) {
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = run_steps(b, s);
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return bfail(FV_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiateWithFlags(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return bfail(FV_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
  }
  for (int c = 0; c < n_cycles; ++c) {
    if (graphable && b->graph) {
      BCK(cudaGraphLaunch(b->graph, s));
    } else {
      int rc = run_steps(b, s);
      if (rc) return rc;
    }
  }
  return FV_OK;
}

int fv_batch_info(fv_batch *b, int *subiterations, int *kernel_launches) {
  if (!b) return bfail(FV_ERR_INVALID_ARG, "fv_batch_info: NULL batch");
  if (subiterations) *subiterations = 1 << b->thetamax;
  if (kernel_launches) {
    int k = 0;
    for (const auto &st : b->steps) k += st.type == 0 ? (11 + (b->Lmax - 1) + ((b->Lmax - 1) % 2 == 0)) : st.type == 1 ? 4 : 1;
    *kernel_launches = k;
  }
  return FV_OK;
}

int fv_batch_set_launch(fv_batch *b, const int32_t per_sm[4]) {
  if (!b || !per_sm) return bfail(FV_ERR_INVALID_ARG, "fv_batch_set_launch: NULL argument");
  for (int k = 0; k < 4; ++k)
    if (per_sm[k] < 1 || per_sm[k] > 64)
      return bfail(FV_ERR_INVALID_ARG, "fv_batch_set_launch: 1..64 blocks per SM");
  for (int k = 0; k < 4; ++k) b->launch.per_sm[k] = per_sm[k];
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return FV_OK;
}

int fv_batch_get_launch(fv_batch *b, int32_t per_sm[4]) {
  if (!b || !per_sm) return bfail(FV_ERR_INVALID_ARG, "fv_batch_get_launch: NULL argument");
  for (int k = 0; k < 4; ++k) per_sm[k] = b->launch.per_sm[k];
  return FV_OK;
}

int fv_batch_mlp_load(fv_batch *b, const float *params_dev, int n_params, int target, double gate) {
  if (!b || !params_dev || n_params != 4673 || (target != 0 && target != 1) || !std::isfinite(gate) ||
      gate > 1e38)
    return bfail(FV_ERR_INVALID_ARG, "fv_batch_mlp_load: bad argument");
  BCK(cudaSetDevice(b->device));
  if (!b->mlp) {
    int rc = balloc(b, &b->mlp, (size_t)2560);
    if (rc) return rc;
  }
  if (fvk::launch_mlp_pack(params_dev, target, (float)gate, b->mlp, 0) != FV_OK)
    return bfail(FV_ERR_CUDA, "fv_batch_mlp_load: pack launch failed");
  BCK(cudaDeviceSynchronize());
  b->use_mlp = true;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return FV_OK;
}

int fv_batch_set_guess(fv_batch *b, int guess) {
  if (!b || (guess != FV_GUESS_TWO_RAREFACTION && guess != FV_GUESS_MLP))
    return bfail(FV_ERR_INVALID_ARG, "fv_batch_set_guess: bad argument");
  if (guess == FV_GUESS_MLP && !b->mlp)
    return bfail(FV_ERR_INVALID_ARG, "fv_batch_set_guess: no network loaded (fv_batch_mlp_load)");
  b->use_mlp = guess == FV_GUESS_MLP;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return FV_OK;
}

int fv_batch_use_graph(fv_batch *b, int enable) {
  if (!b) return bfail(FV_ERR_INVALID_ARG, "fv_batch_use_graph: NULL batch");
  b->use_graph = enable != 0;
  return FV_OK;
}

}  // extern "C"

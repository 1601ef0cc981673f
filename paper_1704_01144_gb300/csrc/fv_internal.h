// fv_internal.h -- data layout shared by the host side and the kernels of the
// GB300 library (not part of the C ABI).
//
// Layout in HBM (N cells after Morton renumbering, F faces numbered by owner
// cell).  Everything a kernel gathers through an index (a neighbour's or a
// face's cell record, a cell's face records) is a padded record read with
// 16-byte vector loads, so one gather touches one or two 32-byte sectors;
// what is streamed in cell order (the conserved state) is
// structure-of-arrays.
//   cells  vol[N], ivol[N] (ivol32 in FP32 mode), cf4[N] faces of local faces
//          0..3, cnb4[N] neighbours across them (-1 wall, -2 transmissive),
//          cown[N] bit j set when the cell owns local face j, lsw[N][12]
//          least-squares weights (3 per local face; lsw32 in FP32 mode),
//          lev[N] temporal level
//   faces  fcell[F] = (owner, neighbour or -bc), fgeo[F][8] = (unit normal
//          owner -> outside, area, x_R - x_L (ghost centroid on boundary
//          faces), pad) in FP64 and fgeo32 in FP32 mode, flev[F]
//   state  Un[5][N] (FP64), Us[5][N] predicted (FP64 mode) or Un32/Us32
//          (FP32-flux mode: FP32 shadow of U^n and the FP32 predicted
//          state, which only ever feeds fluxes)
//   phase  W[N][8] primitives at the phase time, G[N][16] gradients (FP64 or
//          FP32 by mode); FA[F][6] predictor flux x area (FP64 mode; FA32
//          [F][8] in FP32 mode), then the step's flux time integral in
//          units of the level's half step dt_k/2; ACC[F][6] fine-side
//          integral on level interfaces, in units of the coarse level's
//          half step; BND[F][6] boundary ledger (time units)
//   lists  cl[N] cells sorted by (level, has-finer-neighbour), coff[2L+1],
//          with clf/cln/clb the sorted faces, neighbours and bits of each
//          entry; fl[F] faces sorted by face level, foff[L+1], with flc the
//          sorted cell pairs
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/fv.h"

#define FV_MAXL 8
// record strides (elements)
#define REC_W 8     // primitives (5 used)
#define REC_G 16    // gradients (15 used)
#define REC_FG 8    // face geometry: n[3], A, r[3], pad
#define REC_FA 6    // FP64 face values (5 used)
#define REC_FA32 8  // FP32 face values (5 used)
#define REC_LSW 12  // least-squares weights
#define REC_U32 8   // FP32 shadow state: 5 conserved values, the cell's level, pad
#define FV_STATUS_NONPHYS 1
#define FV_STATUS_RIEMANN 2
#define FV_STATUS_TIMEOUT 4  // a bounded grid barrier gave up

// state of the persistent kernel's grid barrier (reset before each launch)
struct GridBar {
  unsigned count, gen;
};

#define FV_HIST_CAP 4096  // cycles kept by the level history

// largest cell or face count (ids are int32; grid-stride loops overshoot a
// range end by less than 2^22)
#define FV_MAX_ITEMS ((int64_t)0x7fffffff - ((int64_t)1 << 22))

struct DevMesh {
  int N, F, L;
  // cells
  double *vol, *ivol;  // volume and its reciprocal
  float *ivol32;       // FP32 reciprocal volume (FP32-flux mode predictor)
  int4 *cf4, *cnb4;
  uint8_t *cown;
  double *lsw;
  float *lsw32;        // FP32 copy of the weights (FP32-flux mode)
  // faces
  int2 *fcell;
  double *fgeo;
  float *fgeo32;
  // state
  double *Un, *Us, *G;  // Us: predicted state (FP64 mode only)
  float *Un32, *Us32;    // FP32-flux mode: FP32 shadow of U^n, predicted state ([N][REC_U32])
  double *UsD;           // FP32-flux mode, order 1: the provisional end state in FP64 (SoA [5][N])
  float *G32;
  double *FA, *ACC, *BND;
  float *FA32;         // FP32-flux mode: predictor flux x area
  // levels and sorted lists
  int8_t *lev, *lev_tmp, *flev;
  uint8_t *ckey, *fkey;
  uint8_t *cmask;         // per cell: bit j set when the neighbour across face j is
                          // one level finer (that face's integral accumulates)
  int *cl, *fl, *coff, *foff;
  // the sorted lists also carry, per list position, what every phase kernel
  // reads first about its item, so that a kernel reaches the item's
  // neighbours and faces one dependent load earlier: cells their faces
  // (clf = cf4[cl]), neighbours (cln = cnb4[cl]) and the bits own | finer << 4
  // (clb); faces their two cells (flc = fcell[fl]).  Written by the level
  // sort with the lists.
  int4 *clf, *cln;
  uint8_t *clb;
  int2 *flc;
  int *sort_cnt;          // bucket x block counts, scratch of the level sort
  double *dt;             // exact local time steps (where dteps = 0)
  float *dt32;            // FP32 estimates of the local time steps (where dteps > 0)
  float *dteps;           // relative bound of the estimate (0: dt holds the exact value)
  unsigned long long *dthi_bits;  // smallest upper bound of the estimates (bit pattern)
  unsigned long long *dtmin_bits;  // bit pattern of dt_min (positive double)
  int *sweep_changed;     // per smoothing sweep of the level rule: 1 if it lowered a level
  double *tdev;           // physical time
  int *status;            // sticky status bits
  long long *counters;    // [0] cycles, [1] weighted cell updates, [2] face evaluations
  int *hist;              // per cycle (ring of FV_HIST_CAP): cells per level [FV_MAXL]
  double *hist_dt;        // per cycle: dt_min
  // phase scratch: primitives at the phase time (FP64 or FP32 records)
  void *W;
  int precision;
  // starting guess of the Riemann solver's Newton iteration: FV_GUESS_TR or
  // FV_GUESS_MLP with the packed network weights (device, PK_WORDS words)
  int guess;
  const uint32_t *mlp;
  // FP32-flux mode: phases with at most this many faces fuse their gradients
  // into the flux kernel (0: never)
  int fuse_faces;
  // FP32-flux mode: the predictor's residual sum in FP64 (FV_SUM_FP64) or
  // FP32 (FV_SUM_FP32)
  int pred_sum64;
  // FP32-flux mode, two-rarefaction guess, no fusion: the flux kernel stages
  // its gathered inputs through shared memory (k_flux_staged)
  int flux_staged;
  // the update's gather: one thread per cell (0) or four lanes per cell (1)
  int gather_quad;
  // physics
  double gamma, cfl, tol;
  int maxit;
};

// Per-level view of the phase time: mode 0 = U^n, 1 = U*, 2 = interpolate
// U^n + w (U* - U^n).
struct PhaseLevels {
  double w[FV_MAXL];
  int mode[FV_MAXL];
};

// What one phase does on one mesh: the kind of update (stage 1 begins the
// levels 0..level, stage 2 ends the step of `level`), the view of every level
// at the phase time, and the bucket ranges of the level-sorted lists each
// kernel covers (cells: coff buckets [b0, b1); faces: foff buckets).
struct PhaseDesc {
  PhaseLevels pl;
  int stage, level;  // stage 1 begin, 2 end, 3 correct, 4 commit (see phase_desc)
  int pb0, pb1;  // primitives
  int gb0, gb1;  // gradients
  int fb0, fb1;  // faces
  int ub0, ub1;  // cell updates
  int active;    // 0: the mesh sits this phase out (batches)
  int end_cycle; // 1: the mesh's cycle ends with this phase (batches)
};

#define FV_MAXB 64  // instances per batch

// grid sizes of the phase kernels, in blocks per SM (256 threads for
// primitives / gradients / updates, 128 for fluxes); results do not depend
// on them (items are independent), so an autotuner may pick any
struct LaunchCfg {
  int per_sm[4];  // prim, grad, flux, update
};
inline LaunchCfg default_launch() { return LaunchCfg{{8, 8, 16, 8}}; }

// ---- host schedule of one cycle (the subiteration loop of Alg. 2) ----
// kind 0: begin (predict) levels 0..level at T; kind 1: end the step of
// `level` at T (order 0); kind 2: correct `level` at the end T of its step,
// giving its provisional end state (order 1); kind 3: commit levels 0..level
// at T with the deferred interface correction (order 1)
struct SchedPhase {
  int kind;
  int level;
  int64_t T;  // time in dt_min units from the cycle start
};

// Order 0 (FV_ORDER_FINEST_FIRST): for s = 1..2^theta, B(s) then the ends of
// the levels k with s mod 2^k == 0, finest first.  Order 1 (FV_ORDER_PAPER):
// the loops of Alg. 2 -- for s > 1 the commit of levels 0..tau(s) at s - 1,
// B(s), then the correctors of tau' = tau(s) down to 0 at s - 1 + 2^tau' --
// and the final commit of every level (the extra subiteration of Alg. 3).
inline std::vector<SchedPhase> make_phases(int theta, int order = 0) {
  std::vector<SchedPhase> out;
  int nsub = 1 << theta;
  for (int s = 1; s <= nsub; ++s) {
    int tau = 0;
    for (int tmp = 1; tmp <= theta; ++tmp)
      if ((s - 1) % (1 << tmp) == 0) tau = tmp;
    if (order == 1) {
      if (s > 1) out.push_back({3, tau, (int64_t)(s - 1)});
      out.push_back({0, tau, (int64_t)(s - 1)});
      for (int k = tau; k >= 0; --k) out.push_back({2, k, (int64_t)(s - 1) + ((int64_t)1 << k)});
    } else {
      out.push_back({0, tau, (int64_t)(s - 1)});
      for (int k = 0; k <= theta && s % (1 << k) == 0; ++k) out.push_back({1, k, (int64_t)s});
    }
  }
  if (order == 1) out.push_back({3, theta, (int64_t)nsub});
  return out;
}

// the view of every level at time T from each level's step start tn and
// whether its predicted (or, order 1, provisional end) state exists; with
// `extrapolate` (order 1 correctors) a level may be taken up to one step past
// its predicted state, linearly
inline PhaseLevels levels_at(int L, const int64_t *tn, const bool *pred, int64_t T, bool extrapolate = false) {
  PhaseLevels pl;
  for (int j = 0; j < FV_MAXL; ++j) {
    pl.w[j] = 0.0;
    pl.mode[j] = 0;
    if (j >= L) continue;
    int64_t dd = T - tn[j];
    int64_t span = (int64_t)1 << j;
    if (dd <= 0 || dd > (extrapolate ? 2 * span : span) || !pred[j]) continue;  // U^n (or not needed)
    if (dd == span) {
      pl.mode[j] = 1;
    } else {
      pl.mode[j] = 2;
      pl.w[j] = (double)dd / (double)span;
    }
  }
  return pl;
}

// what a phase covers: begin(tau) -> primitives of levels <= tau+2,
// gradients of levels <= tau plus the level-(tau+1) cells next to level tau,
// faces of level <= tau, updates of levels <= tau; end(k) and correct(k) ->
// primitives of levels k-1..k+2, gradients of level k plus the halo of k+1,
// faces of level k, updates of level k; commit(tau) -> updates of levels
// <= tau only (cell buckets: 2 level + no-finer-neighbour).  Stages: 1
// begin, 2 end, 3 correct, 4 commit.
inline PhaseDesc phase_desc(int L, const int64_t *tn, const bool *pred, const SchedPhase &ph) {
  const int nb = 2 * L;
  auto cl = [nb](int b) { return b < 0 ? 0 : (b > nb ? nb : b); };
  auto fclip = [L](int b) { return b < 0 ? 0 : (b > L ? L : b); };
  PhaseDesc pd;
  memset(&pd, 0, sizeof pd);
  pd.pl = levels_at(L, tn, pred, ph.T, ph.kind == 2);
  pd.active = 1;
  pd.level = ph.level;
  if (ph.kind == 0) {
    int tau = ph.level;
    pd.stage = 1;
    pd.pb0 = 0; pd.pb1 = cl(2 * (tau + 3));
    pd.gb0 = 0; pd.gb1 = cl(2 * tau + 3);
    pd.fb0 = 0; pd.fb1 = fclip(tau + 1);
    pd.ub0 = 0; pd.ub1 = cl(2 * tau + 2);
  } else if (ph.kind == 3) {
    pd.stage = 4;
    pd.ub0 = 0; pd.ub1 = cl(2 * ph.level + 2);
  } else {
    int k = ph.level;
    pd.stage = ph.kind == 1 ? 2 : 3;
    pd.pb0 = cl(2 * (k - 1)); pd.pb1 = cl(2 * (k + 3));
    pd.gb0 = cl(2 * k); pd.gb1 = cl(2 * k + 3);
    pd.fb0 = fclip(k); pd.fb1 = fclip(k + 1);
    pd.ub0 = cl(2 * k); pd.ub1 = cl(2 * k + 2);
  }
  return pd;
}

inline void phase_apply(int64_t *tn, bool *pred, const SchedPhase &ph) {
  if (ph.kind == 0) {
    for (int j = 0; j <= ph.level; ++j) pred[j] = true;
  } else if (ph.kind == 1) {
    tn[ph.level] = ph.T;
    pred[ph.level] = false;
  } else if (ph.kind == 3) {
    for (int j = 0; j <= ph.level; ++j) {
      tn[j] = ph.T;
      pred[j] = false;
    }
  }
}

// host-side mesh preprocessing result (fv_host.cpp)
struct HostMesh {
  int64_t N = 0, F = 0;
  std::vector<int64_t> new2old, old2new;
  std::vector<double> vol;                   // N
  std::vector<double> xc;                    // 3N (SoA)
  std::vector<int> cf, cnb;                  // 4N (SoA, j-major)
  std::vector<uint8_t> cown;                 // N
  std::vector<double> lsw;                   // 12N (SoA)
  std::vector<int> fown, fnb;                // F
  std::vector<double> fn, farea, fr;         // 3F, F, 3F (SoA)
};

// Builds faces, geometry, Morton order.  Returns FV_OK or FV_ERR_* and sets
// *err on failure.
int fv_host_build(const double *xyz, int64_t n_nodes, const int64_t *tets, int64_t n_tets,
                  const int8_t *face_bc, HostMesh &out, std::string *err);

// sets the message fv_last_error() returns to the calling thread
void fv_internal_set_error(const std::string &msg);

// Optional per-kernel-class timing: events recorded on the launching stream
// around each launch when a hook is active.
struct ProfHook {
  bool on = false;
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  double ms[FV_PROF_N] = {0, 0, 0, 0, 0};
  long long launches[FV_PROF_N] = {0, 0, 0, 0, 0};
};

struct ProfScope {
  ProfHook *h;
  int cls;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(ProfHook *hook, int c, cudaStream_t st) : h(hook), cls(c), s(st) {
    if (h && h->on) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (h && h->on) {
      cudaEventRecord(b, s);
      h->recs.push_back({cls, a, b});
    }
  }
};

// a mesh handle (C ABI type fv_mesh)
struct fv_mesh {
  fv_config cfg;
  DevMesh d;
  int L = 1, theta = 0;
  int *new2old_dev = nullptr;  // Morton index -> caller's index
  void *W = nullptr;           // phase-time primitives (FP64 or FP32)
  double *FAt = nullptr;       // residual-hook scratch (REC_FA x F; also host staging)
  int *cnt_scratch = nullptr;  // level-sort counts
  std::vector<SchedPhase> phases;
  int order = 0;               // FV_ORDER_FINEST_FIRST or FV_ORDER_PAPER
  // the boundary faces (the only faces whose ledger entries are ever
  // written) and whether the interface accumulators may hold values: they
  // are all zero after every completed cycle
  int *bfaces_dev = nullptr;
  int n_bfaces = 0;
  bool acc_dirty = false;
  bool in_cycle = false;
  int next_phase = 0;
  int64_t tn[FV_MAXL];
  bool pred[FV_MAXL];
  std::vector<void *> allocs;
  ProfHook prof;
  bool use_graph = true;
  cudaGraphExec_t cycle_graph = nullptr;
  bool have_dt = false;
  bool in_batch = false;       // owned by a batch's schedule while advancing
  LaunchCfg launch = default_launch();
  bool use_persistent = false;    // whole cycles as one cooperative launch
  PhaseDesc *pds_dev = nullptr;   // the cycle's phase descriptors (persistent mode)
  GridBar *bar = nullptr;
  int levels_step = 0;            // split level assignment: 1 after the local steps, 2 after classifying
};

// kernels (fv_kernels.cu)
namespace fvk {
void init_device_info();
int launch_assign_levels(const DevMesh &d, int L, int *cnt_scratch, ProfHook *ph, cudaStream_t s);
// its three parts (a sharded run inserts its exchanges between them)
int launch_levels_local_dt(const DevMesh &d, cudaStream_t s);
int launch_set_dt_min(const DevMesh &d, double dt_min, cudaStream_t s);
int launch_levels_classify(const DevMesh &d, int L, cudaStream_t s);
int launch_levels_sort(const DevMesh &d, cudaStream_t s);
// ghost-cell records of a sharded run (fv_shard.cu)
int launch_halo(const DevMesh &d, const int *cells, int n, int what, void *buf, bool pack, cudaStream_t s);
int launch_phase(const DevMesh &d, const PhaseDesc &pd, const LaunchCfg &lc, ProfHook *ph,
                 cudaStream_t s);
// batches: ms/pds are device arrays of n meshes / descriptors of one phase
int launch_phase_multi(const DevMesh *ms, const PhaseDesc *pds, int n, const DevMesh &d0,
                       int64_t max_cells, int64_t max_faces, const LaunchCfg &lc, const uint32_t *mlp,
                       cudaStream_t s);
int launch_assign_multi(const DevMesh *ms, const int *active, int n, int Lmax, int64_t max_cells,
                        int64_t max_faces, int64_t max_cell_blocks, int64_t max_face_blocks,
                        int *cnt_scratch, const int *blk_pref_c, const int *blk_pref_f, cudaStream_t s);
int launch_time_advance_multi(const DevMesh *ms, const PhaseDesc *pds, int n, cudaStream_t s);
int launch_residual(const DevMesh &d, int precision, const PhaseLevels &pl, int level, void *Wbuf,
                    double *FAt, double *R, const int *new2old, cudaStream_t s);
int launch_time_advance(const DevMesh &d, int theta, cudaStream_t s);
int launch_set_state(const DevMesh &d, const double *prim, const int *new2old, cudaStream_t s);
int launch_set_cons(const DevMesh &d, const double *cons, const int *new2old, cudaStream_t s);
int launch_zero_faces(double *rec, const int *faces, int n, cudaStream_t s);
int launch_get_state(const DevMesh &d, double *cons, const int *new2old, cudaStream_t s);
int launch_get_levels(const DevMesh &d, int8_t *lev, const int *new2old, cudaStream_t s);
int launch_check_state(const DevMesh &d, cudaStream_t s);
int launch_flux_batch(const double *WL, const double *WR, const double *nrm, int n, double gamma,
                      double tol, int maxit, int precision, int bc, double *F, int *iters,
                      const uint32_t *mlp, cudaStream_t s);
int launch_harvest(const DevMesh &d, double *out, int m, long long a, long long b, cudaStream_t s);
// every phase of a cycle in one cooperative launch (pds: the cycle's nph
// phase descriptors in device memory; bar: barrier state, reset here)
int launch_persistent_cycle(const DevMesh &d, const PhaseDesc *pds, int nph, GridBar *bar,
                            cudaStream_t s);
int launch_barrier_probe(GridBar *bar, int *status, int rounds, unsigned extra, cudaStream_t s);
// fv_mlp.cu: FP32 parameters -> packed bf16 fragments (PK_WORDS words)
int launch_mlp_pack(const float *params, int target, float gate, uint32_t *packed, cudaStream_t s);
}  // namespace fvk

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
//          [F][8] in FP32 mode), then the step's flux time integral;
//          ACC[F][6] fine-side integral on level interfaces; BND[F][6]
//          boundary ledger
//   lists  cl[N] cells sorted by (level, has-finer-neighbour), coff[2L+1];
//          fl[F] faces sorted by face level, foff[L+1]
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
#define FV_STATUS_NONPHYS 1
#define FV_STATUS_RIEMANN 2

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
  float *Un32, *Us32;    // FP32-flux mode: FP32 shadow of U^n, predicted state
  float *G32;
  double *FA, *ACC, *BND;
  float *FA32;         // FP32-flux mode: predictor flux x area
  // levels and sorted lists
  int8_t *lev, *lev_tmp, *flev;
  uint8_t *ckey, *fkey;
  int *cl, *fl, *coff, *foff;
  int *sort_cnt;          // bucket x block counts, scratch of the level sort
  double *dt;             // local time steps
  unsigned long long *dtmin_bits;  // bit pattern of dt_min (positive double)
  double *tdev;           // physical time
  int *status;            // sticky status bits
  long long *counters;    // [0] cycles, [1] weighted cell updates, [2] face evaluations
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

// kernels (fv_kernels.cu)
namespace fvk {
void init_device_info();
int launch_assign_levels(const DevMesh &d, int L, int *cnt_scratch, ProfHook *ph, cudaStream_t s);
int launch_phase(const DevMesh &d, int precision, const PhaseLevels &pl, int stage, int level,
                 int pb0, int pb1, int gb0, int gb1, int fb0, int fb1, int ub0, int ub1, void *Wbuf,
                 ProfHook *ph, cudaStream_t s);
int launch_residual(const DevMesh &d, int precision, const PhaseLevels &pl, int level, void *Wbuf,
                    double *FAt, double *R, const int *new2old, cudaStream_t s);
int launch_time_advance(const DevMesh &d, int theta, cudaStream_t s);
int launch_set_state(const DevMesh &d, const double *prim, const int *new2old, cudaStream_t s);
int launch_set_cons(const DevMesh &d, const double *cons, const int *new2old, cudaStream_t s);
int launch_get_state(const DevMesh &d, double *cons, const int *new2old, cudaStream_t s);
int launch_get_levels(const DevMesh &d, int8_t *lev, const int *new2old, cudaStream_t s);
int launch_check_state(const DevMesh &d, cudaStream_t s);
int launch_flux_batch(const double *WL, const double *WR, const double *nrm, int n, double gamma,
                      double tol, int maxit, int precision, int bc, double *F, int *iters,
                      cudaStream_t s);
}  // namespace fvk

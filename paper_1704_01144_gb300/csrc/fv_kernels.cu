// fv_kernels.cu -- the hot path of one temporally adaptive cycle (Alg. 2)
// as CUDA kernels for sm_103a.
//
// Per cycle:  k_dt32 (certified FP32 local steps) -> k_dt_min_exact (exact
//             FP64 minimum) -> k_levels0_certified -> k_smooth x (L-1) ->
//             cell/face keys -> counting sort (hist, scan, scatter) for
//             cells and faces.
// Per phase:  [FP64 mode: k_prim (states at the phase time, time-
//             interpolated)] ->
//             gradients (least squares; the FP32-flux mode computes the
//                        primitives of the cell and its neighbours here) ->
//             flux (MUSCL-minmod + exact Riemann, optionally the learned
//                   starting guess; predictor stash or corrector time
//                   integral + interface accumulation) ->
//             update (per-cell gather over the 4 faces in fixed order, no
//                     atomics; predictor U* or corrector U^{n+1}).
//
// Every phase kernel grid-strides over a range of a level-sorted list whose
// bounds are read from device memory, so inactive levels cost a few idle
// blocks and the launch sequence of a cycle is fixed (graph-capturable).
// Gathered data (cell state, primitive and gradient records, face geometry
// and flux records) are padded records read with 16-byte vector loads; the
// FP64 state is structure-of-arrays.  Cells follow a Morton curve, faces
// their owner cell.
#include <cuda_runtime.h>

#include <cstring>

#include "fv_internal.h"
#include "fv_riemann.cuh"
#include "fv_mlp.cuh"

namespace fvk {

static int g_num_sms = 0;
static int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

static inline int grid_for(int64_t items, int block, int per_sm) {
  int64_t need = (items + block - 1) / block;
  int64_t cap = (int64_t)num_sms() * per_sm;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

#define FV_LAUNCH_CHECK()                        \
  do {                                           \
    cudaError_t e_ = cudaGetLastError();         \
    if (e_ != cudaSuccess) return FV_ERR_CUDA;   \
  } while (0)

// ------------------------------------------------------------- helpers ---
// Programmatic dependent launch: a kernel of the cycle waits (in hardware) for the
// kernel before it to finish and flush before it reads anything, and lets
// the next one be launched once its own items are done, so launch and
// ramp-up of the next kernel overlap the drain of this one.  Without a
// programmatic predecessor the wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// N-element record loads/stores with 16-byte vector accesses (records are
// 16-byte aligned: cudaMalloc bases and strides that are multiples of 16 B)
template <int NE>
__device__ __forceinline__ void ldrec(const float *p, float *o) {
  static_assert(NE % 4 == 0, "record of float4");
#pragma unroll
  for (int k = 0; k < NE / 4; ++k) {
    float4 v = reinterpret_cast<const float4 *>(p)[k];
    o[4 * k] = v.x;
    o[4 * k + 1] = v.y;
    o[4 * k + 2] = v.z;
    o[4 * k + 3] = v.w;
  }
}
template <int NE>
__device__ __forceinline__ void ldrec(const double *p, double *o) {
  static_assert(NE % 2 == 0, "record of double2");
#pragma unroll
  for (int k = 0; k < NE / 2; ++k) {
    double2 v = reinterpret_cast<const double2 *>(p)[k];
    o[2 * k] = v.x;
    o[2 * k + 1] = v.y;
  }
}
template <int NE>
__device__ __forceinline__ void strec(float *p, const float *o) {
#pragma unroll
  for (int k = 0; k < NE / 4; ++k)
    reinterpret_cast<float4 *>(p)[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
}
template <int NE>
__device__ __forceinline__ void strec(double *p, const double *o) {
#pragma unroll
  for (int k = 0; k < NE / 2; ++k) reinterpret_cast<double2 *>(p)[k] = make_double2(o[2 * k], o[2 * k + 1]);
}
// x 2^k for a positive normal x whose scaled value stays normal (dt_min and
// the level steps 2^k dt_min): the exponent field plus k -- exact, the value
// ldexp gives, in integer instructions only
__device__ __forceinline__ double scale2(double x, int k) {
  return __longlong_as_double(__double_as_longlong(x) + ((long long)k << 52));
}
__device__ __forceinline__ int nbr_of(const int4 &v, int j) {
  return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}
template <typename T>
__device__ __forceinline__ void cons_to_prim(const T U[5], T gm1, T W[5]) {
  T r = U[0];
  T ri = qdiv(T(1), r);  // FP32: the fast quotient (about 2 ulps)
  T u = U[1] * ri, v = U[2] * ri, w = U[3] * ri;
  T ke = T(0.5) * r * ((u * u + v * v) + w * w);
  W[0] = r;
  W[1] = u;
  W[2] = v;
  W[3] = w;
  W[4] = gm1 * (U[4] - ke);
}

// FP64 primitives without an FP64 division: the single-precision reciprocal
// of rho refined by two Newton steps r <- r (2 - rho r) (error ~1e-16)
__device__ __forceinline__ void prim_fp64(const double U[5], double gm1, double W[5]) {
  double r = U[0];
  double ri = (double)(1.0f / (float)r);
  ri = ri * (2.0 - r * ri);
  ri = ri * (2.0 - r * ri);
  double u = U[1] * ri, v = U[2] * ri, w = U[3] * ri;
  double ke = 0.5 * r * ((u * u + v * v) + w * w);
  W[0] = r;
  W[1] = u;
  W[2] = v;
  W[3] = w;
  W[4] = gm1 * (U[4] - ke);
}

__device__ __forceinline__ double minmod(double a, double b) {
  if (a > 0.0 && b > 0.0) return a < b ? a : b;
  if (a < 0.0 && b < 0.0) return a > b ? a : b;
  return 0.0;
}
// FP32: as max(min(a, b), 0) + min(max(a, b), 0), four min/max and an add
// without comparisons or selects; the same value as the branches above for
// every pair of numbers (one term is the result and the other zero, so the
// add is exact; a pair of opposite signs or with a zero gives a zero)
__device__ __forceinline__ float minmod(float a, float b) {
  return fmaxf(fminf(a, b), 0.f) + fminf(fmaxf(a, b), 0.f);
}

// ------------------------------------------------ level assignment (a1-a2)
// dt_i = 2 CFL V_i / sum_j A_j (|u_i . n_j| + c_i), with rho_i multiplied
// through: dt_i = 2 CFL V_i rho_i / sum_j A_j (|m_i . n_j| + sqrt(g p rho)),
// p = (g-1)(E - (|m|^2/2)/rho).  Evaluated with round-to-nearest intrinsics
// (no fused multiply-add) in the fixed order j = 0..3, so that it is bitwise
// the same number as a plain FP64 host evaluation of the same formula:
// temporal levels are integer decisions taken on it.
__device__ __forceinline__ double local_dt_of(const DevMesh &d, int i) {
  const size_t N = d.N;
  double r = d.Un[i];
  double mx = d.Un[N + i], my = d.Un[2 * N + i], mz = d.Un[3 * N + i];
  double mm = __dadd_rn(__dadd_rn(__dmul_rn(mx, mx), __dmul_rn(my, my)), __dmul_rn(mz, mz));
  double p = __dmul_rn(d.gamma - 1.0, __dsub_rn(d.Un[4 * N + i], __ddiv_rn(__dmul_rn(0.5, mm), r)));
  double rc = __dsqrt_rn(__dmul_rn(__dmul_rn(d.gamma, p), r));
  double S = 0.0;
  int4 cf = d.cf4[i];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const double *g = d.fgeo + (size_t)nbr_of(cf, j) * REC_FG;
    double2 n01 = reinterpret_cast<const double2 *>(g)[0];
    double2 n2A = reinterpret_cast<const double2 *>(g)[1];
    double mn = __dadd_rn(__dadd_rn(__dmul_rn(mx, n01.x), __dmul_rn(my, n01.y)), __dmul_rn(mz, n2A.x));
    S = __dadd_rn(S, __dmul_rn(n2A.y, __dadd_rn(fabs(mn), rc)));
  }
  double dt = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, d.cfl), d.vol[i]), r), S);
  if (!(p > 0.0) || !(r > 0.0) || !isfinite(dt)) {
    atomicOr(d.status, FV_STATUS_NONPHYS);
    dt = __longlong_as_double(0x7ff0000000000000LL);
  }
  d.dt[i] = dt;
  return dt;
}

// block minimum, then one atomic per block on the bit pattern (positive
// doubles order like their bit patterns): order-independent, exact.  Every
// thread of the block must call it.
__device__ __forceinline__ void block_min_to(double local_min, unsigned long long *bits) {
  __shared__ double sm[32];
  for (int o = 16; o > 0; o >>= 1) local_min = fmin(local_min, __shfl_xor_sync(0xffffffff, local_min, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = local_min;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : __longlong_as_double(0x7ff0000000000000LL);
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffff, v, o));
    if (threadIdx.x == 0) atomicMin(bits, (unsigned long long)__double_as_longlong(v));
  }
}

__global__ void k_init_min2(unsigned long long *a, unsigned long long *b) {
  pdl_wait();
  *a = 0x7ff0000000000000ULL;
  *b = 0x7ff0000000000000ULL;
  pdl_trigger();
}

// ---- certified FP32 estimate of the local step.  The estimate dt~ comes
// with a relative bound e such that the exact FP64 value of local_dt_of lies
// in [dt~ (1 - e), dt~ (1 + e)]; the bound is built from first-order error
// propagation (u = 2^-24 per rounding of the state, the geometry and every
// operation; the cancellation in E - |m|^2/(2 rho) enters as
// u (E + 8 ke) / (E - ke)), then widened by 1.25 plus 16 u and a 1e-13 term
// for the FP64 evaluation's own rounding.  A cell whose bound exceeds 2^-12,
// or whose pressure is not clearly positive, gets the exact FP64 value
// (which also raises the non-physical status as before).  The exact minimum
// and every level decision an estimate cannot settle are then taken on exact
// FP64 values, so levels and dt_min are bit for bit those of the all-FP64
// evaluation.
// Returns true with the estimate val and its bound eps, or false after the
// exact value was computed (local_dt_of: stored in d.dt[i], returned in
// exact).
__device__ __forceinline__ bool local_dt32(const DevMesh &d, int i, float &val, float &eps, double &exact) {
  const float u = 5.9604645e-8f;  // 2^-24
  float r, mx, my, mz, E, iv;
  if (d.Un32) {
    float a[REC_U32];
    ldrec<REC_U32>(d.Un32 + (size_t)i * REC_U32, a);
    r = a[0]; mx = a[1]; my = a[2]; mz = a[3]; E = a[4];
    iv = d.ivol32[i];
  } else {
    const size_t N = d.N;
    r = (float)d.Un[i]; mx = (float)d.Un[N + i]; my = (float)d.Un[2 * N + i];
    mz = (float)d.Un[3 * N + i]; E = (float)d.Un[4 * N + i];
    iv = (float)d.ivol[i];
  }
  const float g = (float)d.gamma, gm1 = (float)(d.gamma - 1.0);
  const float mm = mx * mx + my * my + mz * mz;
  const float ke = 0.5f * mm / r;
  const float P = E - ke;
  const float eP = u * (E + 8.0f * ke + P);              // |P~ - P| to first order
  if (!(r > 0.0f) || !(P > 4.0f * eP) || !isfinite(E + mm)) {
    exact = local_dt_of(d, i);
    return false;
  }
  const float relP = eP / (P - eP);
  const float p = gm1 * P;
  const float relq = relP + 6.0f * u;                     // gamma p rho
  const float rc = sqrtf(g * p * r);
  const float relc = 0.5f * relq + u;
  float S = 0.0f, eS = 0.0f;
  int4 cf = d.cf4[i];
  const float *fg = d.fgeo32;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float n0, n1, n2, A;
    const int f = nbr_of(cf, j);
    if (fg) {
      float4 q = *reinterpret_cast<const float4 *>(fg + (size_t)f * REC_FG);
      n0 = q.x; n1 = q.y; n2 = q.z; A = q.w;
    } else {
      const double *gd = d.fgeo + (size_t)f * REC_FG;
      n0 = (float)gd[0]; n1 = (float)gd[1]; n2 = (float)gd[2]; A = (float)gd[3];
    }
    const float amn = fabsf(mx * n0) + fabsf(my * n1) + fabsf(mz * n2);
    const float mn = fabsf(mx * n0 + my * n1 + mz * n2);
    const float t = mn + rc;
    S += A * t;
    eS += A * (6.0f * u * amn + relc * rc + 4.0f * u * t);
  }
  val = 2.0f * (float)d.cfl * r / (iv * S);
  float e = eS / S + 3.0f * u + 10.0f * u;
  e = 1.25f * e + 16.0f * u + 1e-13f;
  if (!(e <= 2.44140625e-4f) || !isfinite(val) || !(val > 0.0f)) {  // 2^-12
    exact = local_dt_of(d, i);
    return false;
  }
  eps = e;
  return true;
}

// The passes below compare in FP32 with directed rounding, which is exact
// for these questions: lo = val (1 - e) rounded down and hi = val (1 + e)
// rounded up enclose the cell's exact step, and for a float x and a double t,
// t <= x exactly when t rounded up to FP32 is <= x (x <= t when x <= t
// rounded down).  FP64 arithmetic -- a small fraction of the SM's FP32 rate
// on this GPU -- is left to the cells an interval cannot settle.

// pass 1 of one cell: its estimate (dt32, dteps) or its exact value (dt,
// dteps = 0); lowers the FP32 upper bound hi32 or the exact minimum hi64
__device__ __forceinline__ void dt32_cell(const DevMesh &d, int i, float &hi32, double &hi64) {
  float v, e;
  double x;
  if (local_dt32(d, i, v, e, x)) {
    d.dt32[i] = v;
    d.dteps[i] = e;
    hi32 = fminf(hi32, __fmul_ru(v, __fadd_ru(1.0f, e)));
  } else {
    d.dteps[i] = 0.0f;
    hi64 = fmin(hi64, x);
  }
}

// pass 2 of one cell: exact if its lower bound reaches the smallest upper
// bound hi (hi_rd: hi rounded down to FP32), so that it can hold the
// minimum; lowers m by its exact value then
__device__ __forceinline__ void dt_min_exact_cell(const DevMesh &d, int i, float e, float v, double hi,
                                                  float hi_rd, double &m) {
  if (e > 0.0f) {
    if (__fmul_rd(v, __fsub_rd(1.0f, e)) <= hi_rd) {
      m = fmin(m, local_dt_of(d, i));
      d.dteps[i] = 0.0f;
    }
  } else {
    const double dt = d.dt[i];
    if (dt <= hi) m = fmin(m, dt);
  }
}

// pass 1: estimates and the smallest upper bound
__global__ void __launch_bounds__(256) k_dt32(DevMesh d) {
  float hi32 = __int_as_float(0x7f800000);
  double hi64 = __longlong_as_double(0x7ff0000000000000LL);
  pdl_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x)
    dt32_cell(d, i, hi32, hi64);
  block_min_to(fmin((double)hi32, hi64), d.dthi_bits);
  pdl_trigger();
}

// a cell's estimate and its bound for the passes below, DT_UNROLL cells per
// thread at a time: both loads of every cell issued before any is used, so
// a thread keeps 2 x DT_UNROLL loads in flight instead of waiting on the
// bound, then on the estimate, cell after cell
#define DT_UNROLL 4
__device__ __forceinline__ void load_estimates(const DevMesh &d, int i0, int stride, float e[DT_UNROLL],
                                               float v[DT_UNROLL]) {
#pragma unroll
  for (int u = 0; u < DT_UNROLL; ++u) {
    const int i = i0 + u * stride;
    e[u] = i < d.N ? d.dteps[i] : 0.0f;
    v[u] = i < d.N ? d.dt32[i] : 0.0f;
  }
}

// pass 2: every cell that can hold the minimum (lower bound <= the smallest
// upper bound) is made exact; dt_min = the exact minimum over them (a
// minimum: the same in any order)
__global__ void __launch_bounds__(256) k_dt_min_exact(DevMesh d) {
  pdl_wait();
  const double hi = __longlong_as_double((long long)*d.dthi_bits);
  const float hi_rd = __double2float_rd(hi);
  double m = __longlong_as_double(0x7ff0000000000000LL);
  const int stride = gridDim.x * blockDim.x;
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < d.N; i0 += DT_UNROLL * stride) {
    float e[DT_UNROLL], v[DT_UNROLL];
    load_estimates(d, i0, stride, e, v);
#pragma unroll
    for (int u = 0; u < DT_UNROLL; ++u)
      if (i0 + u * stride < d.N) dt_min_exact_cell(d, i0 + u * stride, e[u], v[u], hi, hi_rd, m);
  }
  block_min_to(m, d.dtmin_bits);
  pdl_trigger();
}

// the thresholds of the level rule, t[k] = 2^k dt_min for k < L, and t[k]
// rounded up to FP32, filled once per block (every thread calls it)
struct LevelRule {
  double t[FV_MAXL];
  float tu[FV_MAXL];
};
__device__ __forceinline__ void level_rule_fill(LevelRule &r, const DevMesh &d) {
  if (threadIdx.x < d.L) {
    const double t = ldexp(__longlong_as_double((long long)*d.dtmin_bits), (int)threadIdx.x);
    r.t[threadIdx.x] = t;
    r.tu[threadIdx.x] = __double2float_ru(t);
  }
  __syncthreads();
}

// k_i = max{k <= L-1 : 2^k dt_min <= dt_i}, taken on the exact value, or on
// the estimate's interval when no threshold falls inside it
__device__ __forceinline__ int8_t level0_certified_of(const DevMesh &d, const LevelRule &r, int i, float e,
                                                     float v) {
  if (e > 0.0f) {
    const float lo = __fmul_rd(v, __fsub_rd(1.0f, e)), hi = __fmul_ru(v, __fadd_ru(1.0f, e));
    int klo = 0, khi = 0;
    for (int k = 1; k < d.L; ++k) {
      klo += r.tu[k] <= lo;
      khi += r.tu[k] <= hi;
    }
    if (klo == khi) return (int8_t)klo;
    local_dt_of(d, i);
    d.dteps[i] = 0.0f;
  }
  const double dt = d.dt[i];
  int k = 0;
  while (k + 1 < d.L && r.t[k + 1] <= dt) ++k;
  return (int8_t)k;
}

__global__ void __launch_bounds__(256) k_levels0_certified(DevMesh d) {
  __shared__ LevelRule r;
  pdl_wait();
  if (blockIdx.x == 0 && threadIdx.x < FV_MAXL) d.sweep_changed[threadIdx.x] = 0;
  level_rule_fill(r, d);
  const int stride = gridDim.x * blockDim.x;
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < d.N; i0 += DT_UNROLL * stride) {
    float e[DT_UNROLL], v[DT_UNROLL];
    load_estimates(d, i0, stride, e, v);
#pragma unroll
    for (int u = 0; u < DT_UNROLL; ++u)
      if (i0 + u * stride < d.N) d.lev_tmp[i0 + u * stride] = level0_certified_of(d, r, i0 + u * stride, e[u], v[u]);
  }
  pdl_trigger();
}

// one Jacobi sweep of k_i <- min(k_i, 1 + min_j k_j); L-1 sweeps reach the
// fixed point (the result is min_j (k0_j + graph distance), and k0 <= L-1)
__device__ __forceinline__ int8_t smooth_of(const DevMesh &d, const int8_t *src, int i) {
  int k = src[i];
  int4 nb4 = d.cnb4[i];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int nb = nbr_of(nb4, j);
    if (nb >= 0) k = min(k, src[nb] + 1);
  }
  return (int8_t)k;
}

// Sweep number sw.  A sweep that lowers no level has reached the fixed point
// and written it to dst, so src and dst both hold it: every later sweep
// returns at once (sweep_changed is cleared by k_levels0_certified).
__global__ void __launch_bounds__(256) k_smooth(DevMesh d, const int8_t *__restrict__ src,
                                                int8_t *__restrict__ dst, int sw) {
  pdl_wait();
  if (sw == 0 || d.sweep_changed[sw - 1]) {
    bool lowered = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x) {
      const int8_t k = smooth_of(d, src, i);
      lowered |= k != src[i];
      dst[i] = k;
    }
    if (__syncthreads_or(lowered) && threadIdx.x == 0) d.sweep_changed[sw] = 1;
  }
  pdl_trigger();
}

// cell sort key: 2 level + (1 unless a neighbour is one level finer), so the
// cells a phase touches are contiguous: levels <= tau followed by the
// level-(tau+1) cells next to level tau.  Also stored: the mask of the faces
// whose neighbour is finer (the corrector update takes their accumulated
// integrals) and, in the FP32-flux mode, the cycle's level in the cell's FP32
// state record (read with the state, so the phase kernels need no separate
// level lookup).
__device__ __forceinline__ int cell_key_store(const DevMesh &d, int i) {
  const int k = d.lev[i];
  unsigned finer = 0;
  int4 nb4 = d.cnb4[i];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int nb = nbr_of(nb4, j);
    if (nb >= 0 && d.lev[nb] < k) finer |= 1u << j;
  }
  const int key = 2 * k + (finer ? 0 : 1);
  d.ckey[i] = (uint8_t)key;
  d.cmask[i] = (uint8_t)finer;
  // written only where it changed (a few cells per thousand a cycle), so
  // the other records are read here but not written back
  if (d.Un32) {
    float *lv = d.Un32 + (size_t)i * REC_U32 + 5;
    if (*lv != (float)k) *lv = (float)k;
  }
  return key;
}

// face level = min of the two cell levels; faces sort by it
__device__ __forceinline__ int face_key_of(const DevMesh &d, int f) {
  int2 fc = d.fcell[f];
  int a = d.lev[fc.x];
  int k = fc.y >= 0 ? min(a, (int)d.lev[fc.y]) : a;
  d.flev[f] = (int8_t)k;
  d.fkey[f] = (uint8_t)k;
  return k;
}

// ---- stable counting sort of small keys (< 16 buckets), in tiles of
// SORT_TILE (batches) or SORT_TILE1 (one mesh) items
#define SORT_TILE 1024
#define SORT_THREADS 256
// items per tile of one large mesh's sort (from SORT_LARGE_CELLS cells):
// larger tiles, fewer (bucket, tile) counts for the single-block scan (at
// 80M cells, 1024-item tiles made the scan a millisecond per cycle); a
// smaller mesh keeps SORT_TILE, which fills the GPU with more blocks
#define SORT_TILE1 8192
#define SORT_LARGE_CELLS (1 << 23)

// per-tile bucket counts -> cnt[bucket * nblk + tile]
__device__ __forceinline__ void sort_hist_tile(const uint8_t *__restrict__ key, int n, int nb, int *cnt,
                                               int tile, int nblk) {
  __shared__ int h[16];
  if (threadIdx.x < 16) h[threadIdx.x] = 0;
  __syncthreads();
  int base = tile * SORT_TILE;
  for (int r = 0; r < SORT_TILE / SORT_THREADS; ++r) {
    int i = base + r * SORT_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[key[i]], 1);
  }
  __syncthreads();
  if (threadIdx.x < nb) cnt[threadIdx.x * nblk + tile] = h[threadIdx.x];
}


// exclusive scan over the bucket-major (bucket, tile) counts by one block of
// 1024 threads; also writes the bucket offsets off[0..nb]
__device__ __forceinline__ void sort_scan_block(int *cnt, int total, int nblk, int nb, int *off) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < total; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < total ? cnt[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffff, x, o);
      if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) warp_sums[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      int s = warp_sums[threadIdx.x];
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffff, s, o);
        if (threadIdx.x >= o) s += y;
      }
      warp_sums[threadIdx.x] = s;
    }
    __syncthreads();
    int warp_prefix = (threadIdx.x >= 32) ? warp_sums[(threadIdx.x >> 5) - 1] : 0;
    int excl = carry + warp_prefix + x - v;
    if (i < total) {
      cnt[i] = excl;
      if (i % nblk == 0) off[i / nblk] = excl;
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[nb] = carry;
}


// what a list entry carries: the item and, for cells, its faces, neighbours
// and own | finer bits; for faces, its two cells
template <bool FACES>
__device__ __forceinline__ void emit_entry(const DevMesh &d, int i, int pos) {
  if (FACES) {
    d.fl[pos] = i;
    d.flc[pos] = d.fcell[i];
  } else {
    d.cl[pos] = i;
    d.clf[pos] = d.cf4[i];
    d.cln[pos] = d.cnb4[i];
    d.clb[pos] = (uint8_t)(d.cown[i] | (d.cmask[i] << 4));
  }
}

// stable scatter of one tile: lanes with equal keys rank in lane (= item)
// order, warps in order, earlier rounds first
template <bool FACES, int TILE = SORT_TILE>
__device__ __forceinline__ void sort_scatter_tile(const DevMesh &d, const uint8_t *__restrict__ key, int n,
                                                  int nb, const int *__restrict__ cnt, int tile, int nblk) {
  __shared__ int wcount[SORT_THREADS / 32][16];
  __shared__ int run[16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 16) run[threadIdx.x] = threadIdx.x < nb ? cnt[threadIdx.x * nblk + tile] : 0;
  int base = tile * TILE;
  for (int r = 0; r < TILE / SORT_THREADS; ++r) {
    int i = base + r * SORT_THREADS + threadIdx.x;
    int k = i < n ? (int)key[i] : -1;
    if (lane < 16) wcount[warp][lane] = 0;
    __syncthreads();
    unsigned mask = __match_any_sync(0xffffffff, k);
    int rank = __popc(mask & ((1u << lane) - 1));
    if (k >= 0 && rank == 0) wcount[warp][k] = __popc(mask);
    __syncthreads();
    if (k >= 0) {
      int pre = run[k];
      for (int w = 0; w < warp; ++w) pre += wcount[w][k];
      emit_entry<FACES>(d, i, pre + rank);
    }
    __syncthreads();
    if (threadIdx.x < 16) {
      int s = 0;
      for (int w = 0; w < SORT_THREADS / 32; ++w) s += wcount[w][threadIdx.x];
      run[threadIdx.x] += s;
    }
    __syncthreads();
  }
}


// One mesh's cell and face sorts share each launch: the key computation and
// the per-tile counts (tiles 0..nc-1 are cells, the rest faces), the two
// scans (block 0 cells, block 1 faces), the two stable scatters.  The cell
// counts sit at sort_cnt[0 .. 2L nc), the face counts after them.
template <int TILE>
__global__ void __launch_bounds__(SORT_THREADS) k_keys_hist(DevMesh d, int nc, int nf) {
  __shared__ int h[16];
  pdl_wait();
  if (threadIdx.x < 16) h[threadIdx.x] = 0;
  __syncthreads();
  const bool faces = (int)blockIdx.x >= nc;
  const int tile = faces ? blockIdx.x - nc : blockIdx.x, n = faces ? d.F : d.N;
  for (int r = 0; r < TILE / SORT_THREADS; ++r) {
    const int i = tile * TILE + r * SORT_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[faces ? face_key_of(d, i) : cell_key_store(d, i)], 1);
  }
  __syncthreads();
  if (!faces && threadIdx.x < 2 * d.L) d.sort_cnt[threadIdx.x * nc + tile] = h[threadIdx.x];
  if (faces && threadIdx.x < d.L) d.sort_cnt[2 * d.L * nc + threadIdx.x * nf + tile] = h[threadIdx.x];
  pdl_trigger();
}

__global__ void __launch_bounds__(1024) k_sort_scan2(DevMesh d, int nc, int nf) {
  pdl_wait();
  if (blockIdx.x == 0)
    sort_scan_block(d.sort_cnt, 2 * d.L * nc, nc, 2 * d.L, d.coff);
  else
    sort_scan_block(d.sort_cnt + 2 * d.L * nc, d.L * nf, nf, d.L, d.foff);
  pdl_trigger();
}

template <int TILE>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_scatter2(DevMesh d, int nc, int nf) {
  pdl_wait();
  if ((int)blockIdx.x < nc)
    sort_scatter_tile<false, TILE>(d, d.ckey, d.N, 2 * d.L, d.sort_cnt, blockIdx.x, nc);
  else
    sort_scatter_tile<true, TILE>(d, d.fkey, d.F, d.L, d.sort_cnt + 2 * d.L * nc, blockIdx.x - nc, nf);
  pdl_trigger();
}

// ---- batched level assignment: block b of a grid covering every instance's
// tiles maps to (instance, tile) through a prefix over per-instance tile
// counts; blocks of instances that do not start a cycle return at once
struct MultiTiles {
  const DevMesh *ms;
  const int *active;  // per instance
  const int *tpref;   // n+1 prefix of tile counts (cells or faces, 1024 per tile)
  int n;
};

__device__ __forceinline__ bool tile_of(const MultiTiles &a, int &inst, int &tile) {
  __shared__ int s_inst, s_tile;
  if (threadIdx.x == 0) {
    int lo = 0, hi = a.n;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (a.tpref[mid] <= (int)blockIdx.x) lo = mid; else hi = mid;
    }
    s_inst = lo;
    s_tile = (int)blockIdx.x - a.tpref[lo];
  }
  __syncthreads();
  inst = s_inst;
  tile = s_tile;
  return a.active[inst] != 0 && (int)blockIdx.x < a.tpref[a.n];
}

__global__ void k_init_min_multi(const DevMesh *ms, const int *active, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && active[i]) {
    *ms[i].dtmin_bits = 0x7ff0000000000000ULL;
    *ms[i].dthi_bits = 0x7ff0000000000000ULL;
  }
}

// the certified local step of a batch: pass 1 (op 0) and pass 2 (op 1) per
// instance, as k_dt32 and k_dt_min_exact do for one mesh
__global__ void __launch_bounds__(256) k_dt_multi(MultiTiles a, int op) {
  int inst, tile;
  if (!tile_of(a, inst, tile)) return;
  const DevMesh &d = a.ms[inst];
  double m = __longlong_as_double(0x7ff0000000000000LL);
  const int end = min(d.N, (tile + 1) * SORT_TILE);
  if (op == 0) {
    float hi32 = __int_as_float(0x7f800000);
    for (int i = tile * SORT_TILE + threadIdx.x; i < end; i += blockDim.x) dt32_cell(d, i, hi32, m);
    block_min_to(fmin((double)hi32, m), d.dthi_bits);
  } else {
    const double hi = __longlong_as_double((long long)*d.dthi_bits);
    const float hi_rd = __double2float_rd(hi);
    for (int i = tile * SORT_TILE + threadIdx.x; i < end; i += blockDim.x)
      dt_min_exact_cell(d, i, d.dteps[i], d.dt32[i], hi, hi_rd, m);
    block_min_to(m, d.dtmin_bits);
  }
}

// op 0: levels0; 1: copy lev_tmp -> lev; 2: sweep lev_tmp -> lev;
// 3: sweep lev -> lev_tmp; 4: cell keys
__global__ void __launch_bounds__(256) k_cells_multi(MultiTiles a, int op) {
  int inst, tile;
  if (!tile_of(a, inst, tile)) return;
  const DevMesh &d = a.ms[inst];
  __shared__ LevelRule r;
  if (op == 0) level_rule_fill(r, d);
  for (int i = tile * SORT_TILE + threadIdx.x; i < min(d.N, (tile + 1) * SORT_TILE); i += blockDim.x) {
    if (op == 0) d.lev_tmp[i] = level0_certified_of(d, r, i, d.dteps[i], d.dt32[i]);
    else if (op == 1) d.lev[i] = d.lev_tmp[i];
    else if (op == 2) d.lev[i] = smooth_of(d, d.lev_tmp, i);
    else if (op == 3) d.lev_tmp[i] = smooth_of(d, d.lev, i);
    else cell_key_store(d, i);
  }
}

__global__ void __launch_bounds__(256) k_face_keys_multi(MultiTiles a) {
  int inst, tile;
  if (!tile_of(a, inst, tile)) return;
  const DevMesh &d = a.ms[inst];
  for (int f = tile * SORT_TILE + threadIdx.x; f < min(d.F, (tile + 1) * SORT_TILE); f += blockDim.x)
    face_key_of(d, f);
}

// faces = 0: cell keys (2L buckets) into cl/coff; 1: face keys (L) into fl/foff
__global__ void __launch_bounds__(SORT_THREADS) k_sort_hist_multi(MultiTiles a, int faces) {
  int inst, tile;
  if (!tile_of(a, inst, tile)) return;
  const DevMesh &d = a.ms[inst];
  int n = faces ? d.F : d.N;
  sort_hist_tile(faces ? d.fkey : d.ckey, n, faces ? d.L : 2 * d.L, d.sort_cnt, tile,
                 (n + SORT_TILE - 1) / SORT_TILE);
}

__global__ void __launch_bounds__(1024) k_sort_scan_multi(const DevMesh *ms, const int *active, int faces) {
  if (!active[blockIdx.x]) return;
  const DevMesh &d = ms[blockIdx.x];
  int n = faces ? d.F : d.N;
  int nb = faces ? d.L : 2 * d.L;
  int nblk = (n + SORT_TILE - 1) / SORT_TILE;
  sort_scan_block(d.sort_cnt, nb * nblk, nblk, nb, faces ? d.foff : d.coff);
}

__global__ void __launch_bounds__(SORT_THREADS) k_sort_scatter_multi(MultiTiles a, int faces) {
  int inst, tile;
  if (!tile_of(a, inst, tile)) return;
  const DevMesh &d = a.ms[inst];
  int n = faces ? d.F : d.N;
  if (faces)
    sort_scatter_tile<true>(d, d.fkey, n, d.L, d.sort_cnt, tile, (n + SORT_TILE - 1) / SORT_TILE);
  else
    sort_scatter_tile<false>(d, d.ckey, n, 2 * d.L, d.sort_cnt, tile, (n + SORT_TILE - 1) / SORT_TILE);
}

// ------------------------------------------------------ state at a time --
// whether some level of the phase reads its predicted (or interpolated)
// state
__device__ __forceinline__ bool reads_predicted(const PhaseLevels &pl) {
  bool any = false;
#pragma unroll
  for (int j = 0; j < FV_MAXL; ++j) any |= pl.mode[j] != 0;
  return any;
}

// the state of cell c at the phase time (FP64 mode); returns its level
__device__ __forceinline__ int load_state(const DevMesh &d, const PhaseLevels &pl, int c,
                                          double U[5], bool = false) {
  const size_t N = d.N;
  int k = d.lev[c];
  int mode = pl.mode[k];
  if (mode == 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) U[q] = d.Un[q * N + c];
  } else if (mode == 1) {
#pragma unroll
    for (int q = 0; q < 5; ++q) U[q] = d.Us[q * N + c];
  } else {
    double w = pl.w[k];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      double a = d.Un[q * N + c], b = d.Us[q * N + c];
      U[q] = a + w * (b - a);
    }
  }
  return k;
}

// FP32-flux mode: the state at the phase time from the FP32 records of U^n
// and of the predicted state; the record of U^n carries the cell's level.
// With `both` (the phase reads some level's predicted state) the predicted
// record is loaded together with U^n rather than after its level is known.
// Returns the level.
__device__ __forceinline__ int load_state(const DevMesh &d, const PhaseLevels &pl, int c,
                                          float U[5], bool both = false) {
  float a[REC_U32], b[REC_U32];
  ldrec<REC_U32>(d.Un32 + (size_t)c * REC_U32, a);
  if (both) ldrec<REC_U32>(d.Us32 + (size_t)c * REC_U32, b);
  const int k = (int)a[5];
  const int mode = pl.mode[k];
  if (mode == 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) U[q] = a[q];
  } else {
    if (!both) ldrec<REC_U32>(d.Us32 + (size_t)c * REC_U32, b);
    if (mode == 1) {
#pragma unroll
      for (int q = 0; q < 5; ++q) U[q] = b[q];
    } else {
      float w = (float)pl.w[k];
#pragma unroll
      for (int q = 0; q < 5; ++q) U[q] = a[q] + w * (b[q] - a[q]);
    }
  }
  return k;
}

__device__ __forceinline__ void to_prim(const double U[5], double gm1, double W[5]) {
  prim_fp64(U, gm1, W);
}
__device__ __forceinline__ void to_prim(const float U[5], double gm1, float W[5]) {
  cons_to_prim(U, (float)gm1, W);
}

// record arrays of the flux type
__device__ __forceinline__ const double *grec(const DevMesh &d, double) { return d.G; }
__device__ __forceinline__ const float *grec(const DevMesh &d, float) { return d.G32; }
__device__ __forceinline__ double *grec_w(const DevMesh &d, double) { return d.G; }
__device__ __forceinline__ float *grec_w(const DevMesh &d, float) { return d.G32; }
__device__ __forceinline__ const double *lswrec(const DevMesh &d, double) { return d.lsw; }
__device__ __forceinline__ const float *lswrec(const DevMesh &d, float) { return d.lsw32; }
__device__ __forceinline__ const double *georec(const DevMesh &d, double) { return d.fgeo; }
__device__ __forceinline__ const float *georec(const DevMesh &d, float) { return d.fgeo32; }

// primitives of the cell at list position idx at the phase time into its W
// record: FP64 (FP64 mode) or FP32 (FP32-flux mode, no FP64 work)
template <typename WT>
__device__ __forceinline__ void prim_item(const DevMesh &d, const PhaseLevels &pl, int idx) {
  int i = d.cl[idx];
  WT U[5], Wt[REC_W];
  load_state(d, pl, i, U);
  to_prim(U, d.gamma - 1.0, Wt);
#pragma unroll
  for (int q = 5; q < REC_W; ++q) Wt[q] = WT(0);
  strec<REC_W>((WT *)d.W + (size_t)i * REC_W, Wt);
}

// least-squares gradient of the primitives of cell i, whose own primitives
// are Wi: g = sum_j w_j (W_nb(j) - W_i), ghost states on boundary faces.
// FP64 mode: neighbours from the W records the primitives kernel wrote;
// FP32-flux mode: from their states at the phase time (`both`: load the
// predicted record together with U^n).
// nb4: the cell's neighbours; cfp: where its faces are (read only for a
// wall face's normal)
template <typename T>
__device__ __forceinline__ void lsq_grad(const DevMesh &d, const PhaseLevels &pl, bool both, int i,
                                         const T Wi[5], T g[REC_G], const int4 nb4, const int4 *cfp) {
  constexpr bool INLINE_W = sizeof(T) == 4;
  const T *W = (const T *)d.W;
  const T *fgeo = georec(d, T(0));
  const double gm1 = d.gamma - 1.0;
  T w[REC_LSW];
  ldrec<REC_LSW>(lswrec(d, T(0)) + (size_t)i * REC_LSW, w);
#pragma unroll
  for (int q = 0; q < REC_G; ++q) g[q] = T(0);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int nb = nbr_of(nb4, j);
    T Wn[REC_W];
    if (nb >= 0) {
      if (INLINE_W) {
        T U[5];
        load_state(d, pl, nb, U, both);
        to_prim(U, gm1, Wn);
      } else {
        ldrec<REC_W>(W + (size_t)nb * REC_W, Wn);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 5; ++q) Wn[q] = Wi[q];
      if (nb == -FV_BC_WALL) {
        const T *gf = fgeo + (size_t)nbr_of(*cfp, j) * REC_FG;
        T n0 = gf[0], n1 = gf[1], n2 = gf[2];
        T un = (Wi[1] * n0 + Wi[2] * n1) + Wi[3] * n2;
        Wn[1] = Wi[1] - (T(2) * un) * n0;
        Wn[2] = Wi[2] - (T(2) * un) * n1;
        Wn[3] = Wi[3] - (T(2) * un) * n2;
      }
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      T dd = Wn[c] - Wi[c];
      g[3 * c] += w[3 * j] * dd;
      g[3 * c + 1] += w[3 * j + 1] * dd;
      g[3 * c + 2] += w[3 * j + 2] * dd;
    }
  }
}

// gradient item of the cell at list position idx.  FP64 mode: from the W
// records the primitives kernel wrote.  FP32-flux mode (INLINE_W): the
// primitives of the cell and of its neighbours are computed here from their
// states at the phase time, and the cell's own primitives are stored in its W
// record for the flux kernel, with its level in slot 5; there is no separate
// primitives kernel.  Both records are stored after every load.
template <typename T>
__device__ __forceinline__ void grad_cell(const DevMesh &d, const PhaseLevels &pl, int i, const int4 nb4,
                                          const int4 *cfp) {
  constexpr bool INLINE_W = sizeof(T) == 4;
  const bool both = INLINE_W && reads_predicted(pl);
  T Wi[REC_W], g[REC_G];
  if (INLINE_W) {
    T U[5];
    const int k = load_state(d, pl, i, U, both);
    to_prim(U, d.gamma - 1.0, Wi);
    Wi[5] = T(k);
#pragma unroll
    for (int q = 6; q < REC_W; ++q) Wi[q] = T(0);
  } else {
    ldrec<REC_W>((const T *)d.W + (size_t)i * REC_W, Wi);
  }
  lsq_grad<T>(d, pl, both, i, Wi, g, nb4, cfp);
  strec<REC_G>(grec_w(d, T(0)) + (size_t)i * REC_G, g);
  if (INLINE_W) strec<REC_W>((T *)d.W + (size_t)i * REC_W, Wi);
}

// the cell at list position idx, its neighbours from the list entry
template <typename T>
__device__ __forceinline__ void grad_item(const DevMesh &d, const PhaseLevels &pl, int idx) {
  grad_cell<T>(d, pl, d.cl[idx], d.cln[idx], d.clf + idx);
}

// gradients (and, FP32-flux mode, primitives) of every cell by plain index:
// the hooks' pass, independent of the level-sorted lists
template <typename T>
__global__ void __launch_bounds__(256, 2) k_grad_all(DevMesh d, const __grid_constant__ PhaseLevels pl) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x)
    grad_cell<T>(d, pl, i, d.cnb4[i], d.cf4 + i);
}

// the learned starting guess of one face (warp-collective): where the
// two-rarefaction estimate shows a shock stronger than the packed gate, the
// network (on the tensor cores, run by the warp if any of its lanes needs it)
// gives either an absolute guess pbar e^y (target 0) or a factor e^(s(q) y)
// on the two-rarefaction guess (target 1).
// Elsewhere, and for invalid values, the solver keeps the two-rarefaction
// guess.
template <typename T>
__device__ __forceinline__ void mlp_guess(const uint32_t *__restrict__ sw, float gamma, const T WL[5],
                                          const T WR[5], const T n[3], T &gabs, T &gmul) {
  T unL = (WL[1] * n[0] + WL[2] * n[1]) + WL[3] * n[2];
  T unR = (WR[1] * n[0] + WR[2] * n[1]) + WR[3] * n[2];
  const float rL = (float)WL[0], uL = (float)unL, pL = (float)WL[4];
  const float rR = (float)WR[0], uR = (float)unR, pR = (float)WR[4];
  const float gate = __uint_as_float(sw[PK_GATE]);
  const float q = shock_strength(gamma, rL, uL, pL, rR, uR, pR);
  const bool use = gate < 0.0f || q > gate;
  gabs = T(0);
  gmul = T(1);
  if (!__any_sync(0xffffffffu, use)) return;
  float x[6];
  float pb = mlp_features<T>((T)gamma, WL[0], unL, WL[4], WR[0], unR, WR[4], x);
  float y = mlp_eval_warp(sw, x);
  if (!use) return;
  if (sw[PK_TARGET] == 0u) {
    gabs = (T)(pb * __expf(y));
  } else {
    float e = __expf(shock_scale(q) * y);
    if (e > 0.0f && e < 3.0e38f) gmul = (T)e;
  }
}

// FP32: the MUSCL-minmod reconstruction of both sides of an interior face
// with Blackwell's paired FP32 instructions (two independent multiplies or
// fused multiply-adds per instruction): each component's left and right
// gradient projections g_i.r and g_j.r, the limiter arguments 2 g.r - dW
// and the reconstructed values W_i + m/2, W_j - m/2 go pairwise; the
// limiter itself stays per side.  The same operations as the plain form
// (the projections accumulate x, then y, then z).
__device__ __forceinline__ void reconstruct_pair(const float Wi[], const float gi[], const float Wj[],
                                                 const float gj[], const float r[3], float WL[5],
                                                 float WR[5]) {
  const float2 r0 = make_float2(r[0], r[0]), r1 = make_float2(r[1], r[1]), r2 = make_float2(r[2], r[2]);
  const float2 two = make_float2(2.0f, 2.0f), half = make_float2(0.5f, -0.5f);
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    float2 g = __fmul2_rn(make_float2(gi[3 * c], gj[3 * c]), r0);
    g = __ffma2_rn(make_float2(gi[3 * c + 1], gj[3 * c + 1]), r1, g);
    g = __ffma2_rn(make_float2(gi[3 * c + 2], gj[3 * c + 2]), r2, g);
    const float dW = Wj[c] - Wi[c];
    const float2 a = __ffma2_rn(two, g, make_float2(-dW, -dW));
    const float2 m = make_float2(minmod(a.x, dW), minmod(a.y, dW));
    const float2 w = __ffma2_rn(half, m, make_float2(Wi[c], Wj[c]));
    WL[c] = w.x;
    WR[c] = w.y;
  }
}

// FP32, one side of an interior face with the operations of one lane of
// reconstruct_pair (explicit round-to-nearest products and fused
// multiply-adds, so that the result is bitwise the paired one): the value
// Wc + half * minmod(2 g.r - dW, dW), half = +1/2 (left), -1/2 (right)
__device__ __forceinline__ float reconstruct_side(float Wc, const float *g, const float r[3], float dW,
                                                  float half) {
  float gr = __fmul_rn(g[0], r[0]);
  gr = __fmaf_rn(g[1], r[1], gr);
  gr = __fmaf_rn(g[2], r[2], gr);
  const float a = __fmaf_rn(2.0f, gr, -dW);
  return __fmaf_rn(half, minmod(a, dW), Wc);
}

// the reconstructed inputs of face f's Riemann problem from the phase-time
// primitive and gradient records: WL, WR (a boundary face copies WL into WR),
// unit normal n and area A; fc = fcell[f], the face's cells.  Returns fc.y:
// the right cell, or minus the boundary tag.
template <typename T>
__device__ __forceinline__ int face_states(const DevMesh &d, const T *__restrict__ W,
                                           const T *__restrict__ Gr, const T *__restrict__ fgeo, int f,
                                           const int2 fc, T WL[5], T WR[5], T n[3], T &A) {
  const int L = fc.x, R = fc.y;
  T geo[REC_FG];
  ldrec<REC_FG>(fgeo + (size_t)f * REC_FG, geo);
  n[0] = geo[0];
  n[1] = geo[1];
  n[2] = geo[2];
  A = geo[3];
  const T r[3] = {geo[4], geo[5], geo[6]};
  T Wi[REC_W], gi[REC_G];
  ldrec<REC_W>(W + (size_t)L * REC_W, Wi);
  ldrec<REC_G>(Gr + (size_t)L * REC_G, gi);
  if (R >= 0) {
    T Wj[REC_W], gj[REC_G];
    ldrec<REC_W>(W + (size_t)R * REC_W, Wj);
    ldrec<REC_G>(Gr + (size_t)R * REC_G, gj);
    if constexpr (sizeof(T) == 4) {
      reconstruct_pair(Wi, gi, Wj, gj, r, WL, WR);
    } else {
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        T dW = Wj[c] - Wi[c];
        T gir = (gi[3 * c] * r[0] + gi[3 * c + 1] * r[1]) + gi[3 * c + 2] * r[2];
        T gjr = (gj[3 * c] * r[0] + gj[3 * c + 1] * r[1]) + gj[3 * c + 2] * r[2];
        WL[c] = Wi[c] + T(0.5) * minmod(T(2) * gir - dW, dW);
        WR[c] = Wj[c] - T(0.5) * minmod(T(2) * gjr - dW, dW);
      }
    }
  } else {
    // reconstruct toward the ghost (mirror image of the cell in the face)
    T Wg[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) Wg[c] = Wi[c];
    if (R == -FV_BC_WALL) {
      T un = (Wi[1] * n[0] + Wi[2] * n[1]) + Wi[3] * n[2];
#pragma unroll
      for (int e = 0; e < 3; ++e) Wg[1 + e] = Wi[1 + e] - (T(2) * un) * n[e];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      T dW = Wg[c] - Wi[c];
      T gir = (gi[3 * c] * r[0] + gi[3 * c + 1] * r[1]) + gi[3 * c + 2] * r[2];
      WL[c] = Wi[c] + T(0.5) * minmod(T(2) * gir - dW, dW);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) WR[c] = WL[c];
  }
  return R;
}

// face flux of face f: F A in FA[5].  Returns a nonzero status on Riemann
// failure.  With MLP the whole warp calls it together (the learned guess is
// warp-collective); a lane without a face passes f < 0 and gets nothing.
template <typename T, bool G14, bool MLP = false>
__device__ __forceinline__ int face_flux(const DevMesh &d, const GasT<T> &G, const T *__restrict__ W,
                                         const T *__restrict__ Gr, const T *__restrict__ fgeo, int f,
                                         const int2 fc, T FA[5], const uint32_t *sw = nullptr) {
  T WL[5], WR[5], n[3], A;
  int R = 0;
  if (!MLP || f >= 0) {
    R = face_states<T>(d, W, Gr, fgeo, f, fc, WL, WR, n, A);
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) WL[c] = WR[c] = c == 0 || c == 4 ? T(1) : T(0);
    n[0] = T(1);
    n[1] = n[2] = T(0);
    A = T(0);
  }
  T gabs = T(0), gmul = T(1);
  if (MLP) {
    __syncwarp();
    mlp_guess<T>(sw, (float)G.g, WL, WR, n, gabs, gmul);
    if (f < 0) return 0;
  }
  int it, rc;
  T Fx[5];
  if (R >= 0)
    rc = godunov_flux<T, G14, MLP>(G, WL, WR, n, Fx, it, gabs, gmul);
  else
    rc = boundary_flux<T, G14>(G, -R, WL, n, Fx, it);
#pragma unroll
  for (int c = 0; c < 5; ++c) FA[c] = Fx[c] * A;
  return rc;
}

// exact sign flip through the bit pattern (no floating-point instruction)
__device__ __forceinline__ double flip(double v, bool neg) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
}
__device__ __forceinline__ float flip(float v, bool neg) {
  return __int_as_float(__float_as_int(v) ^ ((int)neg << 31));
}

// stage 1 (predictor): the flux F1 A is stashed (FP32 in the FP32-flux mode,
// where it is an FP32 result of the FP32 flux).  stage 2 (corrector of
// `level` k): the step's flux time integral Phi = h_k (F1 A + F2 A), h_k =
// dt_k/2, is kept in units of h_k: Psi = F1 A + F2 A, formed in FP64 (in the
// FP32-flux mode each FP32 flux is widened first, so the sum is an FP64
// operation), and stored; the cells of level k take h_k once per cell in
// their update.  On a level interface (iface) Phi is added to ACC[f], the
// coarse side's integral, in the coarse level's units h_{k+1} = 2 h_k (the
// level rule keeps neighbours within one level): ACC += Psi / 2.  On a
// boundary face (bnd) Phi itself goes to BND[f] (the conservation ledger,
// which spans cycles and so stays in time units).
template <typename T>
__device__ __forceinline__ void flux_store(const DevMesh &d, int stage, int level, int f, const T FAt[5],
                                           bool iface, bool bnd) {
  const bool f32 = sizeof(T) == 4;
  if (stage == 1) {
    if (f32) {
      float v[REC_FA32] = {(float)FAt[0], (float)FAt[1], (float)FAt[2], (float)FAt[3], (float)FAt[4], 0.f, 0.f, 0.f};
      strec<REC_FA32>(d.FA32 + (size_t)f * REC_FA32, v);
    } else {
      double v[REC_FA] = {(double)FAt[0], (double)FAt[1], (double)FAt[2], (double)FAt[3], (double)FAt[4], 0.0};
      strec<REC_FA>(d.FA + (size_t)f * REC_FA, v);
    }
    return;
  }
  double psi[REC_FA];
  if (f32) {
    float a[REC_FA32];
    ldrec<REC_FA32>(d.FA32 + (size_t)f * REC_FA32, a);
#pragma unroll
    for (int c = 0; c < 5; ++c) psi[c] = (double)a[c] + (double)FAt[c];
  } else {
    double a[REC_FA];
    ldrec<REC_FA>(d.FA + (size_t)f * REC_FA, a);
#pragma unroll
    for (int c = 0; c < 5; ++c) psi[c] = a[c] + (double)FAt[c];
  }
  psi[5] = 0.0;
  strec<REC_FA>(d.FA + (size_t)f * REC_FA, psi);
  if (iface || bnd) {
    double *dst = (iface ? d.ACC : d.BND) + (size_t)f * REC_FA;
    // Psi / 2 in the coarse side's units, or h_k Psi in time units
    const double w = iface ? 0.5 : scale2(__longlong_as_double((long long)*d.dtmin_bits), level - 1);
    double acc[REC_FA];
    ldrec<REC_FA>(dst, acc);
#pragma unroll
    for (int c = 0; c < 5; ++c) acc[c] = fma(w, psi[c], acc[c]);
    strec<REC_FA>(dst, acc);
  }
}

// flux item of the face at list position idx, from the phase's primitive and
// gradient records
template <typename T, bool G14, bool MLP = false>
__device__ __forceinline__ void flux_item(const DevMesh &d, const GasT<T> &G, int stage, int level,
                                          int idx, const uint32_t *sw = nullptr) {
  const bool f32 = sizeof(T) == 4;
  int f = (!MLP || idx >= 0) ? d.fl[idx] : -1;
  const int2 fc = (!MLP || idx >= 0) ? d.flc[idx] : make_int2(0, 0);  // the entry's cells
  T FAt[5];
  int rc = face_flux<T, G14, MLP>(d, G, (const T *)d.W, grec(d, T(0)), georec(d, T(0)), f, fc, FAt, sw);
  if (MLP && f < 0) return;
  if (rc) atomicOr(d.status, FV_STATUS_RIEMANN);
  bool iface = false, bnd = false;
  if (stage != 1) {
    // the FP32-flux mode has the cells' levels in slot 5 of the W records
    // the face states were just read from
    const T *Wr = (const T *)d.W;
    iface = fc.y >= 0 && (f32 ? Wr[(size_t)fc.x * REC_W + 5] != Wr[(size_t)fc.y * REC_W + 5]
                              : d.lev[fc.x] != d.lev[fc.y]);
    bnd = fc.y < 0;
  }
  flux_store<T>(d, stage, level, f, FAt, iface, bnd);
}

// FP32-flux mode, phases with few faces (fused_phase): the Riemann inputs of
// face f with both cells' primitives and gradients computed here from the
// states at the phase time -- the arithmetic of the gradient kernel followed
// by that of face_states -- so the phase needs no gradient records.  Returns
// fcell.y; iface: the two cells are on different levels.
__device__ __forceinline__ int face_states_fused(const DevMesh &d, const PhaseLevels &pl, bool both, int f,
                                                 float WL[5], float WR[5], float n[3], float &A,
                                                 bool &iface) {
  int2 fc = d.fcell[f];
  const int L = fc.x, R = fc.y;
  float geo[REC_FG];
  ldrec<REC_FG>(d.fgeo32 + (size_t)f * REC_FG, geo);
  n[0] = geo[0];
  n[1] = geo[1];
  n[2] = geo[2];
  A = geo[3];
  const float r[3] = {geo[4], geo[5], geo[6]};
  const double gm1 = d.gamma - 1.0;
  float U[5], Wi[5], g[REC_G];
  const int kL = load_state(d, pl, L, U, both);
  to_prim(U, gm1, Wi);
  lsq_grad<float>(d, pl, both, L, Wi, g, d.cnb4[L], d.cf4 + L);
  iface = false;
  if (R >= 0) {
    float Wj[5];
    const int kR = load_state(d, pl, R, U, both);
    to_prim(U, gm1, Wj);
    iface = kL != kR;
#pragma unroll
    for (int c = 0; c < 5; ++c) WL[c] = reconstruct_side(Wi[c], g + 3 * c, r, Wj[c] - Wi[c], 0.5f);
    lsq_grad<float>(d, pl, both, R, Wj, g, d.cnb4[R], d.cf4 + R);
#pragma unroll
    for (int c = 0; c < 5; ++c) WR[c] = reconstruct_side(Wj[c], g + 3 * c, r, Wj[c] - Wi[c], -0.5f);
  } else {
    float Wg[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) Wg[c] = Wi[c];
    if (R == -FV_BC_WALL) {
      float un = (Wi[1] * n[0] + Wi[2] * n[1]) + Wi[3] * n[2];
#pragma unroll
      for (int e = 0; e < 3; ++e) Wg[1 + e] = Wi[1 + e] - (2.0f * un) * n[e];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      float dW = Wg[c] - Wi[c];
      float gir = (g[3 * c] * r[0] + g[3 * c + 1] * r[1]) + g[3 * c + 2] * r[2];
      WL[c] = Wi[c] + 0.5f * minmod(2.0f * gir - dW, dW);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) WR[c] = WL[c];
  }
  return R;
}

template <bool G14>
__device__ __forceinline__ void flux_item_fused(const DevMesh &d, const GasT<float> &G, int stage, int level,
                                                const PhaseLevels &pl, bool both, int idx) {
  const int f = d.fl[idx];
  float WL[5], WR[5], n[3], A, Fx[5], FAt[5];
  bool iface;
  const int R = face_states_fused(d, pl, both, f, WL, WR, n, A, iface);
  int it, rc;
  if (R >= 0)
    rc = godunov_flux<float, G14, false>(G, WL, WR, n, Fx, it, 0.0f, 1.0f);
  else
    rc = boundary_flux<float, G14>(G, -R, WL, n, Fx, it);
#pragma unroll
  for (int c = 0; c < 5; ++c) FAt[c] = Fx[c] * A;
  if (rc) atomicOr(d.status, FV_STATUS_RIEMANN);
  flux_store<float>(d, stage, level, f, FAt, iface, R < 0);
}

// per-cell gather over its 4 faces in local order (deterministic, no
// atomics), signs applied by flipping bits:
//  stage 1: U* = U^n + dt_k (-S/V), S = sum sigma F1 A.  In the FP32-flux mode
//           the predictor is all FP32 (U* only feeds fluxes).
//  stage 2 (level k): U^{n+1} = U^n - (h_k/V) S, S = sum sigma Psi in FP64
//           (the flux time integrals in units of h_k = dt_k/2), where faces
//           to finer neighbours contribute (and reset) their accumulated
//           integral, kept in the same units; the FP32 shadow of U^n is
//           refreshed.
// Positivity is checked by the next level assignment and on demand
// (fv_status), not here.
// Order 1 (the paper's order), the corrector of the cell at list position
// idx, of `level` k: the
// provisional end state U^n - (h_k/V) S, S = sum sigma psi over the cell's
// faces in units of h_k = dt_k/2, psi = Psi on its own-level faces (and
// faces to coarser neighbours) and the provisional dt_k F1 A = h_k (2 F1 A)
// on faces to finer neighbours, whose accumulators start from minus that
// value (the finer side adds its integrals to them, in the same units).
// The state goes to the FP64 predicted-state array (FP64 mode) or to UsD
// and the FP32 predicted record (FP32-flux mode), where the finer levels
// interpolate it.  Every load before the first store.
template <bool F32>
__device__ __forceinline__ void correct_cell(const DevMesh &d, int level, int idx) {
  const size_t N = d.N;
  const double hk = scale2(__longlong_as_double((long long)*d.dtmin_bits), level - 1);
  const int i = d.cl[idx];
  const unsigned bits = d.clb[idx];
  const unsigned own = bits & 15u, finer = bits >> 4;
  const int4 cf = d.clf[idx];
  double S[5];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int f = nbr_of(cf, j);
    const bool neg = !((own >> j) & 1u);
    double v[REC_FA];
    if ((finer >> j) & 1u) {
      if (F32) {
        float a[REC_FA32];
        ldrec<REC_FA32>(d.FA32 + (size_t)f * REC_FA32, a);
#pragma unroll
        for (int c = 0; c < 5; ++c) v[c] = 2.0 * (double)a[c];
      } else {
        ldrec<REC_FA>(d.FA + (size_t)f * REC_FA, v);
#pragma unroll
        for (int c = 0; c < 5; ++c) v[c] = 2.0 * v[c];
      }
    } else {
      ldrec<REC_FA>(d.FA + (size_t)f * REC_FA, v);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) S[c] = j == 0 ? flip(v[c], neg) : S[c] + flip(v[c], neg);
  }
  const double hV = hk * d.ivol[i];
  double u[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) u[c] = d.Un[c * N + i];
#pragma unroll
  for (int c = 0; c < 5; ++c) u[c] = u[c] - hV * S[c];
  double *Up = F32 ? d.UsD : d.Us;
#pragma unroll
  for (int c = 0; c < 5; ++c) Up[c * N + i] = u[c];
  if (F32) {
    float r[REC_U32];
#pragma unroll
    for (int c = 0; c < 5; ++c) r[c] = (float)u[c];
    r[5] = (float)level;
    r[6] = r[7] = 0.0f;
    strec<REC_U32>(d.Us32 + (size_t)i * REC_U32, r);
  }
  // the accumulators of the faces to finer neighbours start from minus the
  // provisional integral (re-read: the loads above must not wait on these)
  if (finer) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!((finer >> j) & 1u)) continue;
      const int f = nbr_of(cf, j);
      double p[REC_FA], acc[REC_FA];
      if (F32) {
        float a[REC_FA32];
        ldrec<REC_FA32>(d.FA32 + (size_t)f * REC_FA32, a);
#pragma unroll
        for (int c = 0; c < 5; ++c) p[c] = (double)a[c];
      } else {
        ldrec<REC_FA>(d.FA + (size_t)f * REC_FA, p);
      }
      ldrec<REC_FA>(d.ACC + (size_t)f * REC_FA, acc);
#pragma unroll
      for (int c = 0; c < 5; ++c) acc[c] = fma(-2.0, p[c], acc[c]);
      strec<REC_FA>(d.ACC + (size_t)f * REC_FA, acc);
    }
  }
}

// Order 1, the commit of the cell at list position idx at the end of its step (Alg. 2's intensive
// correction): U^{n+1} = Up - (h_k/V) sum sigma ACC over the faces to finer
// neighbours (ACC = their integral minus the provisional one, in units of
// the cell's h_k = dt_k/2), which are reset; a cell without finer
// neighbours takes its provisional state as it is.
template <bool F32>
__device__ __forceinline__ void commit_cell(const DevMesh &d, int idx) {
  const size_t N = d.N;
  const int i = d.cl[idx];
  const unsigned bits = d.clb[idx];
  const unsigned finer = bits >> 4;
  const double *Up = F32 ? d.UsD : d.Us;
  double u[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) u[c] = Up[c * N + i];
  if (finer) {
    const unsigned own = bits & 15u;
    const int4 cf = d.clf[idx];
    double S[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!((finer >> j) & 1u)) continue;
      const bool neg = !((own >> j) & 1u);
      double v[REC_FA];
      ldrec<REC_FA>(d.ACC + (size_t)nbr_of(cf, j) * REC_FA, v);
#pragma unroll
      for (int c = 0; c < 5; ++c) S[c] += flip(v[c], neg);
    }
    const double hV = scale2(__longlong_as_double((long long)*d.dtmin_bits), (int)d.lev[i] - 1) * d.ivol[i];
#pragma unroll
    for (int c = 0; c < 5; ++c) u[c] = u[c] - hV * S[c];
    const double z[REC_FA] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((finer >> j) & 1u) strec<REC_FA>(d.ACC + (size_t)nbr_of(cf, j) * REC_FA, z);
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) d.Un[c * N + i] = u[c];
  if (F32) {
    float r[REC_U32];
#pragma unroll
    for (int c = 0; c < 5; ++c) r[c] = (float)u[c];
    r[5] = (float)d.lev[i];
    r[6] = r[7] = 0.0f;
    strec<REC_U32>(d.Un32 + (size_t)i * REC_U32, r);
  }
}

template <bool F32>
__device__ __forceinline__ void update_item(const DevMesh &d, int stage, int level, int idx) {
  const size_t N = d.N;
  double dtmin = __longlong_as_double((long long)*d.dtmin_bits);
  // the cell, its faces and its bits from the list entry
  const int i = d.cl[idx];
  const unsigned bits = d.clb[idx];
  const unsigned own = bits & 15u;
  const int4 cf = d.clf[idx];
  if (stage == 1 && F32 && d.pred_sum64) {
    // the predictor's residual sum in FP64 (each FP32 flux widened) and U*
    // from the FP64 U^n; U* is rounded to its FP32 record, which only feeds
    // fluxes
    double S[5];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      bool neg = !((own >> j) & 1u);
      float v[REC_FA32];
      ldrec<REC_FA32>(d.FA32 + (size_t)nbr_of(cf, j) * REC_FA32, v);
#pragma unroll
      for (int c = 0; c < 5; ++c) S[c] = j == 0 ? flip((double)v[c], neg) : S[c] + flip((double)v[c], neg);
    }
    const int k = d.lev[i];
    double u[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) u[c] = d.Un[c * N + i];
    const double cdt = -scale2(dtmin, k) * d.ivol[i];
    float r[REC_U32];
#pragma unroll
    for (int c = 0; c < 5; ++c) r[c] = (float)(u[c] + cdt * S[c]);
    r[5] = (float)k;
    r[6] = r[7] = 0.0f;
    strec<REC_U32>(d.Us32 + (size_t)i * REC_U32, r);
    return;
  }
  if (stage == 1 && F32) {
    float S[5];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      bool neg = !((own >> j) & 1u);
      float v[REC_FA32];
      ldrec<REC_FA32>(d.FA32 + (size_t)nbr_of(cf, j) * REC_FA32, v);
#pragma unroll
      for (int c = 0; c < 5; ++c) S[c] = j == 0 ? flip(v[c], neg) : S[c] + flip(v[c], neg);
    }
    float a[REC_U32];
    ldrec<REC_U32>(d.Un32 + (size_t)i * REC_U32, a);
    float cdt = -(float)scale2(dtmin, (int)a[5]) * d.ivol32[i];
#pragma unroll
    for (int c = 0; c < 5; ++c) a[c] = a[c] + cdt * S[c];
    strec<REC_U32>(d.Us32 + (size_t)i * REC_U32, a);
    return;
  }
  // every load comes before the first store (the reset of the accumulated
  // integrals is last), so the four face loads and the state loads overlap
  // instead of waiting on one another behind possibly aliasing stores.  At
  // the end of a step, faces to finer neighbours (cmask) contribute their
  // accumulated integrals.
  const unsigned finer = stage == 2 ? bits >> 4 : 0u;
  bool reset[4];
  const double *src[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    reset[j] = (finer >> j) & 1u;
    src[j] = (reset[j] ? d.ACC : d.FA) + (size_t)nbr_of(cf, j) * REC_FA;
  }
  double S[5];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    bool neg = !((own >> j) & 1u);
    double v[REC_FA];
    ldrec<REC_FA>(src[j], v);
#pragma unroll
    for (int c = 0; c < 5; ++c) S[c] = j == 0 ? flip(v[c], neg) : S[c] + flip(v[c], neg);
  }
  const double iV = d.ivol[i];
  double u[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) u[c] = d.Un[c * N + i];
  if (stage == 1) {
    double cdt = -scale2(dtmin, (int)d.lev[i]) * iV;
#pragma unroll
    for (int c = 0; c < 5; ++c) d.Us[c * N + i] = u[c] + cdt * S[c];
  } else {
    const double hV = scale2(dtmin, level - 1) * iV;
    float r[REC_U32];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      u[c] = u[c] - hV * S[c];
      r[c] = (float)u[c];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) d.Un[c * N + i] = u[c];
    if (F32) {
      r[5] = (float)level;  // the cell ends the step of its own level
      r[6] = r[7] = 0.0f;
      strec<REC_U32>(d.Un32 + (size_t)i * REC_U32, r);
    }
    const double z[REC_FA] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (reset[j]) strec<REC_FA>(const_cast<double *>(src[j]), z);
  }
}

// The update with the gather shared by four lanes per cell (the quad of the
// cell's four faces, `fv_set_gather`): lane j loads face j's record and
// applies its sign, the quad's first lane adds the four values in face order
// ((v0 + v1) + v2) + v3 -- the order of update_item, so the results are
// bitwise the same -- and updates the cell; lane j resets face j's
// accumulated integral.  A warp covers 8 cells per step of its loop, which
// every lane runs the same number of times (the shuffles take the whole
// warp).  The paper's order and the FP64 predictor sum keep update_item.
template <bool F32>
__device__ __forceinline__ void update_range_quad(const DevMesh &d, int stage, int level, int beg, int end) {
  const unsigned FULL = 0xffffffffu;
  const size_t N = d.N;
  const double dtmin = __longlong_as_double((long long)*d.dtmin_bits);
  const int lane = threadIdx.x & 31, j = lane & 3, lead = lane & ~3;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int base = beg + warp * 8; base < end; base += nwarps * 8) {
    const int idx = base + (lane >> 2);
    const bool valid = idx < end;
    int i = 0, f = 0;
    unsigned bits = 0;
    if (valid) {
      i = d.cl[idx];
      bits = d.clb[idx];
      f = reinterpret_cast<const int *>(d.clf + idx)[j];
    }
    const bool neg = !((bits >> j) & 1u);
    if (stage == 1 && F32) {
      float v[REC_FA32];
      if (valid) {
        ldrec<REC_FA32>(d.FA32 + (size_t)f * REC_FA32, v);
      } else {
#pragma unroll
        for (int c = 0; c < REC_FA32; ++c) v[c] = 0.0f;
      }
      float S[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const float x = flip(v[c], neg);
        const float x1 = __shfl_sync(FULL, x, lead + 1), x2 = __shfl_sync(FULL, x, lead + 2),
                    x3 = __shfl_sync(FULL, x, lead + 3);
        S[c] = ((x + x1) + x2) + x3;
      }
      if (valid && j == 0) {
        float a[REC_U32];
        ldrec<REC_U32>(d.Un32 + (size_t)i * REC_U32, a);
        const float cdt = -(float)scale2(dtmin, (int)a[5]) * d.ivol32[i];
#pragma unroll
        for (int c = 0; c < 5; ++c) a[c] = a[c] + cdt * S[c];
        strec<REC_U32>(d.Us32 + (size_t)i * REC_U32, a);
      }
      continue;
    }
    const bool reset = stage == 2 && ((bits >> (4 + j)) & 1u);
    double *src = (reset ? d.ACC : d.FA) + (size_t)f * REC_FA;
    double v[REC_FA];
    if (valid) {
      ldrec<REC_FA>(src, v);
    } else {
#pragma unroll
      for (int c = 0; c < REC_FA; ++c) v[c] = 0.0;
    }
    double S[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const double x = flip(v[c], neg);
      const double x1 = __shfl_sync(FULL, x, lead + 1), x2 = __shfl_sync(FULL, x, lead + 2),
                   x3 = __shfl_sync(FULL, x, lead + 3);
      S[c] = ((x + x1) + x2) + x3;
    }
    if (valid && j == 0) {
      const double iV = d.ivol[i];
      double u[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) u[c] = d.Un[c * N + i];
      if (stage == 1) {
        const double cdt = -scale2(dtmin, (int)d.lev[i]) * iV;
#pragma unroll
        for (int c = 0; c < 5; ++c) d.Us[c * N + i] = u[c] + cdt * S[c];
      } else {
        const double hV = scale2(dtmin, level - 1) * iV;
        float r[REC_U32];
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          u[c] = u[c] - hV * S[c];
          r[c] = (float)u[c];
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) d.Un[c * N + i] = u[c];
        if (F32) {
          r[5] = (float)level;
          r[6] = r[7] = 0.0f;
          strec<REC_U32>(d.Un32 + (size_t)i * REC_U32, r);
        }
      }
    }
    if (valid && reset) {
      const double z[REC_FA] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      strec<REC_FA>(src, z);
    }
  }
}

// ---- phase drivers: one kernel kind over the phase's list range of one
// mesh (k_phase1), or over the concatenated ranges of a batch of meshes
// (k_phaseN: a flattened work index, split by a per-block prefix over the
// instances' range lengths)
enum { K_PRIM = 0, K_GRAD = 1, K_FLUX = 2, K_UPD = 3, K_CORR = 4, K_COMMIT = 5 };  // K_CORR, K_COMMIT:
// the cell updates of order 1's correct (stage 3) and commit (stage 4) phases


__device__ __forceinline__ void kind_range(const DevMesh &d, const PhaseDesc &p, int kind, int &beg,
                                           int &end) {
  if (kind == K_FLUX) {
    beg = d.foff[p.fb0];
    end = d.foff[p.fb1];
  } else {
    int b0 = kind == K_PRIM ? p.pb0 : kind == K_GRAD ? p.gb0 : p.ub0;
    int b1 = kind == K_PRIM ? p.pb1 : kind == K_GRAD ? p.gb1 : p.ub1;
    beg = d.coff[b0];
    end = d.coff[b1];
  }
}

template <int KIND, typename T, bool G14>
__device__ __forceinline__ void run_item(const DevMesh &d, const PhaseDesc &p, const GasT<T> &G,
                                         int idx) {
  if (KIND == K_PRIM)
    prim_item<T>(d, p.pl, idx);
  else if (KIND == K_GRAD)
    grad_item<T>(d, p.pl, idx);
  else if (KIND == K_FLUX)
    flux_item<T, G14>(d, G, p.stage, p.level, idx);
  else if (KIND == K_UPD)
    update_item<sizeof(T) == 4>(d, p.stage, p.level, idx);
  else if (KIND == K_CORR)
    correct_cell<sizeof(T) == 4>(d, p.level, idx);
  else
    commit_cell<sizeof(T) == 4>(d, idx);
}

// flux: 128 threads, 8 blocks per SM in FP32 (64 registers), 4 in FP64;
// FP64 gradients need ~96 registers (2 blocks of 256); the update (a gather
// with all of its loads in flight at once) fits in 48 registers for 5
// resident blocks of 256; the rest fit in 64
#ifndef FV_FLUX32_BLOCKS
#define FV_FLUX32_BLOCKS 8
#endif
#define KBOUNDS(KIND, T)                                                                      \
  __launch_bounds__((KIND) == K_FLUX ? 128 : 256,                                             \
                    (KIND) == K_FLUX ? (sizeof(T) == 4 ? FV_FLUX32_BLOCKS : 4)                \
                    : (KIND) == K_UPD ? 5                                                     \
                                      : ((KIND) == K_GRAD && sizeof(T) == 8 ? 2 : 4))

// FP32-flux mode with the two-rarefaction guess: a phase with at most
// d.fuse_faces faces is latency-bound (about a wave of faces or less, each a
// chain of dependent loads), so its flux kernel computes the gradients it
// needs itself (a cell's gradient once per face of the cell) and its
// gradient kernel does nothing.  Decided on the device from the phase's
// face count, so a captured cycle follows every level assignment.
__device__ __forceinline__ bool fused_phase(const DevMesh &d, const PhaseDesc &p) {
  return d.fuse_faces > 0 && d.guess == FV_GUESS_TWO_RAREFACTION &&
         d.foff[p.fb1] - d.foff[p.fb0] <= d.fuse_faces;
}

template <int KIND, typename T, bool G14>
__global__ void KBOUNDS(KIND, T) k_phase1(DevMesh d, const __grid_constant__ PhaseDesc p, GasT<T> G) {
  pdl_wait();
  int beg, end;
  kind_range(d, p, KIND, beg, end);
  bool fused = false;
  if constexpr (sizeof(T) == 4 && (KIND == K_GRAD || KIND == K_FLUX)) fused = fused_phase(d, p);
  if (!fused)
    for (int idx = beg + blockIdx.x * blockDim.x + threadIdx.x; idx < end; idx += gridDim.x * blockDim.x)
      run_item<KIND, T, G14>(d, p, G, idx);
  pdl_trigger();
}

// the update with the quad gather (fv_set_gather), a kernel of its own so
// that the per-thread update keeps its registers
template <typename T>
__global__ void __launch_bounds__(256, 5) k_update_quad(DevMesh d, const __grid_constant__ PhaseDesc p) {
  pdl_wait();
  int beg, end;
  kind_range(d, p, K_UPD, beg, end);
  update_range_quad<sizeof(T) == 4>(d, p.stage, p.level, beg, end);
  pdl_trigger();
}

// the flux of a fused phase (FP32-flux mode): with both cells' gradients to
// compute per face it needs more registers than the plain flux kernel, and
// runs where a wave of faces or less is in flight anyway.  Launched after the
// plain flux kernel of every phase; exactly one of the two has work.
#ifndef FV_FUSED_BLOCKS
#define FV_FUSED_BLOCKS 4  // resident 128-thread blocks per SM (up to 128 registers)
#endif
template <bool G14>
__global__ void __launch_bounds__(128, FV_FUSED_BLOCKS) k_flux_fused(DevMesh d, const __grid_constant__ PhaseDesc p,
                                                                     GasT<float> G) {
  pdl_wait();
  if (fused_phase(d, p)) {
    int beg, end;
    kind_range(d, p, K_FLUX, beg, end);
    const bool both = reads_predicted(p.pl);
    for (int idx = beg + blockIdx.x * blockDim.x + threadIdx.x; idx < end; idx += gridDim.x * blockDim.x)
      flux_item_fused<G14>(d, G, p.stage, p.level, p.pl, both, idx);
  }
  pdl_trigger();
}

// ---- the FP32 flux with its inputs staged through shared memory.  Each
// thread copies the records of its next face (geometry, both cells'
// primitives and gradients: 14 chunks of 16 bytes) into its own slots of
// shared memory with asynchronous copies (cp.async) while it solves the
// Riemann problem of the current face, and loads the list entry of the face
// after that into registers; the gathers of a face are in flight during the
// previous face's arithmetic instead of stalling its warp.  Slots are
// chunk-major ([chunk][thread]), so a warp's 16-byte reads of one chunk hit
// consecutive banks.  The same operations as flux_item on the same values.
#define FLUX_STAGE_CHUNKS 14
#define FLUX_STAGE_THREADS 128
#ifndef FV_STAGED_BLOCKS
#define FV_STAGED_BLOCKS 7  // 28 KB of shared memory per block: 7 resident blocks per SM
#endif

__device__ __forceinline__ void cp_async16(float4 *dst_smem, const void *src) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(a), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// copies of face f's records (fc its cells) into slot t of st
__device__ __forceinline__ void stage_face(const DevMesh &d, float4 (*st)[FLUX_STAGE_THREADS], int t, int f,
                                           int2 fc) {
  const float4 *geo = reinterpret_cast<const float4 *>(d.fgeo32 + (size_t)f * REC_FG);
  const float4 *W = reinterpret_cast<const float4 *>(d.W);
  const float4 *G = reinterpret_cast<const float4 *>(d.G32);
  cp_async16(&st[0][t], geo);
  cp_async16(&st[1][t], geo + 1);
  cp_async16(&st[2][t], W + (size_t)fc.x * (REC_W / 4));
  cp_async16(&st[3][t], W + (size_t)fc.x * (REC_W / 4) + 1);
#pragma unroll
  for (int k = 0; k < 4; ++k) cp_async16(&st[4 + k][t], G + (size_t)fc.x * (REC_G / 4) + k);
  if (fc.y >= 0) {
    cp_async16(&st[8][t], W + (size_t)fc.y * (REC_W / 4));
    cp_async16(&st[9][t], W + (size_t)fc.y * (REC_W / 4) + 1);
#pragma unroll
    for (int k = 0; k < 4; ++k) cp_async16(&st[10 + k][t], G + (size_t)fc.y * (REC_G / 4) + k);
  }
}

// face_states from the staged records (R = fc.y); iface: the two cells'
// levels (slot 5 of their primitive records) differ
__device__ __forceinline__ void face_states_staged(const float4 (*st)[FLUX_STAGE_THREADS], int t, int R,
                                                   float WL[5], float WR[5], float n[3], float &A,
                                                   bool &iface) {
  const float4 g0 = st[0][t], g1 = st[1][t];
  n[0] = g0.x;
  n[1] = g0.y;
  n[2] = g0.z;
  A = g0.w;
  const float r[3] = {g1.x, g1.y, g1.z};
  const float4 a0 = st[2][t], a1 = st[3][t];
  const float Wi[6] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y};
  float gi[16];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 v = st[4 + k][t];
    gi[4 * k] = v.x;
    gi[4 * k + 1] = v.y;
    gi[4 * k + 2] = v.z;
    gi[4 * k + 3] = v.w;
  }
  if (R >= 0) {
    const float4 b0 = st[8][t], b1 = st[9][t];
    const float Wj[6] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y};
    float gj[16];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float4 v = st[10 + k][t];
      gj[4 * k] = v.x;
      gj[4 * k + 1] = v.y;
      gj[4 * k + 2] = v.z;
      gj[4 * k + 3] = v.w;
    }
    iface = Wi[5] != Wj[5];
    reconstruct_pair(Wi, gi, Wj, gj, r, WL, WR);
  } else {
    iface = false;
    float Wg[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) Wg[c] = Wi[c];
    if (R == -FV_BC_WALL) {
      float un = (Wi[1] * n[0] + Wi[2] * n[1]) + Wi[3] * n[2];
#pragma unroll
      for (int e = 0; e < 3; ++e) Wg[1 + e] = Wi[1 + e] - (2.0f * un) * n[e];
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      float dW = Wg[c] - Wi[c];
      float gir = (gi[3 * c] * r[0] + gi[3 * c + 1] * r[1]) + gi[3 * c + 2] * r[2];
      WL[c] = Wi[c] + 0.5f * minmod(2.0f * gir - dW, dW);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) WR[c] = WL[c];
  }
}

template <bool G14>
__global__ void __launch_bounds__(FLUX_STAGE_THREADS, FV_STAGED_BLOCKS)
    k_flux_staged(DevMesh d, const __grid_constant__ PhaseDesc p, GasT<float> G) {
  __shared__ float4 st[FLUX_STAGE_CHUNKS][FLUX_STAGE_THREADS];
  pdl_wait();
  int beg, end;
  kind_range(d, p, K_FLUX, beg, end);
  const int t = threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  int idx = beg + blockIdx.x * blockDim.x + t;
  // entries of the current face (its records staged) and of the next one
  int f0 = -1, f1 = -1;
  int2 c0 = make_int2(0, 0), c1 = make_int2(0, 0);
  if (idx < end) {
    f0 = d.fl[idx];
    c0 = d.flc[idx];
    stage_face(d, st, t, f0, c0);
  }
  cp_async_commit();
  if (idx + stride < end) {
    f1 = d.fl[idx + stride];
    c1 = d.flc[idx + stride];
  }
  for (; idx < end; idx += stride) {
    cp_async_wait_all();
    float WL[5], WR[5], n[3], A;
    bool iface;
    face_states_staged(st, t, c0.y, WL, WR, n, A, iface);
    // the slots are free: the next face's records go in flight, and the
    // entry of the face after it
    if (f1 >= 0) stage_face(d, st, t, f1, c1);
    cp_async_commit();
    int f2 = -1;
    int2 c2 = make_int2(0, 0);
    if (idx + 2 * stride < end) {
      f2 = d.fl[idx + 2 * stride];
      c2 = d.flc[idx + 2 * stride];
    }
    int it, rc;
    float Fx[5], FAt[5];
    if (c0.y >= 0)
      rc = godunov_flux<float, G14, false>(G, WL, WR, n, Fx, it, 0.0f, 1.0f);
    else
      rc = boundary_flux<float, G14>(G, -c0.y, WL, n, Fx, it);
#pragma unroll
    for (int c = 0; c < 5; ++c) FAt[c] = Fx[c] * A;
    if (rc) atomicOr(d.status, FV_STATUS_RIEMANN);
    flux_store<float>(d, p.stage, p.level, f0, FAt, p.stage != 1 && iface, p.stage != 1 && c0.y < 0);
    f0 = f1;
    c0 = c1;
    f1 = f2;
    c1 = c2;
  }
  cp_async_wait_all();
  pdl_trigger();
}

// flux with the learned guess: the packed network staged in shared memory,
// the loop warp-uniform (lanes past the end ride along without a face)
#ifndef FV_MLP_FLUX_BLOCKS
#define FV_MLP_FLUX_BLOCKS 8  // resident 128-thread blocks per SM (64 registers)
#endif
template <typename T, bool G14>
__global__ void __launch_bounds__(128, FV_MLP_FLUX_BLOCKS) k_flux_mlp1(DevMesh d, const __grid_constant__ PhaseDesc p,
                                                      GasT<T> G) {
  __shared__ __align__(16) uint32_t sw[PK_WORDS];
  mlp_stage(sw, d.mlp);  // the weights do not depend on the previous kernel
  pdl_wait();
  int beg, end;
  kind_range(d, p, K_FLUX, beg, end);
  const int lane = threadIdx.x & 31;
  for (int base = beg + blockIdx.x * blockDim.x + (threadIdx.x - lane); base < end;
       base += gridDim.x * blockDim.x) {
    const int idx = base + lane;
    flux_item<T, G14, true>(d, G, p.stage, p.level, idx < end ? idx : -1, sw);
  }
  pdl_trigger();
}

// a batch's flattened work index: the first warp of the block writes the
// exclusive prefix of the active instances' range lengths (pref[0..n], total
// in pref[FV_MAXB]) and their range starts (base) to shared memory
__device__ __forceinline__ void batch_prefix(const DevMesh *__restrict__ ms,
                                             const PhaseDesc *__restrict__ ps, int n, int kind,
                                             int *pref, int *base) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int len[2], b[2];
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      int i = lane + 32 * hh;
      len[hh] = 0;
      b[hh] = 0;
      if (i < n && ps[i].active) {
        int e;
        kind_range(ms[i], ps[i], kind, b[hh], e);
        len[hh] = e - b[hh];
      }
    }
    int x0 = len[0], x1 = len[1];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y0 = __shfl_up_sync(0xffffffff, x0, o), y1 = __shfl_up_sync(0xffffffff, x1, o);
      if (lane >= o) {
        x0 += y0;
        x1 += y1;
      }
    }
    int tot0 = __shfl_sync(0xffffffff, x0, 31);
    pref[lane] = x0 - len[0];
    pref[lane + 32] = tot0 + x1 - len[1];
    if (lane == 31) pref[FV_MAXB] = tot0 + x1;
    base[lane] = b[0];
    base[lane + 32] = b[1];
  }
  __syncthreads();
}

// the instance of flattened index g (binary search of the prefix)
__device__ __forceinline__ int batch_instance(const int *pref, int n, int g) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (pref[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// the batch's flux with the learned guess: one packed network for every
// instance, the warp-uniform loop over the flattened face index
template <typename T, bool G14>
__global__ void __launch_bounds__(128, FV_MLP_FLUX_BLOCKS) k_flux_mlpN(const DevMesh *__restrict__ ms,
                                                                       const PhaseDesc *__restrict__ ps,
                                                                       int n, GasT<T> G,
                                                                       const uint32_t *__restrict__ mlp) {
  __shared__ __align__(16) uint32_t sw[PK_WORDS];
  __shared__ int pref[FV_MAXB + 1];
  __shared__ int base[FV_MAXB];
  mlp_stage(sw, mlp);
  pdl_wait();
  batch_prefix(ms, ps, n, K_FLUX, pref, base);
  const int total = pref[FV_MAXB];
  const int lane = threadIdx.x & 31;
  for (int gb = blockIdx.x * blockDim.x + (threadIdx.x - lane); gb < total; gb += gridDim.x * blockDim.x) {
    // one call for every lane (the guess inside is warp-collective): lanes
    // past the end pass no face
    const int g = gb + lane;
    const bool ok = g < total;
    const int lo = ok ? batch_instance(pref, n, g) : 0;
    const int idx = ok ? base[lo] + (g - pref[lo]) : -1;
    flux_item<T, G14, true>(ms[lo], G, ps[lo].stage, ps[lo].level, idx, sw);
  }
  pdl_trigger();
}

template <int KIND, typename T, bool G14>
__global__ void KBOUNDS(KIND, T) k_phaseN(const DevMesh *__restrict__ ms, const PhaseDesc *__restrict__ ps,
                                          int n, GasT<T> G) {
  __shared__ int pref[FV_MAXB + 1];
  __shared__ int base[FV_MAXB];
  pdl_wait();
  batch_prefix(ms, ps, n, KIND, pref, base);
  const int total = pref[FV_MAXB];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    const int lo = batch_instance(pref, n, g);
    run_item<KIND, T, G14>(ms[lo], ps[lo], G, base[lo] + (g - pref[lo]));
  }
  pdl_trigger();
}

// ---- persistent cycle: every phase of a cycle in one cooperative launch,
// the kernel kinds of a phase separated by a grid barrier.  The blocks all
// run the same sequence (phase by phase, prim -> grad -> flux -> update, a
// barrier after each), so every block meets every barrier.  The barrier is a
// counter and a generation number; waiting is bounded: after 2^21 polls of
// the generation (each an L2 round trip, about a second in all) a block
// records FV_STATUS_TIMEOUT and every block leaves at its next barrier.
#define FV_BAR_SPIN_LIMIT (1u << 21)

__device__ __forceinline__ bool grid_barrier(GridBar *b, int *status, unsigned expected) {
  __shared__ int go;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = &b->gen;
    volatile int *vst = status;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(&b->count, 1u) == expected - 1) {
      b->count = 0;
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      unsigned spins = 0;
      while (*vgen == g) {
        if (++spins > FV_BAR_SPIN_LIMIT) {
          atomicOr(status, FV_STATUS_TIMEOUT);
          break;
        }
        if ((spins & 1023u) == 0 && (*vst & FV_STATUS_TIMEOUT)) break;  // another block gave up
      }
    }
    __threadfence();
    go = (*(volatile int *)status & FV_STATUS_TIMEOUT) == 0;
  }
  __syncthreads();
  return go != 0;
}

// the barrier on its own, for failure-detection tests: `rounds` barriers
// over the grid, each expecting gridDim.x + extra arrivals (extra > 0: a
// count that is never reached, so every wait runs out)
__global__ void k_barrier_probe(GridBar *bar, int *status, int rounds, unsigned extra) {
  for (int r = 0; r < rounds; ++r)
    if (!grid_barrier(bar, status, gridDim.x + extra)) return;
}

int launch_barrier_probe(GridBar *bar, int *status, int rounds, unsigned extra, cudaStream_t s) {
  if (cudaMemsetAsync(bar, 0, sizeof(GridBar), s) != cudaSuccess) return FV_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(num_sms());
  cfg.blockDim = dim3(64);
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_barrier_probe, bar, status, rounds, extra) != cudaSuccess) return FV_ERR_CUDA;
  return FV_OK;
}

// 256-thread blocks, 4 per SM at 64 registers (FP32), 2 at 128 (FP64)
template <typename T>
struct PersistThreads {
  static constexpr int value = 256;
  static constexpr int blocks = sizeof(T) == 4 ? 4 : 2;
};

template <typename T, bool G14>
__global__ void __launch_bounds__(PersistThreads<T>::value, PersistThreads<T>::blocks)
    k_persist(DevMesh d, const PhaseDesc *__restrict__ pds, int nph, GasT<T> G, GridBar *bar) {
  const int stride = gridDim.x * blockDim.x;
  for (int p = 0; p < nph; ++p) {
    const PhaseDesc &pd = pds[p];
    int beg, end;
    if (sizeof(T) == 8) {  // the FP32-flux mode computes primitives in the gradient step
      kind_range(d, pd, K_PRIM, beg, end);
      for (int idx = beg + blockIdx.x * blockDim.x + threadIdx.x; idx < end; idx += stride)
        prim_item<T>(d, pd.pl, idx);
      if (!grid_barrier(bar, d.status, gridDim.x)) return;
    }
    kind_range(d, pd, K_GRAD, beg, end);
    for (int idx = beg + blockIdx.x * blockDim.x + threadIdx.x; idx < end; idx += stride)
      grad_item<T>(d, pd.pl, idx);
    if (!grid_barrier(bar, d.status, gridDim.x)) return;
    kind_range(d, pd, K_FLUX, beg, end);
    for (int idx = beg + blockIdx.x * blockDim.x + threadIdx.x; idx < end; idx += stride)
      flux_item<T, G14>(d, G, pd.stage, pd.level, idx);
    if (!grid_barrier(bar, d.status, gridDim.x)) return;
    kind_range(d, pd, K_UPD, beg, end);
    for (int idx = beg + blockIdx.x * blockDim.x + threadIdx.x; idx < end; idx += stride)
      update_item<sizeof(T) == 4>(d, pd.stage, pd.level, idx);
    if (!grid_barrier(bar, d.status, gridDim.x)) return;
  }
}

template <typename T, bool G14>
static int persist_launch(const DevMesh &d, const PhaseDesc *pds, int nph, const GasT<T> &G,
                          GridBar *bar, cudaStream_t s) {
  static int per_sm[2][2] = {{0, 0}, {0, 0}};
  int &bps = per_sm[sizeof(T) == 4][G14];
  if (!bps) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_persist<T, G14>, PersistThreads<T>::value,
                                                      0) != cudaSuccess ||
        bps < 1)
      return FV_ERR_CUDA;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(num_sms() * bps);
  cfg.blockDim = dim3(PersistThreads<T>::value);
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_persist<T, G14>, d, pds, nph, G, bar) != cudaSuccess) return FV_ERR_CUDA;
  return FV_OK;
}

// positivity and finiteness of U^n (rho > 0, 2 rho E > |rho u|^2)
__global__ void __launch_bounds__(256) k_check_state(DevMesh d) {
  const size_t N = d.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x) {
    double U[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) U[c] = d.Un[c * N + i];
    double m2 = (U[1] * U[1] + U[2] * U[2]) + U[3] * U[3];
    if (!(U[0] > 0.0) || !(2.0 * U[0] * U[4] > m2) || !isfinite(m2 + U[4]))
      atomicOr(d.status, FV_STATUS_NONPHYS);
  }
}

int launch_check_state(const DevMesh &d, cudaStream_t s) {
  k_check_state<<<grid_for(d.N, 256, 8), 256, 0, s>>>(d);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

// R = -(1/V) sum sigma F A for the cells of one level (residual hook);
// written in the caller's order
__global__ void __launch_bounds__(256) k_residual(DevMesh d, int level, const double *__restrict__ FAt,
                                                  double *__restrict__ R, const int *__restrict__ new2old) {
  const size_t N = d.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x) {
    int o = new2old[i];
    if (d.lev[i] != level) {
#pragma unroll
      for (int c = 0; c < 5; ++c) R[c * N + o] = 0.0;
      continue;
    }
    unsigned own = d.cown[i];
    int4 cf = d.cf4[i];
    double S[5];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      bool neg = !((own >> j) & 1u);
      double v[REC_FA];
      ldrec<REC_FA>(FAt + (size_t)nbr_of(cf, j) * REC_FA, v);
#pragma unroll
      for (int c = 0; c < 5; ++c) S[c] = j == 0 ? flip(v[c], neg) : S[c] + flip(v[c], neg);
    }
    double iV = d.ivol[i];
#pragma unroll
    for (int c = 0; c < 5; ++c) R[c * N + o] = -S[c] * iV;
  }
}

// F A of every face touching a level-`level` cell into FAt (residual hook)
template <typename T, bool G14>
__global__ void __launch_bounds__(128) k_flux_all(DevMesh d, GasT<T> G, int level, const T *__restrict__ W,
                                                  const T *__restrict__ Gr, const T *__restrict__ fgeo,
                                                  double *__restrict__ FAt) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < d.F; f += gridDim.x * blockDim.x) {
    int2 fc = d.fcell[f];
    bool touch = d.lev[fc.x] == level || (fc.y >= 0 && d.lev[fc.y] == level);
    if (!touch) continue;
    T FAx[5];
    if (face_flux<T, G14>(d, G, W, Gr, fgeo, f, fc, FAx)) atomicOr(d.status, FV_STATUS_RIEMANN);
    double v[REC_FA] = {(double)FAx[0], (double)FAx[1], (double)FAx[2], (double)FAx[3], (double)FAx[4], 0.0};
    strec<REC_FA>(FAt + (size_t)f * REC_FA, v);
  }
}

// primitives of every cell (residual hook: a plain, unsorted pass)
template <typename WT>
__global__ void __launch_bounds__(256) k_prim_all(DevMesh d, const __grid_constant__ PhaseLevels pl, WT *W) {
  double gm1 = d.gamma - 1.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x) {
    WT U[5], Wt[REC_W];
    load_state(d, pl, i, U);
    to_prim(U, gm1, Wt);
#pragma unroll
    for (int q = 5; q < REC_W; ++q) Wt[q] = WT(0);
    strec<REC_W>(W + (size_t)i * REC_W, Wt);
  }
}

// end of a cycle: t += 2^theta dt_min, and the work counters of the cost
// model: sum_k 2^(theta-k) |Omega_k| cell updates, twice that over faces
// The cycle's level distribution also goes into the level history (cells
// per level and dt_min, a ring of FV_HIST_CAP cycles).
__device__ __forceinline__ void time_advance_of(const DevMesh &d, int theta) {
  const double dtmin = __longlong_as_double((long long)*d.dtmin_bits);
  d.tdev[0] += ldexp(dtmin, theta);
  long long cu = 0, fe = 0;
  const long long slot = d.counters[0] % FV_HIST_CAP;
  for (int k = 0; k < FV_MAXL; ++k) {
    const int nk = k <= theta ? d.coff[2 * k + 2] - d.coff[2 * k] : 0;
    d.hist[slot * FV_MAXL + k] = nk;
    if (k <= theta) {
      cu += (long long)nk << (theta - k);
      fe += (long long)(d.foff[k + 1] - d.foff[k]) << (theta - k + 1);
    }
  }
  d.hist_dt[slot] = dtmin;
  d.counters[0] += 1;
  d.counters[1] += cu;
  d.counters[2] += fe;
}

__global__ void k_time_advance(DevMesh d, int theta) { time_advance_of(d, theta); }

__global__ void k_time_advance_multi(const DevMesh *ms, const PhaseDesc *pds, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && pds[i].end_cycle) time_advance_of(ms[i], ms[i].L - 1);
}

// caller-order primitives -> Morton-order conserved state
__global__ void __launch_bounds__(256) k_set_state(DevMesh d, const double *__restrict__ prim,
                                                   const int *__restrict__ new2old) {
  const size_t N = d.N;
  double gm1 = d.gamma - 1.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x) {
    int o = new2old[i];
    double r = prim[o], u = prim[N + o], v = prim[2 * N + o], w = prim[3 * N + o], p = prim[4 * N + o];
    if (!(r > 0.0) || !(p > 0.0)) atomicOr(d.status, FV_STATUS_NONPHYS);
    d.Un[i] = r;
    d.Un[N + i] = __dmul_rn(r, u);
    d.Un[2 * N + i] = __dmul_rn(r, v);
    d.Un[3 * N + i] = __dmul_rn(r, w);
    double uu = __dadd_rn(__dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)), __dmul_rn(w, w));
    d.Un[4 * N + i] = __dadd_rn(__ddiv_rn(p, gm1), __dmul_rn(__dmul_rn(0.5, r), uu));
    if (d.Un32) {
      float r[REC_U32];
#pragma unroll
      for (int c = 0; c < 5; ++c) r[c] = (float)d.Un[c * N + i];
      r[5] = r[6] = r[7] = 0.0f;  // level: stamped by the next level assignment
      strec<REC_U32>(d.Un32 + (size_t)i * REC_U32, r);
    }
  }
}

__global__ void __launch_bounds__(256) k_set_cons(DevMesh d, const double *__restrict__ cons,
                                                  const int *__restrict__ new2old) {
  const size_t N = d.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x) {
    int o = new2old[i];
#pragma unroll
    for (int c = 0; c < 5; ++c) d.Un[c * N + i] = cons[c * N + o];
    if (d.Un32) {
      float r[REC_U32];
#pragma unroll
      for (int c = 0; c < 5; ++c) r[c] = (float)cons[c * N + o];
      r[5] = r[6] = r[7] = 0.0f;  // level: stamped by the next level assignment
      strec<REC_U32>(d.Un32 + (size_t)i * REC_U32, r);
    }
    if (!(cons[o] > 0.0)) atomicOr(d.status, FV_STATUS_NONPHYS);
  }
}

__global__ void __launch_bounds__(256) k_get_state(DevMesh d, double *__restrict__ cons,
                                                   const int *__restrict__ new2old) {
  const size_t N = d.N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x) {
    int o = new2old[i];
#pragma unroll
    for (int c = 0; c < 5; ++c) cons[c * N + o] = d.Un[c * N + i];
  }
}

__global__ void __launch_bounds__(256) k_get_levels(DevMesh d, int8_t *__restrict__ lev,
                                                    const int *__restrict__ new2old) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.N; i += gridDim.x * blockDim.x)
    lev[new2old[i]] = d.lev[i];
}

// Godunov flux of independent face states (test / harvesting hook)
template <typename T, bool G14>
__global__ void __launch_bounds__(128) k_flux_batch(const double *__restrict__ WL,
                                                    const double *__restrict__ WR,
                                                    const double *__restrict__ nrm, int n, GasT<T> G,
                                                    int bc, double *__restrict__ F,
                                                    int *__restrict__ iters) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T wl[5], wr[5], nn[3], Fx[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      wl[c] = (T)WL[(size_t)c * n + i];
      wr[c] = (T)WR[(size_t)c * n + i];
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) nn[e] = (T)nrm[(size_t)e * n + i];
    int it = 0, rc;
    if (bc == 0)
      rc = godunov_flux<T, G14>(G, wl, wr, nn, Fx, it);
    else
      rc = boundary_flux<T, G14>(G, bc, wl, nn, Fx, it);
#pragma unroll
    for (int c = 0; c < 5; ++c) F[(size_t)c * n + i] = rc ? 0.0 : (double)Fx[c];
    iters[i] = rc ? -1 : it;
  }
}

// the same with the learned starting guess (interior faces; warp-uniform
// loop, packed network staged in shared memory)
template <typename T, bool G14>
__global__ void __launch_bounds__(128, 4) k_flux_batch_mlp(const double *__restrict__ WL,
                                                           const double *__restrict__ WR,
                                                           const double *__restrict__ nrm, int n,
                                                           GasT<T> G, const uint32_t *__restrict__ mlp,
                                                           double *__restrict__ F,
                                                           int *__restrict__ iters) {
  __shared__ __align__(16) uint32_t sw[PK_WORDS];
  mlp_stage(sw, mlp);
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x - lane); base < n;
       base += gridDim.x * blockDim.x) {
    const int i = base + lane;
    const bool ok = i < n;
    T wl[5], wr[5], nn[3], Fx[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      wl[c] = ok ? (T)WL[(size_t)c * n + i] : T(c == 0 || c == 4);
      wr[c] = ok ? (T)WR[(size_t)c * n + i] : T(c == 0 || c == 4);
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) nn[e] = ok ? (T)nrm[(size_t)e * n + i] : T(e == 0);
    T gabs, gmul;
    __syncwarp();
    mlp_guess<T>(sw, (float)G.g, wl, wr, nn, gabs, gmul);
    if (!ok) continue;
    int it = 0;
    int rc = godunov_flux<T, G14, true>(G, wl, wr, nn, Fx, it, gabs, gmul);
#pragma unroll
    for (int c = 0; c < 5; ++c) F[(size_t)c * n + i] = rc ? 0.0 : (double)Fx[c];
    iters[i] = rc ? -1 : it;
  }
}

int launch_flux_batch(const double *WL, const double *WR, const double *nrm, int n, double gamma,
                      double tol, int maxit, int precision, int bc, double *F, int *iters,
                      const uint32_t *mlp, cudaStream_t s) {
  int g = grid_for(n, 128, 16);
  bool g14 = gamma == 1.4;
  if (mlp) {
    int gm = grid_for(n, 128, 4);
    if (precision == FV_FP64) {
      GasT<double> G = GasT<double>::make(gamma, tol, maxit);
      if (g14)
        k_flux_batch_mlp<double, true><<<gm, 128, 0, s>>>(WL, WR, nrm, n, G, mlp, F, iters);
      else
        k_flux_batch_mlp<double, false><<<gm, 128, 0, s>>>(WL, WR, nrm, n, G, mlp, F, iters);
    } else {
      GasT<float> G = GasT<float>::make(gamma, tol > 2e-6 ? tol : 2e-6, maxit);
      if (g14)
        k_flux_batch_mlp<float, true><<<gm, 128, 0, s>>>(WL, WR, nrm, n, G, mlp, F, iters);
      else
        k_flux_batch_mlp<float, false><<<gm, 128, 0, s>>>(WL, WR, nrm, n, G, mlp, F, iters);
    }
    FV_LAUNCH_CHECK();
    return FV_OK;
  }
  if (precision == FV_FP64) {
    GasT<double> G = GasT<double>::make(gamma, tol, maxit);
    if (g14)
      k_flux_batch<double, true><<<g, 128, 0, s>>>(WL, WR, nrm, n, G, bc, F, iters);
    else
      k_flux_batch<double, false><<<g, 128, 0, s>>>(WL, WR, nrm, n, G, bc, F, iters);
  } else {
    GasT<float> G = GasT<float>::make(gamma, tol > 2e-6 ? tol : 2e-6, maxit);
    if (g14)
      k_flux_batch<float, true><<<g, 128, 0, s>>>(WL, WR, nrm, n, G, bc, F, iters);
    else
      k_flux_batch<float, false><<<g, 128, 0, s>>>(WL, WR, nrm, n, G, bc, F, iters);
  }
  FV_LAUNCH_CHECK();
  return FV_OK;
}

// ================================================================ hosts ==
void init_device_info() { num_sms(); }

// launch with a programmatic dependency on the previous kernel of the stream
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// the three parts of the level assignment: local steps and their minimum;
// levels from dt_min (classification and smoothing); keys and sorted lists.
// A sharded run puts the global minimum in between the first two and the
// owners' levels of its ghost cells in between the last two.
int launch_levels_local_dt(const DevMesh &d, cudaStream_t s) {
  int g = grid_for(d.N, 256, 8);
  launch_pdl(k_init_min2, 1, 1, s, d.dtmin_bits, d.dthi_bits);
  launch_pdl(k_dt32, g, 256, s, d);
  launch_pdl(k_dt_min_exact, g, 256, s, d);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

__global__ void k_set_bits(unsigned long long *bits, unsigned long long v) { *bits = v; }

int launch_set_dt_min(const DevMesh &d, double dt_min, cudaStream_t s) {
  unsigned long long v;
  memcpy(&v, &dt_min, sizeof v);
  launch_pdl(k_set_bits, 1, 1, s, d.dtmin_bits, v);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

int launch_levels_classify(const DevMesh &d, int L, cudaStream_t s) {
  int g = grid_for(d.N, 256, 8);
  launch_pdl(k_levels0_certified, g, 256, s, d);
  // L-1 Jacobi sweeps between lev_tmp and lev; the result must land in lev
  const int8_t *src = d.lev_tmp;
  int8_t *dst = d.lev;
  if (L == 1) {
    cudaMemcpyAsync(d.lev, d.lev_tmp, d.N, cudaMemcpyDeviceToDevice, s);
  } else {
    // with an even number of sweeps, start with a copy so the last one writes lev
    if ((L - 1) % 2 == 0) {
      cudaMemcpyAsync(d.lev, d.lev_tmp, d.N, cudaMemcpyDeviceToDevice, s);
      src = d.lev;
      dst = d.lev_tmp;
    }
    for (int sw = 0; sw < L - 1; ++sw) {
      launch_pdl(k_smooth, g, 256, s, d, src, dst, sw);
      const int8_t *t = dst;
      dst = (int8_t *)src;
      src = t;
    }
  }
  FV_LAUNCH_CHECK();
  return FV_OK;
}

template <int TILE>
static void launch_sort_tiles(const DevMesh &d, cudaStream_t s) {
  // cell keys (2L buckets) and face keys (L buckets), sorted together
  const int nc = (d.N + TILE - 1) / TILE, nf = (d.F + TILE - 1) / TILE;
  launch_pdl(k_keys_hist<TILE>, nc + nf, SORT_THREADS, s, d, nc, nf);
  launch_pdl(k_sort_scan2, 2, 1024, s, d, nc, nf);
  launch_pdl(k_sort_scatter2<TILE>, nc + nf, SORT_THREADS, s, d, nc, nf);
}

int launch_levels_sort(const DevMesh &d, cudaStream_t s) {
  if (d.N >= SORT_LARGE_CELLS)
    launch_sort_tiles<SORT_TILE1>(d, s);
  else
    launch_sort_tiles<SORT_TILE>(d, s);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

int launch_assign_levels(const DevMesh &d, int L, int *cnt_scratch, ProfHook *ph, cudaStream_t s) {
  (void)cnt_scratch;  // d.sort_cnt
  ProfScope scope(ph, FV_PROF_LEVELS, s);
  int rc = launch_levels_local_dt(d, s);
  if (rc == FV_OK) rc = launch_levels_classify(d, L, s);
  if (rc == FV_OK) rc = launch_levels_sort(d, s);
  return rc;
}

template <typename T, bool G14>
static void phase1_all(const DevMesh &d, const PhaseDesc &pd, const GasT<T> &G, const LaunchCfg &lc,
                       ProfHook *ph, cudaStream_t s) {
  const int g0 = grid_for(d.N, 256, lc.per_sm[0]), g1 = grid_for(d.N, 256, lc.per_sm[1]);
  const int g2 = grid_for(d.F, 128, lc.per_sm[2]), g3 = grid_for(d.N, 256, lc.per_sm[3]);
  if (pd.stage == 4) {  // a commit (order 1) updates cells only
    ProfScope sc(ph, FV_PROF_UPDATE, s);
    launch_pdl(k_phase1<K_COMMIT, T, G14>, g3, 256, s, d, pd, G);
    return;
  }
  if (sizeof(T) == 8) {  // FP32-flux mode: primitives computed inside the gradient kernel
    ProfScope sc(ph, FV_PROF_PRIM, s);
    launch_pdl(k_phase1<K_PRIM, T, G14>, g0, 256, s, d, pd, G);
  }
  { ProfScope sc(ph, FV_PROF_GRAD, s); launch_pdl(k_phase1<K_GRAD, T, G14>, g1, 256, s, d, pd, G); }
  {
    ProfScope sc(ph, FV_PROF_FLUX, s);
    if (d.guess == FV_GUESS_MLP)
      launch_pdl(k_flux_mlp1<T, G14>,
                 grid_for(d.F, 128, lc.per_sm[2] < FV_MLP_FLUX_BLOCKS ? lc.per_sm[2] : FV_MLP_FLUX_BLOCKS),
                 128, s, d, pd, G);
    else {
      bool staged = false;
      if constexpr (sizeof(T) == 4) {
        if (d.fuse_faces == 0 && d.flux_staged) {
          launch_pdl(k_flux_staged<G14>,
                     grid_for(d.F, FLUX_STAGE_THREADS,
                              lc.per_sm[2] < FV_STAGED_BLOCKS ? lc.per_sm[2] : FV_STAGED_BLOCKS),
                     FLUX_STAGE_THREADS, s, d, pd, G);
          staged = true;
        }
      }
      if (!staged) launch_pdl(k_phase1<K_FLUX, T, G14>, g2, 128, s, d, pd, G);
    }
    if constexpr (sizeof(T) == 4)
      if (d.guess == FV_GUESS_TWO_RAREFACTION && d.fuse_faces > 0)
        launch_pdl(k_flux_fused<G14>,
                   grid_for(d.F, 128, lc.per_sm[2] < FV_FUSED_BLOCKS ? lc.per_sm[2] : FV_FUSED_BLOCKS), 128, s,
                   d, pd, G);
  }
  {
    ProfScope sc(ph, FV_PROF_UPDATE, s);
    if (pd.stage == 3)
      launch_pdl(k_phase1<K_CORR, T, G14>, g3, 256, s, d, pd, G);
    else if (d.gather_quad && !(sizeof(T) == 4 && pd.stage == 1 && d.pred_sum64))
      launch_pdl(k_update_quad<T>, grid_for(4 * (int64_t)d.N, 256, lc.per_sm[3]), 256, s, d, pd);
    else
      launch_pdl(k_phase1<K_UPD, T, G14>, g3, 256, s, d, pd, G);
  }
}

static GasT<double> gas64(const DevMesh &d) { return GasT<double>::make(d.gamma, d.tol, d.maxit); }
static GasT<float> gas32(const DevMesh &d) {
  return GasT<float>::make(d.gamma, d.tol > 2e-6 ? d.tol : 2e-6, d.maxit);
}

int launch_persistent_cycle(const DevMesh &d, const PhaseDesc *pds, int nph, GridBar *bar,
                            cudaStream_t s) {
  if (cudaMemsetAsync(bar, 0, sizeof(GridBar), s) != cudaSuccess) return FV_ERR_CUDA;
  const bool g14 = d.gamma == 1.4;
  int rc;
  if (d.precision == FV_FP64)
    rc = g14 ? persist_launch<double, true>(d, pds, nph, gas64(d), bar, s)
             : persist_launch<double, false>(d, pds, nph, gas64(d), bar, s);
  else
    rc = g14 ? persist_launch<float, true>(d, pds, nph, gas32(d), bar, s)
             : persist_launch<float, false>(d, pds, nph, gas32(d), bar, s);
  return rc;
}

int launch_phase(const DevMesh &d, const PhaseDesc &pd, const LaunchCfg &lc, ProfHook *ph,
                 cudaStream_t s) {
  const bool g14 = d.gamma == 1.4;
  if (d.precision == FV_FP64) {
    if (g14) phase1_all<double, true>(d, pd, gas64(d), lc, ph, s);
    else phase1_all<double, false>(d, pd, gas64(d), lc, ph, s);
  } else {
    if (g14) phase1_all<float, true>(d, pd, gas32(d), lc, ph, s);
    else phase1_all<float, false>(d, pd, gas32(d), lc, ph, s);
  }
  FV_LAUNCH_CHECK();
  return FV_OK;
}

template <typename T, bool G14>
static void phaseN_all(const DevMesh *ms, const PhaseDesc *pds, int n, const GasT<T> &G,
                       int64_t cells, int64_t faces, const LaunchCfg &lc, const uint32_t *mlp,
                       cudaStream_t s) {
  const int g0 = grid_for(cells, 256, lc.per_sm[0]), g1 = grid_for(cells, 256, lc.per_sm[1]);
  const int g2 = grid_for(faces, 128, lc.per_sm[2]), g3 = grid_for(cells, 256, lc.per_sm[3]);
  if (sizeof(T) == 8) launch_pdl(k_phaseN<K_PRIM, T, G14>, g0, 256, s, ms, pds, n, G);
  launch_pdl(k_phaseN<K_GRAD, T, G14>, g1, 256, s, ms, pds, n, G);
  if (mlp)
    launch_pdl(k_flux_mlpN<T, G14>,
               grid_for(faces, 128, lc.per_sm[2] < FV_MLP_FLUX_BLOCKS ? lc.per_sm[2] : FV_MLP_FLUX_BLOCKS),
               128, s, ms, pds, n, G, mlp);
  else
    launch_pdl(k_phaseN<K_FLUX, T, G14>, g2, 128, s, ms, pds, n, G);
  launch_pdl(k_phaseN<K_UPD, T, G14>, g3, 256, s, ms, pds, n, G);
}

int launch_phase_multi(const DevMesh *ms, const PhaseDesc *pds, int n, const DevMesh &d0,
                       int64_t max_cells, int64_t max_faces, const LaunchCfg &lc, const uint32_t *mlp,
                       cudaStream_t s) {
  const bool g14 = d0.gamma == 1.4;
  if (d0.precision == FV_FP64) {
    if (g14) phaseN_all<double, true>(ms, pds, n, gas64(d0), max_cells, max_faces, lc, mlp, s);
    else phaseN_all<double, false>(ms, pds, n, gas64(d0), max_cells, max_faces, lc, mlp, s);
  } else {
    if (g14) phaseN_all<float, true>(ms, pds, n, gas32(d0), max_cells, max_faces, lc, mlp, s);
    else phaseN_all<float, false>(ms, pds, n, gas32(d0), max_cells, max_faces, lc, mlp, s);
  }
  FV_LAUNCH_CHECK();
  return FV_OK;
}

int launch_residual(const DevMesh &d, int precision, const PhaseLevels &pl, int level, void *Wbuf,
                    double *FAt, double *R, const int *new2old, cudaStream_t s) {
  (void)Wbuf;
  int gc = grid_for(d.N, 256, 8);
  int gfx = grid_for(d.F, 128, 16);
  const bool g14 = d.gamma == 1.4;
  if (precision == FV_FP64) {
    double *W = (double *)d.W;
    GasT<double> G = gas64(d);
    k_prim_all<double><<<gc, 256, 0, s>>>(d, pl, W);
    k_grad_all<double><<<gc, 256, 0, s>>>(d, pl);
    if (g14)
      k_flux_all<double, true><<<gfx, 128, 0, s>>>(d, G, level, W, d.G, d.fgeo, FAt);
    else
      k_flux_all<double, false><<<gfx, 128, 0, s>>>(d, G, level, W, d.G, d.fgeo, FAt);
  } else {
    float *W = (float *)d.W;
    GasT<float> G = gas32(d);
    // the FP32 gradient pass writes every cell's primitives too (view pl)
    k_grad_all<float><<<gc, 256, 0, s>>>(d, pl);
    if (g14)
      k_flux_all<float, true><<<gfx, 128, 0, s>>>(d, G, level, W, d.G32, d.fgeo32, FAt);
    else
      k_flux_all<float, false><<<gfx, 128, 0, s>>>(d, G, level, W, d.G32, d.fgeo32, FAt);
  }
  k_residual<<<gc, 256, 0, s>>>(d, level, FAt, R, new2old);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

// Riemann pairs of the current state U^n for training the learned guess:
// pair j is face (a j + b) mod F (a coprime with F, so no face repeats within
// a call), written as (rho, u_n, p) left and right in the face frame; a wall
// face gives its mirrored problem
template <typename T>
__global__ void __launch_bounds__(128) k_harvest(DevMesh d, const T *__restrict__ W, const T *__restrict__ Gr,
                                                 const T *__restrict__ fgeo, double *__restrict__ out,
                                                 int m, long long a, long long b) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    int f = (int)((a * (long long)j + b) % (long long)d.F);
    T WL[5], WR[5], n[3], A;
    int R = face_states<T>(d, W, Gr, fgeo, f, d.fcell[f], WL, WR, n, A);
    T unL = (WL[1] * n[0] + WL[2] * n[1]) + WL[3] * n[2];
    T unR = (WR[1] * n[0] + WR[2] * n[1]) + WR[3] * n[2];
    if (R == -FV_BC_WALL) unR = -unL;
    double *o = out + 6 * (size_t)j;
    o[0] = (double)WL[0];
    o[1] = (double)unL;
    o[2] = (double)WL[4];
    o[3] = (double)WR[0];
    o[4] = (double)unR;
    o[5] = (double)WR[4];
  }
}

int launch_harvest(const DevMesh &d, double *out, int m, long long a, long long b, cudaStream_t s) {
  int gc = grid_for(d.N, 256, 8);
  PhaseLevels pl;  // every level at U^n
  memset(&pl, 0, sizeof pl);
  int gh = grid_for(m, 128, 8);
  if (d.precision == FV_FP64) {
    double *W = (double *)d.W;
    k_prim_all<double><<<gc, 256, 0, s>>>(d, pl, W);
    k_grad_all<double><<<gc, 256, 0, s>>>(d, pl);
    k_harvest<double><<<gh, 128, 0, s>>>(d, W, d.G, d.fgeo, out, m, a, b);
  } else {
    float *W = (float *)d.W;
    k_grad_all<float><<<gc, 256, 0, s>>>(d, pl);
    k_harvest<float><<<gh, 128, 0, s>>>(d, W, d.G32, d.fgeo32, out, m, a, b);
  }
  FV_LAUNCH_CHECK();
  return FV_OK;
}

int launch_assign_multi(const DevMesh *ms, const int *active, int n, int Lmax, int64_t max_cells,
                        int64_t max_faces, int64_t max_cell_blocks, int64_t max_face_blocks,
                        int *cnt_scratch, const int *blk_pref_c, const int *blk_pref_f, cudaStream_t s) {
  (void)max_cells;
  (void)max_faces;
  (void)cnt_scratch;
  MultiTiles ac{ms, active, blk_pref_c, n}, af{ms, active, blk_pref_f, n};
  const int gc = (int)max_cell_blocks, gf = (int)max_face_blocks;
  k_init_min_multi<<<1, FV_MAXB, 0, s>>>(ms, active, n);
  k_dt_multi<<<gc, 256, 0, s>>>(ac, 0);
  k_dt_multi<<<gc, 256, 0, s>>>(ac, 1);
  k_cells_multi<<<gc, 256, 0, s>>>(ac, 0);
  // Lmax-1 sweeps for every instance (extra sweeps keep the fixed point); the
  // last one must write lev
  int sweeps = Lmax - 1;
  bool from_tmp = true;
  if (sweeps % 2 == 0) {
    k_cells_multi<<<gc, 256, 0, s>>>(ac, 1);
    from_tmp = false;
  }
  for (int sw = 0; sw < sweeps; ++sw) {
    k_cells_multi<<<gc, 256, 0, s>>>(ac, from_tmp ? 2 : 3);
    from_tmp = !from_tmp;
  }
  k_cells_multi<<<gc, 256, 0, s>>>(ac, 4);
  k_sort_hist_multi<<<gc, SORT_THREADS, 0, s>>>(ac, 0);
  k_sort_scan_multi<<<n, 1024, 0, s>>>(ms, active, 0);
  k_sort_scatter_multi<<<gc, SORT_THREADS, 0, s>>>(ac, 0);
  k_face_keys_multi<<<gf, 256, 0, s>>>(af);
  k_sort_hist_multi<<<gf, SORT_THREADS, 0, s>>>(af, 1);
  k_sort_scan_multi<<<n, 1024, 0, s>>>(ms, active, 1);
  k_sort_scatter_multi<<<gf, SORT_THREADS, 0, s>>>(af, 1);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

int launch_time_advance_multi(const DevMesh *ms, const PhaseDesc *pds, int n, cudaStream_t s) {
  k_time_advance_multi<<<1, FV_MAXB, 0, s>>>(ms, pds, n);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

int launch_time_advance(const DevMesh &d, int theta, cudaStream_t s) {
  k_time_advance<<<1, 1, 0, s>>>(d, theta);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

int launch_set_state(const DevMesh &d, const double *prim, const int *new2old, cudaStream_t s) {
  k_set_state<<<grid_for(d.N, 256, 8), 256, 0, s>>>(d, prim, new2old);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

// zero the [REC_FA] double records of the listed faces
__global__ void __launch_bounds__(256) k_zero_faces(double *__restrict__ rec, const int *__restrict__ faces, int n) {
  const double z[REC_FA] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    strec<REC_FA>(rec + (size_t)faces[i] * REC_FA, z);
}

int launch_zero_faces(double *rec, const int *faces, int n, cudaStream_t s) {
  if (n <= 0) return FV_OK;
  k_zero_faces<<<grid_for(n, 256, 8), 256, 0, s>>>(rec, faces, n);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

int launch_set_cons(const DevMesh &d, const double *cons, const int *new2old, cudaStream_t s) {
  k_set_cons<<<grid_for(d.N, 256, 8), 256, 0, s>>>(d, cons, new2old);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

int launch_get_state(const DevMesh &d, double *cons, const int *new2old, cudaStream_t s) {
  k_get_state<<<grid_for(d.N, 256, 8), 256, 0, s>>>(d, cons, new2old);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

int launch_get_levels(const DevMesh &d, int8_t *lev, const int *new2old, cudaStream_t s) {
  k_get_levels<<<grid_for(d.N, 256, 8), 256, 0, s>>>(d, lev, new2old);
  FV_LAUNCH_CHECK();
  return FV_OK;
}

}  // namespace fvk

// fv_mlp.cu -- the learned starting guess of the exact Riemann solver's Newton
// iteration (Sec. 2.1: Godunov fluxes from the exact face Riemann problem;
// the network itself is not in the paper): labelling of harvested Riemann
// pairs, FP32 training kernels (forward + backward per tile, deterministic
// reduction, Adam), packing to bfloat16 fragments, standalone inference, and
// the C ABI that installs the network in a mesh's flux kernel.
//
// Training is deterministic: every sum runs in a fixed order (samples of a
// tile in order inside a block, blocks in order in the reduction), so the
// same data, seed and launch give the same weights bit for bit.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fv_internal.h"
#include "fv_mlp.cuh"
#include "fv_riemann.cuh"

namespace fvk {

constexpr int TILE = 128;        // samples per block tile (one per thread)
constexpr int TS = TILE + 1;     // padded row stride of the per-sample arrays
constexpr int WPAD = 4676;       // parameters staged in shared memory (float4 multiple)

// shared-memory layout of k_mlp_fwdbwd (floats)
constexpr int SM_W = 0;
constexpr int SM_H1 = SM_W + WPAD;
constexpr int SM_D1 = SM_H1 + MLP_H * TS;   // gelu'(a1), then d1
constexpr int SM_H2 = SM_D1 + MLP_H * TS;
constexpr int SM_D2 = SM_H2 + MLP_H * TS;   // gelu'(a2), then d2
constexpr int SM_X = SM_D2 + MLP_H * TS;
constexpr int SM_DY = SM_X + MLP_NIN * TS;
constexpr int SM_ACC = SM_DY + TS;
constexpr int SM_LOSS = SM_ACC + WPAD;
constexpr int SM_FLOATS = SM_LOSS + TILE;
constexpr size_t SM_BYTES = sizeof(float) * SM_FLOATS;
static_assert(SM_BYTES <= 227 * 1024, "fwd/bwd tile exceeds shared memory");

// training activation: the tanh form in FP32 and its derivative
__device__ __forceinline__ float gelu_train(float x, float &dg) {
  const float K = 0.7978845608028654f, C = 0.044715f;
  float x2 = x * x;
  float th = tanhf(K * (x + C * x2 * x));
  dg = 0.5f * (1.0f + th) + 0.5f * x * (1.0f - th * th) * (K * (1.0f + 3.0f * C * x2));
  return 0.5f * x * (1.0f + th);
}

// forward and backward of the mean squared loss over `count` samples
// (sample k is sel[k], or k), tiles of 128 samples round-robin over the
// blocks; each block writes its partial gradient sum (in order of its tiles,
// samples in order within a tile) to part[block] and its partial loss sum.
__global__ void __launch_bounds__(TILE, 1) k_mlp_fwdbwd(const float *__restrict__ theta,
                                                       const float *__restrict__ X,
                                                       const float *__restrict__ Y,
                                                       const int *__restrict__ sel, int count,
                                                       float inv_n, float *__restrict__ part,
                                                       float *__restrict__ lossp) {
  extern __shared__ __align__(16) float sm[];
  float *w = sm + SM_W;
  float *H1 = sm + SM_H1, *D1 = sm + SM_D1, *H2 = sm + SM_H2, *D2 = sm + SM_D2;
  float *Xs = sm + SM_X, *DY = sm + SM_DY, *ACC = sm + SM_ACC, *LS = sm + SM_LOSS;
  const int s = threadIdx.x;
  for (int k = s; k < WPAD; k += TILE) {
    w[k] = k < MLP_NPARAM ? theta[k] : 0.0f;
    ACC[k] = 0.0f;
  }
  __syncthreads();
  const float *W1 = w + MP_W1, *b1 = w + MP_B1, *b2 = w + MP_B2, *w3 = w + MP_W3;
  const float4 *W2v = reinterpret_cast<const float4 *>(w + MP_W2);
  float lsum = 0.0f;
  const int ntiles = (count + TILE - 1) / TILE;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int pos = tile * TILE + s;
    const bool valid = pos < count;
    const int sid = valid ? (sel ? sel[pos] : pos) : 0;
    float x[MLP_NIN];
#pragma unroll
    for (int i = 0; i < MLP_NIN; ++i) {
      x[i] = valid ? X[(size_t)MLP_NIN * sid + i] : 0.0f;
      Xs[i * TS + s] = x[i];
    }
    // layer 1
    float h[MLP_H];
#pragma unroll
    for (int o = 0; o < MLP_H; ++o) {
      float a = b1[o];
#pragma unroll
      for (int i = 0; i < MLP_NIN; ++i) a += W1[o * MLP_NIN + i] * x[i];
      float dg;
      h[o] = gelu_train(a, dg);
      H1[o * TS + s] = h[o];
      D1[o * TS + s] = dg;
    }
    // layer 2 and the output
    float y = w[MP_B3];
    for (int o = 0; o < MLP_H; ++o) {
      float a = b2[o];
#pragma unroll
      for (int q = 0; q < MLP_H / 4; ++q) {
        float4 r = W2v[o * (MLP_H / 4) + q];
        a += r.x * h[4 * q] + r.y * h[4 * q + 1] + r.z * h[4 * q + 2] + r.w * h[4 * q + 3];
      }
      float dg;
      float h2 = gelu_train(a, dg);
      H2[o * TS + s] = h2;
      D2[o * TS + s] = dg;
      y += w3[o] * h2;
    }
    const float e = valid ? y - Y[sid] : 0.0f;
    lsum += e * e;
    const float dy = 2.0f * e * inv_n;
    DY[s] = dy;
    // backward: d2 = dy w3 gelu'(a2); d1 = (W2^T d2) gelu'(a1)
    float s1[MLP_H];
#pragma unroll
    for (int i = 0; i < MLP_H; ++i) s1[i] = 0.0f;
    for (int o = 0; o < MLP_H; ++o) {
      float d2 = dy * w3[o] * D2[o * TS + s];
      D2[o * TS + s] = d2;
#pragma unroll
      for (int q = 0; q < MLP_H / 4; ++q) {
        float4 r = W2v[o * (MLP_H / 4) + q];
        s1[4 * q] += r.x * d2;
        s1[4 * q + 1] += r.y * d2;
        s1[4 * q + 2] += r.z * d2;
        s1[4 * q + 3] += r.w * d2;
      }
    }
#pragma unroll
    for (int i = 0; i < MLP_H; ++i) D1[i * TS + s] *= s1[i];
    __syncthreads();
    // parameter gradients of this tile, summed over its samples in order
    for (int k = s; k < MLP_NPARAM; k += TILE) {
      float g = 0.0f;
      if (k < MP_B1) {
        const float *a = D1 + (k / MLP_NIN) * TS, *b = Xs + (k % MLP_NIN) * TS;
        for (int j = 0; j < TILE; ++j) g += a[j] * b[j];
      } else if (k < MP_W2) {
        const float *a = D1 + (k - MP_B1) * TS;
        for (int j = 0; j < TILE; ++j) g += a[j];
      } else if (k < MP_B2) {
        const int q = k - MP_W2;
        const float *a = D2 + (q / MLP_H) * TS, *b = H1 + (q % MLP_H) * TS;
        for (int j = 0; j < TILE; ++j) g += a[j] * b[j];
      } else if (k < MP_W3) {
        const float *a = D2 + (k - MP_B2) * TS;
        for (int j = 0; j < TILE; ++j) g += a[j];
      } else if (k < MP_B3) {
        const float *b = H2 + (k - MP_W3) * TS;
        for (int j = 0; j < TILE; ++j) g += DY[j] * b[j];
      } else {
        for (int j = 0; j < TILE; ++j) g += DY[j];
      }
      ACC[k] += g;
    }
    __syncthreads();
  }
  float *dst = part + (size_t)blockIdx.x * MLP_NPARAM;
  for (int k = s; k < MLP_NPARAM; k += TILE) dst[k] = ACC[k];
  LS[s] = lsum;
  __syncthreads();
  if (s == 0) {
    float t = 0.0f;
    for (int j = 0; j < TILE; ++j) t += LS[j];
    lossp[blockIdx.x] = t;
  }
}

// sum of the blocks' partial gradients in block order; then either store
// the gradient or take one Adam step (bias corrections c1 = 1 - b1^t,
// c2 = 1 - b2^t).  Block 0 also writes the mean loss.
template <bool ADAM>
__global__ void __launch_bounds__(256) k_mlp_reduce(const float *__restrict__ part, int nblk,
                                                    const float *__restrict__ lossp, float inv_n,
                                                    float *__restrict__ grad, float *__restrict__ loss,
                                                    float *__restrict__ theta, float *__restrict__ m,
                                                    float *__restrict__ v, float lr, float b1, float b2,
                                                    float c1, float c2, float eps) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < MLP_NPARAM) {
    float g = 0.0f;
    for (int b = 0; b < nblk; ++b) g += part[(size_t)b * MLP_NPARAM + k];
    if (ADAM) {
      float mk = b1 * m[k] + (1.0f - b1) * g;
      float vk = b2 * v[k] + (1.0f - b2) * g * g;
      m[k] = mk;
      v[k] = vk;
      theta[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    } else {
      grad[k] = g;
    }
  }
  if (k == 0 && loss) {
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += (double)lossp[b];
    *loss = (float)(t * (double)inv_n);
  }
}

// FP32 parameters -> fragment-ordered bfloat16 weights + FP32 biases
__global__ void k_mlp_pack(const float *__restrict__ th, int target, float gate, uint32_t *__restrict__ pk) {
  for (int wd = threadIdx.x; wd < PK_WORDS; wd += blockDim.x) {
    uint32_t val = 0u;
    if (wd < PK_W2) {
      // m16n8k8 B fragment: k = 2t, 2t+1 of hidden unit n = 8j + g
      const int j = wd / 32, lane = wd % 32, g = lane >> 2, t = lane & 3, n = 8 * j + g;
      const int k0 = 2 * t;
      float lo = k0 < MLP_NIN ? th[MP_W1 + n * MLP_NIN + k0] : 0.0f;
      float hi = k0 + 1 < MLP_NIN ? th[MP_W1 + n * MLP_NIN + k0 + 1] : 0.0f;
      val = pack_bf16x2(lo, hi);
    } else if (wd < PK_B1) {
      // m16n8k16 B fragment of k-step kk, n-tile j: register r holds
      // k = 16 kk + 2t + 8r (+1) of unit n = 8j + g
      const int q = wd - PK_W2, r = q & 1, idx = q >> 1;
      const int lane = idx % 32, j = (idx / 32) % 8, kk = idx / 256;
      const int g = lane >> 2, t = lane & 3, n = 8 * j + g, k0 = 16 * kk + 2 * t + 8 * r;
      val = pack_bf16x2(th[MP_W2 + n * MLP_H + k0], th[MP_W2 + n * MLP_H + k0 + 1]);
    } else if (wd < PK_B2) {
      val = __float_as_uint(th[MP_B1 + (wd - PK_B1)]);
    } else if (wd < PK_W3) {
      val = __float_as_uint(th[MP_B2 + (wd - PK_B2)]);
    } else if (wd < PK_B3) {
      val = __float_as_uint(th[MP_W3 + (wd - PK_W3)]);
    } else if (wd == PK_B3) {
      val = __float_as_uint(th[MP_B3]);
    } else if (wd == PK_TARGET) {
      val = (uint32_t)target;
    } else if (wd == PK_GATE) {
      val = __float_as_uint(gate);
    }
    pk[wd] = val;
  }
}

// standalone bfloat16 inference (the flux kernel's device function)
template <bool EXACT>
__global__ void __launch_bounds__(128, 4) k_mlp_infer(const uint32_t *__restrict__ pk,
                                                      const float *__restrict__ X, int n,
                                                      float *__restrict__ Y) {
  __shared__ __align__(16) uint32_t sw[PK_WORDS];
  mlp_stage(sw, pk);
  const int lane = threadIdx.x & 31;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x - lane); base < n;
       base += gridDim.x * blockDim.x) {
    const int i = base + lane;
    const bool ok = i < n;
    float x[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) x[c] = ok ? X[6 * (size_t)i + c] : (c == 1 || c == 4 ? 0.0f : 1.0f);
    __syncwarp();
    float y = mlp_eval_warp<EXACT>(sw, x);
    if (ok) Y[i] = y;
  }
}

// labels of harvested pairs: p* by the FP64 exact solver to a tight
// tolerance, the features, and the target log(p*/pbar) or
// log(p*/p_TR) / s(q)
__global__ void __launch_bounds__(128) k_mlp_label(const double *__restrict__ pairs, int n,
                                                   GasT<double> G, int target, float *__restrict__ X,
                                                   float *__restrict__ Y, double *__restrict__ pstar,
                                                   float *__restrict__ Q, int *__restrict__ status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double *q = pairs + 6 * (size_t)i;
    double ps = 0.0, us = 0.0;
    int it = 0;
    int rc = riemann_star<double>(G, q[0], q[1], q[2], q[3], q[4], q[5], ps, us, it);
    float x[6];
    float pb = mlp_features<double>(G.g, q[0], q[1], q[2], q[3], q[4], q[5], x);
#pragma unroll
    for (int c = 0; c < 6; ++c) X[6 * (size_t)i + c] = x[c];
    double aL = sqrt(G.g * q[2] / q[0]), aR = sqrt(G.g * q[5] / q[3]);
    double num = aL + aR - 0.5 * G.gm1 * (q[4] - q[1]);
    double den = aL / pow(q[2], G.z) + aR / pow(q[5], G.z);
    double ptr = pow(num / den, G.inv_z);
    double qs = ptr / fmin(q[2], q[5]) - 1.0;
    if (Q) Q[i] = (float)qs;
    if (rc) {
      atomicOr(status, 1);
      ps = nan("");
    }
    pstar[i] = ps;
    double y;
    if (target == 0) {
      y = log(ps / (double)pb);
    } else {
      double r = qs / (1.0 + qs), sc = qs > 0.0 ? r * r * r : 0.0;
      y = sc > 0.0 ? log(ps / ptr) / sc : 0.0;
    }
    Y[i] = (float)y;
  }
}

int launch_mlp_pack(const float *params, int target, float gate, uint32_t *packed, cudaStream_t s) {
  k_mlp_pack<<<1, 256, 0, s>>>(params, target, gate, packed);
  return cudaGetLastError() == cudaSuccess ? FV_OK : FV_ERR_CUDA;
}

}  // namespace fvk

using namespace fvk;

// ===================================================================== C ABI
namespace {

int mfail(int code, const std::string &msg) {
  fv_internal_set_error(msg);
  return code;
}

#define MCK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return mfail(FV_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// splitmix64 (Steele, Lea, Flood 2014): the shuffles' and the
// initialisation's random stream
struct SplitMix {
  uint64_t x;
  uint64_t next() {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

int fwdbwd_ready() {
  static int done = 0;
  if (!done) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_fwdbwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SM_BYTES);
    if (e != cudaSuccess) return mfail(FV_ERR_CUDA, std::string("fwd/bwd shared memory: ") + cudaGetErrorString(e));
    done = 1;
  }
  return FV_OK;
}

// one forward/backward over `count` samples into part / lossp; returns the
// number of partial blocks
int run_fwdbwd(const float *theta, const float *X, const float *Y, const int *sel, int count,
               float *part, float *lossp, int max_blocks, cudaStream_t s) {
  const int ntiles = (count + TILE - 1) / TILE;
  const int grid = ntiles < max_blocks ? ntiles : max_blocks;
  k_mlp_fwdbwd<<<grid, TILE, SM_BYTES, s>>>(theta, X, Y, sel, count, 1.0f / (float)count, part, lossp);
  return grid;
}

int gcd64(int64_t a, int64_t b) {
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return (int)a;
}

}  // namespace

extern "C" {

int fv_mlp_init(float *params, int n_params, uint64_t seed) {
  if (!params || n_params != MLP_NPARAM) return mfail(FV_ERR_INVALID_ARG, "fv_mlp_init: need 4673 parameters");
  SplitMix r{seed};
  auto fill = [&](int off, int fan_in, int fan_out, int count) {
    // Glorot-uniform: U(-a, a), a = sqrt(6 / (fan_in + fan_out))
    double a = std::sqrt(6.0 / (double)(fan_in + fan_out));
    for (int k = 0; k < count; ++k) params[off + k] = (float)((2.0 * r.uniform() - 1.0) * a);
  };
  std::memset(params, 0, sizeof(float) * MLP_NPARAM);
  fill(MP_W1, MLP_NIN, MLP_H, MLP_H * MLP_NIN);
  fill(MP_W2, MLP_H, MLP_H, MLP_H * MLP_H);
  fill(MP_W3, MLP_H, 1, MLP_H);
  return FV_OK;
}

int fv_mlp_pack(const float *params_dev, int n_params, int target, double gate, void *packed_dev,
                void *stream) {
  if (!params_dev || !packed_dev || n_params != MLP_NPARAM || (target != 0 && target != 1) ||
      !std::isfinite(gate) || gate > 1e38)
    return mfail(FV_ERR_INVALID_ARG, "fv_mlp_pack: bad argument");
  if ((uintptr_t)packed_dev % 16) return mfail(FV_ERR_INVALID_ARG, "fv_mlp_pack: packed buffer not 16-byte aligned");
  k_mlp_pack<<<1, 256, 0, (cudaStream_t)stream>>>(params_dev, target, (float)gate, (uint32_t *)packed_dev);
  MCK(cudaGetLastError());
  return FV_OK;
}

static int mlp_infer(const void *packed_dev, const float *x_dev, int64_t count, float *y_dev, void *stream,
                     bool exact) {
  if (!packed_dev || (count > 0 && (!x_dev || !y_dev)) || count < 0 || count > 0x7fffffff)
    return mfail(FV_ERR_INVALID_ARG, "fv_mlp_infer: bad argument");
  if ((uintptr_t)packed_dev % 16) return mfail(FV_ERR_INVALID_ARG, "fv_mlp_infer: packed buffer not 16-byte aligned");
  if (count == 0) return FV_OK;
  int n = (int)count;
  int grid = (n + 127) / 128, cap = 4 * sm_count();
  if (exact)
    k_mlp_infer<true><<<grid < cap ? grid : cap, 128, 0, (cudaStream_t)stream>>>((const uint32_t *)packed_dev, x_dev,
                                                                                 n, y_dev);
  else
    k_mlp_infer<false><<<grid < cap ? grid : cap, 128, 0, (cudaStream_t)stream>>>((const uint32_t *)packed_dev, x_dev,
                                                                                  n, y_dev);
  MCK(cudaGetLastError());
  return FV_OK;
}

int fv_mlp_infer(const void *packed_dev, const float *x_dev, int64_t count, float *y_dev, void *stream) {
  return mlp_infer(packed_dev, x_dev, count, y_dev, stream, false);
}

int fv_mlp_infer_exact_tanh(const void *packed_dev, const float *x_dev, int64_t count, float *y_dev,
                            void *stream) {
  return mlp_infer(packed_dev, x_dev, count, y_dev, stream, true);
}

int fv_mlp_label(const double *pairs_dev, int64_t count, double gamma, int target, float *x_dev,
                 float *y_dev, double *pstar_dev, float *q_dev, void *stream) {
  if (count < 0 || count > 0x7fffffff || !(gamma > 1.0) || (target != 0 && target != 1) ||
      (count > 0 && (!pairs_dev || !x_dev || !y_dev || !pstar_dev)))
    return mfail(FV_ERR_INVALID_ARG, "fv_mlp_label: bad argument");
  if (count == 0) return FV_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int *st = nullptr;
  MCK(cudaMalloc(&st, sizeof(int)));
  cudaMemsetAsync(st, 0, sizeof(int), s);
  GasT<double> G = GasT<double>::make(gamma, 1e-14, 100);
  int n = (int)count, grid = (n + 127) / 128, cap = 16 * sm_count();
  k_mlp_label<<<grid < cap ? grid : cap, 128, 0, s>>>(pairs_dev, n, G, target, x_dev, y_dev, pstar_dev, q_dev, st);
  int h = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(st);
  if (e != cudaSuccess) return mfail(FV_ERR_CUDA, std::string("fv_mlp_label: ") + cudaGetErrorString(e));
  if (h) return mfail(FV_ERR_RIEMANN, "fv_mlp_label: a pair has no star state (vacuum or no convergence)");
  return FV_OK;
}

int fv_mlp_loss_grad(const float *params_dev, const float *x_dev, const float *y_dev,
                     const int32_t *sel_dev, int64_t count, float *grad_dev, double *loss_out,
                     void *stream) {
  if (!params_dev || !x_dev || !y_dev || count <= 0 || count > 0x7fffffff)
    return mfail(FV_ERR_INVALID_ARG, "fv_mlp_loss_grad: bad argument");
  int rc = fwdbwd_ready();
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int maxb = 2 * sm_count();
  float *part = nullptr, *lossp = nullptr, *loss = nullptr, *g = grad_dev;
  MCK(cudaMalloc(&part, sizeof(float) * (size_t)maxb * MLP_NPARAM));
  cudaError_t e = cudaMalloc(&lossp, sizeof(float) * (maxb + 1));
  if (e == cudaSuccess && !g) e = cudaMalloc(&g, sizeof(float) * MLP_NPARAM);
  if (e == cudaSuccess) {
    loss = lossp + maxb;
    int nb = run_fwdbwd(params_dev, x_dev, y_dev, sel_dev, (int)count, part, lossp, maxb, s);
    k_mlp_reduce<false><<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(
        part, nb, lossp, 1.0f / (float)count, g, loss, nullptr, nullptr, nullptr, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
    e = cudaGetLastError();
  }
  float hl = 0.0f;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hl, loss, sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(part);
  cudaFree(lossp);
  if (g != grad_dev) cudaFree(g);
  if (e != cudaSuccess) return mfail(FV_ERR_CUDA, std::string("fv_mlp_loss_grad: ") + cudaGetErrorString(e));
  if (loss_out) *loss_out = (double)hl;
  return FV_OK;
}

int fv_mlp_adam(float *params_dev, float *m_dev, float *v_dev, const float *grad_dev, int step,
                double lr, double beta1, double beta2, double eps, void *stream) {
  if (!params_dev || !m_dev || !v_dev || !grad_dev || step < 1 || !(lr > 0.0) || !(beta1 >= 0.0) ||
      !(beta1 < 1.0) || !(beta2 >= 0.0) || !(beta2 < 1.0) || !(eps > 0.0))
    return mfail(FV_ERR_INVALID_ARG, "fv_mlp_adam: bad argument");
  // the gradient enters as one block's partial sum
  float c1 = (float)(1.0 - std::pow(beta1, step)), c2 = (float)(1.0 - std::pow(beta2, step));
  k_mlp_reduce<true><<<(MLP_NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      grad_dev, 1, nullptr, 0.f, nullptr, nullptr, params_dev, m_dev, v_dev, (float)lr, (float)beta1,
      (float)beta2, c1, c2, (float)eps);
  MCK(cudaGetLastError());
  return FV_OK;
}

int fv_mlp_train(float *params_dev, const float *x_dev, const float *y_dev, const int32_t *sel_host,
                 int64_t n_sel, const fv_train_config *tc, float *loss_hist_dev, void *stream) {
  if (!params_dev || !x_dev || !y_dev || !tc || n_sel <= 0 || n_sel > 0x7fffffff || tc->epochs < 1 ||
      tc->batch < 1 || tc->batch > (1 << 20) || !(tc->lr0 > 0.0) || !(tc->lr1 > 0.0) ||
      !(tc->beta1 >= 0.0 && tc->beta1 < 1.0) || !(tc->beta2 >= 0.0 && tc->beta2 < 1.0) || !(tc->eps > 0.0))
    return mfail(FV_ERR_INVALID_ARG, "fv_mlp_train: bad argument");
  int rc = fwdbwd_ready();
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = (int)n_sel, B = tc->batch;
  const int maxb = (B + TILE - 1) / TILE;
  const int64_t steps_per_epoch = (n + B - 1) / B, total = steps_per_epoch * tc->epochs;
  float *m = nullptr, *v = nullptr, *part = nullptr, *lossp = nullptr;
  int *idx = nullptr;
  MCK(cudaMalloc(&m, sizeof(float) * 2 * MLP_NPARAM));
  v = m + MLP_NPARAM;
  cudaError_t e = cudaMalloc(&part, sizeof(float) * (size_t)maxb * MLP_NPARAM);
  if (e == cudaSuccess) e = cudaMalloc(&lossp, sizeof(float) * maxb);
  if (e == cudaSuccess) e = cudaMalloc(&idx, sizeof(int) * (size_t)n);
  if (e == cudaSuccess) e = cudaMemsetAsync(m, 0, sizeof(float) * 2 * MLP_NPARAM, s);
  std::vector<int> perm(n), order(n);
  SplitMix r{tc->seed};
  int64_t step = 0;
  for (int ep = 0; ep < tc->epochs && e == cudaSuccess; ++ep) {
    // Fisher-Yates shuffle of the selected samples
    for (int k = 0; k < n; ++k) perm[k] = k;
    for (int k = n - 1; k > 0; --k) {
      int j = (int)(r.next() % (uint64_t)(k + 1));
      int t = perm[k];
      perm[k] = perm[j];
      perm[j] = t;
    }
    for (int k = 0; k < n; ++k) order[k] = sel_host ? sel_host[perm[k]] : perm[k];
    e = cudaStreamSynchronize(s);  // the previous epoch's copy of `order` is done
    if (e == cudaSuccess) e = cudaMemcpyAsync(idx, order.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, s);
    for (int64_t b = 0; b < steps_per_epoch && e == cudaSuccess; ++b, ++step) {
      const int off = (int)(b * B), cnt = n - off < B ? n - off : B;
      // cosine decay from lr0 to lr1
      const double frac = total > 1 ? (double)step / (double)(total - 1) : 1.0;
      const double lr = tc->lr1 + 0.5 * (tc->lr0 - tc->lr1) * (1.0 + std::cos(3.141592653589793 * frac));
      const int nb = run_fwdbwd(params_dev, x_dev, y_dev, idx + off, cnt, part, lossp, maxb, s);
      const float c1 = (float)(1.0 - std::pow(tc->beta1, (double)(step + 1)));
      const float c2 = (float)(1.0 - std::pow(tc->beta2, (double)(step + 1)));
      k_mlp_reduce<true><<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(
          part, nb, lossp, 1.0f / (float)cnt, nullptr, loss_hist_dev ? loss_hist_dev + step : nullptr,
          params_dev, m, v, (float)lr, (float)tc->beta1, (float)tc->beta2, c1, c2, (float)tc->eps);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(m);
  cudaFree(part);
  cudaFree(lossp);
  cudaFree(idx);
  if (e != cudaSuccess) return mfail(FV_ERR_CUDA, std::string("fv_mlp_train: ") + cudaGetErrorString(e));
  return FV_OK;
}

int fv_mlp_train_steps(const fv_train_config *tc, int64_t n_sel) {
  if (!tc || tc->batch < 1 || n_sel <= 0) return 0;
  return (int)(((n_sel + tc->batch - 1) / tc->batch) * tc->epochs);
}

int fv_mlp_load(fv_mesh *m, const float *params_dev, int n_params, int target, double gate) {
  if (!m || !params_dev || n_params != MLP_NPARAM || (target != 0 && target != 1) || !std::isfinite(gate) || gate > 1e38)
    return mfail(FV_ERR_INVALID_ARG, "fv_mlp_load: bad argument");
  if (m->in_batch || (m->in_cycle && m->next_phase > 0))
    return mfail(FV_ERR_INVALID_ARG, "fv_mlp_load: mesh is inside a cycle or a batch");
  MCK(cudaSetDevice(m->cfg.device));
  if (!m->d.mlp) {
    void *p = nullptr;
    MCK(cudaMalloc(&p, sizeof(uint32_t) * PK_WORDS));
    m->allocs.push_back(p);
    m->d.mlp = (const uint32_t *)p;
  }
  k_mlp_pack<<<1, 256>>>(params_dev, target, (float)gate, (uint32_t *)m->d.mlp);
  MCK(cudaGetLastError());
  MCK(cudaDeviceSynchronize());
  m->d.guess = FV_GUESS_MLP;
  m->cfg.guess = FV_GUESS_MLP;
  if (m->cycle_graph) {
    cudaGraphExecDestroy(m->cycle_graph);
    m->cycle_graph = nullptr;
  }
  return FV_OK;
}

int fv_set_guess(fv_mesh *m, int guess) {
  if (!m || (guess != FV_GUESS_TWO_RAREFACTION && guess != FV_GUESS_MLP))
    return mfail(FV_ERR_INVALID_ARG, "fv_set_guess: bad argument");
  if (guess == FV_GUESS_MLP && !m->d.mlp)
    return mfail(FV_ERR_INVALID_ARG, "fv_set_guess: no network loaded (fv_mlp_load)");
  if (m->in_batch || (m->in_cycle && m->next_phase > 0))
    return mfail(FV_ERR_INVALID_ARG, "fv_set_guess: mesh is inside a cycle or a batch");
  m->d.guess = guess;
  m->cfg.guess = guess;
  if (m->cycle_graph) {
    cudaGraphExecDestroy(m->cycle_graph);
    m->cycle_graph = nullptr;
  }
  return FV_OK;
}

int fv_harvest_pairs(fv_mesh *m, double *pairs_dev, int64_t count, uint64_t seed, void *stream) {
  if (!m || count < 0 || (count > 0 && !pairs_dev)) return mfail(FV_ERR_INVALID_ARG, "fv_harvest_pairs: bad argument");
  if (count > m->d.F) return mfail(FV_ERR_INVALID_ARG, "fv_harvest_pairs: more pairs than faces");
  if (m->in_cycle && m->next_phase > 0) return mfail(FV_ERR_INVALID_ARG, "fv_harvest_pairs: inside a cycle");
  if (count == 0) return FV_OK;
  MCK(cudaSetDevice(m->cfg.device));
  SplitMix r{seed};
  const int64_t F = m->d.F;
  int64_t a = (int64_t)(r.next() % (uint64_t)F) | 1;
  while (gcd64(a, F) != 1) a = (a + 2) % F;
  if (a == 0) a = 1;
  const int64_t b = (int64_t)(r.next() % (uint64_t)F);
  int rc = fvk::launch_harvest(m->d, pairs_dev, (int)count, a, b, (cudaStream_t)stream);
  if (rc) return mfail(rc, std::string("fv_harvest_pairs: launch failed: ") + cudaGetErrorString(cudaGetLastError()));
  return FV_OK;
}

int fv_godunov_flux_batch_mlp(const double *WL_dev, const double *WR_dev, const double *n_dev,
                              int64_t count, const fv_config *cfg, const void *packed_dev,
                              double *F_dev, int32_t *iters_dev, void *stream) {
  if (!WL_dev || !WR_dev || !n_dev || !cfg || !packed_dev || !F_dev || !iters_dev)
    return mfail(FV_ERR_INVALID_ARG, "fv_godunov_flux_batch_mlp: NULL argument");
  if (count < 0 || count > 0x7fffffff || !(cfg->gamma > 1.0) || !(cfg->newton_tol > 0.0) ||
      cfg->newton_max_iter < 1 || (cfg->precision != FV_FP64 && cfg->precision != FV_FP32_FLUX) ||
      (uintptr_t)packed_dev % 16)
    return mfail(FV_ERR_INVALID_ARG, "fv_godunov_flux_batch_mlp: bad argument");
  if (count == 0) return FV_OK;
  MCK(cudaSetDevice(cfg->device));
  int rc = fvk::launch_flux_batch(WL_dev, WR_dev, n_dev, (int)count, cfg->gamma, cfg->newton_tol,
                                  cfg->newton_max_iter, cfg->precision, FV_BC_INTERIOR, F_dev, iters_dev,
                                  (const uint32_t *)packed_dev, (cudaStream_t)stream);
  if (rc) return mfail(rc, "fv_godunov_flux_batch_mlp: launch failed");
  return FV_OK;
}

}  // extern "C"

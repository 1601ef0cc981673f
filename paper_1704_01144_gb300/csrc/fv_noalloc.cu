// fv_noalloc.cu -- level assignment on caller-owned device arrays that
// allocates nothing.
//
// Who needs it: code that cannot call cudaMalloc at the point where it wants
// the temporal levels -- for example a host application that hands the
// solver only memory from its own fixed-budget pool and accounts for every
// byte of it, or one that runs under an allocator which must see every
// device allocation, so that a library allocating behind its back breaks
// the budget.  Such a caller keeps its own dt[] and neighbour arrays on the
// device and gets the levels and dt_min written into buffers it owns.
//
// Scratch (the dt_min reduction word and the ping-pong level buffer of the
// smoothing sweeps) lives in one file-scope __device__ array of fixed size,
// so the entry point never allocates.  Every GPU that loads this library
// holds that array (FV_NOALLOC_MAX_CELLS + 256 bytes) until the process
// exits.  All calls share it: each call re-initialises what it needs, and
// calls whose kernels overlap on the GPU (different streams, or different
// host threads on the same device) race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "fv_internal.h"

#define FV_NOALLOC_MAX_DEVICES 64

// bytes [0, 8): bit pattern of dt_min; bytes [256, 256 + max cells): one
// int8 level per cell for the smoothing ping-pong
static __device__ __align__(256) unsigned char g_noalloc_scratch[256 + FV_NOALLOC_MAX_CELLS];

namespace {

void *g_scratch_addr[FV_NOALLOC_MAX_DEVICES];
std::mutex g_setup_mutex;

__global__ void k_na_init(unsigned long long *bits) { *bits = 0x7ff0000000000000ULL; }

__global__ void __launch_bounds__(256) k_na_min(const double *__restrict__ dt, int n,
                                                unsigned long long *bits) {
  double m = __longlong_as_double(0x7ff0000000000000LL);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = fmin(m, dt[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffff, m, o));
  __shared__ double sm[8];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : __longlong_as_double(0x7ff0000000000000LL);
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffff, v, o));
    if (threadIdx.x == 0) atomicMin(bits, (unsigned long long)__double_as_longlong(v));
  }
}

// k_i = max{k <= L-1 : 2^k dt_min <= dt_i}
__global__ void __launch_bounds__(256) k_na_levels0(const double *__restrict__ dt, int n, int L,
                                                    const unsigned long long *bits, int8_t *out) {
  double dtmin = __longlong_as_double((long long)*bits);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < L && ldexp(dtmin, k + 1) <= dt[i]) ++k;
    out[i] = (int8_t)k;
  }
}

// one Jacobi sweep k_i <- min(k_i, 1 + min over neighbours)
__global__ void __launch_bounds__(256) k_na_smooth(const int32_t *__restrict__ nbr, int n,
                                                   const int8_t *__restrict__ src,
                                                   int8_t *__restrict__ dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int k = src[i];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int nb = nbr[(size_t)j * n + i];
      if (nb >= 0 && nb < n) k = min(k, src[nb] + 1);
    }
    dst[i] = (int8_t)k;
  }
}

__global__ void k_na_finish(const unsigned long long *bits, double *dt_min_out) {
  *dt_min_out = __longlong_as_double((long long)*bits);
}

int na_fail(int code, const std::string &msg) {
  fv_internal_set_error(msg);
  return code;
}

}  // namespace

extern "C" int fv_assign_levels_noalloc(const double *dt_dev, const int32_t *nbr_dev,
                                        int64_t n_cells, int max_levels, int8_t *levels_dev,
                                        double *dt_min_dev, void *stream) {
  if (!dt_dev || !nbr_dev || !levels_dev || !dt_min_dev)
    return na_fail(FV_ERR_INVALID_ARG, "fv_assign_levels_noalloc: NULL pointer");
  if (n_cells < 1 || n_cells > FV_NOALLOC_MAX_CELLS)
    return na_fail(FV_ERR_INVALID_ARG,
                   "fv_assign_levels_noalloc: n_cells must be in [1, " +
                       std::to_string(FV_NOALLOC_MAX_CELLS) +
                       "] (the size of its static scratch), got " + std::to_string((long long)n_cells));
  if (max_levels < 1 || max_levels > FV_MAXL)
    return na_fail(FV_ERR_INVALID_ARG, "fv_assign_levels_noalloc: max_levels must be in [1, 8]");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return na_fail(FV_ERR_CUDA, std::string("fv_assign_levels_noalloc: cudaGetDevice: ") +
                                    cudaGetErrorString(e));
  if (dev < 0 || dev >= FV_NOALLOC_MAX_DEVICES)
    return na_fail(FV_ERR_INVALID_ARG, "fv_assign_levels_noalloc: current device " + std::to_string(dev) +
                                           " is beyond the " + std::to_string(FV_NOALLOC_MAX_DEVICES) +
                                           " devices whose scratch address it caches");
  // once per device, with that device current: the device address of the
  // static scratch (the host-side symbol is only a stand-in).  The address
  // is cached for the life of the process; a cudaDeviceReset destroys the
  // context it belongs to, and the library does not support use after one.
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return na_fail(FV_ERR_CUDA, std::string("fv_assign_levels_noalloc: cudaGetSymbolAddress: ") +
                                        cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long *bits = (unsigned long long *)base;
  int8_t *tmp = (int8_t *)((unsigned char *)base + 256);
  const int n = (int)n_cells;
  int dev_sms = 1;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev);
  int need = (n + 255) / 256;
  int grid = need < dev_sms * 8 ? need : dev_sms * 8;
  k_na_init<<<1, 1, 0, s>>>(bits);  // the reduction word must start at +inf
  k_na_min<<<grid, 256, 0, s>>>(dt_dev, n, bits);
  // L-1 sweeps; the last one must write into levels_dev
  int sweeps = max_levels - 1;
  int8_t *a = (sweeps % 2 == 0) ? levels_dev : tmp;
  int8_t *b = (sweeps % 2 == 0) ? tmp : levels_dev;
  k_na_levels0<<<grid, 256, 0, s>>>(dt_dev, n, max_levels, bits, a);
  for (int sw = 0; sw < sweeps; ++sw) {
    k_na_smooth<<<grid, 256, 0, s>>>(nbr_dev, n, a, b);
    int8_t *t = a;
    a = b;
    b = t;
  }
  k_na_finish<<<1, 1, 0, s>>>(bits, dt_min_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return na_fail(FV_ERR_CUDA, std::string("fv_assign_levels_noalloc: launch: ") + cudaGetErrorString(e));
  return FV_OK;
}

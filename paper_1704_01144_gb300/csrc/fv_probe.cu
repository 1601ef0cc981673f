// fv_probe.cu -- arithmetic peak probe: independent fused multiply-add
// chains (8 per thread, 256 threads per block, 16 blocks per SM), timed with
// CUDA events.  Gives the measured FP64 / FP32 FMA ceiling of the device for
// the roofline of the ALU-bound kernels.
#include <cuda_runtime.h>

#include <string>

#include "fv_internal.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T *out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == T(12345.678)) out[0] = s;  // keeps the chains alive
}

template <typename T>
int probe(int iters, double *tflops) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  T *out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return FV_ERR_NOMEM;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int blocks = sms * 16, threads = 256;
  k_fma_chain<T><<<blocks, threads>>>(out, iters / 8, T(0.999999), T(1e-7));  // warm-up
  cudaEventRecord(a);
  k_fma_chain<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-7));
  cudaEventRecord(b);
  cudaError_t e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess || ms <= 0.f) return FV_ERR_CUDA;
  double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return FV_OK;
}

}  // namespace

extern "C" int fv_probe_fma_peak(int device, int precision, double *tflops_out) {
  if (!tflops_out || (precision != FV_FP64 && precision != FV_FP32_FLUX)) {
    fv_internal_set_error("fv_probe_fma_peak: bad argument");
    return FV_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    fv_internal_set_error("fv_probe_fma_peak: cudaSetDevice failed");
    return FV_ERR_CUDA;
  }
  int rc = precision == FV_FP64 ? probe<double>(1 << 14, tflops_out) : probe<float>(1 << 18, tflops_out);
  if (rc) fv_internal_set_error("fv_probe_fma_peak: probe failed");
  return rc;
}

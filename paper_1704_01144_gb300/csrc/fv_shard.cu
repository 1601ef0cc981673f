// fv_shard.cu -- the ghost-cell exchange of a sharded run.
//
// The paper's distributed version (Sec. 3.3, and the MPI + task version of
// Sec. 4.3) splits the mesh into subdomains whose cells each belong to one
// subdomain; ghost cells hold copies of the neighbouring subdomains' border
// cells, and the border faces are computed on both sides.  Here a subdomain
// is an fv_mesh of its own cells plus ghost layers; a halo plan lists cells
// of one mesh (by the caller's order of that mesh's tets) whose records are
// packed into, or unpacked from, a flat device buffer that the caller moves
// between subdomains (a device copy, NCCL, or host staging).
//
// Packed per cell: the level (FV_HALO_LEVELS, one byte), or the state
// (FV_HALO_STATE, FV_HALO_STATE_DOUBLES doubles): U^n, and the predicted
// state of the mode -- FP64: U*; FP32-flux: the FP32 records of U^n and U*
// (bit copies) and, when allocated, the FP64 provisional end state of the
// paper's order.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "fv_internal.h"

struct fv_halo {
  fv_mesh *m = nullptr;
  int n = 0;
  int *cells_dev = nullptr;  // internal (renumbered) cell ids
};

namespace fvk {

__global__ void __launch_bounds__(256) k_halo(DevMesh d, const int *__restrict__ cells, int n, int what,
                                              void *buf, bool pack) {
  const size_t N = d.N;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int i = cells[k];
    if (what == FV_HALO_LEVELS) {
      int8_t *b = (int8_t *)buf;
      if (pack)
        b[k] = d.lev[i];
      else
        d.lev[i] = b[k];
      continue;
    }
    double *r = (double *)buf + (size_t)k * FV_HALO_STATE_DOUBLES;
    if (pack) {
#pragma unroll
      for (int c = 0; c < 5; ++c) r[c] = d.Un[c * N + i];
      if (d.Us) {
#pragma unroll
        for (int c = 0; c < 5; ++c) r[5 + c] = d.Us[c * N + i];
      } else {
        const double *a = (const double *)(d.Un32 + (size_t)i * REC_U32);
        const double *b = (const double *)(d.Us32 + (size_t)i * REC_U32);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          r[5 + q] = a[q];
          r[9 + q] = b[q];
        }
        if (d.UsD) {
#pragma unroll
          for (int c = 0; c < 5; ++c) r[13 + c] = d.UsD[c * N + i];
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < 5; ++c) d.Un[c * N + i] = r[c];
      if (d.Us) {
#pragma unroll
        for (int c = 0; c < 5; ++c) d.Us[c * N + i] = r[5 + c];
      } else {
        double *a = (double *)(d.Un32 + (size_t)i * REC_U32);
        double *b = (double *)(d.Us32 + (size_t)i * REC_U32);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a[q] = r[5 + q];
          b[q] = r[9 + q];
        }
        if (d.UsD) {
#pragma unroll
          for (int c = 0; c < 5; ++c) d.UsD[c * N + i] = r[13 + c];
        }
      }
    }
  }
}

int launch_halo(const DevMesh &d, const int *cells, int n, int what, void *buf, bool pack, cudaStream_t s) {
  if (n <= 0) return FV_OK;
  int blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_halo<<<blocks, 256, 0, s>>>(d, cells, n, what, buf, pack);
  return cudaGetLastError() == cudaSuccess ? FV_OK : FV_ERR_CUDA;
}

}  // namespace fvk

namespace {

int halo_fail(int code, const std::string &msg) {
  fv_internal_set_error(msg);
  return code;
}

}  // namespace

extern "C" {

int fv_halo_create(fv_mesh *m, const int64_t *cells, int64_t n, fv_halo **out) {
  if (!m || !out || n < 0 || (n > 0 && !cells)) return halo_fail(FV_ERR_INVALID_ARG, "fv_halo_create: bad argument");
  *out = nullptr;
  if (cudaSetDevice(m->cfg.device) != cudaSuccess) return halo_fail(FV_ERR_CUDA, "fv_halo_create: cudaSetDevice");
  const int N = m->d.N;
  std::vector<int> n2o(N), o2n(N, -1), ids((size_t)n);
  if (cudaMemcpy(n2o.data(), m->new2old_dev, sizeof(int) * N, cudaMemcpyDeviceToHost) != cudaSuccess)
    return halo_fail(FV_ERR_CUDA, "fv_halo_create: reading the cell numbering");
  for (int i = 0; i < N; ++i) o2n[n2o[i]] = i;
  for (int64_t k = 0; k < n; ++k) {
    if (cells[k] < 0 || cells[k] >= N)
      return halo_fail(FV_ERR_INVALID_ARG, "fv_halo_create: cell " + std::to_string((long long)cells[k]) +
                                               " outside the mesh");
    ids[k] = o2n[cells[k]];
  }
  fv_halo *h = new fv_halo;
  h->m = m;
  h->n = (int)n;
  if (n > 0) {
    if (cudaMalloc(&h->cells_dev, sizeof(int) * n) != cudaSuccess) {
      delete h;
      cudaGetLastError();
      return halo_fail(FV_ERR_NOMEM, "fv_halo_create: cudaMalloc");
    }
    if (cudaMemcpy(h->cells_dev, ids.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(h->cells_dev);
      delete h;
      return halo_fail(FV_ERR_CUDA, "fv_halo_create: upload");
    }
  }
  *out = h;
  return FV_OK;
}

int fv_halo_pack(fv_halo *h, int what, void *buf_dev, void *stream) {
  if (!h || (what != FV_HALO_LEVELS && what != FV_HALO_STATE) || (h->n > 0 && !buf_dev))
    return halo_fail(FV_ERR_INVALID_ARG, "fv_halo_pack: bad argument");
  if (fvk::launch_halo(h->m->d, h->cells_dev, h->n, what, buf_dev, true, (cudaStream_t)stream))
    return halo_fail(FV_ERR_CUDA, std::string("fv_halo_pack: ") + cudaGetErrorString(cudaGetLastError()));
  return FV_OK;
}

int fv_halo_unpack(fv_halo *h, int what, const void *buf_dev, void *stream) {
  if (!h || (what != FV_HALO_LEVELS && what != FV_HALO_STATE) || (h->n > 0 && !buf_dev))
    return halo_fail(FV_ERR_INVALID_ARG, "fv_halo_unpack: bad argument");
  if (h->m->in_batch) return halo_fail(FV_ERR_INVALID_ARG, "fv_halo_unpack: mesh is inside a batch");
  if (fvk::launch_halo(h->m->d, h->cells_dev, h->n, what, const_cast<void *>(buf_dev), false,
                       (cudaStream_t)stream))
    return halo_fail(FV_ERR_CUDA, std::string("fv_halo_unpack: ") + cudaGetErrorString(cudaGetLastError()));
  return FV_OK;
}

int64_t fv_halo_size(fv_halo *h) { return h ? h->n : -1; }

void fv_halo_free(fv_halo *h) {
  if (!h) return;
  if (h->cells_dev) {
    cudaSetDevice(h->m->cfg.device);
    cudaFree(h->cells_dev);
  }
  delete h;
}

}  // extern "C"

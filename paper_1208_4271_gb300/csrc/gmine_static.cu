// gmine_static.cu -- gmine_compute_batch_static: the batch computation with
// its working memory in a fixed array inside the library instead of a
// workspace that the caller allocates.
//
// Some callers cannot allocate device memory: code that runs inside a host
// application that owns the GPU's memory through its own pool and does not
// let plug-ins call cudaMalloc, and code on a latency-critical path where
// the device-wide synchronisation that cudaMalloc and cudaFree imply is not
// acceptable.  They still pass their own inputs and outputs; only the
// scratch memory comes from here.
//
// The array is a file-scope __device__ object of this file's module: under
// lazy module loading (the runtime's default) a GPU reserves its
// kStaticScratchBytes when this call first runs there, under eager loading
// whenever the process uses that GPU; it stays until the process exits.  On
// the first call on a device (with that device current) its device address
// is looked up with cudaGetSymbolAddress and kept (a device reset after that
// is not supported: the kept address would be stale); host code never passes
// the array's name itself to a kernel, since in host code that name is only
// a stand-in for the device object.
#include <mutex>

#include "gmine.h"
#include "gmine_internal.cuh"
#include "kernels.h"

namespace {

constexpr int64_t kStaticScratchBytes = int64_t(64) << 20;  // 64 MiB per GPU
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_addr[kMaxDevices];  // device address per device, once looked up

// Device address of the array on the current device (set up on first use).
int static_scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GMINE_E_NODEVICE;
  if (dev < 0 || dev >= kMaxDevices) return GMINE_E_LIMIT;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_addr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) {
      gm::note_cuda_error(e);
      return GMINE_E_CUDA;
    }
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return GMINE_OK;
}

}  // namespace

extern "C" int gmine_compute_batch_static(const double* d_vars, int64_t p, int64_t n,
                                          const int32_t* d_pairs, int64_t n_pairs,
                                          const gmine_param* param, int32_t precision,
                                          gmine_pair_score* d_scores, double* d_M,
                                          void* stream) {
  int64_t cells = 0, need = 0;
  int rc = gmine_plan(p, n, n_pairs, param, precision, 0, &cells, &need);
  if (rc != GMINE_OK) return rc;
  if (need > kStaticScratchBytes) return GMINE_E_WORKSPACE;  // nothing was touched
  void* ws = nullptr;
  rc = static_scratch_address(&ws);
  if (rc != GMINE_OK) return rc;
  // The batch path writes every part of its working memory before reading
  // it (its counters are reset at each call), so whatever an earlier call
  // left in the array does not matter.
  return gmine_compute_batch(d_vars, p, n, d_pairs, n_pairs, param, precision, ws, need, d_scores,
                             d_M, stream);
}

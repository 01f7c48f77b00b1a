// acr_residual_noalloc: the FP64 residual r = b - A x with relative norms,
// for callers that must not allocate device memory during the call -- for
// example code running under a fixed memory budget that was reserved up
// front, or a latency-critical loop where an allocation's implicit
// synchronisation is not acceptable.  It does the same work as acr_residual,
// but its reduction scratch (per-block partial sums of ||r||^2 and ||b||^2)
// is a fixed array in device global memory that is part of the library image
// instead of memory obtained from the allocator at call time.
//
// Limits and sharing: at most kMaxRhs right-hand sides per call; the array
// (about 1 MiB) is held by every GPU that loads the library until the process
// exits; all calls share it and it keeps the previous call's contents (every
// entry a call reads is first written by that same call, so nothing needs
// clearing).  Calls that overlap on the GPU -- on two streams, or from two
// threads -- race on the array and must be serialised by the caller.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/acr.h"
#include "acr_internal.h"

namespace {

constexpr int kMaxRhs = 64;
constexpr int kMaxBlocks = 1024;  // partial sums per column (grid-stride residual kernel)
constexpr size_t kPartElems = (size_t)kMaxBlocks * kMaxRhs * 2;
constexpr size_t kScratchElems = kPartElems + 2 * kMaxRhs;

// Scratch of the residual reduction.  In host code this name is only a
// host-side stand-in for the symbol; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) double g_resid_scratch[kScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return ACR_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_resid_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return ACR_ERR_CUDA;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return ACR_OK;
}

}  // namespace

namespace acr {
// Access to a handle's stream and face coefficients (defined with the handle).
int handle_residual_view(acr_handle h, cudaStream_t* st, int* n, const double** coef);
}  // namespace acr

extern "C" int acr_residual_noalloc(acr_handle h, const double* b, const double* x, double* r, int nrhs, long ld,
                                    double* rel_norms) {
  cudaStream_t st = nullptr;
  int n = 0;
  const double* coef = nullptr;
  if (!h || !b || !x || !r) return ACR_ERR_ARG;
  if (nrhs < 1 || nrhs > kMaxRhs) return ACR_ERR_ARG;  // beyond the fixed scratch
  if (acr::handle_residual_view(h, &st, &n, &coef) != ACR_OK) return ACR_ERR_ARG;
  if (ld < (long)n * n * n) return ACR_ERR_ARG;
  double* scratch = nullptr;
  int s = scratch_address(&scratch);
  if (s != ACR_OK) return s;
  double* part = scratch;
  double* pairs = scratch + kPartElems;
  acr::stencil_norms_scratch(st, n, nrhs, coef, x, ld, b, r, part, kMaxBlocks, pairs);
  // A failed launch must not fall through to reading the previous call's
  // norms out of the shared array.
  if (cudaGetLastError() != cudaSuccess) return ACR_ERR_CUDA;
  double hn[2 * kMaxRhs];
  if (cudaMemcpyAsync(hn, pairs, 2 * sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return ACR_ERR_CUDA;
  }
  if (rel_norms)
    for (int k = 0; k < nrhs; ++k)
      rel_norms[k] = hn[2 * k + 1] > 0 ? std::sqrt(hn[2 * k] / hn[2 * k + 1]) : std::sqrt(hn[2 * k]);
  return ACR_OK;
}

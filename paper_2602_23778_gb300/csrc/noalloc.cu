// eigref_product_dense_noalloc: the FP64 product P = (A - shift I) X with no
// device allocation.  The internal row-major copies of X and P live in one
// fixed array of device memory that is part of the library image, so the
// call works for code that is not allowed to allocate device memory.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace eigref {

constexpr int64_t kNoAllocMaxElems = EIGREF_NOALLOC_MAX_ELEMS;

// X (row-major) in the first half, P (row-major) in the second.  Every GPU
// that loads the library holds these 16 MiB until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxElems];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (returned in
// *dev), looked up once per device and cached.  In host code the array's name
// is only a host-side stand-in, never a device address.  A cudaDeviceReset of
// the device makes the cached address stale; the library does not detect it.
int scratch_for_current_device(double** out, int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return EIGREF_E_CUDA;
  }
  *dev_out = dev;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return EIGREF_E_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return EIGREF_OK;
}

bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}
}  // namespace

}  // namespace eigref

using namespace eigref;

extern "C" int eigref_product_dense_noalloc(const double* A, int64_t n, int64_t lda, const double* X, int64_t ldx,
                                            int k, double shift, double* P, int64_t ldp, void* stream) {
  if (!A || !X || !P) return EIGREF_E_INVALID;
  if (n < 1 || k < 1 || lda < n || ldx < n || ldp < n) return EIGREF_E_INVALID;
  if (n * (int64_t)k > kNoAllocMaxElems) return EIGREF_E_INVALID;  // beyond the fixed scratch
  // An error already pending on this thread belongs to the caller's earlier
  // work: report it without consuming it, so that the check after the
  // launches below sees only this call's own launches.
  if (cudaPeekAtLastError() != cudaSuccess) return EIGREF_E_CUDA;
  double* scratch = nullptr;
  int dev = 0;
  int st = scratch_for_current_device(&scratch, &dev);
  if (st) return st;
  if (!on_device(A, dev) || !on_device(X, dev) || !on_device(P, dev)) return EIGREF_E_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* xi = scratch;                     // every entry written by copy_in before it is read
  double* pi = scratch + kNoAllocMaxElems;  // every entry written by the product before it is read
  launch_copy_in(X, ldx, xi, n, k, nullptr, s);
  launch_gemm_fp64(A, lda, xi, pi, n, k, shift, nullptr, s);
  launch_copy_out(pi, P, ldp, n, k, nullptr, s);
  if (cudaGetLastError() != cudaSuccess) return EIGREF_E_CUDA;
  return EIGREF_OK;
}

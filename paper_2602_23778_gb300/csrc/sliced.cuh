// Split-precision (error-free sliced) evaluation of the dense product
// W = (A - shift I) X on the tensor cores.  See sliced.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace eigref {

cudaError_t init_sliced_attributes();

class SlicedA {
 public:
  // Host-side plan for A (device, n x n, lda) and k columns; no device work.
  int configure(const double* A, int64_t n, int64_t lda, int k, int precision, int slices);
  size_t workspace_bytes() const;
  void bind_workspace(char* p);
  // Slice A into its low-precision planes (once per refinement call).
  int prepare(cudaStream_t s);
  // P = (A - shift I) X for row-major X, P (n x k).  ev0/ev1 (may be null)
  // are recorded around the tensor-core kernel; returns the kernels launched.
  int product(const double* X, double* P, double shift, const Control* ctl, cudaStream_t s,
              cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, unsigned ev_flags = 0);
  const char* error() const { return err_; }

 private:
  const double* A_ = nullptr;
  int64_t n_ = 0, lda_ = 0;
  int k_ = 0, precision_ = 0, slices_ = 0;
  char* ws_ = nullptr;
  char err_[256] = {0};
};

}  // namespace eigref

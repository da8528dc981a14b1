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
  // Slice A into its digit planes and encode the tensor maps (once per call).
  int prepare(cudaStream_t s);
  // P = (A - shift I) X for row-major X, P (n x k).  ev0/ev1 (may be null)
  // are recorded around the tensor-core kernel; returns the kernels launched.
  int product(const double* X, double* P, double shift, const Control* ctl, cudaStream_t s,
              cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, unsigned ev_flags = 0);
  // 1 if a bounded wait inside the tensor-core kernel gave up (synchronises s).
  int timed_out(cudaStream_t s) const;
  // Tensor-core flops one product executes (all digit pairs, padded sizes).
  double executed_flops() const;
  int slices() const { return slices_; }
  const char* error() const { return err_; }

 private:
  const double* A_ = nullptr;
  int64_t n_ = 0, lda_ = 0;
  int k_ = 0, precision_ = 0, slices_ = 0;
  int n_pad_ = 0, k_pad_ = 0;
  char* ws_ = nullptr;
  alignas(64) unsigned char tmA_[128];
  alignas(64) unsigned char tmX_[128];
  char err_[256] = {0};
};

}  // namespace eigref

// Split-precision (error-free sliced) evaluation on the tensor cores of the
// dense products of a sweep: W = (A - shift I) X, the Gram products X^T X and
// X^T W, and the row update X - X F.  See sliced.cu.
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
  // The GPU is shared with `problems` - 1 other problems running side by side:
  // no product split-K, Gram split-K only down to about 4096 rows per CTA.
  // Call before workspace_bytes().
  void share_gpu(int problems);
  size_t workspace_bytes() const;
  void bind_workspace(char* p);
  // Slice A into its digit planes and encode the tensor maps (once per call).
  int prepare(cudaStream_t s);
  // P = (A - shift I) X for row-major X, P (n x k); keeps X's column planes
  // for gram().  ev0/ev1 (may be null) are recorded around the tensor-core
  // kernel; returns the kernels launched.
  int product(const double* X, double* P, double shift, const Control* ctl, cudaStream_t s,
              cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, unsigned ev_flags = 0);
  // out[0] = X^T X, out[1] = X^T P (k x k column-major, all n rows), with X the
  // operand of the last product(); part = split-K scratch (null: internal).
  int gram(const double* P, double* part, double* out, const Control* ctl, cudaStream_t s);
  // Rows k..n-1 of X' = X + (W - X D) D^-1 - X F (F k x k column-major) and
  // per-row-tile column sums of X'^2 and (W - X D)^2 into upart[update_grid()][2k].
  int update(const double* X, const double* W, const double* F, const double* d, const double* dinv, double* Xn,
             double* upart, const Control* ctl, cudaStream_t s);
  int update_grid() const;
  // 1 if a bounded wait inside a tensor-core kernel gave up (synchronises s).
  int timed_out(cudaStream_t s) const;
  // Tensor-core flops one product executes (all digit pairs, padded sizes).
  double executed_flops() const;
  int slices() const { return slices_; }
  const char* error() const { return err_; }

 private:
  size_t layout_total() const;
  const double* A_ = nullptr;
  int64_t n_ = 0, lda_ = 0;
  int k_ = 0, precision_ = 0, slices_ = 0;
  int n_pad_ = 0, k_pad_ = 0, kr_ = 0, ksplit_ = 1, psplit_ = 1;
  char* ws_ = nullptr;
  alignas(64) unsigned char tmA_[128];
  alignas(64) unsigned char tmX_[128];
  alignas(64) unsigned char tmXA_[128];
  alignas(64) unsigned char tmP_[128];
  alignas(64) unsigned char tmXR_[128];
  alignas(64) unsigned char tmF_[128];
  char err_[256] = {0};
};

}  // namespace eigref

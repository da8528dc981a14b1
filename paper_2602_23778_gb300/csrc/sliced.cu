// Split-precision dense product (placeholder until the tensor-core kernel lands).
#include <stdio.h>

#include "sliced.cuh"

namespace eigref {

cudaError_t init_sliced_attributes() { return cudaSuccess; }

int SlicedA::configure(const double* A, int64_t n, int64_t lda, int k, int precision, int slices) {
  A_ = A;
  n_ = n;
  lda_ = lda;
  k_ = k;
  precision_ = precision;
  slices_ = slices;
  snprintf(err_, sizeof(err_), "split-precision product not built yet");
  return EIGREF_E_UNSUPPORTED;
}
size_t SlicedA::workspace_bytes() const { return 0; }
void SlicedA::bind_workspace(char* p) { ws_ = p; }
int SlicedA::prepare(cudaStream_t) { return EIGREF_E_UNSUPPORTED; }
int SlicedA::product(const double*, double*, double, const Control*, cudaStream_t, cudaEvent_t, cudaEvent_t,
                     unsigned) {
  return 0;
}

}  // namespace eigref

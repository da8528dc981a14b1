// CSR SpMM over k right-hand columns: P = A X - shift X (the product of
// Algorithm 4 for sparse A; Table tab:cost prices it at O(nnz(A) k)).
//
// X and P are row-major n x k, so the k values a nonzero a_il multiplies sit
// in one contiguous row of X (128 bytes at k = 16): a group of lanes loads
// that row with 16-byte vector loads, and the row of P is written the same
// way.  The CSR arrays are read once (streaming, no L1 allocation); the X
// rows a 5-point stencil touches stay in L2 between neighbouring rows.  The
// kernel is HBM-bound: per launch it moves the CSR arrays, X once and P once.
#include <cuda_runtime.h>

#include "common.cuh"

namespace eigref {

__device__ __forceinline__ int ld_stream_i32(const int32_t* p) {
  int v;
  asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_stream_f64(const double* p) {
  double v;
  asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

// LPR lanes per row; each lane owns column pairs c2 = lane, lane + LPR, ...
// GB300 issues about 2 DFMA per clock per SM, so this kernel is bound by the
// FP64 pipe (nnz k DFMA per launch, ~130 us at n = 1,024,000, k = 16), not by
// HBM (~48 us for its 328 MB): it is kept lean -- one X row load and two DFMA
// per nonzero and lane.  With the shift folded into the stored diagonal
// (SHIFT = false, see csr_fold_diag) there is no separate shift term.
// cmax (optional): column maxima of |P| as ordered bit patterns (atomicMax),
// for the slicing of P that follows in the split form.
template <int LPR, bool SHIFT>
__global__ void __launch_bounds__(256) spmm_csr_vec2_kernel(const int32_t* __restrict__ rp,
                                                            const int32_t* __restrict__ ci,
                                                            const double* __restrict__ val,
                                                            const double* __restrict__ X, double* __restrict__ P,
                                                            int64_t n, int k, double shift,
                                                            const double* __restrict__ Xs, const Control* ctl,
                                                            unsigned long long* __restrict__ cmax) {
  if (ctl && ctl->done) return;
  __shared__ unsigned long long colm[kMaxK];
  // this lane's column pairs (at most two): max |P| as ordered bit patterns,
  // compared as integers (the FP64 pipe is the kernel's bottleneck)
  unsigned long long mx[2][2] = {{0ull, 0ull}, {0ull, 0ull}};
  const int lane = threadIdx.x % LPR;
  const int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LPR;
  const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / LPR;
  const int k2 = k >> 1;
  const double2* X2 = reinterpret_cast<const double2*>(X);
  double2* P2 = reinterpret_cast<double2*>(P);
  for (int64_t i = g; i < n; i += ng) {
    const int32_t b = ld_stream_i32(rp + i), e = ld_stream_i32(rp + i + 1);
    for (int c2 = lane; c2 < k2; c2 += LPR) {
      double ax = 0.0, ay = 0.0;
#pragma unroll 4
      for (int32_t p = b; p < e; ++p) {
        const double a = ld_stream_f64(val + p);
        const int64_t col = ld_stream_i32(ci + p);
        const double2 x = __ldg(X2 + col * k2 + c2);
        ax = fma(a, x.x, ax);
        ay = fma(a, x.y, ay);
      }
      if (SHIFT) {
        const double2 xi = __ldg(reinterpret_cast<const double2*>(Xs) + i * k2 + c2);
        ax = fma(-shift, xi.x, ax);
        ay = fma(-shift, xi.y, ay);
      }
      P2[i * k2 + c2] = make_double2(ax, ay);
      if (cmax) {
        const unsigned long long a = (unsigned long long)__double_as_longlong(ax) & 0x7FFFFFFFFFFFFFFFull;
        const unsigned long long b = (unsigned long long)__double_as_longlong(ay) & 0x7FFFFFFFFFFFFFFFull;
        if (c2 < lane + LPR) {
          mx[0][0] = umax64(mx[0][0], a);
          mx[0][1] = umax64(mx[0][1], b);
        } else {
          mx[1][0] = umax64(mx[1][0], a);
          mx[1][1] = umax64(mx[1][1], b);
        }
      }
    }
  }
  if (cmax) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) colm[j] = 0ull;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c2 = lane + q * LPR;
      if (c2 < k2) {
        atomicMax(&colm[2 * c2], mx[q][0]);
        atomicMax(&colm[2 * c2 + 1], mx[q][1]);
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      if (colm[j]) atomicMax(cmax + j, colm[j]);
  }
}

// val_out = val with the shift subtracted on the diagonal; missing[0] is set
// when some row has no stored diagonal entry (then the folded copy is unusable).
__global__ void csr_fold_diag_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const double* __restrict__ val, int64_t n, double shift,
                                     double* __restrict__ val_out, int* __restrict__ missing) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    bool found = false;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
      const bool diag = ci[p] == i;
      val_out[p] = diag ? val[p] - shift : val[p];
      found = found || diag;
    }
    if (!found) atomicExch(missing, 1);
  }
}

void launch_csr_fold_diag(const int32_t* rp, const int32_t* ci, const double* val, int64_t n, double shift,
                          double* val_out, int* missing, cudaStream_t s) {
  cudaMemsetAsync(missing, 0, sizeof(int), s);
  const int grid = (int)((n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16);
  csr_fold_diag_kernel<<<grid, 256, 0, s>>>(rp, ci, val, n, shift, val_out, missing);
}

__global__ void __launch_bounds__(256) spmm_csr_scalar_kernel(const int32_t* __restrict__ rp,
                                                              const int32_t* __restrict__ ci,
                                                              const double* __restrict__ val,
                                                              const double* __restrict__ X, double* __restrict__ P,
                                                              int64_t n, int k, double shift,
                                                              const double* __restrict__ Xs, const Control* ctl) {
  if (ctl && ctl->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w; i < n; i += nw) {
    const int32_t b = rp[i], e = rp[i + 1];
    for (int c = lane; c < k; c += 32) {
      double acc = 0.0;
      for (int32_t p = b; p < e; ++p) acc = fma(val[p], X[(int64_t)ci[p] * k + c], acc);
      P[i * k + c] = acc - shift * Xs[i * k + c];
    }
  }
}

void launch_spmm_csr(const int32_t* rp, const int32_t* ci, const double* val, const double* X, double* P,
                     int64_t n, int k, double shift, const Control* ctl, cudaStream_t s, const double* Xs,
                     unsigned long long* cmax) {
  if (!Xs) Xs = X;
  if ((k & 1) || k > 2 * 2 * 32) cmax = nullptr;   // maxima only from the paired-column kernel
  const int grid = 152 * 8;  // 8 resident CTAs of 256 threads per SM, grid-stride over rows
  if ((k & 1) == 0) {
    const int k2 = k >> 1;
#define EIGREF_SPMM(L)                                                                                       \
  if (shift != 0.0)                                                                                         \
    spmm_csr_vec2_kernel<L, true><<<grid, 256, 0, s>>>(rp, ci, val, X, P, n, k, shift, Xs, ctl, cmax);       \
  else                                                                                                      \
    spmm_csr_vec2_kernel<L, false><<<grid, 256, 0, s>>>(rp, ci, val, X, P, n, k, shift, Xs, ctl, cmax);
    if (k2 <= 2) {
      EIGREF_SPMM(2)
    } else if (k2 <= 4) {
      EIGREF_SPMM(4)
    } else if (k2 <= 8) {
      EIGREF_SPMM(8)
    } else if (k2 <= 16) {
      EIGREF_SPMM(16)
    } else {
      EIGREF_SPMM(32)
    }
#undef EIGREF_SPMM
  } else {
    spmm_csr_scalar_kernel<<<grid, 256, 0, s>>>(rp, ci, val, X, P, n, k, shift, Xs, ctl);
  }
}

}  // namespace eigref

// CSR SpMM over k right-hand columns: P = A X - shift X (line 1 of
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

// A CTA takes 64 consecutive rows at a time.  Their row pointers and then
// their nonzeros (a contiguous range of the CSR arrays) are staged in shared
// memory with coalesced loads; then each group of LPR lanes takes two rows
// and requests every X row they touch before using any, so each 64-row block
// costs three memory latencies and keeps many X rows in flight.  Blocks whose
// nonzeros do not fit the stage read them from global memory directly.
constexpr int SP_ROWS = 64;
constexpr int SP_CAP = 2048;   // staged nonzeros per block

template <int LPR>
__global__ void __launch_bounds__(256) spmm_csr_vec2_kernel(const int32_t* __restrict__ rp,
                                                            const int32_t* __restrict__ ci,
                                                            const double* __restrict__ val,
                                                            const double* __restrict__ X, double* __restrict__ P,
                                                            int64_t n, int k, double shift, const Control* ctl) {
  if (ctl && ctl->done) return;
  __shared__ int32_t rps[SP_ROWS + 1];
  __shared__ int32_t cis[SP_CAP];
  __shared__ double vals[SP_CAP];
  constexpr int GROUPS = 256 / LPR;
  const int tid = threadIdx.x, lane = tid % LPR, grp = tid / LPR;
  const int k2 = k >> 1;
  const double2* X2 = reinterpret_cast<const double2*>(X);
  double2* P2 = reinterpret_cast<double2*>(P);
  const int64_t nblk = (n + SP_ROWS - 1) / SP_ROWS;
  for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int64_t r0 = blk * SP_ROWS;
    const int rows = (int)(n - r0 < SP_ROWS ? n - r0 : SP_ROWS);
    if (tid <= rows) rps[tid] = ld_stream_i32(rp + r0 + tid);
    __syncthreads();
    const int32_t nb = rps[0], cnt = rps[rows] - nb;
    const bool staged = cnt <= SP_CAP;
    if (staged)
      for (int q = tid; q < cnt; q += 256) {
        cis[q] = ld_stream_i32(ci + nb + q);
        vals[q] = ld_stream_f64(val + nb + q);
      }
    __syncthreads();
    for (int r = grp; r < rows; r += GROUPS) {
      const int32_t b = rps[r], e = rps[r + 1];
      const int64_t i = r0 + r;
      for (int c2 = lane; c2 - lane < k2; c2 += LPR) {
        double ax = 0.0, ay = 0.0;
        for (int32_t p0 = b; p0 < e; p0 += 8) {
          double2 xs[8];
          double as[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int32_t p = p0 + t;
            const bool on = p < e && c2 < k2;
            const int64_t col = on ? (staged ? cis[p - nb] : ci[p]) : 0;
            as[t] = on ? (staged ? vals[p - nb] : val[p]) : 0.0;
            xs[t] = on ? __ldg(X2 + col * k2 + c2) : make_double2(0.0, 0.0);
          }
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            ax = fma(as[t], xs[t].x, ax);
            ay = fma(as[t], xs[t].y, ay);
          }
        }
        if (c2 < k2) {
          const double2 xi = __ldg(X2 + i * k2 + c2);
          P2[i * k2 + c2] = make_double2(ax - shift * xi.x, ay - shift * xi.y);
        }
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) spmm_csr_scalar_kernel(const int32_t* __restrict__ rp,
                                                              const int32_t* __restrict__ ci,
                                                              const double* __restrict__ val,
                                                              const double* __restrict__ X, double* __restrict__ P,
                                                              int64_t n, int k, double shift, const Control* ctl) {
  if (ctl && ctl->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w; i < n; i += nw) {
    const int32_t b = rp[i], e = rp[i + 1];
    for (int c = lane; c < k; c += 32) {
      double acc = 0.0;
      for (int32_t p = b; p < e; ++p) acc = fma(val[p], X[(int64_t)ci[p] * k + c], acc);
      P[i * k + c] = acc - shift * X[i * k + c];
    }
  }
}

void launch_spmm_csr(const int32_t* rp, const int32_t* ci, const double* val, const double* X, double* P,
                     int64_t n, int k, double shift, const Control* ctl, cudaStream_t s) {
  const int grid = 152 * 6;  // resident CTAs of 256 threads, grid-stride over 64-row blocks
  if ((k & 1) == 0) {
    const int k2 = k >> 1;
    if (k2 <= 2)
      spmm_csr_vec2_kernel<2><<<grid, 256, 0, s>>>(rp, ci, val, X, P, n, k, shift, ctl);
    else if (k2 <= 4)
      spmm_csr_vec2_kernel<4><<<grid, 256, 0, s>>>(rp, ci, val, X, P, n, k, shift, ctl);
    else if (k2 <= 8)
      spmm_csr_vec2_kernel<8><<<grid, 256, 0, s>>>(rp, ci, val, X, P, n, k, shift, ctl);
    else if (k2 <= 16)
      spmm_csr_vec2_kernel<16><<<grid, 256, 0, s>>>(rp, ci, val, X, P, n, k, shift, ctl);
    else
      spmm_csr_vec2_kernel<32><<<grid, 256, 0, s>>>(rp, ci, val, X, P, n, k, shift, ctl);
  } else {
    spmm_csr_scalar_kernel<<<grid, 256, 0, s>>>(rp, ci, val, X, P, n, k, shift, ctl);
  }
}

}  // namespace eigref

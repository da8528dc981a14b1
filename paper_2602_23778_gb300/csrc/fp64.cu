// FP64 kernels of one refinement sweep of Algorithm 4: the product W = B X
// (plain FP64 form), the Gram reductions X^T X and X^T W (Rayleigh quotients,
// Eq. Rayleigh), the row update of the rows below the leading k x k block
// (Eq. update-X in the folded form), the per-sweep statistics and stopping test
// (Section 3.1.3), and column normalisation.
//
// GB300 runs FP64 at about 2 DFMA per clock per SM (1.1 TFLOP/s measured for
// the whole GPU), so every FP64 kernel here is bound by the FP64 pipe, not by
// HBM: they are organised for enough independent DFMAs per thread, not for
// bandwidth.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace eigref {

// ---------------------------------------------------------------------------
// P = A X - shift Xs (Xs = X unless given).  A n x n row-major (lda), X, Xs
// and P n x k row-major.
// 16 x 16 output tile per CTA, one output per thread: the K sum is a single
// FMA chain over l = 0 .. n-1, operands read through L1 (a warp reads two
// elements of A, one per row, and one 128-byte row of X a step).  GB300 issues
// about 2 DFMA a clock and SM, so the kernel is bound by the FP64 pipe, not by
// its loads; n k / 256 CTAs (8192 at n = 16384, k = 128) leave no tail
// worth the name, where 64 x 64 tiles with a shared-memory K panel ran 1.68
// waves and reached 0.83 of this kernel's rate.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) gemm_fp64_kernel(const double* __restrict__ A, int64_t lda,
                                                        const double* __restrict__ X,
                                                        double* __restrict__ P, int64_t n, int k,
                                                        double shift, const double* __restrict__ Xs,
                                                        const Control* ctl) {
  if (ctl && ctl->done) return;
  const int tid = threadIdx.x;
  const int64_t row = (int64_t)blockIdx.x * 16 + (tid >> 4);
  const int col = blockIdx.y * 16 + (tid & 15);
  if (row >= n || col >= k) return;
  const double* a = A + row * lda;
  const double* x = X + col;
  double acc = 0.0;
  int64_t l = 0;
  for (; l + 4 <= n; l += 4) {
    const double a0 = __ldg(a + l), a1 = __ldg(a + l + 1), a2 = __ldg(a + l + 2), a3 = __ldg(a + l + 3);
    const double x0 = __ldg(x + l * k), x1 = __ldg(x + (l + 1) * k), x2 = __ldg(x + (l + 2) * k),
                 x3 = __ldg(x + (l + 3) * k);
    acc = fma(a0, x0, acc);
    acc = fma(a1, x1, acc);
    acc = fma(a2, x2, acc);
    acc = fma(a3, x3, acc);
  }
  for (; l < n; ++l) acc = fma(__ldg(a + l), __ldg(x + l * k), acc);
  P[row * k + col] = acc - shift * Xs[row * k + col];
}

void launch_gemm_fp64(const double* A, int64_t lda, const double* X, double* P, int64_t n, int k,
                      double shift, const Control* ctl, cudaStream_t s, const double* Xs) {
  const dim3 grid((unsigned)((n + 15) / 16), (unsigned)((k + 15) / 16));
  gemm_fp64_kernel<<<grid, 256, 0, s>>>(A, lda, X, P, n, k, shift, Xs ? Xs : X, ctl);
}

// ---------------------------------------------------------------------------
// Gram partials over a row range: part[z][c] = (X^T Y)[rows of chunk c],
// z = 0: Y = X (G), z = 1: Y = P (S).  T x T output tile per CTA (T = 16 for
// k <= 16, else 32), 256 threads.  Deterministic: partials are summed in
// chunk order by gram_reduce.  G is symmetric and fma(a, b, c) = fma(b, a, c),
// so for z = 0 only tiles ti <= tj are formed (and at T = 16 only the 136
// outputs i <= j, on 5 of the 8 warps) and mirrored on the way out, with the
// same bits as forming both.
// ---------------------------------------------------------------------------
template <int T>
__global__ void __launch_bounds__(256) gram_partial_kernel(const double* __restrict__ X,
                                                           const double* __restrict__ P, int k, int64_t r0,
                                                           int64_t r1, int64_t chunk_rows, int nchunks,
                                                           double* __restrict__ part, const Control* ctl) {
  if (ctl && ctl->done) return;
  constexpr int RB = 2048 / T;              // rows staged per step (T x RB doubles per operand, < 48 KB)
  constexpr int OUT = T * T / 256;          // outputs per thread
  __shared__ double Xa[RB][T + 1];
  __shared__ double Xb[RB][T + 1];
  const int c = blockIdx.x;
  const int tiles = (k + T - 1) / T;
  const int ti = blockIdx.y % tiles, tj = blockIdx.y / tiles;
  const int z = blockIdx.z;
  if (z == 0 && ti > tj) return;            // the mirror of tile (tj, ti)
  const double* Yb = z ? P : X;
  const int tid = threadIdx.x;
  int i = tid % T, jg = tid / T;            // outputs (i, jg * OUT + q)
  const bool tri = (T == 16 && z == 0);     // upper triangle of the single G tile
  bool active = true;
  if (tri) {
    // thread t < 136 takes the t-th pair (i, j), i <= j, row by row
    int t = tid, r = 0;
    while (r < 16 && t >= 16 - r) {
      t -= 16 - r;
      ++r;
    }
    active = r < 16;
    i = active ? r : 0;
    jg = active ? r + t : 0;
  }
  double acc[OUT];
#pragma unroll
  for (int q = 0; q < OUT; ++q) acc[q] = 0.0;
  const int64_t rb = r0 + (int64_t)c * chunk_rows;
  const int64_t re = r1 < rb + chunk_rows ? r1 : rb + chunk_rows;
  for (int64_t row0 = rb; row0 < re; row0 += RB) {
    for (int e = tid; e < RB * T; e += 256) {
      const int rr = e / T, cc = e % T;
      const int64_t row = row0 + rr;
      const int ca = ti * T + cc, cb = tj * T + cc;
      Xa[rr][cc] = (row < re && ca < k) ? X[row * k + ca] : 0.0;
      Xb[rr][cc] = (row < re && cb < k) ? Yb[row * k + cb] : 0.0;
    }
    __syncthreads();
    if (active) {
#pragma unroll 8
      for (int rr = 0; rr < RB; ++rr) {
        const double a = Xa[rr][i];
#pragma unroll
        for (int q = 0; q < OUT; ++q) acc[q] = fma(a, Xb[rr][jg * OUT + q], acc[q]);
      }
    }
    __syncthreads();
  }
  double* out = part + ((int64_t)z * nchunks + c) * k * k;
  const int gi = ti * T + i;
  if (!active) return;
#pragma unroll
  for (int q = 0; q < OUT; ++q) {
    const int gj = tj * T + jg * OUT + q;
    if (gi < k && gj < k) {
      out[gi + (int64_t)gj * k] = acc[q];
      if (z == 0) out[gj + (int64_t)gi * k] = acc[q];   // G(j, i) = G(i, j)
    }
  }
}

// One warp per output: lane l sums chunks l, l + 32, ... in order, then a
// fixed butterfly combines the lanes, so the result is the same every run.
__device__ __forceinline__ void gram_reduce_body(const double* __restrict__ part, int k, int nchunks,
                                                 double* __restrict__ out, int64_t w0, int64_t nw) {
  const int64_t kk = (int64_t)k * k;
  const int lane = threadIdx.x & 31;
  for (int64_t e = w0; e < 2 * kk; e += nw) {
    const int z = (int)(e / kk);
    const int64_t o = e % kk;
    const double* p = part + (int64_t)z * nchunks * kk + o;
    double s = 0.0;
    for (int c = lane; c < nchunks; c += 32) s += p[(int64_t)c * kk];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (lane == 0) out[e] = s;
  }
}

__global__ void gram_reduce_kernel(const double* __restrict__ part, int k, int nchunks, double* __restrict__ out,
                                   const Control* ctl) {
  if (ctl && ctl->done) return;
  gram_reduce_body(part, k, nchunks, out, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5,
                   ((int64_t)gridDim.x * blockDim.x) >> 5);
}

void launch_gram_reduce(const double* part, int k, int nchunks, double* out, const Control* ctl, cudaStream_t s) {
  const int64_t warps = 2LL * k * k;
  const int rg = (int)std::min<int64_t>((warps + 7) / 8, 152 * 8);
  gram_reduce_kernel<<<rg, 256, 0, s>>>(part, k, nchunks, out, ctl);
}

// Gram products of the leading k x k block: out[0] = X1^T X1, out[1] = X1^T P1
// (16 x 16 output tiles, k-term dot products).
__device__ __forceinline__ void top_gram_body(const double* __restrict__ X, const double* __restrict__ P, int k,
                                              double* __restrict__ out, int bx, int by, int bz) {
  __shared__ double As[16][17];
  __shared__ double Bs[16][17];
  const double* Y = bz ? P : X;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i = bx * 16 + tx, j = by * 16 + ty;
  double acc = 0.0;
  for (int l0 = 0; l0 < k; l0 += 16) {
    const int l = l0 + ty;
    const int ai = bx * 16 + tx, bj = by * 16 + tx;
    As[ty][tx] = (l < k && ai < k) ? X[(int64_t)l * k + ai] : 0.0;   // X1(l, i)
    Bs[ty][tx] = (l < k && bj < k) ? Y[(int64_t)l * k + bj] : 0.0;   // Y1(l, j)
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 16; ++c) acc = fma(As[c][tx], Bs[c][ty], acc);
    __syncthreads();
  }
  if (i < k && j < k) out[(int64_t)bz * k * k + i + (int64_t)j * k] = acc;
}

__global__ void __launch_bounds__(256) top_gram_kernel(const double* __restrict__ X, const double* __restrict__ P,
                                                       int k, double* __restrict__ out, const Control* ctl) {
  if (ctl && ctl->done) return;
  top_gram_body(X, P, k, out, blockIdx.x, blockIdx.y, blockIdx.z);
}

void launch_top_gram(const double* X, const double* P, int k, double* out, const Control* ctl, cudaStream_t s) {
  dim3 g((k + 15) / 16, (k + 15) / 16, 2);
  top_gram_kernel<<<g, 256, 0, s>>>(X, P, k, out, ctl);
}

// Batch: blockIdx.z = 2 problem + (0: G1, 1: S1).
__global__ void __launch_bounds__(256) top_gram_grouped_kernel(const GroupItem* __restrict__ items, int parity) {
  const GroupItem& it = items[blockIdx.z >> 1];
  const SweepBufs& b = it.b[parity];
  if ((int)blockIdx.x * 16 >= it.k || (int)blockIdx.y * 16 >= it.k || b.ctl->done) return;
  top_gram_body(b.x, b.p, it.k, b.gtop, blockIdx.x, blockIdx.y, blockIdx.z & 1);
}

void launch_top_gram_grouped(const GroupItem* items, const GroupDims& gd, int parity, cudaStream_t s) {
  const int t = (gd.max_k + 15) / 16;
  top_gram_grouped_kernel<<<dim3(t, t, 2 * gd.count), 256, 0, s>>>(items, parity);
}

void launch_gram(const double* X, const double* P, int k, int64_t r0, int64_t r1, int64_t chunk_rows,
                 int nchunks, double* part, double* out, const Control* ctl, cudaStream_t s) {
  if (k <= 16) {
    dim3 grid(nchunks, 1, 2);
    gram_partial_kernel<16><<<grid, 256, 0, s>>>(X, P, k, r0, r1, chunk_rows, nchunks, part, ctl);
  } else {
    const int tiles = (k + 31) / 32;
    dim3 grid(nchunks, tiles * tiles, 2);
    gram_partial_kernel<32><<<grid, 256, 0, s>>>(X, P, k, r0, r1, chunk_rows, nchunks, part, ctl);
  }
  launch_gram_reduce(part, k, nchunks, out, ctl, s);
}

// ---------------------------------------------------------------------------
// Row update below the leading block (rows k..n-1), folded form of the update
// X-tilde = X-hat + H-hat E-tilde_L (Algorithm 4, Eq. update-X):
//   x' = x + (w - x o d) / d - x F,   F = M D^-1 + N
// with per-CTA partial column sums of x'^2, of the residual r = w - x o d and
// of the rows of V2 = R2 - X2 M (E21 = V2 D^-1, the lower block of E-tilde_L
// in Algorithm 4): ||E21||_F is formed from explicit rows, as the stopping test of
// Section 3.1.3 reads it, not from k x k Gram quantities (whose difference
// cancels once the correction falls below sqrt(u)).
// ---------------------------------------------------------------------------
constexpr int UPD_ROWS = 16;     // rows per step at k = 128; smaller k takes UPD_ROWS * 128 / k
constexpr int UPD_GRID = 2 * 152;

int update_rows_grid() { return UPD_GRID; }

__host__ __device__ inline int update_rows_per_step(int k) { return (UPD_ROWS * kMaxK) / k > 0 ? (UPD_ROWS * kMaxK) / k : 1; }
// Column parts: above 64 columns a CTA takes half of them, so that its panels
// of F and M (k x columns each) fit in shared memory together.
__host__ __device__ inline int update_rows_parts(int k) { return k > 64 ? 2 : 1; }
__host__ __device__ inline int update_rows_cols(int k) { return (k + update_rows_parts(k) - 1) / update_rows_parts(k); }

// CTA (g, h): row blocks g, g + gridDim.x, ... and columns h kc .. h kc + kc - 1.
// Column sums are formed in a fixed order (no atomics), so results are
// bitwise reproducible run to run.  upart[g][3k]: sums of x'^2, r^2, v2^2.
__global__ void __launch_bounds__(256) update_rows_kernel(const double* __restrict__ X,
                                                          const double* __restrict__ P,
                                                          double* __restrict__ Xn, int64_t n, int k,
                                                          const double* __restrict__ F,
                                                          const double* __restrict__ M,
                                                          const double* __restrict__ d,
                                                          double* __restrict__ upart, const Control* ctl) {
  if (ctl && ctl->done) return;
  extern __shared__ double sm[];
  const int kc = update_rows_cols(k);
  const int j0 = (int)blockIdx.y * kc;
  const int jn = min(kc, k - j0);           // columns of this CTA
  const int rb = update_rows_per_step(k);   // rows per step: rb k ~ 2048 inputs
  double* Fs = sm;                          // Fs[l * kc + jj] = F(l, j0 + jj)
  double* Ms = Fs + k * kc;                 // Ms[l * kc + jj] = M(l, j0 + jj)
  double* xs = Ms + k * kc;                 // [rb][k]: whole rows of X
  double* sq = xs + rb * k;                 // [rb][jn]: x'^2
  double* rq = sq + rb * kc;                // [rb][jn]: r^2
  double* vq = rq + rb * kc;                // [rb][jn]: v2^2
  double* dinv = vq + rb * kc;              // [jn]
  double* dv = dinv + kc;                   // [jn]
  const int tid = threadIdx.x;
  for (int e = tid; e < k * jn; e += blockDim.x) {
    const int l = e % k, jj = e / k;        // F, M column-major
    Fs[l * kc + jj] = F[l + (int64_t)(j0 + jj) * k];
    Ms[l * kc + jj] = M[l + (int64_t)(j0 + jj) * k];
  }
  for (int jj = tid; jj < jn; jj += blockDim.x) {
    dv[jj] = d[j0 + jj];
    dinv[jj] = 1.0 / d[j0 + jj];
  }
  // column sums: thread tid owns column tid % jn and rows tid / jn, tid / jn + gstride, ...
  const int gstride = blockDim.x / jn > 0 ? blockDim.x / jn : 1;
  const int scol = tid % jn, srow0 = tid / jn;
  double accx = 0.0, accr = 0.0, accv = 0.0;
  __syncthreads();
  const int64_t rows = n - k;
  const int64_t nblk = (rows + rb - 1) / rb;
  const int per = rb * jn;
  for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    const int64_t row0 = k + b * rb;
    for (int e = tid; e < rb * k; e += blockDim.x) {
      int64_t row = row0 + e / k;
      xs[e] = row < n ? X[row0 * k + e] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < per; e += blockDim.x) {
      const int r = e / jn, jj = e % jn, j = j0 + jj;
      const int64_t row = row0 + r;
      double xn = 0.0, rr = 0.0, v = 0.0;
      if (row < n) {
        const double* xr = xs + r * k;
        const double x = xr[j];
        rr = P[row * k + j] - x * dv[jj];
        double s = 0.0, sm2 = 0.0;
        for (int l = 0; l < k; ++l) {
          s = fma(xr[l], Fs[l * kc + jj], s);
          sm2 = fma(xr[l], Ms[l * kc + jj], sm2);
        }
        xn = x + rr * dinv[jj] - s;
        v = rr - sm2;                       // row of V2 = R2 - X2 M
        Xn[row * k + j] = xn;
      }
      sq[e] = xn * xn;
      rq[e] = rr * rr;
      vq[e] = v * v;
    }
    __syncthreads();
    if (srow0 < gstride && tid < gstride * jn)
      for (int r = srow0; r < rb; r += gstride) {
        accx += sq[r * jn + scol];
        accr += rq[r * jn + scol];
        accv += vq[r * jn + scol];
      }
    __syncthreads();
  }
  // combine the gstride partial sums of each column in a fixed order
  __shared__ double cs[3][256];
  cs[0][tid] = accx;
  cs[1][tid] = accr;
  cs[2][tid] = accv;
  __syncthreads();
  if (tid < jn) {
    double sx = 0.0, sr = 0.0, sv = 0.0;
    for (int g = 0; g < gstride; ++g) {
      sx += cs[0][g * jn + tid];
      sr += cs[1][g * jn + tid];
      sv += cs[2][g * jn + tid];
    }
    double* up = upart + (int64_t)blockIdx.x * 3 * k + j0 + tid;
    up[0] = sx;
    up[k] = sr;
    up[2 * k] = sv;
  }
}

static size_t update_smem(int k) {
  const size_t kc = (size_t)update_rows_cols(k), rb = (size_t)update_rows_per_step(k);
  return sizeof(double) * (2 * (size_t)k * kc + rb * (size_t)k + 3 * rb * kc + 2 * kc);
}

static size_t update_smem_max() {
  size_t m = 0;
  for (int k = 1; k <= kMaxK; ++k) m = std::max(m, update_smem(k));
  return m;
}

void launch_update_rows(const SweepBufs& b, int64_t n, int k, cudaStream_t s) {
  size_t smem = update_smem(k);
  update_rows_kernel<<<dim3(UPD_GRID, update_rows_parts(k)), 256, smem, s>>>(b.x, b.p, b.xn, n, k, b.f, b.m, b.d,
                                                                              b.upart, b.ctl);
}

// ---------------------------------------------------------------------------
// Per-sweep statistics and control (one CTA).
//   ||R||_F^2  = sum_j r1sq_j + sum_blocks r^2
//   ||E||_F^2  = ||E11||_F^2 + sum_j ||v2_j||^2 / d_j^2   (E21 = V2 D^-1, rows of V2 summed by the update)
//   nu_j = 1 / ||x'_j||
// Stopping, divergence and non-finite tests of Section 3.1.3 / Section 4.3.1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finalize_body(const SweepBufs& b, int k) {
  Control* ctl = b.ctl;
  __shared__ double xsq_s[kMaxK], r2_s[kMaxK];
  __shared__ double red[3][32];
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  // The kernel is a chain of latencies, so every control field it needs is
  // loaded here, together with the partials below; the stop flag is acted on
  // once they are in (reading partials of a finished run writes nothing).
  const int done = ctl->done, judge = ctl->judge;
  int it = 0, stop = 0, max_iters = 0;
  double tol = 0.0, norm_a = 1.0, div_factor = 0.0, div_floor = 0.0, emin = 0.0;
  if (tid == 0) {
    it = ctl->iterations;
    stop = ctl->stop;
    max_iters = ctl->max_iters;
    tol = ctl->tol;
    norm_a = ctl->norm_a;
    div_factor = ctl->div_factor;
    div_floor = ctl->div_floor;
    emin = ctl->emin;
    bad = 0;
  }
  // Column sums of the update partials [ugrid][3k] and of the squares of the
  // leading block's rows: row group rg = tid / 128 (8 of them) takes rows
  // rg, rg + 8, ... and its 128 threads the columns c, c + 128, c + 256, so
  // each thread has all its loads (about 50 at 3k = 384) in flight at once;
  // the 8 row-group sums of a column are then added in order (fixed order,
  // reproducible).
  constexpr int kRG = 8;
  __shared__ double part_s[kRG][3 * kMaxK];
  __shared__ double top_s[kRG * kMaxK];
  __shared__ double v2_s[kMaxK];
  {
    const int w3 = 3 * k, rg = tid >> 7, t = tid & 127;
    if (rg < kRG) {
      double acc[3] = {0.0, 0.0, 0.0};
      for (int g = rg; g < b.ugrid; g += kRG) {
        const double* row = b.upart + (int64_t)g * w3;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (t + 128 * q < w3) acc[q] += row[t + 128 * q];
      }
      // the leading block's rows i = rg, rg + 8, ... of column t (X' row-major)
      double top = 0.0;
      if (t < k)
        for (int i = rg; i < k; i += kRG) {
          const double v = b.xn[(int64_t)i * k + t];
          top = fma(v, v, top);
        }
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (t + 128 * q < w3) part_s[rg][t + 128 * q] = acc[q];
      if (t < k) top_s[rg * k + t] = top;
    }
    __syncthreads();
    if (tid < k) {
      const int j = tid;
      double xsq = 0.0, r2 = 0.0, v2 = 0.0, tp = 0.0;
      for (int g = 0; g < kRG; ++g) {
        xsq += part_s[g][j];
        r2 += part_s[g][k + j];
        v2 += part_s[g][2 * k + j];
        tp += top_s[g * k + j];
      }
      xsq_s[j] = xsq + tp;
      r2_s[j] = r2;
      v2_s[j] = v2;
    }
  }
  if (done) {
    if (tid == 0) ctl->pending_norm = 0;
    return;
  }
  __syncthreads();
  double rsum = 0.0, esum = 0.0, e11 = 0.0;
  if (tid < k) {
    const int j = tid;
    const double xsq = xsq_s[j], r2 = r2_s[j], dj = b.d[j];
    const double e21 = v2_s[j] / (dj * dj);   // ||E21(:, j)||^2 from the explicit rows of V2
    // the correction of the judged leading columns decides stop and divergence
    esum = j < judge ? e21 : 0.0;
    rsum = b.r1sq[j] + r2;
    e11 = j < judge ? b.e11sq[j] : 0.0;
    b.nu[j] = 1.0 / sqrt(xsq);
    if (!isfinite(xsq) || !(xsq > 0.0)) atomicExch(&bad, 1);
  }
  for (int o = 16; o > 0; o >>= 1) {
    rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
    esum += __shfl_xor_sync(0xffffffffu, esum, o);
    e11 += __shfl_xor_sync(0xffffffffu, e11, o);
  }
  if (lane == 0) {
    red[0][warp] = rsum;
    red[1][warp] = esum;
    red[2][warp] = e11;
  }
  __syncthreads();
  // the warps' sums by a shuffle tree in warp 0 (fixed order)
  if (warp != 0) return;
  double rs = lane < nwarp ? red[0][lane] : 0.0, es = lane < nwarp ? red[1][lane] : 0.0,
         ee = lane < nwarp ? red[2][lane] : 0.0;
  for (int o = 16; o > 0; o >>= 1) {
    rs += __shfl_xor_sync(0xffffffffu, rs, o);
    es += __shfl_xor_sync(0xffffffffu, es, o);
    ee += __shfl_xor_sync(0xffffffffu, ee, o);
  }
  if (tid != 0) return;
  const double res = sqrt(rs) / norm_a;
  const double corr = sqrt(es + ee);
  if (bad || !isfinite(res) || !isfinite(corr)) {
    ctl->status = EIGREF_E_NONFINITE;
    ctl->nonfinite = 1;
    ctl->done = 1;
    ctl->pending_norm = 0;
    return;
  }
  b.hist_res[it] = res;
  b.hist_corr[it] = corr;
  ctl->last_res = res;
  ctl->last_corr = corr;
  ctl->iterations = it + 1;
  ctl->pending_norm = 1;
  const double crit = stop == EIGREF_STOP_CORRECTION ? corr : res;
  if (tol > 0.0 && crit <= tol) {
    ctl->status = EIGREF_OK;
    ctl->done = 1;
  } else if (corr >= 1.0 || (corr > div_factor * emin && corr > div_floor)) {
    ctl->status = EIGREF_E_DIVERGED;
    ctl->done = 1;
  } else if (it + 1 >= max_iters) {
    ctl->status = tol > 0.0 ? EIGREF_E_NOT_CONVERGED : EIGREF_OK;
    ctl->done = 1;
  }
  if (corr < emin) ctl->emin = corr;
}

__global__ void __launch_bounds__(1024) finalize_kernel(SweepBufs b, int k) { finalize_body(b, k); }

// Batch: one CTA per problem.
__global__ void __launch_bounds__(1024) finalize_grouped_kernel(const GroupItem* __restrict__ items, int parity) {
  const GroupItem& it = items[blockIdx.x];
  finalize_body(it.b[parity], it.k);
}

void launch_finalize_grouped(const GroupItem* items, const GroupDims& gd, int parity, cudaStream_t s) {
  finalize_grouped_kernel<<<gd.count, 1024, 0, s>>>(items, parity);
}

cudaError_t init_fp64_attributes() {
  return cudaFuncSetAttribute(update_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)update_smem_max());
}

void launch_finalize(const SweepBufs& b, int k, double, cudaStream_t s) {
  finalize_kernel<<<1, 1024, 0, s>>>(b, k);
}

__device__ __forceinline__ void normalize_body(double* __restrict__ X, int64_t n, int k, const double* __restrict__ nu,
                                               int64_t t0, int64_t stride) {
  const int64_t total = n * k;
  for (int64_t e = t0; e < total; e += stride) X[e] *= nu[e % k];
}

__global__ void normalize_kernel(double* __restrict__ X, int64_t n, int k, const double* __restrict__ nu,
                                 const Control* ctl) {
  if (!ctl->pending_norm) return;
  normalize_body(X, n, k, nu, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

__global__ void normalize_grouped_kernel(const GroupItem* __restrict__ items, int parity) {
  const GroupItem& it = items[blockIdx.z];
  const SweepBufs& b = it.b[parity];
  if (!b.ctl->pending_norm) return;
  normalize_body(b.xn, it.n, it.k, b.nu, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                 (int64_t)gridDim.x * blockDim.x);
}

void launch_normalize_grouped(const GroupItem* items, const GroupDims& gd, int parity, cudaStream_t s) {
  const int64_t total = gd.max_n * gd.max_k;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 64);
  normalize_grouped_kernel<<<dim3(grid, 1, gd.count), 256, 0, s>>>(items, parity);
}

// The same, also forming the column maxima of the normalised |X| (the next
// sweep's slicing of X needs them).  The grid makes the thread count a
// multiple of k, so every thread stays on one column.
__global__ void __launch_bounds__(256) normalize_max_kernel(double* __restrict__ X, int64_t n, int k,
                                                            const double* __restrict__ nu, const Control* ctl,
                                                            unsigned long long* __restrict__ cmax) {
  if (!ctl->pending_norm) return;
  __shared__ unsigned long long colm[kMaxK];
  for (int j = threadIdx.x; j < k; j += blockDim.x) colm[j] = 0ull;
  __syncthreads();
  const int64_t total = n * k;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const double sc = nu[t % k];
  unsigned long long m = 0ull;   // max |X| as an ordered bit pattern (integer compares)
  for (int64_t e = t; e < total; e += T) {
    const double v = X[e] * sc;
    X[e] = v;
    m = umax64(m, (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull);
  }
  if (t < total) atomicMax(&colm[t % k], m);
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x)
    if (colm[j]) atomicMax(cmax + j, colm[j]);
}

// The same for even k with 16-byte accesses: a thread takes column pairs
// (2 c, 2 c + 1), c fixed (the thread count is a multiple of k / 2), and keeps
// four pairs in flight a step, so that HBM, not the latency of one load a
// thread, sets the pace.
__global__ void __launch_bounds__(256) normalize_max2_kernel(double* __restrict__ X, int64_t n, int k,
                                                             const double* __restrict__ nu, const Control* ctl,
                                                             unsigned long long* __restrict__ cmax) {
  if (!ctl->pending_norm) return;
  __shared__ unsigned long long colm[kMaxK];
  for (int j = threadIdx.x; j < k; j += blockDim.x) colm[j] = 0ull;
  __syncthreads();
  const int h = k / 2;
  const int64_t total = n * h;                       // pairs
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int c = (int)(t % h);
  const double s0 = nu[2 * c], s1 = nu[2 * c + 1];
  double2* X2 = reinterpret_cast<double2*>(X);
  unsigned long long m0 = 0ull, m1 = 0ull;
  int64_t e = t;
  for (; e + 3 * T < total; e += 4 * T) {
    double2 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = X2[e + q * T];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[q].x *= s0;
      v[q].y *= s1;
      X2[e + q * T] = v[q];
      m0 = umax64(m0, (unsigned long long)__double_as_longlong(v[q].x) & 0x7FFFFFFFFFFFFFFFull);
      m1 = umax64(m1, (unsigned long long)__double_as_longlong(v[q].y) & 0x7FFFFFFFFFFFFFFFull);
    }
  }
  for (; e < total; e += T) {
    double2 v = X2[e];
    v.x *= s0;
    v.y *= s1;
    X2[e] = v;
    m0 = umax64(m0, (unsigned long long)__double_as_longlong(v.x) & 0x7FFFFFFFFFFFFFFFull);
    m1 = umax64(m1, (unsigned long long)__double_as_longlong(v.y) & 0x7FFFFFFFFFFFFFFFull);
  }
  if (t < total) {
    atomicMax(&colm[2 * c], m0);
    atomicMax(&colm[2 * c + 1], m1);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x)
    if (colm[j]) atomicMax(cmax + j, colm[j]);
}

void launch_normalize(const SweepBufs& b, int64_t n, int k, cudaStream_t s, unsigned long long* cmax) {
  int64_t total = n * k;
  if (cmax && k % 2 == 0 && (reinterpret_cast<uintptr_t>(b.xn) & 15) == 0) {
    // blocks: about 8 per SM, the thread count a multiple of k / 2
    int g = 256, kk = k / 2;
    while (kk % 2 == 0 && g % 2 == 0) { kk /= 2; g /= 2; }
    const int blocks = ((152 * 8 + kk - 1) / kk) * kk;
    normalize_max2_kernel<<<blocks, 256, 0, s>>>(b.xn, n, k, b.nu, b.ctl, cmax);
    return;
  }
  if (cmax) {
    // blocks: about 8 per SM, a multiple of k / gcd(k, 256)
    int g = 256, kk = k;
    while (kk % 2 == 0 && g % 2 == 0) { kk /= 2; g /= 2; }
    const int blocks = ((152 * 8 + kk - 1) / kk) * kk;
    normalize_max_kernel<<<blocks, 256, 0, s>>>(b.xn, n, k, b.nu, b.ctl, cmax);
    return;
  }
  int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  normalize_kernel<<<grid, 256, 0, s>>>(b.xn, n, k, b.nu, b.ctl);
}

// ---------------------------------------------------------------------------
// Layout conversion between the caller's column-major X (ldx) and the
// internal row-major X, with the column signs sigma (sigma may be NULL).
// ---------------------------------------------------------------------------
__global__ void copy_in_kernel(const double* __restrict__ Xu, int64_t ldx, double* __restrict__ X, int64_t n,
                               int k, const double* __restrict__ sigma) {
  const int64_t total = n * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % n;
    int j = (int)(e / n);
    double v = Xu[i + j * ldx];
    X[i * k + j] = sigma ? v * sigma[j] : v;
  }
}

__global__ void copy_out_kernel(const double* __restrict__ X, double* __restrict__ Xu, int64_t ldx, int64_t n,
                                int k, const double* __restrict__ sigma) {
  const int64_t total = n * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e % n;
    int j = (int)(e / n);
    double v = X[i * k + j];
    Xu[i + j * ldx] = sigma ? v * sigma[j] : v;
  }
}

static int grid_for(int64_t total) { return (int)std::min<int64_t>((total + 255) / 256, 152 * 16); }

void launch_copy_in(const double* Xu, int64_t ldx, double* X, int64_t n, int k, const double* sigma,
                    cudaStream_t s) {
  copy_in_kernel<<<grid_for(n * k), 256, 0, s>>>(Xu, ldx, X, n, k, sigma);
}

void launch_copy_out(const double* X, double* Xu, int64_t ldx, int64_t n, int k, const double* sigma,
                     cudaStream_t s) {
  copy_out_kernel<<<grid_for(n * k), 256, 0, s>>>(X, Xu, ldx, n, k, sigma);
}

void launch_rowmajor_to_colmajor(const double* X, double* Xu, int64_t ldx, int64_t n, int k, cudaStream_t s) {
  copy_out_kernel<<<grid_for(n * k), 256, 0, s>>>(X, Xu, ldx, n, k, nullptr);
}

// ---------------------------------------------------------------------------
// ||A||_inf = max_i sum_l |a_il| (the computable bound used for the shift of
// Section 5.1).  Non-negative doubles order like their bit patterns, so the
// maximum is an integer atomicMax.
// ---------------------------------------------------------------------------
__global__ void norm_inf_dense_kernel(const double* __restrict__ A, int64_t n, int64_t lda,
                                      unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    double s = 0.0;
    for (int64_t l = lane; l < n; l += 32) s += fabs(A[i * lda + l]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(s));
  }
}

__global__ void norm_inf_csr_kernel(const int32_t* __restrict__ rp, const double* __restrict__ val, int64_t n,
                                    unsigned long long* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) s += fabs(val[p]);
    atomicMax(out, (unsigned long long)__double_as_longlong(s));
  }
}

void launch_norm_inf_dense(const double* A, int64_t n, int64_t lda, double* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(double), s);
  norm_inf_dense_kernel<<<152 * 8, 256, 0, s>>>(A, n, lda, reinterpret_cast<unsigned long long*>(out));
}

void launch_norm_inf_csr(const int32_t* rp, const double* val, int64_t n, double* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(double), s);
  norm_inf_csr_kernel<<<grid_for(n), 256, 0, s>>>(rp, val, n, reinterpret_cast<unsigned long long*>(out));
}

}  // namespace eigref

// The k x k stage of one sweep of Algorithm 4 (everything between the product
// and the row update, and the top block of the update), in the folded form the
// GPU uses.  With B the refined operator,
// W = B X, subscript 1 = rows 0..k-1 and 2 = rows k..n-1:
//
//   G = X^T X, S = X^T W (split into the top block G1, S1 and the rest G2, S2)
//   alpha_j = G_jj, d_j = S_jj / G_jj                  (Eq. Rayleigh)
//   R1 = W1 - X1 D,  Y1 = X1 - I                       (Algorithm 1: Y = X - I_{n,k})
//   Y^T R = (S - G D) - R1,  Z = S2 - G2 D = X2^T R2
//   M = T^T (Y^T R) = -Y1^{-1} (Y^T R)                 (T = -Y1^{-T})
//   V1 = R1 - Y1 M = S - G D (= X^T R: top rows of V = H^T R, Eq. V-def;
//        V2 = R2 - X2 M is formed by the row update)
//   E11 by the four cases of Algorithm 4 (Eqs. Ediag, Eoffdiag, beta)
//   Y^T E = Y1^T E11 + (Z - G2 M) D^-1                  (E21 = V2 D^-1)
// V1 needs no product: R1 + Y^T R = X1^T R1 + X2^T R2 = X^T R = S - G D, and
// R1 - Y1 M = R1 + Y^T R.  (S - G D is the difference the sweep forms for
// Y^T R anyway, so V1 carries the same rounding as before.)
//   N = T (Y^T E) = -Y1^{-T} (Y^T E)
//   X1' = X1 + E11 - Y1 N,  F = M D^-1 + N             (H E = E - Y N)
// The rows below are updated by update_rows: X2' = X2 + (W2 - X2 D) D^-1 - X2 F.
// This equals H-hat applied through its compact WY factors (Section 3.1.2);
// Y-hat is never formed and T-hat enters only through the LU of Y1.
//
// All k x k matrices are FP64 column-major with leading dimension k.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"

namespace eigref {

// Sum over the first vb threads of the block (the others pass 0), in a fixed
// order that depends on vb only: a grouped launch with more threads gives the
// same bits as a launch of exactly vb threads.
__device__ __forceinline__ double block_sum(double v, double* sh, int vb) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = vb >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < nw; ++q) s += sh[q];
  return s;
}

// One block per column j.  In the split form g2 arrives holding the Gram
// products over all rows; the block turns its column into G2 = G - G1,
// S2 = S - S1 in place (only this block touches column j).
__device__ __forceinline__ void kk_prep_body(const SweepBufs& b, int k, int j, int vb) {
  __shared__ double sh[32];
  const int64_t kk = (int64_t)k * k;
  const double* G1 = b.gtop;
  const double* S1 = b.gtop + kk;
  double* G2 = b.g2;
  double* S2 = b.g2 + kk;
  const bool full = b.mixed != 0;
  const int64_t jj = j + (int64_t)j * k;
  const double al = full ? G2[jj] : G1[jj] + G2[jj];
  const double dj = (full ? S2[jj] : S1[jj] + S2[jj]) / al;
  __syncthreads();
  double r1s = 0.0;
  for (int i = threadIdx.x; i < k && (int)threadIdx.x < vb; i += vb) {
    const int64_t e = i + (int64_t)j * k;
    const double G = full ? G2[e] : G1[e] + G2[e];
    const double S = full ? S2[e] : S1[e] + S2[e];
    const double g2 = full ? G2[e] - G1[e] : G2[e];
    const double s2 = full ? S2[e] - S1[e] : S2[e];
    if (full) {
      G2[e] = g2;
      S2[e] = s2;
    }
    const double x = b.x[(int64_t)i * k + j];
    const double r1 = b.p[(int64_t)i * k + j] - x * dj;
    const double v1 = S - G * dj;   // V1 = X^T R
    b.r1[e] = r1;
    b.v1[e] = v1;
    b.t1[e] = v1 - r1;
    b.z[e] = s2 - g2 * dj;
    b.y1[e] = x - (i == j ? 1.0 : 0.0);
    r1s += r1 * r1;
  }
  if (b.fm_cmax && j == 0)   // read by the last update's slicing; formed again below by the X1 product
    for (int c = threadIdx.x; c < kfm_cols(k); c += blockDim.x) b.fm_cmax[c] = 0ull;
  r1s = block_sum(r1s, sh, vb);
  if (threadIdx.x == 0) {
    if (j == 0) b.ctl->ns_twice = 0;
    b.alpha[j] = al;
    b.d[j] = dj;
    b.dinv[j] = 1.0 / dj;
    b.r1sq[j] = r1s;
  }
}

// Threads of the one-column-per-block kernels for a given k.
__host__ __device__ __forceinline__ int kk_threads(int k) { return k >= 128 ? 128 : ((k + 31) / 32) * 32; }

__global__ void kk_prep_kernel(SweepBufs b, int k) {
  if (b.ctl->done) return;
  kk_prep_body(b, k, blockIdx.x, blockDim.x);
}

__device__ __forceinline__ double nan_max(double a, double b) {   // NaN-propagating max
  return (a != a || b != b) ? __longlong_as_double(0x7FF8000000000000ll) : fmax(a, b);
}

// LU with partial pivoting of Y1 in shared memory (one CTA).  A pivot below
// k u max|Y1| means Y1 is singular to working precision: Algorithm 1 cannot
// proceed, the sweep stops with EIGREF_E_SINGULAR_WY.
__global__ void __launch_bounds__(512) kk_lu_kernel(SweepBufs b, int k) {
  Control* ctl = b.ctl;
  if (ctl->done) return;
  extern __shared__ double a[];
  __shared__ double sh[32];
  __shared__ int s_piv, s_sing;
  const int tid = threadIdx.x;
  const int64_t kk = (int64_t)k * k;
  double amax = 0.0;
  for (int64_t e = tid; e < kk; e += blockDim.x) {
    a[e] = b.y1[e];
    amax = nan_max(amax, fabs(a[e]));
  }
  for (int o = 16; o > 0; o >>= 1) amax = nan_max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((tid & 31) == 0) sh[tid >> 5] = amax;
  if (tid == 0) s_sing = 0;
  __syncthreads();
  amax = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) amax = nan_max(amax, sh[q]);
  if (!isfinite(amax)) {                 // Inf / NaN in X: not a singularity
    if (tid == 0) {
      ctl->nonfinite = 1;
      ctl->status = EIGREF_E_NONFINITE;
      ctl->done = 1;
    }
    return;
  }
  const double thresh = k * kUnitRoundoff * amax;
  for (int p = 0; p < k; ++p) {
    if (tid < 32) {
      double best = -1.0;
      int bi = p;
      for (int i = p + tid; i < k; i += 32) {
        double v = fabs(a[i + (int64_t)p * k]);
        if (v > best) { best = v; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        s_piv = bi;
        b.piv[p] = bi;
        if (!(best > thresh)) s_sing = 1;
      }
    }
    __syncthreads();
    if (s_sing) break;
    const int q = s_piv;
    if (q != p)
      for (int c = tid; c < k; c += blockDim.x) {
        double t = a[p + (int64_t)c * k];
        a[p + (int64_t)c * k] = a[q + (int64_t)c * k];
        a[q + (int64_t)c * k] = t;
      }
    __syncthreads();
    const double pv = a[p + (int64_t)p * k];
    for (int i = p + 1 + tid; i < k; i += blockDim.x) a[i + (int64_t)p * k] /= pv;
    __syncthreads();
    const int m = k - p - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int i = p + 1 + e % m, c = p + 1 + e / m;
      a[i + (int64_t)c * k] -= a[i + (int64_t)p * k] * a[p + (int64_t)c * k];
    }
    __syncthreads();
  }
  if (s_sing) {
    if (tid == 0) {
      ctl->singular = 1;
      ctl->status = EIGREF_E_SINGULAR_WY;
      ctl->done = 1;
    }
    return;
  }
  for (int64_t e = tid; e < kk; e += blockDim.x) b.lu[e] = a[e];
}

// One block per right-hand side column.  MODE 0: out = -Y1^{-1} rhs;
// MODE 1: out = -Y1^{-T} rhs.  With P Y1 = L U (P the row swaps piv):
// Y1 x = b  <=>  L U x = P b;   Y1^T x = b  <=>  U^T L^T (P x) = b.
template <int MODE>
__global__ void kk_solve_kernel(const double* __restrict__ LU, const int* __restrict__ piv,
                                const double* __restrict__ rhs, double* __restrict__ out, int k,
                                const Control* ctl) {
  if (ctl->done) return;
  __shared__ double x[kMaxK];
  const int j = blockIdx.x, tid = threadIdx.x;
  for (int i = tid; i < k; i += blockDim.x) x[i] = rhs[i + (int64_t)j * k];
  __syncthreads();
  if (MODE == 0) {
    if (tid == 0)
      for (int p = 0; p < k; ++p) {
        int q = piv[p];
        double t = x[p]; x[p] = x[q]; x[q] = t;
      }
    __syncthreads();
    for (int p = 0; p < k - 1; ++p) {          // L y = P b (unit lower)
      const double xp = x[p];
      for (int i = p + 1 + tid; i < k; i += blockDim.x) x[i] -= LU[i + (int64_t)p * k] * xp;
      __syncthreads();
    }
    for (int p = k - 1; p >= 0; --p) {         // U x = y
      if (tid == 0) x[p] /= LU[p + (int64_t)p * k];
      __syncthreads();
      const double xp = x[p];
      for (int i = tid; i < p; i += blockDim.x) x[i] -= LU[i + (int64_t)p * k] * xp;
      __syncthreads();
    }
  } else {
    for (int p = 0; p < k; ++p) {              // U^T z = b (lower, diagonal U_pp)
      if (tid == 0) x[p] /= LU[p + (int64_t)p * k];
      __syncthreads();
      const double xp = x[p];
      for (int i = p + 1 + tid; i < k; i += blockDim.x) x[i] -= LU[p + (int64_t)i * k] * xp;
      __syncthreads();
    }
    for (int p = k - 1; p > 0; --p) {          // L^T w = z (unit upper)
      const double xp = x[p];
      for (int i = tid; i < p; i += blockDim.x) x[i] -= LU[p + (int64_t)i * k] * xp;
      __syncthreads();
    }
    if (tid == 0)
      for (int p = k - 1; p >= 0; --p) {       // x = P^T w
        int q = piv[p];
        double t = x[p]; x[p] = x[q]; x[q] = t;
      }
    __syncthreads();
  }
  for (int i = tid; i < k; i += blockDim.x) out[i + (int64_t)j * k] = -x[i];
}

enum { KG_YTE = 2, KG_X1 = 3 };

// The TT rows of op(A) and TT columns of B a tile needs, whole (every load in
// flight at once: these products are latency-bound), into As[r][l] = op(A)(i0
// + r, l) and Bs[l][c] = B(l, j0 + c); zero outside k.
template <int TT>
__device__ __forceinline__ void kk_load_panels(const double* __restrict__ A, bool transA, const double* __restrict__ B,
                                               int k, int i0, int j0, double (*As)[kMaxK + 1],
                                               double (*Bs)[TT + 1]) {
  const int nt = blockDim.x;
  for (int e = threadIdx.x; e < TT * k; e += nt) {
    int r, l;
    if (transA) {   // op(A)(i, l) = A(l, i): l runs along memory
      l = e % k;
      r = e / k;
    } else {
      r = e % TT;
      l = e / TT;
    }
    const int ai = i0 + r;
    As[r][l] = ai < k ? (transA ? A[l + (int64_t)ai * k] : A[ai + (int64_t)l * k]) : 0.0;
  }
  for (int e = threadIdx.x; e < TT * k; e += nt) {
    const int l = e % k, c = e / k;
    const int bj = j0 + c;
    Bs[l][c] = bj < k ? B[l + (int64_t)bj * k] : 0.0;
  }
}

// TT x TT output tile per CTA (TT^2 threads), one output per thread:
// s = op(A)(i,:) . Bm(:,j), summed in the order l = 0, 1, ... for any TT.
//   KG_YTE: Y^T E = Y1^T E11 + (Z - W2) D^-1 with W2 = G2 M formed here too
//           (second panel pair, loaded after the first product)
//   KG_X1:  X1' = X1 + E11 - Y1 N, F = M D^-1 + N (and the [F | M] panel)
template <int MODE, int TT = 16>
__device__ __forceinline__ void kk_gemm_body(const SweepBufs& b, int k, int bx, int by, int done = 0) {
  __shared__ double As[TT][kMaxK + 1];
  __shared__ double Bs[kMaxK][TT + 1];
  const int tx = threadIdx.x % TT, ty = threadIdx.x / TT;
  const int i = bx * TT + tx, j = by * TT + ty;
  const int64_t kk = (int64_t)k * k;
  const double* Bm = (MODE == KG_YTE) ? b.e11 : b.nmat;
  const bool transA = (MODE == KG_YTE);
  kk_load_panels<TT>(b.y1, transA, Bm, k, bx * TT, by * TT, As, Bs);
  __syncthreads();
  if (done) return;
  double s = 0.0;
  for (int l = 0; l < k; ++l) s = fma(As[tx][l], Bs[l][ty], s);
  if (MODE == KG_YTE) {
    __syncthreads();                      // every thread is done with the first panels
    kk_load_panels<TT>(b.g2, false, b.m, k, bx * TT, by * TT, As, Bs);   // G2 = b.g2[0 .. k*k)
    __syncthreads();
    double w2 = 0.0;
    for (int l = 0; l < k; ++l) w2 = fma(As[tx][l], Bs[l][ty], w2);
    if (i >= k || j >= k) return;
    const int64_t e = i + (int64_t)j * k;
    b.yte[e] = s + (b.z[e] - w2) / b.d[j];
    return;
  }
  const bool live = i < k && j < k;
  const int64_t e = i + (int64_t)j * k;
  double f = 0.0, mv = 0.0;
  if (live) {
    b.xn[(int64_t)i * k + j] = b.x[(int64_t)i * k + j] + b.e11[e] - s;
    f = b.m[e] / b.d[j] + b.nmat[e];
    mv = b.m[e];
    b.f[e] = f;
    if (b.fm) {   // the tensor-core update's operand: F and M side by side (X2 F and X2 M in one pass)
      const int64_t c = kfm_col(j);
      b.fm[i + c * k] = f;
      b.fm[i + (c + 16) * k] = mv;
    }
  }
  if (b.fm_cmax) {
    // the panel's column maxima: the TT rows of column j sit on TT consecutive
    // lanes (tx = threadIdx % TT); their maximum, then one atomic a column and tile
    unsigned long long mf = live ? (unsigned long long)__double_as_longlong(f) & 0x7FFFFFFFFFFFFFFFull : 0ull;
    unsigned long long mm = live ? (unsigned long long)__double_as_longlong(mv) & 0x7FFFFFFFFFFFFFFFull : 0ull;
#pragma unroll
    for (int o = 1; o < TT && o < 32; o <<= 1) {
      mf = umax64(mf, __shfl_xor_sync(0xffffffffu, mf, o));
      mm = umax64(mm, __shfl_xor_sync(0xffffffffu, mm, o));
    }
    if (tx == 0 && j < k) {
      const int c = kfm_col(j);
      atomicMax(b.fm_cmax + c, mf);
      atomicMax(b.fm_cmax + c + 16, mm);
    }
  }
  (void)kk;
}

// The stop flag is loaded first and acted on after the panel loads, so the
// two latencies overlap (reading the inputs of a finished run writes nothing).
template <int MODE, int TT>
__global__ void __launch_bounds__(256) kk_gemm_kernel(SweepBufs b, int k) {
  const int done = b.ctl->done;
  kk_gemm_body<MODE, TT>(b, k, blockIdx.x, blockIdx.y, done);
}

// E11 by the cases of Algorithm 4 (Eqs. Ediag, Eoffdiag), one block per column j, plus the
// column sum the finalize step needs: ||E11(:,j)||^2.
__device__ __forceinline__ void kk_e11_body(const SweepBufs& b, int k, double delta, int beta_zero, int j, int vb) {
  __shared__ double sh[32];
  const int64_t kk = (int64_t)k * k;
  const double dj = b.d[j];
  double es = 0.0;
  for (int i = threadIdx.x; i < k && (int)threadIdx.x < vb; i += vb) {
    const int64_t e = i + (int64_t)j * k;
    const double di = b.d[i];
    double v;
    if (i == j) {
      v = (1.0 - b.alpha[i]) * 0.5;                       // Eq. (Ediag)
    } else if (fabs(dj - di) <= delta) {
      v = beta_zero ? 0.0 : -0.5 * (b.gtop[e] + b.g2[e]);  // beta_ij = -x_i^T x_j / 2
    } else {
      v = b.v1[e] / (dj - di);                            // Eq. (Eoffdiag), i, j <= k
    }
    b.e11[e] = v;
    es += v * v;
  }
  es = block_sum(es, sh, vb);
  if (threadIdx.x == 0) b.e11sq[j] = es;
  (void)kk;
}

__global__ void kk_e11_kernel(SweepBufs b, int k, double delta, int beta_zero) {
  if (b.ctl->done) return;
  kk_e11_body(b, k, delta, beta_zero, blockIdx.x, blockDim.x);
}


// ---------------------------------------------------------------------------
// Y1^{-1} for the split form.  An LU of Y1 is a long chain of dependent steps
// on one SM; instead the inverse Z is computed once per call (LU) and then
// corrected every sweep by two Newton-Schulz steps, Z <- Z + Z (I - Y1 Z).
// Each step squares the error ||I - Y1 Z||, which at the start of a sweep is
// of the order of the change of X1 in the last update.  All of it is k x k
// FP64 GEMMs spread over many CTAs.
// ---------------------------------------------------------------------------

// C = add_i I + beta C0 + alpha op(A) B  (k x k, column-major).  check > 0:
// flags Y1 as singular when an entry of C exceeds it (Newton-Schulz diverging).
template <int TRANS, int TT = 16>
__device__ __forceinline__ void kk_gemm_generic_body(const double* __restrict__ A, const double* __restrict__ B,
                                                     const double* __restrict__ C0, double* __restrict__ C, int k,
                                                     double alpha, double beta, int add_i, double check, Control* ctl,
                                                     int bx, int by, int done = 0, double twice_above = 0.0) {
  __shared__ double As[TT][kMaxK + 1];
  __shared__ double Bs[kMaxK][TT + 1];
  const int tx = threadIdx.x % TT, ty = threadIdx.x / TT;
  const int i = bx * TT + tx, j = by * TT + ty;
  kk_load_panels<TT>(A, TRANS != 0, B, k, bx * TT, by * TT, As, Bs);
  __syncthreads();
  if (done) return;
  double acc = 0.0;
  for (int l = 0; l < k; ++l) acc = fma(As[tx][l], Bs[l][ty], acc);
  if (i < k && j < k) {
    const int64_t e = i + (int64_t)j * k;
    double v = alpha * acc;
    if (C0) v += beta * C0[e];
    if (add_i && i == j) v += 1.0;
    C[e] = v;
    if (check > 0.0 && !(fabs(v) <= check)) {
      ctl->singular = 1;
      ctl->status = EIGREF_E_SINGULAR_WY;
      ctl->done = 1;
    }
    if (twice_above > 0.0 && !(fabs(v) <= twice_above)) atomicOr(&ctl->ns_twice, 1);
  }
}

template <int TRANS, int TT>
__global__ void __launch_bounds__(256) kk_gemm_generic_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                                              const double* __restrict__ C0, double* __restrict__ C,
                                                              int k, double alpha, double beta, int add_i,
                                                              double check, Control* ctl) {
  const int done = ctl->done;   // acted on after the panel loads (see kk_gemm_kernel)
  kk_gemm_generic_body<TRANS, TT>(A, B, C0, C, k, alpha, beta, add_i, check, ctl, blockIdx.x, blockIdx.y, done);
}

// Tiles of 8 for k >= 64 (a k x k product then spreads over 64+ SMs), else 16.
__host__ __device__ __forceinline__ int kk_tile(int k) { return k >= 64 ? 8 : 16; }
// Threads of an E11 column block where it shares a launch with a product (TT^2 threads a block).
__host__ __device__ __forceinline__ int kk_e11_vb(int k) {
  const int t = kk_tile(k) * kk_tile(k);
  return kk_threads(k) < t ? kk_threads(k) : t;
}

static void kk_gemm_generic(const double* A, bool transA, const double* B, const double* C0, double* C, int k,
                            double alpha, double beta, int add_i, double check, Control* ctl, cudaStream_t s) {
  if (k >= 64) {
    dim3 g((k + 7) / 8, (k + 7) / 8);
    if (transA)
      kk_gemm_generic_kernel<1, 8><<<g, 64, 0, s>>>(A, B, C0, C, k, alpha, beta, add_i, check, ctl);
    else
      kk_gemm_generic_kernel<0, 8><<<g, 64, 0, s>>>(A, B, C0, C, k, alpha, beta, add_i, check, ctl);
  } else {
    dim3 g((k + 15) / 16, (k + 15) / 16);
    if (transA)
      kk_gemm_generic_kernel<1, 16><<<g, 256, 0, s>>>(A, B, C0, C, k, alpha, beta, add_i, check, ctl);
    else
      kk_gemm_generic_kernel<0, 16><<<g, 256, 0, s>>>(A, B, C0, C, k, alpha, beta, add_i, check, ctl);
  }
}

template <int MODE>
static void kk_gemm(const SweepBufs& b, int k, cudaStream_t s) {
  if (k >= 64)
    kk_gemm_kernel<MODE, 8><<<dim3((k + 7) / 8, (k + 7) / 8), 64, 0, s>>>(b, k);
  else
    kk_gemm_kernel<MODE, 16><<<dim3((k + 15) / 16, (k + 15) / 16), 256, 0, s>>>(b, k);
}

// Y1 = X1 - I from the row-major X, and rhs = -I (so that the LU solve gives Y1^{-1}).
__global__ void kk_inverse_init_kernel(const double* __restrict__ X, int k, double* __restrict__ y1,
                                       double* __restrict__ rhs) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    const int i = e % k, j = e / k;
    y1[e] = X[(int64_t)i * k + j] - (i == j ? 1.0 : 0.0);
    rhs[e] = i == j ? -1.0 : 0.0;
  }
}

void launch_inverse_setup(const SweepBufs& b, int k, cudaStream_t s) {
  const int tpb = kk_threads(k);
  kk_inverse_init_kernel<<<(k * k + 255) / 256, 256, 0, s>>>(b.x, k, b.y1, b.res);
  kk_lu_kernel<<<1, 512, sizeof(double) * (size_t)k * k, s>>>(b, k);
  kk_solve_kernel<0><<<k, tpb, 0, s>>>(b.lu, b.piv, b.res, b.zinv, k, b.ctl);   // Z = -Y1^{-1}(-I)
}

// The Newton-Schulz refresh of Z ~ Y1^{-1} (split form), one step
// Z' = Z + Z T, T = I - Y1 Z, squaring ||T||.  X changes by O(||E||) a sweep,
// so Z kept from the last sweep starts at ||T|| ~ ||E||; a second step runs
// only when the first T has an entry above 2^-27 (then ||T'|| would stay above
// u), and that second T' is the one checked for Y1 turning singular (> 0.5:
// the iteration would not contract).
constexpr double kNsOnce = 7.450580596923828e-09;   // 2^-27

// First product T = I - Y1 Z into res, asking for the second step where due;
// blocks past the product's tiles form E11 (column blk - tiles), which needs
// only the quotients and V1 of the prep step.
template <int TT>
__device__ __forceinline__ void kk_ns_first_body(const SweepBufs& b, int k, double delta, int beta_zero, int blk,
                                                 int done) {
  const int nt = (k + TT - 1) / TT;
  if (blk < nt * nt) {
    kk_gemm_generic_body<0, TT>(b.y1, b.zinv, nullptr, b.res, k, -1.0, 0.0, 1, 0.0, b.ctl, blk % nt, blk / nt, done,
                                kNsOnce);
  } else if (blk - nt * nt < k && !done) {
    kk_e11_body(b, k, delta, beta_zero, blk - nt * nt, kk_e11_vb(k));
  }
}

template <int TT>
__global__ void __launch_bounds__(256) kk_ns_first_kernel(SweepBufs b, int k, double delta, int beta_zero) {
  const int done = b.ctl->done;   // acted on after the panel loads
  kk_ns_first_body<TT>(b, k, delta, beta_zero, blockIdx.x, done);
}

// Second step, T' = I - Y1 Z' (checked) and Z = Z' + Z' T'; without it Z = Z'.
template <int TT>
__device__ __forceinline__ void kk_ns_second_body(const SweepBufs& b, int k, int op, int bx, int by, int done) {
  const int twice = b.ctl->ns_twice;
  if (op == 0) {
    if (!twice) return;
    kk_gemm_generic_body<0, TT>(b.y1, b.zinv2, nullptr, b.res, k, -1.0, 0.0, 1, 0.5, b.ctl, bx, by, done);
  } else if (twice) {
    kk_gemm_generic_body<0, TT>(b.zinv2, b.res, b.zinv2, b.zinv, k, 1.0, 1.0, 0, 0.0, b.ctl, bx, by, done);
  } else if (!done) {
    const int i = bx * TT + (int)threadIdx.x % TT, j = by * TT + (int)threadIdx.x / TT;
    if (i < k && j < k) b.zinv[i + (int64_t)j * k] = b.zinv2[i + (int64_t)j * k];
  }
}

template <int TT>
__global__ void __launch_bounds__(256) kk_ns_second_kernel(SweepBufs b, int k, int op) {
  const int done = b.ctl->done;
  kk_ns_second_body<TT>(b, k, op, blockIdx.x, blockIdx.y, done);
}

template <int TT>
static void kk_ns_launches(const SweepBufs& b, int k, double delta, int beta_zero, cudaStream_t s) {
  const int nt = (k + TT - 1) / TT;
  kk_ns_first_kernel<TT><<<nt * nt + k, TT * TT, 0, s>>>(b, k, delta, beta_zero);                    // T, E11
  kk_gemm_generic(b.zinv, false, b.res, b.zinv, b.zinv2, k, 1.0, 1.0, 0, 0.0, b.ctl, s);             // Z' = Z + Z T
  kk_ns_second_kernel<TT><<<dim3(nt, nt), TT * TT, 0, s>>>(b, k, 0);                                 // T' (if due)
  kk_ns_second_kernel<TT><<<dim3(nt, nt), TT * TT, 0, s>>>(b, k, 1);                                 // Z
}

void launch_kxk_stage(const SweepBufs& b, int k, double delta, int beta_zero, cudaStream_t s) {
  const int tpb = kk_threads(k);
  kk_prep_kernel<<<k, tpb, 0, s>>>(b, k);
  if (b.mixed) {
    if (k >= 64)
      kk_ns_launches<8>(b, k, delta, beta_zero, s);
    else
      kk_ns_launches<16>(b, k, delta, beta_zero, s);
    kk_gemm_generic(b.zinv, false, b.t1, nullptr, b.m, k, -1.0, 0.0, 0, 0.0, b.ctl, s);        // M = -Z (Y^T R)
  } else {
    kk_e11_kernel<<<k, tpb, 0, s>>>(b, k, delta, beta_zero);
    kk_lu_kernel<<<1, 512, sizeof(double) * (size_t)k * k, s>>>(b, k);
    kk_solve_kernel<0><<<k, tpb, 0, s>>>(b.lu, b.piv, b.t1, b.m, k, b.ctl);
  }
  kk_gemm<KG_YTE>(b, k, s);                                                                     // Y^T E (W2 inside)
  if (b.mixed)
    kk_gemm_generic(b.zinv, true, b.yte, nullptr, b.nmat, k, -1.0, 0.0, 0, 0.0, b.ctl, s);     // N = -Z^T (Y^T E)
  else
    kk_solve_kernel<1><<<k, tpb, 0, s>>>(b.lu, b.piv, b.yte, b.nmat, k, b.ctl);
  kk_gemm<KG_X1>(b, k, s);
}

// ---------------------------------------------------------------------------
// The same stage for a batch (split form, Newton-Schulz inverse): each launch
// covers every problem, blockIdx.z selecting it; CTAs outside a problem's
// k x k extent return at once.  Tiles of 16 for every problem.
// ---------------------------------------------------------------------------
__global__ void kk_prep_grouped_kernel(const GroupItem* __restrict__ items, int parity) {
  const GroupItem& it = items[blockIdx.z];
  const SweepBufs& b = it.b[parity];
  if ((int)blockIdx.x >= it.k || b.ctl->done) return;
  kk_prep_body(b, it.k, blockIdx.x, kk_threads(it.k));
}

template <int MODE>
__global__ void __launch_bounds__(256) kk_gemm_grouped_kernel(const GroupItem* __restrict__ items, int parity) {
  const GroupItem& it = items[blockIdx.z];
  const SweepBufs& b = it.b[parity];
  if ((int)blockIdx.x * 16 >= it.k || (int)blockIdx.y * 16 >= it.k) return;
  kk_gemm_body<MODE>(b, it.k, blockIdx.x, blockIdx.y, b.ctl->done);   // the flag is acted on after the loads
}

// First Newton-Schulz product with E11 (16 x 16 tiles: blocks 0 .. nt^2 - 1 of
// the problem's own nt = ceil(k / 16), then its k E11 columns).
__global__ void __launch_bounds__(256) kk_ns_first_grouped_kernel(const GroupItem* __restrict__ items, int parity) {
  const GroupItem& it = items[blockIdx.z];
  const SweepBufs& b = it.b[parity];
  const int nt = (it.k + 15) / 16;
  if ((int)blockIdx.x >= nt * nt + it.k) return;
  const int done = b.ctl->done;
  if ((int)blockIdx.x < nt * nt) {
    kk_gemm_generic_body<0, 16>(b.y1, b.zinv, nullptr, b.res, it.k, -1.0, 0.0, 1, 0.0, b.ctl, blockIdx.x % nt,
                                blockIdx.x / nt, done, kNsOnce);
  } else if (!done) {
    kk_e11_body(b, it.k, it.delta, it.beta_zero, blockIdx.x - nt * nt, kk_e11_vb(it.k));   // as a single problem's
  }
}

__global__ void __launch_bounds__(256) kk_ns_second_grouped_kernel(const GroupItem* __restrict__ items, int parity,
                                                                   int op) {
  const GroupItem& it = items[blockIdx.z];
  const SweepBufs& b = it.b[parity];
  if ((int)blockIdx.x * 16 >= it.k || (int)blockIdx.y * 16 >= it.k) return;
  kk_ns_second_body<16>(b, it.k, op, blockIdx.x, blockIdx.y, b.ctl->done);
}

// The products of the Newton-Schulz refresh and of M, N (see launch_kxk_stage).
enum { NS_Z1 = 1, NS_M = 4, NS_N = 5 };

template <int OP>
__global__ void __launch_bounds__(256) kk_ns_grouped_kernel(const GroupItem* __restrict__ items, int parity) {
  const GroupItem& it = items[blockIdx.z];
  const SweepBufs& b = it.b[parity];
  const int k = it.k;
  if ((int)blockIdx.x * 16 >= k || (int)blockIdx.y * 16 >= k) return;
  const int done = b.ctl->done;   // acted on after the panel loads
  const int bx = blockIdx.x, by = blockIdx.y;
  if (OP == NS_Z1) kk_gemm_generic_body<0>(b.zinv, b.res, b.zinv, b.zinv2, k, 1.0, 1.0, 0, 0.0, b.ctl, bx, by, done);
  if (OP == NS_M) kk_gemm_generic_body<0>(b.zinv, b.t1, nullptr, b.m, k, -1.0, 0.0, 0, 0.0, b.ctl, bx, by, done);
  if (OP == NS_N) kk_gemm_generic_body<1>(b.zinv, b.yte, nullptr, b.nmat, k, -1.0, 0.0, 0, 0.0, b.ctl, bx, by, done);
}

void launch_kxk_stage_grouped(const GroupItem* items, const GroupDims& gd, int parity, cudaStream_t s) {
  const int k = gd.max_k;
  const int tpb = kk_threads(k);
  const int nt = (k + 15) / 16;
  const dim3 gk(k, 1, gd.count);
  const dim3 gt(nt, nt, gd.count);
  kk_prep_grouped_kernel<<<gk, tpb, 0, s>>>(items, parity);
  kk_ns_first_grouped_kernel<<<dim3(nt * nt + k, 1, gd.count), 256, 0, s>>>(items, parity);   // T, E11
  kk_ns_grouped_kernel<NS_Z1><<<gt, 256, 0, s>>>(items, parity);
  kk_ns_second_grouped_kernel<<<gt, 256, 0, s>>>(items, parity, 0);
  kk_ns_second_grouped_kernel<<<gt, 256, 0, s>>>(items, parity, 1);
  kk_ns_grouped_kernel<NS_M><<<gt, 256, 0, s>>>(items, parity);
  kk_gemm_grouped_kernel<KG_YTE><<<gt, 256, 0, s>>>(items, parity);
  kk_ns_grouped_kernel<NS_N><<<gt, 256, 0, s>>>(items, parity);
  kk_gemm_grouped_kernel<KG_X1><<<gt, 256, 0, s>>>(items, parity);
}

// ---------------------------------------------------------------------------
// Rayleigh--Ritz preprocessing (Section 3.3): with G = X^T X and S = X^T B X,
// solve S V = G V D, then Z = X V has Z^T Z = I and Z^T B Z = D.  One CTA:
// Cholesky G = L L^T, C = L^-1 S L^-T, cyclic Jacobi C = Q D Q^T (parallel
// round-robin ordering: each round rotates k/2 disjoint pairs), Ritz pairs
// ordered by |D| descending, V = L^-T Q.  C lives in shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) rr_kernel(const double* __restrict__ gtop, const double* __restrict__ g2,
                                                  int k, double* __restrict__ L, double* __restrict__ W,
                                                  double* __restrict__ Q, double* __restrict__ V,
                                                  double* __restrict__ lam, Control* ctl) {
  extern __shared__ double C[];                  // k x k, column-major
  __shared__ double red[32];
  __shared__ int s_bad;
  __shared__ int perm[kMaxK];
  __shared__ double rot_c[kMaxK / 2 + 1], rot_s[kMaxK / 2 + 1];
  __shared__ int rot_p[kMaxK / 2 + 1], rot_q[kMaxK / 2 + 1];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t kk = (int64_t)k * k;
  if (tid == 0) s_bad = 0;
  // G, S over all rows = leading block + the rest
  for (int64_t e = tid; e < kk; e += nt) {
    L[e] = gtop[e] + g2[e];
    C[e] = gtop[kk + e] + g2[kk + e];
  }
  __syncthreads();
  // symmetrise S (its rounding asymmetry carries no information)
  for (int64_t e = tid; e < kk; e += nt) {
    const int i = (int)(e % k), j = (int)(e / k);
    if (i < j) {
      const double v = 0.5 * (C[e] + C[j + (int64_t)i * k]);
      C[e] = v;
      C[j + (int64_t)i * k] = v;
    }
  }
  // Cholesky of G (right-looking, lower triangle of L)
  for (int p = 0; p < k; ++p) {
    __syncthreads();
    if (tid == 0) {
      const double a = L[p + (int64_t)p * k];
      if (!(a > 0.0) || !isfinite(a)) s_bad = 1;
      L[p + (int64_t)p * k] = sqrt(a);
    }
    __syncthreads();
    if (s_bad) break;
    const double lpp = L[p + (int64_t)p * k];
    for (int i = p + 1 + tid; i < k; i += nt) L[i + (int64_t)p * k] /= lpp;
    __syncthreads();
    const int m = k - p - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int i = p + 1 + e % m, j = p + 1 + e / m;
      if (i >= j) L[i + (int64_t)j * k] -= L[i + (int64_t)p * k] * L[j + (int64_t)p * k];
    }
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) {
      ctl->singular = 1;
      ctl->status = EIGREF_E_SINGULAR_WY;
      ctl->done = 1;
    }
    return;
  }
  // W = L^-1 S (one column per thread), then C = L^-1 W^T
  for (int c = tid; c < k; c += nt)
    for (int i = 0; i < k; ++i) {
      double v = C[i + (int64_t)c * k];
      for (int l = 0; l < i; ++l) v -= L[i + (int64_t)l * k] * W[l + (int64_t)c * k];
      W[i + (int64_t)c * k] = v / L[i + (int64_t)i * k];
    }
  __syncthreads();
  for (int c = tid; c < k; c += nt)
    for (int i = 0; i < k; ++i) {
      double v = W[c + (int64_t)i * k];                     // (W^T)(i, c)
      for (int l = 0; l < i; ++l) v -= L[i + (int64_t)l * k] * C[l + (int64_t)c * k];
      C[i + (int64_t)c * k] = v / L[i + (int64_t)i * k];
    }
  __syncthreads();
  for (int64_t e = tid; e < kk; e += nt) {
    const int i = (int)(e % k), j = (int)(e / k);
    Q[e] = i == j ? 1.0 : 0.0;
    if (i < j) {
      const double v = 0.5 * (C[e] + C[j + (int64_t)i * k]);
      C[e] = v;
      C[j + (int64_t)i * k] = v;
    }
  }
  // cyclic Jacobi, round-robin pairs over m = k rounded up to even players
  const int m = k + (k & 1);
  const int half = m / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    __syncthreads();
    double off = 0.0, tot = 0.0;
    for (int64_t e = tid; e < kk; e += nt) {
      const double v = C[e] * C[e];
      tot += v;
      if (e % k != e / k) off += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = off;
    __syncthreads();
    double offs = 0.0;
    for (int q = 0; q < (nt >> 5); ++q) offs += red[q];
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = tot;
    __syncthreads();
    double tots = 0.0;
    for (int q = 0; q < (nt >> 5); ++q) tots += red[q];
    if (!(offs > kUnitRoundoff * kUnitRoundoff * tots)) break;   // also leaves on NaN
    for (int r = 0; r < m - 1; ++r) {
      __syncthreads();
      if (tid < half) {
        int p, q;
        if (tid == 0) {
          p = r;
          q = m - 1;
        } else {
          p = (r + tid) % (m - 1);
          q = (r - tid + (m - 1)) % (m - 1);
        }
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, sn = 0.0;
        if (q < k) {
          const double apq = C[p + (int64_t)q * k];
          if (apq != 0.0) {
            const double th = (C[q + (int64_t)q * k] - C[p + (int64_t)p * k]) / (2.0 * apq);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
          }
        }
        rot_p[tid] = p;
        rot_q[tid] = q;
        rot_c[tid] = c;
        rot_s[tid] = sn;
      }
      __syncthreads();
      // C <- C J (columns p, q), Q <- Q J
      for (int e = tid; e < half * k; e += nt) {
        const int a = e / k, i = e % k;
        const int p = rot_p[a], q = rot_q[a];
        if (q >= k) continue;
        const double c = rot_c[a], sn = rot_s[a];
        const double cp = C[i + (int64_t)p * k], cq = C[i + (int64_t)q * k];
        C[i + (int64_t)p * k] = c * cp - sn * cq;
        C[i + (int64_t)q * k] = sn * cp + c * cq;
        const double qp = Q[i + (int64_t)p * k], qq = Q[i + (int64_t)q * k];
        Q[i + (int64_t)p * k] = c * qp - sn * qq;
        Q[i + (int64_t)q * k] = sn * qp + c * qq;
      }
      __syncthreads();
      // C <- J^T C (rows p, q)
      for (int e = tid; e < half * k; e += nt) {
        const int a = e / k, j = e % k;
        const int p = rot_p[a], q = rot_q[a];
        if (q >= k) continue;
        const double c = rot_c[a], sn = rot_s[a];
        const double cp = C[p + (int64_t)j * k], cq = C[q + (int64_t)j * k];
        C[p + (int64_t)j * k] = c * cp - sn * cq;
        C[q + (int64_t)j * k] = sn * cp + c * cq;
      }
    }
  }
  __syncthreads();
  // order by |eigenvalue| descending (stable)
  if (tid == 0) {
    for (int i = 0; i < k; ++i) perm[i] = i;
    for (int i = 1; i < k; ++i) {
      const int v = perm[i];
      const double av = fabs(C[v + (int64_t)v * k]);
      int j = i - 1;
      while (j >= 0 && fabs(C[perm[j] + (int64_t)perm[j] * k]) < av) {
        perm[j + 1] = perm[j];
        --j;
      }
      perm[j + 1] = v;
    }
  }
  __syncthreads();
  for (int j = tid; j < k; j += nt) lam[j] = C[perm[j] + (int64_t)perm[j] * k];
  // V = L^-T Q(:, perm): back substitution with the upper factor L^T
  for (int c = tid; c < k; c += nt) {
    const int pc = perm[c];
    for (int i = k - 1; i >= 0; --i) {
      double v = Q[i + (int64_t)pc * k];
      for (int l = i + 1; l < k; ++l) v -= L[l + (int64_t)i * k] * V[l + (int64_t)c * k];
      V[i + (int64_t)c * k] = v / L[i + (int64_t)i * k];
    }
  }
}

// Z = X V for row-major X, Z (n x k) and column-major V (k x k), V in shared memory.
__global__ void __launch_bounds__(256) xv_kernel(const double* __restrict__ X, const double* __restrict__ V,
                                                 double* __restrict__ Z, int64_t n, int k) {
  extern __shared__ double Vs[];
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Vs[e] = V[e];
  __syncthreads();
  const int64_t total = n * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / k;
    const int j = (int)(e % k);
    const double* xr = X + i * k;
    double s = 0.0;
    for (int l = 0; l < k; ++l) s = fma(xr[l], Vs[l + j * k], s);
    Z[e] = s;
  }
}

// Column signs that make each column's largest-magnitude entry (first on ties) positive.
__global__ void colsign_kernel(const double* __restrict__ Z, int64_t n, int k, double* __restrict__ sg) {
  const int lane = threadIdx.x & 31;
  const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (j >= k) return;
  double best = -1.0, val = 0.0;
  int64_t bi = INT64_MAX;
  for (int64_t i = lane; i < n; i += 32) {
    const double v = Z[i * k + j];
    if (fabs(v) > best) { best = fabs(v); val = v; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const double ov = __shfl_xor_sync(0xffffffffu, val, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; val = ov; bi = oi; }
  }
  if (lane == 0) sg[j] = val < 0.0 ? -1.0 : 1.0;
}

// Out = In diag(sg) (row-major n x k).
__global__ void scale_cols_kernel(const double* __restrict__ In, double* __restrict__ Out, int64_t n, int k,
                                  const double* __restrict__ sg) {
  const int64_t total = n * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    Out[e] = In[e] * sg[e % k];
}

// V = (3 I - G) / 2 with G = G1 + G2 (leading block + rest): the first-order
// symmetric (Loewdin) orthonormaliser, X V = X (X^T X)^{-1/2} + O(||G - I||^2).
__global__ void loewdin_kernel(const double* __restrict__ gtop, const double* __restrict__ g2, int k,
                               double* __restrict__ V) {
  const int64_t kk = (int64_t)k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < kk; e += (int64_t)gridDim.x * blockDim.x) {
    const double g = gtop[e] + g2[e];
    V[e] = (e % k == e / k ? 1.5 : 0.0) - 0.5 * g;
  }
}

void launch_reorthonormalise(const SweepBufs& b, int64_t n, int k, double* Xbuf, double* Zbuf, int64_t chunk_rows,
                             int nchunks, cudaStream_t s) {
  const int64_t total = n * k;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  for (int step = 0; step < 2; ++step) {   // each step squares ||X^T X - I||
    launch_gram(Xbuf, Xbuf, k, k, n, chunk_rows, nchunks, b.gpart, b.g2, nullptr, s);
    launch_gram(Xbuf, Xbuf, k, 0, k, k, 1, b.gpart, b.gtop, nullptr, s);
    loewdin_kernel<<<(k * k + 255) / 256, 256, 0, s>>>(b.gtop, b.g2, k, b.f);
    xv_kernel<<<grid, 256, sizeof(double) * (size_t)k * k, s>>>(Xbuf, b.f, Zbuf, n, k);
    cudaMemcpyAsync(Xbuf, Zbuf, (size_t)total * sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
}

void launch_rayleigh_ritz(const SweepBufs& b, int64_t n, int k, double* Xbuf, double* Zbuf, cudaStream_t s) {
  // G, S of X (gtop + g2) must be in place; b.lu, b.res, b.z are k x k scratch, b.f receives V
  rr_kernel<<<1, 1024, sizeof(double) * (size_t)k * k, s>>>(b.gtop, b.g2, k, b.lu, b.res, b.z, b.f, b.d, b.ctl);
  const int64_t total = n * k;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  xv_kernel<<<grid, 256, sizeof(double) * (size_t)k * k, s>>>(Xbuf, b.f, Zbuf, n, k);
  colsign_kernel<<<(k * 32 + 255) / 256, 256, 0, s>>>(Zbuf, n, k, b.nu);
  scale_cols_kernel<<<grid, 256, 0, s>>>(Zbuf, Xbuf, n, k, b.nu);
}

// Signs of Algorithm 2 on the leading k x k block of the caller's X
// (column-major, ldx): sigma_j = -sign(q_jj), sign(0) = +1, unpivoted
// elimination of Q - Sigma.  The shifted pivot |q_jj| + 1 is never zero.
__global__ void __launch_bounds__(512) sign_fix_kernel(const double* __restrict__ X, int64_t rs, int64_t cs, int k,
                                                       double* __restrict__ sigma) {
  extern __shared__ double a[];
  const int tid = threadIdx.x;
  for (int64_t e = tid; e < (int64_t)k * k; e += blockDim.x) {
    int i = (int)(e % k), c = (int)(e / k);
    a[e] = X[i * rs + (int64_t)c * cs];
  }
  __syncthreads();
  for (int p = 0; p < k; ++p) {
    const double app = a[p + (int64_t)p * k];
    const double sg = -(app >= 0.0 ? 1.0 : -1.0);
    __syncthreads();
    if (tid == 0) {
      sigma[p] = sg;
      a[p + (int64_t)p * k] = app - sg;
    }
    __syncthreads();
    const double pv = a[p + (int64_t)p * k];
    for (int i = p + 1 + tid; i < k; i += blockDim.x) a[i + (int64_t)p * k] /= pv;
    __syncthreads();
    const int m = k - p - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int i = p + 1 + e % m, c = p + 1 + e / m;
      a[i + (int64_t)c * k] -= a[i + (int64_t)p * k] * a[p + (int64_t)c * k];
    }
    __syncthreads();
  }
}

cudaError_t init_kxk_attributes() {
  cudaError_t e = cudaFuncSetAttribute(kk_lu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double) * kMaxK * kMaxK));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(rr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double) * kMaxK * kMaxK));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(xv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double) * kMaxK * kMaxK));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sign_fix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(double) * kMaxK * kMaxK));
}

void launch_sign_fix(const double* X, int64_t ldx, int k, double* sigma, int* /*singular*/, cudaStream_t s) {
  sign_fix_kernel<<<1, 512, sizeof(double) * (size_t)k * k, s>>>(X, 1, ldx, k, sigma);
}

void launch_sign_fix_rowmajor(const double* X, int k, double* sigma, cudaStream_t s) {
  sign_fix_kernel<<<1, 512, sizeof(double) * (size_t)k * k, s>>>(X, k, 1, k, sigma);
}

void launch_scale_cols(const double* In, double* Out, int64_t n, int k, const double* sg, cudaStream_t s) {
  const int64_t total = n * k;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
  scale_cols_kernel<<<grid, 256, 0, s>>>(In, Out, n, k, sg);
}

}  // namespace eigref

// The k x k stage of one sweep (Algorithm 4, lines 2-6 and the top block of
// line 7), in the folded form the GPU uses.  With B the refined operator,
// W = B X, subscript 1 = rows 0..k-1 and 2 = rows k..n-1:
//
//   G = X^T X, S = X^T W (split into the top block G1, S1 and the rest G2, S2)
//   alpha_j = G_jj, d_j = S_jj / G_jj                  (lines 3-4, Eq. Rayleigh)
//   R1 = W1 - X1 D,  Y1 = X1 - I                       (Algorithm 1: Y = X - I_{n,k})
//   Y^T R = (S - G D) - R1,  Z = S2 - G2 D = X2^T R2
//   M = T^T (Y^T R) = -Y1^{-1} (Y^T R)                 (T = -Y1^{-T})
//   V1 = R1 - Y1 M   (top rows of V = H^T R, Eq. V-def; V2 = R2 - X2 M)
//   E11 by the four cases of line 6 (Eqs. Ediag, Eoffdiag, beta)
//   Y^T E = Y1^T E11 + (Z - G2 M) D^-1                  (E21 = V2 D^-1)
//   N = T (Y^T E) = -Y1^{-T} (Y^T E)
//   X1' = X1 + E11 - Y1 N,  F = M D^-1 + N             (H E = E - Y N)
// The rows below are updated by update_rows: X2' = X2 + (W2 - X2 D) D^-1 - X2 F.
// This equals H-hat applied through its compact WY factors (Section 3.1.2);
// Y-hat is never formed and T-hat enters only through the LU of Y1.
//
// All k x k matrices are FP64 column-major with leading dimension k.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"

namespace eigref {

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < nw; ++q) s += sh[q];
  return s;
}

// One block per column j.
__global__ void kk_prep_kernel(SweepBufs b, int k) {
  if (b.ctl->done) return;
  __shared__ double sh[32];
  const int j = blockIdx.x;
  const int64_t kk = (int64_t)k * k;
  const double* G1 = b.gtop;
  const double* S1 = b.gtop + kk;
  const double* G2 = b.g2;
  const double* S2 = b.g2 + kk;
  const int64_t jj = j + (int64_t)j * k;
  const double al = G1[jj] + G2[jj];
  const double dj = (S1[jj] + S2[jj]) / al;
  double r1s = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const int64_t e = i + (int64_t)j * k;
    const double G = G1[e] + G2[e], S = S1[e] + S2[e];
    const double x = b.x[(int64_t)i * k + j];
    const double r1 = b.p[(int64_t)i * k + j] - x * dj;
    b.r1[e] = r1;
    b.t1[e] = (S - G * dj) - r1;
    b.z[e] = S2[e] - G2[e] * dj;
    b.y1[e] = x - (i == j ? 1.0 : 0.0);
    r1s += r1 * r1;
  }
  r1s = block_sum(r1s, sh);
  if (threadIdx.x == 0) {
    b.alpha[j] = al;
    b.d[j] = dj;
    b.r1sq[j] = r1s;
  }
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

enum { KG_V1 = 0, KG_W2 = 1, KG_YTE = 2, KG_X1 = 3 };

// 16 x 16 output tile per CTA, one output per thread:  s = op(A)(i,:) . Bm(:,j)
template <int MODE>
__global__ void __launch_bounds__(256) kk_gemm_kernel(SweepBufs b, int k) {
  if (b.ctl->done) return;
  __shared__ double As[16][17];
  __shared__ double Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i = blockIdx.x * 16 + tx, j = blockIdx.y * 16 + ty;
  const int64_t kk = (int64_t)k * k;
  const double* A = (MODE == KG_W2) ? b.g2 : b.y1;   // G2 = b.g2[0 .. k*k)
  const double* Bm = (MODE == KG_YTE) ? b.e11 : (MODE == KG_X1 ? b.nmat : b.m);
  const bool transA = (MODE == KG_YTE);
  double s = 0.0;
  for (int l0 = 0; l0 < k; l0 += 16) {
    // As[r][c] = op(A)(blockIdx.x*16 + r, l0 + c); Bs[r][c] = Bm(l0 + r, blockIdx.y*16 + c)
    {
      const int r = ty, c = tx;  // each thread loads one element of each tile
      const int ai = blockIdx.x * 16 + r, al = l0 + c;
      double av = 0.0;
      if (ai < k && al < k) av = transA ? A[al + (int64_t)ai * k] : A[ai + (int64_t)al * k];
      As[r][c] = av;
      const int bl = l0 + r, bj = blockIdx.y * 16 + c;
      Bs[r][c] = (bl < k && bj < k) ? Bm[bl + (int64_t)bj * k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 16; ++c) s = fma(As[tx][c], Bs[c][ty], s);
    __syncthreads();
  }
  if (i >= k || j >= k) return;
  const int64_t e = i + (int64_t)j * k;
  if (MODE == KG_V1) {
    b.v1[e] = b.r1[e] - s;
  } else if (MODE == KG_W2) {
    b.w2[e] = s;
  } else if (MODE == KG_YTE) {
    b.yte[e] = s + (b.z[e] - b.w2[e]) / b.d[j];
  } else {
    b.xn[(int64_t)i * k + j] = b.x[(int64_t)i * k + j] + b.e11[e] - s;
    b.f[e] = b.m[e] / b.d[j] + b.nmat[e];
  }
  (void)kk;
}

// E11 by the cases of line 6 of Algorithm 4, one block per column j, plus the
// column sums the finalize step needs: ||E11(:,j)||^2, (M^T Z)_jj, (M^T G2 M)_jj.
__global__ void kk_e11_kernel(SweepBufs b, int k, double delta, int beta_zero) {
  if (b.ctl->done) return;
  __shared__ double sh[32];
  const int j = blockIdx.x;
  const int64_t kk = (int64_t)k * k;
  const double dj = b.d[j];
  double es = 0.0, cz = 0.0, cw = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
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
    const double mij = b.m[e];
    cz += mij * b.z[e];
    cw += mij * b.w2[e];
  }
  es = block_sum(es, sh);
  cz = block_sum(cz, sh);
  cw = block_sum(cw, sh);
  if (threadIdx.x == 0) {
    b.e11sq[j] = es;
    b.cz[j] = cz;
    b.cw[j] = cw;
  }
  (void)kk;
}


// ---------------------------------------------------------------------------
// Mixed precision for the two k x k systems of the split form: Y1 is
// factored in FP32 (64x the FP64 rate on this part), each solve is refined
// twice against the FP64 residual, which brings the solution to FP64 accuracy
// for cond(Y1) << 1 / u32 (the sign fix keeps cond(Y1) small).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) kk_lu32_kernel(SweepBufs b, int k) {
  Control* ctl = b.ctl;
  if (ctl->done) return;
  extern __shared__ float af[];
  __shared__ float sh[32];
  __shared__ int s_piv, s_sing, s_bad;
  float* lu32 = reinterpret_cast<float*>(b.lu);
  const int tid = threadIdx.x;
  const int64_t kk = (int64_t)k * k;
  float amax = 0.f;
  int bad = 0;
  for (int64_t e = tid; e < kk; e += blockDim.x) {
    const double v = b.y1[e];
    bad |= !isfinite(v);
    af[e] = (float)v;
    amax = fmaxf(amax, fabsf(af[e]));
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  bad = __any_sync(0xffffffffu, bad);
  if ((tid & 31) == 0) sh[tid >> 5] = amax;
  if (tid == 0) {
    s_sing = 0;
    s_bad = 0;
  }
  __syncthreads();
  if (bad) s_bad = 1;
  __syncthreads();
  if (s_bad) {
    if (tid == 0) {
      ctl->nonfinite = 1;
      ctl->status = EIGREF_E_NONFINITE;
      ctl->done = 1;
    }
    return;
  }
  amax = 0.f;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) amax = fmaxf(amax, sh[q]);
  const float thresh = (float)k * 5.9604645e-08f * amax;   // k u_32 max|Y1|
  for (int p = 0; p < k; ++p) {
    if (tid < 32) {
      float best = -1.f;
      int bi = p;
      for (int i = p + tid; i < k; i += 32) {
        const float v = fabsf(af[i + (int64_t)p * k]);
        if (v > best) { best = v; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
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
        const float t = af[p + (int64_t)c * k];
        af[p + (int64_t)c * k] = af[q + (int64_t)c * k];
        af[q + (int64_t)c * k] = t;
      }
    __syncthreads();
    const float pv = af[p + (int64_t)p * k];
    for (int i = p + 1 + tid; i < k; i += blockDim.x) af[i + (int64_t)p * k] /= pv;
    __syncthreads();
    const int m = k - p - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int i = p + 1 + e % m, c = p + 1 + e / m;
      af[i + (int64_t)c * k] -= af[i + (int64_t)p * k] * af[p + (int64_t)c * k];
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
  for (int64_t e = tid; e < kk; e += blockDim.x) lu32[e] = af[e];
}

// One block per right-hand side: x = op(Y1)^{-1} (neg ? -rhs : rhs) with the
// FP32 factors, then out = x (acc = 0) or out += x (acc = 1), in FP64.
template <int TRANS>
__global__ void kk_solve32_kernel(const float* __restrict__ LU, const int* __restrict__ piv,
                                  const double* __restrict__ rhs, double* __restrict__ out, int k, int neg,
                                  int acc, const Control* ctl) {
  if (ctl->done) return;
  __shared__ float x[kMaxK];
  const int j = blockIdx.x, tid = threadIdx.x;
  for (int i = tid; i < k; i += blockDim.x) {
    const double v = rhs[i + (int64_t)j * k];
    x[i] = (float)(neg ? -v : v);
  }
  __syncthreads();
  if (TRANS == 0) {
    if (tid == 0)
      for (int p = 0; p < k; ++p) {
        const int q = piv[p];
        const float t = x[p]; x[p] = x[q]; x[q] = t;
      }
    __syncthreads();
    for (int p = 0; p < k - 1; ++p) {
      const float xp = x[p];
      for (int i = p + 1 + tid; i < k; i += blockDim.x) x[i] -= LU[i + (int64_t)p * k] * xp;
      __syncthreads();
    }
    for (int p = k - 1; p >= 0; --p) {
      if (tid == 0) x[p] /= LU[p + (int64_t)p * k];
      __syncthreads();
      const float xp = x[p];
      for (int i = tid; i < p; i += blockDim.x) x[i] -= LU[i + (int64_t)p * k] * xp;
      __syncthreads();
    }
  } else {
    for (int p = 0; p < k; ++p) {
      if (tid == 0) x[p] /= LU[p + (int64_t)p * k];
      __syncthreads();
      const float xp = x[p];
      for (int i = p + 1 + tid; i < k; i += blockDim.x) x[i] -= LU[p + (int64_t)i * k] * xp;
      __syncthreads();
    }
    for (int p = k - 1; p > 0; --p) {
      const float xp = x[p];
      for (int i = tid; i < p; i += blockDim.x) x[i] -= LU[p + (int64_t)i * k] * xp;
      __syncthreads();
    }
    if (tid == 0)
      for (int p = k - 1; p >= 0; --p) {
        const int q = piv[p];
        const float t = x[p]; x[p] = x[q]; x[q] = t;
      }
    __syncthreads();
  }
  for (int i = tid; i < k; i += blockDim.x) {
    const int64_t e = i + (int64_t)j * k;
    out[e] = acc ? out[e] + (double)x[i] : (double)x[i];
  }
}

// FP64 residual of the system being refined: res = -rhs - op(Y1) sol.
template <int TRANS>
__global__ void __launch_bounds__(256) kk_resid_kernel(const double* __restrict__ Y1, const double* __restrict__ rhs,
                                                       const double* __restrict__ sol, double* __restrict__ res,
                                                       int k, const Control* ctl) {
  if (ctl->done) return;
  __shared__ double As[16][17];
  __shared__ double Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i = blockIdx.x * 16 + tx, j = blockIdx.y * 16 + ty;
  double acc = 0.0;
  for (int l0 = 0; l0 < k; l0 += 16) {
    const int ai = blockIdx.x * 16 + ty, al = l0 + tx;
    As[ty][tx] = (ai < k && al < k) ? (TRANS ? Y1[al + (int64_t)ai * k] : Y1[ai + (int64_t)al * k]) : 0.0;
    const int bl = l0 + ty, bj = blockIdx.y * 16 + tx;
    Bs[ty][tx] = (bl < k && bj < k) ? sol[bl + (int64_t)bj * k] : 0.0;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 16; ++c) acc = fma(As[tx][c], Bs[c][ty], acc);
    __syncthreads();
  }
  if (i < k && j < k) {
    const int64_t e = i + (int64_t)j * k;
    res[e] = -rhs[e] - acc;
  }
}

// sol = op(Y1)^{-1} (-rhs), FP32 factors + two FP64 refinement steps.
template <int TRANS>
static void solve_refined(const SweepBufs& b, int k, const double* rhs, double* sol, int tpb, cudaStream_t s) {
  const float* lu32 = reinterpret_cast<const float*>(b.lu);
  dim3 g((k + 15) / 16, (k + 15) / 16);
  kk_solve32_kernel<TRANS><<<k, tpb, 0, s>>>(lu32, b.piv, rhs, sol, k, 1, 0, b.ctl);
  for (int it = 0; it < 2; ++it) {
    kk_resid_kernel<TRANS><<<g, 256, 0, s>>>(b.y1, rhs, sol, b.res, k, b.ctl);
    kk_solve32_kernel<TRANS><<<k, tpb, 0, s>>>(lu32, b.piv, b.res, sol, k, 0, 1, b.ctl);
  }
}

void launch_kxk_stage(const SweepBufs& b, int k, double delta, int beta_zero, cudaStream_t s) {
  const int tpb = k >= 128 ? 128 : ((k + 31) / 32) * 32;
  kk_prep_kernel<<<k, tpb, 0, s>>>(b, k);
  if (b.mixed) {
    kk_lu32_kernel<<<1, 512, sizeof(float) * (size_t)k * k, s>>>(b, k);
    solve_refined<0>(b, k, b.t1, b.m, tpb, s);          // M = -Y1^{-1} (Y^T R)
  } else {
    kk_lu_kernel<<<1, 512, sizeof(double) * (size_t)k * k, s>>>(b, k);
    kk_solve_kernel<0><<<k, tpb, 0, s>>>(b.lu, b.piv, b.t1, b.m, k, b.ctl);
  }
  dim3 g((k + 15) / 16, (k + 15) / 16);
  kk_gemm_kernel<KG_V1><<<g, 256, 0, s>>>(b, k);
  kk_gemm_kernel<KG_W2><<<g, 256, 0, s>>>(b, k);
  kk_e11_kernel<<<k, tpb, 0, s>>>(b, k, delta, beta_zero);
  kk_gemm_kernel<KG_YTE><<<g, 256, 0, s>>>(b, k);
  if (b.mixed)
    solve_refined<1>(b, k, b.yte, b.nmat, tpb, s);      // N = -Y1^{-T} (Y^T E)
  else
    kk_solve_kernel<1><<<k, tpb, 0, s>>>(b.lu, b.piv, b.yte, b.nmat, k, b.ctl);
  kk_gemm_kernel<KG_X1><<<g, 256, 0, s>>>(b, k);
}

// Signs of Algorithm 2 on the leading k x k block of the caller's X
// (column-major, ldx): sigma_j = -sign(q_jj), sign(0) = +1, unpivoted
// elimination of Q - Sigma.  The shifted pivot |q_jj| + 1 is never zero.
__global__ void __launch_bounds__(512) sign_fix_kernel(const double* __restrict__ X, int64_t ldx, int k,
                                                       double* __restrict__ sigma) {
  extern __shared__ double a[];
  const int tid = threadIdx.x;
  for (int64_t e = tid; e < (int64_t)k * k; e += blockDim.x) {
    int i = (int)(e % k), c = (int)(e / k);
    a[e] = X[i + (int64_t)c * ldx];
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
  e = cudaFuncSetAttribute(kk_lu32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(float) * kMaxK * kMaxK));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sign_fix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(double) * kMaxK * kMaxK));
}

void launch_sign_fix(const double* X, int64_t ldx, int k, double* sigma, int* /*singular*/, cudaStream_t s) {
  sign_fix_kernel<<<1, 512, sizeof(double) * (size_t)k * k, s>>>(X, ldx, k, sigma);
}

}  // namespace eigref

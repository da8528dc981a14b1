// Shared declarations of the eigref CUDA library (sm_103a).
//
// Internal layouts (all device memory owned by the handle):
//   X, P     : n x k FP64, row-major, leading dimension k (row i = the k
//              entries of row i of the approximate eigenvector block).
//   k x k    : FP64 column-major, leading dimension k.
// The caller's X (column-major, ldx) is converted at entry and exit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/eigref.h"

namespace eigref {

// max of two 64-bit unsigned integers as one compare and one select (PTX,
// so that it stays two integer instructions).  The bit patterns of
// non-negative doubles order like these integers; the column and row maxima
// of the split form are taken this way.
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("{\n .reg .pred p;\n setp.gt.u64 p, %1, %2;\n selp.b64 %0, %1, %2, p;\n}\n" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

constexpr double kUnitRoundoff = 1.1102230246251565e-16;  // 2^-53
constexpr int kMaxK = 128;                                 // k x k stage lives in shared memory

// Device-resident loop state.  Every sweep kernel returns at once when
// `done` is set, so a CUDA graph of several sweeps stops exactly at the
// sweep that met the criterion (or failed).
struct Control {
  int done;           // 1: remaining sweep kernels are no-ops
  int status;         // eigref_status of the loop
  int iterations;     // sweeps applied
  int pending_norm;   // 1: this sweep's update was applied; normalise it
  int max_iters;
  int stop;           // eigref_stop
  int nonfinite;
  int singular;       // set by the LU of Y_1
  int judge;          // columns 0..judge-1 decide the stop and divergence tests
  int ns_twice;       // split form: this sweep's first Newton-Schulz step left ||I - Y1 Z|| above the
                      // threshold, so a second one runs
  double tol;
  double norm_a;
  double div_factor, div_floor;
  double emin;        // smallest ||E_t||_F so far
  double last_res;    // ||R_t||_F / ||A||
  double last_corr;   // ||E_t||_F
};

// Pointers of one sweep (all device).
struct SweepBufs {
  const double* x;    // X_t   (n x k row-major)
  double* xn;         // X_{t+1}
  double* p;          // P = B X_t
  double* gpart;      // Gram partials: [2][nchunks][k*k]
  double* gtop;       // [2][k*k]: G1 = X1^T X1, S1 = X1^T P1
  double* g2;         // [2][k*k]: G2 = X2^T X2, S2 = X2^T P2 (rows >= k)
  double *r1, *t1, *z, *y1, *lu, *m, *v1, *w2, *e11, *yte, *nmat, *f, *res;  // k x k
  double *zinv, *zinv2;  // k x k: Y1^{-1} kept across sweeps (split form) and a scratch copy
  double* fm;         // split form, dense: k x kfm(k) column-major, F and M interleaved in blocks of 16
                      // columns (block q: F(:, 16q .. 16q+15), then M(:, 16q .. 16q+15)), or null
  unsigned long long* fm_cmax;   // or null: fm's column maxima of |.| (bit patterns), cleared by the prep
                                 // step and formed where fm is written
  int mixed;          // 1: Y1^{-1} by Newton-Schulz updates instead of an LU per sweep
  int* piv;           // [k]
  double *alpha, *d, *dinv, *nu, *r1sq, *e11sq, *x1sq;  // [k]
  double* upart;      // update partials [ugrid][3k]: column sums of x'^2, r^2, v2^2
  double *hist_res, *hist_corr;  // [max_iters]
  Control* ctl;
  int nchunks;
  int64_t chunk_rows;
  int ugrid;
};

// One problem of a batch run with grouped launches: every stage of a sweep is
// one launch over all problems, blockIdx.z (or a tile table) selecting the
// problem.  Lives in device memory; b[t & 1] holds the pointers of sweep t.
struct GroupItem {
  SweepBufs b[2];
  int64_t n;
  int k;
  int beta_zero;
  double delta;
  // split-form operands of this problem (see SlicedA)
  int n_pad, k_pad, kr, ksplit;
  void* x_planes;            // BF16 [S][k_pad][n_pad]
  void* p_planes;            // BF16 [S][k_pad][n_pad]
  void* xr_planes;           // BF16 [S][n_pad][kr]
  void* f_planes;            // BF16 [S][k_pad][kr]
  int *x_colexp, *p_colexp, *xr_rowexp, *f_colexp;
  unsigned long long *x_cmax, *p_cmax, *f_cmax;
  void* sgpart;              // tensor-core Gram partials: [2][ksplit][k k] exact (hi, lo) int64 pairs
};

// Columns of the interleaved [F | M] panel: 32 per 16 columns of k.
__host__ __device__ inline int kfm_cols(int k) { return 32 * ((k + 15) / 16); }
// Column of the panel that holds F(:, j) (M(:, j) is 16 further).
__host__ __device__ inline int kfm_col(int j) { return 32 * (j >> 4) + (j & 15); }

// Extent of a grouped launch: blockIdx.z = problem, x/y sized for the largest.
struct GroupDims {
  int count;
  int max_k;
  int64_t max_n;
};

// ---- kernels launched by the driver (definitions in the .cu files) ----
// fp64.cu
void launch_gemm_fp64(const double* A, int64_t lda, const double* X, double* P, int64_t n, int k,
                      double shift, const Control* ctl, cudaStream_t s, const double* Xs = nullptr);
void launch_gram(const double* X, const double* P, int k, int64_t r0, int64_t r1, int64_t chunk_rows,
                 int nchunks, double* part, double* out, const Control* ctl, cudaStream_t s);
void launch_gram_reduce(const double* part, int k, int nchunks, double* out, const Control* ctl, cudaStream_t s);
void launch_top_gram(const double* X, const double* P, int k, double* out, const Control* ctl, cudaStream_t s);
void launch_update_rows(const SweepBufs& b, int64_t n, int k, cudaStream_t s);
void launch_finalize(const SweepBufs& b, int k, double delta_unused, cudaStream_t s);
// cmax (optional): also the column maxima of the normalised |X| (ordered bits, atomicMax).
void launch_normalize(const SweepBufs& b, int64_t n, int k, cudaStream_t s, unsigned long long* cmax = nullptr);
void launch_copy_in(const double* Xu, int64_t ldx, double* X, int64_t n, int k, const double* sigma,
                    cudaStream_t s);
void launch_copy_out(const double* X, double* Xu, int64_t ldx, int64_t n, int k, const double* sigma,
                     cudaStream_t s);
void launch_rowmajor_to_colmajor(const double* X, double* Xu, int64_t ldx, int64_t n, int k, cudaStream_t s);
void launch_norm_inf_dense(const double* A, int64_t n, int64_t lda, double* out, cudaStream_t s);
void launch_norm_inf_csr(const int32_t* rp, const double* val, int64_t n, double* out, cudaStream_t s);
int update_rows_grid();
cudaError_t init_fp64_attributes();
cudaError_t init_kxk_attributes();
// spmm.cu
// cmax (optional, even k only): also the column maxima of |P| (ordered bits, atomicMax).
void launch_spmm_csr(const int32_t* rp, const int32_t* ci, const double* val, const double* X, double* P,
                     int64_t n, int k, double shift, const Control* ctl, cudaStream_t s, const double* Xs = nullptr,
                     unsigned long long* cmax = nullptr);
void launch_csr_fold_diag(const int32_t* rp, const int32_t* ci, const double* val, int64_t n, double shift,
                          double* val_out, int* missing, cudaStream_t s);
// kxk.cu
void launch_kxk_stage(const SweepBufs& b, int k, double delta, int beta_zero, cudaStream_t s);
void launch_sign_fix(const double* X, int64_t ldx, int k, double* sigma, int* singular, cudaStream_t s);
void launch_inverse_setup(const SweepBufs& b, int k, cudaStream_t s);
void launch_sign_fix_rowmajor(const double* X, int k, double* sigma, cudaStream_t s);
void launch_scale_cols(const double* In, double* Out, int64_t n, int k, const double* sg, cudaStream_t s);
// Rayleigh--Ritz (Section 3.3): G, S of Xbuf in b.gtop + b.g2; Xbuf <- its Ritz
// vectors (|Ritz value| descending, largest entry of each positive); Zbuf scratch.
void launch_rayleigh_ritz(const SweepBufs& b, int64_t n, int k, double* Xbuf, double* Zbuf, cudaStream_t s);
// Optional reorthogonalisation (Section 3.1.3): two first-order Loewdin steps
// Xbuf <- Xbuf (3 I - X^T X) / 2; Zbuf scratch.
void launch_reorthonormalise(const SweepBufs& b, int64_t n, int k, double* Xbuf, double* Zbuf, int64_t chunk_rows,
                             int nchunks, cudaStream_t s);

// grouped launches over a batch (parity = t & 1 of the sweep)
void launch_top_gram_grouped(const GroupItem* items, const GroupDims& gd, int parity, cudaStream_t s);
void launch_finalize_grouped(const GroupItem* items, const GroupDims& gd, int parity, cudaStream_t s);
void launch_normalize_grouped(const GroupItem* items, const GroupDims& gd, int parity, cudaStream_t s);
void launch_kxk_stage_grouped(const GroupItem* items, const GroupDims& gd, int parity, cudaStream_t s);

}  // namespace eigref

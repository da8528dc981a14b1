// Split-precision (error-free sliced) evaluation on the tensor cores of the
// dense products of a sweep: W = (A - shift I) X, the Gram products X^T X and
// X^T W, and the row update X - X F.  See sliced.cu.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace eigref {

namespace sl {
enum { MODE_PRODUCT = 0, MODE_GRAM = 1, MODE_UPDATE = 2 };

// Arguments of the tensor-core kernel (one problem, one mode).
struct MmaArgs {
  int a_plane_rows;      // rows between consecutive A-side planes in the A tensor map
  int b_plane_rows;      // rows between consecutive B-side planes in the B tensor maps
  int kb_total;          // K blocks of 64 in the contraction
  int ksplit;            // GRAM: number of K splits (blockIdx.z = job + 2 split)
  const int* rowexp;     // exponents of the output rows (A side)
  const int* colexp;     // exponents of the output columns (B side; GRAM job 0)
  const int* colexp2;    // GRAM job 1: exponents of W's columns
  int64_t m_valid;       // output rows that exist
  int k;                 // output columns that exist
  int row_begin;         // UPDATE: first row written (k)
  const double* X;       // PRODUCT / UPDATE: row-major n x k
  double* P;             // PRODUCT: row-major n x k
  double shift;          // PRODUCT
  const double* Xs;      // PRODUCT: operand of the shift term (row-major n x k)
  longlong2* ppart;      // PRODUCT with ksplit > 1: [ksplit][n x k] row-major exact (hi, lo) partials
  longlong2* gpart;      // GRAM: [2][ksplit][k * k] column-major exact (hi, lo) partials
  const double* W;       // UPDATE: row-major n x k
  const double* d;       // UPDATE: Rayleigh quotients [k]
  const double* dinv;    // UPDATE: 1 / d
  double* Xn;            // UPDATE: row-major n x k (overlaps none of X, W, d, dinv)
  double* upart;         // UPDATE: [m tiles][3k] column sums of X'^2, (W - X D)^2 and V2^2 (V2 = R2 - X2 M)
  const Control* ctl;
  int* err;              // set to 1 on a timed-out wait
  int sk_ranges;         // PRODUCT: > 0: equal-work ranges of (row tile, K block) units per column block
  long long sk_units;    // PRODUCT with sk_ranges: units per column block (row tiles x K blocks)
  unsigned long long wait_ns;   // limit of every bounded wait inside the kernel (0: the default, 2 s)
};
}  // namespace sl

// One launch's worth of tensor-core work for one problem: its tensor maps,
// arguments and tile grid (gx column blocks, gy row tiles, gz splits/jobs).
struct MmaTask {
  CUtensorMap a, b, b2;
  sl::MmaArgs g;
  int gx, gy, gz;
  int wide = 0;   // PRODUCT: 128 x 64 tiles (sliced_wide_kernel); grouped launches take 128 x 32 tasks only
};

// Grouped launches of the split form over a batch (all problems share S).
// Up to 40 tasks per launch, CTAs in task order.  side (optional): one stream
// per launch group, forked from s and joined back with ev[0..groups]
// (groups + 1 events), so the groups run side by side.
void launch_mma_tasks(int S, int mode, const MmaTask* tasks, int count, cudaStream_t s,
                      const cudaStream_t* side = nullptr, const cudaEvent_t* ev = nullptr);
enum { SLICE_X_COLS = 0, SLICE_P_COLS = 1, SLICE_F_COLS = 2, SLICE_X_ROWS = 3, SLICE_ZERO_MAX = 4 };
void launch_sgram_reduce_grouped(int S, const GroupItem* items, const GroupDims& gd, cudaStream_t s);
void launch_slice_grouped(int S, int op, const GroupItem* items, const GroupDims& gd, int max_n_pad, int parity,
                          cudaStream_t s);

cudaError_t init_sliced_attributes();

namespace sl {
// Column maxima of |Y| (row-major rows x k) as non-negative double bit patterns, atomicMax into cmax.
void launch_colmax_rowmajor(const double* Y, int64_t rows, int k, unsigned long long* cmax, const Control* ctl,
                            cudaStream_t s);
}  // namespace sl

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
  // P = A (A X) - alpha X (the shifted square of Section 5.2) through T; X's
  // planes stay in place for gram().
  int product_sq(const double* X, double* T, double* P, double alpha, const Control* ctl, cudaStream_t s,
                 cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, unsigned ev_flags = 0);
  // out[0] = X^T X, out[1] = X^T P (k x k column-major, all n rows), with X the
  // operand of the last product(); part = split-K scratch (null: internal).
  int gram(const double* P, double* part, double* out, const Control* ctl, cudaStream_t s);
  // Rows k..n-1 of X' = X + (W - X D) D^-1 - X F and per-row-tile column
  // sums of X'^2, (W - X D)^2 and V2^2 (V2 = R2 - X2 M, the rows of E21 D)
  // into upart[update_grid()][3k].  FM: the k x kfm_cols(k) panel of F and M
  // interleaved by 16 columns (SweepBufs::fm).
  int update(const double* X, const double* W, const double* FM, const double* d, const double* dinv, double* Xn,
             double* upart, const Control* ctl, cudaStream_t s);
  int update_grid() const;
  // The same three stages as launchable tasks (the batch groups them), and the
  // fields of this problem's GroupItem that describe its planes.
  // b_from_p: the B operand is the planes sliced into the W slot (the second
  // product of the shifted square); Xs: operand of the shift term (default X).
  MmaTask product_task(const double* X, double* P, double shift, const Control* ctl, const double* Xs = nullptr,
                       bool b_from_p = false) const;
  MmaTask gram_task(double* part, const Control* ctl) const;
  MmaTask update_task(const double* X, const double* W, const double* d, const double* dinv, double* Xn,
                      double* upart, const Control* ctl) const;
  void fill_group_item(GroupItem* it) const;
  // 1 if a bounded wait inside a tensor-core kernel gave up (synchronises s).
  int timed_out(cudaStream_t s) const;
  // Tensor-core flops one product executes (all digit pairs, padded sizes).
  double executed_flops() const;
  int slices() const { return slices_; }
  // K decomposition of the product (psplit) and split-K of the Gram products
  // (ksplit).  psplit 1..4: that many equal K splits a tile; kPsplitBalanced:
  // equal-work ranges over (row tile, K block) units, as many as make whole
  // rounds of one CTA per SM.  The partials are exact, so any choice gives
  // the same results bitwise; only the time differs (what the autotuner
  // measures).
  static constexpr int kPsplitBalanced = 8;
  std::vector<int> psplit_candidates() const;
  std::vector<int> ksplit_candidates() const;
  void set_splits(int psplit, int ksplit);
  int psplit() const { return psplit_; }
  int ksplit() const { return ksplit_; }
  // Columns of the product's output tile: 64 (the 128 x 64 kernel, k a
  // multiple of 64), 32, or 0 for the default (64 where it applies).  Single
  // problems only (grouped launches use 32).  Returns EIGREF_E_INVALID for a
  // width this k cannot take.  Either width gives the same results bitwise.
  int set_product_tile(int cols);
  int product_tile() const { return wide_ ? 64 : 32; }
  // Limit of every bounded wait inside the tensor-core kernels (0: 2 s).
  void set_wait_ns(unsigned long long ns) { wait_ns_ = ns; }
  // Fused column maxima (single-problem sweeps, after any autotuning): the
  // slicing of X, P and the [F | M] panel reads maxima that the kernels
  // writing them formed -- X's by the normalisation (launch_normalize with
  // x_cmax()), P's by the product's reduction, the panel's by the k x k stage
  // (SweepBufs::fm_cmax) -- in place of passes of their own.  X's maxima must
  // hold the starting X's when the first sweep begins; P's and the panel's
  // must be zero.  fused_maxima(): the product uses them (it needs the
  // reduction, i.e. a K decomposition other than one split).
  void set_fused_maxima(bool on) { fused_max_ = on; }
  bool fused_maxima() const;
  unsigned long long* x_cmax() const;
  unsigned long long* p_cmax() const;
  unsigned long long* fm_cmax() const;
  const char* error() const { return err_; }

 private:
  unsigned long long wait_ns_ = 0;
  bool fused_max_ = false;
  size_t layout_total() const;
  const double* A_ = nullptr;
  int64_t n_ = 0, lda_ = 0;
  int k_ = 0, precision_ = 0, slices_ = 0;
  int n_pad_ = 0, k_pad_ = 0, kr_ = 0, ksplit_ = 1, psplit_ = 1, ksplit_max_ = 1, psplit_max_ = 1;
  int pslots_ = 4;                      // product partial slots a tile in the workspace
  long long sk_ranges_ = 0, sk_units_ = 0;   // the equal-work plan (ranges and units a column block)
  long long sk_ranges_w_ = 0, sk_units_w_ = 0;   // the same for 64-column blocks
  bool wide_ = false;                   // product on 128 x 64 tiles
  char* ws_ = nullptr;
  alignas(64) unsigned char tmA_[128];
  alignas(64) unsigned char tmX_[128];
  alignas(64) unsigned char tmXA_[128];
  alignas(64) unsigned char tmP_[128];
  alignas(64) unsigned char tmXw_[128];   // X / P planes in 64-row boxes (the 128 x 64 product)
  alignas(64) unsigned char tmPw_[128];
  alignas(64) unsigned char tmXR_[128];
  alignas(64) unsigned char tmF_[128];
  char err_[256] = {0};
};

// The Gram products G = X^T X, S = X^T P (k <= 16, all n rows) as stacked
// F16 digit planes on the tensor cores, without A: the split form of the
// Gram products for CSR matrices (whose product stays an FP64 SpMM).
class SlicedGram {
 public:
  int configure(int64_t n, int k, int slices);
  size_t workspace_bytes() const;
  void bind_workspace(char* p);
  int prepare(cudaStream_t s);
  // out[0] = X^T X, out[1] = X^T P (k x k column-major); X, P row-major n x k
  int gram(const double* X, const double* P, double* out, const Control* ctl, cudaStream_t s);
  // The same with the column maxima of X and P already in x_cmax() / p_cmax()
  // (formed by the kernels that wrote X and P); clears them after use.
  int gram_ready(const double* X, const double* P, double* out, const Control* ctl, cudaStream_t s);
  void colmax_x(const double* X, cudaStream_t s);   // x_cmax() = column maxima of X
  int gram_fused(const double* X, const double* P, double* out, const Control* ctl, cudaStream_t s);
  // X' = X + (W - X D) D^-1 - X F for rows k .. n - 1 on the tensor cores
  // (even k); upart gets update_grid() x 3k column sums (x'^2, (w - x d)^2,
  // v^2 with V2 = R2 - X2 M).  Returns the launch count, or -1 when this k
  // has no such kernel.
  bool update_ready() const { return upd_ok_; }
  int update_grid() const { return upd_grid_; }
  int update(const double* X, const double* W, const double* F, const double* M, const double* d,
             const double* dinv, double* Xn, double* upart, const Control* ctl, cudaStream_t s);
  unsigned long long* x_cmax() const;
  unsigned long long* p_cmax() const;
  int timed_out(cudaStream_t s) const;
  int ksplit() const { return ksplit_; }
  int slices() const { return slices_; }
  void set_wait_ns(unsigned long long ns) { wait_ns_ = ns; }
  const char* error() const { return err_; }

 private:
  unsigned long long wait_ns_ = 0;
  int64_t n_ = 0, n_pad_ = 0;
  int k_ = 0, slices_ = 0, ksplit_ = 1;
  int upd_grid_ = 0;
  bool upd_ok_ = false;
  char* ws_ = nullptr;
  alignas(64) unsigned char tmX_[128];
  alignas(64) unsigned char tmP_[128];
  char err_[256] = {0};
};

}  // namespace eigref

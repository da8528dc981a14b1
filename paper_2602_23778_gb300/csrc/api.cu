// The C ABI of include/eigref.h: handle, workspace, argument checks, host
// buffer staging and the sweep driver (Algorithm 4 iterated with the
// stopping rules of Section 3.1.3).
//
// One sweep is a fixed sequence of kernel launches on the handle's stream;
// check_every sweeps are captured once into a CUDA graph and replayed.  The
// host reads the device Control block only between chunks; a sweep that
// finds the loop finished returns from every kernel at once, so the number of
// sweeps applied does not depend on the chunk length.
#include <cuda_runtime.h>
#include <float.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <map>
#include <memory>
#include <tuple>
#include <string>
#include <vector>

#include "common.cuh"
#include "sliced.cuh"

using namespace eigref;

struct eigref_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char err[512] = {0};
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  Control* host_ctl = nullptr;  // pinned
  // device copy of a host A (refine_dense with A in host memory): kept for the
  // next call, grown when a larger A comes, freed with the handle
  void* a_stage = nullptr;
  size_t a_stage_bytes = 0;
  // split-K choices the autotuner measured, by (n, k, slices, product tile)
  std::map<std::tuple<int64_t, int, int, int>, std::pair<int, int>> tuned;
};

namespace {

int set_err(eigref_ctx* h, int code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CUDA_TRY(h, expr)                                                                   \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return set_err(h, EIGREF_E_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                     __LINE__);                                                             \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Bump allocator over the handle's workspace; every block 256-byte aligned.
struct Carve {
  size_t off = 0;
  char* base = nullptr;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

int ensure_ws(eigref_ctx* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return EIGREF_OK;
  if (h->ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&h->ws, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(h, EIGREF_E_NOMEM, "workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  h->ws_bytes = bytes;
  return EIGREF_OK;
}

struct Params {
  int target, max_iters, stop, precision, slices, beta, check_every, sign_fix, use_graph, profile, rayleigh_ritz,
      judge_cols, reorth, resign, autotune;
  double shift, norm_a, tol, delta_c, div_factor, div_floor;
  unsigned long long wait_ns;  // bounded waits of the tensor-core kernels (0: their default)
};

int read_params(eigref_ctx* h, const eigref_params* p, Params* q) {
  eigref_params d;
  eigref_params_default(&d);
  if (!p) p = &d;
  q->target = p->target;
  q->shift = p->shift;
  q->norm_a = p->norm_a;
  q->max_iters = p->max_iters;
  q->tol = p->tol;
  q->stop = p->stop;
  q->precision = p->precision;
  q->slices = p->slices;
  q->beta = p->beta;
  q->delta_c = p->delta_c > 0 ? p->delta_c : 10.0;
  q->div_factor = p->div_factor > 0 ? p->div_factor : 10.0;
  q->div_floor = p->div_floor > 0 ? p->div_floor : 1e-4;
  q->check_every = p->check_every > 0 ? p->check_every : 32;
  q->check_every += q->check_every & 1;  // even: a chunk starts on the same X buffer
  q->sign_fix = p->sign_fix;
  q->use_graph = p->use_graph;
  q->profile = p->profile;
  q->rayleigh_ritz = p->rayleigh_ritz;
  q->judge_cols = p->judge_cols;
  q->reorth = p->reorth;
  q->resign = p->resign;
  q->autotune = p->autotune;
  q->wait_ns = p->wait_limit_s > 0.0 && isfinite(p->wait_limit_s)
                   ? (unsigned long long)std::max(1.0, std::min(p->wait_limit_s, 3600.0) * 1e9)
                   : 0ull;
  if (q->judge_cols < 0) return set_err(h, EIGREF_E_INVALID, "judge_cols < 0");
  if (q->target < EIGREF_LARGEST_MAG || q->target > EIGREF_SMALLEST_MAG)
    return set_err(h, EIGREF_E_INVALID, "target %d out of range", q->target);
  if (q->max_iters < 0) return set_err(h, EIGREF_E_INVALID, "max_iters < 0");
  if (!(q->tol >= 0.0) || !isfinite(q->tol)) return set_err(h, EIGREF_E_INVALID, "tol must be finite and >= 0");
  if (q->stop != EIGREF_STOP_CORRECTION && q->stop != EIGREF_STOP_RESIDUAL)
    return set_err(h, EIGREF_E_INVALID, "stop %d out of range", q->stop);
  if (q->beta != EIGREF_BETA_CLUSTER && q->beta != EIGREF_BETA_ZERO)
    return set_err(h, EIGREF_E_INVALID, "beta %d out of range", q->beta);
  if (q->precision < EIGREF_FP64 || q->precision > EIGREF_AUTO)
    return set_err(h, EIGREF_E_INVALID, "precision %d out of range", q->precision);
  if (!isfinite(q->shift) || !isfinite(q->norm_a)) return set_err(h, EIGREF_E_INVALID, "shift/norm_a not finite");
  return EIGREF_OK;
}

// Everything one refinement call needs besides the matrix.
struct Problem {
  bool csr = false;
  const double* A = nullptr;  // device
  int64_t lda = 0;
  const int32_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const double* val = nullptr;
  double* val_folded = nullptr;  // CSR values with the shift folded into the diagonal (workspace)
  bool folded = false;
  int64_t n = 0, nnz = 0;
  int k = 0;
  SlicedA* sliced = nullptr;  // split-precision dense product, or null
  SlicedGram* sgram = nullptr;  // CSR split form: tensor-core Gram products (k <= 16), or null
  // CSR split form with even k: the SpMM and the normalisation also form the
  // column maxima the slicing of P and X needs (no separate passes over them)
  unsigned long long* p_cmax = nullptr;
  bool fused_max = false;
  bool square = false;        // B = A^2 - alpha I (Section 5.2): W = A (A X) - alpha X
  double* tbuf = nullptr;     // A X of the shifted square (workspace)
};

// Returns the number of kernels launched.  ev0/ev1 (optional) bracket the
// product kernel; ev_flags is cudaEventRecordExternal inside a graph capture.
int launch_product(const Problem& pr, const double* X, double* P, double shift, const Control* ctl,
                   cudaStream_t s, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, unsigned ev_flags = 0) {
  if (pr.square) {
    // the shifted square of Section 5.2, A^2 never formed: T = A X, W = A T - alpha X
    if (pr.sliced) return pr.sliced->product_sq(X, pr.tbuf, P, shift, ctl, s, ev0, ev1, ev_flags);
    if (ev0) cudaEventRecordWithFlags(ev0, s, ev_flags);
    if (pr.csr) {
      launch_spmm_csr(pr.rp, pr.ci, pr.val, X, pr.tbuf, pr.n, pr.k, 0.0, ctl, s);
      launch_spmm_csr(pr.rp, pr.ci, pr.val, pr.tbuf, P, pr.n, pr.k, shift, ctl, s, X, pr.p_cmax);
    } else {
      launch_gemm_fp64(pr.A, pr.lda, X, pr.tbuf, pr.n, pr.k, 0.0, ctl, s);
      launch_gemm_fp64(pr.A, pr.lda, pr.tbuf, P, pr.n, pr.k, shift, ctl, s, X);
    }
    if (ev1) cudaEventRecordWithFlags(ev1, s, ev_flags);
    return 2;
  }
  if (pr.sliced) return pr.sliced->product(X, P, shift, ctl, s, ev0, ev1, ev_flags);
  if (ev0) cudaEventRecordWithFlags(ev0, s, ev_flags);
  if (pr.csr) {
    if (pr.folded)
      launch_spmm_csr(pr.rp, pr.ci, pr.val_folded, X, P, pr.n, pr.k, 0.0, ctl, s, nullptr, pr.p_cmax);
    else
      launch_spmm_csr(pr.rp, pr.ci, pr.val, X, P, pr.n, pr.k, shift, ctl, s, nullptr, pr.p_cmax);
  } else
    launch_gemm_fp64(pr.A, pr.lda, X, P, pr.n, pr.k, shift, ctl, s);
  if (ev1) cudaEventRecordWithFlags(ev1, s, ev_flags);
  return 1;
}

int launch_sweep(const Problem& pr, SweepBufs b, double shift, double delta, int beta_zero, cudaStream_t s,
                 cudaEvent_t ev0, cudaEvent_t ev1, unsigned ev_flags) {
  const int64_t n = pr.n;
  const int k = pr.k;
  int launches = launch_product(pr, b.x, b.p, shift, b.ctl, s, ev0, ev1, ev_flags);
  if (pr.sgram) {
    // CSR split form: Gram products over all rows on the tensor cores, the
    // leading block in FP64 (the k x k stage forms G2 = G - G1); FP64 update
    if (pr.fused_max)
      launches += pr.sgram->gram_ready(b.x, b.p, b.g2, b.ctl, s);
    else
      launches += pr.sgram->gram(b.x, b.p, b.g2, b.ctl, s);
    launch_top_gram(b.x, b.p, k, b.gtop, b.ctl, s);
    launch_kxk_stage(b, k, delta, beta_zero, s);
    // the row update on the tensor cores where this k has it, else in FP64
    if (pr.sgram->update(b.x, b.p, b.f, b.m, b.d, b.dinv, b.xn, b.upart, b.ctl, s) > 0) {
      b.ugrid = pr.sgram->update_grid();
    } else {
      launch_update_rows(b, n, k, s);
      b.ugrid = update_rows_grid();
    }
    launch_finalize(b, k, delta, s);
    launch_normalize(b, n, k, s, pr.fused_max ? pr.sgram->x_cmax() : nullptr);
    return launches + 1 + 9 + 1 + 2;
  }
  if (pr.sliced) {
    // split form: Gram products over all rows on the tensor cores, the
    // leading k x k block in FP64; the k x k stage forms G2 = G - G1
    pr.sliced->gram(b.p, nullptr, b.g2, b.ctl, s);
    launch_top_gram(b.x, b.p, k, b.gtop, b.ctl, s);
    launches += 5;
  } else {
    // Gram products of the rows below the leading block, then of the block
    launch_gram(b.x, b.p, k, k, n, b.chunk_rows, b.nchunks, b.gpart, b.g2, b.ctl, s);
    launch_gram(b.x, b.p, k, 0, k, k, 1, b.gpart, b.gtop, b.ctl, s);
    launches += 4;
  }
  launch_kxk_stage(b, k, delta, beta_zero, s);
  launches += b.mixed ? 9 : 7;
  if (pr.sliced) {
    pr.sliced->update(b.x, b.p, b.fm, b.d, b.dinv, b.xn, b.upart, b.ctl, s);
    launches += b.fm_cmax ? 3 : 4;
  } else {
    launch_update_rows(b, n, k, s);
    launches += 1;
  }
  launch_finalize(b, k, delta, s);
  // split form with fused maxima: the normalisation also forms X's column maxima
  launch_normalize(b, n, k, s, (pr.sliced && pr.sliced->fused_maxima()) ? pr.sliced->x_cmax() : nullptr);
  return launches + 2;
}

// One refinement in flight: the problem, its parameters and its workspace.
// refine_common drives one Run; eigref_refine_batched drives many at once.
struct Run {
  Problem pr;
  Params q;
  double* X = nullptr;  // caller's X
  int64_t ldx = 0;
  bool x_dev = true;
  SweepBufs b{};
  double* xbuf[2] = {nullptr, nullptr};
  double* xstage = nullptr;
  double* sigma = nullptr;
  double* scal = nullptr;
  const double* sg = nullptr;  // sign vector when the sign fix is on
  int64_t chunk_rows = 0;
  int nchunks = 0;
  int ugrid = 0;
  int hist_len = 0;
  double norm_a = 0.0, shift = 0.0, delta = 0.0;
  double norm_res = 0.0;  // scale of the residual test: ||B|| (||A|| unless B is the shifted square)
  int xoff = 0;           // X_t lives in xbuf[(t + xoff) & 1] (changes when the signs are retaken)
};

void run_plan(Run& r) {
  const int64_t n = r.pr.n;
  const int k = r.pr.k;
  r.chunk_rows = 256;
  while ((n - k + r.chunk_rows - 1) / r.chunk_rows > 1024) r.chunk_rows *= 2;
  r.nchunks = (int)std::max<int64_t>(1, (n - k + r.chunk_rows - 1) / r.chunk_rows);
  r.ugrid = r.pr.sliced ? r.pr.sliced->update_grid() : update_rows_grid();
  if (r.pr.sgram) r.ugrid = std::max(r.ugrid, r.pr.sgram->update_grid());   // either row update may run
  r.hist_len = std::max(1, r.q.max_iters);
}

// Carves the Run's buffers; with c.base == nullptr it only sizes them.  The
// Control block comes from `ctl` when given (one array for a whole batch).
void run_layout(Run& r, Carve& c, Control* ctl) {
  const int64_t n = r.pr.n;
  const int k = r.pr.k;
  const int64_t kk = (int64_t)k * k;
  SweepBufs& b = r.b;
  r.xbuf[0] = c.take<double>(n * k);
  r.xbuf[1] = c.take<double>(n * k);
  b.p = c.take<double>(n * k);
  r.xstage = r.x_dev ? nullptr : c.take<double>(n * k);
  b.gpart = c.take<double>(2 * (int64_t)r.nchunks * kk);
  b.gtop = c.take<double>(2 * kk);
  b.g2 = c.take<double>(2 * kk);
  double** mats[] = {&b.r1, &b.t1, &b.z, &b.y1, &b.lu, &b.m, &b.v1, &b.w2, &b.e11, &b.yte, &b.nmat, &b.f, &b.res,
                     &b.zinv, &b.zinv2};
  for (double** m : mats) *m = c.take<double>(kk);
  // the dense split form's row update reads F and M as one interleaved panel
  b.fm = (r.pr.sliced != nullptr) ? c.take<double>((int64_t)k * kfm_cols(k)) : nullptr;
  b.piv = c.take<int>(k);
  double** vecs[] = {&b.alpha, &b.d, &b.dinv, &b.nu, &b.r1sq, &b.e11sq, &b.x1sq};
  for (double** v : vecs) *v = c.take<double>(k);
  r.sigma = c.take<double>(k);
  b.upart = c.take<double>((int64_t)r.ugrid * 3 * k);
  b.hist_res = c.take<double>(r.hist_len);
  b.hist_corr = c.take<double>(r.hist_len);
  b.ctl = ctl ? ctl : c.take<Control>(1);
  r.scal = c.take<double>(4);
  if (r.pr.csr) r.pr.val_folded = c.take<double>(r.pr.nnz > 0 ? r.pr.nnz : 1);
  r.pr.tbuf = r.pr.square ? c.take<double>(n * k) : nullptr;
  b.nchunks = r.nchunks;
  b.chunk_rows = r.chunk_rows;
  b.ugrid = r.ugrid;
  b.mixed = r.pr.sliced != nullptr || r.pr.sgram != nullptr;  // the split form keeps Y1^{-1} by Newton-Schulz steps
}

// Bytes of workspace the Run needs (its buffers, then the sliced planes).
size_t run_bytes(Run& r, bool own_ctl) {
  Carve c;
  run_layout(r, c, own_ctl ? nullptr : reinterpret_cast<Control*>(16));
  const size_t extra = r.pr.sliced ? r.pr.sliced->workspace_bytes() : (r.pr.sgram ? r.pr.sgram->workspace_bytes() : 0);
  return ((c.off + 255) & ~size_t(255)) + 1024 + extra;
}

void run_bind(Run& r, char* base, Control* ctl) {
  Carve c;
  c.base = base;
  run_layout(r, c, ctl);
  if (r.pr.sliced) r.pr.sliced->bind_workspace(base + ((c.off + 255) & ~size_t(255)));
  if (r.pr.sgram) {
    r.pr.sgram->bind_workspace(base + ((c.off + 255) & ~size_t(255)));
    if (r.pr.fused_max) r.pr.p_cmax = r.pr.sgram->p_cmax();
  }
}

// Shift and delta from ||A|| and the target (Sections 3.1.3, 5.1 and 5.2).
void run_shift(Run& r) {
  r.shift = 0.0;
  if (r.q.target == EIGREF_SHIFT) r.shift = r.q.shift;
  else if (r.q.target == EIGREF_SMALLEST) r.shift = 0.5 * (r.norm_a + r.q.shift);   // Section 5.1
  else if (r.q.target == EIGREF_LARGEST) r.shift = 0.5 * (r.q.shift - r.norm_a);    // its mirror
  else if (r.q.target == EIGREF_SMALLEST_MAG)                                       // Section 5.2, on A^2
    r.shift = 0.5 * (r.norm_a * r.norm_a + r.q.shift * r.q.shift);
  const double norm_b = r.pr.square ? r.norm_a * r.norm_a + fabs(r.shift) : r.norm_a + fabs(r.shift);
  r.norm_res = r.pr.square ? norm_b : r.norm_a;
  r.delta = r.q.delta_c * norm_b * kUnitRoundoff;                                   // Section 3.1.3
}

Control run_control(const Run& r) {
  Control c{};
  c.max_iters = r.q.max_iters;
  c.stop = r.q.stop;
  c.tol = r.q.tol;
  c.norm_a = r.norm_res;
  c.judge = (r.q.judge_cols > 0 && r.q.judge_cols < r.pr.k) ? r.q.judge_cols : r.pr.k;
  c.div_factor = r.q.div_factor;
  c.div_floor = r.q.div_floor;
  c.emin = DBL_MAX;
  c.status = EIGREF_OK;
  c.done = r.q.max_iters == 0;
  return c;
}

// Column maxima the first sweep's slicing reads when the producers form them:
// those of the starting X, and none yet for P (or the [F | M] panel).
void run_setup_maxima(const Run& r, cudaStream_t s) {
  if (r.pr.sliced && r.pr.sliced->fused_maxima()) {
    SlicedA* sl = r.pr.sliced;
    cudaMemsetAsync(sl->p_cmax(), 0, (size_t)r.pr.k * 8, s);
    cudaMemsetAsync(sl->fm_cmax(), 0, (size_t)kfm_cols(r.pr.k) * 8, s);
    cudaMemsetAsync(sl->x_cmax(), 0, (size_t)r.pr.k * 8, s);
    sl::launch_colmax_rowmajor(r.xbuf[0], r.pr.n, r.pr.k, sl->x_cmax(), nullptr, s);
  }
  if (!r.pr.fused_max) return;
  cudaMemsetAsync(r.pr.p_cmax, 0, (size_t)r.pr.k * 8, s);
  r.pr.sgram->colmax_x(r.xbuf[0], s);
}

// Device half of the set-up after ||A|| and the shift are known: the internal
// X (staged, sign-fixed) and the slices of A.
int run_setup_device(eigref_ctx* h, Run& r, cudaStream_t s) {
  const int64_t n = r.pr.n;
  const int k = r.pr.k;
  const double* xu = r.X;
  if (!r.x_dev) {
    CUDA_TRY(h, cudaMemcpy2DAsync(r.xstage, n * sizeof(double), r.X, r.ldx * sizeof(double), n * sizeof(double), k,
                                  cudaMemcpyHostToDevice, s));
    xu = r.xstage;
  }
  const int64_t ldu = r.x_dev ? r.ldx : n;
  r.sg = nullptr;
  // the [F | M] panel's padding columns (past k in its last block) stay zero
  if (r.b.fm) CUDA_TRY(h, cudaMemsetAsync(r.b.fm, 0, sizeof(double) * (size_t)k * kfm_cols(k), s));
  if (!r.q.rayleigh_ritz) {
    if (r.q.sign_fix) {
      launch_sign_fix(xu, ldu, k, r.sigma, nullptr, s);
      r.sg = r.sigma;
    }
    launch_copy_in(xu, ldu, r.xbuf[0], n, k, r.sg, s);
  } else {
    launch_copy_in(xu, ldu, r.xbuf[0], n, k, nullptr, s);
  }
  if (r.pr.sliced) {
    const int st = r.pr.sliced->prepare(s);
    if (st) return set_err(h, st, "%s", r.pr.sliced->error());
  }
  if (r.pr.sgram) {
    const int st = r.pr.sgram->prepare(s);
    if (st) return set_err(h, st, "%s", r.pr.sgram->error());
  }
  if (r.q.rayleigh_ritz) {
    // Section 3.3: X <- its Ritz vectors for B, then the signs of Algorithm 2
    // on that X.  The Ritz vectors are what the call refines and returns.
    SweepBufs& b = r.b;
    // (no Control on these launches: they run even when max_iters = 0)
    launch_product(r.pr, r.xbuf[0], b.p, r.shift, nullptr, s);
    launch_gram(r.xbuf[0], b.p, k, k, n, r.chunk_rows, r.nchunks, b.gpart, b.g2, nullptr, s);
    launch_gram(r.xbuf[0], b.p, k, 0, k, k, 1, b.gpart, b.gtop, nullptr, s);
    launch_rayleigh_ritz(b, n, k, r.xbuf[0], r.xbuf[1], s);
    if (r.q.sign_fix) {
      launch_sign_fix_rowmajor(r.xbuf[0], k, r.sigma, s);
      launch_scale_cols(r.xbuf[0], r.xbuf[0], n, k, r.sigma, s);
      r.sg = r.sigma;
    }
  }
  run_setup_maxima(r, s);
  return EIGREF_OK;
}

// Split form: Y1^{-1} of the starting X, refined every sweep after.  Runs
// after the Control block holds run_control(r).
void run_setup_inverse(const Run& r, cudaStream_t s) {
  if (r.b.mixed && r.q.max_iters > 0) {
    SweepBufs b0 = r.b;
    b0.x = r.xbuf[0];
    launch_inverse_setup(b0, r.pr.k, s);
  }
}

// Issues sweeps t0 .. t0 + count - 1 (X_t lives in xbuf[t % 2]); returns the
// number of kernels launched.
int run_issue(const Run& r, int count, cudaStream_t s, cudaEvent_t* pev, unsigned ev_flags) {
  int launches = 0;
  for (int t = 0; t < count; ++t) {
    SweepBufs bt = r.b;
    bt.x = r.xbuf[t & 1];
    bt.xn = r.xbuf[(t + 1) & 1];
    launches += launch_sweep(r.pr, bt, r.shift, r.delta, r.q.beta == EIGREF_BETA_ZERO, s,
                             pev ? pev[2 * t] : nullptr, pev ? pev[2 * t + 1] : nullptr, ev_flags);
  }
  return launches;
}

// Copies the final iterate back into the caller's X (signs restored), after
// the optional reorthogonalisation.
int run_copy_out(eigref_ctx* h, const Run& r, int iterations, cudaStream_t s) {
  const int64_t n = r.pr.n;
  const int k = r.pr.k;
  const int cur = (iterations + r.xoff) & 1;
  const double* xr = r.xbuf[cur];
  if (r.q.reorth)
    launch_reorthonormalise(r.b, n, k, r.xbuf[cur], r.xbuf[cur ^ 1], r.chunk_rows, r.nchunks, s);
  if (r.x_dev) {
    launch_copy_out(xr, r.X, r.ldx, n, k, r.sg, s);
  } else {
    launch_copy_out(xr, r.xstage, n, n, k, r.sg, s);
    CUDA_TRY(h, cudaMemcpy2DAsync(r.X, r.ldx * sizeof(double), r.xstage, n * sizeof(double), n * sizeof(double), k,
                                  cudaMemcpyDeviceToHost, s));
  }
  return EIGREF_OK;
}

void fill_report(const Run& r, const Control& fin, const double* dvec, eigref_report* rep) {
  int status = fin.status;
  if (r.q.max_iters == 0) status = EIGREF_OK;
  rep->status = status;
  rep->iterations = fin.iterations;
  rep->final_rel_residual = fin.iterations ? fin.last_res : NAN;
  rep->final_corr_norm = fin.iterations ? fin.last_corr : NAN;
  rep->shift = r.shift;
  rep->norm_a = r.norm_a;
  rep->delta = r.delta;
  if (rep->eigenvalues)
    for (int j = 0; j < r.pr.k; ++j) rep->eigenvalues[j] = fin.iterations ? dvec[j] + r.shift : NAN;
}

// A CUDA graph of one chunk of sweeps, destroyed with the guard.
struct GraphGuard {
  cudaGraphExec_t g = nullptr;
  ~GraphGuard() {
    if (g) cudaGraphExecDestroy(g);
  }
};

// The autotuner: times each split-K candidate of the tensor-core product and
// of the Gram products on this problem (3 runs after a warm-up, CUDA events)
// and keeps the fastest for the handle.  The split partials are exact, so the
// choice changes the time only, never the results.
int tune_splits(eigref_ctx* h, Run& r, cudaStream_t s) {
  SlicedA* sl = r.pr.sliced;
  cudaEvent_t e0, e1;
  CUDA_TRY(h, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_err(h, EIGREF_E_CUDA, "autotune events");
  }
  auto time_it = [&](const std::function<void()>& f) {
    f();
    cudaEventRecord(e0, s);
    for (int i = 0; i < 3; ++i) f();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  int best_p = sl->psplit(), best_k = sl->ksplit();
  float best = 1e30f;
  for (int p : sl->psplit_candidates()) {
    sl->set_splits(p, best_k);
    const float ms = time_it([&] { launch_product(r.pr, r.xbuf[0], r.b.p, r.shift, nullptr, s); });
    if (ms < best) {
      best = ms;
      best_p = p;
    }
  }
  best = 1e30f;
  for (int kq : sl->ksplit_candidates()) {
    sl->set_splits(best_p, kq);
    const float ms = time_it([&] { sl->gram(r.b.p, nullptr, r.b.g2, nullptr, s); });
    if (ms < best) {
      best = ms;
      best_k = kq;
    }
  }
  sl->set_splits(best_p, best_k);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CUDA_TRY(h, cudaGetLastError());
  h->tuned[std::make_tuple(r.pr.n, r.pr.k, sl->slices(), sl->product_tile())] = std::make_pair(best_p, best_k);
  return EIGREF_OK;
}

int refine_common(eigref_ctx* h, Problem& pr, double* X, int64_t ldx, const eigref_params* pin,
                  eigref_report* rep) {
  Run r;
  r.pr = pr;
  int st = read_params(h, pin, &r.q);
  if (st) return st;
  const Params& q = r.q;
  const int64_t n = pr.n;
  const int k = pr.k;
  cudaStream_t s = h->stream;
  if (r.pr.sliced) r.pr.sliced->set_wait_ns(q.wait_ns);
  if (r.pr.sgram) r.pr.sgram->set_wait_ns(q.wait_ns);
  r.X = X;
  r.ldx = ldx;
  r.x_dev = is_device_ptr(X);

  // ---- workspace ----
  run_plan(r);
  st = ensure_ws(h, run_bytes(r, true));
  if (st) return st;
  run_bind(r, static_cast<char*>(h->ws), nullptr);
  SweepBufs& b = r.b;

  CUDA_TRY(h, cudaEventRecord(h->ev[0], s));
  // ---- set-up: ||A||, shift, delta, signs, internal X ----
  r.norm_a = q.norm_a;
  if (!(r.norm_a > 0.0)) {
    if (r.pr.csr)
      launch_norm_inf_csr(r.pr.rp, r.pr.val, n, r.scal, s);
    else
      launch_norm_inf_dense(r.pr.A, n, r.pr.lda, r.scal, s);
    CUDA_TRY(h, cudaMemcpyAsync(&h->host_ctl->tol, r.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    r.norm_a = h->host_ctl->tol;
    if (!(r.norm_a > 0.0) || !isfinite(r.norm_a))
      return set_err(h, isfinite(r.norm_a) ? EIGREF_E_INVALID : EIGREF_E_NONFINITE, "||A||_inf = %g", r.norm_a);
  }
  run_shift(r);
  *h->host_ctl = run_control(r);
  CUDA_TRY(h, cudaMemcpyAsync(b.ctl, h->host_ctl, sizeof(Control), cudaMemcpyHostToDevice, s));
  if (r.pr.csr && r.shift != 0.0 && r.pr.nnz > 0 && !r.pr.square) {
    // fold -shift into the stored diagonal once, so the SpMM has no shift term
    int* missing = reinterpret_cast<int*>(r.scal + 2);
    launch_csr_fold_diag(r.pr.rp, r.pr.ci, r.pr.val, n, r.shift, r.pr.val_folded, missing, s);
    int* hmiss = &h->host_ctl->singular;   // the host copy of the Control block is spare here
    CUDA_TRY(h, cudaMemcpyAsync(hmiss, missing, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    r.pr.folded = *hmiss == 0;
  }
  st = run_setup_device(h, r, s);
  if (st) return st;
  if (r.pr.sliced && q.autotune && q.max_iters > 0 &&
      !h->tuned.count(std::make_tuple(r.pr.n, r.pr.k, r.pr.sliced->slices(), r.pr.sliced->product_tile()))) {
    st = tune_splits(h, r, s);
    if (st) return st;
  }
  if (r.pr.sliced && !r.pr.square) {
    // from here on the kernels that write X, P and the [F | M] panel form the
    // column maxima the slicing needs (the autotuner's runs above did not)
    r.pr.sliced->set_fused_maxima(true);
    r.b.fm_cmax = r.pr.sliced->fm_cmax();
    run_setup_maxima(r, s);
  }
  run_setup_inverse(r, s);

  // ---- sweeps: chunks of check_every (no longer than the run), even ----
  const int m = std::min(q.check_every, std::max(2, q.max_iters + (q.max_iters & 1)));
  std::vector<cudaEvent_t> pev;
  if (q.profile) {
    pev.resize(2 * m);
    for (auto& e : pev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        for (auto& f : pev)
          if (f) cudaEventDestroy(f);
        return set_err(h, EIGREF_E_CUDA, "profiling events");
      }
  }
  struct EvGuard {
    std::vector<cudaEvent_t>& v;
    ~EvGuard() {
      for (auto& e : v)
        if (e) cudaEventDestroy(e);
    }
  } ev_guard{pev};
  cudaEvent_t* pe = q.profile ? pev.data() : nullptr;
  GraphGuard graph;
  int chunk_launches = 0;
  if (q.use_graph && q.max_iters > 0) {
    // capture before the sweep timer starts: instantiation is host work
    cudaGraph_t g;
    CUDA_TRY(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    chunk_launches = run_issue(r, m, s, pe, cudaEventRecordExternal);
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (ce != cudaSuccess) return set_err(h, EIGREF_E_CUDA, "graph capture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&graph.g, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return set_err(h, EIGREF_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    CUDA_TRY(h, cudaGraphUpload(graph.g, s));
  }
  CUDA_TRY(h, cudaEventRecord(h->ev[1], s));
  CUDA_TRY(h, cudaGetLastError());
  int launched = 0;
  int64_t kernel_launches = 0;
  double product_ms = 0.0;
  int product_launches = 0;
  int it_before = 0;
  int resigned = 0;
  while (launched < q.max_iters) {
    if (graph.g) {
      CUDA_TRY(h, cudaGraphLaunch(graph.g, s));
      kernel_launches += chunk_launches;
    } else {
      kernel_launches += run_issue(r, m, s, pe, cudaEventRecordDefault);
    }
    launched += m;
    CUDA_TRY(h, cudaMemcpyAsync(h->host_ctl, b.ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    if (q.resign && h->host_ctl->status == EIGREF_E_SINGULAR_WY && resigned < 4) {
      // Y1 lost its conditioning: take the signs of Algorithm 2 for the current
      // X (the choice Algorithm 3 builds into its WY factors), X <- X Sigma, and
      // resume from the same iterate.  The next chunk starts on xbuf[0].
      const int it = h->host_ctl->iterations;
      double* xc = r.xbuf[(it + r.xoff) & 1];
      double* s2 = b.nu;   // scratch: recomputed by every sweep
      launch_sign_fix_rowmajor(xc, k, s2, s);
      launch_scale_cols(xc, r.xbuf[0], n, k, s2, s);
      if (r.sg) {
        launch_scale_cols(r.sigma, r.sigma, 1, k, s2, s);
      } else {
        CUDA_TRY(h, cudaMemcpyAsync(r.sigma, s2, k * sizeof(double), cudaMemcpyDeviceToDevice, s));
        r.sg = r.sigma;
      }
      r.xoff = it & 1;
      Control c = *h->host_ctl;
      c.status = EIGREF_OK;
      c.done = 0;
      c.singular = 0;
      *h->host_ctl = c;
      CUDA_TRY(h, cudaMemcpyAsync(b.ctl, h->host_ctl, sizeof(Control), cudaMemcpyHostToDevice, s));
      run_setup_inverse(r, s);
      run_setup_maxima(r, s);
      ++resigned;
      launched = it;
      it_before = it;
      continue;
    }
    const int ran = h->host_ctl->iterations - it_before;
    it_before = h->host_ctl->iterations;
    for (int t = 0; q.profile && t < ran && t < m; ++t) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pev[2 * t], pev[2 * t + 1]) == cudaSuccess) {
        product_ms += ms;
        ++product_launches;
      }
    }
    if (h->host_ctl->done) break;
  }
  CUDA_TRY(h, cudaEventRecord(h->ev[2], s));
  CUDA_TRY(h, cudaMemcpyAsync(h->host_ctl, b.ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaStreamSynchronize(s));
  const Control fin = *h->host_ctl;

  // ---- result: X_{iterations} lives in xbuf[(iterations + xoff) % 2] ----
  st = run_copy_out(h, r, fin.iterations, s);
  if (st) return st;
  std::vector<double> dvec(k);
  CUDA_TRY(h, cudaMemcpyAsync(dvec.data(), b.d, k * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (rep && rep->hist_residual && fin.iterations > 0)
    CUDA_TRY(h, cudaMemcpyAsync(rep->hist_residual, b.hist_res, fin.iterations * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
  if (rep && rep->hist_corr && fin.iterations > 0)
    CUDA_TRY(h, cudaMemcpyAsync(rep->hist_corr, b.hist_corr, fin.iterations * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaEventRecord(h->ev[3], s));
  CUDA_TRY(h, cudaStreamSynchronize(s));
  CUDA_TRY(h, cudaGetLastError());
  const int status = q.max_iters == 0 ? EIGREF_OK : fin.status;
  if (rep) {
    fill_report(r, fin, dvec.data(), rep);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
    rep->setup_ms = ms;
    cudaEventElapsedTime(&ms, h->ev[1], h->ev[2]);
    rep->sweeps_ms = ms;
    rep->product_ms = product_ms;
    rep->product_launches = product_launches;
    rep->kernel_launches = kernel_launches;
    rep->psplit = r.pr.sliced ? r.pr.sliced->psplit() : 0;
    rep->ksplit = r.pr.sliced ? r.pr.sliced->ksplit() : (r.pr.sgram ? r.pr.sgram->ksplit() : 0);
  }
  if (status != EIGREF_OK)
    set_err(h, status, "%s after %d sweeps", eigref_status_string(status), fin.iterations);
  return status;
}

// EIGREF_AUTO: the split form where the library has one that pays off.
int resolve_precision(int precision, bool csr, int64_t n, int k) {
  if (precision != EIGREF_AUTO) return precision;
  if (csr) return k <= 16 ? EIGREF_BF16_SLICES : EIGREF_FP64;
  return (n >= 1024 && n <= ((int64_t)1 << 18)) ? EIGREF_BF16_SLICES : EIGREF_FP64;
}

int check_dims(eigref_ctx* h, int64_t n, int k, int64_t ldx, const double* X) {
  if (!X) return set_err(h, EIGREF_E_INVALID, "X is NULL");
  if (n < 2 || n > (int64_t)INT32_MAX) return set_err(h, EIGREF_E_INVALID, "n = %lld out of range", (long long)n);
  if (k < 1 || k > kMaxK || k >= n)
    return set_err(h, EIGREF_E_INVALID, "need 1 <= k <= %d and k < n (k = %d, n = %lld)", kMaxK, k, (long long)n);
  if (ldx < n) return set_err(h, EIGREF_E_INVALID, "ldx < n");
  return EIGREF_OK;
}

}  // namespace

extern "C" {

void eigref_params_default(eigref_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->target = EIGREF_LARGEST_MAG;
  p->shift = 0.0;
  p->norm_a = 0.0;
  p->max_iters = 100;
  p->tol = 0.0;
  p->stop = EIGREF_STOP_CORRECTION;
  p->precision = EIGREF_FP64;
  p->slices = 0;
  p->beta = EIGREF_BETA_CLUSTER;
  p->delta_c = 10.0;
  p->div_factor = 10.0;
  p->div_floor = 1e-4;
  p->check_every = 32;
  p->sign_fix = 1;
  p->use_graph = 1;
  p->profile = 0;
  p->rayleigh_ritz = 0;
  p->judge_cols = 0;
  p->reorth = 0;
  p->resign = 0;
  p->autotune = 1;
  p->product_tile = 0;
}

const char* eigref_status_string(int s) {
  switch (s) {
    case EIGREF_OK: return "ok";
    case EIGREF_E_INVALID: return "invalid argument";
    case EIGREF_E_CUDA: return "CUDA error";
    case EIGREF_E_NOMEM: return "out of device memory";
    case EIGREF_E_SINGULAR_WY: return "leading block Y1 singular (Algorithm 1 not applicable)";
    case EIGREF_E_DIVERGED: return "diverged";
    case EIGREF_E_NOT_CONVERGED: return "not converged";
    case EIGREF_E_NONFINITE: return "non-finite values";
    case EIGREF_E_TIMEOUT: return "device wait timed out";
    case EIGREF_E_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

int eigref_create(eigref_handle* out, int device, void* stream) {
  if (!out) return EIGREF_E_INVALID;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return EIGREF_E_INVALID;
  }
  eigref_ctx* h = new eigref_ctx();
  h->device = device;
  if (cudaSetDevice(device) != cudaSuccess) { delete h; return EIGREF_E_CUDA; }
  if (stream) {
    h->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) { delete h; return EIGREF_E_CUDA; }
    h->own_stream = true;
  }
  for (auto& e : h->ev)
    if (cudaEventCreate(&e) != cudaSuccess) { eigref_destroy(h); return EIGREF_E_CUDA; }
  if (cudaMallocHost(reinterpret_cast<void**>(&h->host_ctl), sizeof(Control)) != cudaSuccess ||
      init_fp64_attributes() != cudaSuccess || init_kxk_attributes() != cudaSuccess ||
      init_sliced_attributes() != cudaSuccess) {
    cudaGetLastError();
    eigref_destroy(h);
    return EIGREF_E_CUDA;
  }
  *out = h;
  return EIGREF_OK;
}

int eigref_destroy(eigref_handle h) {
  if (!h) return EIGREF_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->ws) cudaFree(h->ws);
  if (h->a_stage) cudaFree(h->a_stage);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  if (h->host_ctl) cudaFreeHost(h->host_ctl);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return EIGREF_OK;
}

const char* eigref_last_error(eigref_handle h) { return h ? h->err : ""; }

int eigref_refine_dense(eigref_handle h, const double* A, int64_t n, int64_t lda, double* X, int64_t ldx, int k,
                        const eigref_params* p, eigref_report* rep) {
  if (!h) return EIGREF_E_INVALID;
  h->err[0] = 0;
  if (!A) return set_err(h, EIGREF_E_INVALID, "A is NULL");
  int st = check_dims(h, n, k, ldx, X);
  if (st) return st;
  if (lda < n) return set_err(h, EIGREF_E_INVALID, "lda < n");
  if (cudaSetDevice(h->device) != cudaSuccess) return set_err(h, EIGREF_E_CUDA, "cudaSetDevice");
  eigref_params dp;
  eigref_params_default(&dp);
  if (p) dp = *p;
  dp.precision = resolve_precision(dp.precision, false, n, k);
  const eigref_params* pp = &dp;
  Problem pr;
  pr.n = n;
  pr.k = k;
  pr.lda = lda;
  pr.square = pp->target == EIGREF_SMALLEST_MAG;
  if (is_device_ptr(A)) {
    pr.A = A;
  } else {
    // host A: one pitched copy into the handle's staging buffer (kept between
    // calls: a serving host that refines against matrices of one size pays
    // the allocation once)
    const size_t bytes = (size_t)n * n * sizeof(double);
    if (bytes > h->a_stage_bytes) {
      if (h->a_stage) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->a_stage);
        h->a_stage = nullptr;
        h->a_stage_bytes = 0;
      }
      if (cudaMalloc(&h->a_stage, bytes) != cudaSuccess) {
        cudaGetLastError();
        h->a_stage = nullptr;
        return set_err(h, EIGREF_E_NOMEM, "device copy of A");
      }
      h->a_stage_bytes = bytes;
    }
    double* a_dev = static_cast<double*>(h->a_stage);
    cudaError_t e = cudaMemcpy2DAsync(a_dev, n * sizeof(double), A, lda * sizeof(double), n * sizeof(double), n,
                                      cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return set_err(h, EIGREF_E_CUDA, "copy of A: %s", cudaGetErrorString(e));
    pr.A = a_dev;
    pr.lda = n;
  }
  SlicedA sl;
  if (pp->precision != EIGREF_FP64) {
    st = sl.configure(pr.A, n, pr.lda, k, pp->precision, pp->slices);
    if (!st) st = sl.set_product_tile(pp->product_tile);
    if (st) return set_err(h, st, "%s", sl.error());
    auto tk = h->tuned.find(std::make_tuple(n, k, sl.slices(), sl.product_tile()));
    if (tk != h->tuned.end()) sl.set_splits(tk->second.first, tk->second.second);
    pr.sliced = &sl;
  }
  return refine_common(h, pr, X, ldx, pp, rep);
}

int eigref_refine_csr(eigref_handle h, const int32_t* row_ptr, const int32_t* col_idx, const double* val, int64_t n,
                      int64_t nnz, double* X, int64_t ldx, int k, const eigref_params* p, eigref_report* rep) {
  if (!h) return EIGREF_E_INVALID;
  h->err[0] = 0;
  if (!row_ptr || !col_idx || !val) return set_err(h, EIGREF_E_INVALID, "CSR array is NULL");
  int st = check_dims(h, n, k, ldx, X);
  if (st) return st;
  if (nnz < 0) return set_err(h, EIGREF_E_INVALID, "nnz < 0");
  if (cudaSetDevice(h->device) != cudaSuccess) return set_err(h, EIGREF_E_CUDA, "cudaSetDevice");
  Problem pr;
  pr.csr = true;
  pr.n = n;
  pr.k = k;
  pr.nnz = nnz;
  pr.square = p && p->target == EIGREF_SMALLEST_MAG;
  void* bufs[3] = {nullptr, nullptr, nullptr};
  const void* src[3] = {row_ptr, col_idx, val};
  size_t sz[3] = {(size_t)(n + 1) * 4, (size_t)nnz * 4, (size_t)nnz * 8};
  for (int i = 0; i < 3; ++i) {
    if (is_device_ptr(src[i]) || sz[i] == 0) continue;
    if (cudaMalloc(&bufs[i], sz[i]) != cudaSuccess ||
        cudaMemcpyAsync(bufs[i], src[i], sz[i], cudaMemcpyHostToDevice, h->stream) != cudaSuccess) {
      cudaGetLastError();
      for (void* q : bufs)
        if (q) cudaFree(q);
      return set_err(h, EIGREF_E_NOMEM, "device copy of CSR arrays");
    }
  }
  pr.rp = static_cast<const int32_t*>(bufs[0] ? bufs[0] : row_ptr);
  pr.ci = static_cast<const int32_t*>(bufs[1] ? bufs[1] : col_idx);
  pr.val = static_cast<const double*>(bufs[2] ? bufs[2] : val);
  SlicedGram sg;
  eigref_params cp;
  eigref_params_default(&cp);
  if (p) cp = *p;
  cp.precision = resolve_precision(cp.precision, true, n, k);
  if (cp.precision == EIGREF_BF16_SLICES) {
    st = sg.configure(n, k, cp.slices);
    if (st) {
      set_err(h, st, "%s", sg.error());
    } else {
      pr.sgram = &sg;
      pr.fused_max = (k % 2) == 0;
    }
  } else if (cp.precision != EIGREF_FP64) {
    st = set_err(h, EIGREF_E_UNSUPPORTED, "CSR: precision %d not built (FP64 or BF16 slices)", cp.precision);
  }
  if (st == EIGREF_OK) st = refine_common(h, pr, X, ldx, &cp, rep);
  cudaStreamSynchronize(h->stream);
  for (void* q : bufs)
    if (q) cudaFree(q);
  return st;
}

// Many independent problems in one CUDA graph: every problem's sweep chain is
// captured on a stream of its own, forked from and joined back into the
// handle's stream, so one graph launch advances every problem by a chunk of
// sweeps and the GPU runs the chains side by side.  A finished problem's
// kernels return at once (its Control block is done), so problems of uneven
// difficulty share the launches without changing each other's results.
int eigref_refine_batched(eigref_handle h, int count, const eigref_problem* probs, const eigref_params* p,
                          eigref_report* reps) {
  if (!h) return EIGREF_E_INVALID;
  h->err[0] = 0;
  if (count < 1 || !probs) return set_err(h, EIGREF_E_INVALID, "need count >= 1 and a problem array");
  if (cudaSetDevice(h->device) != cudaSuccess) return set_err(h, EIGREF_E_CUDA, "cudaSetDevice");
  Params q;
  int st = read_params(h, p, &q);
  if (st) return st;
  if (q.precision == EIGREF_AUTO) {
    int64_t nmax = 0;
    for (int i = 0; i < count; ++i) nmax = std::max(nmax, probs[i].n);
    q.precision = nmax <= ((int64_t)1 << 18) ? EIGREF_BF16_SLICES : EIGREF_FP64;
  }
  std::vector<Run> runs(count);
  std::unique_ptr<SlicedA[]> sls(new SlicedA[count]);
  for (int i = 0; i < count; ++i) {
    const eigref_problem& pb = probs[i];
    if (!pb.A || !is_device_ptr(pb.A)) return set_err(h, EIGREF_E_INVALID, "problem %d: A must be device memory", i);
    st = check_dims(h, pb.n, pb.k, pb.ldx, pb.X);
    if (st) {
      char why[sizeof(h->err)];
      memcpy(why, h->err, sizeof(why));
      return set_err(h, st, "problem %d: %s", i, why);
    }
    if (!is_device_ptr(pb.X)) return set_err(h, EIGREF_E_INVALID, "problem %d: X must be device memory", i);
    if (pb.lda < pb.n) return set_err(h, EIGREF_E_INVALID, "problem %d: lda < n", i);
    if (pb.target < EIGREF_LARGEST_MAG || pb.target > EIGREF_SHIFT)
      return set_err(h, EIGREF_E_INVALID, "problem %d: target %d out of range", i, pb.target);
    if (!isfinite(pb.shift) || !isfinite(pb.norm_a))
      return set_err(h, EIGREF_E_INVALID, "problem %d: shift/norm_a not finite", i);
    Run& r = runs[i];
    r.q = q;
    r.q.target = pb.target;
    r.q.shift = pb.shift;
    r.q.norm_a = pb.norm_a;
    r.pr.n = pb.n;
    r.pr.k = pb.k;
    r.pr.A = pb.A;
    r.pr.lda = pb.lda;
    r.X = pb.X;
    r.ldx = pb.ldx;
    r.x_dev = true;
    r.pr.square = pb.target == EIGREF_SMALLEST_MAG;
    if (q.precision != EIGREF_FP64) {
      st = sls[i].configure(pb.A, pb.n, pb.lda, pb.k, q.precision, q.slices);
      if (st) return set_err(h, st, "problem %d: %s", i, sls[i].error());
      sls[i].share_gpu(count);
      sls[i].set_wait_ns(q.wait_ns);
      r.pr.sliced = &sls[i];
    }
    run_plan(r);
  }
  // split form: every stage is one grouped launch over all problems
  const bool grouped = q.precision != EIGREF_FP64;
  if (grouped)
    for (int i = 0; i < count; ++i)
      if (runs[i].pr.square)
        return set_err(h, EIGREF_E_UNSUPPORTED, "problem %d: the shifted square is not batched in the split form", i);
  // ---- workspace: the Control array, the GroupItem array, one region per problem ----
  const size_t ctl_bytes = ((size_t)count * sizeof(Control) + 1023) & ~size_t(1023);
  const size_t item_bytes = grouped ? (((size_t)count * sizeof(GroupItem) + 1023) & ~size_t(1023)) : 0;
  std::vector<size_t> off(count);
  size_t total = ctl_bytes + item_bytes;
  for (int i = 0; i < count; ++i) {
    off[i] = total;
    total += (run_bytes(runs[i], false) + 1023) & ~size_t(1023);
  }
  st = ensure_ws(h, total);
  if (st) return st;
  char* base = static_cast<char*>(h->ws);
  Control* ctls = reinterpret_cast<Control*>(base);
  GroupItem* items_dev = reinterpret_cast<GroupItem*>(base + ctl_bytes);
  for (int i = 0; i < count; ++i) run_bind(runs[i], base + off[i], ctls + i);

  // host-side resources of the call, released by the guard
  struct Res {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    Control* hc = nullptr;
    ~Res() {
      for (auto e : events)
        if (e) cudaEventDestroy(e);
      for (auto s : streams)
        if (s) cudaStreamDestroy(s);
      if (hc) cudaFreeHost(hc);
    }
  } res;
  CUDA_TRY(h, cudaMallocHost(reinterpret_cast<void**>(&res.hc), (size_t)count * sizeof(Control)));
  cudaStream_t s = h->stream;
  CUDA_TRY(h, cudaEventRecord(h->ev[0], s));

  // ---- set-up ----
  bool need_norm = false;
  for (int i = 0; i < count; ++i) {
    Run& r = runs[i];
    r.norm_a = r.q.norm_a;
    if (!(r.norm_a > 0.0)) {
      launch_norm_inf_dense(r.pr.A, r.pr.n, r.pr.lda, r.scal, s);
      CUDA_TRY(h, cudaMemcpyAsync(&res.hc[i].tol, r.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
      need_norm = true;
    }
  }
  if (need_norm) CUDA_TRY(h, cudaStreamSynchronize(s));
  for (int i = 0; i < count; ++i) {
    Run& r = runs[i];
    if (!(r.norm_a > 0.0)) {
      r.norm_a = res.hc[i].tol;
      if (!(r.norm_a > 0.0) || !isfinite(r.norm_a))
        return set_err(h, isfinite(r.norm_a) ? EIGREF_E_INVALID : EIGREF_E_NONFINITE, "problem %d: ||A||_inf = %g", i,
                       r.norm_a);
    }
    run_shift(r);
    res.hc[i] = run_control(r);
  }
  CUDA_TRY(h, cudaMemcpyAsync(ctls, res.hc, (size_t)count * sizeof(Control), cudaMemcpyHostToDevice, s));
  for (int i = 0; i < count; ++i) {
    st = run_setup_device(h, runs[i], s);
    if (st) return st;
  }
  for (int i = 0; i < count; ++i) run_setup_inverse(runs[i], s);

  int m = std::min(q.check_every, std::max(2, q.max_iters));
  std::function<int(int)> issue_all;
  // grouped form: per-problem items and tensor-core tasks for both sweep parities
  std::vector<GroupItem> items;
  std::vector<MmaTask> prod[2], gram, upd[2];
  GroupDims gd{count, 0, 0};
  int max_n_pad = 0;
  if (grouped) {
    items.resize(count);
    gram.resize(count);
    for (int par = 0; par < 2; ++par) {
      prod[par].resize(count);
      upd[par].resize(count);
    }
    // tensor-core tasks heaviest first (longest CTAs start first; launch groups
    // hold problems of like size, so a group's CTAs end together)
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return (int64_t)runs[a].pr.n * runs[a].pr.k > (int64_t)runs[b].pr.n * runs[b].pr.k;
    });
    for (int slot = 0; slot < count; ++slot) {
      const int i = order[slot];
      const Run& r = runs[i];
      for (int par = 0; par < 2; ++par) {
        prod[par][slot] = sls[i].product_task(r.xbuf[par], r.b.p, r.shift, r.b.ctl);
        upd[par][slot] = sls[i].update_task(r.xbuf[par], r.b.p, r.b.d, r.b.dinv, r.xbuf[par ^ 1], r.b.upart, r.b.ctl);
      }
      gram[slot] = sls[i].gram_task(nullptr, r.b.ctl);
    }
    for (int i = 0; i < count; ++i) {
      const Run& r = runs[i];
      GroupItem& it = items[i];
      memset(&it, 0, sizeof(it));
      for (int par = 0; par < 2; ++par) {
        it.b[par] = r.b;
        it.b[par].x = r.xbuf[par];
        it.b[par].xn = r.xbuf[par ^ 1];
      }
      it.n = r.pr.n;
      it.k = r.pr.k;
      it.beta_zero = q.beta == EIGREF_BETA_ZERO;
      it.delta = r.delta;
      sls[i].fill_group_item(&it);
      gd.max_k = std::max(gd.max_k, r.pr.k);
      gd.max_n = std::max(gd.max_n, r.pr.n);
      max_n_pad = std::max(max_n_pad, it.n_pad);
    }
    CUDA_TRY(h, cudaMemcpyAsync(items_dev, items.data(), (size_t)count * sizeof(GroupItem), cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    const int S = sls[0].slices();
    m += m & 1;
    const int groups = (count + 39) / 40;
    res.streams.assign(groups, nullptr);
    res.events.assign(groups + 1, nullptr);
    for (auto& x : res.streams) CUDA_TRY(h, cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    for (auto& e : res.events) CUDA_TRY(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    const cudaStream_t* side = groups > 1 ? res.streams.data() : nullptr;
    const cudaEvent_t* evs = res.events.data();
    issue_all = [&, S, groups, side, evs](int count_sweeps) {
      int launches = 0;
      for (int t = 0; t < count_sweeps; ++t) {
        const int par = t & 1;
        launch_slice_grouped(S, SLICE_ZERO_MAX, items_dev, gd, max_n_pad, par, s);
        launch_slice_grouped(S, SLICE_X_COLS, items_dev, gd, max_n_pad, par, s);
        launch_mma_tasks(S, sl::MODE_PRODUCT, prod[par].data(), count, s, side, evs);
        launch_slice_grouped(S, SLICE_P_COLS, items_dev, gd, max_n_pad, par, s);
        launch_mma_tasks(S, sl::MODE_GRAM, gram.data(), count, s, side, evs);
        launch_sgram_reduce_grouped(S, items_dev, gd, s);
        launch_top_gram_grouped(items_dev, gd, par, s);
        launch_kxk_stage_grouped(items_dev, gd, par, s);
        launch_slice_grouped(S, SLICE_X_ROWS, items_dev, gd, max_n_pad, par, s);
        launch_slice_grouped(S, SLICE_F_COLS, items_dev, gd, max_n_pad, par, s);
        launch_mma_tasks(S, sl::MODE_UPDATE, upd[par].data(), count, s, side, evs);
        launch_finalize_grouped(items_dev, gd, par, s);
        launch_normalize_grouped(items_dev, gd, par, s);
        launches += 21 + 3 * groups;
      }
      return launches;
    };
  } else {
    // ---- one stream per problem, forked from and joined into the handle's stream ----
    res.streams.assign(count, nullptr);
    res.events.assign(count + 1, nullptr);
    for (auto& x : res.streams) CUDA_TRY(h, cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
    for (auto& e : res.events) CUDA_TRY(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    // chunk length: about 32k graph nodes per replay, even, at least 2
    m = std::min(m, std::max(2, 32768 / (25 * count)));
    m += m & 1;
    issue_all = [&](int count_sweeps) {
      int launches = 0;
      cudaEventRecord(res.events[count], s);
      for (int i = 0; i < count; ++i) {
        cudaStreamWaitEvent(res.streams[i], res.events[count], 0);
        launches += run_issue(runs[i], count_sweeps, res.streams[i], nullptr, 0);
        cudaEventRecord(res.events[i], res.streams[i]);
        cudaStreamWaitEvent(s, res.events[i], 0);
      }
      return launches;
    };
  }
  GraphGuard graph;
  int chunk_launches = 0;
  if (q.use_graph && q.max_iters > 0) {
    cudaGraph_t g;
    CUDA_TRY(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    chunk_launches = issue_all(m);
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (ce != cudaSuccess) return set_err(h, EIGREF_E_CUDA, "graph capture: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&graph.g, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return set_err(h, EIGREF_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    CUDA_TRY(h, cudaGraphUpload(graph.g, s));
  }
  CUDA_TRY(h, cudaEventRecord(h->ev[1], s));
  CUDA_TRY(h, cudaGetLastError());

  // ---- sweeps ----
  int launched = 0;
  int64_t kernel_launches = 0;
  while (launched < q.max_iters) {
    if (graph.g) {
      CUDA_TRY(h, cudaGraphLaunch(graph.g, s));
      kernel_launches += chunk_launches;
    } else {
      kernel_launches += issue_all(m);
    }
    launched += m;
    CUDA_TRY(h, cudaMemcpyAsync(res.hc, ctls, (size_t)count * sizeof(Control), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    bool all_done = true;
    for (int i = 0; i < count; ++i) all_done = all_done && res.hc[i].done;
    if (all_done) break;
  }
  CUDA_TRY(h, cudaEventRecord(h->ev[2], s));
  CUDA_TRY(h, cudaMemcpyAsync(res.hc, ctls, (size_t)count * sizeof(Control), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(h, cudaStreamSynchronize(s));

  // ---- results ----
  int kmax = 0;
  for (const Run& r : runs) kmax = std::max(kmax, r.pr.k);
  std::vector<double> dvec((size_t)count * kmax);
  for (int i = 0; i < count; ++i) {
    const Run& r = runs[i];
    const Control& fin = res.hc[i];
    st = run_copy_out(h, r, fin.iterations, s);
    if (st) return st;
    CUDA_TRY(h, cudaMemcpyAsync(dvec.data() + (size_t)i * kmax, r.b.d, r.pr.k * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
    eigref_report* rep = reps ? reps + i : nullptr;
    if (rep && rep->hist_residual && fin.iterations > 0)
      CUDA_TRY(h, cudaMemcpyAsync(rep->hist_residual, r.b.hist_res, fin.iterations * sizeof(double),
                                  cudaMemcpyDeviceToHost, s));
    if (rep && rep->hist_corr && fin.iterations > 0)
      CUDA_TRY(h, cudaMemcpyAsync(rep->hist_corr, r.b.hist_corr, fin.iterations * sizeof(double),
                                  cudaMemcpyDeviceToHost, s));
  }
  CUDA_TRY(h, cudaEventRecord(h->ev[3], s));
  CUDA_TRY(h, cudaStreamSynchronize(s));
  CUDA_TRY(h, cudaGetLastError());
  float setup_ms = 0.f, sweeps_ms = 0.f;
  cudaEventElapsedTime(&setup_ms, h->ev[0], h->ev[1]);
  cudaEventElapsedTime(&sweeps_ms, h->ev[1], h->ev[2]);
  int status = EIGREF_OK, first_bad = -1;
  for (int i = 0; i < count; ++i) {
    const int si = q.max_iters == 0 ? EIGREF_OK : res.hc[i].status;
    if (si != EIGREF_OK && first_bad < 0) {
      first_bad = i;
      status = si;
    }
    if (reps) {
      fill_report(runs[i], res.hc[i], dvec.data() + (size_t)i * kmax, reps + i);
      reps[i].setup_ms = setup_ms;
      reps[i].sweeps_ms = sweeps_ms;
      reps[i].product_ms = 0.0;
      reps[i].product_launches = 0;
      reps[i].kernel_launches = kernel_launches;
      reps[i].psplit = runs[i].pr.sliced ? runs[i].pr.sliced->psplit() : 0;
      reps[i].ksplit = runs[i].pr.sliced ? runs[i].pr.sliced->ksplit() : 0;
    }
  }
  if (status != EIGREF_OK)
    set_err(h, status, "problem %d: %s after %d sweeps", first_bad, eigref_status_string(status),
            res.hc[first_bad].iterations);
  return status;
}

// G = X^T X, S = X^T P over all n rows (the Gram sums behind the Rayleigh
// quotients of Algorithm 4, Eq. Rayleigh, on their own) through the kernels
// the sweeps use.
int eigref_gram(eigref_handle h, const double* X, int64_t ldx, const double* P, int64_t ldp, int64_t n, int k,
                int precision, int slices, double* G, double* S) {
  if (!h) return EIGREF_E_INVALID;
  h->err[0] = 0;
  if (!X || !P || !G || !S) return set_err(h, EIGREF_E_INVALID, "NULL argument");
  if (n < 1 || k < 1 || k > kMaxK || ldx < n || ldp < n) return set_err(h, EIGREF_E_INVALID, "bad sizes");
  if (!is_device_ptr(X) || !is_device_ptr(P)) return set_err(h, EIGREF_E_INVALID, "gram needs X and P in device memory");
  if (precision == EIGREF_AUTO) precision = k <= 16 ? EIGREF_BF16_SLICES : EIGREF_FP64;
  if (precision != EIGREF_FP64 && precision != EIGREF_BF16_SLICES)
    return set_err(h, EIGREF_E_UNSUPPORTED, "precision %d not built for the Gram products", precision);
  if (cudaSetDevice(h->device) != cudaSuccess) return set_err(h, EIGREF_E_CUDA, "cudaSetDevice");
  cudaStream_t s = h->stream;
  SlicedGram sg;
  if (precision == EIGREF_BF16_SLICES) {
    const int st = sg.configure(n, k, slices);
    if (st) return set_err(h, st, "%s", sg.error());
  }
  int64_t chunk_rows = 256;
  while ((n + chunk_rows - 1) / chunk_rows > 1024) chunk_rows *= 2;
  const int nchunks = (int)std::max<int64_t>(1, (n + chunk_rows - 1) / chunk_rows);
  const int64_t kk = (int64_t)k * k;
  auto lay = [&](Carve& c, double** xi, double** pi, double** gpart, double** out) {
    *xi = c.take<double>(n * k);
    *pi = c.take<double>(n * k);
    *gpart = c.take<double>(2 * (int64_t)nchunks * kk);
    *out = c.take<double>(2 * kk);
  };
  double *xi, *pi, *gpart, *out;
  Carve c0;
  lay(c0, &xi, &pi, &gpart, &out);
  const size_t extra = precision == EIGREF_BF16_SLICES ? sg.workspace_bytes() : 0;
  int st = ensure_ws(h, c0.off + 1024 + extra);
  if (st) return st;
  Carve c;
  c.base = static_cast<char*>(h->ws);
  lay(c, &xi, &pi, &gpart, &out);
  launch_copy_in(X, ldx, xi, n, k, nullptr, s);
  launch_copy_in(P, ldp, pi, n, k, nullptr, s);
  if (precision == EIGREF_BF16_SLICES) {
    sg.bind_workspace(static_cast<char*>(h->ws) + ((c.off + 255) & ~size_t(255)));
    st = sg.prepare(s);
    if (st) return set_err(h, st, "%s", sg.error());
    sg.gram(xi, pi, out, nullptr, s);
    if (sg.timed_out(s)) return set_err(h, EIGREF_E_TIMEOUT, "tensor-core Gram wait timed out");
  } else {
    launch_gram(xi, pi, k, 0, n, chunk_rows, nchunks, gpart, out, nullptr, s);
  }
  const cudaMemcpyKind kg = is_device_ptr(G) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const cudaMemcpyKind ks = is_device_ptr(S) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(h, cudaMemcpyAsync(G, out, kk * sizeof(double), kg, s));
  CUDA_TRY(h, cudaMemcpyAsync(S, out + kk, kk * sizeof(double), ks, s));
  CUDA_TRY(h, cudaStreamSynchronize(s));
  CUDA_TRY(h, cudaGetLastError());
  return EIGREF_OK;
}

// P = (A - shift I) X through the same product kernels the sweeps use.
static int product_common(eigref_ctx* h, Problem& pr, const double* X, int64_t ldx, double shift, double* P,
                          int64_t ldp) {
  const int64_t n = pr.n;
  const int k = pr.k;
  cudaStream_t s = h->stream;
  Carve c0;
  c0.take<double>(n * k);
  c0.take<double>(n * k);
  c0.take<double>(n * k);
  size_t extra = pr.sliced ? pr.sliced->workspace_bytes() : 0;
  int st = ensure_ws(h, c0.off + 256 + extra);
  if (st) return st;
  Carve c;
  c.base = static_cast<char*>(h->ws);
  double* xs = c.take<double>(n * k);
  double* xi = c.take<double>(n * k);
  double* pi = c.take<double>(n * k);
  if (pr.sliced) pr.sliced->bind_workspace(static_cast<char*>(h->ws) + ((c.off + 255) & ~size_t(255)));
  const double* xu = X;
  int64_t ldu = ldx;
  if (!is_device_ptr(X)) {
    CUDA_TRY(h, cudaMemcpy2DAsync(xs, n * sizeof(double), X, ldx * sizeof(double), n * sizeof(double), k,
                                  cudaMemcpyHostToDevice, s));
    xu = xs;
    ldu = n;
  }
  launch_copy_in(xu, ldu, xi, n, k, nullptr, s);
  if (pr.sliced) {
    st = pr.sliced->prepare(s);
    if (st) return set_err(h, st, "%s", pr.sliced->error());
  }
  launch_product(pr, xi, pi, shift, nullptr, s);
  if (pr.sliced && pr.sliced->timed_out(s)) return set_err(h, EIGREF_E_TIMEOUT, "tensor-core product wait timed out");
  if (is_device_ptr(P)) {
    launch_copy_out(pi, P, ldp, n, k, nullptr, s);
  } else {
    launch_copy_out(pi, xs, n, n, k, nullptr, s);
    CUDA_TRY(h, cudaMemcpy2DAsync(P, ldp * sizeof(double), xs, n * sizeof(double), n * sizeof(double), k,
                                  cudaMemcpyDeviceToHost, s));
  }
  CUDA_TRY(h, cudaStreamSynchronize(s));
  CUDA_TRY(h, cudaGetLastError());
  return EIGREF_OK;
}

int eigref_product_dense(eigref_handle h, const double* A, int64_t n, int64_t lda, const double* X, int64_t ldx,
                         int k, double shift, int precision, int slices, double* P, int64_t ldp) {
  if (!h) return EIGREF_E_INVALID;
  h->err[0] = 0;
  if (!A || !X || !P) return set_err(h, EIGREF_E_INVALID, "NULL argument");
  if (n < 1 || k < 1 || lda < n || ldx < n || ldp < n) return set_err(h, EIGREF_E_INVALID, "bad sizes");
  if (!is_device_ptr(A)) return set_err(h, EIGREF_E_INVALID, "product_dense needs A in device memory");
  if (cudaSetDevice(h->device) != cudaSuccess) return set_err(h, EIGREF_E_CUDA, "cudaSetDevice");
  Problem pr;
  pr.n = n;
  pr.k = k;
  pr.A = A;
  pr.lda = lda;
  SlicedA sl;
  precision = resolve_precision(precision, false, n, k);
  if (precision != EIGREF_FP64) {
    int st = sl.configure(A, n, lda, k, precision, slices);
    if (!st) st = sl.set_product_tile(0);
    if (st) return set_err(h, st, "%s", sl.error());
    auto tk = h->tuned.find(std::make_tuple(n, k, sl.slices(), sl.product_tile()));
    if (tk != h->tuned.end()) sl.set_splits(tk->second.first, tk->second.second);
    pr.sliced = &sl;
  }
  return product_common(h, pr, X, ldx, shift, P, ldp);
}

int eigref_product_csr(eigref_handle h, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                       int64_t n, int64_t nnz, const double* X, int64_t ldx, int k, double shift, double* P,
                       int64_t ldp) {
  if (!h) return EIGREF_E_INVALID;
  h->err[0] = 0;
  if (!row_ptr || !col_idx || !val || !X || !P) return set_err(h, EIGREF_E_INVALID, "NULL argument");
  if (n < 1 || k < 1 || nnz < 0 || ldx < n || ldp < n) return set_err(h, EIGREF_E_INVALID, "bad sizes");
  if (!is_device_ptr(row_ptr) || !is_device_ptr(col_idx) || !is_device_ptr(val))
    return set_err(h, EIGREF_E_INVALID, "product_csr needs the CSR arrays in device memory");
  if (cudaSetDevice(h->device) != cudaSuccess) return set_err(h, EIGREF_E_CUDA, "cudaSetDevice");
  Problem pr;
  pr.csr = true;
  pr.n = n;
  pr.k = k;
  pr.nnz = nnz;
  pr.rp = row_ptr;
  pr.ci = col_idx;
  pr.val = val;
  return product_common(h, pr, X, ldx, shift, P, ldp);
}

}  // extern "C"

/*
 * eigref -- GB300 (sm_103a) refinement of a subset of eigenvectors of a real
 * symmetric matrix.
 *
 * Method: Terao, Ozaki, Imamura and Ogita, "Iterative Refinement for a Subset
 * of Eigenvectors of Symmetric Matrices via Matrix Multiplications".  Given
 * approximate eigenvectors X-hat (n x k, k << n) of a symmetric A, each sweep
 * applies Algorithm 4 (Section 3.1.2): W = A X-hat, the compact-WY matrix
 * H-hat of Algorithm 1, Rayleigh quotients (Eq. Rayleigh), the correction
 * E-tilde_L (Eqs. Ediag, V-def, Eoffdiag), the update X-hat + H-hat E-tilde_L
 * (Eq. update-X), then column normalisation (Section 3.1.3).
 *
 * C ABI.  Plain pointers and sizes, no C++ or framework types.  Every entry
 * point returns an eigref_status; no exception crosses the boundary.
 *
 * Memory: matrix arguments may be device pointers (cudaMalloc, or a framework
 * tensor's storage on the handle's device) or host pointers (pageable or
 * pinned); the library detects which with cudaPointerGetAttributes and copies
 * host data through its own device workspace, inside the call.  The caller
 * owns every argument buffer; the handle owns its workspace.
 *
 * Layouts: A dense is n x n with leading dimension lda >= n (row i starts at
 * A + i*lda; A is symmetric, so row- and column-major agree).  CSR A is
 * row_ptr[n+1], col_idx[nnz] (0-based, int32), val[nnz] (FP64), and must be
 * symmetric; column order within a row is free.  X is n x k column-major with
 * ldx >= n: column j (an approximate eigenvector) starts at X + j*ldx.
 *
 * Threading: a handle is not thread-safe; all its work is issued on its
 * stream and every entry point returns after that work has finished.
 */
#ifndef EIGREF_H
#define EIGREF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct eigref_ctx* eigref_handle;

enum eigref_status {
  EIGREF_OK = 0,
  EIGREF_E_INVALID = 1,        /* bad argument; nothing was written */
  EIGREF_E_CUDA = 2,           /* a CUDA call failed (eigref_last_error has it) */
  EIGREF_E_NOMEM = 3,          /* workspace allocation failed */
  EIGREF_E_SINGULAR_WY = 4,    /* Algorithm 1's Y_1 singular to working precision */
  EIGREF_E_DIVERGED = 5,       /* correction norm grew (advice closing Section 4.3.1) */
  EIGREF_E_NOT_CONVERGED = 6,  /* max_iters sweeps without meeting tol (tol > 0) */
  EIGREF_E_NONFINITE = 7,      /* a sweep produced Inf/NaN; X keeps the last finite iterate */
  EIGREF_E_TIMEOUT = 8,        /* a bounded device wait gave up */
  EIGREF_E_UNSUPPORTED = 9     /* valid request the library does not implement */
};

/* Which eigenvectors the refinement converges to (Section 3.1 and Section 5.1).
 * The operator refined is B = A - alpha I. */
enum eigref_target {
  EIGREF_LARGEST_MAG = 0,  /* k largest |lambda|, alpha = 0 (the paper's default ordering) */
  EIGREF_LARGEST = 1,      /* k algebraically largest, alpha = (lambda_{k+1} - ||A||) / 2 */
  EIGREF_SMALLEST = 2,     /* k algebraically smallest, alpha = (||A|| + lambda_{k+1}) / 2 (Section 5.1) */
  EIGREF_SHIFT = 3,        /* explicit alpha */
  EIGREF_SMALLEST_MAG = 4  /* k smallest |lambda| through B = A^2 - alpha I, alpha = (||A||^2 +
                              lambda_{k+1}^2) / 2 (Section 5.2); W = A (A X) - alpha X, A^2 never
                              formed; eigenvalues reports lambda^2 */
};

/* How W = B X and the Gram products are evaluated. */
enum eigref_precision {
  EIGREF_FP64 = 0,         /* plain FP64 on the CUDA cores */
  EIGREF_BF16_SLICES = 1,  /* error-free digit slices on the tensor cores, FP32 accumulation (8-bit
                              digits, exact in BF16 and F16; the planes are stored as F16) */
  EIGREF_INT8_SLICES = 2,  /* error-free INT8 slices on the tensor cores, INT32 accumulation (not
                              built: GB300's INT8 tensor rate is far below its BF16 rate) */
  EIGREF_AUTO = 3          /* the faster form the build offers for the call: BF16 slices for dense
                              1024 <= n <= 2^18 and for CSR k <= 16, FP64 otherwise */
};

enum eigref_stop {
  EIGREF_STOP_CORRECTION = 0,  /* ||E-tilde_L||_F <= tol (Section 3.1.3) */
  EIGREF_STOP_RESIDUAL = 1     /* ||A X - X D||_F / ||A|| <= tol (Section 3.1.3) */
};

enum eigref_beta {
  EIGREF_BETA_CLUSTER = 0,  /* beta_ij = -x_i^T x_j / 2 for |d_j - d_i| <= delta */
  EIGREF_BETA_ZERO = 1      /* beta_ij = 0 (after Rayleigh--Ritz preprocessing) */
};

typedef struct eigref_params {
  int target;          /* enum eigref_target */
  double shift;        /* EIGREF_SHIFT: alpha.  EIGREF_LARGEST / EIGREF_SMALLEST: an
                          estimate of lambda_{k+1} of A.  Ignored otherwise. */
  double norm_a;       /* ||A|| (spectral norm or an upper bound); <= 0: ||A||_inf is computed */
  int max_iters;       /* maximum number of sweeps (>= 0) */
  double tol;          /* stopping tolerance; 0 = run exactly max_iters sweeps */
  int stop;            /* enum eigref_stop */
  int precision;       /* enum eigref_precision (dense only; CSR is always FP64) */
  int slices;          /* split forms: 8-bit digit planes per operand, 2..8; 0 = default (8:
                          63 bits, FP64-level products) */
  int beta;            /* enum eigref_beta */
  double delta_c;      /* c of delta = c ||B|| u (Section 3.1.3); <= 0: 10 */
  double div_factor;   /* diverged when ||E_t||_F > div_factor * min_{s<t} ||E_s||_F and
                          ||E_t||_F > div_floor, or ||E_t||_F >= 1; <= 0: 10 */
  double div_floor;    /* <= 0: 1e-4 */
  int check_every;     /* sweeps between host reads of the device status; <= 0: 32 */
  int sign_fix;        /* 1: X <- X Sigma at entry with Algorithm 2's signs (undone on exit) */
  int use_graph;       /* 1: replay each chunk of check_every sweeps as one CUDA graph */
  int profile;         /* 1: time the product kernel of every sweep with CUDA events */
  int rayleigh_ritz;   /* 1: replace X by its Ritz vectors for B first (Section 3.3): solve
                          (X^T B X) S = (X^T X) S D, X <- X S, ordered by |D| descending with each
                          column's largest entry positive; X is returned in that basis.  Pairs
                          with beta = EIGREF_BETA_ZERO for clustered targets. */
  int judge_cols;      /* > 0 and < k: only the correction of columns 0..judge_cols-1 decides the
                          stop and divergence tests (K = k refined vectors, convergence judged on
                          the leading ones, Section 4.1); 0 = all columns */
  int reorth;          /* 1: reorthogonalise the result before returning it (the option of Section
                          3.1.3): two symmetric (Loewdin) steps X <- X (3 I - X^T X) / 2, each
                          squaring ||X^T X - I||, so the columns move by O(||X^T X - I||) */
  int resign;          /* 1: when Y_1 = X_1 - I turns singular mid-run (EIGREF_E_SINGULAR_WY), take
                          the signs of Algorithm 2 for the current X -- the choice Algorithm 3 builds
                          into its WY factors -- and resume from the same iterate (at most 4 times
                          per call; the signs are undone on exit).  refine_dense / refine_csr only. */
  int autotune;        /* 1: the first split-form call for a given (n, k, slices) times the split-K
                          candidates of its tensor-core product and Gram products and keeps the
                          fastest on the handle (results are identical for every choice: the split
                          partials are exact).  0: the built-in choice. */
  double wait_limit_s; /* limit, in seconds, of every bounded wait inside the tensor-core kernels
                          (a pipeline stage that never arrives); <= 0: 2 s.  A wait that runs out
                          ends its kernel early and the call returns EIGREF_E_TIMEOUT with X at
                          the last completed iterate; the handle stays usable.  A tiny limit
                          (1e-9) gives up at the first wait that is not already complete. */
  int product_tile;    /* split form, single problems: columns of the dense product's output tile.
                          64: 128 x 64 tiles (one TMEM accumulator set drained group by group; k must
                          lie in (64 j - 32, 64 j]); 32: 128 x 32 tiles (two accumulator sets);
                          0 = default (64 where k allows it, else 32).  Results are identical for
                          either; EIGREF_E_INVALID for another value or a width k cannot take. */
} eigref_params;

/* Report of one refinement call.  The three array pointers are optional,
 * caller-owned host buffers (NULL = not wanted). */
typedef struct eigref_report {
  int status;                 /* same value the call returns */
  int iterations;             /* sweeps applied */
  double final_rel_residual;  /* ||B X_t - X_t D_t||_F / ||A|| of the last sweep */
  double final_corr_norm;     /* ||E-tilde_L||_F of the last sweep */
  double shift;               /* alpha used */
  double norm_a;              /* ||A|| used */
  double delta;               /* delta used */
  double setup_ms;            /* device time before the first sweep (copies, slicing, sign fix) */
  double sweeps_ms;           /* device time of all sweeps */
  double* eigenvalues;        /* [k]: Rayleigh quotients of the last sweep, plus alpha */
  double* hist_residual;      /* [max_iters]: per-sweep ||R_t||_F / ||A|| */
  double* hist_corr;          /* [max_iters]: per-sweep ||E_t||_F */
  double product_ms;          /* profile = 1: summed device time of the product kernel
                                 (W = B X) over the sweeps applied; else 0 */
  int64_t kernel_launches;    /* kernels launched by the call (graph replays included) */
  int product_launches;       /* product kernels timed in product_ms */
  int psplit;                 /* split form: the product's K decomposition: 1..4 equal K splits a tile,
                                 8 equal-work ranges of (row tile, K block) units, whole rounds of one
                                 CTA per SM (0: FP64 form) */
  int ksplit;                 /* split form: split-K of the Gram products used */
} eigref_report;

/* Defaults: LARGEST_MAG, norm_a computed, max_iters 100, tol 0, correction
 * criterion, FP64, beta cluster, delta_c 10, div 10 / 1e-4, check 32,
 * sign_fix 1, use_graph 1, profile 0, rayleigh_ritz 0, judge_cols 0, reorth 0, resign 0, autotune 1,
 * wait_limit_s 0 (2 s), product_tile 0. */
void eigref_params_default(eigref_params* p);

/* Create a handle on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to issue work on, or NULL for a stream the handle creates and owns.
 * Errors: EIGREF_E_INVALID (h NULL, bad device), EIGREF_E_CUDA. */
int eigref_create(eigref_handle* h, int device, void* cuda_stream);

/* Release the handle, its workspace and its staging buffer for host A.
 * NULL is a no-op. */
int eigref_destroy(eigref_handle h);

/* Refine the k columns of X in place against dense symmetric A (Algorithm 4
 * iterated, Section 3.1.3).  1 <= k <= 128, k < n.  On EIGREF_OK,
 * EIGREF_E_NOT_CONVERGED or EIGREF_E_DIVERGED, X holds the last iterate; on
 * EIGREF_E_NONFINITE the last finite one; on EIGREF_E_INVALID it is untouched.
 * A and X may be device or host memory.  A host A is copied into a device
 * buffer that the handle keeps for later calls (grown when a larger A comes,
 * released by eigref_destroy); page-locked host memory copies fastest.
 * rep may be NULL. */
int eigref_refine_dense(eigref_handle h, const double* A, int64_t n, int64_t lda,
                        double* X, int64_t ldx, int k,
                        const eigref_params* p, eigref_report* rep);

/* Same for CSR A.  The product is an FP64 SpMM.  p->precision EIGREF_FP64:
 * FP64 Gram products; EIGREF_BF16_SLICES: the Gram products X^T X and X^T W
 * as error-free digit planes on the tensor cores (k <= 16, else
 * EIGREF_E_UNSUPPORTED); the k x k stage and the row update stay FP64. */
int eigref_refine_csr(eigref_handle h, const int32_t* row_ptr, const int32_t* col_idx,
                      const double* val, int64_t n, int64_t nnz,
                      double* X, int64_t ldx, int k,
                      const eigref_params* p, eigref_report* rep);

/* One dense problem of a batch.  A (n x n, lda >= n) and X (n x k column-major,
 * ldx >= n, in/out) are device memory; target, shift and norm_a have the
 * meaning of the eigref_params fields of the same names and override them. */
typedef struct eigref_problem {
  const double* A;
  int64_t n;
  int64_t lda;
  double* X;
  int64_t ldx;
  int k;
  int target;
  double shift;
  double norm_a;
} eigref_problem;

/* Refine `count` independent dense problems at once (Algorithm 4 iterated on
 * each, as eigref_refine_dense does).  The problems may differ in n and k.
 * Every problem's sweeps are captured on a stream of its own and the whole
 * batch is replayed as one CUDA graph per chunk of sweeps, so the problems run
 * side by side on the GPU; a problem that has stopped (tol met, diverged,
 * max_iters) does no further work while the others continue.  p gives the
 * shared options (max_iters, tol, stop, precision, slices, beta, ...);
 * p->check_every is capped so that one replay stays near 32k graph nodes.
 * reps (NULL or count entries) receives one report per problem; setup_ms and
 * sweeps_ms are those of the whole batch, product_ms is not measured.
 * Returns EIGREF_OK when every problem ended OK, else the status of the first
 * problem that did not (eigref_last_error names it).  On EIGREF_E_INVALID no
 * X is touched.  Errors: as eigref_refine_dense, plus EIGREF_E_INVALID for
 * count < 1 or host-memory A or X. */
int eigref_refine_batched(eigref_handle h, int count, const eigref_problem* probs,
                          const eigref_params* p, eigref_report* reps);

/* Lines 3-4 of Algorithm 4 on their own: G = X^T X and S = X^T P over all n
 * rows, k x k column-major (ld k) into caller-owned G and S (host or device).
 * X (ldx) and P (ldp) are n x k column-major in device memory.  precision
 * EIGREF_FP64: FP64 dot products; EIGREF_BF16_SLICES: error-free digit
 * planes on the tensor cores (the split form used by eigref_refine_csr),
 * k <= 16, each entry exact up to the slice truncation and one rounding.
 * Errors: EIGREF_E_INVALID (NULL, sizes, host X/P), EIGREF_E_UNSUPPORTED
 * (other precisions, k > 16 in the split form), EIGREF_E_CUDA, EIGREF_E_TIMEOUT. */
int eigref_gram(eigref_handle h, const double* X, int64_t ldx, const double* P, int64_t ldp,
                int64_t n, int k, int precision, int slices, double* G, double* S);

/* Line 1 of Algorithm 4 on its own: P = (A - shift I) X for dense A, with the
 * chosen precision (slices as in eigref_params).  P is n x k column-major
 * (ldp >= n), caller-owned, host or device. */
int eigref_product_dense(eigref_handle h, const double* A, int64_t n, int64_t lda,
                         const double* X, int64_t ldx, int k, double shift,
                         int precision, int slices, double* P, int64_t ldp);

/* P = (A - shift I) X for CSR A, FP64. */
int eigref_product_csr(eigref_handle h, const int32_t* row_ptr, const int32_t* col_idx,
                       const double* val, int64_t n, int64_t nnz,
                       const double* X, int64_t ldx, int k, double shift,
                       double* P, int64_t ldp);

/* Largest n * k that eigref_product_dense_noalloc accepts. */
#define EIGREF_NOALLOC_MAX_ELEMS (1LL << 20)

/* P = (A - shift I) X in FP64, like eigref_product_dense with precision
 * EIGREF_FP64, but without allocating any device memory.  The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc at the point
 * they need the product -- code inside a framework or plugin whose memory
 * pool owns the device and forbids allocations behind its back, or code on a
 * path where an allocation's implicit device synchronisation is not allowed.
 *
 * A, X, P: device pointers on the current CUDA device (host memory is
 * rejected), layouts as in eigref_product_dense, n * k <= 2^20.  Work is
 * queued on `stream` (a cudaStream_t, NULL = the legacy default stream) and
 * the call returns without waiting; P is ready when the stream reaches it.
 *
 * Scratch: a fixed 16 MiB array of device memory inside the library, which
 * every GPU that loads the library holds until the process exits.  The first
 * call on a device looks up that array's address (cudaGetSymbolAddress) and
 * keeps it, so make one call on each device before any stream capture; a
 * cudaDeviceReset of that device makes the kept address stale.  All calls
 * share the array and it keeps the last call's contents; calls whose work
 * overlaps on the GPU (different streams, or different host threads) race on
 * it, so serialise them.  Nothing in it needs to start at zero: each call
 * writes every entry it reads.
 * Errors: EIGREF_E_INVALID (NULL or foreign pointers, sizes out of range,
 * n * k above the limit), EIGREF_E_CUDA (a CUDA error was already pending on
 * the calling thread -- left pending for its owner --, or the address look-up
 * or a launch of this call failed). */
int eigref_product_dense_noalloc(const double* A, int64_t n, int64_t lda,
                                 const double* X, int64_t ldx, int k, double shift,
                                 double* P, int64_t ldp, void* cuda_stream);

/* Static text for a status code. */
const char* eigref_status_string(int status);

/* Text of the last error on this handle ("" if none).  Valid until the next
 * call on the handle. */
const char* eigref_last_error(eigref_handle h);

#ifdef __cplusplus
}
#endif

#endif /* EIGREF_H */

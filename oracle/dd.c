/* ORACLE (test infrastructure only): double-double evaluation of the
 * quantities the refinement is judged by -- eigenpair residuals, Rayleigh
 * quotients, orthogonality X^T X - I, sines of angles to reference vectors and
 * single entries of (A - shift I) X.
 *
 * Double-double arithmetic: an unevaluated sum hi + lo of two doubles,
 * |lo| <= ulp(hi)/2, about 106 bits.  Error-free transformations TwoSum
 * (Knuth, TAOCP vol. 2) and TwoProd via fused multiply-add (Ogita, Rump and
 * Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005),
 * renormalised with FastTwoSum (Dekker, 1971).  Compile with
 * -ffp-contract=off so the compiler fuses nothing on its own.
 *
 * Residual quantities follow Section 3.1.3 (stopping criteria) and Section 4
 * (relative residual, sine of the largest principal angle).
 */
#include <math.h>
#include <stdint.h>

typedef struct { double hi, lo; } dd;

static inline dd two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  dd r = {s, (a - (s - bb)) + (b - bb)};
  return r;
}
static inline dd fast_two_sum(double a, double b) {   /* |a| >= |b| */
  double s = a + b;
  dd r = {s, b - (s - a)};
  return r;
}
static inline dd two_prod(double a, double b) {
  double p = a * b;
  dd r = {p, fma(a, b, -p)};
  return r;
}
static inline dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
static inline dd dd_add_prod(dd acc, double a, double b) { return dd_add(acc, two_prod(a, b)); }
static inline dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return fast_two_sum(p.hi, p.lo);
}
static inline dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return fast_two_sum(p.hi, p.lo);
}
static inline dd dd_neg(dd a) { dd r = {-a.hi, -a.lo}; return r; }
static inline dd dd_div(dd a, dd b) {          /* one Newton correction of hi/hi */
  double q1 = a.hi / b.hi;
  dd r = dd_add(a, dd_neg(dd_mul_d(b, q1)));
  double q2 = r.hi / b.hi;
  r = dd_add(r, dd_neg(dd_mul_d(b, q2)));
  double q3 = r.hi / b.hi;
  dd q = fast_two_sum(q1, q2);
  return dd_add(q, (dd){q3, 0.0});
}
static inline dd dd_from(double a) { dd r = {a, 0.0}; return r; }
static inline double dd_sqrt_d(dd a) {         /* sqrt of a dd to double accuracy */
  if (a.hi <= 0.0) return 0.0;
  double x = sqrt(a.hi);
  dd r = dd_add(a, dd_neg(two_prod(x, x)));
  return x + r.hi / (2.0 * x);
}

/* Exported: the building blocks, for tests against exact rational arithmetic. */
void dd_two_prod(double a, double b, double* hi, double* lo) { dd r = two_prod(a, b); *hi = r.hi; *lo = r.lo; }
void dd_two_sum(double a, double b, double* hi, double* lo) { dd r = two_sum(a, b); *hi = r.hi; *lo = r.lo; }
void dd_dot(const double* x, const double* y, int64_t n, double* hi, double* lo) {
  dd acc = {0.0, 0.0};
  for (int64_t i = 0; i < n; ++i) acc = dd_add_prod(acc, x[i], y[i]);
  *hi = acc.hi; *lo = acc.lo;
}

/* y_j = (A - shift I) x_j in dd for one column (A dense, column-major with lda;
 * symmetric, so row i of A is column i). */
static void dense_apply_col(const double* A, int64_t n, int64_t lda, const double* x, double shift, dd* y) {
  for (int64_t i = 0; i < n; ++i) {
    const double* a = A + i * lda;           /* column i == row i */
    dd acc = {0.0, 0.0};
    for (int64_t l = 0; l < n; ++l) acc = dd_add_prod(acc, a[l], x[l]);
    if (shift != 0.0) acc = dd_add(acc, dd_neg(two_prod(shift, x[i])));
    y[i] = acc;
  }
}

static void csr_apply_col(const int32_t* rp, const int32_t* ci, const double* v, int64_t n,
                          const double* x, double shift, dd* y) {
  for (int64_t i = 0; i < n; ++i) {
    dd acc = {0.0, 0.0};
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) acc = dd_add_prod(acc, v[p], x[ci[p]]);
    if (shift != 0.0) acc = dd_add(acc, dd_neg(two_prod(shift, x[i])));
    y[i] = acc;
  }
}

/* Given y = B x in dd: Rayleigh quotient rq = x^T y / x^T x (dd) and the
 * residual norm || y - rq x ||_2 / ||x||_2 evaluated in dd. */
static void rq_and_residual(const double* x, const dd* y, int64_t n, double* rq_out, double* res_out) {
  dd xx = {0.0, 0.0}, xy = {0.0, 0.0};
  for (int64_t i = 0; i < n; ++i) {
    xx = dd_add_prod(xx, x[i], x[i]);
    xy = dd_add(xy, dd_mul_d(y[i], x[i]));
  }
  dd rq = dd_div(xy, xx);
  dd ss = {0.0, 0.0};
  for (int64_t i = 0; i < n; ++i) {
    dd r = dd_add(y[i], dd_neg(dd_mul_d(rq, x[i])));
    ss = dd_add(ss, dd_mul(r, r));
  }
  *rq_out = rq.hi + rq.lo;
  *res_out = dd_sqrt_d(ss) / dd_sqrt_d(xx);
}

/* Per column j of X (n x k, column-major, ldx): the Rayleigh quotient of
 * B = A - shift I and the residual norm ||B x_j - rq_j x_j|| / ||x_j||,
 * both in double-double.  The work buffer holds n dd per thread. */
void dd_residual_dense(const double* A, int64_t n, int64_t lda, const double* X, int64_t ldx,
                       int k, double shift, double* rq, double* res, dd* work, int nthreads_hint) {
  (void)nthreads_hint;
  #pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < k; ++j) {
    dd* y = work + (int64_t)j * n;
    dense_apply_col(A, n, lda, X + (int64_t)j * ldx, shift, y);
    rq_and_residual(X + (int64_t)j * ldx, y, n, rq + j, res + j);
  }
}

void dd_residual_csr(const int32_t* rp, const int32_t* ci, const double* v, int64_t n,
                     const double* X, int64_t ldx, int k, double shift, double* rq, double* res, dd* work) {
  #pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < k; ++j) {
    dd* y = work + (int64_t)j * n;
    csr_apply_col(rp, ci, v, n, X + (int64_t)j * ldx, shift, y);
    rq_and_residual(X + (int64_t)j * ldx, y, n, rq + j, res + j);
  }
}

/* G = X^T X - I in double-double, rounded to double (k x k, column-major). */
void dd_orth(const double* X, int64_t n, int64_t ldx, int k, double* out) {
  #pragma omp parallel for collapse(2) schedule(dynamic, 4)
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) {
      dd acc = {i == j ? -1.0 : 0.0, 0.0};
      const double* xi = X + (int64_t)i * ldx;
      const double* xj = X + (int64_t)j * ldx;
      for (int64_t l = 0; l < n; ++l) acc = dd_add_prod(acc, xi[l], xj[l]);
      out[i + (int64_t)j * k] = acc.hi + acc.lo;
    }
}

/* sin of the angle between x_j and q_j: || x/|x| - q (q^T x)/(|q||x|) || / |q|
 * evaluated in dd (no arccos, which loses half the digits near 0). */
void dd_sin_angles(const double* X, int64_t ldx, const double* Q, int64_t ldq, int64_t n, int k, double* out) {
  #pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < k; ++j) {
    const double* x = X + (int64_t)j * ldx;
    const double* q = Q + (int64_t)j * ldq;
    dd xx = {0, 0}, qq = {0, 0}, qx = {0, 0};
    for (int64_t l = 0; l < n; ++l) {
      xx = dd_add_prod(xx, x[l], x[l]);
      qq = dd_add_prod(qq, q[l], q[l]);
      qx = dd_add_prod(qx, q[l], x[l]);
    }
    dd c = dd_div(qx, qq);                   /* coefficient of q */
    dd ss = {0, 0};
    for (int64_t l = 0; l < n; ++l) {
      dd r = dd_add(dd_from(x[l]), dd_neg(dd_mul_d(c, q[l])));
      ss = dd_add(ss, dd_mul(r, r));
    }
    /* sin^2 = ||x - c q||^2 / ||x||^2 */
    out[j] = dd_sqrt_d(dd_div(ss, xx));
  }
}

/* Entries ((A - shift I) X)[rows[t], cols[t]] in dd, rounded to double. */
void dd_product_entries(const double* A, int64_t n, int64_t lda, const double* X, int64_t ldx,
                        double shift, const int64_t* rows, const int32_t* cols, int64_t count,
                        double* hi, double* lo) {
  #pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < count; ++t) {
    const double* a = A + rows[t] * lda;
    const double* x = X + (int64_t)cols[t] * ldx;
    dd acc = {0.0, 0.0};
    for (int64_t l = 0; l < n; ++l) acc = dd_add_prod(acc, a[l], x[l]);
    if (shift != 0.0) acc = dd_add(acc, dd_neg(two_prod(shift, x[rows[t]])));
    hi[t] = acc.hi;
    lo[t] = acc.lo;
  }
}

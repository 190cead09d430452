/*
 * Plain, slow, FP64 CPU oracle for block-Jacobi preconditioning, Lanczos condition
 * number estimation and preconditioned CG.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the bench's CPU
 * baseline leg load this library.  It shares no code, header or constant with the CUDA
 * path; both read the same seeded inputs and nothing else.
 *
 * Every routine is written as the textbook definition or the algorithm's steps in the
 * order they are stated, with sequential loops and no blocking or reordering:
 *
 *   or_extract_block   - diagonal block A_k of the partition A = diag(A_1..A_k) (Sec. 3.2)
 *   or_cholesky        - A_k = L L^T, column (gaxpy) Cholesky, Golub & Van Loan Alg. 4.2.1
 *   or_tri_inv_lower   - L^{-1} column by column by forward substitution on e_c
 *   or_minv_from_linv  - M_k^{-1} = L^{-T} L^{-1} by its definition (triple loop)
 *   or_block_apply     - z = M^{-1} r etc. by forward/back substitution with L (Sec. 3.3,
 *                        generalised from point Jacobi M_i = diag(A_i)^{-1} to the full block)
 *   or_spmv, or_dot    - y = A x and x.y in natural order
 *   or_lanczos         - symmetric Lanczos with optional full classical Gram-Schmidt
 *                        reorthogonalisation done twice (CGS2)
 *   or_tridiag_eig_k   - k-th smallest eigenvalue of a symmetric tridiagonal matrix by
 *                        Sturm-sequence bisection
 *   or_pcg             - Hestenes-Stiefel preconditioned CG with the relative residual
 *                        ||b - A x|| / ||b|| of Sec. 3.7 as the stopping test
 *   or_grad_val        - adjoint gradient dL/dA_ij = -lambda_i x_j on the pattern
 *   or_grad_edges      - the same adjoint for a matrix assembled from edge coefficients,
 *                        A = sum_e c_e (e_p - e_q)(e_p - e_q)^T + sum_f c_f e_p e_p^T
 *   zor_*              - the same for complex Hermitian positive definite A (Sec. 3.1):
 *                        A_k = L L^H, M^{-1} = L^{-H} L^{-1}, PCG with conjugate dots,
 *                        Lanczos with a complex basis and a real tridiagonal
 *
 * Condition number (Sec. 3.1): for the SPD operators here kappa = lambda_max/lambda_min.
 *
 * Threads (or_set_threads, default 1): when built with OpenMP, the loops over rows, blocks
 * and vector elements are shared among threads.  No loop changes its arithmetic with the
 * thread count: an element loop computes every element the same way whoever runs it, and a
 * dot product always adds its terms in index order within fixed chunks of OR_CHUNK entries,
 * then the chunk sums in chunk order.  Results are therefore identical for any thread count.
 *
 * Status codes returned: 0 ok, 2 not SPD (Cholesky pivot), 3 CG breakdown,
 * 4 no convergence within max_iter.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_NOT_SPD 2
#define OR_BREAKDOWN 3
#define OR_NO_CONVERGENCE 4

/* Loops shorter than OR_PAR_MIN iterations run on the calling thread only (the result is
 * the same either way; this only avoids the cost of waking threads for tiny inputs). */
#define OR_CHUNK 4096
#define OR_PAR_MIN 32768

void or_set_threads(int32_t t) {
#ifdef _OPENMP
  omp_set_num_threads(t > 0 ? t : 1);
#else
  (void)t;
#endif
}

/* Threads the parallel loops use (1 when built without OpenMP). */
int32_t or_get_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

int64_t or_num_blocks(int64_t n, int32_t bs) { return (n + bs - 1) / bs; }

static int32_t block_rows(int64_t n, int32_t bs, int64_t k) {
  int64_t s = k * (int64_t)bs;
  int64_t e = s + bs;
  if (e > n) e = n;
  return (int32_t)(e - s);
}

/* ------------------------------------------------------------------------- */
/* Block extraction: D(i, j) = A(s+i, s+j) if stored, else 0, for 0 <= i, j < b.
 * D is written with row stride bs (only the b x b corner is meaningful).     */
void or_extract_block(int64_t n, const int32_t *row_ptr, const int32_t *col,
                      const double *val, int32_t bs, int64_t k, double *D) {
  int64_t s = k * (int64_t)bs;
  int32_t b = block_rows(n, bs, k);
  for (int32_t i = 0; i < bs; ++i)
    for (int32_t j = 0; j < bs; ++j) D[(int64_t)i * bs + j] = 0.0;
  for (int32_t i = 0; i < b; ++i) {
    int64_t row = s + i;
    for (int64_t e = row_ptr[row]; e < row_ptr[row + 1]; ++e) {
      int64_t c = col[e];
      if (c >= s && c < s + b) D[(int64_t)i * bs + (c - s)] = val[e];
    }
  }
}

/* All diagonal blocks: out has nblocks * bs * bs doubles. */
void or_extract_blocks(int64_t n, const int32_t *row_ptr, const int32_t *col,
                       const double *val, int32_t bs, double *out) {
  int64_t nb = or_num_blocks(n, bs);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
  for (int64_t k = 0; k < nb; ++k)
    or_extract_block(n, row_ptr, col, val, bs, k, out + k * (int64_t)bs * bs);
}

/* ------------------------------------------------------------------------- */
/* Column (gaxpy) Cholesky of the b x b leading corner of D (row stride ld).
 * L is written lower triangular with stride ld, zeros above the diagonal.
 * A pivot v_j <= tol * max_i D_ii (or not finite) is a failure: returns j, else -1. */
int32_t or_cholesky(int32_t b, int32_t ld, const double *D, double *L, double tol) {
  double dmax = 0.0;
  for (int32_t i = 0; i < b; ++i)
    if (D[(int64_t)i * ld + i] > dmax) dmax = D[(int64_t)i * ld + i];
  for (int32_t i = 0; i < b; ++i)
    for (int32_t j = 0; j < ld; ++j) L[(int64_t)i * ld + j] = 0.0;
  double *v = (double *)malloc(sizeof(double) * (b > 0 ? b : 1));
  int32_t fail = -1;
  for (int32_t j = 0; j < b && fail < 0; ++j) {
    /* v(j:b) = A(j:b, j) - sum_{k<j} L(j:b, k) L(j, k) */
    for (int32_t i = j; i < b; ++i) {
      double s = D[(int64_t)i * ld + j];
      for (int32_t k = 0; k < j; ++k) s -= L[(int64_t)i * ld + k] * L[(int64_t)j * ld + k];
      v[i] = s;
    }
    if (!(v[j] > tol * dmax) || !isfinite(v[j])) {
      fail = j;
      break;
    }
    double d = sqrt(v[j]);
    L[(int64_t)j * ld + j] = d;
    for (int32_t i = j + 1; i < b; ++i) L[(int64_t)i * ld + j] = v[i] / d;
  }
  free(v);
  return fail;
}

/* Factor every block.  Returns -1 if all blocks are SPD, else the first failing block. */
int64_t or_cholesky_blocks(int64_t n, int32_t bs, const double *D, double *L, double tol) {
  int64_t nb = or_num_blocks(n, bs);
  int64_t first = -1;
  if (n < OR_PAR_MIN) {
    for (int64_t k = 0; k < nb; ++k) {
      int32_t b = block_rows(n, bs, k);
      int32_t f = or_cholesky(b, bs, D + k * (int64_t)bs * bs, L + k * (int64_t)bs * bs, tol);
      if (f >= 0) return k;
    }
    return -1;
  }
  /* every block is factored; the smallest failing index is the answer */
  first = nb;
#pragma omp parallel for schedule(static) reduction(min : first)
  for (int64_t k = 0; k < nb; ++k) {
    int32_t b = block_rows(n, bs, k);
    int32_t f = or_cholesky(b, bs, D + k * (int64_t)bs * bs, L + k * (int64_t)bs * bs, tol);
    if (f >= 0 && k < first) first = k;
  }
  return first < nb ? first : -1;
}

/* L^{-1}: for each column c solve L y = e_c by forward substitution. */
void or_tri_inv_lower(int32_t b, int32_t ld, const double *L, double *X) {
  for (int32_t i = 0; i < b; ++i)
    for (int32_t j = 0; j < ld; ++j) X[(int64_t)i * ld + j] = 0.0;
  for (int32_t c = 0; c < b; ++c) {
    for (int32_t i = c; i < b; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int32_t k = c; k < i; ++k) s -= L[(int64_t)i * ld + k] * X[(int64_t)k * ld + c];
      X[(int64_t)i * ld + c] = s / L[(int64_t)i * ld + i];
    }
  }
}

/* M^{-1} = L^{-T} L^{-1}:  Minv(i, j) = sum_k Linv(k, i) Linv(k, j). */
void or_minv_from_linv(int32_t b, int32_t ld, const double *X, double *Minv) {
  for (int32_t i = 0; i < b; ++i)
    for (int32_t j = 0; j < ld; ++j) {
      double s = 0.0;
      if (j < b)
        for (int32_t k = 0; k < b; ++k) s += X[(int64_t)k * ld + i] * X[(int64_t)k * ld + j];
      Minv[(int64_t)i * ld + j] = s;
    }
}

void or_tri_inv_blocks(int64_t n, int32_t bs, const double *L, double *X) {
  int64_t nb = or_num_blocks(n, bs);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
  for (int64_t k = 0; k < nb; ++k)
    or_tri_inv_lower(block_rows(n, bs, k), bs, L + k * (int64_t)bs * bs, X + k * (int64_t)bs * bs);
}

void or_minv_blocks(int64_t n, int32_t bs, const double *X, double *Minv) {
  int64_t nb = or_num_blocks(n, bs);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
  for (int64_t k = 0; k < nb; ++k)
    or_minv_from_linv(block_rows(n, bs, k), bs, X + k * (int64_t)bs * bs, Minv + k * (int64_t)bs * bs);
}

/* ------------------------------------------------------------------------- */
/* Block solves with the Cholesky factors (L blocks, nblocks * bs * bs).
 * mode 0: z = L^{-T} L^{-1} r  (z = M^{-1} r)
 * mode 2: z = L^{-1} r         (forward substitution)
 * mode 3: z = L^{-T} r         (back substitution with L^T)                   */
static void forward_block(int32_t b, int32_t ld, const double *L, const double *r, double *y) {
  for (int32_t i = 0; i < b; ++i) {
    double s = r[i];
    for (int32_t k = 0; k < i; ++k) s -= L[(int64_t)i * ld + k] * y[k];
    y[i] = s / L[(int64_t)i * ld + i];
  }
}

static void backward_block(int32_t b, int32_t ld, const double *L, const double *y, double *z) {
  for (int32_t i = b - 1; i >= 0; --i) {
    double s = y[i];
    for (int32_t k = i + 1; k < b; ++k) s -= L[(int64_t)k * ld + i] * z[k];
    z[i] = s / L[(int64_t)i * ld + i];
  }
}

void or_block_apply(int64_t n, int32_t bs, const double *L, int32_t mode, const double *r,
                    double *z) {
  int64_t nb = or_num_blocks(n, bs);
#pragma omp parallel if (n >= OR_PAR_MIN)
  {
    double *y = (double *)malloc(sizeof(double) * bs);
#pragma omp for schedule(static)
    for (int64_t k = 0; k < nb; ++k) {
      int64_t s = k * (int64_t)bs;
      int32_t b = block_rows(n, bs, k);
      const double *Lk = L + k * (int64_t)bs * bs;
      if (mode == 0) {
        forward_block(b, bs, Lk, r + s, y);
        backward_block(b, bs, Lk, y, z + s);
      } else if (mode == 2) {
        forward_block(b, bs, Lk, r + s, z + s);
      } else {
        backward_block(b, bs, Lk, r + s, z + s);
      }
    }
    free(y);
  }
}

/* ------------------------------------------------------------------------- */
void or_spmv(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val,
             const double *x, double *y) {
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) s += val[e] * x[col[e]];
    y[i] = s;
  }
}

/* x.y: the terms of each chunk of OR_CHUNK entries added in index order, then the chunk
 * sums added in chunk order. */
static double dot_chunk(int64_t lo, int64_t hi, const double *x, const double *y) {
  double s = 0.0;
  for (int64_t i = lo; i < hi; ++i) s += x[i] * y[i];
  return s;
}

static double dot_serial(int64_t n, const double *x, const double *y) {
  double s = 0.0;
  for (int64_t lo = 0; lo < n; lo += OR_CHUNK)
    s += dot_chunk(lo, lo + OR_CHUNK < n ? lo + OR_CHUNK : n, x, y);
  return s;
}

double or_dot(int64_t n, const double *x, const double *y) {
  if (n < OR_PAR_MIN) return dot_serial(n, x, y);
  int64_t nc = (n + OR_CHUNK - 1) / OR_CHUNK;
  double *part = (double *)malloc(sizeof(double) * nc);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    int64_t lo = c * OR_CHUNK;
    part[c] = dot_chunk(lo, lo + OR_CHUNK < n ? lo + OR_CHUNK : n, x, y);
  }
  double s = 0.0;
  for (int64_t c = 0; c < nc; ++c) s += part[c];
  free(part);
  return s;
}

/* Symmetric preconditioned operator y = L^{-1} A L^{-T} v (block L). */
void or_sym_apply(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val,
                  int32_t bs, const double *L, const double *v, double *y, double *tmp1,
                  double *tmp2) {
  or_block_apply(n, bs, L, 3, v, tmp1);
  or_spmv(n, row_ptr, col, val, tmp1, tmp2);
  or_block_apply(n, bs, L, 2, tmp2, y);
}

/* ------------------------------------------------------------------------- */
/* Lanczos on Op = A (L == NULL) or Op = L^{-1} A L^{-T}.
 *   q_1 = v0/||v0|| (or L^{-1} v0 / ||L^{-1} v0|| when preconditioned)
 *   for j = 1..m:  w = Op q_j - beta_{j-1} q_{j-1};  alpha_j = q_j.w;  w -= alpha_j q_j
 *                  reorth: twice { c_i = q_i.w for i <= j;  w -= sum_i c_i q_i }
 *                  beta_j = ||w||;  stop if beta_j <= tol * max(|alpha|, |beta|) so far
 *                  q_{j+1} = w / beta_j
 * alpha[0..steps), beta[0..steps) are written (beta[steps-1] is the last norm).
 * basis: caller workspace of m * n doubles.  Returns the number of steps. */
int32_t or_lanczos(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val,
                   int32_t bs, const double *L, const double *v0, int32_t m, double tol,
                   int32_t reorth, double *alpha, double *beta, double *basis) {
  double *w = (double *)malloc(sizeof(double) * n);
  double *t1 = (double *)malloc(sizeof(double) * n);
  double *t2 = (double *)malloc(sizeof(double) * n);
  double *c = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
  double *q0 = basis;
  if (L) or_block_apply(n, bs, L, 2, v0, q0);
  else memcpy(q0, v0, sizeof(double) * n);
  double nrm = sqrt(or_dot(n, q0, q0));
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
  for (int64_t i = 0; i < n; ++i) q0[i] = q0[i] / nrm;
  double tnorm = 0.0;
  int32_t steps = 0;
  for (int32_t j = 0; j < m; ++j) {
    double *qj = basis + (int64_t)j * n;
    if (L) or_sym_apply(n, row_ptr, col, val, bs, L, qj, w, t1, t2);
    else or_spmv(n, row_ptr, col, val, qj, w);
    if (j > 0) {
      double *qp = basis + (int64_t)(j - 1) * n;
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
      for (int64_t i = 0; i < n; ++i) w[i] -= beta[j - 1] * qp[i];
    }
    double a = or_dot(n, qj, w);
    alpha[j] = a;
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) w[i] -= a * qj[i];
    if (reorth) {
      for (int pass = 0; pass < 2; ++pass) {
        /* c_l = q_l . w (each the chunked dot of or_dot, computed one per thread) */
#pragma omp parallel for schedule(dynamic, 1) if (n >= OR_PAR_MIN)
        for (int32_t l = 0; l <= j; ++l) c[l] = dot_serial(n, basis + (int64_t)l * n, w);
        /* w -= sum_l c_l q_l: every w_i takes its subtractions in the order l = 0, 1, ..., j
           (the loops run over chunks of i, then l, then i within the chunk) */
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
        for (int64_t lo = 0; lo < n; lo += OR_CHUNK) {
          int64_t hi = lo + OR_CHUNK < n ? lo + OR_CHUNK : n;
          for (int32_t l = 0; l <= j; ++l) {
            const double *ql = basis + (int64_t)l * n;
            for (int64_t i = lo; i < hi; ++i) w[i] -= c[l] * ql[i];
          }
        }
      }
    }
    double bj = sqrt(or_dot(n, w, w));
    beta[j] = bj;
    steps = j + 1;
    if (fabs(a) > tnorm) tnorm = fabs(a);
    if (bj > tnorm) tnorm = bj;
    if (bj <= tol * tnorm || j + 1 == m) break;
    if ((int64_t)(j + 1) >= n) break; /* the Krylov space is the whole space */
    double *qn = basis + (int64_t)(j + 1) * n;
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) qn[i] = w[i] / bj;
  }
  free(w); free(t1); free(t2); free(c);
  return steps;
}

/* Number of eigenvalues of the symmetric tridiagonal T (diag a[0..m), off-diag b[0..m-1))
 * that are smaller than x: count of negative pivots of the LDL^T factorisation of T - xI. */
int32_t or_sturm_count(int32_t m, const double *a, const double *b, double x) {
  double bmax2 = 0.0;
  for (int32_t i = 0; i + 1 < m; ++i)
    if (b[i] * b[i] > bmax2) bmax2 = b[i] * b[i];
  double pivmin = DBL_MIN * (bmax2 > 1.0 ? bmax2 : 1.0);
  int32_t cnt = 0;
  double d = 1.0;
  for (int32_t i = 0; i < m; ++i) {
    d = (a[i] - x) - (i > 0 ? (b[i - 1] * b[i - 1]) / d : 0.0);
    if (fabs(d) < pivmin) d = -pivmin;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

/* k-th smallest eigenvalue (0-based) of T by bisection on the Sturm count, starting from
 * the Gershgorin interval and halving until the midpoint no longer moves. */
double or_tridiag_eig_k(int32_t m, const double *a, const double *b, int32_t k) {
  double lo = a[0], hi = a[0];
  for (int32_t i = 0; i < m; ++i) {
    double r = 0.0;
    if (i > 0) r += fabs(b[i - 1]);
    if (i + 1 < m) r += fabs(b[i]);
    if (a[i] - r < lo) lo = a[i] - r;
    if (a[i] + r > hi) hi = a[i] + r;
  }
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (or_sturm_count(m, a, b, mid) > k) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------- */
/* Preconditioned CG (Hestenes-Stiefel) with M = blockdiag(L_k L_k^T):
 *   r = b - A x;  z = M^{-1} r;  p = z;  rho = r.z
 *   loop: q = A p;  alpha = rho / p.q;  x += alpha p;  r -= alpha q;  it++
 *         stop when ||r|| <= tol ||b||
 *         z = M^{-1} r;  rho' = r.z;  beta = rho'/rho;  rho = rho';  p = z + beta p
 * then the true residual b - A x is recomputed; if it is above tol the iteration
 * restarts from the current x (at most max_restarts times).
 * L == NULL means no preconditioner (M = I).
 * out[0] = iterations, out[1] = recurrence rel. residual, out[2] = true rel. residual,
 * out[3] = restarts.  alphas/betas (optional, length max_iter) receive the coefficients
 * of the first cycle.  Returns a status code. */
int32_t or_pcg(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *val,
               int32_t bs, const double *L, const double *b, double *x, double tol,
               int32_t max_iter, int32_t max_restarts, double *out, double *alphas,
               double *betas) {
  double *r = (double *)malloc(sizeof(double) * n);
  double *z = (double *)malloc(sizeof(double) * n);
  double *p = (double *)malloc(sizeof(double) * n);
  double *q = (double *)malloc(sizeof(double) * n);
  int32_t status = OR_OK;
  int32_t it = 0, restarts = 0;
  double bnorm = sqrt(or_dot(n, b, b));
  double rnorm = 0.0, tnorm = 0.0;
  int first_cycle = 1;
  if (bnorm == 0.0) {
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    goto done;
  }
  for (;;) {
    /* (re)start: r = b - A x, z = M^{-1} r, p = z, rho = r.z */
    or_spmv(n, row_ptr, col, val, x, q);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    if (L) or_block_apply(n, bs, L, 0, r, z);
    else memcpy(z, r, sizeof(double) * n);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
    double rho = or_dot(n, r, z);
    rnorm = sqrt(or_dot(n, r, r));
    int converged = rnorm <= tol * bnorm;
    while (!converged) {
      if (it >= max_iter) { status = OR_NO_CONVERGENCE; goto done; }
      if (!(rho > 0.0) || !isfinite(rho)) { status = OR_BREAKDOWN; goto done; }
      or_spmv(n, row_ptr, col, val, p, q);
      double pq = or_dot(n, p, q);
      if (!(pq > 0.0) || !isfinite(pq)) { status = OR_BREAKDOWN; goto done; }
      double alpha = rho / pq;
      if (first_cycle && alphas) alphas[it] = alpha;
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
      for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
      for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
      ++it;
      rnorm = sqrt(or_dot(n, r, r));
      if (rnorm <= tol * bnorm) { converged = 1; break; }
      if (L) or_block_apply(n, bs, L, 0, r, z);
      else memcpy(z, r, sizeof(double) * n);
      double rho_new = or_dot(n, r, z);
      double beta = rho_new / rho;
      if (first_cycle && betas) betas[it - 1] = beta;
      rho = rho_new;
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    /* true residual check */
    or_spmv(n, row_ptr, col, val, x, q);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    tnorm = sqrt(or_dot(n, r, r));
    if (tnorm <= tol * bnorm) break;
    if (restarts >= max_restarts) { status = OR_NO_CONVERGENCE; goto done; }
    ++restarts;
    first_cycle = 0;
  }
done:
  if (out) {
    out[0] = (double)it;
    out[1] = bnorm > 0.0 ? rnorm / bnorm : 0.0;
    if (bnorm > 0.0) {
      or_spmv(n, row_ptr, col, val, x, q);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
      for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
      tnorm = sqrt(or_dot(n, r, r));
      out[2] = tnorm / bnorm;
    } else {
      out[2] = 0.0;
    }
    out[3] = (double)restarts;
  }
  free(r); free(z); free(p); free(q);
  return status;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of x = A^{-1} b with respect to the stored entries of A:
 * dL/dA_ij = -lambda_i x_j for every stored (i, j), where A^T lambda = dL/dx. */
void or_grad_val(int64_t n, const int32_t *row_ptr, const int32_t *col, const double *lambda,
                 const double *x, double *gval) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) gval[e] = -lambda[i] * x[col[e]];
}

/* Adjoint with respect to edge coefficients.  For A(c) = sum_e c_e (e_p - e_q)(e_p - e_q)^T
 * + sum_f c_f e_p e_p^T (a Dirichlet boundary face f touches one node p, marked q < 0),
 * dA/dc_e is that rank-one term, so dL/dc_e = -lambda^T (dA/dc_e) x
 * = -(lambda_p - lambda_q)(x_p - x_q), and -lambda_p x_p for a boundary face. */
void or_grad_edges(int64_t n_edges, const int32_t *p, const int32_t *q, const double *lambda,
                   const double *x, double *gc) {
  for (int64_t e = 0; e < n_edges; ++e) {
    if (q[e] < 0)
      gc[e] = -lambda[p[e]] * x[p[e]];
    else
      gc[e] = -(lambda[p[e]] - lambda[q[e]]) * (x[p[e]] - x[q[e]]);
  }
}

/* ========================================================================= */
/* Complex Hermitian positive definite systems (Sec. 3.1: A is Hermitian PD).
 * Values are C99 double complex (interleaved re, im in memory).  Same algorithms as the real
 * routines above with the Hermitian transpose: A_k = L L^H (real positive diagonal),
 * M^{-1} = L^{-H} L^{-1}, conjugate dot products, and Lanczos with a real tridiagonal. */
#include <complex.h>

typedef double complex zdbl;

static zdbl zdot_chunk(int64_t lo, int64_t hi, const zdbl *x, const zdbl *y) {
  zdbl s = 0.0;
  for (int64_t i = lo; i < hi; ++i) s += conj(x[i]) * y[i];
  return s;
}

/* x^H y: terms added in index order within chunks of OR_CHUNK, then the chunk sums in order. */
static zdbl zdot_serial(int64_t n, const zdbl *x, const zdbl *y) {
  zdbl s = 0.0;
  for (int64_t lo = 0; lo < n; lo += OR_CHUNK)
    s += zdot_chunk(lo, lo + OR_CHUNK < n ? lo + OR_CHUNK : n, x, y);
  return s;
}

static zdbl zdot(int64_t n, const zdbl *x, const zdbl *y) {
  if (n < OR_PAR_MIN) return zdot_serial(n, x, y);
  int64_t nc = (n + OR_CHUNK - 1) / OR_CHUNK;
  zdbl *part = (zdbl *)malloc(sizeof(zdbl) * nc);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    int64_t lo = c * OR_CHUNK;
    part[c] = zdot_chunk(lo, lo + OR_CHUNK < n ? lo + OR_CHUNK : n, x, y);
  }
  zdbl s = 0.0;
  for (int64_t c = 0; c < nc; ++c) s += part[c];
  free(part);
  return s;
}

/* x^H y written to out[0] (re), out[1] (im). */
void zor_dotc(int64_t n, const zdbl *x, const zdbl *y, double *out) {
  zdbl s = zdot(n, x, y);
  out[0] = creal(s);
  out[1] = cimag(s);
}

void zor_spmv(int64_t n, const int32_t *row_ptr, const int32_t *col, const zdbl *val, const zdbl *x,
              zdbl *y) {
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
  for (int64_t i = 0; i < n; ++i) {
    zdbl s = 0.0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) s += val[e] * x[col[e]];
    y[i] = s;
  }
}

void zor_extract_blocks(int64_t n, const int32_t *row_ptr, const int32_t *col, const zdbl *val,
                        int32_t bs, zdbl *out) {
  int64_t nb = or_num_blocks(n, bs);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
  for (int64_t k = 0; k < nb; ++k) {
    zdbl *D = out + k * (int64_t)bs * bs;
    int64_t s = k * (int64_t)bs;
    int32_t b = block_rows(n, bs, k);
    for (int64_t t = 0; t < (int64_t)bs * bs; ++t) D[t] = 0.0;
    for (int32_t i = 0; i < b; ++i) {
      int64_t row = s + i;
      for (int64_t e = row_ptr[row]; e < row_ptr[row + 1]; ++e) {
        int64_t c = col[e];
        if (c >= s && c < s + b) D[(int64_t)i * bs + (c - s)] = val[e];
      }
    }
  }
}

/* Column Cholesky A = L L^H of the b x b corner (stride ld): v(j:b) = A(j:b, j) -
 * sum_{k<j} L(j:b, k) conj(L(j, k)); the pivot is the real part of v(j), which must exceed
 * tol * max_i Re A_ii (and be finite); returns the failing column or -1. */
int32_t zor_cholesky(int32_t b, int32_t ld, const zdbl *D, zdbl *L, double tol) {
  double dmax = 0.0;
  for (int32_t i = 0; i < b; ++i)
    if (creal(D[(int64_t)i * ld + i]) > dmax) dmax = creal(D[(int64_t)i * ld + i]);
  for (int32_t i = 0; i < b; ++i)
    for (int32_t j = 0; j < ld; ++j) L[(int64_t)i * ld + j] = 0.0;
  zdbl *v = (zdbl *)malloc(sizeof(zdbl) * (b > 0 ? b : 1));
  int32_t fail = -1;
  for (int32_t j = 0; j < b && fail < 0; ++j) {
    for (int32_t i = j; i < b; ++i) {
      zdbl s = D[(int64_t)i * ld + j];
      for (int32_t k = 0; k < j; ++k) s -= L[(int64_t)i * ld + k] * conj(L[(int64_t)j * ld + k]);
      v[i] = s;
    }
    double piv = creal(v[j]);
    if (!(piv > tol * dmax) || !isfinite(piv)) {
      fail = j;
      break;
    }
    double d = sqrt(piv);
    L[(int64_t)j * ld + j] = d;
    for (int32_t i = j + 1; i < b; ++i) L[(int64_t)i * ld + j] = v[i] / d;
  }
  free(v);
  return fail;
}

int64_t zor_cholesky_blocks(int64_t n, int32_t bs, const zdbl *D, zdbl *L, double tol) {
  int64_t nb = or_num_blocks(n, bs);
  for (int64_t k = 0; k < nb; ++k) {
    int32_t f = zor_cholesky(block_rows(n, bs, k), bs, D + k * (int64_t)bs * bs, L + k * (int64_t)bs * bs, tol);
    if (f >= 0) return k;
  }
  return -1;
}

/* mode 0: z = L^{-H} L^{-1} r;  2: z = L^{-1} r;  3: z = L^{-H} r. */
static void zforward(int32_t b, int32_t ld, const zdbl *L, const zdbl *r, zdbl *y) {
  for (int32_t i = 0; i < b; ++i) {
    zdbl s = r[i];
    for (int32_t k = 0; k < i; ++k) s -= L[(int64_t)i * ld + k] * y[k];
    y[i] = s / creal(L[(int64_t)i * ld + i]);
  }
}

static void zbackward(int32_t b, int32_t ld, const zdbl *L, const zdbl *y, zdbl *z) {
  for (int32_t i = b - 1; i >= 0; --i) {
    zdbl s = y[i];
    for (int32_t k = i + 1; k < b; ++k) s -= conj(L[(int64_t)k * ld + i]) * z[k];
    z[i] = s / creal(L[(int64_t)i * ld + i]);
  }
}

void zor_block_apply(int64_t n, int32_t bs, const zdbl *L, int32_t mode, const zdbl *r, zdbl *z) {
  int64_t nb = or_num_blocks(n, bs);
#pragma omp parallel if (n >= OR_PAR_MIN)
  {
    zdbl *y = (zdbl *)malloc(sizeof(zdbl) * bs);
#pragma omp for schedule(static)
    for (int64_t k = 0; k < nb; ++k) {
      int64_t s = k * (int64_t)bs;
      int32_t b = block_rows(n, bs, k);
      const zdbl *Lk = L + k * (int64_t)bs * bs;
      if (mode == 0) {
        zforward(b, bs, Lk, r + s, y);
        zbackward(b, bs, Lk, y, z + s);
      } else if (mode == 2) {
        zforward(b, bs, Lk, r + s, z + s);
      } else {
        zbackward(b, bs, Lk, r + s, z + s);
      }
    }
    free(y);
  }
}

/* Preconditioned CG for Hermitian PD A with M = blockdiag(L_k L_k^H), x0 given (x in/out):
 *   r = b - A x;  z = M^{-1} r;  p = z;  rho = r^H z (real)
 *   loop: q = A p;  alpha = rho / Re(p^H q);  x += alpha p;  r -= alpha q;  stop at ||r|| <= tol ||b||
 *         z = M^{-1} r;  rho' = Re(r^H z);  beta = rho'/rho;  p = z + beta p
 * with the same true-residual restarts as or_pcg.  out: iterations, recurrence and true
 * relative residuals, restarts. */
int32_t zor_pcg(int64_t n, const int32_t *row_ptr, const int32_t *col, const zdbl *val, int32_t bs,
                const zdbl *L, const zdbl *b, zdbl *x, double tol, int32_t max_iter,
                int32_t max_restarts, double *out) {
  zdbl *r = (zdbl *)malloc(sizeof(zdbl) * n);
  zdbl *z = (zdbl *)malloc(sizeof(zdbl) * n);
  zdbl *p = (zdbl *)malloc(sizeof(zdbl) * n);
  zdbl *q = (zdbl *)malloc(sizeof(zdbl) * n);
  int32_t status = OR_OK;
  int32_t it = 0, restarts = 0;
  double bnorm = sqrt(creal(zdot(n, b, b)));
  double rnorm = 0.0, tnorm = 0.0;
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    goto done;
  }
  for (;;) {
    zor_spmv(n, row_ptr, col, val, x, q);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    if (L) zor_block_apply(n, bs, L, 0, r, z);
    else memcpy(z, r, sizeof(zdbl) * n);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
    double rho = creal(zdot(n, r, z));
    rnorm = sqrt(creal(zdot(n, r, r)));
    int converged = rnorm <= tol * bnorm;
    while (!converged) {
      if (it >= max_iter) { status = OR_NO_CONVERGENCE; goto done; }
      if (!(rho > 0.0) || !isfinite(rho)) { status = OR_BREAKDOWN; goto done; }
      zor_spmv(n, row_ptr, col, val, p, q);
      double pq = creal(zdot(n, p, q));
      if (!(pq > 0.0) || !isfinite(pq)) { status = OR_BREAKDOWN; goto done; }
      double alpha = rho / pq;
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
      for (int64_t i = 0; i < n; ++i) x[i] += alpha * p[i];
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
      for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
      ++it;
      rnorm = sqrt(creal(zdot(n, r, r)));
      if (rnorm <= tol * bnorm) { converged = 1; break; }
      if (L) zor_block_apply(n, bs, L, 0, r, z);
      else memcpy(z, r, sizeof(zdbl) * n);
      double rho_new = creal(zdot(n, r, z));
      double beta = rho_new / rho;
      rho = rho_new;
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    zor_spmv(n, row_ptr, col, val, x, q);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    tnorm = sqrt(creal(zdot(n, r, r)));
    if (tnorm <= tol * bnorm) break;
    if (restarts >= max_restarts) { status = OR_NO_CONVERGENCE; goto done; }
    ++restarts;
  }
done:
  if (out) {
    out[0] = (double)it;
    out[1] = bnorm > 0.0 ? rnorm / bnorm : 0.0;
    if (bnorm > 0.0) {
      zor_spmv(n, row_ptr, col, val, x, q);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
      for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
      out[2] = sqrt(creal(zdot(n, r, r))) / bnorm;
    } else {
      out[2] = 0.0;
    }
    out[3] = (double)restarts;
  }
  free(r); free(z); free(p); free(q);
  return status;
}

/* Hermitian Lanczos on Op = A (L == NULL) or L^{-1} A L^{-H}, complex basis, real tridiagonal:
 *   q_1 = v0/||v0|| (L^{-1} v0 normalised when preconditioned)
 *   w = Op q_j - beta_{j-1} q_{j-1};  alpha_j = Re(q_j^H w);  w -= alpha_j q_j
 *   reorth: twice { c_l = q_l^H w for l <= j;  w -= sum_l c_l q_l }
 *   beta_j = ||w||; stop as or_lanczos.  basis: m * n complex workspace. */
int32_t zor_lanczos(int64_t n, const int32_t *row_ptr, const int32_t *col, const zdbl *val, int32_t bs,
                    const zdbl *L, const zdbl *v0, int32_t m, double tol, int32_t reorth, double *alpha,
                    double *beta, zdbl *basis) {
  zdbl *w = (zdbl *)malloc(sizeof(zdbl) * n);
  zdbl *t1 = (zdbl *)malloc(sizeof(zdbl) * n);
  zdbl *t2 = (zdbl *)malloc(sizeof(zdbl) * n);
  zdbl *c = (zdbl *)malloc(sizeof(zdbl) * (m > 0 ? m : 1));
  zdbl *q0 = basis;
  if (L) zor_block_apply(n, bs, L, 2, v0, q0);
  else memcpy(q0, v0, sizeof(zdbl) * n);
  double nrm = sqrt(creal(zdot(n, q0, q0)));
  for (int64_t i = 0; i < n; ++i) q0[i] = q0[i] / nrm;
  double tnorm = 0.0;
  int32_t steps = 0;
  for (int32_t j = 0; j < m; ++j) {
    zdbl *qj = basis + (int64_t)j * n;
    if (L) {
      zor_block_apply(n, bs, L, 3, qj, t1);
      zor_spmv(n, row_ptr, col, val, t1, t2);
      zor_block_apply(n, bs, L, 2, t2, w);
    } else {
      zor_spmv(n, row_ptr, col, val, qj, w);
    }
    if (j > 0) {
      zdbl *qp = basis + (int64_t)(j - 1) * n;
      for (int64_t i = 0; i < n; ++i) w[i] -= beta[j - 1] * qp[i];
    }
    double a = creal(zdot(n, qj, w));
    alpha[j] = a;
    for (int64_t i = 0; i < n; ++i) w[i] -= a * qj[i];
    if (reorth) {
      for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel for schedule(dynamic, 1) if (n >= OR_PAR_MIN)
        for (int32_t l = 0; l <= j; ++l) c[l] = zdot_serial(n, basis + (int64_t)l * n, w);
#pragma omp parallel for schedule(static) if (n >= OR_PAR_MIN)
        for (int64_t lo = 0; lo < n; lo += OR_CHUNK) {
          int64_t hi = lo + OR_CHUNK < n ? lo + OR_CHUNK : n;
          for (int32_t l = 0; l <= j; ++l) {
            const zdbl *ql = basis + (int64_t)l * n;
            for (int64_t i = lo; i < hi; ++i) w[i] -= c[l] * ql[i];
          }
        }
      }
    }
    double bj = sqrt(creal(zdot(n, w, w)));
    beta[j] = bj;
    steps = j + 1;
    if (fabs(a) > tnorm) tnorm = fabs(a);
    if (bj > tnorm) tnorm = bj;
    if (bj <= tol * tnorm || j + 1 == m) break;
    if ((int64_t)(j + 1) >= n) break;
    zdbl *qn = basis + (int64_t)(j + 1) * n;
    for (int64_t i = 0; i < n; ++i) qn[i] = w[i] / bj;
  }
  free(w); free(t1); free(t2); free(c);
  return steps;
}

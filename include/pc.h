/*
 * pc.h - C ABI of libpc: GB300-native block-Jacobi preconditioning, Lanczos condition
 * number estimation and preconditioned CG for sparse SPD systems A x = b.
 *
 * What the paper defines (arXiv 2410.02408):
 *   Sec. 3.1  A is sparse, Hermitian (here: real symmetric) positive definite; the cost
 *             driver is kappa(A) = ||A|| ||A^{-1}|| (= lambda_max / lambda_min for SPD).
 *   Sec. 3.2  A and b are partitioned into contiguous diagonal blocks A_1..A_k of size nb.
 *   Sec. 3.3  each block is preconditioned (point Jacobi M_i = diag(A_i)^{-1} in the
 *             paper; here the full block, M = blockdiag(A_kk) = blockdiag(L_k L_k^T), which
 *             equals the paper's preconditioner at block_size 1).
 *   Sec. 3.6  block solutions are concatenated (z = M^{-1} r writes disjoint slices).
 *   Sec. 3.7  accuracy is the relative residual ||A x - b|| / ||b||.
 *
 * Conventions for every entry point:
 *   - All array arguments are DEVICE pointers owned by the caller, unless stated.  They
 *     are read (or written) during the call only; nothing is retained, except that a
 *     pc_handle keeps the CSR pointers given to pc_setup and reads them in later
 *     pc_apply / pcg_solve_h calls, so the caller keeps that CSR alive and unchanged
 *     until pc_destroy.
 *   - Handles and their workspaces are owned by the library: created by pc_setup,
 *     released by pc_destroy.  Their device memory comes from a memory pool of the library
 *     (one per device) that keeps released memory for later handles rather than returning
 *     it to the driver (an allocation that would fail first trims the pool); pc_destroy
 *     waits for the device, as cudaFree does, and must run with the handle's device
 *     current.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).  Work is
 *     enqueued on it; calls that report a device-side status (setup, solve, kappa)
 *     synchronise the stream before returning.
 *   - No call aborts, prints or traps.  Every failure is a pc_status; details are in the
 *     info structs.  Device-side waits are bounded (PC_ERR_TIMEOUT).
 *   - CSR: square, int32 indices, column indices sorted and unique in each row, explicit
 *     diagonal.  n < 2^31, nnz < 2^31.  Every entry point that takes a CSR without a handle
 *     (pc_setup, hence pcg_solve and kappa_estimate with block_size > 0; kappa_estimate and
 *     kappa_estimate_h without a handle; pcg_solve_noalloc; pc_spmv; pc_extract_blocks;
 *     pc_grad_val) first runs an O(nnz) structure check on the device (pc_csr_check) and
 *     returns PC_ERR_INVALID_ARG before any other kernel reads the matrix when it fails; the
 *     check reads only row_ptr[0..n] and col_idx[0..nnz) and synchronises the stream.
 *   - Block partition: block k covers rows [k*bs, min(n, (k+1)*bs)); the last block may
 *     be shorter and is padded with the identity internally (the result is unchanged).
 *     1 <= block_size <= 64.
 *
 * Environment variables (read when the setting is needed; the pc_set_* calls take
 * precedence where both exist):
 *   PC_CG_ENGINE=graph|persistent   CG engine (pc_set_cg_engine).
 *   PC_WAIT_BUDGET=<cycles>         bound of every device-side wait (pc_set_wait_budget).
 *   PC_BIN_SPMV=pipe|plain          row loop of the binned CG SpMV, read when a handle first
 *                                   solves: pipelined (default, 2 CTAs per SM) or plain (4).
 *   PC_CG_PROFILE=1                 graph engine: launch the loop body kernels one by one with
 *                                   events around each (per-kernel times, pc_get_trace); every
 *                                   step starts with a 40 us spacer kernel so that the event
 *                                   intervals exclude the host's launch latency.
 *   PC_TRACE_BARRIERS=N             persistent engine: record N barrier timestamps.
 *   PC_BATCH_PROFILE=1              batched mode: per-phase device timers (pc_batch_profile).
 */
#ifndef PC_H_
#define PC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PC_OK = 0,
  PC_ERR_INVALID_ARG = 1,    /* bad size, pointer, block size, mode or precision      */
  PC_ERR_NOT_SPD = 2,        /* a block's Cholesky pivot <= tol * max diag of the block */
  PC_ERR_BREAKDOWN = 3,      /* CG: p.q <= 0, r.z <= 0 or a non-finite scalar          */
  PC_ERR_NO_CONVERGENCE = 4, /* max_iter reached (x holds the last iterate)            */
  PC_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up                    */
  PC_ERR_CUDA = 6,           /* a CUDA runtime call failed                            */
  PC_ERR_OOM = 7             /* device allocation failed                              */
} pc_status;

typedef enum { PC_F64 = 0, PC_F32 = 1 } pc_dtype; /* type of the CSR values */

/* Precision of the block factors and of their application.  PC_PREC_FP64: factor and
 * apply in FP64.  PC_PREC_FP32: factor and apply in FP32 (FP32 accumulation); CG vectors,
 * residual update, dot products and scalars stay FP64, so the outer FP64 CG is the
 * iterative refinement that recovers full accuracy.  PC_PREC_TF32: as PC_PREC_FP32, except
 * that M_k^{-1} = L_k^{-T} L_k^{-1} is formed on the tensor cores (mma.sync m16n8k8) from
 * L_k^{-1} rounded to TF32 (round to nearest, ties away from zero) with FP32 accumulation;
 * the Cholesky factor and L_k^{-1} are FP32, and the stored M_k^{-1} is exactly symmetric. */
typedef enum { PC_PREC_FP64 = 0, PC_PREC_FP32 = 1, PC_PREC_TF32 = 2 } pc_prec;

/* pc_apply modes (L_k is the Cholesky factor of the diagonal block A_kk):
 *   INV   : out = M^{-1} in = L^{-T} L^{-1} in          (the PCG preconditioner)
 *   SYM   : out = L^{-1} A L^{-T} in                    (symmetric preconditioned operator;
 *                                                        same spectrum as M^{-1} A)
 *   LINV  : out = L^{-1} in
 *   LTINV : out = L^{-T} in                                                            */
typedef enum { PC_APPLY_INV = 0, PC_APPLY_SYM = 1, PC_APPLY_LINV = 2, PC_APPLY_LTINV = 3 } pc_apply_mode;

typedef struct {
  int64_t n;               /* rows = columns                                  */
  int64_t nnz;             /* stored entries                                  */
  const int32_t *row_ptr;  /* device [n+1], row_ptr[0] = 0, row_ptr[n] = nnz */
  const int32_t *col_idx;  /* device [nnz]                                    */
  const void *val;         /* device [nnz], double (PC_F64) or float (PC_F32) */
  int32_t dtype;           /* pc_dtype                                        */
} pc_csr;

typedef struct pc_handle pc_handle; /* opaque, library-owned */

typedef struct {
  int32_t status;            /* same value the call returns                           */
  int32_t iterations;        /* CG iterations (matrix-vector products with p)         */
  int32_t restarts;          /* true-residual restarts taken                          */
  int32_t failed_block;      /* PC_ERR_NOT_SPD: first failing block index, else -1    */
  double rel_residual;       /* recurrence ||r|| / ||b|| at exit                      */
  double true_rel_residual;  /* ||b - A x|| / ||b|| recomputed at exit                */
  double setup_ms;           /* pc_setup time inside pcg_solve (0 for pcg_solve_h)    */
  double solve_ms;           /* CG kernel time (CUDA events on the stream)            */
  int32_t grid_ctas;         /* CTAs of the persistent CG launch (0: graph engine)     */
  int32_t block_size;
  int32_t prec;              /* pc_prec used                                          */
  int32_t reserved;
} pc_solve_info;

typedef struct {
  int32_t status;
  int32_t steps;         /* Lanczos steps taken (<= max_steps)              */
  double kappa;          /* theta_max / theta_min of the Lanczos tridiagonal */
  double lambda_min;     /* theta_min                                      */
  double lambda_max;     /* theta_max                                      */
  double *alpha;         /* optional HOST array [max_steps] (caller-owned) receiving the
                            tridiagonal's diagonal, or NULL                  */
  double *beta;          /* optional HOST array [max_steps]: beta[j] = ||w_j|| after step
                            j (the off-diagonal for j < steps-1), or NULL     */
  double elapsed_ms;
} pc_kappa_info;

/* ---------------------------------------------------------------------------------
 * pc_setup - build the block-Jacobi preconditioner (Sec. 3.2-3.3): extract the diagonal
 * blocks A_kk from CSR and factor each one, A_kk = L_k L_k^T, storing L_k^{-1} and
 * M_k^{-1} = L_k^{-T} L_k^{-1} on the device.
 *   A          CSR (device arrays; kept by the handle, see conventions).
 *   block_size 1..64.
 *   tol        pivot threshold: a pivot <= tol * max_i (A_kk)_ii fails (PC_ERR_NOT_SPD).
 *   prec       pc_prec.
 *   out        receives the new handle (NULL on failure, except PC_ERR_NOT_SPD, where
 *              the handle is still returned so that pc_handle_failed_block can be read;
 *              destroy it with pc_destroy).
 */
pc_status pc_setup(const pc_csr *A, int32_t block_size, double tol, int32_t prec, void *stream,
                   pc_handle **out);

/* pc_csr_check - the O(nnz) structure check that the CSR entry points run: row_ptr[0] = 0,
 * row ranges non-decreasing and inside [0, nnz], row_ptr[n] = nnz, every column index in
 * [0, n), columns strictly increasing within each row, and the diagonal entry stored in every
 * row (Sec. 3.1 takes A sparse and Hermitian positive definite; these are the storage rules
 * this library's kernels rely on).  One device thread per row reads only row_ptr[0..n] and
 * col_idx[0..nnz); no value is read and nothing is gathered through a column index.
 *   flags  (host, may be NULL) receives the OR of the violations found: 1 row pointers,
 *          2 a column out of range, 4 columns not strictly increasing, 8 a missing diagonal.
 * Returns PC_OK or PC_ERR_INVALID_ARG (also for a malformed descriptor: n <= 0, null
 * pointers, bad dtype).  Synchronises the stream. */
pc_status pc_csr_check(const pc_csr *A, uint32_t *flags, void *stream);

/* First failing block of the last pc_setup on h (-1 if none). */
int64_t pc_handle_failed_block(const pc_handle *h);

/* 1 if the handle was created with FP32/TF32 factors and an FP32 pivot broke down, so that
 * pc_setup factored every block again in FP64 arithmetic (the stored factors stay FP32);
 * NOT_SPD is reported only if that FP64 factorisation fails too.  0 otherwise. */
int32_t pc_handle_refactored_fp64(const pc_handle *h);

/* pc_apply - out = op(in) for op in pc_apply_mode; in and out are device [n] doubles and
 * must not overlap.  Stream-ordered, does not synchronise. */
pc_status pc_apply(pc_handle *h, int32_t mode, const double *in, double *out, void *stream);

/* pc_apply_tol - pc_apply with a refinement tolerance for z = M^{-1} r (Sec. 3.3's per-block
 * solve; the mixed-precision pattern "FP32 factors, FP64 refinement").  tol = 0: exactly
 * pc_apply (any mode).  tol > 0 (mode PC_APPLY_INV only, else PC_ERR_INVALID_ARG): z starts as
 * the apply with the stored factors, then while ||r - blockdiag(A) z|| > tol ||r|| (the
 * diagonal blocks of the partition read from the CSR in FP64) and fewer than 20 corrections
 * were made, z += M^{-1} (r - blockdiag(A) z).  *steps (HOST, may be NULL): corrections made;
 * *rel_residual (HOST, may be NULL): the last ||r - blockdiag(A) z|| / ||r|| (0 for r = 0).
 * Returns PC_ERR_NO_CONVERGENCE when the tolerance was not reached (out holds the last z) and
 * PC_ERR_BREAKDOWN for a non-finite residual.  With tol > 0 it synchronises the stream and
 * allocates a workspace of about 2n + 521 doubles on the handle at its first use. */
pc_status pc_apply_tol(pc_handle *h, int32_t mode, const double *in, double *out, double tol,
                       int32_t *steps, double *rel_residual, void *stream);

/* pc_get_factor - copy the stored factor of h into dense row-major blocks
 * out[k][i][j] (device, nblocks * bs * bs doubles): which = 0 gives L_k^{-1} (lower
 * triangular), which = 1 gives M_k^{-1}.  Padding rows/columns of the last block are
 * written as the identity. */
pc_status pc_get_factor(const pc_handle *h, int32_t which, double *out, void *stream);

/* pc_destroy - free the handle and its device workspace (synchronises nothing; the
 * caller must not have work using h still in flight). */
pc_status pc_destroy(pc_handle *h);

/* pc_extract_blocks - the diagonal blocks of the partition (Sec. 3.2) as dense row-major
 * tiles out[k][i][j] = A(k*bs+i, k*bs+j) (0 where not stored or beyond n), device
 * nblocks * bs * bs doubles.  Values are copied bit-exactly (float values are widened). */
pc_status pc_extract_blocks(const pc_csr *A, int32_t block_size, double *out, void *stream);

/* pc_spmv - y = A x (device [n] doubles). */
pc_status pc_spmv(const pc_csr *A, const double *x, double *y, void *stream);

/* pc_dot - *result = x . y (device scalar), fixed-order reduction (bit-reproducible). */
pc_status pc_dot(int64_t n, const double *x, const double *y, double *result, void *stream);

/* pc_debug_convert - the float <-> double conversions that the mixed-precision kernels
 * (FP32 factors applied to FP64 vectors, FP32 CSR values in FP64 products) perform on the
 * integer pipe instead of the FP64 pipe, exposed element by element so that they can be
 * checked against IEEE-754 conversion: out_f[i] = in_d[i] rounded to float (round to nearest,
 * ties to even; overflow to infinity), out_d[i] = in_f[i] widened exactly.  Support call; the
 * paper has no counterpart.  Device arrays of n elements.  Stream-ordered, no synchronisation. */
pc_status pc_debug_convert(int64_t n, const double *in_d, float *out_f, const float *in_f, double *out_d,
                           void *stream);

/* pc_debug_mma_tf32 - one tensor-core product as PC_PREC_TF32's setup issues it: d = a b with
 * a 16 x 8 and b 8 x 8 (device, row-major FP32), both rounded to TF32 (round to nearest, ties
 * away from zero), FP32 accumulation; d is 16 x 8 row-major.  Support call for checking the
 * fragment mapping; the paper has no counterpart.  Stream-ordered, no synchronisation. */
pc_status pc_debug_mma_tf32(const float *a, const float *b, float *d, void *stream);

/* ---------------------------------------------------------------------------------
 * kappa_estimate - Lanczos estimate of kappa (Sec. 3.1) for A (block_size == 0) or for
 * the block-Jacobi preconditioned operator L^{-1} A L^{-T} (block_size > 0, FP64
 * factors), whose spectrum is that of M^{-1} A.
 *   max_steps  Lanczos steps m (<= 256).
 *   tol        early stop when beta_j <= tol * max(|alpha|, |beta|) so far.
 *   v0         device [n] start vector (q_1 = v0/||v0||, or L^{-1} v0 / ||L^{-1} v0||
 *              when preconditioned); must be non-zero.
 *   reorth     0: plain three-term recurrence; 1: full reorthogonalisation against all
 *              previous Lanczos vectors, classical Gram-Schmidt applied twice.
 * The extreme Ritz values are found by Sturm-count bisection in FP64 on the device.
 * Workspace (max_steps * n doubles for the basis) is allocated and freed by the call. */
pc_status kappa_estimate(const pc_csr *A, int32_t block_size, int32_t max_steps, double tol,
                         const double *v0, int32_t reorth, pc_kappa_info *info, void *stream);

/* Same on an existing handle (any precision; NULL handle = unpreconditioned, then A is
 * taken from the csr argument). */
pc_status kappa_estimate_h(pc_handle *h, const pc_csr *A, int32_t max_steps, double tol,
                           const double *v0, int32_t reorth, pc_kappa_info *info, void *stream);

/* ---------------------------------------------------------------------------------
 * pcg_solve - solve A x = b by block-Jacobi preconditioned CG until the recurrence
 * residual satisfies ||r|| <= tol ||b|| (Sec. 3.7), then recompute b - A x; if that is
 * above tol, restart from x (at most 3 times).  Default engine: a CUDA graph whose device-
 * driven `while` node runs three kernels per iteration (q = A p with p.q; r update,
 * z = M^{-1} r with r.z and r.r; x and p updates) until the last kernel's last CTA clears the
 * loop condition, with the host out of the loop; the alternative (pc_set_cg_engine(1)) is one
 * persistent cooperative kernel with two reductions and one plain grid barrier per step.
 * Both use fixed-order reductions (bit-reproducible for a given device).
 *   x    device [n]: in = initial guess x0, out = solution (last iterate on failure).
 *   prec pc_prec of the preconditioner; CG itself is FP64.
 * pcg_solve builds (and frees) the preconditioner; pcg_solve_h reuses a handle. */
pc_status pcg_solve(const pc_csr *A, int32_t block_size, const double *b, double *x, double tol,
                    int32_t max_iter, int32_t prec, pc_solve_info *info, void *stream);

pc_status pcg_solve_h(pc_handle *h, const double *b, double *x, double tol, int32_t max_iter,
                      pc_solve_info *info, void *stream);

/* pcg_solve_noalloc - the same solve as pcg_solve with the persistent engine
 * (pc_set_cg_engine(1): same kernels, same grid, same wait budget, same results), for
 * callers that cannot allocate device memory.  The paper has no counterpart; this is a
 * deployment variant.  Examples of such callers: plug-ins hosted by a framework whose
 * caching allocator owns the device memory (a cudaMalloc behind its back can fail or fragment
 * the pool it manages), and latency-critical loops that must not enter the driver's allocator
 * (cudaMalloc and cudaFree can block and synchronise the device).  The caller passes only
 * inputs and outputs (A, b, x as in pcg_solve); every byte of scratch (block factors, four CG
 * vectors, reduction partials, barrier and status words) comes from one fixed device array of
 * PC_NOALLOC_SCRATCH_BYTES that the library defines statically, so every GPU that loads libpc
 * holds that much memory until the process exits.
 *   Limit: the problem must fit, i.e. roughly (K+1 + bs) * n * e + 32 n bytes plus a few KB
 *   for factors of element size e (8 for PC_PREC_FP64, 4 otherwise), K = bs/2, with the
 *   factor arrays padded to whole 32-row warp units and the vectors to multiples of 32 rows;
 *   larger problems return PC_ERR_INVALID_ARG before any work is enqueued.
 *   The call runs the CSR structure check (pc_csr_check), then setup, then the solve, and
 *   synchronises the stream after each of them (and after the FP64 refactorisation that
 *   follows an FP32 pivot breakdown, as in pc_setup) to read their status words back.
 *   The first call on each device looks up the array's device address (cudaGetSymbolAddress
 *   with that device current) and caches it.  All calls share the one array and it keeps the
 *   previous call's contents (the call clears what must start at zero): calls that overlap on
 *   the GPU (different streams or threads on the same device) race and must be serialised by
 *   the caller.  No cudaMalloc, cudaFree or allocating library routine is called;
 *   info->solve_ms and info->setup_ms are not measured (0). */
#define PC_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
pc_status pcg_solve_noalloc(const pc_csr *A, int32_t block_size, const double *b, double *x,
                            double tol, int32_t max_iter, int32_t prec, pc_solve_info *info,
                            void *stream);

/* pc_grad_val - adjoint of x = A^{-1} b with respect to the stored entries of A:
 * grad_val[e] = -lambda[row(e)] * x[col(e)] for every stored entry e, where lambda solves
 * A^T lambda = dL/dx (A symmetric here).  Device arrays: lambda, x [n]; grad_val [nnz]. */
pc_status pc_grad_val(const pc_csr *A, const double *lambda, const double *x, double *grad_val,
                      void *stream);

/* pc_grad_edges - the same adjoint for a matrix assembled from edge coefficients,
 * A(c) = sum_e c_e (e_p - e_q)(e_p - e_q)^T + sum_f c_f e_p e_p^T (graph Laplacians and the
 * variable-coefficient diffusion stencils: an interior face couples cells p and q, a
 * Dirichlet boundary face touches cell p only and is marked q < 0).  dA/dc_e is that
 * rank-one term, so
 *     grad_c[e] = -(lambda[p[e]] - lambda[q[e]]) * (x[p[e]] - x[q[e]])   (q[e] >= 0)
 *     grad_c[e] = -lambda[p[e]] * x[p[e]]                                 (q[e] <  0)
 * Device arrays: p, q int32 [n_edges]; lambda, x [n]; grad_c [n_edges] (written).  Edges
 * whose indices fall outside 0..n-1 get NaN.  Enqueued on stream; PC_ERR_INVALID_ARG for
 * null pointers, negative sizes or n > INT32_MAX. */
pc_status pc_grad_edges(int64_t n_edges, const int32_t *p, const int32_t *q, const double *lambda,
                        const double *x, int64_t n, double *grad_c, void *stream);

/* ---------------------------------------------------------------------------------
 * Complex Hermitian positive definite systems (Sec. 3.1 takes A Hermitian PD).  Values are
 * complex doubles stored as interleaved (real, imaginary) pairs, vectors likewise.
 *
 * A z = f is solved as the real system K y = g with y = (Re z_0, Im z_0, Re z_1, ...): the
 * 2x2 block (i, j) of K is [[b, -c], [c, b]] for a_ij = b + i c.  K is SPD exactly when A is
 * Hermitian PD and has A's eigenvalues (each twice).  The Cholesky factor of the real form of a
 * complex diagonal block is the real form of its complex factor A_kk = L_k L_k^H (uniqueness of
 * the Cholesky factor), so block-Jacobi on K with block size 2 bs is the complex block-Jacobi
 * preconditioner M = blockdiag(L_k L_k^H), and because every CG and Lanczos scalar of a Hermitian
 * PD system is real, PCG and Lanczos on K follow the complex iterations step for step.
 * The CSR structure rules (and pc_csr_check) are those of real matrices; Hermitian symmetry is
 * the caller's contract (an input that is not Hermitian gives an unsymmetric K and typically a
 * CG breakdown).  n < 2^30, nnz < 2^29 (K has 2n rows and 4 nnz entries). */
typedef struct {
  int64_t n;               /* rows = columns                                            */
  int64_t nnz;             /* stored complex entries                                    */
  const int32_t *row_ptr;  /* device [n+1]                                              */
  const int32_t *col_idx;  /* device [nnz], sorted and unique per row, diagonal stored  */
  const double *val;       /* device [2 nnz]: (re, im) of every entry                   */
} pc_csr_z;

/* pc_hermitian_real_form - the real form K of A into caller-owned device arrays: row_ptr
 * [2n+1], col_idx [4 nnz], val [4 nnz] (FP64); real rows 2i and 2i+1 hold the real and the
 * imaginary parts of complex row i, columns 2j and 2j+1 for complex column j.  Runs the CSR
 * structure check first (synchronises the stream). */
pc_status pc_hermitian_real_form(const pc_csr_z *A, int32_t *row_ptr, int32_t *col_idx, double *val,
                                 void *stream);

/* pcg_solve_z - block-Jacobi PCG for Hermitian PD A (complex block size 1..32; b, x device
 * [2n] interleaved, x in = x0).  Builds K in library-owned device memory (freed before return)
 * and runs pcg_solve on it with block size 2 * block_size; info as pcg_solve (failed_block is
 * the complex block index, block_size the complex one). */
pc_status pcg_solve_z(const pc_csr_z *A, int32_t block_size, const double *b, double *x, double tol,
                      int32_t max_iter, int32_t prec, pc_solve_info *info, void *stream);

/* kappa_estimate_z - Lanczos kappa of A (block_size 0) or of L^{-1} A L^{-H} (complex block size
 * 1..32), v0 device [2n] interleaved; as kappa_estimate on K. */
pc_status kappa_estimate_z(const pc_csr_z *A, int32_t block_size, int32_t max_steps, double tol,
                           const double *v0, int32_t reorth, pc_kappa_info *info, void *stream);

/* ---------------------------------------------------------------------------------
 * Batched mode: many independent SPD systems of uneven size, each with its own block
 * size.  Block-Jacobi setup (Sec. 3.2-3.3) and PCG to ||b_s - A_s x_s|| <= tol ||b_s||
 * (Sec. 3.7) for every system run inside ONE persistent cooperative kernel launch, which
 * pc_batch_solve captures in a CUDA graph (a counter reset plus that launch) and replays.
 *
 * Each system is handled by a team of co-resident CTAs sized by its estimated work (a
 * power of two up to the team limit); teams take queue slots in order of decreasing
 * work and synchronise through their own bounded release/acquire barriers.  Reductions
 * are fixed-order, so results are bit-reproducible for a given schedule.
 *
 *   n_sys          number of systems (>= 1).
 *   sys_row        device int64 [n_sys+1]: system s owns rows [sys_row[s], sys_row[s+1])
 *                  of the concatenated CSR (sys_row[0] = 0, sys_row[n_sys] = n_rows);
 *                  row_ptr holds global nnz offsets (row_ptr[0] = 0, row_ptr[n_rows] = nnz).
 *   col_idx        LOCAL column indices (0 .. N_s - 1) of each system, sorted per row,
 *                  with the diagonal stored.  A system with rows must store entries.
 *   val            FP64 values.
 *   block_size     device int32 [n_sys], each 1..max_block_size (<= 64).
 *   b, x           device [n_rows]; x is overwritten (x0 = 0).
 * All arrays are caller-owned device memory and must stay valid while a handle that was
 * created from them is used.  A system with zero rows is reported converged. */
typedef struct {
  int32_t n_sys;
  int64_t n_rows;           /* total rows */
  int64_t nnz;              /* total nnz  */
  const int64_t *sys_row;   /* device [n_sys+1] */
  const int32_t *row_ptr;   /* device [n_rows+1] */
  const int32_t *col_idx;   /* device [nnz], local */
  const double *val;        /* device [nnz] */
  const int32_t *block_size;/* device [n_sys] */
  int32_t max_block_size;   /* host: max over block_size (<= 64) */
} pc_batch;

typedef struct pc_batch_handle pc_batch_handle;

/* pc_batch_create - validate the batch (an O(nnz) device pass: row pointers
 * non-decreasing, local columns inside their system, strictly increasing within each row,
 * diagonal stored), schedule the teams and allocate the
 * library-owned workspace (4 FP64 vectors of n_rows, the M^{-1} factors, team counters).
 * prec: PC_PREC_FP64, or PC_PREC_FP32 / PC_PREC_TF32 (FP32 factors applied in FP32, FP64
 * CG).  pivot_tol: a Cholesky pivot <= pivot_tol * (largest diagonal entry of its block)
 * marks the system not SPD.  Synchronises the stream.  Errors: PC_ERR_INVALID_ARG
 * (arguments or CSR structure), PC_ERR_OOM, PC_ERR_CUDA. */
pc_status pc_batch_create(const pc_batch *B, int32_t prec, double pivot_tol, void *stream,
                          pc_batch_handle **out);

/* pc_batch_solve - setup + PCG for every system in one launch (graph replay when b, x,
 * tol and max_iter match the previous call, else a new capture).  max_iter bounds each
 * system's CG iterations; up to 3 restarts from the true residual.
 * Outputs (device arrays, each may be NULL): iters, status (pc_status values) int32
 * [n_sys]; relres double [n_sys] = ||b_s - A_s x_s|| / ||b_s|| (0 for b_s = 0, -1 when
 * not computed).  info (host, may be NULL): status = first non-OK system status (or
 * PC_ERR_TIMEOUT), failed_block = the index of that SYSTEM, iterations = max over
 * systems, true_rel_residual = worst system, solve_ms = device time of the launch,
 * grid_ctas = persistent grid size, reserved = 1 if the launch went through the graph.
 * Synchronises the stream. */
pc_status pc_batch_solve(pc_batch_handle *h, const double *b, double *x, double tol,
                         int32_t max_iter, int32_t *iters, int32_t *status, double *relres,
                         pc_solve_info *info, void *stream);

pc_status pc_batch_destroy(pc_batch_handle *h);

/* Launch shape of a handle, host out[]: grid CTAs, CTAs per SM, queue slots, team limit,
 * dynamic shared memory, setup warps per CTA, graph captured (1/0).  Returns the count
 * written (<= max_entries). */
int32_t pc_batch_info(const pc_batch_handle *h, int32_t *out, int32_t max_entries);

/* Phase profile of a handle created with the environment variable PC_BATCH_PROFILE=1:
 * nanoseconds summed over all CTAs and over every solve since creation, per phase:
 * setup, start (x0 = 0 pass), SpMV, unit pass (r, x, z), p update, true residual,
 * reductions and team waits, queue and idle (8 entries, host out[]).  Returns the count
 * copied, 0 when profiling is off.  Synchronous. */
int32_t pc_batch_profile(const pc_batch_handle *h, uint64_t *out, int32_t max_entries);

/* Team size and first queue slot of every system (host arrays [n_sys], may be NULL).
 * Returns n_sys. */
int32_t pc_batch_teams(const pc_batch_handle *h, int32_t *team, int32_t *slot0);

/* The scheduler, host only (no GPU): team sizes, first slots and slot order for systems
 * of n_rows[s] rows, nnz[s] entries and block size block_size[s] on a grid of n_ctas
 * CTAs.  A system's cost is its bytes per CG iteration times N^(1/3) (the growth of the
 * PCG iteration count with kappa ~ N^(2/3) on 3D meshes and geometric graphs); a team
 * doubles while it stays within team_max and n_ctas, keeps >= 4 warp units per member
 * and each member keeps >= total / (slots_per_cta * n_ctas) of the cost.  Slots go to
 * larger teams first, then to longer slots.  Host arrays [n_sys]: team, slot0, order
 * (systems in slot order).  Returns the number of slots, or -1 on invalid input. */
int32_t pc_batch_schedule(int32_t n_sys, const int64_t *n_rows, const int64_t *nnz,
                          const int32_t *block_size, int32_t n_ctas, int32_t team_max,
                          double slots_per_cta, int32_t *team, int32_t *slot0, int32_t *order);

/* Tuning of handles created afterwards: CTAs per SM of the persistent grid (0 =
 * occupancy maximum), team limit (0 = 32) and slots per CTA of the scheduler (0 = 2).
 * Process-wide. */
void pc_batch_set_tuning(int32_t ctas_per_sm, int32_t team_max, double slots_per_cta);

/* Shared memory (KB) that pc_batch_create gives to setup slots: the number of warps of a
 * CTA that factor blocks concurrently is this budget over one slot (a slot holds the
 * dense A and L^{-1} tiles of one warp unit of the largest block size).  0 = 70 KB.
 * Process-wide. */
void pc_batch_set_setup_smem(int32_t kb);

/* Autotuner of the batched launch: solves the batch (setup + PCG, right-hand side b) with
 * up to max_trials candidate launch shapes (0 = all 36: CTAs per SM {occupancy maximum, 1}
 * x team limit {4, 8, 32} x slots per CTA {8, 4, 2} x setup shared memory {70, 140} KB),
 * timing the second (graph-replayed) solve of each, and records the fastest for this batch
 * signature (n_sys, n_rows, nnz, prec): later pc_batch_create calls on a matching batch use
 * it unless explicit tuning was set.  Allocates a scratch x.  best_ms (host, may be NULL):
 * its solve time; best_cfg (host int32 [4], may be NULL): CTAs per SM (0 = maximum), team
 * limit, slots per CTA x 1000, setup KB.  Synchronous. */
pc_status pc_batch_autotune(const pc_batch *B, int32_t prec, const double *b, double tol,
                            int32_t max_iter, int32_t max_trials, void *stream, double *best_ms,
                            int32_t *best_cfg);

/* Forget every autotuned launch shape. */
void pc_batch_clear_tuned(void);

/* One-shot form: pc_batch_create (pivot_tol 0) + pc_batch_solve + pc_batch_destroy. */
pc_status pcg_solve_batched(const pc_batch *B, const double *b, double *x, double tol,
                            int32_t max_iter, int32_t prec, int32_t *iters, int32_t *status,
                            double *relres, pc_solve_info *info, void *stream);

/* ---------------------------------------------------------------------------------
 * Library options and diagnostics. */

/* Cycle budget of every bounded device-side wait (grid barrier spin).  <= 0 restores the
 * default (about 4e9 cycles).  Process-wide; not thread-safe against concurrent calls. */
void pc_set_wait_budget(int64_t cycles);

/* Number of CTAs per SM used by the persistent CG kernel (0 = occupancy maximum). */
void pc_set_ctas_per_sm(int32_t ctas);

/* CG engine of pcg_solve / pcg_solve_h: 0 = CUDA-graph loop (a device-driven `while`
 * conditional node over three full-occupancy kernels per iteration; the default),
 * 1 = one persistent cooperative kernel with grid-wide barriers.  Both compute the same
 * recurrences; reductions are fixed-order in each.  Any other value restores the default
 * (or the PC_CG_ENGINE environment variable: "graph" / "persistent"). */
void pc_set_cg_engine(int32_t engine);

/* Row order of the graph engine's CG SpMV (one row per lane, every lane running to the
 * longest row of its warp).  Mode -1 (default): on the first solve of a handle, measure the
 * FP64 operations that order would spend (sum over 32-row groups of 32 x the longest row)
 * and, if they exceed 1.25 x nnz (irregular row lengths, e.g. power-law rows), sort the rows
 * by length inside windows of 2048 rows (a stable, deterministic counting sort; 4 bytes per
 * row of workspace).  0: natural order always; 1: binned always.  Applies to handles that
 * have not solved yet.  Process-wide. */
void pc_set_row_binning(int32_t mode);

/* 1 if the handle's CG SpMV uses the binned row order, else 0. */
int32_t pc_handle_row_binned(const pc_handle *h);

/* Column segments of the binned CG SpMV.  The binned SpMV sweeps its rows once per segment
 * of columns [s * ceil(n/S), (s+1) * ceil(n/S)), each sweep gathering only that part of x
 * (so that it stays in L2 while the matrix streams), and adds the sweeps' partial sums in
 * order.  segs -1 (default): S = 1 (on an 8M-row power-law matrix every S > 1 measured
 * slower: the extra sweeps cost more dependent load rounds than the L2 hits save); 1..8:
 * exactly that many.
 * Workspace: 4 (S + 1) bytes per row, plus 8 per row when S > 1.  Segments need sorted
 * column indices; a matrix whose rows are not strictly increasing is swept whole (S = 1).
 * Applies to binned handles that have not solved yet.  Process-wide. */
void pc_set_col_segments(int32_t segs);

/* Column segments of the handle's binned CG SpMV (1 if unsegmented or not binned). */
int32_t pc_handle_col_segments(const pc_handle *h);

/* Launch shape of the graph engine's CG loop kernels (the paper fixes none; these are
 * implementation choices that change speed, and results only through the order of the
 * per-CTA partial sums).  0 in a field: the library default. */
typedef struct {
  int32_t spmv_ctas_per_sm;   /* natural-order SpMV: resident CTAs per SM, 1..8 (default 4)  */
  int32_t ring_stages;        /* warp-ring preconditioner: stages per warp, 2..4 (default:
                                 the deepest that fits 110 KB of shared memory per CTA)       */
  int32_t bin_pipe;           /* binned SpMV row loop: -1 default (2), 0 plain, 1 pipelined,
                                 2 pipelined with the groups of rows up to 64 entries read
                                 from a sliced copy built at the first solve (entry k of the
                                 group's 32 rows contiguous; 8 or 12 bytes per entry of those
                                 rows, padded to each group's longest row); with column
                                 segments 2 runs as 1.  Natural row order: 2 walks a sliced
                                 copy of all rows (groups of 32 consecutive rows; only when no
                                 row exceeds 64 entries), any other value the CSR (default)   */
  int32_t fuse_update;        /* x += alpha p and p = z + beta p: 0 default (1 with FP64
                                 factors, 2 otherwise), 1 fused into the warp-ring
                                 preconditioner kernel (x updated unit by unit as it goes; p
                                 after its CTAs have waited, under the wait budget, for its
                                 last CTA's beta; one cooperative launch), 2 a separate
                                 kernel.  Fused only where the preconditioner is the warp-ring
                                 kernel (block sizes up to 32); pc_handle_shape reports 1 or
                                 2, what the graph runs                                       */
  double us_per_iteration;    /* time per CG iteration measured for this shape (0: none)     */
} pc_shape;

/* pc_autotune - kernel-shape autotuner of the single-system solve.  Sets up a handle for A
 * (block_size, prec), then for each candidate shape (natural row order: SpMV CTAs per SM
 * {2, 3, 4, 6, 8} x ring stages {2, 3, 4}; binned: row loop {plain, pipelined, sliced} x ring stages;
 * each with the default update; then the best of them with the other update, fused or a
 * separate kernel, and in natural order with the other row walk, CSR or sliced copy, each
 * kept only when at least 1% faster)
 * runs `iterations` CG iterations twice (right-hand side of ones, tolerance 0) and times the
 * second run with CUDA events; max_trials > 0 caps the candidates before that last trial.  The fastest shape is
 * recorded for A's key (block size, precision, ceil(log2 n), round(log2(nnz / n)), SM count
 * of the current device); handles with that key use it when they build their loop graph (at
 * their first solve), and when the environment variable PC_TUNE_CACHE names a file it is
 * saved there.  best (HOST, may be NULL) receives the shape with its time per iteration.
 * Allocates and frees its own buffers; synchronises the stream.  1 <= iterations <= 10000. */
pc_status pc_autotune(const pc_csr *A, int32_t block_size, int32_t prec, int32_t iterations,
                      int32_t max_trials, void *stream, pc_shape *best);

/* Records (pc_tune_set) or looks up (pc_tune_get: 1 if found, 0 if not) the shape for the key
 * of a system with n rows, nnz entries, this block size and precision on the current device.
 * Host-only (no device work; with no device the SM count of the key is 0).  pc_tune_set
 * returns PC_ERR_INVALID_ARG for a field outside its range. */
pc_status pc_tune_set(int32_t block_size, int32_t prec, int64_t n, int64_t nnz, const pc_shape *shape);
int32_t pc_tune_get(int32_t block_size, int32_t prec, int64_t n, int64_t nnz, pc_shape *shape);

/* Forgets every recorded shape, single-system and batched (a file named by PC_TUNE_CACHE is
 * not read again until pc_tune_load). */
void pc_tune_clear(void);

/* Cache file of the recorded shapes: one flat JSON object per line, "kind" "cg" (the key and
 * pc_shape fields) or "batch" (the batch signature of pc_batch_autotune and its launch
 * shape).  pc_tune_save writes every recorded shape (through a temporary file renamed into
 * place); pc_tune_load merges a file into the table, skipping lines that do not parse, and
 * reports the entries taken in *entries (HOST, may be NULL).  PC_ERR_INVALID_ARG when the
 * file cannot be written or opened.  The file named by PC_TUNE_CACHE is loaded once per
 * process at the first lookup.  Host-only. */
pc_status pc_tune_save(const char *path);
pc_status pc_tune_load(const char *path, int32_t *entries);

/* The launch shape h's loop graph was built with (after its first solve with the graph engine;
 * PC_ERR_INVALID_ARG before).  us_per_iteration is that of the recorded shape, if any. */
pc_status pc_handle_shape(const pc_handle *h, pc_shape *out);

/* Phase trace of the last pcg_solve_h on h, when the environment variable
 * PC_TRACE_BARRIERS=N (N > 0) was set for that solve: out[0] is the device globaltimer (ns)
 * at kernel start and out[k] the time after the k-th grid-wide synchronisation (entries
 * never reached are 0).  Copies at most max_entries values to the HOST array out and
 * returns how many were copied (0 if tracing was off).  Synchronous.
 * With the graph engine and PC_CG_PROFILE=1 (the loop body kernels are then launched one by
 * one from the host, with events around each) it returns 3 entries instead: the mean
 * nanoseconds per iteration of the SpMV, preconditioner and vector-update kernels. */
int32_t pc_get_trace(const pc_handle *h, int64_t *out, int32_t max_entries);

/* Static description of a status code. */
const char *pc_status_string(int32_t status);

/* Library version (major * 10000 + minor * 100 + patch). */
int32_t pc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PC_H_ */

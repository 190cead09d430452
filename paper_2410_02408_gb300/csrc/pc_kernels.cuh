// Kernel argument structs and host-side launchers shared between the libpc translation
// units (internal; the public interface is include/pc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pc_common.cuh"

namespace pc {

struct SetupArgs {
  Layout lay;
  const int32_t* row_ptr;
  const int32_t* col;
  const void* val;
  double tol;
  void* minv;                     // unit layout, FT
  void* linv;                     // unit layout, FT
  unsigned long long* failed;     // min failing block index (init: all ones)
};

struct PcgOut {
  int32_t status;
  int32_t iterations;
  int32_t restarts;
  int32_t pad;
  double rel_residual;
  double true_rel_residual;
};

// Shared-memory plan of the persistent CG kernel (identical on host and device).
constexpr int PCG_BLOCK = 256;    // threads per CTA
constexpr int PCG_NW = PCG_BLOCK / 32;
constexpr int PCG_NSTW = 2;       // pipeline stages per warp
constexpr int PCG_TCAP = 512;     // SpMV chunk table capacity (entries)
constexpr int PCG_WSTAGE = 3328;  // bytes per warp stage
constexpr int PCG_CHUNK = 32;     // rows per SpMV chunk (one row per lane)

struct PcgSmem {
  int wstage;      // bytes per warp stage
  int off_col;     // column window offset in an SpMV stage (after the row-pointer window)
  int off_val;     // value window offset
  int tnnz;        // entries an SpMV stage holds
  int fac_smem;    // 1 if one warp unit of M^{-1} fits a stage
  int total;       // dynamic shared memory bytes
};

__host__ __device__ inline PcgSmem pcg_smem_plan(int val_bytes, int64_t unit_bytes) {
  PcgSmem p;
  p.wstage = PCG_WSTAGE;
  p.off_col = 176;                                  // row-pointer window: <= 33*4 + 32 bytes
  int t = (PCG_WSTAGE - p.off_col - 32 - 32 - 16) / (4 + val_bytes);
  t &= ~7;
  p.tnnz = t;                                        // col window <= 4t+32, value window <= vb*t+32
  p.off_val = (p.off_col + t * 4 + 32 + 15) & ~15;
  p.fac_smem = unit_bytes <= PCG_WSTAGE ? 1 : 0;
  p.total = 256 + PCG_TCAP * 4 + PCG_NW * PCG_NSTW * PCG_WSTAGE;
  return p;
}

struct PcgArgs {
  Layout lay;
  int64_t nnz;
  int32_t tr;            // rows per SpMV tile
  int32_t pad0;
  PcgSmem sp;
  const int32_t* rp;
  const int32_t* ci;
  const void* va;
  const void* minv;
  const double* b;
  double* x;
  double* r;
  double* z;
  double* p;
  double* q;
  double* part;          // 2 * gridDim * 2 doubles (double-buffered per-CTA partials)
  const int64_t* split;  // gridDim + 1 SpMV row boundaries
  GridSync* gs;
  PcgOut* out;
  double tol;
  int32_t max_iter;
  int32_t max_restarts;
  long long budget;
  unsigned long long* trace;   // optional: globaltimer (ns) at kernel start and after each grid barrier
  int32_t trace_len;           // entries available in trace
  int32_t pad1;
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// pc_setup.cu
cudaError_t launch_setup(const SetupArgs& a, bool val_f32, bool fac_f32, cudaStream_t st);
// PC_PREC_TF32: FP32 factorisation, M^{-1} formed on the tensor cores (TF32 operands, FP32 accumulation).
cudaError_t launch_setup_tf32(const SetupArgs& a, bool val_f32, cudaStream_t st);
cudaError_t launch_extract(int64_t n, const int32_t* rp, const int32_t* ci, const void* va, bool val_f32,
                           int32_t bs, double* out, cudaStream_t st);
cudaError_t launch_get_factor(const Layout& L, const void* fac, bool fac_f32, int which, double* out,
                              cudaStream_t st);

// pc_ops.cu
// CSR structure check (sets *flags to the OR of the CSR_BAD_* bits found; 0 = valid).
constexpr unsigned CSR_BAD_ROW_PTR = 1u;   // row_ptr[0] != 0, row_ptr[n] != nnz, or a row range outside [0, nnz]
constexpr unsigned CSR_BAD_COLUMN = 2u;    // a column index outside [0, n)
constexpr unsigned CSR_BAD_ORDER = 4u;     // columns of a row not strictly increasing
constexpr unsigned CSR_NO_DIAGONAL = 8u;   // a row without its diagonal entry
cudaError_t launch_validate_csr(int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci, unsigned* flags,
                                cudaStream_t st);
// D (16x8) = A (16x8) B (8x8), row-major, on the tensor cores with TF32 operands (one warp)
cudaError_t launch_mma_tf32_check(const float* A, const float* B, float* D, cudaStream_t st);
// out_f[i] = d2f(in_d[i]), out_d[i] = f2d(in_f[i]) (the conversions of pc_common.cuh)
cudaError_t launch_convert(int64_t n, const double* in_d, float* out_f, const float* in_f, double* out_d,
                           cudaStream_t st);
cudaError_t launch_spmv(int64_t n, const int32_t* rp, const int32_t* ci, const void* va, bool val_f32,
                        const double* x, double* y, cudaStream_t st);
cudaError_t launch_dot(int64_t n, const double* x, const double* y, double* result, double* part,
                       cudaStream_t st);
int dot_partials();
cudaError_t launch_apply(const Layout& L, const void* fac, bool fac_f32, int mode, const double* in,
                         double* out, cudaStream_t st);
// d = r - blockdiag(A) z (FP64, the diagonal blocks of the partition read from the CSR); z += e.
cudaError_t launch_block_residual(int64_t n, int32_t bs, const int32_t* rp, const int32_t* ci, const void* va,
                                  bool val_f32, const double* r, const double* z, double* d, cudaStream_t st);
cudaError_t launch_add(int64_t n, const double* e, double* z, cudaStream_t st);
// out = L^{-1} (A t) (+ optional Lanczos epilogue, see pc_ops.cu)
struct SymPhase2Args {
  Layout lay;
  const int32_t* rp;
  const int32_t* ci;
  const void* va;
  const void* linv;
  const double* t;      // L^{-T} v
  double* out;
  // Lanczos epilogue (q_prev == nullptr: none)
  const double* q_cur;
  const double* q_prev;
  const double* beta;   // device scalar array, beta[j-1] used
  int32_t j;
  double* part;         // per-CTA partial of q_cur . out
  unsigned* counter;
  double* alpha_out;    // alpha[j]
  const int* done;
};
cudaError_t launch_sym_phase2(const SymPhase2Args& a, bool val_f32, bool fac_f32, int grid, cudaStream_t st);
cudaError_t launch_split(int64_t n, int64_t nnz, const int32_t* rp, int parts, int64_t* split, cudaStream_t st);
cudaError_t launch_grad_val(int64_t n, const int32_t* rp, const int32_t* ci, const double* lam, const double* x,
                            double* g, cudaStream_t st);
cudaError_t launch_grad_edges(int64_t n_edges, const int32_t* ep, const int32_t* eq, const double* lam,
                              const double* x, int64_t n, double* g, cudaStream_t st);

// pc_api.cu: settings of the persistent engine (wait budget in cycles; grid for a matrix).
long long wait_budget_cycles();
cudaError_t persistent_grid(const Layout& L, int64_t nnz, bool val_f32, bool fac_f32, int* grid);
// pc_setup.cu: FP64 arithmetic with FP32 stored factors (fallback of the FP32 setup).
cudaError_t launch_setup_f64_store_f32(const SetupArgs& a, bool val_f32, cudaStream_t st);

// pc_pcg_*.cu
cudaError_t launch_pcg(const PcgArgs& a, bool val_f32, bool fac_f32, int grid, int block, cudaStream_t st);
cudaError_t pcg_occupancy(const Layout& L, bool val_f32, bool fac_f32, int block, int smem, int* ctas_per_sm);
// Fill the launch plan fields of a (nnz, tr, sp) for this matrix and factor precision.
void pcg_plan(PcgArgs& a, int64_t nnz, bool val_f32, bool fac_f32);

// pc_cg_graph.cu
struct CgResult {
  int32_t status, iterations, restarts, pad;
  double rel_residual, true_rel_residual;
  double kernel_us[3];   // profiling mode: mean time of the SpMV, preconditioner and update kernels
};
int cg_graph_partials();
size_t cg_scalars_bytes();
// Binned SpMV order of the graph engine (built by pc_rowbin.cu).
struct CgBinned {
  const int32_t* perm;     // [n] the row at each binned position
  const int32_t* gsplit;   // [n_warps + 1] each SpMV warp's first work item (runs of about equal cost)
  const int32_t* items;    // [m_items] work items: group g (>= 0) or the row at position -(v + 1)
  const int32_t* gmax;     // [ceil(n/32)] longest row of each group (selects the lanes per row)
  const int32_t* bnd;      // [(nseg + 1) * bstride] entry boundaries of the column segments, by position
  int64_t bstride;
  double* spart;           // [n] partial sums between segment sweeps (nseg > 1), by position
  int32_t nseg;            // column segments swept one after another (1: whole rows)
  int32_t pipe;            // 1: pipelined row loop (gsplit sized for cg_spmv_bin_warps(true))
  // Sliced copy of the one-lane-per-row groups (null: none; used with nseg 1 and the
  // pipelined loop): group g (gmax[g] <= BIN_SLICED_LANE_ROWS) holds 32 * gmax[g] entries ending at
  // sincl[g], entry k of the row at position 32 g + l at 32 k + l, padded past the row's end.
  // With perm null (natural order) the groups are 32 consecutive rows, each with its slab.
  const int32_t* scol;
  const void* sval;        // VT, as the CSR values
  const int64_t* sincl;    // [ceil(n/32)] inclusive prefix of the slab sizes
};
// bin: null (or bin->perm null) for the natural row order.
// Launch shape of the graph engine's loop kernels (0: the default of each field).
struct CgShape {
  int32_t spmv_ctas_per_sm;   // natural-order SpMV: resident CTAs per SM (1..8; default 4)
  int32_t ring_stages;        // warp-ring preconditioner: stages per warp (2..4; default the deepest that fits)
  int32_t fuse_update;        // 0 default (fused where possible), 1 fused, 2 separate update kernel
};
cudaError_t cg_graph_create(void** out, const Layout& L, const int32_t* rp, const int32_t* ci, const void* va,
                            bool val_f32, const void* minv, bool fac_f32, const double* b, double* x, double* r,
                            double* z, double* p, double* q, double* part, void* scal, const CgBinned* bin,
                            const CgShape& shape, cudaStream_t st);
// True if the loop graph runs the x / p update as the tail of the preconditioner kernel.
bool cg_graph_fused(const void* g);

// Row binning (pc_rowbin.cu): rows sorted by length inside windows of ROWBIN_W rows.
constexpr int ROWBIN_W = 2048;
// Longest row of a 32-row group that the binned SpMV walks one lane per row: 64 over the CSR,
// 256 over the sliced copy (whose loads stay coalesced and whose rounds are pipelined, so a
// longer group costs rounds, not scattered loads); longer groups take 8 lanes per row (CSR
// walk, up to 256) or are split into single-row items (above 256).
constexpr int BIN_LANE_ROWS = 64;
constexpr int BIN_SLICED_LANE_ROWS = 256;
// d_out[0] += sum over 32-row groups of 32 * (longest row in the group).
cudaError_t row_bin_waste(int64_t n, const int32_t* rp, unsigned long long* d_out, cudaStream_t st);
// perm[n]: the rows of every window, stably sorted by length bucket.
cudaError_t row_bin_build(int64_t n, const int32_t* rp, int32_t* perm, cudaStream_t st);
// Work items of the binned SpMV (see pc_rowbin.cu): whole 32-row groups, and the single rows of
// groups whose longest row exceeds 256 entries.  Step 1: per group its longest row (gmax
// [ceil(n/32)]), the cost of the whole-group item (gcost) and the inclusive prefix of the item
// counts (gcount_incl, int64 [ceil(n/32)]; its last entry is the number of items).  Step 2: the
// items (items [m_items]: g >= 0 for group g, -(pos + 1) for the row at binned position pos), their
// cost prefix (icost, int64 [m_items]) and each warp's first item (isplit [n_warps + 1]).
// scan_ws: scratch of ceil(m / 8192) int64 for the prefix sums over m entries (m: groups or
// items).
cudaError_t row_bin_group_stats(int64_t n, const int32_t* rp, const int32_t* perm, int64_t* gcost, int32_t* gmax,
                                int64_t* gcount_incl, int lane_max, int64_t* scan_ws, cudaStream_t st);
cudaError_t row_bin_items(int64_t n, const int32_t* rp, const int32_t* perm, const int32_t* gmax, const int64_t* gcost,
                          const int64_t* gcount_incl, int64_t m_items, int n_warps, int32_t* items, int64_t* icost,
                          int32_t* isplit, int64_t* scan_ws, cudaStream_t st);
// Column segments of the binned SpMV: for the row at binned position idx, bnd[s * stride + idx]
// is its first entry (s = 0), one past its last entry (s = nseg), or its first entry with
// column >= s * seg_cols (0 < s < nseg; columns sorted within the row).  *unsorted (device
// int, zeroed by the caller) is set when some row's columns are not strictly increasing.
cudaError_t row_seg_bounds(int64_t n, const int32_t* rp, const int32_t* ci, const int32_t* perm, int nseg,
                           int64_t seg_cols, int64_t stride, int32_t* bnd, int* unsorted, cudaStream_t st);
// Sliced copy of the one-lane-per-row groups (CgBinned::scol): step 1 writes the inclusive
// prefix of the slab sizes (32 * gmax[g] entries for gmax[g] <= lane_max, else 0) to sincl
// [ceil(n/32)]; step 2 fills scol / sval (sincl's last entry of each, VT = float when
// val_f32) from the whole-row bounds bnd (nseg 1): padding entries get column 0 and value 0.
cudaError_t row_sliced_sizes(int64_t n, const int32_t* gmax, int64_t* sincl, int lane_max, int64_t* scan_ws,
                             cudaStream_t st);
// Natural order: gmax[g] = the longest of rows 32 g .. 32 g + 31, and *dmax (device int,
// zeroed by the caller) their maximum.  The fill then takes bnd = rp, stride = 1.
cudaError_t row_natural_gmax(int64_t n, const int32_t* rp, int32_t* gmax, int* dmax, cudaStream_t st);
cudaError_t row_sliced_fill(int64_t n, const int32_t* bnd, int64_t stride, const int32_t* ci, const void* va,
                            bool val_f32, const int32_t* gmax, const int64_t* sincl, int lane_max, int32_t* scol,
                            void* sval, cudaStream_t st);
// Warps of the binned SpMV grid (the number of work items of its split), plain or pipelined.
int cg_spmv_bin_warps(bool pipe);
void cg_graph_destroy(void* g);
cudaError_t cg_graph_round(void* g, bool val_f32, bool fac_f32, cudaStream_t st);
cudaError_t cg_graph_solve(void* g, double tol, int max_iter, int max_restarts, bool val_f32, bool fac_f32,
                           cudaStream_t st, CgResult* res);

// pc_lanczos.cu
struct LanczosState {
  int64_t n;
  int32_t m;
  double tol;
  double* V;          // m * n
  double* w;          // n
  double* t;          // n (L^{-T} q_j)
  double* alpha;      // m
  double* beta;       // m
  double* coef;       // 2 * m
  double* part;       // grid * m
  unsigned* counter;  // 1
  int* ctl;           // [0] done, [1] steps
  double* tnorm;      // 1
  double* result;     // [0] theta_min [1] theta_max
};
cudaError_t lanczos_init(const LanczosState& s, const double* v0, bool precond, const Layout& L, const void* linv,
                         bool fac_f32, cudaStream_t st);
cudaError_t lanczos_step(const LanczosState& s, int j, int reorth, bool precond, const Layout& L,
                         const int32_t* rp, const int32_t* ci, const void* va, bool val_f32, const void* linv,
                         bool fac_f32, cudaStream_t st);
cudaError_t lanczos_finish(const LanczosState& s, cudaStream_t st);
cudaError_t lanczos_configure(int m);
int lanczos_grid();

}  // namespace pc

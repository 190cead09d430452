// Host side of the libpc C ABI (include/pc.h): argument checks, handle and workspace
// management, kernel dispatch and status reporting.  No call prints, aborts or traps.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pc.h"
#include "pc_kernels.cuh"
#include "pc_tune.h"

using pc::Layout;

struct pc_handle {
  pc_csr A;
  int32_t bs;
  int32_t prec;
  double tol;
  Layout L;
  bool val_f32;
  bool fac_f32;
  void* minv;
  void* linv;
  double* tmp;
  unsigned long long* failed_d;
  int64_t failed_block;
  int refactored_fp64;   // FP32 factors recomputed in FP64 arithmetic after an FP32 breakdown
  // CG workspace (allocated on first solve)
  double* cg;            // r, z, p, q: 4 n
  double* part;          // grid * 2
  int64_t* split;        // grid + 1
  unsigned char* ctl;    // GridSync + PcgOut
  int grid;
  int block;
  unsigned long long* trace_d;   // optional barrier trace (PC_TRACE_BARRIERS)
  int trace_len;
  // graph engine
  void* graph;           // instantiated loop graph (pc::cg_graph_create)
  double* gbx;           // copies of b and x: 2 n
  int32_t* perm;         // SpMV row order for irregular row lengths (null: natural order)
  int32_t* gsplit;       // with perm: each SpMV warp's first work item (balanced runs)
  int32_t* items;        // with perm: work items (32-row groups, or single rows of hub-row groups)
  int32_t* gmax;         // with perm: longest row of each 32-row group
  int32_t* bnd;          // with perm: column-segment entry boundaries by binned position
  double* spart;         // with nseg > 1: partial sums between segment sweeps
  int32_t* scol;         // row loop 2: sliced copy of the one-lane-per-row groups (columns)
  void* sval;            // ... (values, as the CSR's)
  int64_t* sincl;        // ... (inclusive prefix of the slab sizes, per group)
  int32_t nseg;          // column segments of the binned SpMV
  int32_t bin_pipe;      // row loop of the binned SpMV: 0 plain, 1 pipelined, 2 pipelined + sliced
  int perm_checked;      // the row-length statistics have been taken
  double* gpart;         // per-CTA partials
  void* gscal;           // CG scalars
  int64_t prof_ns[3];    // graph engine, profiling mode: mean ns per iteration of the 3 kernels
  int prof_valid;
  // launch shape of the loop graph: forced (autotuner trials), else the tuned table, else defaults
  double* ref_ws;        // pc_apply_tol: residual, correction, dot partials and results
  int shape_forced;
  pc_shape shape_force;
  pc_shape shape_used;   // valid once the graph exists
};

namespace {

long long g_budget = 0;          // 0 = default
int g_ctas_per_sm = 0;           // 0 = occupancy maximum
int g_engine = -1;               // -1: from PC_CG_ENGINE (default graph); 0 graph; 1 persistent
int g_row_binning = -1;          // -1: decided per matrix; 0 off; 1 on
int g_col_segments = -1;         // -1: default (1); 1..8 forced

int cg_engine() {
  if (g_engine >= 0) return g_engine;
  const char* e = getenv("PC_CG_ENGINE");
  if (e && strcmp(e, "persistent") == 0) return 1;
  return 0;
}
const long long kDefaultBudget = 4000000000LL;

long long wait_budget() {
  if (g_budget > 0) return g_budget;
  const char* e = getenv("PC_WAIT_BUDGET");
  if (e) {
    long long v = atoll(e);
    if (v > 0) return v;
  }
  return kDefaultBudget;
}

// NVTX range around an entry point (visible in profilers that collect NVTX; the header-only
// NVTX library does nothing when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

pc_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return PC_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA;
}

#define PC_TRY(expr)                         \
  do {                                       \
    cudaError_t _e = (expr);                 \
    if (_e != cudaSuccess) return from_cuda(_e); \
  } while (0)

// Device memory of the single-system handles comes from a memory pool of this library, one
// per device, that keeps freed memory for later allocations instead of returning it to the
// driver: a handle per solve (the one-call API) then costs no page mapping and unmapping
// (3.2 ms of destroy alone on an 8M-row matrix with raw cudaMalloc / cudaFree).  The
// semantics stay those of cudaMalloc / cudaFree: dalloc returns memory ready for any stream
// (its stream-ordered allocation, on a private stream, is synchronized), dfree first waits
// for the device (as cudaFree does) so that no kernel still reads the memory.  An allocation
// that fails trims the pool's cached memory and tries once more.  Without pool support the
// raw calls are used.
struct LibPool {
  cudaMemPool_t pool = nullptr;
  cudaStream_t stream = nullptr;
  bool tried = false;   // creation attempted (once per device)
  bool ok = false;      // pool and stream usable
};
constexpr int kMaxDevices = 64;
LibPool g_pools[kMaxDevices];
std::mutex g_pool_mu;

LibPool* lib_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  LibPool& lp = g_pools[dev];
  if (!lp.tried) {
    lp.tried = true;
    int supported = 0;
    cudaDeviceGetAttribute(&supported, cudaDevAttrMemoryPoolsSupported, dev);
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaError_t e = supported ? cudaMemPoolCreate(&lp.pool, &props) : cudaErrorNotSupported;
    if (e == cudaSuccess) {
      uint64_t keep = UINT64_MAX;   // freed memory stays in the pool
      e = cudaMemPoolSetAttribute(lp.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&lp.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      cudaGetLastError();   // raw allocations from now on
      return nullptr;
    }
    lp.ok = true;
  }
  return lp.ok ? &lp : nullptr;
}

template <typename T>
pc_status dalloc(T** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  LibPool* lp = lib_pool();
  cudaError_t e;
  if (lp) {
    e = cudaMallocFromPoolAsync((void**)p, bytes, lp->pool, lp->stream);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      cudaStreamSynchronize(lp->stream);
      cudaMemPoolTrimTo(lp->pool, 0);
      e = cudaMallocFromPoolAsync((void**)p, bytes, lp->pool, lp->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(lp->stream);
  } else {
    e = cudaMalloc((void**)p, bytes);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA;
  }
  return PC_OK;
}

void dfree(void* p) {
  if (!p) return;
  LibPool* lp = lib_pool();
  if (lp) {
    cudaDeviceSynchronize();
    cudaFreeAsync(p, lp->stream);
  } else {
    cudaFree(p);
  }
}

bool csr_ok(const pc_csr* A) {
  if (!A) return false;
  if (A->n <= 0 || A->n >= (int64_t)INT32_MAX || A->nnz < 0 || A->nnz >= (int64_t)INT32_MAX) return false;
  if (!A->row_ptr || !A->col_idx || (A->nnz > 0 && !A->val)) return false;
  if (A->dtype != PC_F64 && A->dtype != PC_F32) return false;
  return true;
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Element stride of the CG work vectors inside one allocation: a multiple of 32 doubles, so
// that every vector (and every 16-byte row window a bulk copy reads) starts 16-byte aligned
// whatever n is.  The allocation is 4 strides + 64 doubles of padding (bulk copies of the
// last rows round their size up to 16 bytes).
int64_t vec_stride(int64_t n) { return (n + 31) & ~(int64_t)31; }

// Per-device scratch for pc_dot.
std::mutex g_mu;
double* g_dot_scratch[64] = {nullptr};

// Per-device result word of the CSR structure check for calls without a handle; the mutex is
// held from the check's launch until its result has been read.
std::mutex g_check_mu;
unsigned* g_check_word[64] = {nullptr};

// O(nnz) structure check of A on the device (row_ptr[0] = 0, non-decreasing row ranges inside
// [0, nnz], row_ptr[n] = nnz, columns in [0, n), strictly increasing within each row, diagonal
// stored).  word: one device unsigned.  Synchronises the stream; *flags (may be null) receives
// the pc::CSR_BAD_* bits found.
pc_status check_csr_with(const pc_csr* A, unsigned* word, cudaStream_t st, unsigned* flags) {
  unsigned f = 0u;
  cudaError_t e = pc::launch_validate_csr(A->n, A->nnz, A->row_ptr, A->col_idx, word, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&f, word, sizeof(f), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return from_cuda(e);
  if (flags) *flags = f;
  return f ? PC_ERR_INVALID_ARG : PC_OK;
}

pc_status check_csr(const pc_csr* A, cudaStream_t st, unsigned* flags) {
  int dev = 0;
  PC_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return PC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_check_mu);
  if (!g_check_word[dev]) {
    pc_status s = dalloc(&g_check_word[dev], 256);
    if (s != PC_OK) return s;
  }
  return check_csr_with(A, g_check_word[dev], st, flags);
}

}  // namespace

namespace pc {
// Settings shared with the allocation-free solve (pc_static.cu), so that it runs the persistent
// engine with the same grid and wait budget as pcg_solve_h.
long long wait_budget_cycles() { return wait_budget(); }

// Grid of the persistent CG kernel for this matrix: resident CTAs per SM (capped by
// pc_set_ctas_per_sm) times the SM count, at most one CTA per 8 warp units.
cudaError_t persistent_grid(const Layout& L, int64_t nnz, bool val_f32, bool fac_f32, int* grid) {
  PcgArgs plan;
  plan.lay = L;
  pcg_plan(plan, nnz, val_f32, fac_f32);
  int per_sm = 0;
  cudaError_t e = pcg_occupancy(L, val_f32, fac_f32, PCG_BLOCK, plan.sp.total, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (g_ctas_per_sm > 0 && g_ctas_per_sm < per_sm) per_sm = g_ctas_per_sm;
  int g = per_sm * sm_count();
  const int64_t max_useful = (L.n_units + 7) / 8;   // at least 8 warp units per CTA
  if (g > max_useful) g = (int)(max_useful > 0 ? max_useful : 1);
  *grid = g;
  return cudaSuccess;
}
}  // namespace pc

extern "C" {

int32_t pc_version(void) { return 100; }

void pc_set_wait_budget(int64_t cycles) { g_budget = cycles > 0 ? (long long)cycles : 0; }

void pc_set_ctas_per_sm(int32_t ctas) { g_ctas_per_sm = ctas > 0 ? ctas : 0; }

void pc_set_cg_engine(int32_t engine) { g_engine = (engine == 0 || engine == 1) ? engine : -1; }

void pc_set_row_binning(int32_t mode) { g_row_binning = (mode == 0 || mode == 1) ? mode : -1; }

int32_t pc_handle_row_binned(const pc_handle* h) { return h && h->perm ? 1 : 0; }

void pc_set_col_segments(int32_t segs) { g_col_segments = (segs >= 1 && segs <= 8) ? segs : -1; }

int32_t pc_handle_col_segments(const pc_handle* h) { return h && h->perm ? h->nseg : 1; }

const char* pc_status_string(int32_t s) {
  switch (s) {
    case PC_OK: return "ok";
    case PC_ERR_INVALID_ARG: return "invalid argument";
    case PC_ERR_NOT_SPD: return "diagonal block is not SPD (Cholesky pivot below threshold)";
    case PC_ERR_BREAKDOWN: return "CG breakdown (non-positive or non-finite curvature)";
    case PC_ERR_NO_CONVERGENCE: return "no convergence within max_iter";
    case PC_ERR_TIMEOUT: return "bounded device-side wait timed out";
    case PC_ERR_CUDA: return "CUDA runtime error";
    case PC_ERR_OOM: return "device allocation failed";
    default: return "unknown status";
  }
}

pc_status pc_destroy(pc_handle* h) {
  if (!h) return PC_ERR_INVALID_ARG;
  dfree(h->minv);
  dfree(h->linv);
  dfree(h->tmp);
  dfree(h->failed_d);
  dfree(h->cg);
  dfree(h->part);
  dfree(h->split);
  dfree(h->ctl);
  dfree(h->trace_d);
  if (h->graph) pc::cg_graph_destroy(h->graph);
  dfree(h->gbx);
  dfree(h->perm);
  dfree(h->gsplit);
  dfree(h->items);
  dfree(h->gmax);
  dfree(h->bnd);
  dfree(h->spart);
  dfree(h->scol);
  dfree(h->sval);
  dfree(h->sincl);
  dfree(h->gpart);
  dfree(h->gscal);
  dfree(h->ref_ws);
  delete h;
  return PC_OK;
}

int32_t pc_get_trace(const pc_handle* h, int64_t* out, int32_t max_entries) {
  if (!h || !out || max_entries <= 0) return 0;
  if (h->prof_valid) {
    const int n = max_entries < 3 ? max_entries : 3;
    for (int i = 0; i < n; ++i) out[i] = h->prof_ns[i];
    return n;
  }
  if (!h->trace_d) return 0;
  const int n = max_entries < h->trace_len ? max_entries : h->trace_len;
  if (cudaMemcpy(out, h->trace_d, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int64_t pc_handle_failed_block(const pc_handle* h) { return h ? h->failed_block : -1; }

pc_status pc_csr_check(const pc_csr* A, uint32_t* flags, void* stream) {
  NvtxRange nv("pc_csr_check");
  if (flags) *flags = 0u;
  if (!csr_ok(A)) return PC_ERR_INVALID_ARG;
  unsigned f = 0u;
  const pc_status s = check_csr(A, (cudaStream_t)stream, &f);
  if (flags) *flags = f;
  return s;
}

int32_t pc_handle_refactored_fp64(const pc_handle* h) { return h ? h->refactored_fp64 : 0; }

pc_status pc_setup(const pc_csr* A, int32_t block_size, double tol, int32_t prec, void* stream, pc_handle** out) {
  NvtxRange nv("pc_setup");
  if (!out) return PC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!csr_ok(A) || block_size < 1 || block_size > 64 || !(tol >= 0.0)) return PC_ERR_INVALID_ARG;
  if (prec != PC_PREC_FP64 && prec != PC_PREC_FP32 && prec != PC_PREC_TF32) return PC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  pc_handle* h = new pc_handle();
  memset(h, 0, sizeof(*h));
  h->A = *A;
  h->bs = block_size;
  h->prec = prec;
  h->tol = tol;
  h->L = pc::make_layout(A->n, block_size);
  h->val_f32 = A->dtype == PC_F32;
  h->fac_f32 = prec != PC_PREC_FP64;
  h->failed_block = -1;
  const size_t es = h->fac_f32 ? 4 : 8;
  pc_status s = dalloc(&h->minv, es * (size_t)(h->L.n_units * pc::unit_elems_minv(h->L)));
  if (s == PC_OK) s = dalloc(&h->linv, es * (size_t)(h->L.n_units * pc::unit_elems_linv(h->L)));
  if (s == PC_OK) s = dalloc(&h->tmp, sizeof(double) * (size_t)A->n);
  if (s == PC_OK) s = dalloc(&h->failed_d, sizeof(unsigned long long));
  if (s != PC_OK) {
    pc_destroy(h);
    return s;
  }
  // the CSR structure is checked before any kernel reads it through its indices
  s = check_csr_with(A, reinterpret_cast<unsigned*>(h->failed_d), st, nullptr);
  if (s != PC_OK) {
    pc_destroy(h);
    return s;
  }
  cudaError_t e = cudaMemsetAsync(h->failed_d, 0xff, sizeof(unsigned long long), st);
  pc::SetupArgs a;
  a.lay = h->L;
  a.row_ptr = A->row_ptr;
  a.col = A->col_idx;
  a.val = A->val;
  a.tol = tol;
  a.minv = h->minv;
  a.linv = h->linv;
  a.failed = h->failed_d;
  if (e == cudaSuccess)
    e = prec == PC_PREC_TF32 ? pc::launch_setup_tf32(a, h->val_f32, st) : pc::launch_setup(a, h->val_f32, h->fac_f32, st);
  unsigned long long failed = ~0ull;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&failed, h->failed_d, sizeof(failed), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && failed != ~0ull && h->fac_f32) {
    // An FP32 pivot broke down: factor every block again in FP64 arithmetic (stored as FP32)
    // and report NOT_SPD only if that fails too.
    e = cudaMemsetAsync(h->failed_d, 0xff, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = pc::launch_setup_f64_store_f32(a, h->val_f32, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&failed, h->failed_d, sizeof(failed), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    h->refactored_fp64 = 1;
  }
  if (e != cudaSuccess) {
    pc_destroy(h);
    return from_cuda(e);
  }
  *out = h;
  if (failed != ~0ull) {
    h->failed_block = (int64_t)failed;
    return PC_ERR_NOT_SPD;
  }
  return PC_OK;
}

pc_status pc_apply(pc_handle* h, int32_t mode, const double* in, double* out, void* stream) {
  NvtxRange nv("pc_apply");
  if (!h || !in || !out || in == out) return PC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  switch (mode) {
    case PC_APPLY_INV: return from_cuda(pc::launch_apply(h->L, h->minv, h->fac_f32, 0, in, out, st));
    case PC_APPLY_LINV: return from_cuda(pc::launch_apply(h->L, h->linv, h->fac_f32, 2, in, out, st));
    case PC_APPLY_LTINV: return from_cuda(pc::launch_apply(h->L, h->linv, h->fac_f32, 3, in, out, st));
    case PC_APPLY_SYM: {
      PC_TRY(pc::launch_apply(h->L, h->linv, h->fac_f32, 3, in, h->tmp, st));
      pc::SymPhase2Args a;
      memset(&a, 0, sizeof(a));
      a.lay = h->L;
      a.rp = h->A.row_ptr;
      a.ci = h->A.col_idx;
      a.va = h->A.val;
      a.linv = h->linv;
      a.t = h->tmp;
      a.out = out;
      return from_cuda(pc::launch_sym_phase2(a, h->val_f32, h->fac_f32, 0, st));
    }
    default: return PC_ERR_INVALID_ARG;
  }
}

pc_status pc_apply_tol(pc_handle* h, int32_t mode, const double* in, double* out, double tol, int32_t* steps,
                       double* rel_residual, void* stream) {
  NvtxRange nv("pc_apply_tol");
  if (steps) *steps = 0;
  if (rel_residual) *rel_residual = -1.0;
  if (!h || !in || !out || in == out || !(tol >= 0.0) || !isfinite(tol)) return PC_ERR_INVALID_ARG;
  if (tol == 0.0) return pc_apply(h, mode, in, out, stream);
  if (mode != PC_APPLY_INV) return PC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = h->A.n;
  const int64_t vs = vec_stride(n);
  if (!h->ref_ws) {
    const pc_status sa = dalloc(&h->ref_ws, sizeof(double) * (size_t)(2 * vs + pc::dot_partials() + 8));
    if (sa != PC_OK) return sa;
  }
  double* d = h->ref_ws;
  double* e = h->ref_ws + vs;
  double* part = h->ref_ws + 2 * vs;
  double* res = part + pc::dot_partials();   // res[0] = r.r, res[1] = d.d
  PC_TRY(pc::launch_dot(n, in, in, res, part, st));
  double rr = 0.0;
  PC_TRY(cudaMemcpyAsync(&rr, res, sizeof(double), cudaMemcpyDeviceToHost, st));
  PC_TRY(pc::launch_apply(h->L, h->minv, h->fac_f32, 0, in, out, st));
  PC_TRY(cudaStreamSynchronize(st));
  if (rr == 0.0) {
    if (rel_residual) *rel_residual = 0.0;
    return PC_OK;
  }
  constexpr int kMaxSteps = 20;
  double rel = 0.0;
  int k = 0;
  for (;;) {
    // d = r - blockdiag(A) z in FP64; stop when ||d|| <= tol ||r||, else z += M^{-1} d
    PC_TRY(pc::launch_block_residual(n, h->bs, h->A.row_ptr, h->A.col_idx, h->A.val, h->val_f32, in, out, d, st));
    PC_TRY(pc::launch_dot(n, d, d, res + 1, part, st));
    double dd = 0.0;
    PC_TRY(cudaMemcpyAsync(&dd, res + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    PC_TRY(cudaStreamSynchronize(st));
    rel = sqrt(dd / rr);
    if (!(rel > tol) || k >= kMaxSteps) break;
    PC_TRY(pc::launch_apply(h->L, h->minv, h->fac_f32, 0, d, e, st));
    PC_TRY(pc::launch_add(n, e, out, st));
    ++k;
  }
  if (steps) *steps = k;
  if (rel_residual) *rel_residual = rel;
  if (!isfinite(rel)) return PC_ERR_BREAKDOWN;
  return rel <= tol ? PC_OK : PC_ERR_NO_CONVERGENCE;
}

pc_status pc_get_factor(const pc_handle* h, int32_t which, double* out, void* stream) {
  if (!h || !out || (which != 0 && which != 1)) return PC_ERR_INVALID_ARG;
  return from_cuda(pc::launch_get_factor(h->L, which == 0 ? h->linv : h->minv, h->fac_f32, which, out,
                                         (cudaStream_t)stream));
}

pc_status pc_extract_blocks(const pc_csr* A, int32_t block_size, double* out, void* stream) {
  if (!csr_ok(A) || block_size < 1 || !out) return PC_ERR_INVALID_ARG;
  const pc_status s = check_csr(A, (cudaStream_t)stream, nullptr);
  if (s != PC_OK) return s;
  return from_cuda(pc::launch_extract(A->n, A->row_ptr, A->col_idx, A->val, A->dtype == PC_F32, block_size, out,
                                      (cudaStream_t)stream));
}

pc_status pc_spmv(const pc_csr* A, const double* x, double* y, void* stream) {
  if (!csr_ok(A) || !x || !y || x == y) return PC_ERR_INVALID_ARG;
  const pc_status s = check_csr(A, (cudaStream_t)stream, nullptr);
  if (s != PC_OK) return s;
  return from_cuda(pc::launch_spmv(A->n, A->row_ptr, A->col_idx, A->val, A->dtype == PC_F32, x, y,
                                   (cudaStream_t)stream));
}

pc_status pc_debug_convert(int64_t n, const double* in_d, float* out_f, const float* in_f, double* out_d,
                           void* stream) {
  if (n < 0 || (n > 0 && (!in_d || !out_f || !in_f || !out_d))) return PC_ERR_INVALID_ARG;
  if (n == 0) return PC_OK;
  return from_cuda(pc::launch_convert(n, in_d, out_f, in_f, out_d, (cudaStream_t)stream));
}

pc_status pc_debug_mma_tf32(const float* a, const float* b, float* d, void* stream) {
  if (!a || !b || !d) return PC_ERR_INVALID_ARG;
  return from_cuda(pc::launch_mma_tf32_check(a, b, d, (cudaStream_t)stream));
}

pc_status pc_dot(int64_t n, const double* x, const double* y, double* result, void* stream) {
  if (n < 0 || !x || !y || !result) return PC_ERR_INVALID_ARG;
  int dev = 0;
  PC_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return PC_ERR_INVALID_ARG;
  double* scratch;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dot_scratch[dev]) {
      pc_status s = dalloc(&g_dot_scratch[dev], sizeof(double) * (size_t)pc::dot_partials());
      if (s != PC_OK) return s;
    }
    scratch = g_dot_scratch[dev];
  }
  return from_cuda(pc::launch_dot(n, x, y, result, scratch, (cudaStream_t)stream));
}

pc_status pc_grad_val(const pc_csr* A, const double* lambda, const double* x, double* grad_val, void* stream) {
  if (!csr_ok(A) || !lambda || !x || !grad_val) return PC_ERR_INVALID_ARG;
  const pc_status s = check_csr(A, (cudaStream_t)stream, nullptr);
  if (s != PC_OK) return s;
  return from_cuda(pc::launch_grad_val(A->n, A->row_ptr, A->col_idx, lambda, x, grad_val, (cudaStream_t)stream));
}

pc_status pc_grad_edges(int64_t n_edges, const int32_t* p, const int32_t* q, const double* lambda, const double* x,
                        int64_t n, double* grad_c, void* stream) {
  if (n_edges < 0 || n < 0) return PC_ERR_INVALID_ARG;
  if (n_edges == 0) return PC_OK;
  if (!p || !q || !lambda || !x || !grad_c || n == 0 || n > INT32_MAX) return PC_ERR_INVALID_ARG;
  return from_cuda(pc::launch_grad_edges(n_edges, p, q, lambda, x, n, grad_c, (cudaStream_t)stream));
}

// ------------------------------------------------------------------ PCG
static pc_status ensure_cg_workspace(pc_handle* h, cudaStream_t st) {
  const int block = pc::PCG_BLOCK;
  int grid = 0;
  PC_TRY(pc::persistent_grid(h->L, h->A.nnz, h->val_f32, h->fac_f32, &grid));
  if (h->cg && h->grid == grid) return PC_OK;
  dfree(h->part);
  dfree(h->split);
  h->part = nullptr;
  h->split = nullptr;
  pc_status s = PC_OK;
  if (!h->cg) s = dalloc(&h->cg, sizeof(double) * (4 * (size_t)vec_stride(h->A.n) + 64));
  if (s == PC_OK && !h->ctl) s = dalloc(&h->ctl, sizeof(pc::GridSync) + sizeof(pc::PcgOut));
  if (s == PC_OK) s = dalloc(&h->part, sizeof(double) * 4 * (size_t)grid);   // 2 buffers x 2 values
  if (s == PC_OK) s = dalloc(&h->split, sizeof(int64_t) * (size_t)(grid + 1));
  if (s != PC_OK) return s;
  PC_TRY(pc::launch_split(h->A.n, h->A.nnz, h->A.row_ptr, grid, h->split, st));
  h->grid = grid;
  h->block = block;
  return PC_OK;
}

// Column segments of the binned SpMV: sweeping the rows once per column segment keeps each
// sweep's part of x resident in L2 while the matrix streams.  On the 8M-row power-law matrix
// every segment count above 1 measured slower (each extra sweep adds rounds of dependent loads
// that outweigh the gathers it saves), so whole rows are the default; pc_set_col_segments
// forces a count.
static int col_segments() { return g_col_segments >= 1 ? g_col_segments : 1; }

// Row loop of the binned SpMV: 0 plain (column indices and values, then the gathers; 4 CTAs
// per SM), 1 pipelined (the next round's column indices load during the gathers; 2 CTAs per
// SM), 2 pipelined with the one-lane-per-row groups read from a sliced copy (coalesced index
// and value loads; the copy takes 8 or 12 bytes per entry of those groups, built at the
// first solve).  On the 8M-row power-law matrix the pipelined loop measured 1659 against
// 1694 us per SpMV for the plain one.  PC_BIN_SPMV=plain|pipe|sliced overrides the choice.
constexpr int kBinLoopDefault = 2;

// Natural row order: the CSR walk or, for matrices whose rows have at most 64 entries, the
// same walk over a sliced copy (groups of 32 consecutive rows, entry k of each row at 32 k +
// lane).  PC_NAT_SPMV=sliced|csr first, then the launch shape (bin_pipe 2: sliced).
constexpr bool kNatSlicedDefault = false;

static bool nat_spmv_sliced(int shape_pipe) {
  const char* e = getenv("PC_NAT_SPMV");
  if (e && strcmp(e, "sliced") == 0) return true;
  if (e && strcmp(e, "csr") == 0) return false;
  if (shape_pipe >= 0) return shape_pipe == 2;
  return kNatSlicedDefault;
}

static void release_binning(pc_handle* h);

// Sliced copy of the natural-order groups (every row at most 64 entries, else none: the CSR
// walk).  Sets bin_pipe to 2 when built.
static pc_status build_natural_sliced(pc_handle* h, cudaStream_t st) {
  const int64_t n = h->A.n;
  const int64_t n_groups = (n + 31) / 32;
  int* dmax = reinterpret_cast<int*>(h->tmp);   // n >= 1 doubles of scratch
  int gmax_all = 0;
  pc_status s = dalloc(&h->gmax, sizeof(int32_t) * (size_t)n_groups);
  cudaError_t e = cudaSuccess;
  if (s == PC_OK) e = cudaMemsetAsync(dmax, 0, sizeof(int), st);
  if (s == PC_OK && e == cudaSuccess) e = pc::row_natural_gmax(n, h->A.row_ptr, h->gmax, dmax, st);
  if (s == PC_OK && e == cudaSuccess) e = cudaMemcpyAsync(&gmax_all, dmax, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (s == PC_OK && e == cudaSuccess) e = cudaStreamSynchronize(st);
  int64_t total = 0;
  if (s == PC_OK && e == cudaSuccess && gmax_all >= 1 && gmax_all <= 64) {
    s = dalloc(&h->sincl, sizeof(int64_t) * (size_t)n_groups);
    if (s == PC_OK)
      e = pc::row_sliced_sizes(n, h->gmax, h->sincl, pc::BIN_LANE_ROWS, reinterpret_cast<int64_t*>(h->tmp), st);
    if (s == PC_OK && e == cudaSuccess)
      e = cudaMemcpyAsync(&total, h->sincl + n_groups - 1, sizeof(total), cudaMemcpyDeviceToHost, st);
    if (s == PC_OK && e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (s == PC_OK && e == cudaSuccess) {
      const size_t vb = h->val_f32 ? sizeof(float) : sizeof(double);
      s = dalloc(&h->scol, sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
      if (s == PC_OK) s = dalloc(&h->sval, vb * (size_t)(total > 0 ? total : 1));
      if (s == PC_OK)
        e = pc::row_sliced_fill(n, h->A.row_ptr, 1, h->A.col_idx, h->A.val, h->val_f32 != 0, h->gmax, h->sincl,
                                pc::BIN_LANE_ROWS, h->scol, h->sval, st);
    }
  }
  if (s == PC_OK && e != cudaSuccess) s = from_cuda(e);
  if (s != PC_OK || !h->scol) {
    release_binning(h);
    return s;
  }
  h->bin_pipe = 2;
  return PC_OK;
}

// PC_BIN_SPMV first, then the handle's launch shape (bin_pipe 0 / 1 / 2), then the default.
static int bin_spmv_loop(int shape_pipe) {
  const char* e = getenv("PC_BIN_SPMV");
  if (e && strcmp(e, "sliced") == 0) return 2;
  if (e && strcmp(e, "pipe") == 0) return 1;
  if (e && strcmp(e, "plain") == 0) return 0;
  if (shape_pipe >= 0 && shape_pipe <= 2) return shape_pipe;
  return kBinLoopDefault;
}

static void release_binning(pc_handle* h) {
  dfree(h->perm);
  dfree(h->gsplit);
  dfree(h->items);
  h->items = nullptr;
  dfree(h->gmax);
  dfree(h->bnd);
  dfree(h->spart);
  dfree(h->scol);
  dfree(h->sval);
  dfree(h->sincl);
  h->scol = nullptr;
  h->sval = nullptr;
  h->sincl = nullptr;
  h->perm = nullptr;
  h->gsplit = nullptr;
  h->gmax = nullptr;
  h->bnd = nullptr;
  h->spart = nullptr;
  h->nseg = 0;
}

// Graph engine: the CG loop is a CUDA graph `while` node over three kernels (pc_cg_graph.cu).
// Row order of the graph engine's SpMV: rows are binned by length (pc_rowbin.cu) when the
// natural order would make the warp-uniform SpMV spend more than 1.25x the FP64 operations
// of the stored entries.  g_row_binning: -1 decide, 0 never, 1 always.
static pc_status choose_row_order(pc_handle* h, cudaStream_t st) {
  h->perm_checked = 1;
  const int64_t n = h->A.n;
  bool bin = g_row_binning == 1;
  if (g_row_binning < 0) {
    unsigned long long* d = reinterpret_cast<unsigned long long*>(h->tmp);   // n >= 1 doubles
    unsigned long long waste = 0;
    PC_TRY(cudaMemsetAsync(d, 0, sizeof(waste), st));
    PC_TRY(pc::row_bin_waste(n, h->A.row_ptr, d, st));
    PC_TRY(cudaMemcpyAsync(&waste, d, sizeof(waste), cudaMemcpyDeviceToHost, st));
    PC_TRY(cudaStreamSynchronize(st));
    bin = (double)waste > 1.25 * (double)h->A.nnz;
  }
  if (!bin) {
    h->bin_pipe = 0;
    if (nat_spmv_sliced(h->shape_used.bin_pipe)) return build_natural_sliced(h, st);
    return PC_OK;
  }
  h->bin_pipe = bin_spmv_loop(h->shape_used.bin_pipe);
  const int n_warps = pc::cg_spmv_bin_warps(h->bin_pipe != 0);
  const int64_t stride = vec_stride(n);
  const int64_t n_groups = (n + 31) / 32;
  int nseg = col_segments();
  int64_t* gscr = nullptr;    // per group: whole-group cost, inclusive prefix of the item counts
  pc_status s = dalloc(&h->perm, sizeof(int32_t) * (size_t)n);
  if (s == PC_OK) s = dalloc(&h->gsplit, sizeof(int32_t) * (size_t)(n_warps + 1));
  if (s == PC_OK) s = dalloc(&h->gmax, sizeof(int32_t) * (size_t)n_groups);
  if (s == PC_OK) s = dalloc(&h->bnd, sizeof(int32_t) * (size_t)(nseg + 1) * (size_t)stride);
  if (s == PC_OK && nseg > 1) s = dalloc(&h->spart, sizeof(double) * (size_t)stride);
  if (s == PC_OK) s = dalloc(&gscr, sizeof(int64_t) * 2 * (size_t)n_groups);
  if (s != PC_OK) {
    dfree(gscr);
    release_binning(h);
    return s;
  }
  int64_t m_items = 0;
  int64_t* icost = nullptr;
  cudaError_t e = pc::row_bin_build(n, h->A.row_ptr, h->perm, st);
  // the sliced copy (row loop 2, whole rows) serves longer one-lane-per-row groups
  const bool sliced = h->bin_pipe == 2 && nseg == 1;
  const int lane_max = sliced ? pc::BIN_SLICED_LANE_ROWS : pc::BIN_LANE_ROWS;
  if (e == cudaSuccess)
    e = pc::row_bin_group_stats(n, h->A.row_ptr, h->perm, gscr, h->gmax, gscr + n_groups, lane_max,
                                reinterpret_cast<int64_t*>(h->tmp), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&m_items, gscr + 2 * n_groups - 1, sizeof(m_items), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && (m_items < n_groups || m_items > n)) e = cudaErrorInvalidValue;   // cannot happen
  if (e == cudaSuccess) {
    s = dalloc(&h->items, sizeof(int32_t) * (size_t)m_items);
    if (s == PC_OK) s = dalloc(&icost, sizeof(int64_t) * (size_t)m_items);
    if (s == PC_OK)
      e = pc::row_bin_items(n, h->A.row_ptr, h->perm, h->gmax, gscr, gscr + n_groups, m_items, n_warps, h->items,
                            icost, h->gsplit, reinterpret_cast<int64_t*>(h->tmp), st);
    if (s == PC_OK && e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  dfree(icost);
  dfree(gscr);
  if (s == PC_OK && e != cudaSuccess) s = from_cuda(e);
  if (s != PC_OK) {
    release_binning(h);
    return s;
  }
  // entry boundaries per binned position; segments need sorted columns, else whole rows
  int* d_unsorted = reinterpret_cast<int*>(h->tmp);   // after the split's use of the scratch
  int unsorted = 0;
  PC_TRY(cudaMemsetAsync(d_unsorted, 0, sizeof(int), st));
  PC_TRY(pc::row_seg_bounds(n, h->A.row_ptr, h->A.col_idx, h->perm, nseg, (n + nseg - 1) / nseg, stride, h->bnd,
                            d_unsorted, st));
  if (nseg > 1) {
    PC_TRY(cudaMemcpyAsync(&unsorted, d_unsorted, sizeof(int), cudaMemcpyDeviceToHost, st));
    PC_TRY(cudaStreamSynchronize(st));
    if (unsorted) {
      nseg = 1;
      PC_TRY(pc::row_seg_bounds(n, h->A.row_ptr, h->A.col_idx, h->perm, 1, n, stride, h->bnd, d_unsorted, st));
    }
  }
  h->nseg = nseg;
  if (sliced) {
    // sliced copy of the one-lane-per-row groups
    s = dalloc(&h->sincl, sizeof(int64_t) * (size_t)n_groups);
    int64_t total = 0;
    cudaError_t e2 = cudaSuccess;
    if (s == PC_OK) e2 = pc::row_sliced_sizes(n, h->gmax, h->sincl, lane_max, reinterpret_cast<int64_t*>(h->tmp), st);
    if (s == PC_OK && e2 == cudaSuccess)
      e2 = cudaMemcpyAsync(&total, h->sincl + n_groups - 1, sizeof(total), cudaMemcpyDeviceToHost, st);
    if (s == PC_OK && e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
    if (s == PC_OK && e2 == cudaSuccess) {
      const size_t vb = h->val_f32 ? sizeof(float) : sizeof(double);
      s = dalloc(&h->scol, sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
      if (s == PC_OK) s = dalloc(&h->sval, vb * (size_t)(total > 0 ? total : 1));
      if (s == PC_OK)
        e2 = pc::row_sliced_fill(n, h->bnd, stride, h->A.col_idx, h->A.val, h->val_f32 != 0, h->gmax, h->sincl,
                                 lane_max, h->scol, h->sval, st);
    }
    if (s == PC_OK && e2 != cudaSuccess) s = from_cuda(e2);
    if (s != PC_OK) {
      release_binning(h);
      return s;
    }
  } else if (h->bin_pipe == 2) {
    h->bin_pipe = 1;   // segments: the CSR walk
  }
  return PC_OK;
}

static pc_status pcg_solve_graph(pc_handle* h, const double* b, double* x, double tol, int32_t max_iter,
                                 pc_solve_info* info, cudaStream_t st) {
  const int64_t n = h->A.n;
  pc_status s = PC_OK;
  const int64_t vs = vec_stride(n);
  if (!h->cg) s = dalloc(&h->cg, sizeof(double) * (4 * (size_t)vs + 64));
  if (s == PC_OK && !h->gbx) s = dalloc(&h->gbx, sizeof(double) * 2 * (size_t)vs);
  if (s == PC_OK && !h->gpart) s = dalloc(&h->gpart, sizeof(double) * (size_t)pc::cg_graph_partials());
  if (s == PC_OK && !h->gscal) s = dalloc(&h->gscal, pc::cg_scalars_bytes());
  if (s != PC_OK) return s;
  if (!h->graph) {
    // the launch shape: forced, else recorded for this system's key, else the defaults
    memset(&h->shape_used, 0, sizeof(h->shape_used));
    h->shape_used.bin_pipe = -1;
    if (h->shape_forced) {
      h->shape_used = h->shape_force;
    } else {
      pc_shape t;
      if (pc::tune_lookup(pc::tune_key(h->bs, h->prec, h->A.n, h->A.nnz), &t)) h->shape_used = t;
    }
    if (!h->perm_checked) {
      s = choose_row_order(h, st);
      if (s != PC_OK) return s;
    }
    pc::CgBinned bin;
    memset(&bin, 0, sizeof(bin));
    if (h->perm) {
      bin.perm = h->perm;
      bin.gsplit = h->gsplit;
      bin.items = h->items;
      bin.gmax = h->gmax;
      bin.bnd = h->bnd;
      bin.bstride = vec_stride(n);
      bin.spart = h->spart;
      bin.nseg = h->nseg;
      bin.pipe = h->bin_pipe;
    }
    bin.scol = h->scol;   // sliced copy (binned one-lane groups, or the natural-order groups)
    bin.sval = h->sval;
    bin.sincl = h->sincl;
    PC_TRY(pc::cg_graph_create(&h->graph, h->L, h->A.row_ptr, h->A.col_idx, h->A.val, h->val_f32, h->minv,
                               h->fac_f32, h->gbx, h->gbx + vs, h->cg, h->cg + vs, h->cg + 2 * vs, h->cg + 3 * vs,
                               h->gpart, h->gscal, &bin,
                               pc::CgShape{h->shape_used.spmv_ctas_per_sm, h->shape_used.ring_stages,
                                           h->shape_used.fuse_update},
                               st));
    // report what the graph runs: 1 fused update, 2 separate update kernel
    h->shape_used.fuse_update = pc::cg_graph_fused(h->graph) ? 1 : 2;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PC_TRY(cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->gbx, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->gbx + vs, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  pc::CgResult res;
  memset(&res, 0, sizeof(res));
  if (e == cudaSuccess) e = pc::cg_graph_solve(h->graph, tol, max_iter, 3, h->val_f32, h->fac_f32, st, &res);
  if (e == cudaSuccess) e = cudaMemcpyAsync(x, h->gbx + vs, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return from_cuda(e);
  const pc_status status = (pc_status)res.status;
  h->prof_valid = res.kernel_us[0] > 0.0 ? 1 : 0;
  for (int i = 0; i < 3; ++i) h->prof_ns[i] = (int64_t)(1000.0 * res.kernel_us[i]);
  if (info) {
    info->status = status;
    info->iterations = res.iterations;
    info->restarts = res.restarts;
    info->rel_residual = res.rel_residual;
    info->true_rel_residual = res.true_rel_residual;
    info->solve_ms = ms;
    info->grid_ctas = 0;
    info->block_size = h->bs;
    info->prec = h->prec;
  }
  return status;
}

pc_status pcg_solve_h(pc_handle* h, const double* b, double* x, double tol, int32_t max_iter, pc_solve_info* info,
                      void* stream) {
  NvtxRange nv("pcg_solve_h");
  if (info) {
    memset(info, 0, sizeof(*info));
    info->failed_block = -1;
  }
  if (!h || !b || !x || !(tol >= 0.0) || max_iter < 0) return PC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cg_engine() == 0) return pcg_solve_graph(h, b, x, tol, max_iter, info, st);
  pc_status s = ensure_cg_workspace(h, st);
  if (s != PC_OK) return s;
  const int64_t n = h->A.n;
  pc::PcgArgs a;
  a.lay = h->L;
  pc::pcg_plan(a, h->A.nnz, h->val_f32, h->fac_f32);
  a.rp = h->A.row_ptr;
  a.ci = h->A.col_idx;
  a.va = h->A.val;
  a.minv = h->minv;
  a.b = b;
  a.x = x;
  a.r = h->cg;
  a.z = h->cg + vec_stride(n);
  a.p = h->cg + 2 * vec_stride(n);
  a.q = h->cg + 3 * vec_stride(n);
  a.part = h->part;
  a.split = h->split;
  a.gs = reinterpret_cast<pc::GridSync*>(h->ctl);
  a.out = reinterpret_cast<pc::PcgOut*>(h->ctl + sizeof(pc::GridSync));
  a.tol = tol;
  a.max_iter = max_iter;
  a.max_restarts = 3;
  a.budget = wait_budget();
  a.trace = nullptr;
  a.trace_len = 0;
  {
    const char* tv = getenv("PC_TRACE_BARRIERS");
    const int want = tv ? atoi(tv) : 0;
    if (want > 0) {
      if (!h->trace_d || h->trace_len != want) {
        dfree(h->trace_d);
        h->trace_d = nullptr;
        h->trace_len = 0;
        if (dalloc(&h->trace_d, sizeof(unsigned long long) * (size_t)want) == PC_OK) h->trace_len = want;
      }
      if (h->trace_d) {
        PC_TRY(cudaMemsetAsync(h->trace_d, 0, sizeof(unsigned long long) * (size_t)h->trace_len, st));
        a.trace = h->trace_d;
        a.trace_len = h->trace_len;
      }
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PC_TRY(cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ctl, 0, sizeof(pc::GridSync) + sizeof(pc::PcgOut), st);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = pc::launch_pcg(a, h->val_f32, h->fac_f32, h->grid, h->block, st);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  unsigned char hostctl[sizeof(pc::GridSync) + sizeof(pc::PcgOut)];
  if (e == cudaSuccess) e = cudaMemcpyAsync(hostctl, h->ctl, sizeof(hostctl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return from_cuda(e);
  pc::GridSync gs;
  pc::PcgOut out;
  memcpy(&gs, hostctl, sizeof(gs));
  memcpy(&out, hostctl + sizeof(gs), sizeof(out));
  pc_status status = gs.status != 0 ? (pc_status)gs.status : (pc_status)out.status;
  if (info) {
    info->status = status;
    info->iterations = out.iterations;
    info->restarts = out.restarts;
    info->rel_residual = out.rel_residual;
    info->true_rel_residual = out.true_rel_residual;
    info->solve_ms = ms;
    info->grid_ctas = h->grid;
    info->block_size = h->bs;
    info->prec = h->prec;
  }
  return status;
}

pc_status pcg_solve(const pc_csr* A, int32_t block_size, const double* b, double* x, double tol, int32_t max_iter,
                    int32_t prec, pc_solve_info* info, void* stream) {
  NvtxRange nv("pcg_solve");
  if (info) {
    memset(info, 0, sizeof(*info));
    info->failed_block = -1;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PC_TRY(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce == cudaSuccess) ce = cudaEventRecord(e0, st);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return from_cuda(ce);
  }
  pc_handle* h = nullptr;
  pc_status s = pc_setup(A, block_size, 0.0, prec, stream, &h);
  float setup_ms = 0.f;
  if (cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess)
    cudaEventElapsedTime(&setup_ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != PC_OK) {
    if (info) {
      info->status = s;
      info->failed_block = h ? (int32_t)h->failed_block : -1;
      info->setup_ms = setup_ms;
    }
    if (h) pc_destroy(h);
    return s;
  }
  s = pcg_solve_h(h, b, x, tol, max_iter, info, stream);
  if (info) info->setup_ms = setup_ms;
  pc_destroy(h);
  return s;
}

pc_status pc_handle_shape(const pc_handle* h, pc_shape* out) {
  if (!h || !out || !h->graph) return PC_ERR_INVALID_ARG;
  *out = h->shape_used;
  return PC_OK;
}

pc_status pc_autotune(const pc_csr* A, int32_t block_size, int32_t prec, int32_t iterations, int32_t max_trials,
                      void* stream, pc_shape* best) {
  NvtxRange nv("pc_autotune");
  if (!csr_ok(A) || iterations < 1 || iterations > 10000 || max_trials < 0) return PC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = A->n;
  pc_handle* h = nullptr;
  pc_status s = pc_setup(A, block_size, 0.0, prec, stream, &h);
  if (s != PC_OK) {
    if (h) pc_destroy(h);
    return s;
  }
  double *b = nullptr, *x = nullptr;
  s = dalloc(&b, sizeof(double) * (size_t)n);
  if (s == PC_OK) s = dalloc(&x, sizeof(double) * (size_t)n);
  if (s == PC_OK) {
    const std::vector<double> ones((size_t)n, 1.0);
    const cudaError_t e = cudaMemcpy(b, ones.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) s = from_cuda(e);
  }
  // one solve under the default shape decides the row order (natural or binned)
  auto run = [&](double* ms_per_it) -> pc_status {
    PC_TRY(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, st));
    pc_solve_info info;
    memset(&info, 0, sizeof(info));
    const pc_status r = pcg_solve_graph(h, b, x, 0.0, iterations, &info, st);
    if (r != PC_OK && r != PC_ERR_NO_CONVERGENCE) return r;
    if (ms_per_it) *ms_per_it = info.iterations > 0 ? info.solve_ms / info.iterations : 1e300;
    return PC_OK;
  };
  if (s == PC_OK) s = run(nullptr);
  std::vector<pc_shape> cands;
  if (s == PC_OK) {
    pc_shape c;
    memset(&c, 0, sizeof(c));
    c.bin_pipe = -1;
    if (h->perm) {
      for (int pipe : {2, 1, 0})
        for (int ring : {4, 3, 2}) {
          c.bin_pipe = pipe;
          c.ring_stages = ring;
          cands.push_back(c);
        }
    } else {
      for (int ctas : {4, 2, 3, 6, 8})
        for (int ring : {4, 3, 2}) {
          c.spmv_ctas_per_sm = ctas;
          c.ring_stages = ring;
          cands.push_back(c);
        }
    }
    if (max_trials > 0 && (size_t)max_trials < cands.size()) cands.resize((size_t)max_trials);
  }
  // the candidates run the default update (fused with FP64 factors, a separate kernel
  // otherwise); the best of them is also tried with the other one
  const size_t n_main = cands.size();
  const bool natural = !h->perm;
  int extra = 0;   // final trials on the best shape: the other update, then (natural order) the other walk
  pc_shape bestc;
  memset(&bestc, 0, sizeof(bestc));
  bestc.bin_pipe = -1;
  double best_ms = 1e300;
  for (size_t i = 0; s == PC_OK && i <= cands.size(); ++i) {
    if (i == cands.size()) {
      if (n_main == 0) break;
      pc_shape c = bestc;
      if (extra == 0) {
        // bestc.fuse_update is what its graph ran (1 fused, 2 separate); a system whose
        // preconditioner cannot take the fused tail resolves 1 to 2 again, a repeat of bestc
        c.fuse_update = bestc.fuse_update == 1 ? 2 : 1;
      } else if (extra == 1 && natural) {
        c.bin_pipe = bestc.bin_pipe == 2 ? 1 : 2;   // CSR walk <-> sliced copy
      } else {
        break;
      }
      ++extra;
      cands.push_back(c);
    }
    // a new loop graph (and, for another row loop, a new binned split) with this shape
    if (h->graph) {
      pc::cg_graph_destroy(h->graph);
      h->graph = nullptr;
    }
    // another row loop (resolved as choose_row_order would) needs the row order rebuilt
    const int want = natural ? (nat_spmv_sliced(cands[i].bin_pipe) ? 2 : 0) : bin_spmv_loop(cands[i].bin_pipe);
    if (want != h->bin_pipe) {
      release_binning(h);
      h->perm_checked = 0;
    }
    h->shape_forced = 1;
    h->shape_force = cands[i];
    double ms = 0.0;
    s = run(nullptr);   // builds the graph and warms it
    if (s == PC_OK) s = run(&ms);
    // a final trial's option replaces the best shape's only when at least 1% faster (the
    // sliced natural walk also costs a copy of the matrix at setup, outside these timings)
    if (s == PC_OK && ms < (i < n_main ? best_ms : 0.99 * best_ms)) {
      best_ms = ms;
      bestc = h->shape_used;   // the candidate as its graph resolved it (fuse_update 1 or 2)
    }
  }
  cudaStreamSynchronize(st);
  dfree(b);
  dfree(x);
  pc_destroy(h);
  if (s != PC_OK) return s;
  bestc.us_per_iteration = best_ms < 1e299 ? 1000.0 * best_ms : 0.0;
  pc::tune_record(pc::tune_key(block_size, prec, A->n, A->nnz), bestc);
  if (best) *best = bestc;
  return pc::tune_save_env();
}

// ------------------------------------------------------------------ Lanczos
pc_status kappa_estimate_h(pc_handle* h, const pc_csr* A, int32_t max_steps, double tol, const double* v0,
                           int32_t reorth, pc_kappa_info* info, void* stream) {
  NvtxRange nv("kappa_estimate");
  double* ha = info ? info->alpha : nullptr;
  double* hb = info ? info->beta : nullptr;
  if (info) {
    memset(info, 0, sizeof(*info));
    info->alpha = ha;
    info->beta = hb;
  }
  const pc_csr* M = h ? &h->A : A;
  if (!csr_ok(M) || !v0 || max_steps < 1 || max_steps > 256 || !(tol >= 0.0) || (reorth != 0 && reorth != 1))
    return PC_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!h) {   // a handle's CSR was checked by pc_setup
    const pc_status cs = check_csr(M, st, nullptr);
    if (cs != PC_OK) return cs;
  }
  const int64_t n = M->n;
  const int m = max_steps;
  const int G = pc::lanczos_grid();
  pc::LanczosState s;
  memset(&s, 0, sizeof(s));
  s.n = n;
  s.m = m;
  s.tol = tol;
  double* small = nullptr;
  unsigned char* ctlbuf = nullptr;
  pc_status st_ = dalloc(&s.V, sizeof(double) * (size_t)m * (size_t)n);
  if (st_ == PC_OK) st_ = dalloc(&s.w, sizeof(double) * (size_t)n);
  if (st_ == PC_OK) st_ = dalloc(&s.t, sizeof(double) * (size_t)n);
  if (st_ == PC_OK) st_ = dalloc(&small, sizeof(double) * (size_t)(4 * m + 4));
  if (st_ == PC_OK) st_ = dalloc(&s.part, sizeof(double) * (size_t)G * (size_t)m);
  if (st_ == PC_OK) st_ = dalloc(&ctlbuf, 64);
  auto cleanup = [&]() {
    dfree(s.V);
    dfree(s.w);
    dfree(s.t);
    dfree(small);
    dfree(s.part);
    dfree(ctlbuf);
  };
  if (st_ != PC_OK) {
    cleanup();
    return st_;
  }
  s.alpha = small;
  s.beta = small + m;
  s.coef = small + 2 * m;
  s.result = small + 4 * m;
  s.tnorm = small + 4 * m + 2;
  s.counter = reinterpret_cast<unsigned*>(ctlbuf);
  s.ctl = reinterpret_cast<int*>(ctlbuf + 16);
  const bool precond = h != nullptr;
  const Layout L = precond ? h->L : pc::make_layout(n, 1);
  const void* linv = precond ? h->linv : nullptr;
  const bool f32 = precond ? h->fac_f32 : false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = pc::lanczos_configure(m);
  if (e == cudaSuccess) e = pc::lanczos_init(s, v0, precond, L, linv, f32, st);
  for (int j = 0; j < m && e == cudaSuccess; ++j) {
    e = pc::lanczos_step(s, j, reorth, precond, L, M->row_ptr, M->col_idx, M->val, M->dtype == PC_F32, linv, f32,
                         st);
    if (e == cudaSuccess && (j % 16) == 15 && j + 1 < m) {
      int done = 0;
      e = cudaMemcpyAsync(&done, s.ctl, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e == cudaSuccess && done) break;
    }
  }
  if (e == cudaSuccess) e = pc::lanczos_finish(s, st);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  double res[2] = {0.0, 0.0};
  int ctl[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, s.result, sizeof(res), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctl, s.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && ha) e = cudaMemcpyAsync(ha, s.alpha, sizeof(double) * m, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && hb) e = cudaMemcpyAsync(hb, s.beta, sizeof(double) * m, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cleanup();
  if (e != cudaSuccess) return from_cuda(e);
  if (info) {
    info->status = PC_OK;
    info->steps = ctl[1];
    info->lambda_min = res[0];
    info->lambda_max = res[1];
    info->kappa = res[1] / res[0];
    info->elapsed_ms = ms;
  }
  return PC_OK;
}

pc_status kappa_estimate(const pc_csr* A, int32_t block_size, int32_t max_steps, double tol, const double* v0,
                         int32_t reorth, pc_kappa_info* info, void* stream) {
  if (block_size < 0 || block_size > 64) return PC_ERR_INVALID_ARG;
  if (block_size == 0) return kappa_estimate_h(nullptr, A, max_steps, tol, v0, reorth, info, stream);
  pc_handle* h = nullptr;
  pc_status s = pc_setup(A, block_size, 0.0, PC_PREC_FP64, stream, &h);
  if (s != PC_OK) {
    if (h) pc_destroy(h);
    if (info) info->status = s;
    return s;
  }
  s = kappa_estimate_h(h, A, max_steps, tol, v0, reorth, info, stream);
  pc_destroy(h);
  return s;
}

// Batched mode: pc_batched.cu.

}  // extern "C"

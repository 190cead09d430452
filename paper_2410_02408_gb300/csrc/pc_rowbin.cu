// Row binning for the thread-per-row SpMV on matrices with irregular row lengths.
//
// The CG SpMV gives one row to each lane and runs every lane for the longest row of its
// warp (predicated FP64 FMAs still occupy this GPU's narrow FP64 pipe), so a warp that
// holds one hub row among short rows pays for 32 hub rows.  Sorting the rows by length
// inside windows of ROWBIN_W consecutive rows makes the 32 rows of a warp similar in length
// while keeping each warp's vector accesses inside the window (L1/L2 reuse).
//
// The permutation is a stable counting sort per window (deterministic: slices of 32 rows
// in row order, ranks inside a slice by lane order), so the SpMV stays bit-reproducible.
#include "pc_kernels.cuh"

namespace pc {

constexpr int ROWBIN_THREADS = 256;
constexpr int ROWBIN_SLICES = ROWBIN_W / 32;           // 64 slices of 32 rows
constexpr int ROWBIN_BUCKETS = 128;

// Length bucket: exact up to 64 entries, then 8 buckets per octave (ratio 2^(1/8) within a
// bucket).
__device__ __forceinline__ int row_bucket(int32_t len) {
  if (len <= 64) return len;
  const int b = 64 + (int)ceilf(8.0f * log2f((float)len * (1.0f / 64.0f)));
  return b < ROWBIN_BUCKETS - 1 ? b : ROWBIN_BUCKETS - 1;
}

// Sum over 32-row groups of 32 * (longest row of the group): the FP64 lane-operations the
// unbinned SpMV spends.  out[0] += that sum (integer atomics: exact).
__global__ void row_waste_kernel(int64_t n, const int32_t* __restrict__ rp, unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  unsigned long long mine = 0;
  for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) - lane; base < n;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = base + lane;
    const int32_t len = row < n ? __ldg(rp + row + 1) - __ldg(rp + row) : 0;
    const int32_t m = __reduce_max_sync(FULL, len);
    if (lane == 0) mine += 32ull * (unsigned long long)m;
  }
  if (lane == 0 && mine) atomicAdd(out, mine);
}

// perm[w0 .. w0+W) = the rows of window [w0, w0+W) sorted by length bucket (stable).
__global__ void __launch_bounds__(ROWBIN_THREADS) row_bin_kernel(int64_t n, const int32_t* __restrict__ rp,
                                                                 int32_t* __restrict__ perm) {
  __shared__ int cnt[ROWBIN_SLICES][ROWBIN_BUCKETS];
  __shared__ int base_b[ROWBIN_BUCKETS];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int NW = ROWBIN_THREADS / 32;
  const int64_t n_win = (n + ROWBIN_W - 1) / ROWBIN_W;
  for (int64_t win = blockIdx.x; win < n_win; win += gridDim.x) {
    const int64_t w0 = win * ROWBIN_W;
    for (int t = threadIdx.x; t < ROWBIN_SLICES * ROWBIN_BUCKETS; t += ROWBIN_THREADS) (&cnt[0][0])[t] = 0;
    __syncthreads();
    // per slice: bucket of every lane's row, rank among equal buckets of the slice
    int bk[ROWBIN_SLICES / NW], rk[ROWBIN_SLICES / NW];
#pragma unroll
    for (int k = 0; k < ROWBIN_SLICES / NW; ++k) {
      const int slice = k * NW + warp;
      const int64_t row = w0 + (int64_t)slice * 32 + lane;
      const bool valid = row < n;
      const int b = valid ? row_bucket(__ldg(rp + row + 1) - __ldg(rp + row)) : -1;
      const unsigned peers = __match_any_sync(FULL, b);
      const unsigned lower = peers & ((1u << lane) - 1u);
      bk[k] = b;
      rk[k] = __popc(lower);
      if (valid && lower == 0u) cnt[slice][b] = __popc(peers);
    }
    __syncthreads();
    // bucket totals, exclusive scan over buckets, then per bucket over slices in order
    if (threadIdx.x < ROWBIN_BUCKETS) {
      int tot = 0;
      for (int s = 0; s < ROWBIN_SLICES; ++s) tot += cnt[s][threadIdx.x];
      base_b[threadIdx.x] = tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = 0;
      for (int b = 0; b < ROWBIN_BUCKETS; ++b) {
        const int t = base_b[b];
        base_b[b] = run;
        run += t;
      }
    }
    __syncthreads();
    if (threadIdx.x < ROWBIN_BUCKETS) {
      int off = base_b[threadIdx.x];
      for (int s = 0; s < ROWBIN_SLICES; ++s) {
        const int t = cnt[s][threadIdx.x];
        cnt[s][threadIdx.x] = off;
        off += t;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ROWBIN_SLICES / NW; ++k) {
      const int slice = k * NW + warp;
      const int64_t row = w0 + (int64_t)slice * 32 + lane;
      if (bk[k] >= 0) perm[w0 + cnt[slice][bk[k]] + rk[k]] = (int32_t)row;
    }
    __syncthreads();
  }
}

// Work items of the binned SpMV and their cost.  The SpMV is bound by each warp's chain of
// dependent memory round trips (a round = the column indices and values, then the gathers of x
// they address), so the cost of an item is the length of its chain, weighted by the 256 entries
// a warp of short rows handles per round, or its FP64 lane-operations if that is larger, plus a
// per-item overhead.  Item kinds, as the SpMV walks them:
//   a 32-row group whose longest row has <= lane_max entries (64, or 256 over the sliced copy):
//     one lane per row, 8 entries per lane and
//     round: 1 + 2 ceil(max/8) round trips (the bounds load, then two per round);
//   a group whose longest row has <= 256 entries: 8 lanes per row, 4 rows per pass, 8 passes,
//     each taking the rounds of its longest row (64 entries per round);
//   a single row of a group whose longest row has more than 256 entries: the whole warp on that
//     row, 256 entries per round.  Such groups are split into their rows so that no warp's chain
//     is a whole group of hub rows.
__device__ __forceinline__ int64_t item_cost(int64_t ops, int64_t trips) {
  return (ops > 256 * trips ? ops : 256 * trips) + 256;
}

// Per 32-row group g of the binned order: gmax[g] = its longest row, gcount[g] = its number of
// items (1, or its rows when the longest row exceeds 256 entries), gcost[g] = the cost of the
// whole-group item (unused for split groups).
__global__ void group_stats_kernel(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ perm,
                                   int64_t* __restrict__ gcost, int32_t* __restrict__ gmax,
                                   int64_t* __restrict__ gcount, int lane_max) {
  const int lane = threadIdx.x & 31;
  const int64_t n_groups = (n + 31) / 32;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_groups;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t idx = g * 32 + lane;
    int32_t len = 0;
    if (idx < n) {
      const int32_t row = __ldg(perm + idx);
      len = __ldg(rp + row + 1) - __ldg(rp + row);
    }
    const int32_t m = __reduce_max_sync(FULL, len);
    const int32_t sum = __reduce_add_sync(FULL, len);
    // longest row of each pass of 4 rows (lanes 4p .. 4p+3), in lane 4p
    int32_t pm = max(len, __shfl_xor_sync(FULL, len, 1));
    pm = max(pm, __shfl_xor_sync(FULL, pm, 2));
    const int32_t pass_trips = __reduce_add_sync(FULL, (lane & 3) == 0 ? 2 * ((pm + 63) / 64) : 0);
    int64_t ops, trips;
    if (m <= lane_max) {
      ops = 32ll * m;
      trips = 1 + 2ll * ((m + 7) / 8);
    } else {
      ops = (int64_t)sum + 32ll * 3;
      trips = 1 + pass_trips;
    }
    if (lane == 0) {
      gcost[g] = item_cost(ops, trips);
      gmax[g] = m;
      const int64_t rows = n - g * 32 < 32 ? n - g * 32 : 32;
      gcount[g] = m > 256 ? rows : 1;
    }
  }
}

// Fill the items: for group g (first item incl[g] - count[g]), either the group itself (value g)
// or each of its rows (value -(pos + 1), pos = its binned position) with the cost of a warp on
// that row.
__global__ void item_fill_kernel(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ perm,
                                 const int32_t* __restrict__ gmax, const int64_t* __restrict__ gcost,
                                 const int64_t* __restrict__ gcount_incl, int32_t* __restrict__ items,
                                 int64_t* __restrict__ icost) {
  const int lane = threadIdx.x & 31;
  const int64_t n_groups = (n + 31) / 32;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_groups;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t incl = __ldg(gcount_incl + g);
    const int64_t first = g > 0 ? __ldg(gcount_incl + g - 1) : 0;
    const int64_t cnt = incl - first;
    if (__ldg(gmax + g) > 256) {
      const int64_t pos = g * 32 + lane;
      if (lane < cnt) {
        const int32_t row = __ldg(perm + pos);
        const int32_t len = __ldg(rp + row + 1) - __ldg(rp + row);
        items[first + lane] = (int32_t)(-(pos + 1));
        icost[first + lane] = item_cost((int64_t)len + 160, 1 + 2ll * ((len + 255) / 256));
      }
    } else if (lane == 0) {
      items[first] = (int32_t)g;
      icost[first] = __ldg(gcost + g);
    }
  }
}

// Inclusive prefix sum of cost[0..m) in place, in three launches: per chunk of
// SCAN_CHUNK entries its total (one CTA each), an exclusive scan of the chunk totals (one
// CTA), then each chunk's scan from its offset (each thread a contiguous run of SCAN_PER
// entries, the runs' totals scanned across the CTA).  Integer sums: exact in any order.
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER = 8;
constexpr int64_t SCAN_CHUNK = (int64_t)SCAN_THREADS * SCAN_PER;

// Exclusive scan of one value per thread across the CTA (SCAN_THREADS threads); *total gets
// the sum.  ws: 33 int64 of shared memory.
__device__ __forceinline__ int64_t cta_exclusive_scan(int64_t v, int64_t* ws, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int64_t w = ws[lane];
    int64_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(FULL, wi, o);
      if (lane >= o) wi += t;
    }
    ws[lane] = wi - w;   // exclusive offset of each warp
    if (lane == 31) ws[32] = wi;
  }
  __syncthreads();
  const int64_t r = ws[warp] + incl - v;
  *total = ws[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_chunk_totals(int64_t m, const int64_t* __restrict__ cost,
                                                                  int64_t* __restrict__ totals) {
  __shared__ int64_t ws[33];
  const int64_t c0 = (int64_t)blockIdx.x * SCAN_CHUNK;
  int64_t v = 0;
  for (int64_t i = c0 + threadIdx.x; i < m && i < c0 + SCAN_CHUNK; i += SCAN_THREADS) v += cost[i];
  int64_t tot;
  cta_exclusive_scan(v, ws, &tot);
  if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

// Exclusive scan of the nc chunk totals in place (one CTA; nc <= SCAN_THREADS * SCAN_PER).
__global__ void __launch_bounds__(SCAN_THREADS) scan_totals(int64_t nc, int64_t* __restrict__ totals) {
  __shared__ int64_t ws[33];
  const int64_t lo = (int64_t)threadIdx.x * SCAN_PER;
  int64_t v = 0;
  for (int64_t i = lo; i < lo + SCAN_PER && i < nc; ++i) v += totals[i];
  int64_t tot;
  int64_t run = cta_exclusive_scan(v, ws, &tot);
  for (int64_t i = lo; i < lo + SCAN_PER && i < nc; ++i) {
    const int64_t t = totals[i];
    totals[i] = run;
    run += t;
  }
}

__global__ void __launch_bounds__(SCAN_THREADS) scan_chunks(int64_t m, int64_t* __restrict__ cost,
                                                            const int64_t* __restrict__ offsets) {
  __shared__ int64_t ws[33];
  const int64_t lo = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_PER;
  int64_t v = 0;
  for (int64_t i = lo; i < lo + SCAN_PER && i < m; ++i) v += cost[i];
  int64_t tot;
  int64_t run = offsets[blockIdx.x] + cta_exclusive_scan(v, ws, &tot);
  for (int64_t i = lo; i < lo + SCAN_PER && i < m; ++i) {
    run += cost[i];
    cost[i] = run;
  }
}

// Scratch the scan needs for m entries: one int64 per chunk.
static int64_t scan_chunks_for(int64_t m) { return (m + SCAN_CHUNK - 1) / SCAN_CHUNK; }

static cudaError_t inclusive_scan(int64_t m, int64_t* cost, int64_t* scratch, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int64_t nc = scan_chunks_for(m);
  if (nc > SCAN_CHUNK) return cudaErrorInvalidValue;   // more than 2^26 entries: not needed here
  scan_chunk_totals<<<(unsigned)nc, SCAN_THREADS, 0, st>>>(m, cost, scratch);
  scan_totals<<<1, SCAN_THREADS, 0, st>>>(nc, scratch);
  scan_chunks<<<(unsigned)nc, SCAN_THREADS, 0, st>>>(m, cost, scratch);
  return cudaGetLastError();
}

// gsplit[w] = first item of warp w: the first item whose inclusive cost prefix exceeds
// w * total / n_items (so every warp gets a contiguous run of about equal cost).
__global__ void group_split_kernel(int64_t m, const int64_t* __restrict__ prefix, int n_items,
                                   int32_t* __restrict__ gsplit) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w > n_items) return;
  if (w == n_items) {
    gsplit[w] = (int32_t)m;
    return;
  }
  const int64_t total = m > 0 ? prefix[m - 1] : 0;
  const int64_t target = (int64_t)((double)total * (double)w / (double)n_items);
  int64_t lo = 0, hi = m;   // first index with prefix > target
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (prefix[mid] > target) hi = mid;
    else lo = mid + 1;
  }
  gsplit[w] = (int32_t)(w == 0 ? 0 : lo);
}

static int64_t group_grid(int64_t n) {
  const int64_t m = (n + 31) / 32;
  int64_t grid = (m * 32 + 255) / 256;
  if (grid > (int64_t)device_sms() * 16) grid = (int64_t)device_sms() * 16;
  return grid < 1 ? 1 : grid;
}

cudaError_t row_bin_group_stats(int64_t n, const int32_t* rp, const int32_t* perm, int64_t* gcost, int32_t* gmax,
                                int64_t* gcount_incl, int lane_max, int64_t* scan_ws, cudaStream_t st) {
  const int64_t m = (n + 31) / 32;
  group_stats_kernel<<<(unsigned)group_grid(n), 256, 0, st>>>(n, rp, perm, gcost, gmax, gcount_incl, lane_max);
  const cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : inclusive_scan(m, gcount_incl, scan_ws, st);
}

cudaError_t row_bin_items(int64_t n, const int32_t* rp, const int32_t* perm, const int32_t* gmax, const int64_t* gcost,
                          const int64_t* gcount_incl, int64_t m_items, int n_warps, int32_t* items, int64_t* icost,
                          int32_t* isplit, int64_t* scan_ws, cudaStream_t st) {
  item_fill_kernel<<<(unsigned)group_grid(n), 256, 0, st>>>(n, rp, perm, gmax, gcost, gcount_incl, items, icost);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = inclusive_scan(m_items, icost, scan_ws, st);
  if (e != cudaSuccess) return e;
  group_split_kernel<<<(n_warps + 1 + 255) / 256, 256, 0, st>>>(m_items, icost, n_warps, isplit);
  return cudaGetLastError();
}

// One thread per binned position: the row's entry boundaries of every column segment, from a
// scan of its column indices (which also checks that they increase).
__global__ void row_seg_bounds_kernel(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                      const int32_t* __restrict__ perm, int nseg, int64_t seg_cols, int64_t stride,
                                      int32_t* __restrict__ bnd, int* unsorted) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    const int32_t row = __ldg(perm + idx);
    const int32_t rs = __ldg(rp + row), re = __ldg(rp + row + 1);
    bnd[idx] = rs;
    bnd[(int64_t)nseg * stride + idx] = re;
    if (nseg < 2) continue;
    int sg = 1;                    // next boundary to place
    int64_t edge = seg_cols;       // its first column
    int32_t prev = -1;
    bool bad = false;
    for (int32_t k = rs; k < re; ++k) {
      const int32_t c = __ldg(ci + k);
      bad |= c <= prev;
      prev = c;
      while (sg < nseg && (int64_t)c >= edge) {
        bnd[(int64_t)sg * stride + idx] = k;
        ++sg;
        edge += seg_cols;
      }
    }
    for (; sg < nseg; ++sg) bnd[(int64_t)sg * stride + idx] = re;
    if (bad) atomicExch(unsorted, 1);
  }
}

cudaError_t row_seg_bounds(int64_t n, const int32_t* rp, const int32_t* ci, const int32_t* perm, int nseg,
                           int64_t seg_cols, int64_t stride, int32_t* bnd, int* unsorted, cudaStream_t st) {
  int64_t grid = (n + 255) / 256;
  if (grid > (int64_t)device_sms() * 16) grid = (int64_t)device_sms() * 16;
  if (grid < 1) grid = 1;
  row_seg_bounds_kernel<<<(unsigned)grid, 256, 0, st>>>(n, rp, ci, perm, nseg, seg_cols, stride, bnd, unsorted);
  return cudaGetLastError();
}

cudaError_t row_bin_waste(int64_t n, const int32_t* rp, unsigned long long* d_out, cudaStream_t st) {
  int64_t grid = (n + 255) / 256;
  if (grid > (int64_t)device_sms() * 16) grid = (int64_t)device_sms() * 16;
  if (grid < 1) grid = 1;
  row_waste_kernel<<<(unsigned)grid, 256, 0, st>>>(n, rp, d_out);
  return cudaGetLastError();
}

cudaError_t row_bin_build(int64_t n, const int32_t* rp, int32_t* perm, cudaStream_t st) {
  const int64_t n_win = (n + ROWBIN_W - 1) / ROWBIN_W;
  int64_t grid = n_win < (int64_t)device_sms() * 8 ? n_win : (int64_t)device_sms() * 8;
  if (grid < 1) grid = 1;
  row_bin_kernel<<<(unsigned)grid, ROWBIN_THREADS, 0, st>>>(n, rp, perm);
  return cudaGetLastError();
}


// Sliced copy of the one-lane-per-row groups.  Slab sizes: 32 * gmax[g] entries for groups
// whose longest row has at most lane_max entries, 0 for the others (they keep the CSR walk).
__global__ void sliced_size_kernel(int64_t m, const int32_t* __restrict__ gmax, int64_t* __restrict__ size,
                                   int lane_max) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < m; g += (int64_t)gridDim.x * blockDim.x) {
    const int32_t gm = __ldg(gmax + g);
    size[g] = gm <= lane_max ? 32ll * gm : 0;
  }
}

cudaError_t row_sliced_sizes(int64_t n, const int32_t* gmax, int64_t* sincl, int lane_max, int64_t* scan_ws,
                             cudaStream_t st) {
  const int64_t m = (n + 31) / 32;
  int64_t grid = (m + 255) / 256;
  if (grid > (int64_t)device_sms() * 16) grid = (int64_t)device_sms() * 16;
  if (grid < 1) grid = 1;
  sliced_size_kernel<<<(unsigned)grid, 256, 0, st>>>(m, gmax, sincl, lane_max);
  const cudaError_t e = cudaGetLastError();
  return e != cudaSuccess ? e : inclusive_scan(m, sincl, scan_ws, st);
}

// One warp per group with a slab: lane l copies the row at binned position 32 g + l, entry k to
// 32 k + l of the slab (the stores of one k are one contiguous run), padding past the row's
// end (and for positions past n) with column 0 and value 0.
template <typename VT>
__global__ void sliced_fill_kernel(int64_t n, const int32_t* __restrict__ bnd, int64_t stride,
                                   const int32_t* __restrict__ ci, const VT* __restrict__ va,
                                   const int32_t* __restrict__ gmax, const int64_t* __restrict__ sincl,
                                   int lane_max, int32_t* __restrict__ scol, VT* __restrict__ sval) {
  const int lane = threadIdx.x & 31;
  const int64_t m = (n + 31) / 32;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < m;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t gm = __ldg(gmax + g);
    if (gm > lane_max || gm <= 0) continue;   // warp-uniform
    const int64_t base = __ldg(sincl + g) - 32ll * gm;
    const int64_t pos = g * 32 + lane;
    const int32_t lo = pos < n ? __ldg(bnd + pos) : 0;
    const int32_t cnt = pos < n ? __ldg(bnd + stride + pos) - lo : 0;
    for (int32_t k = 0; k < gm; ++k) {
      const bool ok = k < cnt;
      scol[base + 32ll * k + lane] = ok ? __ldg(ci + lo + k) : 0;
      sval[base + 32ll * k + lane] = ok ? __ldg(va + lo + k) : VT(0);
    }
  }
}

cudaError_t row_sliced_fill(int64_t n, const int32_t* bnd, int64_t stride, const int32_t* ci, const void* va,
                            bool val_f32, const int32_t* gmax, const int64_t* sincl, int lane_max, int32_t* scol,
                            void* sval, cudaStream_t st) {
  const unsigned grid = (unsigned)group_grid(n);
  if (val_f32)
    sliced_fill_kernel<float><<<grid, 256, 0, st>>>(n, bnd, stride, ci, static_cast<const float*>(va), gmax, sincl,
                                                    lane_max, scol, static_cast<float*>(sval));
  else
    sliced_fill_kernel<double><<<grid, 256, 0, st>>>(n, bnd, stride, ci, static_cast<const double*>(va), gmax,
                                                     sincl, lane_max, scol, static_cast<double*>(sval));
  return cudaGetLastError();
}

// Longest row of each group of 32 consecutive rows (one warp per group) and their maximum.
__global__ void natural_gmax_kernel(int64_t n, const int32_t* __restrict__ rp, int32_t* __restrict__ gmax,
                                    int* dmax) {
  const int lane = threadIdx.x & 31;
  const int64_t m = (n + 31) / 32;
  int mine = 0;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < m;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t row = g * 32 + lane;
    const int32_t len = row < n ? __ldg(rp + row + 1) - __ldg(rp + row) : 0;
    const int32_t gm = __reduce_max_sync(FULL, len);
    if (lane == 0) gmax[g] = gm;
    mine = gm > mine ? gm : mine;
  }
  if (lane == 0 && mine) atomicMax(dmax, mine);
}

cudaError_t row_natural_gmax(int64_t n, const int32_t* rp, int32_t* gmax, int* dmax, cudaStream_t st) {
  natural_gmax_kernel<<<(unsigned)group_grid(n), 256, 0, st>>>(n, rp, gmax, dmax);
  return cudaGetLastError();
}

}  // namespace pc

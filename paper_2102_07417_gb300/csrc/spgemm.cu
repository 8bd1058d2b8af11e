// spgemm.cu -- the Galerkin product of Algorithm 1 (Eq. AcDef) as a GPU SpGEMM,
// C = X Y, used twice per level: A P, then R (A P) with R = P^T.
//
// Canonical summation order (part of the method in this library, see the
// set-up's file comment): C_iJ = sum over p ascending in row i of X of
// x_ip * Y_{k_p J}, each product rounded (__dmul_rn) and added left to right
// from 0 (__dadd_rn).  Every output row lists its columns in ascending order
// and keeps every structurally produced entry.  Compiled with --fmad=false.
//
// Rows are binned by the bound ub_i = sum_{p in X_i} nnz(Y_{k_p}) on the
// number of products:
//   tier 0  ub <= 32     a warp per row, one candidate product per lane, kept
//                        in registers; duplicates found with __match_any_sync,
//                        each group summed by its lowest lane in lane order
//                        (lane order = p order, so the sum is canonical);
//   tier 1-3 ub <= 64 / 256 / 1024   a warp per row, shared-memory hash set
//                        of 128 / 512 / 2048 slots, keys bitonic-sorted, then
//                        the values summed p by p into a shared accumulator;
//   tier 4  ub <= 4096   a block per row, 8192-slot table in shared memory;
//   tier 5  larger       a block per row, table in a global scratch slice.
// Each tier runs twice: a symbolic pass (distinct-column count per row, then
// a scan gives the row pointers) and a fill pass (columns + values).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TPB = 256;
constexpr int WARPS = TPB / 32;
constexpr int NTIER = 6;
constexpr int BTAB = 8192;  // tier-4 table slots

// flags[3] is set on a full hash table (cannot happen while ub <= slots / 2).
__device__ __forceinline__ bool hash_insert(int *table, unsigned mask, int key, int *flags) {
  unsigned h = ((unsigned)key * 2654435761u) & mask;
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const int prev = atomicCAS(&table[h], -1, key);
    if (prev == -1) return true;
    if (prev == key) return false;
    h = (h + 1) & mask;
  }
  flags[3] = 1;
  return false;
}

__device__ __forceinline__ int lower_bound(const int *a, int len, int key) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

__global__ void k_bin_rows(int m, const int *__restrict__ xrp, const int *__restrict__ xci,
                           const int *__restrict__ yrp, int *__restrict__ lists, int *__restrict__ counts,
                           int *__restrict__ max_ub, int *flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int cls = -1;
  if (i < m) {
    int64_t ub = 0;
    for (int p = xrp[i]; p < xrp[i + 1]; ++p) {
      const int k = xci[p];
      ub += yrp[k + 1] - yrp[k];
    }
    if (ub > (1 << 30)) {
      flags[3] = 1;
      ub = 1 << 30;
    }
    cls = ub <= 32 ? 0 : ub <= 64 ? 1 : ub <= 256 ? 2 : ub <= 1024 ? 3 : ub <= 4096 ? 4 : 5;
    if (cls == NTIER - 1) atomicMax(max_ub, (int)ub);
  }
  for (int c = 0; c < NTIER; ++c) {
    const unsigned mask = __ballot_sync(FULL, cls == c);
    if (!mask) continue;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&counts[c], __popc(mask));
    base = __shfl_sync(FULL, base, leader);
    if (cls == c) lists[(int64_t)c * m + base + __popc(mask & ((1u << lane) - 1u))] = i;
  }
}

// ---------------------------------------------------------- tier 0 ----
template <bool FILL>
__global__ void __launch_bounds__(TPB) k_spgemm_reg(const int *__restrict__ rows, int nrows,
                                                    const int *__restrict__ xrp, const int *__restrict__ xci,
                                                    const double *__restrict__ xv, const int *__restrict__ yrp,
                                                    const int *__restrict__ yci, const double *__restrict__ yv,
                                                    const int *__restrict__ crp, int *__restrict__ cci,
                                                    double *__restrict__ cv, int *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = gw; r < nrows; r += nw) {
    const int i = rows[r];
    int key = INT_MAX;
    double val = 0.0;
    int off = 0;
    for (int p = xrp[i]; p < xrp[i + 1]; ++p) {
      const int k = xci[p];
      const int yb = yrp[k], len = yrp[k + 1] - yb;
      if (lane >= off && lane < off + len) {
        const int q = yb + lane - off;
        key = yci[q];
        if (FILL) val = __dmul_rn(xv[p], yv[q]);
      }
      off += len;
    }
    const bool valid = lane < off;
    const unsigned grp = __match_any_sync(FULL, key);
    const bool leader = valid && (__ffs(grp) - 1) == lane;
    const unsigned lmask = __ballot_sync(FULL, leader);
    if (!FILL) {
      if (lane == 0) cnt[i] = __popc(lmask);
      continue;
    }
    int rank = 0;
    for (int j = 0; j < 32; ++j) {
      const int kj = __shfl_sync(FULL, key, j);
      rank += ((lmask >> j) & 1u) && kj < key;
    }
    const int maxg = (int)__reduce_max_sync(FULL, leader ? (unsigned)__popc(grp) : 0u);
    double acc = 0.0;
    unsigned mm = grp;
    for (int it = 0; it < maxg; ++it) {
      const int src = mm ? __ffs(mm) - 1 : lane;
      const double v = __shfl_sync(FULL, val, src);
      if (leader && mm) acc = __dadd_rn(acc, v);
      mm &= mm - 1u;
    }
    if (leader) {
      const int pos = crp[i] + rank;
      cci[pos] = key;
      cv[pos] = acc;
    }
  }
}

// -------------------------------------------------------- tiers 1-3 ----
// Shared memory per warp: TAB ints (hash table, then reused as TAB/2 double
// accumulators) + TAB/2 ints (the row's distinct columns, then sorted).
template <int TAB, bool FILL>
__global__ void __launch_bounds__(TPB) k_spgemm_hash(const int *__restrict__ rows, int nrows,
                                                     const int *__restrict__ xrp, const int *__restrict__ xci,
                                                     const double *__restrict__ xv, const int *__restrict__ yrp,
                                                     const int *__restrict__ yci, const double *__restrict__ yv,
                                                     const int *__restrict__ crp, int *__restrict__ cci,
                                                     double *__restrict__ cv, int *__restrict__ cnt, int *flags) {
  constexpr int HALF = TAB / 2;
  extern __shared__ __align__(16) int smem_i[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int *table = smem_i + warp * (TAB + HALF);
  int *keys = table + TAB;
  double *acc = reinterpret_cast<double *>(table);
  const int gw = blockIdx.x * WARPS + warp, nw = gridDim.x * WARPS;
  for (int r = gw; r < nrows; r += nw) {
    const int i = rows[r];
    for (int t = lane; t < TAB; t += 32) table[t] = -1;
    __syncwarp();
    const int xb = xrp[i], xe = xrp[i + 1];
    for (int p = xb; p < xe; ++p) {
      const int k = xci[p];
      for (int q = yrp[k] + lane; q < yrp[k + 1]; q += 32) hash_insert(table, TAB - 1, yci[q], flags);
    }
    __syncwarp();
    int count = 0;
    for (int t0 = 0; t0 < TAB; t0 += 32) {
      const int key = table[t0 + lane];
      const unsigned bal = __ballot_sync(FULL, key >= 0);
      if (key >= 0) keys[count + __popc(bal & ((1u << lane) - 1u))] = key;
      count += __popc(bal);
    }
    if (!FILL) {
      if (lane == 0) cnt[i] = count;
      __syncwarp();
      continue;
    }
    const int np2 = next_pow2(count);
    for (int t = count + lane; t < np2; t += 32) keys[t] = INT_MAX;
    __syncwarp();
    for (int kk = 2; kk <= np2; kk <<= 1)
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int t = lane; t < np2; t += 32) {
          const int u = t ^ jj;
          if (u > t) {
            const int a = keys[t], b = keys[u];
            if ((a > b) == ((t & kk) == 0)) {
              keys[t] = b;
              keys[u] = a;
            }
          }
        }
        __syncwarp();
      }
    const int cb = crp[i];
    for (int e = lane; e < count; e += 32) {
      cci[cb + e] = keys[e];
      acc[e] = 0.0;
    }
    __syncwarp();
    for (int p = xb; p < xe; ++p) {
      const int k = xci[p];
      const double x = xv[p];
      for (int q = yrp[k] + lane; q < yrp[k + 1]; q += 32) {
        const int pos = lower_bound(keys, count, yci[q]);
        acc[pos] = __dadd_rn(acc[pos], __dmul_rn(x, yv[q]));
      }
      __syncwarp();
    }
    for (int e = lane; e < count; e += 32) cv[cb + e] = acc[e];
    __syncwarp();
  }
}

// -------------------------------------------------------- tiers 4-5 ----
// A block per row; table of `cap` slots (then cap/2 double accumulators) and
// cap/2 keys, in shared memory (GLOBAL = false, cap = BTAB) or in this block's
// slice of global scratch (GLOBAL = true).
template <bool FILL, bool GLOBAL>
__global__ void __launch_bounds__(TPB) k_spgemm_block(const int *__restrict__ rows, int nrows,
                                                      const int *__restrict__ xrp, const int *__restrict__ xci,
                                                      const double *__restrict__ xv, const int *__restrict__ yrp,
                                                      const int *__restrict__ yci, const double *__restrict__ yv,
                                                      const int *__restrict__ crp, int *__restrict__ cci,
                                                      double *__restrict__ cv, int *__restrict__ cnt, int *flags,
                                                      int *gscratch, int gcap) {
  extern __shared__ __align__(16) int smem_b[];
  __shared__ int s_count;
  const int cap = GLOBAL ? gcap : BTAB;
  int *table = GLOBAL ? gscratch + (size_t)blockIdx.x * ((size_t)cap + cap / 2) : smem_b;
  int *keys = table + cap;
  double *acc = reinterpret_cast<double *>(table);
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int i = rows[r];
    for (int t = threadIdx.x; t < cap; t += blockDim.x) table[t] = -1;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    const int xb = xrp[i], xe = xrp[i + 1];
    for (int p = xb; p < xe; ++p) {
      const int k = xci[p];
      for (int q = yrp[k] + threadIdx.x; q < yrp[k + 1]; q += blockDim.x) hash_insert(table, cap - 1, yci[q], flags);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < cap; t += blockDim.x) {
      const int key = table[t];
      if (key >= 0) keys[atomicAdd(&s_count, 1)] = key;
    }
    __syncthreads();
    const int count = s_count;
    if (!FILL) {
      if (threadIdx.x == 0) cnt[i] = count;
      __syncthreads();
      continue;
    }
    const int np2 = next_pow2(count);
    for (int t = count + threadIdx.x; t < np2; t += blockDim.x) keys[t] = INT_MAX;
    __syncthreads();
    for (int kk = 2; kk <= np2; kk <<= 1)
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int t = threadIdx.x; t < np2; t += blockDim.x) {
          const int u = t ^ jj;
          if (u > t) {
            const int a = keys[t], b = keys[u];
            if ((a > b) == ((t & kk) == 0)) {
              keys[t] = b;
              keys[u] = a;
            }
          }
        }
        __syncthreads();
      }
    const int cb = crp[i];
    for (int e = threadIdx.x; e < count; e += blockDim.x) {
      cci[cb + e] = keys[e];
      acc[e] = 0.0;
    }
    __syncthreads();
    for (int p = xb; p < xe; ++p) {
      const int k = xci[p];
      const double x = xv[p];
      for (int q = yrp[k] + threadIdx.x; q < yrp[k + 1]; q += blockDim.x) {
        const int pos = lower_bound(keys, count, yci[q]);
        acc[pos] = __dadd_rn(acc[pos], __dmul_rn(x, yv[q]));
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < count; e += blockDim.x) cv[cb + e] = acc[e];
    __syncthreads();
  }
}

template <int TAB>
constexpr size_t hash_smem() {
  return (size_t)WARPS * (TAB + TAB / 2) * sizeof(int);
}
constexpr size_t block_smem = (size_t)(BTAB + BTAB / 2) * sizeof(int);

template <int TAB, bool FILL>
void launch_hash(int nr, const int *list, const DCsr &X, const DCsr &Y, DCsr &C, int *cnt, int *flags, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    AMG_CUDA(cudaFuncSetAttribute(k_spgemm_hash<TAB, FILL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)hash_smem<TAB>()));
    attr = true;
  }
  const int grid = std::max(1, std::min(ceil_div(nr, WARPS), kNumSMs * 32));
  k_spgemm_hash<TAB, FILL><<<grid, TPB, hash_smem<TAB>(), s>>>(list, nr, X.rp, X.ci, X.v, Y.rp, Y.ci, Y.v, C.rp,
                                                               C.ci, C.v, cnt, flags);
  AMG_CHECK_LAUNCH();
}

}  // namespace

void spgemm(Mem &m, int *flags, const DCsr &X, const DCsr &Y, int ncols, DCsr &C) {
  cudaStream_t s = m.stream;
  const int rows = X.n;
  Buf<int> lists(m, (size_t)rows * NTIER);
  Buf<int> meta(m, NTIER + 1);  // per-tier counts, max ub of the last tier
  AMG_CUDA(cudaMemsetAsync(meta.p, 0, sizeof(int) * (NTIER + 1), s));
  const double xy_bytes = 4.0 * (rows + 1) + 12.0 * X.nnz + 4.0 * (Y.n + 1) + 12.0 * Y.nnz;
  {
    ProfScope ps(s, AMG_K_SPGEMM, 4.0 * (rows + 1) + 4.0 * X.nnz + 4.0 * (Y.n + 1) + 4.0 * rows);
    k_bin_rows<<<ceil_div(rows, TPB), TPB, 0, s>>>(rows, X.rp, X.ci, Y.rp, lists.p, meta.p, meta.p + NTIER, flags);
    AMG_CHECK_LAUNCH();
  }
  int hm[NTIER + 1];
  AMG_CUDA(cudaMemcpyAsync(hm, meta.p, sizeof(hm), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  if (hm[NTIER] > (1 << 22)) {
    set_error("SpGEMM row product bound above 2^22 entries");
    throw Status{AMG_ERR_UNSUPPORTED};
  }
  int gcap = 2;
  while (gcap < 2 * std::max(hm[NTIER], 1)) gcap <<= 1;
  const int gblocks = std::min(hm[5], kNumSMs * 2);
  Buf<int> gscr;
  if (hm[5] > 0) gscr = Buf<int>(m, (size_t)gblocks * ((size_t)gcap + gcap / 2));
  static bool attr = false;
  if (!attr) {
    AMG_CUDA(cudaFuncSetAttribute(k_spgemm_block<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)block_smem));
    AMG_CUDA(cudaFuncSetAttribute(k_spgemm_block<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)block_smem));
    attr = true;
  }
  auto list = [&](int t) { return lists.p + (size_t)t * rows; };
  Buf<int> cnt(m, (size_t)rows + 1);
  for (int pass = 0; pass < 2; ++pass) {
    const bool fill = pass == 1;
    if (fill) {
      C.n = rows;
      C.ncols = ncols;
      C.rp = m.get_n<int>((size_t)rows + 1);
      C.nnz = scan_counts(m, cnt.p, C.rp, rows);
      C.ci = m.get_n<int>(std::max<int64_t>(C.nnz, 1));
      C.v = m.get_n<double>(std::max<int64_t>(C.nnz, 1));
    }
    ProfScope ps(s, AMG_K_SPGEMM, fill ? xy_bytes + 12.0 * C.nnz + 4.0 * (rows + 1) : xy_bytes - 8.0 * (X.nnz + Y.nnz));
    if (hm[0] > 0) {
      const int grid = std::max(1, std::min(ceil_div(hm[0], WARPS), kNumSMs * 32));
      if (fill)
        k_spgemm_reg<true><<<grid, TPB, 0, s>>>(list(0), hm[0], X.rp, X.ci, X.v, Y.rp, Y.ci, Y.v, C.rp, C.ci, C.v, cnt.p);
      else
        k_spgemm_reg<false><<<grid, TPB, 0, s>>>(list(0), hm[0], X.rp, X.ci, X.v, Y.rp, Y.ci, Y.v, nullptr, nullptr, nullptr, cnt.p);
      AMG_CHECK_LAUNCH();
    }
    if (hm[1] > 0) fill ? launch_hash<128, true>(hm[1], list(1), X, Y, C, cnt.p, flags, s)
                        : launch_hash<128, false>(hm[1], list(1), X, Y, C, cnt.p, flags, s);
    if (hm[2] > 0) fill ? launch_hash<512, true>(hm[2], list(2), X, Y, C, cnt.p, flags, s)
                        : launch_hash<512, false>(hm[2], list(2), X, Y, C, cnt.p, flags, s);
    if (hm[3] > 0) fill ? launch_hash<2048, true>(hm[3], list(3), X, Y, C, cnt.p, flags, s)
                        : launch_hash<2048, false>(hm[3], list(3), X, Y, C, cnt.p, flags, s);
    if (hm[4] > 0) {
      const int grid = std::max(1, std::min(hm[4], kNumSMs * 4));
      if (fill)
        k_spgemm_block<true, false><<<grid, TPB, block_smem, s>>>(list(4), hm[4], X.rp, X.ci, X.v, Y.rp, Y.ci, Y.v, C.rp, C.ci, C.v, cnt.p, flags, nullptr, 0);
      else
        k_spgemm_block<false, false><<<grid, TPB, block_smem, s>>>(list(4), hm[4], X.rp, X.ci, X.v, Y.rp, Y.ci, Y.v, nullptr, nullptr, nullptr, cnt.p, flags, nullptr, 0);
      AMG_CHECK_LAUNCH();
    }
    if (hm[5] > 0) {
      if (fill)
        k_spgemm_block<true, true><<<gblocks, TPB, 0, s>>>(list(5), hm[5], X.rp, X.ci, X.v, Y.rp, Y.ci, Y.v, C.rp, C.ci, C.v, cnt.p, flags, gscr.p, gcap);
      else
        k_spgemm_block<false, true><<<gblocks, TPB, 0, s>>>(list(5), hm[5], X.rp, X.ci, X.v, Y.rp, Y.ci, Y.v, nullptr, nullptr, nullptr, cnt.p, flags, gscr.p, gcap);
      AMG_CHECK_LAUNCH();
    }
  }
}

}  // namespace amg

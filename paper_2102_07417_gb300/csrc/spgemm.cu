// spgemm.cu -- the Galerkin product of Algorithm 1 (Eq. AcDef) as a GPU SpGEMM,
// C = X Y, used twice per level: A P, then R (A P) with R = P^T.
//
// Canonical summation order (part of the method in this library, see the
// set-up's file comment): C_iJ = sum over p ascending in row i of X of
// x_ip * Y_{k_p J}, each product rounded (__dmul_rn) and added left to right
// from 0 (__dadd_rn).  Every output row lists its columns in ascending order
// and keeps every structurally produced entry.  Compiled with --fmad=false.
//
// One numeric pass.  Each row i gets ub_i = sum_{p in X_i} nnz(Y_{k_p})
// slots of scratch (an upper bound on its distinct columns); the row's sorted
// columns and sums are written there with their count, and a compaction
// copies the rows into CSR.  (Leaving A P in that slot form for R (A P) to
// read skips its compaction but doubles its footprint; at the 128^3 level 0
// R (A P) then read 2.8 GB from DRAM and ran 1.5x longer.)  Rows are binned by
// ub_i into tiers (lists filled tile by tile, so neighbouring warps work on
// neighbouring rows):
//   tier 0    ub <= 32     a warp per row, one candidate product per lane in
//                          registers; duplicates found with __match_any_sync,
//                          each group summed by its lowest lane in lane order
//                          (lane order = p order, so the sum is canonical);
//   tier 1-2  ub <= 64, 128   a warp per row, a shared-memory hash set of
//                          2 ub_max slots (128, 256) with a running sum per
//                          slot; products fetched 32 at a time, equal columns
//                          grouped and added in p order; the columns
//                          bitonic-sorted at the end;
//   tier 3    ub > 128     the same with 256 slots, sized for the columns a
//                          row has rather than its product bound (Galerkin
//                          rows have far fewer: at most 122 distinct columns
//                          among the 128^3 Poisson rows with ub <= 4096); a
//                          row that finds more than 128 is retried with 1024
//                          slots, then with an exact table (2 ub slots) and
//                          a block per row -- in shared memory for ub <=
//                          4096, else in a global scratch slice.  (Tables of
//                          2 ub slots for every row had left 16 warps per SM
//                          at ub <= 512.)
//   merge     X row <= 8 entries and ub <= 64 (taken first when X has at least
//                          2^16 rows): a thread per row merging the row's
//                          sorted Y rows.  (Splitting it into lists by ub, for
//                          similar step counts per warp, measured slower: 1.52
//                          against 1.35 ms at level 0.)
// (A thread-per-row variant with a private accumulator in shared memory for
// every short row was bit-exact but twice as slow over a 128^3 set-up: its
// lanes gather Y entries of 32 different rows at once, uncoalesced.)
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TPB = 256;
constexpr int WARPS = TPB / 32;
constexpr int NTIER = 5;
constexpr int T_OPT = 3;     // ub > 128: warp tables sized for the row's distinct columns, retried on overflow
constexpr int T_THREAD = 4;  // thread per row, k-way merge
constexpr int MERGE_L = 8;   // longest X row of the merge tier
constexpr int BTAB = 8192;  // shared-memory table slots of the exact block tier (ub <= 4096)
constexpr int TILE = 1024;  // rows per binning tile

// The merge tier serialises a row's products in one thread: it is taken only
// when X has enough rows to fill the GPU with threads (on the coarse levels'
// few rows the warp tiers finish several times sooner).
constexpr int MERGE_MIN_ROWS = 1 << 16;

__device__ __forceinline__ int tier_of(int64_t ub, int xlen, bool merge_ok) {
  if (merge_ok && xlen <= MERGE_L && ub <= 64) return T_THREAD;
  return ub <= 32 ? 0 : ub <= 64 ? 1 : ub <= 128 ? 2 : T_OPT;
}

// Inserts key into an open-addressing set (linear probing) and returns its
// slot; flags[3] is set, and -1 returned, on a full table (cannot happen while
// ub <= slots / 2).
// *added tells whether the key was new to the set.
__device__ __forceinline__ int hash_insert_slot(int *table, unsigned mask, int key, int *flags, bool *added) {
  unsigned h = ((unsigned)key * 2654435761u) & mask;
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const int prev = atomicCAS(&table[h], -1, key);
    if (prev == -1 || prev == key) {
      *added = prev == -1;
      return (int)h;
    }
    h = (h + 1) & mask;
  }
  flags[3] = 1;
  *added = false;
  return -1;
}

// Slot of a key known to be in the table.
__device__ __forceinline__ int hash_find(const int *table, unsigned mask, int key) {
  unsigned h = ((unsigned)key * 2654435761u) & mask;
  for (unsigned probe = 0; probe < mask && table[h] != key; ++probe) h = (h + 1) & mask;
  return (int)h;
}

// Running sums start from -0.0 instead of the canonical +0.0: -0.0 + w == w
// exactly for every w, so the first product of a column is assigned rather
// than added (one FP64 add saved per output entry), and the two sequences
// agree at every step except while every product so far was -0.0 (then the
// canonical sum is +0.0: it never takes the value -0.0, since it starts at
// +0.0 and rounding to nearest gives +0.0 for x + (-x)).  canon0() maps the
// final -0.0 back to +0.0.
constexpr long long NEG0_BITS = (long long)0x8000000000000000ull;
__device__ __forceinline__ bool is_neg0(double a) { return __double_as_longlong(a) == NEG0_BITS; }
__device__ __forceinline__ double canon0(double a) { return is_neg0(a) ? 0.0 : a; }

__device__ __forceinline__ int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}


// Rows of the right operand Y: [rp[k], rp[k + 1]).
struct YRows {
  const int *rp;
  __device__ __forceinline__ int b(int k) const { return rp[k]; }
  __device__ __forceinline__ int e(int k) const { return rp[k + 1]; }
};

// ------------------------------------------------------------- binning ----
// ub_i = sum over the entries p of X row i of nnz(Y_{k_p}), G lanes per row
// (G = 1 for short X rows, up to 32 for long ones: the coarse levels' rows are
// long and few, and a thread walking a whole row left most SMs idle); the
// row's tier; per-tier row counts (block-aggregated) and the largest ub of
// the T_OPT rows in tcount[NTIER].  ub_out receives the row's scratch slice
// length, ub_i rounded up to 8.
template <int G>
__global__ void __launch_bounds__(TPB) k_row_ub(int m, const int *__restrict__ xrp, const int *__restrict__ xci,
                                                YRows y, int *__restrict__ ub_out, int8_t *__restrict__ tier,
                                                int *__restrict__ tcount, int *flags) {
  __shared__ int cnt[NTIER];
  if (threadIdx.x < NTIER) cnt[threadIdx.x] = 0;
  __syncthreads();
  constexpr int RPW = 32 / G;  // rows per warp step
  const int lane = threadIdx.x & 31, sub = lane & (G - 1), grp = lane / G;
  const int gw = (blockIdx.x * TPB + threadIdx.x) >> 5, nw = (gridDim.x * TPB) >> 5;
  for (int base = gw * RPW; base < m; base += nw * RPW) {  // the whole warp iterates together
    const int i = base + grp;
    int64_t ub = 0;
    if (i < m)
      for (int p = xrp[i] + sub; p < xrp[i + 1]; p += G) {
        const int k = xci[p];
        ub += y.e(k) - y.b(k);
      }
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) ub += __shfl_xor_sync(FULL, ub, o);
    if (i < m && sub == 0) {
      if (ub > (1 << 30)) {
        flags[3] = 1;
        ub = 1 << 30;
      }
      // the row's scratch slice, rounded up to 8 entries: every slice starts
      // on a 32-byte sector of column indices (two of values), so no sector
      // is shared by two rows written at different times (a partly written
      // sector costs DRAM a read-modify-write when it leaves L2)
      ub_out[i] = (int)((ub + 7) & ~(int64_t)7);
      const int t = tier_of(ub, xrp[i + 1] - xrp[i], m >= MERGE_MIN_ROWS);
      tier[i] = (int8_t)t;
      atomicAdd(&cnt[t], 1);
      if (t == T_OPT) atomicMax(&tcount[NTIER], (int)ub);
    }
  }
  __syncthreads();
  if (threadIdx.x < NTIER && cnt[threadIdx.x]) atomicAdd(&tcount[threadIdx.x], cnt[threadIdx.x]);
}

// Appends each row to its tier's list: tiles of TILE consecutive rows reserve a
// range of each list with one atomic per (tile, tier) and fill it in row order,
// so neighbouring rows stay together (the order affects speed only: a row's
// output position comes from its own offset).
__global__ void __launch_bounds__(TPB) k_tier_scatter(int m, const int8_t *__restrict__ tier,
                                                      const int *__restrict__ start, int *__restrict__ cursor,
                                                      int *__restrict__ lists) {
  __shared__ int run[NTIER];
  __shared__ int wcnt[NTIER][WARPS];
  __shared__ int tot[NTIER];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x < NTIER) tot[threadIdx.x] = 0;
  __syncthreads();
  for (int t0 = 0; t0 < TILE; t0 += TPB) {
    const int i = blockIdx.x * TILE + t0 + threadIdx.x;
    if (i < m) atomicAdd(&tot[tier[i]], 1);
  }
  __syncthreads();
  if (threadIdx.x < NTIER) run[threadIdx.x] = tot[threadIdx.x] ? start[threadIdx.x] +
                                                                 atomicAdd(&cursor[threadIdx.x], tot[threadIdx.x])
                                                               : 0;
  __syncthreads();
  for (int t0 = 0; t0 < TILE; t0 += TPB) {
    const int i = blockIdx.x * TILE + t0 + threadIdx.x;
    const int c = i < m ? tier[i] : -1;
    unsigned myb = 0;
    for (int t = 0; t < NTIER; ++t) {
      const unsigned b = __ballot_sync(FULL, c == t);
      if (lane == 0) wcnt[t][w] = __popc(b);
      if (c == t) myb = b;
    }
    __syncthreads();
    if (c >= 0) {
      int pos = run[c] + __popc(myb & ((1u << lane) - 1u));
      for (int ww = 0; ww < w; ++ww) pos += wcnt[c][ww];
      lists[pos] = i;
    }
    __syncthreads();
    if (threadIdx.x < NTIER) {
      int s = 0;
      for (int ww = 0; ww < WARPS; ++ww) s += wcnt[threadIdx.x][ww];
      run[threadIdx.x] += s;
    }
    __syncthreads();
  }
}

// ------------------------------------------------- warp row helpers ----
// Metadata of one chunk of up to 32 entries of X row [c0, xe): lane l holds
// entry c0 + l's Y row start and length, the X value, and the exclusive
// prefix of the lengths; *total is the chunk's number of products.
struct XChunk {
  int ys, len, excl;
  double xv;
};

__device__ __forceinline__ XChunk x_chunk(int c0, int xe, const int *__restrict__ xci, const double *__restrict__ xv,
                                          const YRows &y, int lane, int *total) {
  XChunk c{0, 0, 0, 0.0};
  const int p = c0 + lane;
  if (p < xe) {
    const int k = xci[p];
    c.ys = y.b(k);
    c.len = y.e(k) - c.ys;
    c.xv = xv[p];
  }
  int incl = c.len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  c.excl = incl - c.len;
  *total = __shfl_sync(FULL, incl, 31);
  return c;
}

// Source lane (X entry) of product u of a chunk: the last lane whose
// exclusive prefix is <= u (it always has a nonzero length).  All lanes call.
__device__ __forceinline__ int x_source(const XChunk &c, int u) {
  int lo = 0;
#pragma unroll
  for (int step = 16; step; step >>= 1) {
    const int e = __shfl_sync(FULL, c.excl, lo + step);
    if (e <= u) lo += step;
  }
  return lo;
}

// ------------------------------------------------------ merge tier ----
// A thread per row for short X rows (<= MERGE_L entries, ub <= 64): a k-way
// merge of the row's Y rows, which are sorted.  Each iteration takes ONE
// product: the head with the smallest column, ties to the lowest t (= lowest
// p), so the products of one output column arrive in ascending p and are
// added left to right from 0 -- the canonical order -- and the output comes
// out sorted.  One product per iteration keeps every FP64 instruction useful:
// the kernel is bound by the FP64 pipe, and the earlier form (all heads at
// the current column per iteration, unrolled) issued a predicated multiply and
// add for each of the MERGE_L heads at every output column (81% of the FP64
// pipe busy for ~2 products per output on the 128^3 Poisson A P).
__global__ void __launch_bounds__(TPB) k_spgemm_merge(const int *__restrict__ rows, int nrows,
                                                      const int *__restrict__ xrp, const int *__restrict__ xci,
                                                      const double *__restrict__ xv, YRows y,
                                                      const int *__restrict__ yci, const double *__restrict__ yv,
                                                      const int *__restrict__ off, int *__restrict__ tci,
                                                      double *__restrict__ tcv, int *__restrict__ cnt) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gridDim.x * blockDim.x) {
    const int i = rows[r];
    const int xb = xrp[i], len = xrp[i + 1] - xb;
    int hp[MERGE_L], he[MERGE_L], hc[MERGE_L];
    double xa[MERGE_L];
#pragma unroll
    for (int t = 0; t < MERGE_L; ++t) {
      hp[t] = he[t] = 0;
      hc[t] = INT_MAX;
      xa[t] = 0.0;
      if (t < len) {
        const int k = xci[xb + t];
        xa[t] = xv[xb + t];
        hp[t] = y.b(k);
        he[t] = y.e(k);
        if (hp[t] < he[t]) hc[t] = yci[hp[t]];
      }
    }
    const int base = off[i];
    int count = 0, ccol = -1;
    double acc = 0.0;
    for (;;) {
      // smallest head column; the strict < keeps the lowest t among equals
      int bc = hc[0], bt = 0;
#pragma unroll
      for (int t = 1; t < MERGE_L; ++t)
        if (hc[t] < bc) {
          bc = hc[t];
          bt = t;
        }
      if (bc == INT_MAX) break;
      int q = 0, e = 0;
      double x = 0.0;
#pragma unroll
      for (int t = 0; t < MERGE_L; ++t)
        if (t == bt) {
          q = hp[t];
          e = he[t];
          x = xa[t];
        }
      const double prod = __dmul_rn(x, yv[q]);
      const int cn = q + 1 < e ? yci[q + 1] : INT_MAX;
#pragma unroll
      for (int t = 0; t < MERGE_L; ++t)
        if (t == bt) {
          hp[t] = q + 1;
          hc[t] = cn;
        }
      if (bc != ccol) {  // a new column: its sum starts as -0.0 + prod == prod
        if (ccol >= 0) {
          tci[base + count] = ccol;
          tcv[base + count] = canon0(acc);
          ++count;
        }
        ccol = bc;
        acc = prod;
      } else {
        acc = __dadd_rn(acc, prod);
      }
    }
    if (ccol >= 0) {
      tci[base + count] = ccol;
      tcv[base + count] = canon0(acc);
      ++count;
    }
    cnt[i] = count;
  }
}

// ---------------------------------------------------------- tier 0 ----
__global__ void __launch_bounds__(TPB) k_spgemm_reg(const int *__restrict__ rows, int nrows,
                                                    const int *__restrict__ xrp, const int *__restrict__ xci,
                                                    const double *__restrict__ xv, YRows y,
                                                    const int *__restrict__ yci, const double *__restrict__ yv,
                                                    const int *__restrict__ off, int *__restrict__ tci,
                                                    double *__restrict__ tcv, int *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = gw; r < nrows; r += nw) {
    const int i = rows[r];
    const int xb = xrp[i], xe = xrp[i + 1];
    int key = INT_MAX;
    double val = 0.0;
    int o = 0;  // products placed so far (ub <= 32, so product t sits in lane t)
    for (int c0 = xb; c0 < xe; c0 += 32) {
      int total;
      const XChunk c = x_chunk(c0, xe, xci, xv, y, lane, &total);
      const int u = lane - o;
      const int src = x_source(c, u < 0 ? 0 : u);
      const int ys = __shfl_sync(FULL, c.ys, src), ex = __shfl_sync(FULL, c.excl, src);
      const double xs = __shfl_sync(FULL, c.xv, src);
      if (u >= 0 && u < total) {
        const int q = ys + u - ex;
        key = yci[q];
        val = __dmul_rn(xs, yv[q]);
      }
      o += total;
    }
    const bool valid = lane < o;
    const unsigned grp = __match_any_sync(FULL, key);
    const bool leader = valid && (__ffs(grp) - 1) == lane;
    const unsigned lmask = __ballot_sync(FULL, leader);
    int rank = 0;
    for (int j = 0; j < 32; ++j) {
      const int kj = __shfl_sync(FULL, key, j);
      rank += ((lmask >> j) & 1u) && kj < key;
    }
    const int maxg = (int)__reduce_max_sync(FULL, leader ? (unsigned)__popc(grp) : 0u);
    // the leader is its group's first member: the sum starts as -0.0 + val == val
    double acc = val;
    unsigned mm = grp & (grp - 1u);
    for (int it = 1; it < maxg; ++it) {
      const int sl = mm ? __ffs(mm) - 1 : lane;
      const double v = __shfl_sync(FULL, val, sl);
      if (leader && mm) acc = __dadd_rn(acc, v);
      mm &= mm - 1u;
    }
    const int base = off[i];
    if (leader) {
      tci[base + rank] = key;
      tcv[base + rank] = canon0(acc);
    }
    if (lane == 0) cnt[i] = __popc(lmask);
  }
}

// ------------------------------------------------- hash tiers 1-3 ----
// Shared memory per warp: acc[TAB] the running sum of each slot's column
// (doubles), table[TAB] the hash set of the row's columns, keys[TAB/2] the
// distinct columns (then sorted).
// The products are fetched 32 at a time in (p, q) order over the whole row
// (all lanes busy), each inserted into the set and added into its slot's sum
// at once: lanes holding the same column form a group (__match_any_sync)
// whose lowest lane adds the members in lane order, which is p order -- the
// canonical order.  The sorted columns then find their sums by their slots.
// A row may hold at most TAB/2 distinct columns.  The exact tiers (ub <=
// TAB/2) never reach that.  With a retry list (the optimistic tier, tables
// sized for the columns a row has rather than its product bound) a row that
// passes the limit is dropped after that chunk -- at most TAB/2 + 31 keys are
// then in the table, so probes always end -- and appended to the list for a
// larger table.  nrows_dev (if set) holds the length of the row list, filled
// by the previous kernel of the stream.
template <int TAB>
constexpr size_t hash_smem_warp() {
  return (size_t)TAB * sizeof(double) + (size_t)(TAB + TAB / 2) * sizeof(int);
}

// (At most 32 registers: eight blocks per SM where shared memory allows, up
// from six at 37; no spills.  128^3 set-up SpGEMM 4.10 -> 4.00 ms.)
template <int TAB>
__global__ void __launch_bounds__(TPB, 8) k_spgemm_hash(const int *__restrict__ rows, int nrows,
                                                     const int *__restrict__ nrows_dev,
                                                     const int *__restrict__ xrp, const int *__restrict__ xci,
                                                     const double *__restrict__ xv, YRows y,
                                                     const int *__restrict__ yci, const double *__restrict__ yv,
                                                     const int *__restrict__ off, int *__restrict__ tci,
                                                     double *__restrict__ tcv, int *__restrict__ cnt, int *flags,
                                                     int *__restrict__ retry, int *retry_n) {
  extern __shared__ __align__(16) int smem_i[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double *acc = reinterpret_cast<double *>(smem_i) + (size_t)warp * TAB;
  int *table = smem_i + 2 * WARPS * TAB + warp * (TAB + TAB / 2);
  int *keys = table + TAB;
  if (nrows_dev) nrows = *nrows_dev;
  const int gw = blockIdx.x * WARPS + warp, nw = gridDim.x * WARPS;
  for (int r = gw; r < nrows; r += nw) {
    const int i = rows[r];
    for (int t = lane; t < TAB; t += 32) {
      table[t] = -1;
      acc[t] = -0.0;
    }
    __syncwarp();
    const int xb = xrp[i], xe = xrp[i + 1];
    int ndist = 0;
    bool over = false;
    for (int c0 = xb; c0 < xe && !over; c0 += 32) {
      int total;
      const XChunk c = x_chunk(c0, xe, xci, xv, y, lane, &total);
      for (int u0 = 0; u0 < total; u0 += 32) {
        const int u = u0 + lane;
        const int src = x_source(c, u);
        const int ys = __shfl_sync(FULL, c.ys, src), ex = __shfl_sync(FULL, c.excl, src);
        const double xs = __shfl_sync(FULL, c.xv, src);
        int slot = -1;
        bool added = false;
        double v = 0.0;
        if (u < total) {
          const int q = ys + u - ex;
          v = __dmul_rn(xs, yv[q]);
          slot = hash_insert_slot(table, TAB - 1, yci[q], flags, &added);
        }
        ndist += __popc(__ballot_sync(FULL, added));
        const bool valid = slot >= 0;
        if (!valid) slot = -1 - lane;  // a group of its own
        const unsigned grp = __match_any_sync(FULL, slot);
        const bool leader = valid && (__ffs(grp) - 1) == lane;
        const int maxg = (int)__reduce_max_sync(FULL, leader ? (unsigned)__popc(grp) : 0u);
        double a = leader ? acc[slot] : 0.0;
        unsigned mm = grp;
        for (int it = 0; it < maxg; ++it) {
          const int sl = mm ? __ffs(mm) - 1 : lane;
          const double w = __shfl_sync(FULL, v, sl);
          const bool add = leader && mm != 0u;
          // a sum still at -0.0 takes w without an add (-0.0 + w == w)
          if (__any_sync(FULL, add && !is_neg0(a))) {
            if (add) a = is_neg0(a) ? w : __dadd_rn(a, w);
          } else if (add) {
            a = w;
          }
          mm &= mm - 1u;
        }
        if (leader) acc[slot] = a;
        __syncwarp();
        if (ndist > TAB / 2) {
          over = true;
          break;
        }
      }
    }
    if (over) {
      if (lane == 0) {
        if (retry) retry[atomicAdd(retry_n, 1)] = i;
        else flags[3] = 1;
      }
      __syncwarp();
      continue;
    }
    __syncwarp();
    int count = 0;
    for (int t0 = 0; t0 < TAB; t0 += 32) {
      const int key = table[t0 + lane];
      const unsigned bal = __ballot_sync(FULL, key >= 0);
      if (key >= 0) keys[count + __popc(bal & ((1u << lane) - 1u))] = key;
      count += __popc(bal);
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
    const int base = off[i];
    for (int e = lane; e < count; e += 32) {
      const int key = keys[e];
      tci[base + e] = key;
      tcv[base + e] = canon0(acc[hash_find(table, TAB - 1, key)]);
    }
    if (lane == 0) cnt[i] = count;
    __syncwarp();
  }
}

// ------------------------------------------- exact block-per-row retry ----
// A block per row: acc[cap] running sums (doubles) indexed by the hash slot,
// table[cap] the hash set and keys[cap/2] the distinct columns, in shared
// memory (GLOBAL = false, cap = BTAB) or in this block's slices of global
// scratch (GLOBAL = true).  One pass over the row's X entries in order: the
// threads split Y row k_p (distinct columns, so no two threads meet on a
// slot), insert each column and add the product into its slot's sum; a
// barrier between X entries keeps every column's sum in p order.
template <bool GLOBAL>
__global__ void __launch_bounds__(TPB) k_spgemm_block(const int *__restrict__ rows, int nrows,
                                                      const int *__restrict__ nrows_dev,
                                                      const int *__restrict__ xrp, const int *__restrict__ xci,
                                                      const double *__restrict__ xv, YRows y,
                                                      const int *__restrict__ yci, const double *__restrict__ yv,
                                                      const int *__restrict__ off, int *__restrict__ tci,
                                                      double *__restrict__ tcv, int *__restrict__ cnt, int *flags,
                                                      int *gscratch, double *gacc, int gcap) {
  extern __shared__ __align__(16) int smem_b[];
  __shared__ int s_count;
  const int cap = GLOBAL ? gcap : BTAB;
  double *acc = GLOBAL ? gacc + (size_t)blockIdx.x * cap : reinterpret_cast<double *>(smem_b);
  int *table = GLOBAL ? gscratch + (size_t)blockIdx.x * ((size_t)cap + cap / 2) : smem_b + 2 * BTAB;
  int *keys = table + cap;
  if (nrows_dev) nrows = *nrows_dev;
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int i = rows[r];
    for (int t = threadIdx.x; t < cap; t += blockDim.x) {
      table[t] = -1;
      acc[t] = -0.0;
    }
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    const int xb = xrp[i], xe = xrp[i + 1];
    for (int p = xb; p < xe; ++p) {
      const int k = xci[p];
      const double x = xv[p];
      for (int q = y.b(k) + threadIdx.x; q < y.e(k); q += blockDim.x) {
        bool added;
        const int slot = hash_insert_slot(table, cap - 1, yci[q], flags, &added);
        if (slot >= 0) {
          const double w = __dmul_rn(x, yv[q]);
          const double a = acc[slot];
          acc[slot] = is_neg0(a) ? w : __dadd_rn(a, w);
        }
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < cap; t += blockDim.x) {
      const int key = table[t];
      if (key >= 0) keys[atomicAdd(&s_count, 1)] = key;
    }
    __syncthreads();
    const int count = s_count;
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
    const int base = off[i];
    for (int e = threadIdx.x; e < count; e += blockDim.x) {
      const int key = keys[e];
      tci[base + e] = key;
      tcv[base + e] = canon0(acc[hash_find(table, cap - 1, key)]);
    }
    if (threadIdx.x == 0) cnt[i] = count;
    __syncthreads();
  }
}

// Copies each row's count entries from its scratch slot to the final CSR:
// G lanes per row (G = 8 when rows are short, so that most lanes of a warp
// copy something; a warp per row otherwise).
template <int G>
__global__ void __launch_bounds__(TPB) k_compact(int m, const int *__restrict__ off, const int *__restrict__ tci,
                                                 const double *__restrict__ tcv, const int *__restrict__ crp,
                                                 int *__restrict__ cci, double *__restrict__ cv) {
  const int sub = threadIdx.x & (G - 1);
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) / G, ng = (gridDim.x * blockDim.x) / G;
  for (int i = g; i < m; i += ng) {
    const int src = off[i], dst = crp[i], len = crp[i + 1] - dst;
    for (int e = sub; e < len; e += G) {
      cci[dst + e] = tci[src + e];
      cv[dst + e] = tcv[src + e];
    }
  }
}

template <int TAB>
constexpr size_t hash_smem() {
  return (size_t)WARPS * hash_smem_warp<TAB>();
}
static_assert(hash_smem<1024>() <= 232448, "hash-tier shared memory above the per-block limit");
constexpr size_t block_smem = (size_t)BTAB * sizeof(double) + (size_t)(BTAB + BTAB / 2) * sizeof(int);

struct Args {
  const DCsr *X;
  YRows y;
  const int *yci;
  const double *yv;
  const int *off;
  int *tci;
  double *tcv;
  int *cnt, *flags;
  cudaStream_t s;
};

// nr: the list's length, or (with nr_dev) a bound on the length held at
// nr_dev; retry / retry_n: where rows beyond TAB/2 distinct columns go.
template <int TAB>
void launch_hash(int nr, const int *list, const int *nr_dev, int *retry, int *retry_n, int max_blocks,
                 const Args &a) {
  static std::atomic<unsigned long long> attr{0};
  ensure_smem_attr(k_spgemm_hash<TAB>, (int)hash_smem<TAB>(), attr);
  const int grid = std::max(1, std::min(ceil_div(nr, WARPS), max_blocks));
  k_spgemm_hash<TAB><<<grid, TPB, hash_smem<TAB>(), a.s>>>(list, nr, nr_dev, a.X->rp, a.X->ci, a.X->v, a.y, a.yci,
                                                           a.yv, a.off, a.tci, a.tcv, a.cnt, a.flags, retry, retry_n);
  AMG_CHECK_LAUNCH();
}

}  // namespace

void spgemm(Mem &m, int *flags, const DCsr &X, const DCsr &Y, int ncols, DCsr &C, int level) {
  cudaStream_t s = m.stream;
  const int rows = X.n;
  const int ntiles = ceil_div(rows, TILE);
  const YRows y{Y.rp};
  Buf<int> ub(m, (size_t)rows + 1), off(m, (size_t)rows + 1), lists(m, (size_t)std::max(rows, 1));
  Buf<int8_t> tier(m, (size_t)std::max(rows, 1));
  Buf<int> meta(m, 2 * NTIER + 1);  // per-tier row counts, max ub of the T_OPT rows, list cursors
  AMG_CUDA(cudaMemsetAsync(meta.p, 0, sizeof(int) * (2 * NTIER + 1), s));
  {
    ProfScope ps(s, AMG_K_SPGEMM, 0.0, level);  // bookkeeping: no algorithmic bytes
    const double xavg = rows ? (double)X.nnz / rows : 0.0;
    const int G = xavg <= 8.0 ? 1 : xavg <= 24.0 ? 8 : 32;
    const int grid = std::max(1, std::min(ceil_div((int64_t)rows * G, TPB), kNumSMs * 32));
    if (G == 1) k_row_ub<1><<<grid, TPB, 0, s>>>(rows, X.rp, X.ci, y, ub.p, tier.p, meta.p, flags);
    else if (G == 8) k_row_ub<8><<<grid, TPB, 0, s>>>(rows, X.rp, X.ci, y, ub.p, tier.p, meta.p, flags);
    else k_row_ub<32><<<grid, TPB, 0, s>>>(rows, X.rp, X.ci, y, ub.p, tier.p, meta.p, flags);
    AMG_CHECK_LAUNCH();
  }
  // the scan's total and the tier counts come back in one synchronisation
  Buf<long long> ub_tot(m, 1);
  scan_counts_async(m, ub.p, off.p, rows, ub_tot.p);
  int hm[NTIER + 1];
  long long total_ub = 0;
  AMG_CUDA(cudaMemcpyAsync(hm, meta.p, sizeof(hm), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaMemcpyAsync(&total_ub, ub_tot.p, sizeof(total_ub), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  check_scan_total(total_ub);
  if (hm[NTIER] > (1 << 22)) {
    set_error("SpGEMM row product bound above 2^22 entries");
    throw Status{AMG_ERR_UNSUPPORTED};
  }
  int start[NTIER + 1];
  start[0] = 0;
  for (int t = 0; t < NTIER; ++t) start[t + 1] = start[t] + hm[t];
  Buf<int> startd(m, NTIER);
  AMG_CUDA(cudaMemcpyAsync(startd.p, start, sizeof(int) * NTIER, cudaMemcpyHostToDevice, s));
  {
    ProfScope ps(s, AMG_K_SPGEMM, 0.0, level);
    k_tier_scatter<<<std::max(1, ntiles), TPB, 0, s>>>(rows, tier.p, startd.p, meta.p + NTIER + 1, lists.p);
    AMG_CHECK_LAUNCH();
  }
  // rows of the optimistic tier that overflow a 256-slot table are retried
  // with 1024 slots, then with an exact table (a block per row: shared memory
  // for ub <= BTAB / 2, else a global scratch slice of gcap >= 2 ub slots)
  const int nopt = hm[T_OPT];
  const bool gtab = hm[NTIER] > BTAB / 2;
  int gcap = 2;
  while (gcap < 2 * std::max(hm[NTIER], 1)) gcap <<= 1;
  const int gblocks = std::max(1, std::min(nopt, kNumSMs * 2));
  Buf<int> retry, rn, gscr;
  Buf<double> gacc;
  if (nopt > 0) {
    retry = Buf<int>(m, 2 * (size_t)nopt);
    rn = Buf<int>(m, 2);
    AMG_CUDA(cudaMemsetAsync(rn.p, 0, 2 * sizeof(int), s));
    if (gtab) {
      gscr = Buf<int>(m, (size_t)gblocks * ((size_t)gcap + gcap / 2));
      gacc = Buf<double>(m, (size_t)gblocks * gcap);
    }
  }
  static std::atomic<unsigned long long> attr{0};
  ensure_smem_attr(k_spgemm_block<false>, (int)block_smem, attr);
  Buf<int> tci(m, (size_t)std::max<int64_t>(total_ub, 1));
  Buf<double> tcv(m, (size_t)std::max<int64_t>(total_ub, 1));
  Buf<int> cnt(m, (size_t)rows + 1);
  auto list = [&](int t) { return lists.p + start[t]; };
  const Args a{&X, y, Y.ci, Y.v, off.p, tci.p, tcv.p, cnt.p, flags, s};
  // Algorithmic bytes (the byte model of A_c = R (A P)): X and Y read once
  // here, C written once (charged to the compaction).
  const double xy_bytes = 4.0 * (rows + 1) + 12.0 * (double)X.nnz + 4.0 * (Y.n + 1) + 12.0 * (double)Y.nnz;
  {
    ProfScope ps(s, AMG_K_SPGEMM, xy_bytes, level);
    for (int t = T_THREAD; t <= T_THREAD; ++t) {
      if (hm[t] == 0) continue;
      const int grid = std::max(1, std::min(ceil_div(hm[t], TPB), kNumSMs * 16));
      k_spgemm_merge<<<grid, TPB, 0, s>>>(list(t), hm[t], X.rp, X.ci, X.v, y, Y.ci, Y.v, off.p, tci.p, tcv.p,
                                          cnt.p);
      AMG_CHECK_LAUNCH();
    }
    if (hm[0] > 0) {
      const int grid = std::max(1, std::min(ceil_div(hm[0], WARPS), kNumSMs * 32));
      k_spgemm_reg<<<grid, TPB, 0, s>>>(list(0), hm[0], X.rp, X.ci, X.v, y, Y.ci, Y.v, off.p, tci.p, tcv.p, cnt.p);
      AMG_CHECK_LAUNCH();
    }
    if (hm[1] > 0) launch_hash<128>(hm[1], list(1), nullptr, nullptr, nullptr, kNumSMs * 32, a);
    if (hm[2] > 0) launch_hash<256>(hm[2], list(2), nullptr, nullptr, nullptr, kNumSMs * 32, a);
    if (nopt > 0) {
      launch_hash<256>(nopt, list(T_OPT), nullptr, retry.p, rn.p, kNumSMs * 32, a);
      // a row with ub <= 512 has at most 512 columns: the 1024-slot set holds it
      const bool exact = hm[NTIER] > 512;
      launch_hash<1024>(nopt, retry.p, rn.p, exact ? retry.p + nopt : nullptr, rn.p + 1, kNumSMs * 2, a);
      if (exact && !gtab) {
        k_spgemm_block<false><<<gblocks, TPB, block_smem, s>>>(retry.p + nopt, nopt, rn.p + 1, X.rp, X.ci, X.v, y,
                                                               Y.ci, Y.v, off.p, tci.p, tcv.p, cnt.p, flags, nullptr,
                                                               nullptr, 0);
      } else if (exact) {
        k_spgemm_block<true><<<gblocks, TPB, 0, s>>>(retry.p + nopt, nopt, rn.p + 1, X.rp, X.ci, X.v, y, Y.ci, Y.v,
                                                     off.p, tci.p, tcv.p, cnt.p, flags, gscr.p, gacc.p, gcap);
      }
      AMG_CHECK_LAUNCH();
    }
  }
  C.n = rows;
  C.ncols = ncols;
  C.rp = m.get_n<int>((size_t)rows + 1);
  C.nnz = scan_counts(m, cnt.p, C.rp, rows);
  C.ci = m.get_n<int>(std::max<int64_t>(C.nnz, 1));
  C.v = m.get_n<double>(std::max<int64_t>(C.nnz, 1));
  {
    ProfScope ps(s, AMG_K_SPGEMM, 4.0 * (rows + 1) + 12.0 * C.nnz, level);
    if (C.nnz <= 12LL * rows)
      k_compact<8><<<std::max(1, std::min(ceil_div(rows, TPB / 8), kNumSMs * 32)), TPB, 0, s>>>(
          rows, off.p, tci.p, tcv.p, C.rp, C.ci, C.v);
    else
      k_compact<32><<<std::max(1, std::min(ceil_div(rows, WARPS), kNumSMs * 32)), TPB, 0, s>>>(
          rows, off.p, tci.p, tcv.p, C.rp, C.ci, C.v);
    AMG_CHECK_LAUNCH();
  }
}

}  // namespace amg

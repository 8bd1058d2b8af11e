// setup.cu -- Algorithm 1 (AMG_SetUp) on the GPU.
//
// Per level k, all on the device:
//   strength of connection   (Sec. 2.2, Eq. cla read as Ruge-Stueben, threshold filter)
//   PMIS C/F splitting       (Sec. 2.2; synchronous rounds, SplitMix64 measures)
//   direct interpolation     P = [W; I] in the original ordering (Eq. prolOperator)
//   R = P^T                  (CSR transpose, rows sorted)
//   A_{k+1} = R (A P)        (Eq. AcDef) by a hash-based SpGEMM with a canonical summation order
// and a dense Cholesky of the last level (Algorithm 1, direct factorisation).
//
// This translation unit is compiled with --fmad=false and uses explicit
// round-to-nearest intrinsics for every floating-point operation that
// decides the hierarchy, so that the hierarchy is reproducible bit for bit:
//   (A P)_{iJ} = sum over j ascending of a_ij * P_jJ, each product rounded,
//   then added left to right from 0; (A_c)_{IJ} likewise over i ascending in
//   row I of R.  A one-ulp difference at an exact strength tie would change
//   the next level's strong graph, so this order is part of the method here.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr int TPB = 256;

// ------------------------------------------------------------------ scan --
constexpr int SCAN_T = 256, SCAN_ITEMS = 8, SCAN_TILE = SCAN_T * SCAN_ITEMS;

__device__ __forceinline__ long long warp_incl_scan(long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the block total in *total.
__device__ long long block_excl_scan(long long v, long long *total) {
  __shared__ long long warp_tot[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long inc = warp_incl_scan(v);
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    long long t = lane < nw ? warp_tot[lane] : 0;
    long long ti = warp_incl_scan(t);
    if (lane < nw) warp_tot[lane] = ti - t;
    if (lane == nw - 1) warp_tot[31] = ti;
  }
  __syncthreads();
  long long res = warp_tot[w] + inc - v;
  *total = warp_tot[31];
  __syncthreads();
  return res;
}

__global__ void k_scan_reduce(const int *__restrict__ in, int n, long long *__restrict__ bsum) {
  long long s = 0;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  for (int t = threadIdx.x; t < SCAN_TILE; t += SCAN_T) {
    int64_t i = base + t;
    if (i < n) s += in[i];
  }
  long long tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_blocks(long long *bsum, int nb) {
  long long carry = 0;
  for (int c = 0; c < nb; c += SCAN_T) {
    int i = c + threadIdx.x;
    long long v = i < nb ? bsum[i] : 0, tot;
    long long ex = block_excl_scan(v, &tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_apply(const int *__restrict__ in, int n, const long long *__restrict__ boff,
                             int *__restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  long long v[SCAN_ITEMS], s = 0;
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    int64_t i = base + t;
    v[t] = i < n ? in[i] : 0;
    s += v[t];
  }
  long long tot;
  long long ex = block_excl_scan(s, &tot) + boff[blockIdx.x];
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    int64_t i = base + t;
    if (i < n) out[i] = static_cast<int>(ex);
    ex += v[t];
  }
}

__global__ void k_set_last(int *out, int n, const long long *total) { out[n] = static_cast<int>(*total); }

// Second pass of the two-kernel scan (at most kScan2Blocks tiles): each block
// first sums the totals of the tiles before it (so no pass over the block
// totals is needed), then scans its own tile; the last block writes out[n]
// and *total.
constexpr int kScan2Blocks = 4096;
__global__ void k_scan_apply2(const int *__restrict__ in, int n, const long long *__restrict__ bsum,
                              int *__restrict__ out, long long *__restrict__ total) {
  long long pre = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += SCAN_T) pre += bsum[b];
  long long boff;
  block_excl_scan(pre, &boff);
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  long long v[SCAN_ITEMS], s = 0;
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    int64_t i = base + t;
    v[t] = i < n ? in[i] : 0;
    s += v[t];
  }
  long long tot;
  long long ex = block_excl_scan(s, &tot) + boff;
#pragma unroll
  for (int t = 0; t < SCAN_ITEMS; ++t) {
    int64_t i = base + t;
    if (i < n) out[i] = static_cast<int>(ex);
    ex += v[t];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    out[n] = static_cast<int>(boff + tot);
    *total = boff + tot;
  }
}

// Whole exclusive scan in one block (small n): tiles in order with a carry;
// out[n] and *total receive the sum.
__global__ void k_scan_single(const int *__restrict__ in, int n, int *__restrict__ out, long long *total) {
  long long carry = 0;
  for (int64_t base0 = 0; base0 < n; base0 += SCAN_TILE) {
    const int64_t base = base0 + (int64_t)threadIdx.x * SCAN_ITEMS;
    long long v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int t = 0; t < SCAN_ITEMS; ++t) {
      const int64_t i = base + t;
      v[t] = i < n ? in[i] : 0;
      s += v[t];
    }
    long long tot;
    long long ex = block_excl_scan(s, &tot) + carry;
#pragma unroll
    for (int t = 0; t < SCAN_ITEMS; ++t) {
      const int64_t i = base + t;
      if (i < n) out[i] = static_cast<int>(ex);
      ex += v[t];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) {
    out[n] = static_cast<int>(carry);
    *total = carry;
  }
}

// ------------------------------------------------------- validation --
// flags[0]: malformed CSR, flags[1]: non-positive or missing diagonal,
// flags[2]: pattern not structurally symmetric, flags[3]: hash table overflow,
// flags[4]: Cholesky pivot <= 0
__global__ void k_validate(int n, int64_t nnz, const int *__restrict__ rp, const int *__restrict__ ci,
                           const double *__restrict__ a, int *flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = rp[i], e = rp[i + 1];
  if (b < 0 || e < b || e > nnz || (i == 0 && b != 0) || (i == n - 1 && e != nnz)) {
    flags[0] = 1;
    return;
  }
  bool diag = false;
  for (int p = b; p < e; ++p) {
    const int j = ci[p];
    if (j < 0 || j >= n || (p > b && j <= ci[p - 1])) {
      flags[0] = 1;
      return;
    }
    if (((unsigned long long)__double_as_longlong(a[p]) & 0x7ff0000000000000ULL) == 0x7ff0000000000000ULL) {
      flags[0] = 1;  // NaN or infinity
      return;
    }
    if (j == i) {
      diag = true;
      if (!(a[p] > 0.0)) flags[1] = 1;
    }
  }
  if (!diag) flags[1] = 1;
}

// ----------------------------------------------------------- strength --
// S[p] = 1 iff ci[p] != i, m_i = max_{k != i} (-a_ik) > 0 and -a[p] >= theta * m_i.
// Strength of connection, S[p] = 1 iff j = ci[p] != i and -a_ij >= thr_i =
// theta m_i, m_i = max_{k != i} -a_ik, only when m_i > 0.  The decisions are
// taken on bit patterns with integer instructions (FP64 comparisons kept
// GB300's FP64 pipe busy; FP64 instructions issue at a small fraction of the
// integer rate), exactly equivalent for finite values (the set-up rejects
// others):
//   m_i > 0 iff some off-diagonal a_ik is negative (nonzero), and then m_i is
//   the largest magnitude among them -- the largest magnitude bit pattern, as
//   non-negative doubles order as their patterns;
//   thr_i = fl(theta m_i) is formed in FP64 as before; for thr_i > 0,
//   -a_ij >= thr_i iff a_ij is negative and |a_ij|'s pattern >= thr_i's; for
//   thr_i = +0 (an underflow), iff a_ij <= 0.
constexpr unsigned long long kMagMask = 0x7fffffffffffffffULL;

__device__ __forceinline__ bool strong_entry(long long bits, unsigned long long tbits) {
  if (tbits == 0ULL) return bits < 0 || bits == 0;  // a_ij <= 0
  return bits < 0 && ((unsigned long long)bits & kMagMask) >= tbits;
}

__global__ void k_strength(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                           const double *__restrict__ a, double theta, uint8_t *__restrict__ S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = rp[i], e = rp[i + 1];
  unsigned long long mk = 0ULL;  // largest |a_ik| over negative off-diagonals (0: none)
  for (int p = b; p < e; ++p) {
    const long long bits = __double_as_longlong(a[p]);
    if (bits < 0 && ci[p] != i) mk = max(mk, (unsigned long long)bits & kMagMask);
  }
  const unsigned long long tbits = (unsigned long long)__double_as_longlong(__dmul_rn(theta, __longlong_as_double((long long)mk)));
  for (int p = b; p < e; ++p)
    S[p] = (mk != 0ULL && ci[p] != i && strong_entry(__double_as_longlong(a[p]), tbits)) ? 1 : 0;
}

// SplitMix64 (Steele, Lea & Flood 2014) evaluated at counter c: the c-th output
// of the generator seeded with `seed`.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
  uint64_t z = seed + c * 0x9E3779B97F4A7C15ull;
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

enum : int8_t { ST_U = 0, ST_C = 1, ST_F = 2, ST_NEWC = 3 };

__device__ __forceinline__ int find_col(const int *__restrict__ ci, int b, int e, int key) {
  int lo = b, hi = e - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int c = ci[mid];
    if (c == key) return mid;
    if (c < key) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

// ST[p] = S at the mirrored position (j, i): 1 iff i strongly influences j.
// lambda_i = |S_i^T| + u_i, u_i from the counter-based stream; points that
// influence nobody start as F.
__global__ void k_pmis_init(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                            const uint8_t *__restrict__ S, uint8_t *__restrict__ ST, double *__restrict__ lam,
                            int8_t *__restrict__ st, uint64_t seed, int level, int *flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cnt = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    uint8_t t = 0;
    if (j != i) {
      const int q = find_col(ci, rp[j], rp[j + 1], i);
      if (q < 0) flags[2] = 1;
      else t = S[q];
    }
    ST[p] = t;
    cnt += t;
  }
  const uint64_t c = ((uint64_t)(uint32_t)level << 32) + (uint64_t)(uint32_t)i + 1ull;
  const double u = (double)(splitmix64_at(seed, c) >> 11) * 0x1.0p-53;
  lam[i] = __dadd_rn((double)cnt, u);
  st[i] = cnt == 0 ? ST_F : ST_U;
}

// A measure's bit pattern as a signed integer.  Measures are finite and
// non-negative (|S_i^T| + u with u in [0, 1)), and for non-negative doubles the
// bit patterns order exactly as the values do, so the comparisons below take
// the same decisions as FP64 comparisons, on the integer pipe.
__device__ __forceinline__ long long lam_key(const double *__restrict__ lam, int i) {
  return __double_as_longlong(lam[i]);
}

// Selection step of a round: an undecided point beating every undecided
// strong neighbour (either direction) becomes a new C point.
__global__ void k_pmis_select(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                              const uint8_t *__restrict__ S, const uint8_t *__restrict__ ST,
                              const double *__restrict__ lam, const int8_t *__restrict__ st_old,
                              int8_t *__restrict__ st_new, const int *__restrict__ prev_undecided) {
  if (prev_undecided && *prev_undecided == 0) return;  // the splitting is complete
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int8_t s = st_old[i];
  if (s != ST_U) {
    st_new[i] = s;
    return;
  }
  const long long li = lam_key(lam, i);
  bool is_max = true;
  for (int p = rp[i]; p < rp[i + 1] && is_max; ++p) {
    if (!(S[p] | ST[p])) continue;
    const int j = ci[p];
    if (st_old[j] != ST_U) continue;
    const long long lj = lam_key(lam, j);
    if (lj > li || (lj == li && j > i)) is_max = false;
  }
  st_new[i] = is_max ? ST_NEWC : ST_U;
}

// Update step: undecided points that depend strongly on a new C point become
// F; new C points become C.  Counts the points still undecided.
__global__ void k_pmis_update(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                              const uint8_t *__restrict__ S, const int8_t *__restrict__ st_new,
                              int8_t *__restrict__ st_next, int *undecided,
                              const int *__restrict__ prev_undecided) {
  if (prev_undecided && *prev_undecided == 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool und = false;
  if (i < n) {
    const int8_t s = st_new[i];
    int8_t o = s;
    if (s == ST_NEWC) {
      o = ST_C;
    } else if (s == ST_U) {
      bool f = false;
      for (int p = rp[i]; p < rp[i + 1] && !f; ++p)
        if (S[p] && st_new[ci[p]] == ST_NEWC) f = true;
      o = f ? ST_F : ST_U;
      und = !f;
    }
    st_next[i] = o;
  }
  const unsigned b = __ballot_sync(0xffffffffu, und);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(undecided, __popc(b));
}

__global__ void k_cf_out(int n, const int8_t *__restrict__ st, int8_t *__restrict__ cf, int *__restrict__ isC) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = st[i] == ST_C;
  cf[i] = (int8_t)c;
  isC[i] = c;
}

// ---------------------------------------------- systems: nodal blocks --
// Unknowns are node-major: unknown i is component i % bs of node i / bs, and
// every coupled node pair stores its full bs x bs block (checked by
// k_block_check), so node I's rows share one column pattern of whole blocks.

// flags[5] = 1 if some node's rows are not whole, aligned bs x bs blocks.
__global__ void k_block_check(int nn, int bs, const int *__restrict__ rp, const int *__restrict__ ci, int *flags) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  const int b0 = rp[I * bs], len = rp[I * bs + 1] - b0;
  bool ok = len % bs == 0;
  for (int c = 1; c < bs && ok; ++c) ok = rp[I * bs + c + 1] - rp[I * bs + c] == len;
  for (int t = 0; ok && t < len; t += bs) {
    const int J = ci[b0 + t] / bs;
    for (int c = 0; c < bs && ok; ++c)
      for (int d = 0; d < bs && ok; ++d) ok = ci[rp[I * bs + c] + t + d] == J * bs + d;
  }
  if (!ok) flags[5] = 1;
}

// Node graph: nrp[I] = rp[bs I] / bs^2, nci = the node of each block.
__global__ void k_node_graph(int nn, int bs, const int *__restrict__ rp, const int *__restrict__ ci,
                             int *__restrict__ nrp, int *__restrict__ nci) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I > nn) return;
  const int b0 = rp[I * bs];
  nrp[I] = b0 / (bs * bs);
  if (I == nn) return;
  const int len = rp[I * bs + 1] - b0;
  for (int t = 0; t < len; t += bs) nci[b0 / (bs * bs) + t / bs] = ci[b0 + t] / bs;
}

// ||A_IJ||_F of the block at offset t of node I's rows: a^2 summed over the
// rows in order and the block's columns in ascending order.
__device__ __forceinline__ double block_fnorm(int I, int bs, int t, const int *__restrict__ rp,
                                              const double *__restrict__ a) {
  double f2 = 0.0;
  for (int c = 0; c < bs; ++c) {
    const int q = rp[I * bs + c] + t;
    for (int d = 0; d < bs; ++d) {
      const double v = a[q + d];
      f2 = __dadd_rn(f2, __dmul_rn(v, v));
    }
  }
  return __dsqrt_rn(f2);
}

// dn[I] = ||A_II||_F.
__global__ void k_block_dnorm(int nn, int bs, const int *__restrict__ rp, const int *__restrict__ ci,
                              const double *__restrict__ a, double *__restrict__ dn) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  const int b0 = rp[I * bs], len = rp[I * bs + 1] - b0;
  double f = 0.0;
  for (int t = 0; t < len; t += bs)
    if (ci[b0 + t] / bs == I) f = block_fnorm(I, bs, t, rp, a);
  dn[I] = f;
}

// Nodal strength: s_IJ = ||A_IJ||_F / sqrt(||A_II||_F ||A_JJ||_F); J strong
// for I iff J != I, m_I = max_{K != I} s_IK > 0 and s_IJ >= theta m_I.
// sv holds s_IJ per node-graph entry (scratch).
__global__ void k_block_strength(int nn, int bs, const int *__restrict__ rp, const double *__restrict__ a,
                                 const int *__restrict__ nrp, const int *__restrict__ nci,
                                 const double *__restrict__ dn, double theta, double *__restrict__ sv,
                                 uint8_t *__restrict__ SN) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  const int e0 = nrp[I], e1 = nrp[I + 1];
  const double dI = dn[I];
  double m = 0.0;
  for (int e = e0; e < e1; ++e) {
    const int J = nci[e];
    const double f = block_fnorm(I, bs, (e - e0) * bs, rp, a);
    const double den = __dsqrt_rn(__dmul_rn(dI, dn[J]));
    const double sIJ = den > 0.0 ? __ddiv_rn(f, den) : 0.0;
    sv[e] = sIJ;
    if (J != I && sIJ > m) m = sIJ;
  }
  const double thr = __dmul_rn(theta, m);
  for (int e = e0; e < e1; ++e) SN[e] = (nci[e] != I && m > 0.0 && sv[e] >= thr) ? 1 : 0;
}

// Every unknown takes its node's C/F label.
__global__ void k_cf_expand(int nn, int bs, const int8_t *__restrict__ st, int8_t *__restrict__ cf,
                            int *__restrict__ isC) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nn) return;
  const int c = st[I] == ST_C;
  for (int k = 0; k < bs; ++k) {
    cf[I * bs + k] = (int8_t)c;
    isC[I * bs + k] = c;
  }
}

// Unknown-wise strength: S[p] = 1 iff column ci[p] has row i's component,
// lies in another node J, and J strongly influences node I.
__global__ void k_dof_strength(int n, int bs, const int *__restrict__ rp, const int *__restrict__ ci,
                               const int *__restrict__ nrp, const uint8_t *__restrict__ SN, uint8_t *__restrict__ S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int I = i / bs, comp = i % bs, b = rp[i];
  for (int p = b; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    S[p] = (j % bs == comp && j / bs != I && SN[nrp[I] + (p - b) / bs]) ? 1 : 0;
  }
}

// ------------------------------------------------------ interpolation --
// -1 if v < 0, +1 if v > 0, 0 for +-0 and NaN (what the FP64 comparisons
// v < 0.0 and v > 0.0 decide), from the bit pattern: the interpolation
// kernels are bound by the FP64 pipe, which FP64 comparisons also occupy.
__device__ __forceinline__ int sign_class(double v) {
  const long long bits = __double_as_longlong(v);
  const unsigned long long mag = (unsigned long long)bits & 0x7fffffffffffffffULL;
  if (mag == 0ULL || mag > 0x7ff0000000000000ULL) return 0;
  return bits < 0 ? -1 : 1;
}

// RN(a / b) from y = RN(1 / b), by two FMA corrections:
//   q0 = RN(a y) is within two ulps of a / b (y carries half an ulp of error
//     and the product another half);
//   q1 = RN(q0 + r0 y) with r0 = RN(a - b q0) is within one ulp (a faithful
//     quotient): r0 y differs from a / b - q0 by about 2^-52 of |q0 - a/b|;
//   q = RN(q1 + r1 y) with r1 = a - b q1, exact in one FMA since q1 is
//     faithful, is RN(a / b) by Markstein's theorem (P. W. Markstein,
//     "Computation of elementary functions on the IBM RISC System/6000
//     processor", IBM J. Res. Develop. 34(1), 1990; the FMA division theorem
//     in Muller et al., Handbook of Floating-Point Arithmetic).
// So the result is the correctly rounded quotient a division gives, away
// from overflow and underflow: operands whose exponents leave a safe range
// (|x| in [2^-822, 2^776], where no remainder or product underflows) take
// the division itself.  Quotients that share a divisor then cost one
// correctly rounded reciprocal and a multiply and four FMAs each, where each
// division is a longer instruction sequence on GB300's narrow FP64 pipe.
__device__ __forceinline__ bool div_safe(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  return e > 200 && e < 1800;
}

__device__ __forceinline__ double div_by(double a, double b, double y) {
  const double q0 = __dmul_rn(a, y);
  if (!(div_safe(a) && div_safe(b) && div_safe(q0))) return __ddiv_rn(a, b);
  const double r0 = __fma_rn(-q0, b, a);
  const double q1 = __fma_rn(r0, y, q0);
  const double r1 = __fma_rn(-q1, b, a);
  return __fma_rn(r1, y, q1);
}

__global__ void k_interp_count(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                               const uint8_t *__restrict__ S, const int8_t *__restrict__ cf,
                               int *__restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (cf[i]) {
    cnt[i] = 1;
    return;
  }
  int c = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    if (j != i && S[p] && cf[j]) ++c;
  }
  cnt[i] = c;
}

// Direct interpolation with every sum over the row in ascending column order:
//   alpha = sum_{N_i} a^- / sum_{P_i} a^-,  beta = sum_{N_i} a^+ / sum_{P_i} a^+,
//   at = a_ii + sum_{N_i} a^+ when P_i holds no positive entry, else a_ii,
//   w_ij = -(alpha a_ij) / at for a_ij < 0, -(beta a_ij) / at for a_ij > 0
// (the product rounded, negated, then divided, as the formula reads).
// Systems (bs > 1, node-major unknowns): unknown-wise, row i sees only the
// columns of its own component (j % bs == i % bs).
__global__ void k_interp_fill(int n, int bs, const int *__restrict__ rp, const int *__restrict__ ci,
                              const double *__restrict__ a, const uint8_t *__restrict__ S,
                              const int8_t *__restrict__ cf, const int *__restrict__ cidx,
                              const int *__restrict__ prp, int *__restrict__ pci, double *__restrict__ pv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int pos = prp[i];
  if (cf[i]) {
    pci[pos] = cidx[i];
    pv[pos] = 1.0;
    return;
  }
  double aii = 0.0, sn_neg = 0.0, sn_pos = 0.0, sp_neg = 0.0, sp_pos = 0.0;
  int np = 0;
  const int b = rp[i], e = rp[i + 1];
  const int comp = i % bs;
  for (int p = b; p < e; ++p) {
    const int j = ci[p];
    const double v = a[p];
    if (j % bs != comp) continue;
    if (j == i) {
      aii = v;
      continue;
    }
    const int sg = sign_class(v);
    const bool strong_c = S[p] && cf[j];
    np += strong_c;
    if (sg) {  // one add into the sum of v's sign (the same additions, in the same order)
      const double sn = __dadd_rn(sg < 0 ? sn_neg : sn_pos, v);
      if (sg < 0) sn_neg = sn;
      else sn_pos = sn;
      if (strong_c) {
        const double sp = __dadd_rn(sg < 0 ? sp_neg : sp_pos, v);
        if (sg < 0) sp_neg = sp;
        else sp_pos = sp;
      }
    }
  }
  if (np == 0) return;
  const double alpha = sp_neg != 0.0 ? __ddiv_rn(sn_neg, sp_neg) : 0.0;
  const double beta = sp_pos != 0.0 ? __ddiv_rn(sn_pos, sp_pos) : 0.0;
  const double at = sp_pos != 0.0 ? aii : __dadd_rn(aii, sn_pos);
  const double yat = __drcp_rn(at);  // the row's weights share the divisor
  for (int p = b; p < e; ++p) {
    const int j = ci[p];
    if (j == i || !S[p] || !cf[j]) continue;
    const double v = a[p];
    const int sg = sign_class(v);
    const double w = sg ? div_by(-__dmul_rn(sg < 0 ? alpha : beta, v), at, yat) : 0.0;
    pci[pos] = cidx[j];
    pv[pos] = w;
    ++pos;
  }
}

// ------------------------------------------- warp-per-row variants --
// Used on small levels whose rows are long (mean length >= 12): a warp per row,
// lanes over the row's entries, so the dependent loads of one row are issued
// in parallel instead of walked by one thread.  Results are identical to the
// thread-per-row kernels (maxima, counts and flags do not depend on order;
// the interpolation's FP64 sums are still formed left to right by one lane).
#define WARP_ROW_BEGIN                                                              \
  const int lane = threadIdx.x & 31;                                                \
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);       \
  if (i >= n) return;

__global__ void k_strength_w(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                             const double *__restrict__ a, double theta, uint8_t *__restrict__ S) {
  WARP_ROW_BEGIN
  const int b = rp[i], e = rp[i + 1];
  unsigned long long mk = 0ULL;  // as in k_strength
  for (int p = b + lane; p < e; p += 32) {
    const long long bits = __double_as_longlong(a[p]);
    if (bits < 0 && ci[p] != i) mk = max(mk, (unsigned long long)bits & kMagMask);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) mk = max(mk, __shfl_xor_sync(0xffffffffu, mk, o));
  const unsigned long long tbits = (unsigned long long)__double_as_longlong(__dmul_rn(theta, __longlong_as_double((long long)mk)));
  for (int p = b + lane; p < e; p += 32)
    S[p] = (mk != 0ULL && ci[p] != i && strong_entry(__double_as_longlong(a[p]), tbits)) ? 1 : 0;
}

// The same with G lanes per row (rows of moderate length).
template <int G>
__global__ void __launch_bounds__(256) k_strength_g(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                    const double *__restrict__ a, double theta,
                                                    uint8_t *__restrict__ S) {
  const int lane = threadIdx.x & 31, sub = lane & (G - 1);
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G);  // rows in whole G-lane groups
  const bool live = i < n;
  const int b = live ? rp[i] : 0, e = live ? rp[i + 1] : 0;
  unsigned long long mk = 0ULL;
  for (int p = b + sub; p < e; p += G) {
    const long long bits = __double_as_longlong(a[p]);
    if (bits < 0 && ci[p] != i) mk = max(mk, (unsigned long long)bits & kMagMask);
  }
#pragma unroll
  for (int o = G / 2; o >= 1; o >>= 1) mk = max(mk, __shfl_xor_sync(0xffffffffu, mk, o));
  if (!live) return;
  const unsigned long long tbits = (unsigned long long)__double_as_longlong(__dmul_rn(theta, __longlong_as_double((long long)mk)));
  for (int p = b + sub; p < e; p += G)
    S[p] = (mk != 0ULL && ci[p] != i && strong_entry(__double_as_longlong(a[p]), tbits)) ? 1 : 0;
}

__global__ void k_pmis_init_w(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                              const uint8_t *__restrict__ S, uint8_t *__restrict__ ST, double *__restrict__ lam,
                              int8_t *__restrict__ st, uint64_t seed, int level, int *flags) {
  WARP_ROW_BEGIN
  int cnt = 0;
  for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
    const int j = ci[p];
    uint8_t t = 0;
    if (j != i) {
      const int q = find_col(ci, rp[j], rp[j + 1], i);
      if (q < 0) flags[2] = 1;
      else t = S[q];
    }
    ST[p] = t;
    cnt += t;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) {
    const uint64_t c = ((uint64_t)(uint32_t)level << 32) + (uint64_t)(uint32_t)i + 1ull;
    const double u = (double)(splitmix64_at(seed, c) >> 11) * 0x1.0p-53;
    lam[i] = __dadd_rn((double)cnt, u);
    st[i] = cnt == 0 ? ST_F : ST_U;
  }
}

__global__ void k_pmis_select_w(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                const uint8_t *__restrict__ S, const uint8_t *__restrict__ ST,
                                const double *__restrict__ lam, const int8_t *__restrict__ st_old,
                                int8_t *__restrict__ st_new, const int *__restrict__ prev_undecided) {
  if (prev_undecided && *prev_undecided == 0) return;
  WARP_ROW_BEGIN
  const int8_t s0 = st_old[i];
  if (s0 != ST_U) {
    if (lane == 0) st_new[i] = s0;
    return;
  }
  const long long li = lam_key(lam, i);
  bool beaten = false;
  for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
    if (!(S[p] | ST[p])) continue;
    const int j = ci[p];
    if (st_old[j] != ST_U) continue;
    const long long lj = lam_key(lam, j);
    if (lj > li || (lj == li && j > i)) beaten = true;
  }
  beaten = __any_sync(0xffffffffu, beaten);
  if (lane == 0) st_new[i] = beaten ? ST_U : ST_NEWC;
}

__global__ void k_pmis_update_w(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                const uint8_t *__restrict__ S, const int8_t *__restrict__ st_new,
                                int8_t *__restrict__ st_next, int *undecided,
                                const int *__restrict__ prev_undecided) {
  if (prev_undecided && *prev_undecided == 0) return;
  __shared__ int und_blk;
  if (threadIdx.x == 0) und_blk = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i < n) {
    const int8_t s0 = st_new[i];
    if (s0 == ST_U) {
      bool f = false;
      for (int p = rp[i] + lane; p < rp[i + 1]; p += 32)
        if (S[p] && st_new[ci[p]] == ST_NEWC) f = true;
      f = __any_sync(0xffffffffu, f);
      if (lane == 0) {
        st_next[i] = f ? ST_F : ST_U;
        if (!f) atomicAdd(&und_blk, 1);
      }
    } else if (lane == 0) {
      st_next[i] = s0 == ST_NEWC ? ST_C : s0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && und_blk) atomicAdd(undecided, und_blk);
}

// PMIS initialisation with G lanes per row, for large levels whose rows are of
// moderate length: a thread per row walked the row's mirror searches serially
// (128^3 level 1, 18 entries per row: 120 us with 8 lanes per row against
// 192 us).  The count combines over the row's lanes with shuffles every lane of
// the warp executes; one lane per row writes.  (The selection and update
// kernels were slower this way: 88 and 162 us against 38 and 53 us on level 0
// with 4 lanes per row.)
template <int G>
__global__ void __launch_bounds__(256) k_pmis_init_g(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                     const uint8_t *__restrict__ S, uint8_t *__restrict__ ST,
                                                     double *__restrict__ lam, int8_t *__restrict__ st, uint64_t seed,
                                                     int level, int *flags) {
  const int sub = threadIdx.x & (G - 1);
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G);
  const bool live = i < n;
  int cnt = 0;
  if (live) {
    for (int p = rp[i] + sub; p < rp[i + 1]; p += G) {
      const int j = ci[p];
      uint8_t t = 0;
      if (j != i) {
        const int q = find_col(ci, rp[j], rp[j + 1], i);
        if (q < 0) flags[2] = 1;
        else t = S[q];
      }
      ST[p] = t;
      cnt += t;
    }
  }
#pragma unroll
  for (int o = G / 2; o >= 1; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (live && sub == 0) {
    const uint64_t c = ((uint64_t)(uint32_t)level << 32) + (uint64_t)(uint32_t)i + 1ull;
    const double u = (double)(splitmix64_at(seed, c) >> 11) * 0x1.0p-53;
    lam[i] = __dadd_rn((double)cnt, u);
    st[i] = cnt == 0 ? ST_F : ST_U;
  }
}


__global__ void k_interp_count_w(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                 const uint8_t *__restrict__ S, const int8_t *__restrict__ cf,
                                 int *__restrict__ cnt) {
  WARP_ROW_BEGIN
  if (cf[i]) {
    if (lane == 0) cnt[i] = 1;
    return;
  }
  int c = 0;
  for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
    const int j = ci[p];
    if (j != i && S[p] && cf[j]) ++c;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[i] = c;
}

// Direct interpolation, warp per row: lanes stage a chunk of 32 entries in
// shared memory, lane 0 adds them in ascending column order (the canonical
// order of the thread-per-row kernel), then lanes form the weights.
__global__ void __launch_bounds__(256) k_interp_fill_w(int n, int bs, const int *__restrict__ rp, const int *__restrict__ ci,
                                                       const double *__restrict__ a, const uint8_t *__restrict__ S,
                                                       const int8_t *__restrict__ cf, const int *__restrict__ cidx,
                                                       const int *__restrict__ prp, int *__restrict__ pci,
                                                       double *__restrict__ pv) {
  __shared__ double sv[8][32];
  __shared__ uint8_t sk[8][32];  // bit 0: off-diagonal, bit 1: in P_i (strong C neighbour), bit 2: other component
  const int w = threadIdx.x >> 5;
  WARP_ROW_BEGIN
  int pos = prp[i];
  if (cf[i]) {
    if (lane == 0) {
      pci[pos] = cidx[i];
      pv[pos] = 1.0;
    }
    return;
  }
  const int b = rp[i], e = rp[i + 1];
  double aii = 0.0, sn_neg = 0.0, sn_pos = 0.0, sp_neg = 0.0, sp_pos = 0.0;
  int np = 0;
  for (int c0 = b; c0 < e; c0 += 32) {
    const int p = c0 + lane;
    if (p < e) {
      const int j = ci[p];
      sv[w][lane] = a[p];
      sk[w][lane] = (uint8_t)((j != i ? 1 : 0) | ((j != i && S[p] && cf[j]) ? 2 : 0) | (j % bs != i % bs ? 4 : 0));
    }
    __syncwarp();
    if (lane == 0) {
      const int cnt = min(32, e - c0);
      for (int t = 0; t < cnt; ++t) {
        const double v = sv[w][t];
        const uint8_t k = sk[w][t];
        if (k & 4) continue;
        if (!(k & 1)) {
          aii = v;
          continue;
        }
        const int sg = sign_class(v);
        np += (k & 2) ? 1 : 0;
        if (sg) {
          const double sn = __dadd_rn(sg < 0 ? sn_neg : sn_pos, v);
          if (sg < 0) sn_neg = sn;
          else sn_pos = sn;
          if (k & 2) {
            const double sp = __dadd_rn(sg < 0 ? sp_neg : sp_pos, v);
            if (sg < 0) sp_neg = sp;
            else sp_pos = sp;
          }
        }
      }
    }
    __syncwarp();
  }
  np = __shfl_sync(0xffffffffu, np, 0);
  if (np == 0) return;
  double alpha = 0.0, beta = 0.0, at = 0.0;
  if (lane == 0) {
    alpha = sp_neg != 0.0 ? __ddiv_rn(sn_neg, sp_neg) : 0.0;
    beta = sp_pos != 0.0 ? __ddiv_rn(sn_pos, sp_pos) : 0.0;
    at = sp_pos != 0.0 ? aii : __dadd_rn(aii, sn_pos);
  }
  alpha = __shfl_sync(0xffffffffu, alpha, 0);
  beta = __shfl_sync(0xffffffffu, beta, 0);
  at = __shfl_sync(0xffffffffu, at, 0);
  const double yat = __drcp_rn(at);  // the row's weights share the divisor
  for (int c0 = b; c0 < e; c0 += 32) {
    const int p = c0 + lane;
    bool sel = false;
    int j = 0;
    if (p < e) {
      j = ci[p];
      sel = j != i && S[p] && cf[j];
    }
    const unsigned bal = __ballot_sync(0xffffffffu, sel);
    if (sel) {
      const double v = a[p];
      const int sg = sign_class(v);
      const double wv = sg ? div_by(-__dmul_rn(sg < 0 ? alpha : beta, v), at, yat) : 0.0;
      const int q = pos + __popc(bal & ((1u << lane) - 1u));
      pci[q] = cidx[j];
      pv[q] = wv;
    }
    pos += __popc(bal);
  }
}

// -------------------------------------------- extended+i interpolation --
// Sec. 2.3's distance-two formula, evaluated in the order the oracle fixes:
//   Chat_i = C_i^S u (union over strong F neighbours k of C_k^S);
//   d_k = sum over row k (ascending l) of a_kl < 0 with l in Chat_i u {i};
//   at  = a_ii + over row i's off-diagonals in ascending order either
//         (a_ik a_ki) / d_k (strong F neighbour, a_ki < 0, d_k != 0), a_ik
//         (strong F neighbour with d_k = 0), or a_in (weak, not in Chat_i);
//   w_ij = -((a_ij + sum over strong F k ascending of (a_ik a_kj) / d_k) / at)
//         for j in Chat_i ascending, terms with a_kj >= 0 or d_k = 0 skipped.
// A warp per row builds Chat_i in a shared-memory hash set (the candidates:
// strong C neighbours and the strong C neighbours of each strong F
// neighbour), sorts its keys, then forms d_k (a lane per F neighbour), at
// (one lane, serial like the oracle) and the weights (a lane per j).
constexpr int kExtWarps = 4;  // most warps per block of the extended+i kernels

// sc[i] = number of strong C neighbours of row i.
__global__ void k_strong_c(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                           const uint8_t *__restrict__ S, const int8_t *__restrict__ cf, int *__restrict__ sc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) c += (ci[p] != i && S[p] && cf[ci[p]]) ? 1 : 0;
  sc[i] = c;
}

// mx[0] = largest candidate bound of a row (its strong C neighbours plus those of
// its strong F neighbours, repeats counted), mx[1] = longest row.
__global__ void k_ext_bound(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                            const uint8_t *__restrict__ S, const int8_t *__restrict__ cf,
                            const int *__restrict__ sc, int *mx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int bnd = 0, len = 0;
  if (i < n) {
    len = rp[i + 1] - rp[i];
    bnd = sc[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const int k = ci[p];
      if (k != i && S[p] && !cf[k]) bnd += sc[k];
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    bnd = max(bnd, __shfl_xor_sync(0xffffffffu, bnd, o));
    len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&mx[0], bnd);
    atomicMax(&mx[1], len);
  }
}

// Inserts key into the warp's open-addressing set (T slots, T a power of two
// above the row's candidate bound, so a free slot always exists).
__device__ __forceinline__ void ext_insert(int *table, int T, int key) {
  unsigned h = ((unsigned)key * 2654435761u) & (unsigned)(T - 1);
  for (;;) {
    const int prev = atomicCAS(&table[h], -1, key);
    if (prev == -1 || prev == key) return;
    h = (h + 1) & (unsigned)(T - 1);
  }
}

// Chat_i of F row i into keys[0..m) ascending; returns m (all lanes).  The
// strong F neighbours' rows are walked as one flattened sequence (lane u of
// a 32-product step takes product u of the chunk, found by a shuffle search
// over the chunk's prefix of row lengths), so the rows are gathered in
// parallel rather than one after another.
__device__ int ext_set(int i, int lane, const int *__restrict__ rp, const int *__restrict__ ci,
                       const uint8_t *__restrict__ S, const int8_t *__restrict__ cf, int *table, int *keys, int T) {
  for (int t = lane; t < T; t += 32) table[t] = -1;
  __syncwarp();
  const int b = rp[i], e = rp[i + 1];
  for (int c0 = b; c0 < e; c0 += 32) {
    const int p = c0 + lane;
    int ks = 0, len = 0;
    if (p < e) {
      const int k = ci[p];
      if (k != i && S[p]) {
        if (cf[k]) {
          ext_insert(table, T, k);
        } else {
          ks = rp[k];
          len = rp[k + 1] - ks;
        }
      }
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int excl = incl - len;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int u0 = 0; u0 < total; u0 += 32) {
      const int u = u0 + lane;
      int lo = 0;  // the last lane whose exclusive prefix is <= u
#pragma unroll
      for (int step = 16; step; step >>= 1) {
        const int ex = __shfl_sync(0xffffffffu, excl, lo + step);
        if (ex <= u) lo += step;
      }
      const int sks = __shfl_sync(0xffffffffu, ks, lo), sex = __shfl_sync(0xffffffffu, excl, lo);
      const int sk = __shfl_sync(0xffffffffu, p < e ? ci[min(p, e - 1)] : 0, lo);
      if (u < total) {
        const int q = sks + u - sex;
        const int l = ci[q];
        if (S[q] && l != sk && cf[l]) ext_insert(table, T, l);
      }
    }
  }
  __syncwarp();
  int m = 0;
  for (int t0 = 0; t0 < T; t0 += 32) {
    const int key = table[t0 + lane];
    const unsigned bal = __ballot_sync(0xffffffffu, key >= 0);
    if (key >= 0) keys[m + __popc(bal & ((1u << lane) - 1u))] = key;
    m += __popc(bal);
  }
  int np2 = 1;
  while (np2 < m) np2 <<= 1;
  for (int t = m + lane; t < np2; t += 32) keys[t] = INT_MAX;
  __syncwarp();
  for (int kk = 2; kk <= np2; kk <<= 1)
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      for (int t = lane; t < np2; t += 32) {
        const int u = t ^ jj;
        if (u > t) {
          const int x = keys[t], y = keys[u];
          if ((x > y) == ((t & kk) == 0)) {
            keys[t] = y;
            keys[u] = x;
          }
        }
      }
      __syncwarp();
    }
  return m;
}

// Rank of key among Chat_i's sorted keys, or -1: one probe sequence in the
// warp's hash set, whose slots hold, after ext_rank, the key's rank beside it.
__device__ __forceinline__ int key_pos(const int *table, const int *rank, int T, int key) {
  unsigned h = ((unsigned)key * 2654435761u) & (unsigned)(T - 1);
  for (;;) {
    const int kk = table[h];
    if (kk == key) return rank[h];
    if (kk < 0) return -1;
    h = (h + 1) & (unsigned)(T - 1);
  }
}

// rank[slot of keys[t]] = t for every key of the set.
__device__ __forceinline__ void ext_rank(int lane, const int *table, int *rank, int T, const int *keys, int m) {
  for (int t = lane; t < m; t += 32) {
    const int key = keys[t];
    unsigned h = ((unsigned)key * 2654435761u) & (unsigned)(T - 1);
    while (table[h] != key) h = (h + 1) & (unsigned)(T - 1);
    rank[h] = t;
  }
  __syncwarp();
}

// Shared memory per warp of k_ext_interp: num[T], dv[maxrow], cv[maxrow],
// bv[kExtBatch] (doubles), table[T], keys[T], rank[T], code[maxrow],
// flist[maxrow], bt[kExtBatch], bs[kExtBatch], sstart[kExtSegs + 1],
// sp[kExtSegs] (ints).
constexpr int kExtBatch = 512;  // numerator terms per batch of divisions
constexpr int kExtSegs = 128;   // F-neighbour segments per batch
__host__ __device__ inline size_t ext_warp_bytes(int T, int maxrow, bool fill = true) {
  if (!fill) return (size_t)2 * T * sizeof(int);  // the count pass: table[T], keys[T]
  const size_t b = (size_t)T * sizeof(double) + (size_t)2 * maxrow * sizeof(double) + (size_t)kExtBatch * sizeof(double) +
                   (size_t)3 * T * sizeof(int) + (size_t)2 * maxrow * sizeof(int) + (size_t)2 * kExtBatch * sizeof(int) +
                   (size_t)(2 * kExtSegs + 1) * sizeof(int);
  return (b + 15) & ~(size_t)15;  // keeps the next warp's doubles aligned
}

// FILL = false: cnt[i] = |Chat_i| (1 for C rows).  FILL = true: row i of P.
// GB300 issues FP64 per warp at a small fraction of the FP32 rate, so every
// FP64 step keeps its lanes dense:
//   the strong F neighbours k of row i are listed (ascending); a lane per k
//   forms d_k walking row k in ascending order;
//   a lane per entry p of row i forms its term of at -- (a_ik a_ki) / d_k for a
//   strong F neighbour (a_ki < 0, d_k != 0), a_ik for one with d_k = 0, a_in
//   for a weak coupling outside Chat_i -- and one lane adds them to a_ii in
//   the row's order;
//   the numerators start at a_ij (0 off the row); their terms
//   (a_ik a_kj) / d_k are gathered for the listed k in ascending order into
//   batches (qualifying entries of row k: a_kj < 0, j in Chat_i), divided with
//   all lanes busy, then added k segment by k segment (a column appears once
//   in a row, so each numerator takes its terms in ascending k);
//   w_ij = -(num / at).
// flags[0]: at = 0 met.
template <bool FILL>
__global__ void __launch_bounds__(kExtWarps * 32) k_ext_interp(int n, const int *__restrict__ rp,
                                                               const int *__restrict__ ci, const double *__restrict__ a,
                                                               const uint8_t *__restrict__ S,
                                                               const int8_t *__restrict__ cf,
                                                               const int *__restrict__ cidx, int T, int maxrow,
                                                               int *__restrict__ cnt, const int *__restrict__ prp,
                                                               int *__restrict__ pci, double *__restrict__ pv,
                                                               int *flags) {
  extern __shared__ __align__(16) unsigned char ext_smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  unsigned char *base = ext_smem + ext_warp_bytes(T, maxrow, FILL) * w;
  double *num = reinterpret_cast<double *>(base);
  double *dv = num + T;
  double *cv = dv + maxrow;
  double *bv = cv + maxrow;
  int *table = FILL ? reinterpret_cast<int *>(bv + kExtBatch) : reinterpret_cast<int *>(base);
  int *keys = table + T;
  int *rank = keys + T;
  int *code = rank + T;
  int *flist = code + maxrow;
  int *bt = flist + maxrow;
  int *bs = bt + kExtBatch;
  int *sstart = bs + kExtBatch;
  int *sp = sstart + kExtSegs + 1;
  const int wpb = blockDim.x >> 5;
  const int nw = gridDim.x * wpb;
  for (int i = blockIdx.x * wpb + w; i < n; i += nw) {
    if (cf[i]) {
      if (lane == 0) {
        if (FILL) {
          pci[prp[i]] = cidx[i];
          pv[prp[i]] = 1.0;
        } else {
          cnt[i] = 1;
        }
      }
      continue;
    }
    const int m = ext_set(i, lane, rp, ci, S, cf, table, keys, T);
    if (!FILL) {
      if (lane == 0) {
        cnt[i] = m;
        atomicMax(flags + 1, m);  // the largest |Chat_i|, which sizes the fill pass's set
      }
      __syncwarp();
      continue;
    }
    if (m == 0) continue;
    ext_rank(lane, table, rank, T, keys, m);
    const int b = rp[i], e = rp[i + 1];
    for (int t = lane; t < m; t += 32) num[t] = 0.0;
    // the strong F neighbours in ascending order
    int nf = 0;
    for (int c0 = b; c0 < e; c0 += 32) {
      const int p = c0 + lane;
      const bool f = p < e && ci[p] != i && S[p] && !cf[ci[p]];
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (f) flist[nf + __popc(bal & lt)] = p;
      nf += __popc(bal);
    }
    __syncwarp();
    for (int f = lane; f < nf; f += 32) {  // d_k, a lane per strong F neighbour
      const int p = flist[f], k = ci[p];
      double dk = 0.0;
      for (int q = rp[k]; q < rp[k + 1]; ++q) {
        const int l = ci[q];
        const double v = a[q];
        if (l != k && v < 0.0 && (l == i || key_pos(table, rank, T, l) >= 0)) dk = __dadd_rn(dk, v);
      }
      dv[p - b] = dk;
    }
    __syncwarp();
    for (int p = b + lane; p < e; p += 32) {  // each entry's term of at; numerators start at a_ij
      const int k = ci[p];
      int c = 0;  // bit 0: a term of at; bit 1: a strong F neighbour with d_k != 0
      double term = 0.0;
      if (k != i) {
        if (S[p] && !cf[k]) {
          const double dk = dv[p - b];
          if (dk != 0.0) {
            c = 2;
            const int q = find_col(ci, rp[k], rp[k + 1], i);
            if (q >= 0 && a[q] < 0.0) {
              term = __ddiv_rn(__dmul_rn(a[p], a[q]), dk);
              c |= 1;
            }
          } else {
            term = a[p];
            c = 1;
          }
        } else if (!S[p] && !(cf[k] && key_pos(table, rank, T, k) >= 0)) {
          term = a[p];
          c = 1;
        }
        const int t = key_pos(table, rank, T, k);
        if (t >= 0) num[t] = a[p];
      }
      code[p - b] = c;
      cv[p - b] = term;
    }
    __syncwarp();
    double at = 0.0;
    if (lane == 0) {
      const int pd = find_col(ci, b, e, i);
      at = pd >= 0 ? a[pd] : 0.0;
      for (int p = b; p < e; ++p)
        if (code[p - b] & 1) at = __dadd_rn(at, cv[p - b]);
      if (at == 0.0) flags[0] = 1;
    }
    at = __shfl_sync(0xffffffffu, at, 0);
    // numerator terms in batches: gather, divide (lanes dense), add in k order
    int fill = 0, nseg = 0;
    auto flush = [&]() {
      if (lane == 0) sstart[nseg] = fill;
      __syncwarp();
      for (int x = lane; x < fill; x += 32) {
        const int pp = sp[bs[x]];
        bv[x] = __ddiv_rn(__dmul_rn(a[pp], bv[x]), dv[pp - b]);
      }
      __syncwarp();
      for (int sg = 0; sg < nseg; ++sg) {
        for (int x = sstart[sg] + lane; x < sstart[sg + 1]; x += 32) num[bt[x]] = __dadd_rn(num[bt[x]], bv[x]);
        __syncwarp();
      }
      fill = 0;
      nseg = 0;
    };
    for (int f = 0; f < nf; ++f) {
      const int p = flist[f];
      if (!(code[p - b] & 2)) continue;
      const int k = ci[p];
      bool open = false;  // a segment of this k is open in the current batch
      for (int c0 = rp[k]; c0 < rp[k + 1]; c0 += 32) {
        if (fill + 32 > kExtBatch || (!open && nseg == kExtSegs)) {
          flush();
          open = false;
        }
        if (!open) {
          if (lane == 0) {
            sstart[nseg] = fill;
            sp[nseg] = p;
          }
          ++nseg;
          open = true;
        }
        const int q = c0 + lane;
        int t = -1;
        if (q < rp[k + 1] && a[q] < 0.0 && ci[q] != k) t = key_pos(table, rank, T, ci[q]);
        const unsigned bal = __ballot_sync(0xffffffffu, t >= 0);
        if (t >= 0) {
          const int x = fill + __popc(bal & lt);
          bt[x] = t;
          bv[x] = a[q];
          bs[x] = nseg - 1;
        }
        fill += __popc(bal);
      }
    }
    if (nseg > 0) flush();
    __syncwarp();
    const int off = prp[i];
    for (int t = lane; t < m; t += 32) {
      pci[off + t] = cidx[keys[t]];
      pv[off + t] = -__ddiv_rn(num[t], at);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------- transpose --
__global__ void k_col_count(int64_t nnz, const int *__restrict__ ci, int *__restrict__ cnt) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnz) atomicAdd(&cnt[ci[p]], 1);
}

__global__ void k_transpose_scatter(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                    const double *__restrict__ v, int *__restrict__ fill, int *__restrict__ tci,
                                    double *__restrict__ tv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int q = atomicAdd(&fill[ci[p]], 1);
    tci[q] = i;
    tv[q] = v[p];
  }
}

// Rows of (src_ci, src_v) sorted by column into (dst_ci, dst_v); a warp per
// row, rank of each entry = number of smaller keys in its row (keys distinct).
// Sorts each row of the scattered transpose by column: an entry's position is
// its rank among the row's (distinct) columns.  G lanes per row (8 for short
// rows, so that a warp holds several rows; 32 for long ones).
template <int G>
__global__ void k_sort_rows(int m, const int *__restrict__ rp, const int *__restrict__ src_ci,
                            const double *__restrict__ src_v, int *__restrict__ dst_ci, double *__restrict__ dst_v) {
  const int sub = threadIdx.x & (G - 1);
  const int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G);
  if (row >= m) return;
  const int b = rp[row], e = rp[row + 1];
  for (int p = b + sub; p < e; p += G) {
    const int key = src_ci[p];
    int rank = 0;
    for (int q = b; q < e; ++q) rank += src_ci[q] < key;
    dst_ci[b + rank] = key;
    dst_v[b + rank] = src_v[p];
  }
}

// ------------------------------------------------------------ dense LL^T --
__global__ void k_to_dense(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                           const double *__restrict__ v, double *__restrict__ M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) M[(size_t)i * n + ci[p]] = v[p];
}

// Right-looking dense Cholesky in one block; lower factor in place, upper
// triangle zeroed.  A pivot <= 0 sets flags[4] and stops.
__global__ void k_cholesky(int n, double *M, int *flags) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double d = M[(size_t)j * n + j];
      if (!(d > 0.0)) {
        bad = 1;
        flags[4] = 1;
      } else {
        M[(size_t)j * n + j] = sqrt(d);
      }
    }
    __syncthreads();
    if (bad) return;
    const double ljj = M[(size_t)j * n + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) M[(size_t)i * n + j] = __ddiv_rn(M[(size_t)i * n + j], ljj);
    __syncthreads();
    const int m = n - j - 1;
    for (int64_t t = threadIdx.x; t < (int64_t)m * m; t += blockDim.x) {
      const int i = j + 1 + (int)(t / m), k = j + 1 + (int)(t % m);
      if (k <= i) M[(size_t)i * n + k] = __dadd_rn(M[(size_t)i * n + k], -__dmul_rn(M[(size_t)i * n + j], M[(size_t)k * n + j]));
    }
    __syncthreads();
  }
  for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
    const int i = (int)(t / n), k = (int)(t % n);
    if (k > i) M[t] = 0.0;
  }
}

// Inverse of the lower Cholesky factor, column by column (thread j solves
// L x = e_j by forward substitution); the last level's solve then applies
// L^-1 and L^-T as two dense triangular products.
__global__ void k_tri_inverse(int n, const double *__restrict__ L, double *__restrict__ Li) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int i = 0; i < j; ++i) Li[(size_t)i * n + j] = 0.0;
  for (int i = j; i < n; ++i) {
    double s = (i == j) ? 1.0 : 0.0;
    for (int k = j; k < i; ++k) s = __dadd_rn(s, -__dmul_rn(L[(size_t)i * n + k], Li[(size_t)k * n + j]));
    Li[(size_t)i * n + j] = __ddiv_rn(s, L[(size_t)i * n + i]);
  }
}

// ------------------------------------------------------------ host side --
struct Flags {
  int *d = nullptr;
  int h[8] = {};
};

void read_flags(Mem &m, Flags &f) {
  AMG_CUDA(cudaMemcpyAsync(f.h, f.d, sizeof(f.h), cudaMemcpyDeviceToHost, m.stream));
  AMG_CUDA(cudaStreamSynchronize(m.stream));
}


void fail(int code, const char *msg) {
  set_error("%s", msg);
  throw Status{code};
}

// R = P^T (ncols rows), each row listing fine indices in ascending order.
void transpose(Mem &m, const DCsr &P, int ncols, DCsr &R) {
  cudaStream_t s = m.stream;
  Buf<int> cnt(m, (size_t)ncols + 1);
  AMG_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int) * ((size_t)ncols + 1), s));
  if (P.nnz) {
    ProfScope ps(s, AMG_K_TRANSPOSE, 4.0 * P.nnz + 4.0 * ncols);
    k_col_count<<<ceil_div(P.nnz, TPB), TPB, 0, s>>>(P.nnz, P.ci, cnt.p);
    AMG_CHECK_LAUNCH();
  }
  R.n = ncols;
  R.ncols = P.n;
  R.nnz = P.nnz;
  R.rp = m.get_n<int>((size_t)ncols + 1);
  {
    Buf<long long> tot(m, 1);  // R.nnz = P.nnz is known: no read-back
    scan_counts_async(m, cnt.p, R.rp, ncols, tot.p);
  }
  R.ci = m.get_n<int>(std::max<int64_t>(R.nnz, 1));
  R.v = m.get_n<double>(std::max<int64_t>(R.nnz, 1));
  Buf<int> fill(m, (size_t)ncols + 1);
  AMG_CUDA(cudaMemcpyAsync(fill.p, R.rp, sizeof(int) * ((size_t)ncols + 1), cudaMemcpyDeviceToDevice, s));
  Buf<int> tci(m, std::max<int64_t>(R.nnz, 1));
  Buf<double> tv(m, std::max<int64_t>(R.nnz, 1));
  {
    ProfScope ps(s, AMG_K_TRANSPOSE, 4.0 * (P.n + 1) + 24.0 * P.nnz + 4.0 * ncols);
    k_transpose_scatter<<<ceil_div(P.n, TPB), TPB, 0, s>>>(P.n, P.rp, P.ci, P.v, fill.p, tci.p, tv.p);
    AMG_CHECK_LAUNCH();
  }
  {
    ProfScope ps(s, AMG_K_TRANSPOSE, 4.0 * (ncols + 1) + 24.0 * P.nnz);
    if (P.nnz <= 12LL * ncols)
      k_sort_rows<8><<<ceil_div((int64_t)ncols * 8, TPB), TPB, 0, s>>>(ncols, R.rp, tci.p, tv.p, R.ci, R.v);
    else
      k_sort_rows<32><<<ceil_div((int64_t)ncols * 32, TPB), TPB, 0, s>>>(ncols, R.rp, tci.p, tv.p, R.ci, R.v);
    AMG_CHECK_LAUNCH();
  }
}

void free_csr(Mem &m, DCsr &c) {
  if (c.rp) m.put(c.rp, sizeof(int) * ((size_t)c.n + 1));
  if (c.ci) m.put(c.ci, sizeof(int) * (size_t)std::max<int64_t>(c.nnz, 1));
  if (c.v) m.put(c.v, sizeof(double) * (size_t)std::max<int64_t>(c.nnz, 1));
  c.rp = c.ci = nullptr;
  c.v = nullptr;
}

}  // namespace

void csr_transpose(Mem &m, const DCsr &P, int ncols, DCsr &R) { transpose(m, P, ncols, R); }

// Exclusive scan of n counts into out[0..n] (out[n] = total), enqueued on the
// stream without waiting; *total_dev receives the total.
void scan_counts_async(Mem &m, const int *in, int *out, int n, long long *total_dev) {
  cudaStream_t s = m.stream;
  const int nb = std::max(1, ceil_div(n, SCAN_TILE));
  ProfScope ps(s, AMG_K_SETUP_OTHER, 8.0 * n + 8.0 * nb);
  if (n <= SCAN_TILE) {
    k_scan_single<<<1, SCAN_T, 0, s>>>(in, n, out, total_dev);
    AMG_CHECK_LAUNCH();
  } else if (nb <= kScan2Blocks) {
    Buf<long long> bsum(m, (size_t)nb);  // released in stream order
    k_scan_reduce<<<nb, SCAN_T, 0, s>>>(in, n, bsum.p);
    AMG_CHECK_LAUNCH();
    k_scan_apply2<<<nb, SCAN_T, 0, s>>>(in, n, bsum.p, out, total_dev);
    AMG_CHECK_LAUNCH();
  } else {
    Buf<long long> bsum(m, (size_t)nb + 1);  // released in stream order
    k_scan_reduce<<<nb, SCAN_T, 0, s>>>(in, n, bsum.p);
    AMG_CHECK_LAUNCH();
    k_scan_blocks<<<1, SCAN_T, 0, s>>>(bsum.p, nb);
    AMG_CHECK_LAUNCH();
    k_scan_apply<<<nb, SCAN_T, 0, s>>>(in, n, bsum.p, out);
    AMG_CHECK_LAUNCH();
    k_set_last<<<1, 1, 0, s>>>(out, n, bsum.p + nb);
    AMG_CHECK_LAUNCH();
    AMG_CUDA(cudaMemcpyAsync(total_dev, bsum.p + nb, sizeof(long long), cudaMemcpyDeviceToDevice, s));
  }
}

// Totals of 2^31 - 1 or more fail (the offsets are int32).
void check_scan_total(long long total) {
  if (total >= (1LL << 31) - 1) fail(AMG_ERR_UNSUPPORTED, "more than 2^31-1 nonzeros in one matrix");
}

// Exclusive scan of n counts into out[0..n] (out[n] = total); returns the
// total, read back after the scan has been written (one synchronisation).
// Totals of 2^31 - 1 or more fail; out is then incomplete and must not be used.
int64_t scan_counts(Mem &m, const int *in, int *out, int n) {
  cudaStream_t s = m.stream;
  Buf<long long> tot(m, 1);
  scan_counts_async(m, in, out, n, tot.p);
  long long total = 0;
  AMG_CUDA(cudaMemcpyAsync(&total, tot.p, sizeof(total), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  check_scan_total(total);
  return total;
}

void free_level_csr(Mem &m, DCsr &c) { free_csr(m, c); }

void build_hierarchy(amg_hierarchy *h, const amg_csr &Ain) {
  Mem &m = h->mem;
  cudaStream_t s = m.stream;
  const amg_params &prm = h->prm;
  const int n0 = Ain.n;
  const int64_t nnz0 = Ain.nnz;

  Flags fl;
  Buf<int> flags_buf(m, 8);
  fl.d = flags_buf.p;
  auto sync_flags = [&]() {
    read_flags(m, fl);
    if (fl.h[3]) fail(AMG_ERR_UNSUPPORTED, "SpGEMM hash table overflow");
  };
  AMG_CUDA(cudaMemsetAsync(fl.d, 0, sizeof(int) * 8, s));

  // level 0: copy A
  DCsr &A0 = h->lev[0].A;
  A0.n = A0.ncols = n0;
  A0.nnz = nnz0;
  A0.rp = m.get_n<int>((size_t)n0 + 1);
  A0.ci = m.get_n<int>(std::max<int64_t>(nnz0, 1));
  A0.v = m.get_n<double>(std::max<int64_t>(nnz0, 1));
  const cudaMemcpyKind kind = Ain.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  AMG_CUDA(cudaMemcpyAsync(A0.rp, Ain.rowptr, sizeof(int) * ((size_t)n0 + 1), kind, s));
  AMG_CUDA(cudaMemcpyAsync(A0.ci, Ain.colidx, sizeof(int) * (size_t)nnz0, kind, s));
  AMG_CUDA(cudaMemcpyAsync(A0.v, Ain.val, sizeof(double) * (size_t)nnz0, kind, s));
  {
    ProfScope ps(s, AMG_K_STRENGTH, 4.0 * (n0 + 1) + 12.0 * nnz0);
    k_validate<<<ceil_div(n0, TPB), TPB, 0, s>>>(n0, nnz0, A0.rp, A0.ci, A0.v, fl.d);
    AMG_CHECK_LAUNCH();
  }
  sync_flags();
  if (fl.h[0]) fail(AMG_ERR_INVALID_ARG, "malformed CSR (row pointers, column range, unsorted columns or a non-finite value)");
  if (fl.h[1]) fail(AMG_ERR_NOT_SPD, "a diagonal entry is missing or not positive");

  int k = 0;
  for (;;) {
    Level &L = h->lev[k];
    const DCsr &A = L.A;
    const int n = A.n;
    bool last = n <= prm.max_coarse || k == prm.max_levels - 1;
    // Long rows on a level too small to fill the GPU with a thread per row:
    // the warp-per-row kernels (the interpolation's serial FP64 sums only on
    // the smallest levels, where FP64 issue slots are not the limit).
    const bool wide = (double)A.nnz >= 12.0 * n && n < (1 << 18);
    // The interpolation's FP64 sums are serial per row, and FP64 instructions
    // issue per warp: a thread per row keeps them lane-dense (the 128^3
    // level 3, 24K rows of 60 entries: 113 us against 201 us warp per row,
    // where one lane in 32 issues them); below 8192 rows there are too few rows
    // for that and the warp per row wins (levels 4-6: 40, 22, 14 us against
    // 110, 96, 49 us).  The other set-up kernels (integer work) keep `wide`.
    const bool wide_interp = wide && n < 8192;
    const int gw = ceil_div((int64_t)n * 32, TPB);
    Buf<uint8_t> S, ST;
    Buf<int> cidx;
    int nc = 0;
    if (!last) {
      const int bs = prm.block_size;
      S = Buf<uint8_t>(m, std::max<int64_t>(A.nnz, 1));
      const int g = ceil_div(n, TPB);
      // The graph PMIS runs on: the unknowns (bs = 1) or the nodes (bs > 1).
      int gn = n;
      int64_t gnnz = A.nnz;
      const int *grp = A.rp, *gci = A.ci;
      const uint8_t *gS = S.p;
      Buf<int> nrp, nci;
      Buf<uint8_t> SN;
      if (bs == 1) {
        ProfScope ps(s, AMG_K_STRENGTH, 4.0 * (n + 1) + 13.0 * A.nnz, k);
        // integer work only: rows of 12 to 32 entries with 8 lanes per row, longer
        // ones with a warp (128^3 level 1, 18 entries: 148 us with a thread per row,
        // 144 us with a warp; level 2, 46 entries: 44 us with a warp)
        const double avg = n ? (double)A.nnz / n : 0.0;
        if (avg >= 12.0 && avg <= 32.0)
          k_strength_g<8><<<ceil_div((int64_t)n * 8, TPB), TPB, 0, s>>>(n, A.rp, A.ci, A.v, prm.theta, S.p);
        else if (avg > 32.0)
          k_strength_w<<<gw, TPB, 0, s>>>(n, A.rp, A.ci, A.v, prm.theta, S.p);
        else k_strength<<<g, TPB, 0, s>>>(n, A.rp, A.ci, A.v, prm.theta, S.p);
        AMG_CHECK_LAUNCH();
      } else {
        const int nn = n / bs;
        const int gnn = ceil_div(nn, TPB);
        {
          ProfScope ps(s, AMG_K_STRENGTH, 4.0 * (n + 1) + 4.0 * A.nnz, k);
          k_block_check<<<gnn, TPB, 0, s>>>(nn, bs, A.rp, A.ci, fl.d);
          AMG_CHECK_LAUNCH();
        }
        sync_flags();
        if (fl.h[5]) {
          if (k == 0) fail(AMG_ERR_INVALID_ARG, "block_size > 1 needs every coupled node pair stored as a full block");
          fail(AMG_ERR_SETUP, "a coarse operator lost its block structure");
        }
        const int64_t nne = A.nnz / ((int64_t)bs * bs);
        nrp = Buf<int>(m, (size_t)nn + 1);
        nci = Buf<int>(m, std::max<int64_t>(nne, 1));
        SN = Buf<uint8_t>(m, std::max<int64_t>(nne, 1));
        Buf<double> dn(m, nn), sv(m, std::max<int64_t>(nne, 1));
        {
          ProfScope ps(s, AMG_K_STRENGTH, 4.0 * (n + 1) + 12.0 * A.nnz + 8.0 * nn + 13.0 * nne, k);
          k_node_graph<<<ceil_div(nn + 1, TPB), TPB, 0, s>>>(nn, bs, A.rp, A.ci, nrp.p, nci.p);
          AMG_CHECK_LAUNCH();
          k_block_dnorm<<<gnn, TPB, 0, s>>>(nn, bs, A.rp, A.ci, A.v, dn.p);
          AMG_CHECK_LAUNCH();
          k_block_strength<<<gnn, TPB, 0, s>>>(nn, bs, A.rp, A.v, nrp.p, nci.p, dn.p, prm.theta, sv.p, SN.p);
          AMG_CHECK_LAUNCH();
          k_dof_strength<<<g, TPB, 0, s>>>(n, bs, A.rp, A.ci, nrp.p, SN.p, S.p);
          AMG_CHECK_LAUNCH();
        }
        gn = nn;
        gnnz = nne;
        grp = nrp.p;
        gci = nci.p;
        gS = SN.p;
      }
      const bool gwide = (double)gnnz >= 12.0 * gn && gn < (1 << 18);
      const double gavg = gn ? (double)gnnz / gn : 0.0;
      const int gg = ceil_div(gn, TPB), ggw = ceil_div((int64_t)gn * 32, TPB);
      const int gg8 = ceil_div((int64_t)gn * 8, TPB);
      const double nz = (double)gnnz, rows = 4.0 * (gn + 1);
      ST = Buf<uint8_t>(m, std::max<int64_t>(gnnz, 1));
      Buf<double> lam(m, gn);
      Buf<int8_t> st0(m, gn), st1(m, gn);
      {
        ProfScope ps(s, AMG_K_STRENGTH, rows + 6.0 * nz + 9.0 * gn, k);
        if (gwide) k_pmis_init_w<<<ggw, TPB, 0, s>>>(gn, grp, gci, gS, ST.p, lam.p, st0.p, prm.seed, k, fl.d);
        else if (gavg >= 12.0) k_pmis_init_g<8><<<gg8, TPB, 0, s>>>(gn, grp, gci, gS, ST.p, lam.p, st0.p, prm.seed, k, fl.d);
        else k_pmis_init<<<gg, TPB, 0, s>>>(gn, grp, gci, gS, ST.p, lam.p, st0.p, prm.seed, k, fl.d);
        AMG_CHECK_LAUNCH();
      }
      // Rounds run kPmisBatch at a time between host checks.  Round r's
      // kernels return at once when round r - 1 left no point undecided (a
      // round after that would change nothing), so the batch may run past the
      // end; und[r] counts the points round r leaves undecided, and the last
      // one is read with the error flags (one synchronisation per batch).
      constexpr int kPmisBatch = 8;
      Buf<int> und(m, kPmisBatch);
      for (int round = 0;; round += kPmisBatch) {
        if (round > gn + 1) fail(AMG_ERR_SETUP, "PMIS did not terminate");
        AMG_CUDA(cudaMemsetAsync(und.p, 0, kPmisBatch * sizeof(int), s));
        for (int sub = 0; sub < kPmisBatch; ++sub) {
          const int *prev = sub ? und.p + sub - 1 : nullptr;
          {
            ProfScope ps(s, AMG_K_PMIS, rows + 6.0 * nz + 10.0 * gn, k);
            if (gwide) k_pmis_select_w<<<ggw, TPB, 0, s>>>(gn, grp, gci, gS, ST.p, lam.p, st0.p, st1.p, prev);
            else k_pmis_select<<<gg, TPB, 0, s>>>(gn, grp, gci, gS, ST.p, lam.p, st0.p, st1.p, prev);
            AMG_CHECK_LAUNCH();
          }
          {
            ProfScope ps(s, AMG_K_PMIS, rows + 5.0 * nz + 2.0 * gn, k);
            if (gwide) k_pmis_update_w<<<ggw, TPB, 0, s>>>(gn, grp, gci, gS, st1.p, st0.p, und.p + sub, prev);
            else k_pmis_update<<<gg, TPB, 0, s>>>(gn, grp, gci, gS, st1.p, st0.p, und.p + sub, prev);
            AMG_CHECK_LAUNCH();
          }
        }
        int left = 0;
        AMG_CUDA(cudaMemcpyAsync(&left, und.p + kPmisBatch - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        sync_flags();
        if (fl.h[2]) fail(AMG_ERR_INVALID_ARG, "matrix pattern is not structurally symmetric");
        if (left == 0) break;
      }
      L.cf = m.get_n<int8_t>(n);
      Buf<int> isC(m, n);
      {
        ProfScope ps(s, AMG_K_PMIS, 6.0 * n, k);
        if (bs == 1) k_cf_out<<<g, TPB, 0, s>>>(n, st0.p, L.cf, isC.p);
        else k_cf_expand<<<gg, TPB, 0, s>>>(gn, bs, st0.p, L.cf, isC.p);
        AMG_CHECK_LAUNCH();
      }
      cidx = Buf<int>(m, (size_t)n + 1);
      nc = (int)scan_counts(m, isC.p, cidx.p, n);
      if (nc == 0 || (double)nc > 0.9 * (double)n) {
        last = true;  // stalled coarsening
        m.put(L.cf, n);
        L.cf = nullptr;
      }
    }
    if (last) {
      if (n > kMaxDense) fail(AMG_ERR_SETUP, "coarsening stalled on a level too large for the dense factor");
      h->nL = n;
      h->L = m.get_n<double>((size_t)n * n);
      AMG_CUDA(cudaMemsetAsync(h->L, 0, sizeof(double) * (size_t)n * n, s));
      {
        ProfScope ps(s, AMG_K_SETUP_OTHER, 4.0 * (n + 1) + 12.0 * A.nnz + 16.0 * (double)n * n, k);
        k_to_dense<<<ceil_div(n, TPB), TPB, 0, s>>>(n, A.rp, A.ci, A.v, h->L);
        AMG_CHECK_LAUNCH();
        k_cholesky<<<1, 256, 0, s>>>(n, h->L, fl.d);
        AMG_CHECK_LAUNCH();
      }
      sync_flags();
      if (fl.h[4]) fail(AMG_ERR_NOT_SPD, "dense Cholesky of the last level met a non-positive pivot");
      h->Linv = m.get_n<double>((size_t)n * n);
      {
        ProfScope ps(s, AMG_K_SETUP_OTHER, 16.0 * (double)n * n, k);
        k_tri_inverse<<<ceil_div(n, 64), 64, 0, s>>>(n, h->L, h->Linv);
        AMG_CHECK_LAUNCH();
      }
      h->nlevels = k + 1;
      break;
    }
    // interpolation
    const int g = ceil_div(n, TPB);
    DCsr &P = L.P;
    if (prm.interp == AMG_INTERP_EXT) {
      Buf<int> mx(m, 2), eflag(m, 2), pcnt(m, n);  // eflag[0]: at = 0; eflag[1]: largest |Chat_i|
      AMG_CUDA(cudaMemsetAsync(mx.p, 0, 2 * sizeof(int), s));
      AMG_CUDA(cudaMemsetAsync(eflag.p, 0, sizeof(int), s));
      {
        ProfScope ps(s, AMG_K_INTERP, 8.0 * (n + 1) + 10.0 * A.nnz + 2.0 * n, k);
        k_strong_c<<<g, TPB, 0, s>>>(n, A.rp, A.ci, S.p, L.cf, pcnt.p);
        AMG_CHECK_LAUNCH();
        k_ext_bound<<<g, TPB, 0, s>>>(n, A.rp, A.ci, S.p, L.cf, pcnt.p, mx.p);
        AMG_CHECK_LAUNCH();
      }
      int hmx[2];
      AMG_CUDA(cudaMemcpyAsync(hmx, mx.p, sizeof(hmx), cudaMemcpyDeviceToHost, s));
      AMG_CUDA(cudaStreamSynchronize(s));
      // the count pass sizes its set by the candidate bound (repeats counted),
      // the fill pass by the largest distinct count the count pass found
      auto geometry = [&](int T, bool fill, int *wpb_out) {
        const size_t per = ext_warp_bytes(T, std::max(hmx[1], 1), fill);
        const int wpb = (int)std::max<size_t>(1, std::min<size_t>(kExtWarps, (size_t)(200 * 1024) / per));
        if (per * wpb > 200 * 1024)
          fail(AMG_ERR_UNSUPPORTED, "extended+i: a row's interpolatory candidates exceed the shared-memory set");
        *wpb_out = wpb;
        return per * wpb;
      };
      int T = 32;
      while (T <= hmx[0]) T <<= 1;  // a free slot always remains
      static std::atomic<unsigned long long> attr_c{0}, attr_f{0};
      ensure_smem_attr(k_ext_interp<false>, 200 * 1024, attr_c);
      ensure_smem_attr(k_ext_interp<true>, 200 * 1024, attr_f);
      AMG_CUDA(cudaMemsetAsync(eflag.p, 0, 2 * sizeof(int), s));
      {
        int wpb = 1;
        const size_t smem = geometry(T, false, &wpb);
        const int grid = std::max(1, std::min(ceil_div(n, wpb), kNumSMs * 16));
        ProfScope ps(s, AMG_K_INTERP, 4.0 * (n + 1) + 5.0 * A.nnz + 5.0 * n, k);
        k_ext_interp<false><<<grid, wpb * 32, smem, s>>>(n, A.rp, A.ci, A.v, S.p, L.cf, cidx.p, T,
                                                          std::max(hmx[1], 1), pcnt.p, nullptr, nullptr,
                                                          nullptr, eflag.p);
        AMG_CHECK_LAUNCH();
      }
      P.n = n;
      P.ncols = nc;
      P.rp = m.get_n<int>((size_t)n + 1);
      P.nnz = scan_counts(m, pcnt.p, P.rp, n);
      P.ci = m.get_n<int>(std::max<int64_t>(P.nnz, 1));
      P.v = m.get_n<double>(std::max<int64_t>(P.nnz, 1));
      int hm2[2];
      AMG_CUDA(cudaMemcpyAsync(hm2, eflag.p, sizeof(hm2), cudaMemcpyDeviceToHost, s));
      AMG_CUDA(cudaStreamSynchronize(s));
      int T2 = 32;
      while (T2 <= 2 * hm2[1]) T2 <<= 1;  // the set at most half full
      T2 = std::min(T2, T);
      {
        int wpb = 1;
        const size_t smem = geometry(T2, true, &wpb);
        const int grid = std::max(1, std::min(ceil_div(n, wpb), kNumSMs * 16));
        ProfScope ps(s, AMG_K_INTERP, 8.0 * (n + 1) + 13.0 * A.nnz + 5.0 * n + 12.0 * P.nnz, k);
        k_ext_interp<true><<<grid, wpb * 32, smem, s>>>(n, A.rp, A.ci, A.v, S.p, L.cf, cidx.p, T2,
                                                         std::max(hmx[1], 1), nullptr, P.rp, P.ci, P.v, eflag.p);
        AMG_CHECK_LAUNCH();
      }
      int he = 0;
      AMG_CUDA(cudaMemcpyAsync(&he, eflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
      AMG_CUDA(cudaStreamSynchronize(s));
      if (he) fail(AMG_ERR_SETUP, "extended+i: an F row's modified diagonal is zero");
    } else {
      Buf<int> pcnt(m, n);
      {
        ProfScope ps(s, AMG_K_INTERP, 4.0 * (n + 1) + 5.0 * A.nnz + 5.0 * n, k);
        if (wide) k_interp_count_w<<<gw, TPB, 0, s>>>(n, A.rp, A.ci, S.p, L.cf, pcnt.p);
        else k_interp_count<<<g, TPB, 0, s>>>(n, A.rp, A.ci, S.p, L.cf, pcnt.p);
        AMG_CHECK_LAUNCH();
      }
      P.n = n;
      P.ncols = nc;
      P.rp = m.get_n<int>((size_t)n + 1);
      P.nnz = scan_counts(m, pcnt.p, P.rp, n);
      P.ci = m.get_n<int>(std::max<int64_t>(P.nnz, 1));
      P.v = m.get_n<double>(std::max<int64_t>(P.nnz, 1));
      {
        ProfScope ps(s, AMG_K_INTERP, 8.0 * (n + 1) + 13.0 * A.nnz + 5.0 * n + 12.0 * P.nnz, k);
        if (wide_interp)
          k_interp_fill_w<<<gw, TPB, 0, s>>>(n, prm.block_size, A.rp, A.ci, A.v, S.p, L.cf, cidx.p, P.rp, P.ci, P.v);
        else
          k_interp_fill<<<g, TPB, 0, s>>>(n, prm.block_size, A.rp, A.ci, A.v, S.p, L.cf, cidx.p, P.rp, P.ci, P.v);
        AMG_CHECK_LAUNCH();
      }
    }
    S.reset();
    ST.reset();
    cidx.reset();
    transpose(m, P, nc, L.R);
    DCsr AP;
    spgemm(m, fl.d, A, P, nc, AP, k);
    spgemm(m, fl.d, L.R, AP, nc, h->lev[k + 1].A, k);
    free_csr(m, AP);
    // the SpGEMM's overflow flag is read with the next level's first flag
    // read (every level reads its flags at least once), not with a sync here
    ++k;
  }
}

}  // namespace amg

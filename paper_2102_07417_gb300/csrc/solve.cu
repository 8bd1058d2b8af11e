// solve.cu -- the solve phase: PCG (Sec. 3.1 solver, stopping rule of Sec. 4)
// preconditioned by one V-cycle (Algorithm 2) per iteration.
//
// V-cycle on level k < L with damped Jacobi (S = I - omega D^-1 A, Eq.
// smoother) and zero initial guess; wd_k = omega / diag(A_k):
//   s_k = wd_k .* y_k                 written by whichever kernel produced y_k
//   r_k = y_k - A_k s_k               OpResid
//   y_{k+1} = R_k r_k, s_{k+1}        OpRestrict
//   z_{k+1} = V-cycle(y_{k+1})        recursion; z_L = L^-T L^-1 y_L (k_coarse_solve)
//   t_k = s_k + P_k z_{k+1}           OpProlong  (prolongation + correction)
//   z_k = t_k + wd_k .* (y_k - A_k t_k)   OpJacobi (level 0: OpPost0, fused with the CG dots)
// nu1 > 1 or nu2 > 1 adds plain Jacobi sweeps; nu = 0 drops them.
// With the FSAI smoother (M^-1 = G^T G, Eq. smo) a smoothing step
// s <- s + omega G^T G (y - A s) is three products: w = y - A s (OpResid),
// u = G w and s += (omega G^T) u (OpGemv); the pre-smoothing step from zero
// is u = G y, s = (omega G^T) u, and level 0's last post-smoothing product
// carries the CG bookkeeping (OpPost0 with the G^T product).
//
// FP64 arithmetic on this part runs at ~1.2 TFLOP/s (about 2 DFMA lanes per
// clock per SM), so FP64 issue slots, not HBM bandwidth, bind the FP64 solve:
// one DFMA per stored entry already needs most of the FP64 pipe at full
// bandwidth.  Every sparse kernel is one row "op" (residual, restriction,
// prolongation, smoothing, CG product) run by one of two row kernels:
//   k_sell  -- matrices with >= 32768 rows, stored additionally in sliced
//              ELLPACK (32-row slices, column-major, rows length-sorted within
//              256-row windows when that cuts padding): a lane per row, fully
//              coalesced loads, one FMA issued per stored slot, and residuals
//              y - A x folded into the FMA chain;
//   k_rows  -- smaller CSR matrices, G lanes per row (latency-bound levels).
// Dot products are reduced per block with warp shuffles and finished by the
// last block to arrive (one grid-level reduction, fixed order, deterministic).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <type_traits>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr int TPB = 256;
constexpr int MAX_GRID = kNumSMs * 8;
constexpr unsigned FULL = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T ld(const T *p) {
  return __ldg(p);
}
__device__ __forceinline__ float tof(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float tof(float v) { return v; }
__device__ __forceinline__ double tof(double v) { return v; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Block-reduces NV partial sums, writes them to partials[3*block+c] and
// returns true in every thread of the last block to finish, whose out[c] then
// holds the grid totals (summed in block order).
template <int NV>
__device__ bool grid_reduce(const double (&v)[NV], double *partials, unsigned int *counter, double (&out)[NV]) {
  __shared__ double red[NV][TPB / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    const double s = warp_sum(v[c]);
    if (lane == 0) red[c][w] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double s = 0.0;
      for (int k = 0; k < TPB / 32; ++k) s += red[c][k];
      partials[3 * blockIdx.x + c] = s;
    }
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) acc[c] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int c = 0; c < NV; ++c) acc[c] += __ldcg(&partials[3 * b + c]);
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    const double s = warp_sum(acc[c]);
    if (lane == 0) red[c][w] = s;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    double s = 0.0;
    for (int k = 0; k < TPB / 32; ++k) s += red[c][k];
    out[c] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// v[r] = this lane's partial sum of row r of its G-row group; returns the
// full sum of row `sub` of the group.  Each step halves the rows a lane holds
// (keeping the half its bit selects and adding the partner's copy of that
// half), so a lane performs G/2 + G/4 + ... + 1 = G-1 additions.
template <int G, typename T>
__device__ __forceinline__ T transpose_reduce(T (&v)[G], int sub) {
#pragma unroll
  for (int d = G / 2; d >= 1; d >>= 1) {
    const bool up = (sub & d) != 0;
#pragma unroll
    for (int j = 0; j < d; ++j) {
      const T keep = up ? v[j + d] : v[j];
      const T send = up ? v[j] : v[j + d];
      v[j] = keep + __shfl_xor_sync(FULL, send, d);
    }
  }
  return v[0];
}

template <int NV>
struct Acc {
  double v[NV > 0 ? NV : 1];
};

// Row kernel on CSR, transposed form (TR = true): a warp takes 32 consecutive
// rows; a group of G lanes owns G of them, each lane keeping one partial sum
// per row of its group, then transpose_reduce leaves row base+lane's sum in
// lane `lane` (G-1 additions per row, coalesced epilogue).  Vector form
// (TR = false): G lanes per row, one row per group at a time, butterfly
// reduction; used for levels with few rows, where parallelism matters more
// than the extra additions.  For each row i: sum_i = sum_p mat(p) vec(ci[p])
// (when the op has a matrix; ops with kNeg receive init(i) - sum_i), then
// op.out(i, ., acc); finally op.finish(acc) in every thread.
template <int G, bool TR, class Op>
__global__ void __launch_bounds__(TPB) k_rows(int n, const int *__restrict__ rp, const int *__restrict__ ci, Op op) {
  using T = typename Op::T;
  constexpr int NA = Op::NV > 0 ? Op::NV : 1;
  if (op.skip()) return;
  const int lane = threadIdx.x & 31, sub = lane & (G - 1), grp = lane / G;
  const int gw = (blockIdx.x * TPB + threadIdx.x) >> 5, nw = (gridDim.x * TPB) >> 5;
  Acc<NA> acc;
#pragma unroll
  for (int c = 0; c < NA; ++c) acc.v[c] = 0.0;
  if constexpr (TR) {
    for (int base = gw * 32; base < n; base += nw * 32) {
      T sum = T(0);
      if constexpr (Op::kMatrix) {
        T part[G];
        const int r0 = base + grp * G;
#pragma unroll
        for (int r = 0; r < G; ++r) {
          part[r] = T(0);
          const int row = r0 + r;
          if (row < n) {
            const int e = rp[row + 1];
#pragma unroll 4
            for (int p = rp[row] + sub; p < e; p += G) part[r] = fma(op.mat(p), op.vec(ci[p]), part[r]);
          }
        }
        if constexpr (G == 1) sum = part[0];
        else sum = transpose_reduce<G>(part, sub);
      }
      const int row = base + lane;
      if (row < n) {
        if constexpr (Op::kNeg) sum = op.init(row) - sum;
        op.out(row, sum, acc);
      }
    }
  } else {
    constexpr int RPW = 32 / G;  // rows per warp step
    for (int base = gw * RPW; base < n; base += nw * RPW) {
      const int row = base + grp;
      T sum = T(0);
      if constexpr (Op::kMatrix) {
        if (row < n) {
          const int e = rp[row + 1];
#pragma unroll 4
          for (int p = rp[row] + sub; p < e; p += G) sum = fma(op.mat(p), op.vec(ci[p]), sum);
        }
#pragma unroll
        for (int d = G / 2; d >= 1; d >>= 1) sum += __shfl_xor_sync(FULL, sum, d);
      }
      if (row < n && sub == 0) {
        if constexpr (Op::kNeg) sum = op.init(row) - sum;
        op.out(row, sum, acc);
      }
    }
  }
  op.finish(acc);
}

// Row kernel on the sliced-ELLPACK copy: a warp per 32-row slice, a lane per
// row, the slice's entries read column-major (each warp load is 32
// consecutive entries), exactly one FMA issued per stored slot; ops with
// kNeg start from init(row) and subtract, so y - A x costs no extra add.
// NS slices per warp step (s, s + nw, ...), each an independent chain of
// dependent loads (offsets -> columns and values -> gathered vector).  NS = 1
// is used: two or four slices per step, meant to keep more loads in flight,
// made every level-0 and level-1 kernel slower on the 128^3 hierarchy (FP32
// solve 7.66 ms at NS = 1, 9.89 ms at 2, 11.42 ms at 4).
template <class Op, int NS>
__global__ void __launch_bounds__(TPB) k_sell(int n, int nslices, const int *__restrict__ off,
                                              const int *__restrict__ col, const int *__restrict__ perm, Op op) {
  using T = typename Op::T;
  constexpr int NA = Op::NV > 0 ? Op::NV : 1;
  if (op.skip()) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * TPB + threadIdx.x) >> 5, nw = (gridDim.x * TPB) >> 5;
  Acc<NA> acc;
#pragma unroll
  for (int c = 0; c < NA; ++c) acc.v[c] = 0.0;
  for (int s0 = gw; s0 < nslices; s0 += NS * nw) {
    int row[NS], b[NS], len[NS];
    bool valid[NS];
    T sum[NS];
    int lmax = 0;
#pragma unroll
    for (int u = 0; u < NS; ++u) {
      const int s = s0 + u * nw;
      const bool live = s < nslices;
      const int q = s * 32 + lane;
      valid[u] = live && q < n;
      row[u] = valid[u] ? (perm ? perm[q] : q) : 0;
      const int o0 = live ? off[s] : 0, o1 = live ? off[s + 1] : 0;
      b[u] = o0 + lane;
      len[u] = (o1 - o0) >> 5;
      lmax = max(lmax, len[u]);
      sum[u] = (Op::kNeg && valid[u]) ? op.init(row[u]) : T(0);
    }
#pragma unroll 4
    for (int k = 0; k < lmax; ++k) {
#pragma unroll
      for (int u = 0; u < NS; ++u) {
        if (k < len[u]) {
          const int idx = b[u] + 32 * k;
          const int c = __ldg(col + idx);
          if constexpr (Op::kNeg) sum[u] = fma(-op.mat(idx), op.vec(c), sum[u]);
          else sum[u] = fma(op.mat(idx), op.vec(c), sum[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < NS; ++u)
      if (valid[u]) op.out(row[u], sum[u], acc);
  }
  op.finish(acc);
}

// --------------------------------------------------------- SELL building --
constexpr int SELL_WIN = 256;  // rows per sorting window

// Maximum row length of each 32-row slice, times 32 (entries of the slice).
__global__ void k_sell_count(int n, int nslices, const int *__restrict__ rp, const int *__restrict__ perm,
                             int *__restrict__ cnt) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  int mx = 0;
  for (int l = 0; l < 32; ++l) {
    const int q = s * 32 + l;
    if (q >= n) break;
    const int row = perm ? perm[q] : q;
    mx = max(mx, rp[row + 1] - rp[row]);
  }
  cnt[s] = 32 * mx;
}

// Sorts each window of SELL_WIN rows by length, longest first (ties by row).
__global__ void __launch_bounds__(SELL_WIN) k_sell_perm(int n, const int *__restrict__ rp, int *__restrict__ perm) {
  __shared__ long long key[SELL_WIN];
  const int t = threadIdx.x, row = blockIdx.x * SELL_WIN + t;
  key[t] = row < n ? ((long long)(0x7fffffff - (rp[row + 1] - rp[row])) << 32) | (unsigned)row : LLONG_MAX;
  __syncthreads();
  for (int k = 2; k <= SELL_WIN; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int u = t ^ j;
      if (u > t) {
        const long long a = key[t], b = key[u];
        if ((a > b) == ((t & k) == 0)) {
          key[t] = b;
          key[u] = a;
        }
      }
      __syncthreads();
    }
  if (row < n) perm[row] = (int)(key[t] & 0xffffffffLL);
}

__global__ void k_sell_fill(int n, int nslices, const int *__restrict__ rp, const int *__restrict__ ci,
                            const double *__restrict__ a, const int *__restrict__ perm, const int *__restrict__ off,
                            int *__restrict__ col, double *__restrict__ v, float *__restrict__ v32,
                            __nv_bfloat16 *__restrict__ v16) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = q >> 5, l = q & 31;
  if (s >= nslices) return;
  const int row = q < n ? (perm ? perm[q] : q) : -1;
  const int b = off[s], len = (off[s + 1] - b) >> 5;
  const int rb = row >= 0 ? rp[row] : 0, rl = row >= 0 ? rp[row + 1] - rb : 0;
  for (int k = 0; k < len; ++k) {
    const int idx = b + 32 * k + l;
    const bool in = k < rl;
    const double val = in ? a[rb + k] : 0.0;
    // padding repeats the row's last column (0 for an empty row) with value
    // 0, so the solve kernels need no branch on padding slots
    col[idx] = in ? ci[rb + k] : (rl > 0 ? ci[rb + rl - 1] : 0);
    if (v) v[idx] = val;
    if (v32) v32[idx] = static_cast<float>(val);
    if (v16) v16[idx] = __float2bfloat16_rn(static_cast<float>(val));
  }
}

// ------------------------------------------------------------------ ops --
// Each op: T (arithmetic type of the row sums), NV (number of grid-reduced
// sums), kMatrix, kNeg (the row value is init(i) - sum instead of sum),
// skip(), mat(p), vec(c), init(i), out(i, value, acc), finish(acc).

// r = b - A x;  (b, b), (r, r);  V-cycle input y0 (FP32 modes) and s0.
template <typename TV>
struct OpInit {
  using T = double;
  static constexpr int NV = 2;
  static constexpr bool kMatrix = true, kNeg = true;
  const double *a, *x, *b;
  double *r;
  const TV *wd;
  TV *y0, *s0;
  bool write_y, pre;
  double rtol;
  PcgScalars *sc;
  double *hist, *partials;
  unsigned int *counter;
  __device__ bool skip() const { return false; }
  __device__ double mat(int p) const { return ld(a + p); }
  __device__ double vec(int c) const { return ld(x + c); }
  __device__ double init(int i) const { return b[i]; }
  __device__ void out(int i, double ri, Acc<NV> &acc) const {
    const double bi = b[i];
    r[i] = ri;
    acc.v[0] = fma(bi, bi, acc.v[0]);
    acc.v[1] = fma(ri, ri, acc.v[1]);
    const TV yi = static_cast<TV>(ri);
    if (write_y) y0[i] = yi;
    s0[i] = pre ? wd[i] * yi : TV(0);
  }
  __device__ void finish(Acc<NV> &acc) const {
    double tot[2];
    if (grid_reduce<2>(acc.v, partials, counter, tot) && threadIdx.x == 0) {
      sc->bb = tot[0];
      sc->rr = tot[1];
      sc->tol = rtol * sqrt(tot[0]);
      const double res = sqrt(tot[1]);
      hist[0] = res;
      sc->iters = 0;
      sc->status = AMG_OK;
      sc->done = (res < sc->tol || tot[0] == 0.0) ? 1 : 0;
    }
  }
};

// q = A p;  alpha = rho / (p, q);  breakdown when (p, q) <= 0 or NaN.
struct OpSpmvDot {
  using T = double;
  static constexpr int NV = 1;
  static constexpr bool kMatrix = true, kNeg = false;
  const double *a, *p;
  double *q;
  PcgScalars *sc;
  double *partials;
  unsigned int *counter;
  __device__ bool skip() const { return sc->done; }
  __device__ double mat(int k) const { return ld(a + k); }
  __device__ double vec(int c) const { return ld(p + c); }
  __device__ double init(int) const { return 0.0; }
  __device__ void out(int i, double sum, Acc<NV> &acc) const {
    q[i] = sum;
    acc.v[0] = fma(p[i], sum, acc.v[0]);
  }
  __device__ void finish(Acc<NV> &acc) const {
    double tot[1];
    if (grid_reduce<1>(acc.v, partials, counter, tot) && threadIdx.x == 0) {
      sc->pq = tot[0];
      if (!(tot[0] > 0.0)) {
        sc->status = AMG_ERR_BREAKDOWN;
        sc->done = 1;
      } else {
        sc->alpha = sc->rho / tot[0];
      }
    }
  }
};

// y = A x (FP64, amg_spmv)
struct OpSpmv {
  using T = double;
  static constexpr int NV = 0;
  static constexpr bool kMatrix = true, kNeg = false;
  const double *a, *x;
  double *y;
  __device__ bool skip() const { return false; }
  __device__ double mat(int k) const { return ld(a + k); }
  __device__ double vec(int c) const { return ld(x + c); }
  __device__ double init(int) const { return 0.0; }
  __device__ void out(int i, double sum, Acc<1> &) const { y[i] = sum; }
  __device__ void finish(Acc<1> &) const {}
};

// r = y - A s
template <typename TT>
struct OpResid {
  using T = TT;
  static constexpr int NV = 0;
  static constexpr bool kMatrix = true, kNeg = true;
  const T *a, *s, *y;
  T *r;
  const int *done;
  __device__ bool skip() const { return *done; }
  __device__ T mat(int k) const { return ld(a + k); }
  __device__ T vec(int c) const { return ld(s + c); }
  __device__ T init(int i) const { return y[i]; }
  __device__ void out(int i, T res, Acc<1> &) const { r[i] = res; }
  __device__ void finish(Acc<1> &) const {}
};

// y_c = R r;  s_c = wd_c .* y_c (pre = 1), 0 (pre = 0), not written (pre = -1)
template <typename TT, typename TP>
struct OpRestrict {
  using T = TT;
  static constexpr int NV = 0;
  static constexpr bool kMatrix = true, kNeg = false;
  const TP *rv;
  const T *r, *wd;
  T *yc, *sc;
  int pre;
  const int *done;
  __device__ bool skip() const { return *done; }
  __device__ T mat(int k) const { return static_cast<T>(tof(rv[k])); }
  __device__ T vec(int c) const { return ld(r + c); }
  __device__ T init(int) const { return T(0); }
  __device__ void out(int i, T sum, Acc<1> &) const {
    yc[i] = sum;
    if (pre >= 0) sc[i] = pre ? wd[i] * sum : T(0);
  }
  __device__ void finish(Acc<1> &) const {}
};

// t = s + P z_c
template <typename TT, typename TP>
struct OpProlong {
  using T = TT;
  static constexpr int NV = 0;
  static constexpr bool kMatrix = true, kNeg = false;
  const TP *pv;
  const T *s, *zc;
  T *t;
  const int *done;
  __device__ bool skip() const { return *done; }
  __device__ T mat(int k) const { return static_cast<T>(tof(pv[k])); }
  __device__ T vec(int c) const { return ld(zc + c); }
  __device__ T init(int) const { return T(0); }
  __device__ void out(int i, T sum, Acc<1> &) const { t[i] = s[i] + sum; }
  __device__ void finish(Acc<1> &) const {}
};

// out = M x (+ base when BASE): the FSAI products u = G w and s = base + omega G^T u
template <typename TT, bool BASE>
struct OpGemv {
  using T = TT;
  static constexpr int NV = 0;
  static constexpr bool kMatrix = true, kNeg = false;
  const T *mv, *x, *base;
  T *dst;
  const int *done;
  __device__ bool skip() const { return *done; }
  __device__ T mat(int k) const { return ld(mv + k); }
  __device__ T vec(int c) const { return ld(x + c); }
  __device__ T init(int) const { return T(0); }
  __device__ void out(int i, T sum, Acc<1> &) const { dst[i] = BASE ? base[i] + sum : sum; }
  __device__ void finish(Acc<1> &) const {}
};

// z = t + wd .* (y - A t)
template <typename TT>
struct OpJacobi {
  using T = TT;
  static constexpr int NV = 0;
  static constexpr bool kMatrix = true, kNeg = true;
  const T *a, *wd, *y, *t;
  T *z;
  const int *done;
  __device__ bool skip() const { return *done; }
  __device__ T mat(int k) const { return ld(a + k); }
  __device__ T vec(int c) const { return ld(t + c); }
  __device__ T init(int i) const { return y[i]; }
  __device__ void out(int i, T res, Acc<1> &) const { z[i] = fma(wd[i], res, t[i]); }
  __device__ void finish(Acc<1> &) const {}
};

enum Post0Mode { POST_APPLY = 0, POST_FIRST = 1, POST_ITER = 2 };

// Level-0 post-smoothing fused with the CG bookkeeping:
//   z = t + wd .* (y - A t) (KIND = POST_JACOBI), z = t + (omega G^T) u
//   (POST_FSAI, a = omega G^T's values, u = G (y - A t)) or z = t
//   (POST_NONE), written in FP64;
//   APPLY: nothing else; FIRST: rho = (r, z), p = z;
//   ITER:  beta = (z, r) / rho (standard) or -alpha (z, q) / rho (flexible:
//          (z_{k+1}, r_{k+1} - r_k) with r_{k+1} - r_k = -alpha q_k), rho = (r, z).
enum Post0Kind { POST_NONE = 0, POST_JACOBI = 1, POST_FSAI = 2 };
template <typename TT, int KIND>
struct OpPost0 {
  using T = TT;
  static constexpr int NV = 2;
  static constexpr bool kMatrix = KIND != POST_NONE, kNeg = KIND == POST_JACOBI;
  const T *a, *wd, *y, *t, *u;
  double *z;
  const double *r, *q;
  double *p;
  int mode, flexible;
  PcgScalars *sc;
  const int *done;
  double *partials;
  unsigned int *counter;
  __device__ bool skip() const { return *done; }
  __device__ T mat(int k) const { return ld(a + k); }
  __device__ T vec(int c) const { return KIND == POST_FSAI ? ld(u + c) : ld(t + c); }
  __device__ T init(int i) const { return y[i]; }
  __device__ void out(int i, T res, Acc<NV> &acc) const {
    const T zi = KIND == POST_JACOBI ? fma(wd[i], res, t[i]) : KIND == POST_FSAI ? t[i] + res : t[i];
    const double zd = static_cast<double>(zi);
    z[i] = zd;
    if (mode != POST_APPLY) {
      acc.v[0] = fma(r[i], zd, acc.v[0]);
      if (mode == POST_FIRST) p[i] = zd;
      else if (flexible) acc.v[1] = fma(zd, q[i], acc.v[1]);
    }
  }
  __device__ void finish(Acc<NV> &acc) const {
    if (mode == POST_APPLY) return;
    double tot[2];
    if (grid_reduce<2>(acc.v, partials, counter, tot) && threadIdx.x == 0) {
      sc->rz = tot[0];
      sc->zq = tot[1];
      if (mode == POST_ITER) sc->beta = flexible ? -sc->alpha * tot[1] / sc->rho : tot[0] / sc->rho;
      sc->rho = tot[0];
    }
  }
};

// ------------------------------------------------------ streaming kernels --
template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
  using type = double2;
};
template <>
struct Vec2<float> {
  using type = float2;
};

// x += alpha p;  r -= alpha q;  ||r||;  convergence test;  V-cycle input y0 / s0.
// VEC: two elements per thread with 16-byte loads (all pointers 16-byte aligned).
template <typename T, bool VEC>
__global__ void __launch_bounds__(TPB) k_pcg_update(int n, double *__restrict__ x, double *__restrict__ r,
                                                    const double *__restrict__ p, const double *__restrict__ q,
                                                    const T *__restrict__ wd, T *__restrict__ y0,
                                                    T *__restrict__ s0, bool write_y, bool pre, PcgScalars *sc,
                                                    double *hist, int hist_cap, int *host_done,
                                                    double *partials, unsigned int *counter) {
  if (sc->done) return;
  const double alpha = sc->alpha;
  double v[1] = {0.0};
  if (VEC) {
    using T2 = typename Vec2<T>::type;
    const int n2 = n >> 1;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n2; j += gridDim.x * blockDim.x) {
      double2 xv = reinterpret_cast<double2 *>(x)[j];
      double2 rv = reinterpret_cast<double2 *>(r)[j];
      const double2 pv = reinterpret_cast<const double2 *>(p)[j];
      const double2 qv = reinterpret_cast<const double2 *>(q)[j];
      xv.x = fma(alpha, pv.x, xv.x);
      xv.y = fma(alpha, pv.y, xv.y);
      rv.x = fma(-alpha, qv.x, rv.x);
      rv.y = fma(-alpha, qv.y, rv.y);
      reinterpret_cast<double2 *>(x)[j] = xv;
      reinterpret_cast<double2 *>(r)[j] = rv;
      v[0] = fma(rv.x, rv.x, v[0]);
      v[0] = fma(rv.y, rv.y, v[0]);
      T2 yv, sv;
      yv.x = static_cast<T>(rv.x);
      yv.y = static_cast<T>(rv.y);
      if (write_y) reinterpret_cast<T2 *>(y0)[j] = yv;
      if (pre) {
        const T2 w = reinterpret_cast<const T2 *>(wd)[j];
        sv.x = w.x * yv.x;
        sv.y = w.y * yv.y;
      } else {
        sv.x = sv.y = T(0);
      }
      reinterpret_cast<T2 *>(s0)[j] = sv;
    }
  }
  const int start = VEC ? (n & ~1) : 0;
  for (int i = start + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    v[0] = fma(ri, ri, v[0]);
    const T yi = static_cast<T>(ri);
    if (write_y) y0[i] = yi;
    s0[i] = pre ? wd[i] * yi : T(0);
  }
  double tot[1];
  if (grid_reduce<1>(v, partials, counter, tot) && threadIdx.x == 0) {
    const int it = sc->iters + 1;
    sc->iters = it;
    sc->rr = tot[0];
    const double res = sqrt(tot[0]);
    if (it < hist_cap) hist[it] = res;
    if (res < sc->tol) {
      sc->done = 1;
    } else if (it >= sc->maxit) {
      sc->status = AMG_ERR_NO_CONVERGENCE;
      sc->done = 1;
    }
    if (sc->done && host_done) *(volatile int *)host_done = 1;
  }
}

// p = z + beta p
template <bool VEC>
__global__ void __launch_bounds__(TPB) k_direction(int n, const double *__restrict__ z, double *__restrict__ p,
                                                   const PcgScalars *sc) {
  if (sc->done) return;
  const double beta = sc->beta;
  if (VEC) {
    const int n2 = n >> 1;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n2; j += gridDim.x * blockDim.x) {
      double2 pv = reinterpret_cast<double2 *>(p)[j];
      const double2 zv = reinterpret_cast<const double2 *>(z)[j];
      pv.x = fma(beta, pv.x, zv.x);
      pv.y = fma(beta, pv.y, zv.y);
      reinterpret_cast<double2 *>(p)[j] = pv;
    }
  }
  const int start = VEC ? (n & ~1) : 0;
  for (int i = start + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

// z = L^-T (L^-1 y) on the last level, with Li = L^-1 precomputed from the
// dense Cholesky factor: two triangular matrix-vector products (one block,
// one row per thread), instead of 2n dependent substitution steps.
template <typename T>
__global__ void k_coarse_solve(int n, const double *__restrict__ Li, const T *__restrict__ y, T *__restrict__ z,
                               const int *__restrict__ done) {
  if (*done) return;
  extern __shared__ double sm[];
  double *yy = sm, *w = sm + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) yy[i] = static_cast<double>(y[i]);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j <= i; ++j) s = fma(Li[(size_t)i * n + j], yy[j], s);
    w[i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int k = i; k < n; ++k) s = fma(Li[(size_t)k * n + i], w[k], s);
    z[i] = static_cast<T>(s);
  }
}

// V-cycle input from an FP64 vector: y = (T) src, s = wd .* y or 0
template <typename T>
__global__ void k_load_y0(int n, const double *__restrict__ src, const T *__restrict__ wd, T *__restrict__ y,
                          T *__restrict__ s, bool write_y, bool pre) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const T yi = static_cast<T>(src[i]);
    if (write_y) y[i] = yi;
    s[i] = pre ? wd[i] * yi : T(0);
  }
}

template <typename T>
__global__ void k_copy(int n, const T *__restrict__ a, T *__restrict__ b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = a[i];
}

// wd = omega / a_ii, a thread per row.  (Eight lanes per row with the
// division in one of them was 6.5x slower on the 128^3 level 0: FP64
// instructions issue per warp, so FP64 work must keep its lanes dense.)
__global__ void k_make_wd(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                          const double *__restrict__ a, double omega, double *__restrict__ wd,
                          float *__restrict__ wd32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double d = 1.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] == i) d = a[p];
    const double w = omega / d;
    wd[i] = w;
    if (wd32) wd32[i] = static_cast<float>(w);
  }
}

__global__ void k_to_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = static_cast<float>(a[i]);
}

__global__ void k_to_bf16(int64_t n, const double *__restrict__ a, __nv_bfloat16 *__restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(static_cast<float>(a[i]));
}

// ---------------------------------------------------- dense tail operator --
// Below a level kd with at most kDenseOpRows rows the V-cycle is a fixed
// linear map z_kd = M_kd y_kd (Algorithm 2's steps on levels kd..L are all
// linear in y_kd: Jacobi sweeps from zero, residual, restriction, the
// recursive cycle, prolongation, the dense solve).  The set-up forms M_kd
// explicitly in FP64, level by level from the last one:
//   M_L = L^-T L^-1
//   X   = nu1 Jacobi sweeps from 0 applied to the identity (X = W for nu1 = 1,
//         W = omega D^-1), E = I - A X
//   T   = X + P M_{k+1} R E, then nu2 sweeps T <- T + W (I - A T)
//   M_k = T
// and each V-cycle applies it as one dense matrix-vector product instead of
// the ~4 latency-bound launches per level it replaces (the same operator up to
// rounding).

// out(i, c) = base(i, c) + w_i (diag [i == c] + sgn sum_p m_p D(ci_p, c)),
// out m x ncol row-major; base, wd (w_i = 1) and D may be null.
__global__ void k_dop_sparse(int m, int ncol, const int *__restrict__ rp, const int *__restrict__ ci,
                             const double *__restrict__ mv, const double *__restrict__ D,
                             const double *__restrict__ base, const double *__restrict__ wd, double diag, double sgn,
                             double *__restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * ncol) return;
  const int i = (int)(t / ncol), c = (int)(t % ncol);
  double acc = 0.0;
  if (D)
    for (int p = rp[i]; p < rp[i + 1]; ++p) acc = fma(mv[p], D[(size_t)ci[p] * ncol + c], acc);
  double v = (i == c ? diag : 0.0) + sgn * acc;
  if (wd) v *= wd[i];
  if (base) v += base[t];
  out[t] = v;
}

// out = M V: M m x k, V k x ncol, out m x ncol (row-major).
__global__ void k_dop_gemm(int m, int k, int ncol, const double *__restrict__ M, const double *__restrict__ V,
                           double *__restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * ncol) return;
  const int i = (int)(t / ncol), c = (int)(t % ncol);
  double acc = 0.0;
  for (int j = 0; j < k; ++j) acc = fma(M[(size_t)i * k + j], V[(size_t)j * ncol + c], acc);
  out[t] = acc;
}

// out = base + M V: M m x k, V k x ncol, base and out m x ncol (row-major).
__global__ void k_dop_gemm_add(int m, int k, int ncol, const double *__restrict__ M, const double *__restrict__ V,
                               const double *__restrict__ base, double *__restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * ncol) return;
  const int i = (int)(t / ncol), c = (int)(t % ncol);
  double acc = 0.0;
  for (int j = 0; j < k; ++j) acc = fma(M[(size_t)i * k + j], V[(size_t)j * ncol + c], acc);
  out[t] = base[t] + acc;
}

// out = the CSR matrix (n x n) as a dense row-major array.
__global__ void k_dop_csr_dense(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                const double *__restrict__ v, double *__restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), c = (int)(t % n);
  double x = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == c) x = v[p];
  out[t] = x;
}

// M = Li^T Li for the lower-triangular Li = L^-1 (n x n row-major).
__global__ void k_dop_coarse(int n, const double *__restrict__ Li, double *__restrict__ M) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  double acc = 0.0;
  for (int k = max(i, j); k < n; ++k) acc = fma(Li[(size_t)k * n + i], Li[(size_t)k * n + j], acc);
  M[t] = acc;
}

// z = M y: a block of DOP_TPB threads per row (a row of at most 1024
// entries is then one or a few loads per thread), FP64 accumulation.
constexpr int DOP_TPB = 128;
template <typename T>
__global__ void __launch_bounds__(DOP_TPB) k_dop_apply(int n, const double *__restrict__ M, const T *__restrict__ y,
                                                       T *__restrict__ z, const int *__restrict__ done) {
  __shared__ double red[DOP_TPB / 32];
  if (*done) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    double acc = 0.0;
#pragma unroll 4
    for (int j = threadIdx.x; j < n; j += DOP_TPB)
      acc = fma(__ldg(M + (size_t)i * n + j), static_cast<double>(y[j]), acc);
    acc = warp_sum(acc);
    if (lane == 0) red[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < DOP_TPB / 32; ++k) t += red[k];
      z[i] = static_cast<T>(t);
    }
    __syncthreads();
  }
}

inline int grid_for(int64_t n) { return std::max(1, std::min<int>(ceil_div(n, TPB), MAX_GRID)); }

// How a CSR matrix's rows are mapped to lanes (see k_rows).
template <bool TR, class Op>
void launch_rows_g(int G, int grid, int n, const int *rp, const int *ci, const Op &op, cudaStream_t s) {
  switch (G) {
    case 1: k_rows<1, TR, Op><<<grid, TPB, 0, s>>>(n, rp, ci, op); break;
    case 2: k_rows<2, TR, Op><<<grid, TPB, 0, s>>>(n, rp, ci, op); break;
    case 4: k_rows<4, TR, Op><<<grid, TPB, 0, s>>>(n, rp, ci, op); break;
    case 8: k_rows<8, TR, Op><<<grid, TPB, 0, s>>>(n, rp, ci, op); break;
    case 16: k_rows<16, TR, Op><<<grid, TPB, 0, s>>>(n, rp, ci, op); break;
    default: k_rows<32, TR, Op><<<grid, TPB, 0, s>>>(n, rp, ci, op); break;
  }
}

template <class Op>
void launch_rows(RowMap map, int n, const int *rp, const int *ci, const Op &op, cudaStream_t s) {
  if (map.tr || map.g == 1) {
    launch_rows_g<true>(map.g, grid_for(n), n, rp, ci, op, s);
  } else {
    const int64_t lanes = (int64_t)n * map.g;
    launch_rows_g<false>(map.g, std::max(1, std::min<int>(ceil_div(lanes, TPB), MAX_GRID)), n, rp, ci, op, s);
  }
  AMG_CHECK_LAUNCH();
}

// Matrices with at least kSellSolveRows rows get a SELL copy, used by the
// single-vector kernels and (up to 16 columns) the batched ones; smaller ones
// use the CSR vector form.  From kSellMinRows rows up the CSR form puts at
// most a quarter of the mean row length of lanes on a row (see choose_map):
// there rows are few enough (and on coarse levels long enough) that a few
// lanes per row keep more loads in flight than a lane per row in SELL
// (measured on the 128^3 Poisson hierarchy: level 2, 137K rows of 46
// entries, smoothing 62 us in CSR against 79 us in SELL).  (Copies were once
// built from kSellMinRows rows too, which no kernel read.)
constexpr int kSellMinRows = 1 << 15;
constexpr int kSellSolveRows = 1 << 18;
inline bool on_sell(const DCsr &M) { return M.use_sell && M.n >= kSellSolveRows; }

// Runs `op` over the rows of M: the SELL kernel when on_sell(M) (the op's
// value pointer must then point into the SELL copy), else the CSR row kernel.
template <class Op>
void launch_mat(const DCsr &M, const RowMap &map, const Op &op, cudaStream_t s) {
  if (on_sell(M)) {
    constexpr int NS = 1;
    const int grid = std::max(1, std::min(ceil_div(M.sell.nslices, NS * (TPB / 32)), MAX_GRID));
    k_sell<Op, NS><<<grid, TPB, 0, s>>>(M.n, M.sell.nslices, M.sell.off, M.sell.col, M.sell.perm, op);
    AMG_CHECK_LAUNCH();
  } else {
    launch_rows(map, M.n, M.rp, M.ci, op, s);
  }
}

// Lane mapping of a CSR matrix (used below the SELL threshold).  Large FP64
// matrices: transposed form with G about a quarter of the mean row length
// (each extra lane costs one FP64 add per row).  Otherwise the vector form
// with enough lanes per row to put ~2^19 lanes to work (capped by the row
// length and 32): small coarse levels are latency-bound.
RowMap choose_map(int64_t nnz, int n, bool fp64) {
  RowMap m;
  const double avg = n ? (double)nnz / n : 0.0;
  if (fp64 && n >= (1 << 18)) {
    const double want = avg / 4.0;
    while (m.g < 32 && 2 * m.g <= want) m.g <<= 1;
    m.tr = true;
    return m;
  }
  // lanes per row: at most the mean row length; from 2^15 rows up at most a
  // quarter of it (two or more entries per lane: the measured optimum there,
  // e.g. 4 lanes for 46 entries, 1 lane for P's ~2)
  int cap = 1;
  if (n >= kSellMinRows) {
    while (cap < 32 && 4 * cap <= avg) cap <<= 1;
  } else {
    while (cap < 32 && cap < avg) cap <<= 1;
  }
  // lanes to put to work: 2^19 from 2^15 rows up, 2^17 below (the 128^3
  // hierarchy's level 3, 24K rows of 60 entries, smoothed in 27 us (FP64) with
  // 8 lanes per row against 43 us with 32; level 4, 3.6K rows, keeps 32)
  const int64_t lanes = n >= kSellMinRows ? (1 << 19) : (1 << 17);
  int g = 1;
  while (g < cap && (int64_t)n * g < lanes) g <<= 1;
  m.g = g;
  m.tr = false;
  return m;
}

// Builds M's SELL copy with the requested value types.  Rows are permuted
// (length-sorted within windows) only when that cuts the padding of the
// identity order by more than 3 %.
void build_sell(Mem &m, DCsr &M, bool want64, bool want32, bool want16) {
  cudaStream_t s = m.stream;
  Sell &S = M.sell;
  const int n = M.n;
  S.nslices = ceil_div(n, 32);
  Buf<int> cnt(m, (size_t)S.nslices + 1);
  S.off = m.get_n<int>((size_t)S.nslices + 1);
  {
    ProfScope ps(s, AMG_K_SETUP_OTHER, 8.0 * n);
    k_sell_count<<<ceil_div(S.nslices, TPB), TPB, 0, s>>>(n, S.nslices, M.rp, nullptr, cnt.p);
    AMG_CHECK_LAUNCH();
  }
  S.nent = scan_counts(m, cnt.p, S.off, S.nslices);
  if ((double)S.nent > 1.03 * (double)M.nnz + 32.0) {
    S.perm = m.get_n<int>(n);
    ProfScope ps(s, AMG_K_SETUP_OTHER, 16.0 * n);
    k_sell_perm<<<ceil_div(n, SELL_WIN), SELL_WIN, 0, s>>>(n, M.rp, S.perm);
    AMG_CHECK_LAUNCH();
    k_sell_count<<<ceil_div(S.nslices, TPB), TPB, 0, s>>>(n, S.nslices, M.rp, S.perm, cnt.p);
    AMG_CHECK_LAUNCH();
    S.nent = scan_counts(m, cnt.p, S.off, S.nslices);
  }
  const size_t ne = (size_t)std::max<int64_t>(S.nent, 1);
  S.col = m.get_n<int>(ne);
  if (want64) S.v = m.get_n<double>(ne);
  if (want32) S.v32 = m.get_n<float>(ne);
  if (want16) S.v16 = m.get_n<__nv_bfloat16>(ne);
  {
    ProfScope ps(s, AMG_K_SETUP_OTHER, 4.0 * (n + 1) + 12.0 * M.nnz + 16.0 * S.nent);
    k_sell_fill<<<ceil_div((int64_t)S.nslices * 32, TPB), TPB, 0, s>>>(n, S.nslices, M.rp, M.ci, M.v, S.perm, S.off,
                                                                       S.col, S.v, S.v32, S.v16);
    AMG_CHECK_LAUNCH();
  }
  M.use_sell = true;
}

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ---------------------------------------------------------------- V-cycle --
// Value arrays of A (V-cycle precision or FP64) and of P / R (storage type
// TP) in whichever layout the solve kernels read.
template <typename T>
const T *avals(const DCsr &M);
template <>
const double *avals<double>(const DCsr &M) { return on_sell(M) ? M.sell.v : M.v; }
template <>
const float *avals<float>(const DCsr &M) { return on_sell(M) ? M.sell.v32 : M.v32; }

template <typename TP>
const TP *pvals(const DCsr &M);
template <>
const double *pvals<double>(const DCsr &M) { return on_sell(M) ? M.sell.v : M.v; }
template <>
const float *pvals<float>(const DCsr &M) { return on_sell(M) ? M.sell.v32 : M.v32; }
template <>
const __nv_bfloat16 *pvals<__nv_bfloat16>(const DCsr &M) { return on_sell(M) ? M.sell.v16 : M.v16; }

template <typename T>
const T *wdv(const Level &l);
template <>
const double *wdv<double>(const Level &l) { return l.wd; }
template <>
const float *wdv<float>(const Level &l) { return l.wd32; }

template <typename T>
inline T *vec(void *p) {
  return static_cast<T *>(p);
}

struct CycleCtx {
  const int *done;  // device flag: when set, every kernel returns at once
  int mode;         // Post0Mode
  int flexible;
};

constexpr double idx_bytes = 4.0;

template <typename T>
void jacobi_sweep(amg_hierarchy *h, int k, const T *y, const T *t, T *z, const int *done, int kind) {
  Level &L = h->lev[k];
  const DCsr &A = L.A;
  const double bt = sizeof(T);
  ProfScope ps(h->mem.stream, kind, (idx_bytes + bt) * (double)A.nnz + 4.0 * (A.n + 1) + 4.0 * bt * A.n, k);
  OpJacobi<T> op{avals<T>(A), wdv<T>(L), y, t, z, done};
  launch_mat(A, A.map, op, h->mem.stream);
}

// out = y - A_k s (a residual outside the pre-smoothed one; profiled as `kind`)
template <typename T>
void residual(amg_hierarchy *h, int k, const T *y, const T *sv, T *out, const int *done, int kind) {
  const DCsr &A = h->lev[k].A;
  const double bt = sizeof(T);
  ProfScope ps(h->mem.stream, kind, (idx_bytes + bt) * (double)A.nnz + 4.0 * (A.n + 1) + 3.0 * bt * A.n, k);
  OpResid<T> op{avals<T>(A), sv, y, out, done};
  launch_mat(A, A.map, op, h->mem.stream);
}

// FSAI halves of a smoothing step: u = G w, and out = base + (omega G^T) u
template <typename T>
void fsai_g(amg_hierarchy *h, int k, const T *w, T *u, const int *done) {
  const DCsr &G = h->lev[k].G;
  const double bt = sizeof(T);
  ProfScope ps(h->mem.stream, AMG_K_SMOOTH_FSAI, (idx_bytes + bt) * (double)G.nnz + 4.0 * (G.n + 1) + 2.0 * bt * G.n, k);
  OpGemv<T, false> op{avals<T>(G), w, nullptr, u, done};
  launch_mat(G, G.map, op, h->mem.stream);
}

template <typename T>
void fsai_gt(amg_hierarchy *h, int k, const T *u, const T *base, T *out, const int *done) {
  const DCsr &GT = h->lev[k].GT;
  const double bt = sizeof(T);
  ProfScope ps(h->mem.stream, AMG_K_SMOOTH_FSAI,
               (idx_bytes + bt) * (double)GT.nnz + 4.0 * (GT.n + 1) + (base ? 3.0 : 2.0) * bt * GT.n, k);
  if (base) {
    OpGemv<T, true> op{avals<T>(GT), u, base, out, done};
    launch_mat(GT, GT.map, op, h->mem.stream);
  } else {
    OpGemv<T, false> op{avals<T>(GT), u, nullptr, out, done};
    launch_mat(GT, GT.map, op, h->mem.stream);
  }
}

template <typename T>
void coarse_solve(amg_hierarchy *h, int n, const T *y, T *z, const int *done) {
  cudaStream_t s = h->mem.stream;
  ProfScope ps(s, AMG_K_COARSE, 8.0 * (double)n * n + 2.0 * sizeof(T) * n, h->nlevels - 1);
  const int th = std::min(1024, std::max(32, (n + 31) / 32 * 32));
  k_coarse_solve<T><<<1, th, 2 * sizeof(double) * n, s>>>(n, h->Linv, y, z, done);
  AMG_CHECK_LAUNCH();
}

// Levels k >= 1 (and level 0 up to the prolongation).  On entry y_k and s_k
// are in place; on exit z_k (k > 0) or t_0 (k = 0, in lev[0].r) is written.
template <typename T, typename TP>
void cycle_level(amg_hierarchy *h, int k, const CycleCtx &cc) {
  cudaStream_t s = h->mem.stream;
  Level &L = h->lev[k];
  const DCsr &A = L.A;
  const int n = A.n;
  const double bt = sizeof(T), bp = sizeof(TP);
  if (k == h->nlevels - 1) {
    coarse_solve<T>(h, n, vec<T>(L.y), vec<T>(L.z), cc.done);
    return;
  }
  if (k == h->dense_level) {  // this level and every coarser one: z_k = M_k y_k
    ProfScope ps(s, AMG_K_COARSE, 8.0 * (double)n * n + 2.0 * bt * n, k);
    k_dop_apply<T><<<std::max(1, std::min(n, MAX_GRID)), DOP_TPB, 0, s>>>(n, h->dense_op, vec<T>(L.y), vec<T>(L.z),
                                                                           cc.done);
    AMG_CHECK_LAUNCH();
    return;
  }
  const amg_params &prm = h->prm;
  const bool fsai = prm.smoother == AMG_SMOOTH_FSAI;
  T *y = vec<T>(L.y), *sv = vec<T>(L.s), *r = vec<T>(L.r), *w = vec<T>(L.w);
  if (fsai) {
    if (prm.nu1 > 0) {  // s = omega G^T G y (from s = 0), then further steps in place
      fsai_g<T>(h, k, y, w, cc.done);
      fsai_gt<T>(h, k, w, nullptr, sv, cc.done);
      for (int it = 1; it < prm.nu1; ++it) {
        residual<T>(h, k, y, sv, r, cc.done, AMG_K_SOLVE_OTHER);
        fsai_g<T>(h, k, r, w, cc.done);
        fsai_gt<T>(h, k, w, sv, sv, cc.done);
      }
    }  // nu1 = 0: s = 0 was written by the producer of y
  } else {
    for (int it = 1; it < prm.nu1; ++it) {  // extra pre-smoothing sweeps
      jacobi_sweep<T>(h, k, y, sv, w, cc.done, AMG_K_SOLVE_OTHER);
      std::swap(sv, w);
    }
  }
  {
    ProfScope ps(s, AMG_K_SMOOTH_RESID, (idx_bytes + bt) * (double)A.nnz + 4.0 * (n + 1) + 3.0 * bt * n, k);
    OpResid<T> op{avals<T>(A), sv, y, r, cc.done};
    launch_mat(A, A.map, op, s);
  }
  Level &C = h->lev[k + 1];
  const int nc = C.A.n;
  // no pre-smoothed s on the next level when it is solved directly
  const bool c_last = (k + 1 == h->nlevels - 1) || (k + 1 == h->dense_level);
  {
    const DCsr &R = L.R;
    ProfScope ps(s, AMG_K_RESTRICT, (idx_bytes + bp) * (double)R.nnz + 4.0 * (nc + 1) + bt * n + bt * nc +
                                        (c_last ? 0.0 : 2.0 * bt * nc), k);
    // the coarse level's s: wd .* y (Jacobi), formed by the coarse level itself (FSAI), 0 (nu1 = 0)
    const int pre = c_last ? -1 : prm.nu1 == 0 ? 0 : fsai ? -1 : 1;
    OpRestrict<T, TP> op{pvals<TP>(R), r, pre == 1 ? wdv<T>(C) : nullptr, vec<T>(C.y), vec<T>(C.s), pre, cc.done};
    launch_mat(R, R.map, op, s);
  }
  cycle_level<T, TP>(h, k + 1, cc);
  {
    const DCsr &P = L.P;
    ProfScope ps(s, AMG_K_PROLONG, (idx_bytes + bp) * (double)P.nnz + 4.0 * (n + 1) + 2.0 * bt * n + bt * nc, k);
    OpProlong<T, TP> op{pvals<TP>(P), sv, vec<T>(C.z), r, cc.done};
    launch_mat(P, P.map, op, s);
  }
  if (k == 0) return;  // level 0's post-smoothing is fused with the CG bookkeeping
  T *t = r;
  if (prm.nu2 == 0) {
    ProfScope ps(s, AMG_K_SOLVE_OTHER, 2.0 * bt * n, k);
    k_copy<T><<<grid_for(n), TPB, 0, s>>>(n, t, vec<T>(L.z));
    AMG_CHECK_LAUNCH();
    return;
  }
  if (fsai) {  // w = y - A t, u = G w (in s, free after the prolongation), z = t + omega G^T u
    for (int it = 0; it < prm.nu2; ++it) {
      const bool lastp = it == prm.nu2 - 1;
      T *dst = lastp ? vec<T>(L.z) : t;  // in place: out[i] reads only t[i]
      residual<T>(h, k, y, t, w, cc.done, lastp ? AMG_K_SMOOTH_POST : AMG_K_SOLVE_OTHER);
      fsai_g<T>(h, k, w, sv, cc.done);
      fsai_gt<T>(h, k, sv, t, dst, cc.done);
      t = dst;
    }
    return;
  }
  for (int it = 0; it < prm.nu2; ++it) {
    const bool lastp = it == prm.nu2 - 1;
    T *dst = lastp ? vec<T>(L.z) : (t == r ? w : r);
    jacobi_sweep<T>(h, k, y, t, dst, cc.done, lastp ? AMG_K_SMOOTH_POST : AMG_K_SOLVE_OTHER);
    t = dst;
  }
}

// Whole V-cycle from level-0 input (y0, s0 in place) to z (FP64) with the
// level-0 CG bookkeeping of `cc.mode`.
template <typename T, typename TP>
void vcycle(amg_hierarchy *h, double *z, const CycleCtx &cc) {
  cudaStream_t s = h->mem.stream;
  Level &L0 = h->lev[0];
  const DCsr &A = L0.A;
  const int n = A.n;
  const double bt = sizeof(T);
  const T *y = vec<T>(L0.y);
  const T *t;
  bool sweep = true;
  const bool fsai = h->prm.smoother == AMG_SMOOTH_FSAI && h->nlevels > 1;
  if (h->nlevels == 1) {
    coarse_solve<T>(h, n, y, vec<T>(L0.z), cc.done);
    t = vec<T>(L0.z);
    sweep = false;
  } else {
    cycle_level<T, TP>(h, 0, cc);
    T *tt = vec<T>(L0.r), *w = vec<T>(L0.w);
    if (fsai) {
      T *u = vec<T>(L0.s);  // free after the prolongation
      for (int it = 0; it < h->prm.nu2; ++it) {
        residual<T>(h, 0, y, tt, w, cc.done, it + 1 < h->prm.nu2 ? AMG_K_SOLVE_OTHER : AMG_K_SMOOTH_POST);
        fsai_g<T>(h, 0, w, u, cc.done);
        if (it + 1 < h->prm.nu2) fsai_gt<T>(h, 0, u, tt, tt, cc.done);  // all but the last step, in place
      }
    } else {
      for (int it = 0; it + 1 < h->prm.nu2; ++it) {  // all but the last post sweep
        jacobi_sweep<T>(h, 0, y, tt, w, cc.done, AMG_K_SOLVE_OTHER);
        std::swap(tt, w);
      }
    }
    t = tt;
    sweep = h->prm.nu2 > 0;
  }
  const DCsr &M = fsai ? L0.GT : A;  // matrix of the last post-smoothing product
  double bytes = 8.0 * n + bt * n;   // z (FP64) write, t read
  if (sweep) bytes += (idx_bytes + bt) * (double)M.nnz + 4.0 * (n + 1) + 2.0 * bt * n;
  if (cc.mode != POST_APPLY) bytes += 8.0 * n + (cc.mode == POST_FIRST ? 8.0 * n : (cc.flexible ? 8.0 * n : 0.0));
  ProfScope ps(s, fsai && sweep ? AMG_K_SMOOTH_FSAI : AMG_K_SMOOTH_POST, bytes, 0);
  if (sweep && fsai) {
    OpPost0<T, POST_FSAI> op{avals<T>(M), nullptr, y, t, vec<T>(L0.s), z, h->r, h->q, h->p, cc.mode, cc.flexible,
                             h->sc, cc.done, h->partials, h->counter};
    launch_mat(M, M.map, op, s);
  } else if (sweep) {
    OpPost0<T, POST_JACOBI> op{avals<T>(A), wdv<T>(L0), y, t, nullptr, z, h->r, h->q, h->p, cc.mode, cc.flexible,
                               h->sc, cc.done, h->partials, h->counter};
    launch_mat(A, A.map, op, s);
  } else {
    OpPost0<T, POST_NONE> op{nullptr, wdv<T>(L0), y, t, nullptr, z, h->r, h->q, h->p, cc.mode, cc.flexible,
                             h->sc, cc.done, h->partials, h->counter};
    launch_rows(RowMap{}, n, A.rp, A.ci, op, s);
  }
}

template <typename T>
void load_y0(amg_hierarchy *h, const double *src) {
  Level &L0 = h->lev[0];
  const int n = L0.A.n;
  const bool write_y = !std::is_same<T, double>::value || L0.y != (void *)src;
  k_load_y0<T><<<grid_for(n), TPB, 0, h->mem.stream>>>(n, src, wdv<T>(L0), vec<T>(L0.y), vec<T>(L0.s), write_y,
                                                        h->prm.nu1 > 0 && h->prm.smoother == AMG_SMOOTH_JACOBI);
  AMG_CHECK_LAUNCH();
}

template <typename T, typename TP>
int pcg_impl(amg_hierarchy *h, const double *b, double *x, double rtol, int maxit, int *iters_out, double *hist_out,
             int hist_cap) {
  cudaStream_t s = h->mem.stream;
  Level &L0 = h->lev[0];
  const DCsr &A = L0.A;
  const int n = A.n;
  const double bt = sizeof(T);
  const bool fp64 = std::is_same<T, double>::value;
  const int flexible = fp64 ? 0 : 1;
  if (h->hist_cap < maxit + 1) {
    if (h->hist) h->mem.put(h->hist, sizeof(double) * h->hist_cap);
    h->hist_cap = maxit + 1;
    h->hist = h->mem.get_n<double>(h->hist_cap);
  }
  PcgScalars init{};
  init.maxit = maxit;
  AMG_CUDA(cudaMemcpyAsync(h->sc, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  *h->h_done = 0;
  const int *done = &h->sc->done;
  T *y0 = vec<T>(L0.y);  // aliases r in FP64 mode
  T *s0 = vec<T>(L0.s);
  const T *wd0 = wdv<T>(L0);
  // the pointwise first pre-smoothing step s = wd .* y (Jacobi); FSAI forms s in the cycle
  const bool pre = h->prm.nu1 > 0 && h->prm.smoother == AMG_SMOOTH_JACOBI;
  const double *a64 = avals<double>(A);
  {
    ProfScope ps(s, AMG_K_SOLVE_OTHER, 12.0 * A.nnz + 4.0 * (n + 1) + 8.0 * 3 * n + (fp64 ? 0 : bt * n) + 2 * bt * n);
    OpInit<T> op{a64, x, b, h->r, wd0, y0, s0, !fp64, pre, rtol, h->sc, h->hist, h->partials, h->counter};
    launch_mat(A, A.map64, op, s);
  }
  CycleCtx cc{done, POST_FIRST, flexible};
  vcycle<T, TP>(h, h->z, cc);
  cc.mode = POST_ITER;
  const double spmv_bytes = 12.0 * A.nnz + 4.0 * (n + 1) + 16.0 * n;
  const double upd_bytes = 48.0 + 2.0 * bt + (fp64 ? 0.0 : bt);
  const bool vec_ok = aligned16(x) && aligned16(h->r) && aligned16(h->p) && aligned16(h->q) && aligned16(wd0) &&
                      aligned16(s0) && aligned16(y0) && aligned16(h->z);
  // one iteration: q = A p and (p, q); x, r update; z = M r; p = z + beta p
  auto iteration = [&]() {
    cudaStream_t st = h->mem.stream;
    {
      ProfScope ps(st, AMG_K_SPMV_DOT, spmv_bytes, 0);
      OpSpmvDot op{a64, h->p, h->q, h->sc, h->partials, h->counter};
      launch_mat(A, A.map64, op, st);
    }
    {
      ProfScope ps(st, AMG_K_PCG_UPDATE, upd_bytes * n, 0);
      if (vec_ok)
        k_pcg_update<T, true><<<grid_for((n + 1) / 2), TPB, 0, st>>>(n, x, h->r, h->p, h->q, wd0, y0, s0, !fp64,
                                                                     pre, h->sc, h->hist, h->hist_cap, h->d_done,
                                                                     h->partials, h->counter);
      else
        k_pcg_update<T, false><<<grid_for(n), TPB, 0, st>>>(n, x, h->r, h->p, h->q, wd0, y0, s0, !fp64, pre, h->sc,
                                                            h->hist, h->hist_cap, h->d_done, h->partials, h->counter);
      AMG_CHECK_LAUNCH();
    }
    vcycle<T, TP>(h, h->z, cc);
    {
      ProfScope ps(st, AMG_K_DIRECTION, 24.0 * n, 0);
      if (vec_ok) k_direction<true><<<grid_for((n + 1) / 2), TPB, 0, st>>>(n, h->z, h->p, h->sc);
      else k_direction<false><<<grid_for(n), TPB, 0, st>>>(n, h->z, h->p, h->sc);
      AMG_CHECK_LAUNCH();
    }
  };
  // Unless its kernels are being event-timed, the iteration is captured once (on a stream of the
  // hierarchy's own; capture does not run it) and replayed on the solve's
  // stream: one launch per iteration instead of one per kernel.  Capture and
  // instantiation cost little; launching the ~35 kernels of an iteration one
  // by one is host-bound (a first solve of 128^3 Poisson took 10.6 ms that way
  // against 9.5 ms replayed).
  const bool use_graph = !prof_records_solve();
  if (use_graph && (h->iter_exec == nullptr || h->iter_x != x || h->iter_hist != h->hist)) {
    if (h->iter_exec) AMG_CUDA(cudaGraphExecDestroy(h->iter_exec));
    h->iter_exec = nullptr;
    if (!h->cap_stream) AMG_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    const long long before = g_launches.load();
    h->mem.stream = h->cap_stream;
    AMG_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    try {
      iteration();
    } catch (...) {
      cudaStreamEndCapture(h->cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      h->mem.stream = s;
      throw;
    }
    const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &g);
    h->mem.stream = s;
    AMG_CUDA(ec);
    h->iter_launches = g_launches.load() - before;
    g_launches.fetch_sub(h->iter_launches);
    const cudaError_t ei = cudaGraphInstantiate(&h->iter_exec, g, 0);
    cudaGraphDestroy(g);
    AMG_CUDA(ei);
    h->iter_x = x;
    h->iter_hist = h->hist;
  }
  for (int it = 1; it <= maxit; ++it) {
    if (use_graph) {
      AMG_CUDA(cudaGraphLaunch(h->iter_exec, s));
      g_launches.fetch_add(h->iter_launches);
    } else {
      iteration();
    }
    AMG_CUDA(cudaEventRecord(h->iter_ev[it & 1], s));
    // keep one iteration in flight: wait for the previous one, then test the flag
    if (it > 1) {
      AMG_CUDA(cudaEventSynchronize(h->iter_ev[(it - 1) & 1]));
      if (*(volatile int *)h->h_done) break;
    }
  }
  PcgScalars out{};
  AMG_CUDA(cudaMemcpyAsync(&out, h->sc, sizeof(out), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  prof_collect(s);
  if (iters_out) *iters_out = out.iters;
  if (hist_out && hist_cap > 0) {
    const int cnt = std::min(hist_cap, out.iters + 1);
    AMG_CUDA(cudaMemcpy(hist_out, h->hist, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
  }
  if (out.status != AMG_OK) return out.status;
  if (!out.done) return AMG_ERR_NO_CONVERGENCE;
  return AMG_OK;
}

template <typename T, typename TP>
void vcycle_apply_impl(amg_hierarchy *h, const double *y, double *z) {
  load_y0<T>(h, y);
  CycleCtx cc{h->d_zero, POST_APPLY, 0};
  vcycle<T, TP>(h, z, cc);
}

template <typename T>
void alloc_vectors(amg_hierarchy *h) {
  for (int k = 0; k < h->nlevels; ++k) {
    Level &L = h->lev[k];
    const int n = L.A.n;
    auto get = [&](size_t cnt) { return static_cast<void *>(h->mem.get_n<T>(cnt)); };
    if (k == 0 && std::is_same<T, double>::value) L.y = h->r;  // FP64: V-cycle input is the CG residual
    else L.y = get(n);
    L.z = get(n);
    if (k < h->nlevels - 1 || k == 0) {
      L.s = get(n);
      L.r = get(n);
      L.w = get(n);
    }
  }
}

}  // namespace

// Forms the dense operator of the levels from kd on (see k_dop_sparse): kd is
// the first level below level 0 with at most kDenseOpRows rows, if the
// hierarchy goes further down than that level.
constexpr int kDenseOpRows = 1024;

void build_dense_tail(amg_hierarchy *h) {
  h->dense_level = -1;
  const int Lst = h->nlevels - 1;
  int kd = -1;
  for (int k = 1; k < Lst; ++k)
    if (h->lev[k].A.n <= kDenseOpRows) {
      kd = k;
      break;
    }
  if (kd < 0) return;
  Mem &m = h->mem;
  cudaStream_t s = m.stream;
  const amg_params &prm = h->prm;
  auto blocks = [](int64_t cnt) { return std::max(1, ceil_div(cnt, TPB)); };
  ProfScope ps(s, AMG_K_SETUP_OTHER, 0.0);
  const int nl = h->nL;
  Buf<double> Mn(m, (size_t)nl * nl);
  k_dop_coarse<<<blocks((int64_t)nl * nl), TPB, 0, s>>>(nl, h->Linv, Mn.p);
  AMG_CHECK_LAUNCH();
  const bool fsai = prm.smoother == AMG_SMOOTH_FSAI;
  for (int k = Lst - 1; k >= kd; --k) {
    const Level &L = h->lev[k];
    const DCsr &A = L.A, &P = L.P, &R = L.R;
    const int n = A.n, nc = P.ncols;
    const int64_t nn = (int64_t)n * n;
    // FSAI: the smoothing matrix W = omega G^T G, dense
    Buf<double> W;
    if (fsai) {
      Buf<double> Gd(m, (size_t)nn);
      k_dop_csr_dense<<<blocks(nn), TPB, 0, s>>>(n, L.G.rp, L.G.ci, L.G.v, Gd.p);
      AMG_CHECK_LAUNCH();
      W = Buf<double>(m, (size_t)nn);
      k_dop_sparse<<<blocks(nn), TPB, 0, s>>>(n, n, L.GT.rp, L.GT.ci, L.GT.v, Gd.p, nullptr, nullptr, 0.0, 1.0, W.p);
      AMG_CHECK_LAUNCH();
    }
    // T + W (I - A T): one smoothing sweep applied to the columns of T
    auto sweep = [&](Buf<double> &T) {
      Buf<double> T2(m, (size_t)nn);
      if (fsai) {
        Buf<double> E(m, (size_t)nn);
        k_dop_sparse<<<blocks(nn), TPB, 0, s>>>(n, n, A.rp, A.ci, A.v, T.p, nullptr, nullptr, 1.0, -1.0, E.p);
        AMG_CHECK_LAUNCH();
        k_dop_gemm_add<<<blocks(nn), TPB, 0, s>>>(n, n, n, W.p, E.p, T.p, T2.p);
        AMG_CHECK_LAUNCH();
      } else {
        k_dop_sparse<<<blocks(nn), TPB, 0, s>>>(n, n, A.rp, A.ci, A.v, T.p, T.p, L.wd, 1.0, -1.0, T2.p);
        AMG_CHECK_LAUNCH();
      }
      std::swap(T, T2);
    };
    // X: the pre-smoothing sweeps applied to the identity
    Buf<double> X;
    if (prm.nu1 > 0) {
      X = Buf<double>(m, (size_t)nn);
      if (fsai) {
        AMG_CUDA(cudaMemcpyAsync(X.p, W.p, sizeof(double) * (size_t)nn, cudaMemcpyDeviceToDevice, s));
      } else {
        k_dop_sparse<<<blocks(nn), TPB, 0, s>>>(n, n, A.rp, A.ci, A.v, nullptr, nullptr, L.wd, 1.0, -1.0, X.p);
        AMG_CHECK_LAUNCH();
      }
      for (int j = 1; j < prm.nu1; ++j) sweep(X);
    }
    Buf<double> E(m, (size_t)nn);  // I - A X
    k_dop_sparse<<<blocks(nn), TPB, 0, s>>>(n, n, A.rp, A.ci, A.v, X.p, nullptr, nullptr, 1.0, -1.0, E.p);
    AMG_CHECK_LAUNCH();
    Buf<double> V(m, (size_t)nc * n);  // R E
    k_dop_sparse<<<blocks((int64_t)nc * n), TPB, 0, s>>>(nc, n, R.rp, R.ci, R.v, E.p, nullptr, nullptr, 0.0, 1.0,
                                                         V.p);
    AMG_CHECK_LAUNCH();
    E.reset();
    Buf<double> U(m, (size_t)nc * n);  // M_{k+1} R E
    k_dop_gemm<<<blocks((int64_t)nc * n), TPB, 0, s>>>(nc, nc, n, Mn.p, V.p, U.p);
    AMG_CHECK_LAUNCH();
    V.reset();
    Buf<double> T(m, (size_t)nn);  // X + P U
    k_dop_sparse<<<blocks(nn), TPB, 0, s>>>(n, n, P.rp, P.ci, P.v, U.p, X.p, nullptr, 0.0, 1.0, T.p);
    AMG_CHECK_LAUNCH();
    U.reset();
    X.reset();
    for (int j = 0; j < prm.nu2; ++j) sweep(T);  // post-smoothing sweeps
    Mn = std::move(T);
  }
  h->dense_op = Mn.release();
  h->dense_level = kd;
}

void prepare_solve(amg_hierarchy *h) {
  Mem &m = h->mem;
  cudaStream_t s = m.stream;
  const int prec = h->prm.precision;
  const bool fp64 = prec == AMG_PREC_FP64;
  const int n0 = h->lev[0].A.n;
  AMG_CUDA(cudaFuncSetAttribute(k_coarse_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * sizeof(double) * kMaxDense)));
  AMG_CUDA(cudaFuncSetAttribute(k_coarse_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * sizeof(double) * kMaxDense)));
  for (int k = 0; k < h->nlevels; ++k) {
    Level &L = h->lev[k];
    const int n = L.A.n;
    const bool last = k == h->nlevels - 1;
    L.A.map = choose_map(L.A.nnz, L.A.n, fp64);
    L.A.map64 = choose_map(L.A.nnz, L.A.n, true);
    if (!last) {
      L.P.map = choose_map(L.P.nnz, L.P.n, fp64);
      L.R.map = choose_map(L.R.nnz, L.R.n, fp64);
    }
    L.wd = m.get_n<double>(n);
    if (!fp64) L.wd32 = m.get_n<float>(n);
    {
      ProfScope ps(s, AMG_K_SETUP_OTHER, 4.0 * (n + 1) + 12.0 * L.A.nnz + 12.0 * n);
      k_make_wd<<<grid_for(n), TPB, 0, s>>>(n, L.A.rp, L.A.ci, L.A.v, h->prm.omega, L.wd, L.wd32);
      AMG_CHECK_LAUNCH();
    }
    if (!fp64) {  // CSR FP32 copies (the CSR kernels of small levels and the export keep them)
      L.A.v32 = m.get_n<float>(std::max<int64_t>(L.A.nnz, 1));
      {
        ProfScope ps(s, AMG_K_SETUP_OTHER, 12.0 * L.A.nnz);
        k_to_f32<<<grid_for(L.A.nnz), TPB, 0, s>>>(L.A.nnz, L.A.v, L.A.v32);
        AMG_CHECK_LAUNCH();
      }
      if (!last) {
        for (DCsr *M : {&L.P, &L.R}) {
          ProfScope ps(s, AMG_K_SETUP_OTHER, (prec == AMG_PREC_FP32 ? 12.0 : 10.0) * M->nnz);
          if (prec == AMG_PREC_FP32) {
            M->v32 = m.get_n<float>(std::max<int64_t>(M->nnz, 1));
            k_to_f32<<<grid_for(M->nnz), TPB, 0, s>>>(M->nnz, M->v, M->v32);
          } else {
            M->v16 = m.get_n<__nv_bfloat16>(std::max<int64_t>(M->nnz, 1));
            k_to_bf16<<<grid_for(M->nnz), TPB, 0, s>>>(M->nnz, M->v, M->v16);
          }
          AMG_CHECK_LAUNCH();
        }
      }
    }
    // SELL copies for the large matrices (A also in FP64 on level 0 for the CG products)
    if (n >= kSellSolveRows) build_sell(m, L.A, fp64 || k == 0, !fp64, false);
    if (!last) {
      if (L.P.n >= kSellSolveRows) build_sell(m, L.P, fp64, prec == AMG_PREC_FP32, prec == AMG_PREC_FP32_BF16PR);
      if (L.R.n >= kSellSolveRows) build_sell(m, L.R, fp64, prec == AMG_PREC_FP32, prec == AMG_PREC_FP32_BF16PR);
    }
    if (!last && h->prm.smoother == AMG_SMOOTH_FSAI) {  // G and omega G^T, stored like A
      build_fsai(h, k);
      for (DCsr *M : {&L.G, &L.GT}) {
        M->map = choose_map(M->nnz, M->n, fp64);
        M->map64 = choose_map(M->nnz, M->n, true);
        if (!fp64) {
          M->v32 = m.get_n<float>(std::max<int64_t>(M->nnz, 1));
          ProfScope ps(s, AMG_K_FSAI, 12.0 * M->nnz, k);
          k_to_f32<<<grid_for(M->nnz), TPB, 0, s>>>(M->nnz, M->v, M->v32);
          AMG_CHECK_LAUNCH();
        }
        if (n >= kSellSolveRows) build_sell(m, *M, fp64, !fp64, false);
      }
    }
  }
  // CG vectors (FP64) and scalars
  h->r = m.get_n<double>(n0);
  h->z = m.get_n<double>(n0);
  h->p = m.get_n<double>(n0);
  h->q = m.get_n<double>(n0);
  h->sc = m.get_n<PcgScalars>(1);
  h->d_zero = m.get_n<int>(1);
  AMG_CUDA(cudaMemsetAsync(h->d_zero, 0, sizeof(int), s));
  h->partials = m.get_n<double>(3 * MAX_GRID);
  h->counter = m.get_n<unsigned int>(1);
  AMG_CUDA(cudaMemsetAsync(h->counter, 0, sizeof(unsigned int), s));
  if (fp64) alloc_vectors<double>(h);
  else alloc_vectors<float>(h);
  build_dense_tail(h);
  AMG_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&h->h_done), sizeof(int), cudaHostAllocMapped));
  *h->h_done = 0;
  AMG_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void **>(&h->d_done), h->h_done, 0));
  AMG_CUDA(cudaEventCreateWithFlags(&h->iter_ev[0], cudaEventDisableTiming));
  AMG_CUDA(cudaEventCreateWithFlags(&h->iter_ev[1], cudaEventDisableTiming));
}

void release_solve(amg_hierarchy *h) {
  if (h->iter_exec) cudaGraphExecDestroy(h->iter_exec);
  h->iter_exec = nullptr;
  if (h->vc_exec) cudaGraphExecDestroy(h->vc_exec);
  h->vc_exec = nullptr;
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  h->cap_stream = nullptr;
  if (h->h_done) cudaFreeHost(h->h_done);
  h->h_done = nullptr;
  for (auto &e : h->iter_ev)
    if (e) cudaEventDestroy(e);
  if (h->df_ev) cudaEventDestroy(h->df_ev);
  h->df_ev = nullptr;
}

int pcg_solve(amg_hierarchy *h, const double *b, double *x, double rtol, int maxit, int *iters, double *hist,
              int hist_cap) {
  switch (h->prm.precision) {
    case AMG_PREC_FP64: return pcg_impl<double, double>(h, b, x, rtol, maxit, iters, hist, hist_cap);
    case AMG_PREC_FP32: return pcg_impl<float, float>(h, b, x, rtol, maxit, iters, hist, hist_cap);
    default: return pcg_impl<float, __nv_bfloat16>(h, b, x, rtol, maxit, iters, hist, hist_cap);
  }
}

// One V-cycle z = M^-1 y.  Unless its kernels are being event-timed, the
// launches are captured once per (y, z) pair (on the hierarchy's capture
// stream, which does not run them) and replayed as one graph launch: a
// V-cycle's ~40 launches one by one are host-bound on the small levels (the
// PCG iteration is replayed the same way).
void vcycle_apply(amg_hierarchy *h, const double *y, double *z) {
  auto run = [&]() {
    switch (h->prm.precision) {
      case AMG_PREC_FP64: vcycle_apply_impl<double, double>(h, y, z); break;
      case AMG_PREC_FP32: vcycle_apply_impl<float, float>(h, y, z); break;
      default: vcycle_apply_impl<float, __nv_bfloat16>(h, y, z); break;
    }
  };
  cudaStream_t s = h->mem.stream;
  if (prof_records_solve()) {
    run();
    prof_collect(s);
    return;
  }
  if (h->vc_exec == nullptr || h->vc_y != y || h->vc_z != z) {
    if (h->vc_exec) AMG_CUDA(cudaGraphExecDestroy(h->vc_exec));
    h->vc_exec = nullptr;
    if (!h->cap_stream) AMG_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    const long long before = g_launches.load();
    h->mem.stream = h->cap_stream;
    AMG_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    try {
      run();
    } catch (...) {
      cudaStreamEndCapture(h->cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      h->mem.stream = s;
      throw;
    }
    const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &g);
    h->mem.stream = s;
    AMG_CUDA(ec);
    h->vc_launches = g_launches.load() - before;
    g_launches.fetch_sub(h->vc_launches);
    const cudaError_t ei = cudaGraphInstantiate(&h->vc_exec, g, 0);
    cudaGraphDestroy(g);
    AMG_CUDA(ei);
    h->vc_y = y;
    h->vc_z = z;
  }
  AMG_CUDA(cudaGraphLaunch(h->vc_exec, s));
  g_launches.fetch_add(h->vc_launches);
}

void spmv_level(amg_hierarchy *h, int level, const double *x, double *y) {
  const DCsr &A = h->lev[level].A;
  ProfScope ps(h->mem.stream, AMG_K_SOLVE_OTHER, 12.0 * A.nnz + 4.0 * (A.n + 1) + 16.0 * A.n);
  if (on_sell(A) && A.sell.v) {
    OpSpmv op{A.sell.v, x, y};
    launch_mat(A, A.map64, op, h->mem.stream);
  } else {
    OpSpmv op{A.v, x, y};
    launch_rows(A.map64, A.n, A.rp, A.ci, op, h->mem.stream);
  }
}

}  // namespace amg

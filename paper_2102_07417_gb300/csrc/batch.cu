// batch.cu -- PCG on a block of k right-hand sides at once (Sec. 3.1: dense
// blocks stored row-wise, "efficient for linear systems with multiple
// right-hand-sides").  Vectors are n x k row-major; every sparse product is an
// SpMM in which a group of K >= k lanes owns one row and lane j its column j,
// so a nonzero is read once for all k columns and the k-wide gathers are
// coalesced.  The V-cycle (Algorithm 2) and the CG recurrences are the same
// as the single right-hand side path, with per-column scalars (alpha_j,
// beta_j, rho_j) and a per-column convergence mask: a converged column is
// frozen (its x and r are no longer updated) while the others continue.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr int TPB = 256;
constexpr int MAX_GRID = kNumSMs * 8;
constexpr int KMAX = 32;  // largest block width

struct BScal {
  double rho[KMAX], alpha[KMAX], beta[KMAX], rr[KMAX], bb[KMAX], tol[KMAX];
  int iters[KMAX], done[KMAX], status[KMAX];
  int first[KMAX];  // column admitted since the last iteration (continuous batching): no CG step yet
  unsigned int ticket[KMAX];  // admission number of the request in each column (continuous batching)
  int all_done, maxit, k;
};

__device__ __forceinline__ float tof(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float tof(float v) { return v; }
__device__ __forceinline__ double tof(double v) { return v; }

// ------------------------------------------------------ double-float --
// The FP64 outer product of the FP32 modes in FP32 arithmetic (GB300 runs
// FP32 at many times its FP64 rate): a value v is held as the pair
// hi = fl32(v), lo = fl32(v - hi), and products are accumulated with the
// error-free transformations TwoProd (by FMA) and TwoSum (Knuth), keeping
// about 48 bits -- far below the 1e-8 outer tolerance, with no FP64 FMA.
__device__ __forceinline__ float2 df_split(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

// (sh, sl) += (ah + al) (ph + pl), dropping al * pl.  Intrinsics keep every
// operation rounded as written (no contraction).
__device__ __forceinline__ void df_madd(float ah, float al, float ph, float pl, float &sh, float &sl) {
  const float prod = __fmul_rn(ah, ph);
  const float perr = __fmaf_rn(ah, ph, -prod);
  const float cross = __fmaf_rn(ah, pl, __fmaf_rn(al, ph, perr));
  const float s = __fadd_rn(sh, prod);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(prod, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, cross));
}

// Totals over the grid's block partials, run by every thread of the last
// block: pair (c, j) of the NV x kc (value, column) pairs is summed by
// TPB / P threads over interleaved blocks, then by one thread over those in
// order (a fixed order, so the totals are deterministic).  tot[c][j] in
// shared memory on return.
template <int NV>
__device__ void grid_totals(const double *partials, int nblocks, int kc, double (*tot)[KMAX]) {
  __shared__ double red[TPB];
  const int npairs = NV * kc;
  int P = 1;
  while (P < npairs) P <<= 1;
  const int S = TPB / P;
  const int pair = threadIdx.x % P, sub = threadIdx.x / P;
  double t = 0.0;
  if (pair < npairs) {
    const int c = pair / kc, j = pair % kc;
#pragma unroll 4
    for (int b = sub; b < nblocks; b += S) t += __ldcg(&partials[(b * 3 + c) * KMAX + j]);
  }
  red[threadIdx.x] = t;
  __syncthreads();
  if (threadIdx.x < npairs) {
    double v = 0.0;
    for (int u = 0; u < S; ++u) v += red[u * P + threadIdx.x];
    tot[threadIdx.x / kc][threadIdx.x % kc] = v;
  }
  __syncthreads();
}

// Per-column sums of NV values: v[c] is this thread's partial for column
// (lane % K).  Block partials go to partials[(block * 3 + c) * KMAX + j]; the
// last block to finish gets the totals out[c] for its column j = lane % K
// (summed in block order, deterministic) and returns true.
template <int K, int NV>
__device__ bool col_reduce(const double (&v)[NV], double *partials, unsigned int *counter, double (&out)[NV]) {
  __shared__ double red[NV][TPB];
  __shared__ bool last;
#pragma unroll
  for (int c = 0; c < NV; ++c) red[c][threadIdx.x] = v[c];
  __syncthreads();
  if (threadIdx.x < K) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double s = 0.0;
      for (int m = threadIdx.x; m < TPB; m += K) s += red[c][m];
      partials[(blockIdx.x * 3 + c) * KMAX + threadIdx.x] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  __shared__ double tot[NV][KMAX];
  grid_totals<NV>(partials, gridDim.x, K, tot);
  if (threadIdx.x < K) {
#pragma unroll
    for (int c = 0; c < NV; ++c) out[c] = tot[c][threadIdx.x];
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

template <int NV>
struct BAcc {
  double v[NV > 0 ? NV : 1];
};

// SpMM row kernel: G x K lanes per row (K * G <= 32).  Lane (g, j) takes
// column j (< k) and the row's entries g, g + G, g + 2G, ...; the G partial
// sums of a column are then added with shuffles (a fixed order).  G > 1 keeps
// more loads in flight on the short, long-row coarse levels, where one lane
// walking a whole row for its column was bound by the row's load latency.
// For each (row, j): sum = sum_p mat(p) vec(ci[p], j); op.out(row, j, sum, acc).
template <int K, int G, class Op>
__global__ void __launch_bounds__(TPB) k_brows(int n, int k, const int *__restrict__ rp, const int *__restrict__ ci,
                                               Op op) {
  using T = typename Op::T;
  constexpr int NA = Op::NV > 0 ? Op::NV : 1;
  constexpr int LPR = K * G;  // lanes per row
  constexpr int RPW = 32 / LPR;
  if (op.skip()) return;
  const int lane = threadIdx.x & 31, j = lane & (K - 1), g = (lane / K) & (G - 1), grp = lane / LPR;
  const int gw = (blockIdx.x * TPB + threadIdx.x) >> 5, nw = (gridDim.x * TPB) >> 5;
  BAcc<NA> acc;
#pragma unroll
  for (int c = 0; c < NA; ++c) acc.v[c] = 0.0;
  for (int base = gw * RPW; base < n; base += nw * RPW) {  // the whole warp iterates together
    const int row = base + grp;
    T sum = T(0);
    if constexpr (Op::kMatrix) {
      if (row < n && j < k) {
        const int e = rp[row + 1];
#pragma unroll 4
        for (int p = rp[row] + g; p < e; p += G) sum = fma(op.mat(p), op.vec(ci[p], j), sum);
      }
#pragma unroll
      for (int o = K; o < LPR; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if (row < n && j < k && g == 0) op.out(row, j, sum, acc);
  }
  op.finish(acc);
}

// Per-column sums of NV values when each thread holds all K columns of its
// rows (acc[j].v[c]): warp butterflies, then warps in order, then blocks in
// order (deterministic).  Same partials layout and return convention as
// col_reduce: in the last block thread j < K gets column j's totals.
template <int K, int NV>
__device__ bool rows_reduce(const BAcc<NV> (&acc)[K], double *partials, unsigned int *counter,
                            double (&out)[NV]) {
  __shared__ double red[NV][K][TPB / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < K; ++j) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double v = acc[j].v[c];
#pragma unroll
      for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[c][j][w] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < K) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double t = 0.0;
      for (int ww = 0; ww < TPB / 32; ++ww) t += red[c][threadIdx.x][ww];
      partials[(blockIdx.x * 3 + c) * KMAX + threadIdx.x] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  __shared__ double tot[NV][KMAX];
  grid_totals<NV>(partials, gridDim.x, K, tot);
  if (threadIdx.x < K) {
#pragma unroll
    for (int c = 0; c < NV; ++c) out[c] = tot[c][threadIdx.x];
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// sum[j] += a * p[j] for the K values of one block row, loaded with 16-byte
// vector loads (K * sizeof(T) a multiple of 16), else in 8- or 4-byte pieces.
template <int K, typename T>
__device__ __forceinline__ void fma_row(const T *__restrict__ p, T a, T (&sum)[K]) {
  if constexpr (sizeof(T) * K % 16 == 0) {
#pragma unroll
    for (int v = 0; v < (int)(K * sizeof(T) / 16); ++v) {
      if constexpr (sizeof(T) == 8) {
        const double2 d = __ldg(reinterpret_cast<const double2 *>(p) + v);
        sum[2 * v] = fma(a, d.x, sum[2 * v]);
        sum[2 * v + 1] = fma(a, d.y, sum[2 * v + 1]);
      } else {
        const float4 f = __ldg(reinterpret_cast<const float4 *>(p) + v);
        sum[4 * v] = fma(a, f.x, sum[4 * v]);
        sum[4 * v + 1] = fma(a, f.y, sum[4 * v + 1]);
        sum[4 * v + 2] = fma(a, f.z, sum[4 * v + 2]);
        sum[4 * v + 3] = fma(a, f.w, sum[4 * v + 3]);
      }
    }
  } else if constexpr (sizeof(T) == 4 && K == 2) {
    const float2 f = __ldg(reinterpret_cast<const float2 *>(p));
    sum[0] = fma(a, f.x, sum[0]);
    sum[1] = fma(a, f.y, sum[1]);
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) sum[j] = fma(a, __ldg(p + j), sum[j]);
  }
}

// SpMM on the sliced-ELLPACK copy: a thread per row holding all K columns
// (the matrix entry is loaded once, the block row of the gathered vector with
// vector loads).  vec (k == K and a 16-byte aligned vector) uses the vector
// loads; otherwise k values are loaded one by one.
template <int K, class Op>
__global__ void __launch_bounds__(TPB) k_bsell(int n, int k, bool vec, int nslices, const int *__restrict__ off,
                                               const int *__restrict__ col, const int *__restrict__ perm, Op op) {
  using T = typename Op::T;
  constexpr int NA = Op::NV > 0 ? Op::NV : 1;
  if (op.skip()) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * TPB + threadIdx.x) >> 5, nw = (gridDim.x * TPB) >> 5;
  BAcc<NA> acc[K];
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int c = 0; c < NA; ++c) acc[j].v[c] = 0.0;
  for (int sl = gw; sl < nslices; sl += nw) {
    const int q = sl * 32 + lane;
    const bool valid = q < n;
    const int row = valid ? (perm ? perm[q] : q) : 0;
    T sum[K];
#pragma unroll
    for (int j = 0; j < K; ++j) sum[j] = T(0);
    if constexpr (Op::kMatrix) {
      const int b = off[sl] + lane, len = (off[sl + 1] - off[sl]) >> 5;
#pragma unroll(K <= 4 ? 4 : 2)
      for (int t = 0; t < len; ++t) {
        const int idx = b + 32 * t;
        const int c = __ldg(col + idx);
        const T a = op.mat(idx);
        const T *xr = op.vrow(c);
        if (vec) {
          fma_row<K, T>(xr, a, sum);
        } else {
#pragma unroll
          for (int j = 0; j < K; ++j)
            if (j < k) sum[j] = fma(a, __ldg(xr + j), sum[j]);
        }
      }
    }
    if (valid) {
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j < k) op.out(row, j, sum[j], acc[j]);
    }
  }
  if constexpr (Op::NV > 0) {
    double tot[Op::NV];
    if (rows_reduce<K, Op::NV>(acc, op.partials, op.counter, tot)) op.finish_col(tot);
  }
}

// ------------------------------------------------------------------ ops --
// Block vectors are row-major with leading dimension k: v[i * k + j].

// r = b - A x;  (b_j, b_j), (r_j, r_j);  V-cycle input y0 / s0.
template <int K, typename TV>
struct BInit {
  using T = double;
  static constexpr int NV = 2;
  static constexpr bool kMatrix = true;
  int k;
  const double *a, *x, *b;
  double *r;
  const TV *wd;
  TV *y0, *s0;
  bool write_y, pre;
  double rtol;
  BScal *sc;
  double *hist;
  int hist_cap;
  double *partials;
  unsigned int *counter;
  __device__ bool skip() const { return false; }
  __device__ double mat(int p) const { return __ldg(a + p); }
  __device__ double vec(int c, int j) const { return __ldg(x + (size_t)c * k + j); }
  __device__ const double *vrow(int c) const { return x + (size_t)c * k; }
  __host__ __device__ const double *vbase() const { return x; }
  __device__ void out(int i, int j, double sum, BAcc<NV> &acc) const {
    const size_t o = (size_t)i * k + j;
    const double bi = b[o], ri = bi - sum;
    r[o] = ri;
    acc.v[0] = fma(bi, bi, acc.v[0]);
    acc.v[1] = fma(ri, ri, acc.v[1]);
    const TV yi = static_cast<TV>(ri);
    if (write_y) y0[o] = yi;
    s0[o] = pre ? wd[i] * yi : TV(0);
  }
  __device__ void finish(BAcc<NV> &acc) const {
    double tot[2];
    if (col_reduce<K, 2>(acc.v, partials, counter, tot)) finish_col(tot);
  }
  // Run by every thread of the last block; thread j < k holds column j's totals.
  __device__ void finish_col(const double (&tot)[NV]) const {
    {
      const int j = threadIdx.x;
      if (j < k) {
        sc->bb[j] = tot[0];
        sc->rr[j] = tot[1];
        sc->tol[j] = rtol * sqrt(tot[0]);
        const double res = sqrt(tot[1]);
        if (hist_cap > 0) hist[j] = res;
        sc->iters[j] = 0;
        sc->status[j] = AMG_OK;
        sc->done[j] = (res < sc->tol[j] || tot[0] == 0.0) ? 1 : 0;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int all = 1;
        for (int c = 0; c < k; ++c) all &= sc->done[c];
        sc->all_done = all;
      }
    }
  }
};

// q = A p;  alpha_j = rho_j / (p_j, q_j) (columns not done).
template <int K>
struct BSpmvDot {
  using T = double;
  static constexpr int NV = 1;
  static constexpr bool kMatrix = true;
  int k;
  const double *a, *p;
  double *q;
  BScal *sc;
  double *partials;
  unsigned int *counter;
  __device__ bool skip() const { return sc->all_done; }
  __device__ double mat(int t) const { return __ldg(a + t); }
  __device__ double vec(int c, int j) const { return __ldg(p + (size_t)c * k + j); }
  __device__ const double *vrow(int c) const { return p + (size_t)c * k; }
  __host__ __device__ const double *vbase() const { return p; }
  __device__ void out(int i, int j, double sum, BAcc<NV> &acc) const {
    const size_t o = (size_t)i * k + j;
    q[o] = sum;
    acc.v[0] = fma(p[o], sum, acc.v[0]);
  }
  __device__ void finish(BAcc<NV> &acc) const {
    double tot[1];
    if (col_reduce<K, 1>(acc.v, partials, counter, tot)) finish_col(tot);
  }
  __device__ void finish_col(const double (&tot)[NV]) const {
    {
      const int j = threadIdx.x;
      if (j < k && !sc->done[j] && sc->first[j]) {
        sc->alpha[j] = 0.0;  // p_j = 0: its first step only forms z = M r
      } else if (j < k && !sc->done[j]) {
        if (!(tot[0] > 0.0)) {
          sc->status[j] = AMG_ERR_BREAKDOWN;
          sc->done[j] = 1;
          sc->alpha[j] = 0.0;
        } else {
          sc->alpha[j] = sc->rho[j] / tot[0];
        }
      }
    }
  }
};

// q = A p in double-float on the sliced-ELLPACK copy (a thread per row over
// the K columns; a2 = A as FP32 pairs, p2 = p as FP32 pairs), then the same
// per-column bookkeeping as BSpmvDot (op carries its pointers).
template <int K>
__global__ void __launch_bounds__(TPB) k_bsell_df(int n, int k, bool vec, int nslices, const int *__restrict__ off,
                                                  const int *__restrict__ col, const int *__restrict__ perm,
                                                  const float2 *__restrict__ a2, const float2 *__restrict__ p2,
                                                  BSpmvDot<K> op) {
  if (op.skip()) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * TPB + threadIdx.x) >> 5, nw = (gridDim.x * TPB) >> 5;
  BAcc<1> acc[K];
#pragma unroll
  for (int j = 0; j < K; ++j) acc[j].v[0] = 0.0;
  for (int sl_ = gw; sl_ < nslices; sl_ += nw) {
    const int q = sl_ * 32 + lane;
    const bool valid = q < n;
    const int row = valid ? (perm ? perm[q] : q) : 0;
    float sh[K], sl[K];
#pragma unroll
    for (int j = 0; j < K; ++j) sh[j] = sl[j] = 0.f;
    const int b = off[sl_] + lane, len = (off[sl_ + 1] - off[sl_]) >> 5;
#pragma unroll 2
    for (int t = 0; t < len; ++t) {
      const int idx = b + 32 * t;
      const int c = __ldg(col + idx);
      const float2 a = __ldg(a2 + idx);
      const float2 *pr = p2 + (size_t)c * k;
      if (vec && K % 2 == 0) {
#pragma unroll
        for (int u = 0; u < K / 2; ++u) {
          const float4 v = __ldg(reinterpret_cast<const float4 *>(pr) + u);
          df_madd(a.x, a.y, v.x, v.y, sh[2 * u], sl[2 * u]);
          df_madd(a.x, a.y, v.z, v.w, sh[2 * u + 1], sl[2 * u + 1]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) {
          if (j < k) {
            const float2 v = __ldg(pr + j);
            df_madd(a.x, a.y, v.x, v.y, sh[j], sl[j]);
          }
        }
      }
    }
    if (valid) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        if (j < k) {
          const size_t o = (size_t)row * k + j;
          const double qd = (double)sh[j] + (double)sl[j];
          op.q[o] = qd;
          acc[j].v[0] = fma(op.p[o], qd, acc[j].v[0]);
        }
      }
    }
  }
  double tot[1];
  if (rows_reduce<K, 1>(acc, op.partials, op.counter, tot)) op.finish_col(tot);
}

// A's FP64 values as FP32 pairs.
__global__ void k_split_df(int64_t m, const double *__restrict__ v, float2 *__restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = df_split(v[i]);
}

template <typename TT>
struct BResid {  // r = y - A s
  using T = TT;
  static constexpr int NV = 0;
  static constexpr bool kMatrix = true;
  int k;
  const T *a, *s, *y;
  T *r;
  const int *done;
  __device__ bool skip() const { return *done; }
  __device__ T mat(int p) const { return __ldg(a + p); }
  __device__ T vec(int c, int j) const { return __ldg(s + (size_t)c * k + j); }
  __device__ const T *vrow(int c) const { return s + (size_t)c * k; }
  __host__ __device__ const T *vbase() const { return s; }
  __device__ void out(int i, int j, T sum, BAcc<1> &) const {
    const size_t o = (size_t)i * k + j;
    r[o] = y[o] - sum;
  }
  __device__ void finish(BAcc<1> &) const {}
};

template <typename TT, typename TP>
struct BRestrict {  // y_c = R r;  s_c = wd_c y_c (pre = 1), 0 (pre = 0), not written (pre = -1)
  using T = TT;
  static constexpr int NV = 0;
  static constexpr bool kMatrix = true;
  int k;
  const TP *rv;
  const T *r, *wd;
  T *yc, *sc;
  int pre;
  const int *done;
  __device__ bool skip() const { return *done; }
  __device__ T mat(int p) const { return static_cast<T>(tof(rv[p])); }
  __device__ T vec(int c, int j) const { return __ldg(r + (size_t)c * k + j); }
  __device__ const T *vrow(int c) const { return r + (size_t)c * k; }
  __host__ __device__ const T *vbase() const { return r; }
  __device__ void out(int i, int j, T sum, BAcc<1> &) const {
    const size_t o = (size_t)i * k + j;
    yc[o] = sum;
    if (pre >= 0) sc[o] = pre ? wd[i] * sum : T(0);
  }
  __device__ void finish(BAcc<1> &) const {}
};

template <typename TT, typename TP>
struct BProlong {  // t = s + P z_c
  using T = TT;
  static constexpr int NV = 0;
  static constexpr bool kMatrix = true;
  int k;
  const TP *pv;
  const T *s, *zc;
  T *t;
  const int *done;
  __device__ bool skip() const { return *done; }
  __device__ T mat(int p) const { return static_cast<T>(tof(pv[p])); }
  __device__ T vec(int c, int j) const { return __ldg(zc + (size_t)c * k + j); }
  __device__ const T *vrow(int c) const { return zc + (size_t)c * k; }
  __host__ __device__ const T *vbase() const { return zc; }
  __device__ void out(int i, int j, T sum, BAcc<1> &) const {
    const size_t o = (size_t)i * k + j;
    t[o] = s[o] + sum;
  }
  __device__ void finish(BAcc<1> &) const {}
};

template <typename TT>
struct BJacobi {  // z = t + wd (y - A t)
  using T = TT;
  static constexpr int NV = 0;
  static constexpr bool kMatrix = true;
  int k;
  const T *a, *wd, *y, *t;
  T *z;
  const int *done;
  __device__ bool skip() const { return *done; }
  __device__ T mat(int p) const { return __ldg(a + p); }
  __device__ T vec(int c, int j) const { return __ldg(t + (size_t)c * k + j); }
  __device__ const T *vrow(int c) const { return t + (size_t)c * k; }
  __host__ __device__ const T *vbase() const { return t; }
  __device__ void out(int i, int j, T sum, BAcc<1> &) const {
    const size_t o = (size_t)i * k + j;
    z[o] = fma(wd[i], y[o] - sum, t[o]);
  }
  __device__ void finish(BAcc<1> &) const {}
};

enum { BPOST_APPLY = 0, BPOST_FIRST = 1, BPOST_ITER = 2 };

// Level-0 post-smoothing (or copy) fused with the per-column CG bookkeeping.
template <int K, typename TT, bool SWEEP>
struct BPost0 {
  using T = TT;
  static constexpr int NV = 2;
  static constexpr bool kMatrix = SWEEP;
  int k;
  const T *a, *wd, *y, *t;
  double *z;
  const double *r, *q;
  double *p;
  float2 *p2;  // p as FP32 pairs (double-float outer product), or nullptr
  int mode, flexible;
  BScal *sc;
  const int *done;
  double *partials;
  unsigned int *counter;
  __device__ bool skip() const { return *done; }
  __device__ T mat(int pp) const { return __ldg(a + pp); }
  __device__ T vec(int c, int j) const { return __ldg(t + (size_t)c * k + j); }
  __device__ const T *vrow(int c) const { return t + (size_t)c * k; }
  __host__ __device__ const T *vbase() const { return t; }
  __device__ void out(int i, int j, T sum, BAcc<NV> &acc) const {
    const size_t o = (size_t)i * k + j;
    const T zi = SWEEP ? fma(wd[i], y[o] - sum, t[o]) : t[o];
    const double zd = static_cast<double>(zi);
    z[o] = zd;
    if (mode != BPOST_APPLY) {
      acc.v[0] = fma(r[o], zd, acc.v[0]);
      if (mode == BPOST_FIRST) {
        p[o] = zd;
        if (p2) p2[o] = df_split(zd);
      }
      else if (flexible) acc.v[1] = fma(zd, q[o], acc.v[1]);
    }
  }
  __device__ void finish(BAcc<NV> &acc) const {
    if (mode == BPOST_APPLY) return;
    double tot[2];
    if (col_reduce<K, 2>(acc.v, partials, counter, tot)) finish_col(tot);
  }
  __device__ void finish_col(const double (&tot)[NV]) const {
    if (mode == BPOST_APPLY) return;
    {
      const int j = threadIdx.x;
      if (j < k && !sc->done[j]) {
        if (mode == BPOST_ITER && sc->first[j]) {
          sc->beta[j] = 0.0;  // p_j = 0 + z_j
          sc->first[j] = 0;
        } else if (mode == BPOST_ITER) {
          sc->beta[j] = flexible ? -sc->alpha[j] * tot[1] / sc->rho[j] : tot[0] / sc->rho[j];
        }
        sc->rho[j] = tot[0];
      }
    }
  }
};

// x += alpha_j p;  r -= alpha_j q (columns not done);  ||r_j||;  convergence;  V-cycle input.
// A thread per row holding its k <= K columns (16-byte vector loads when
// k == K); frozen columns (converged, or admitted since the last step) keep
// x and r bit for bit.
template <int K>
__device__ __forceinline__ void load_dr(const double *__restrict__ p, int k, bool vec, double (&v)[K]) {
  if (vec && K % 2 == 0) {
#pragma unroll
    for (int u = 0; u < K / 2; ++u) {
      const double2 d = reinterpret_cast<const double2 *>(p)[u];
      v[2 * u] = d.x;
      v[2 * u + 1] = d.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = j < k ? p[j] : 0.0;
  }
}

template <int K>
__device__ __forceinline__ void store_dr(double *__restrict__ p, int k, bool vec, const double (&v)[K]) {
  if (vec && K % 2 == 0) {
#pragma unroll
    for (int u = 0; u < K / 2; ++u) reinterpret_cast<double2 *>(p)[u] = make_double2(v[2 * u], v[2 * u + 1]);
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (j < k) p[j] = v[j];
  }
}

template <int K, typename T>
__global__ void __launch_bounds__(TPB) k_bupdate(int n, int k, bool vec, double *__restrict__ x, double *__restrict__ r,
                                                 const double *__restrict__ p, const double *__restrict__ q,
                                                 const T *__restrict__ wd, T *__restrict__ y0, T *__restrict__ s0,
                                                 bool write_y, bool pre, BScal *sc, double *hist, int hist_cap,
                                                 int *host_done, double *partials, unsigned int *counter) {
  if (sc->all_done) return;
  __shared__ double s_alpha[KMAX];
  __shared__ int s_frozen[KMAX];
  if (threadIdx.x < KMAX) {
    const int c = threadIdx.x;
    const int fz = c < k ? (sc->done[c] | sc->first[c]) : 1;
    s_frozen[c] = fz;
    s_alpha[c] = fz ? 0.0 : sc->alpha[c];
  }
  __syncthreads();
  double alpha[K];
  bool frozen[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    alpha[j] = s_alpha[j];
    frozen[j] = s_frozen[j];
  }
  BAcc<1> acc[K];
#pragma unroll
  for (int j = 0; j < K; ++j) acc[j].v[0] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const size_t o = (size_t)i * k;
    double xr[K], rr[K], pr[K], qr[K];
    load_dr<K>(r + o, k, vec, rr);
    load_dr<K>(x + o, k, vec, xr);
    load_dr<K>(p + o, k, vec, pr);
    load_dr<K>(q + o, k, vec, qr);
    const T w = pre ? wd[i] : T(0);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (!frozen[j]) {
        xr[j] = fma(alpha[j], pr[j], xr[j]);
        rr[j] = fma(-alpha[j], qr[j], rr[j]);
      }
      acc[j].v[0] = fma(rr[j], rr[j], acc[j].v[0]);
    }
    store_dr<K>(x + o, k, vec, xr);
    store_dr<K>(r + o, k, vec, rr);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (j < k) {
        const T yi = static_cast<T>(rr[j]);
        if (write_y) y0[o + j] = yi;
        s0[o + j] = pre ? w * yi : T(0);
      }
    }
  }
  double tot[1];
  if (!rows_reduce<K, 1>(acc, partials, counter, tot)) return;
  if (threadIdx.x < k) {
    const int c = threadIdx.x;
    if (!sc->done[c] && !sc->first[c]) {
      const int it = sc->iters[c] + 1;
      sc->iters[c] = it;
      sc->rr[c] = tot[0];
      const double res = sqrt(tot[0]);
      if (it < hist_cap) hist[(size_t)it * k + c] = res;
      if (res < sc->tol[c]) {
        sc->done[c] = 1;
      } else if (it >= sc->maxit) {
        sc->status[c] = AMG_ERR_NO_CONVERGENCE;
        sc->done[c] = 1;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int all = 1;
    for (int c = 0; c < k; ++c) all &= sc->done[c];
    sc->all_done = all;
    if (all && host_done) *(volatile int *)host_done = 1;
  }
}

// The same for wide batches (K > 8, where a row's columns do not fit in one
// thread's registers): consecutive threads take consecutive columns.
template <typename T>
__global__ void __launch_bounds__(TPB) k_bupdate_cols(int n, int k, double *__restrict__ x, double *__restrict__ r,
                                                 const double *__restrict__ p, const double *__restrict__ q,
                                                 const T *__restrict__ wd, T *__restrict__ y0, T *__restrict__ s0,
                                                 bool write_y, bool pre, BScal *sc, double *hist, int hist_cap,
                                                 int *host_done, double *partials, unsigned int *counter) {
  if (sc->all_done) return;
  __shared__ double s_alpha[KMAX];
  __shared__ int s_done[KMAX];
  if (threadIdx.x < k) {
    s_done[threadIdx.x] = sc->done[threadIdx.x] | sc->first[threadIdx.x];
    s_alpha[threadIdx.x] = s_done[threadIdx.x] ? 0.0 : sc->alpha[threadIdx.x];
  }
  __syncthreads();
  // thread t handles column t % kk of consecutive entries (kk = power of two >= k)
  int kk = 1;
  while (kk < k) kk <<= 1;
  const int j = threadIdx.x & (kk - 1);
  double v = 0.0;
  if (j < k) {
    const double alpha = s_alpha[j];
    const bool frozen = s_done[j];
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kk; i < n;
         i += (int64_t)gridDim.x * blockDim.x / kk) {
      const size_t o = (size_t)i * k + j;
      double ri = r[o];
      if (!frozen) {
        x[o] = fma(alpha, p[o], x[o]);
        ri = fma(-alpha, q[o], ri);
        r[o] = ri;
      }
      v = fma(ri, ri, v);
      const T yi = static_cast<T>(ri);
      if (write_y) y0[o] = yi;
      s0[o] = pre ? wd[i] * yi : T(0);
    }
  }
  // per-column block partials (column = thread % kk)
  __shared__ double red[TPB];
  __shared__ bool last;
  red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < kk) {
    double s = 0.0;
    for (int m = threadIdx.x; m < TPB; m += kk) s += red[m];
    partials[(blockIdx.x * 3) * KMAX + threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double tot[1][KMAX];
  grid_totals<1>(partials, gridDim.x, kk, tot);
  if (threadIdx.x < k) {
    const int c = threadIdx.x;
    const double s = tot[0][c];
    if (!sc->done[c] && !sc->first[c]) {
      const int it = sc->iters[c] + 1;
      sc->iters[c] = it;
      sc->rr[c] = s;
      const double res = sqrt(s);
      if (it < hist_cap) hist[(size_t)it * k + c] = res;
      if (res < sc->tol[c]) {
        sc->done[c] = 1;
      } else if (it >= sc->maxit) {
        sc->status[c] = AMG_ERR_NO_CONVERGENCE;
        sc->done[c] = 1;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *counter = 0u;
    int all = 1;
    for (int c = 0; c < k; ++c) all &= sc->done[c];
    sc->all_done = all;
    if (all && host_done) *(volatile int *)host_done = 1;
  }
}

// p = z + beta_j p (columns not done)
template <int K>
__global__ void __launch_bounds__(TPB) k_bdirection(int n, int k, bool vec, const double *__restrict__ z,
                                                    double *__restrict__ p, float2 *__restrict__ p2,
                                                    const BScal *sc) {
  if (sc->all_done) return;
  __shared__ double s_beta[KMAX];
  __shared__ int s_act[KMAX];
  if (threadIdx.x < KMAX) {
    const int c = threadIdx.x;
    s_act[c] = c < k && !sc->done[c];
    s_beta[c] = c < k ? sc->beta[c] : 0.0;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const size_t o = (size_t)i * k;
    double zr[K], pr[K];
    load_dr<K>(z + o, k, vec, zr);
    load_dr<K>(p + o, k, vec, pr);
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (s_act[j]) pr[j] = fma(s_beta[j], pr[j], zr[j]);
    store_dr<K>(p + o, k, vec, pr);
    if (p2) {
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j < k && s_act[j]) p2[o + j] = df_split(pr[j]);
    }
  }
}

// Wide batches (K > 8): an entry per thread.
__global__ void __launch_bounds__(TPB) k_bdirection_cols(int64_t total, int k, const double *__restrict__ z,
                                                         double *__restrict__ p, float2 *__restrict__ p2,
                                                         const BScal *sc) {
  if (sc->all_done) return;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(o % k);
    if (!sc->done[j]) {
      const double v = fma(sc->beta[j], p[o], z[o]);
      p[o] = v;
      if (p2) p2[o] = df_split(v);
    }
  }
}

// z = L^-T (L^-1 y) for the k columns of the last level (one block).
template <typename T>
__global__ void k_bcoarse(int n, int k, const double *__restrict__ Li, const T *__restrict__ y, T *__restrict__ z,
                          const int *__restrict__ done) {
  if (*done) return;
  extern __shared__ double sm[];
  double *yy = sm, *w = sm + (size_t)n * k;
  for (int o = threadIdx.x; o < n * k; o += blockDim.x) yy[o] = static_cast<double>(y[o]);
  __syncthreads();
  for (int o = threadIdx.x; o < n * k; o += blockDim.x) {
    const int i = o / k, j = o % k;
    double s = 0.0;
    for (int c = 0; c <= i; ++c) s = fma(Li[(size_t)i * n + c], yy[c * k + j], s);
    w[o] = s;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < n * k; o += blockDim.x) {
    const int i = o / k, j = o % k;
    double s = 0.0;
    for (int c = i; c < n; ++c) s = fma(Li[(size_t)c * n + i], w[c * k + j], s);
    z[o] = static_cast<T>(s);
  }
}

template <typename T>
__global__ void k_bcopy(int64_t total, const T *__restrict__ a, T *__restrict__ b) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x)
    b[o] = a[o];
}

inline int grid_for(int64_t work) { return std::max(1, std::min<int>(ceil_div(work, TPB), MAX_GRID)); }

// Batches of up to 16 columns run on a matrix's sliced-ELLPACK copy from 2^18
// rows up (the op's value pointer must then point into it: bv below); smaller
// matrices use the CSR row kernel with several lanes per row and column.
constexpr int kBSellRows = 1 << 18;
template <int K>
bool bsell(const DCsr &M) {
  return M.use_sell && K <= 16 && M.n >= kBSellRows;
}

// Entry lanes G per (row, column) of k_brows: about a quarter of the mean row
// length, at most 32 / K.
template <int K>
int brows_g(const DCsr &M) {
  const double avg = M.n ? (double)M.nnz / M.n : 0.0;
  int g = 1;
  while (g * 2 * K <= 32 && 4.0 * g * 2 <= avg) g <<= 1;
  return g;
}

template <typename V>
struct VSel;
template <>
struct VSel<double> {
  static const double *csr(const DCsr &M) { return M.v; }
  static const double *sell(const DCsr &M) { return M.sell.v; }
};
template <>
struct VSel<float> {
  static const float *csr(const DCsr &M) { return M.v32; }
  static const float *sell(const DCsr &M) { return M.sell.v32; }
};
template <>
struct VSel<__nv_bfloat16> {
  static const __nv_bfloat16 *csr(const DCsr &M) { return M.v16; }
  static const __nv_bfloat16 *sell(const DCsr &M) { return M.sell.v16; }
};

// Values of M in storage type V, laid out for the kernel launch_b<K> runs.
template <int K, typename V>
const V *bv(const DCsr &M) {
  return bsell<K>(M) ? VSel<V>::sell(M) : VSel<V>::csr(M);
}

template <int K, class Op>
void launch_b(int n, int k, const DCsr &M, const Op &op, cudaStream_t s) {
  bool done = false;
  if constexpr (K <= 16) {
    if (bsell<K>(M)) {
      const int grid = std::max(1, std::min(ceil_div(M.sell.nslices, TPB / 32), MAX_GRID));
      const bool vec = k == K && (reinterpret_cast<uintptr_t>(op.vbase()) & 15) == 0;
      k_bsell<K, Op><<<grid, TPB, 0, s>>>(n, k, vec, M.sell.nslices, M.sell.off, M.sell.col, M.sell.perm, op);
      done = true;
    }
  }
  if (!done) {
    const int g = brows_g<K>(M);
    const int grid = grid_for((int64_t)n * K * g);
    switch (g) {
      case 1: k_brows<K, 1, Op><<<grid, TPB, 0, s>>>(n, k, M.rp, M.ci, op); break;
      case 2: if constexpr (K * 2 <= 32) k_brows<K, 2, Op><<<grid, TPB, 0, s>>>(n, k, M.rp, M.ci, op); break;
      case 4: if constexpr (K * 4 <= 32) k_brows<K, 4, Op><<<grid, TPB, 0, s>>>(n, k, M.rp, M.ci, op); break;
      case 8: if constexpr (K * 8 <= 32) k_brows<K, 8, Op><<<grid, TPB, 0, s>>>(n, k, M.rp, M.ci, op); break;
      case 16: if constexpr (K * 16 <= 32) k_brows<K, 16, Op><<<grid, TPB, 0, s>>>(n, k, M.rp, M.ci, op); break;
      default: if constexpr (K * 32 <= 32) k_brows<K, 32, Op><<<grid, TPB, 0, s>>>(n, k, M.rp, M.ci, op); break;
    }
  }
  AMG_CHECK_LAUNCH();
}

template <int K, typename T>
void launch_bupdate(int n, int k, double *x, double *r, const double *p, const double *q, const T *wd, T *y0, T *s0,
                    bool write_y, bool pre, BScal *sc, double *hist, int hist_cap, int *host_done, double *partials,
                    unsigned int *counter, cudaStream_t s) {
  if constexpr (K <= 8) {
    auto al = [](const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15) == 0; };
    const bool vec = k == K && al(x) && al(r) && al(p) && al(q);
    k_bupdate<K, T><<<grid_for(n), TPB, 0, s>>>(n, k, vec, x, r, p, q, wd, y0, s0, write_y, pre, sc, hist, hist_cap,
                                                 host_done, partials, counter);
  } else {
    k_bupdate_cols<T><<<grid_for((int64_t)n * k), TPB, 0, s>>>(n, k, x, r, p, q, wd, y0, s0, write_y, pre, sc, hist,
                                                               hist_cap, host_done, partials, counter);
  }
  AMG_CHECK_LAUNCH();
}

template <int K>
void launch_bdirection(int n, int k, const double *z, double *p, float2 *p2, const BScal *sc, cudaStream_t s) {
  if constexpr (K <= 8) {
    auto al = [](const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15) == 0; };
    const bool vec = k == K && al(z) && al(p);
    k_bdirection<K><<<grid_for(n), TPB, 0, s>>>(n, k, vec, z, p, p2, sc);
  } else {
    const int64_t nk = (int64_t)n * k;
    k_bdirection_cols<<<grid_for(nk), TPB, 0, s>>>(nk, k, z, p, p2, sc);
  }
  AMG_CHECK_LAUNCH();
}

// --------------------------------------------------------------- driver --
template <typename T>
const T *wdv(const Level &l);
template <>
const double *wdv<double>(const Level &l) { return l.wd; }
template <>
const float *wdv<float>(const Level &l) { return l.wd32; }

// Work vectors of one batched solve (n_k x k per level, V-cycle precision).
template <typename T>
struct BWork {
  std::vector<Buf<T>> y, s, r, z, w;
};

template <int K, typename T, typename TP>
struct Batch {
  amg_hierarchy *h;
  cudaStream_t st;
  int k;
  BWork<T> *wk;
  BScal *sc;
  double *partials;
  unsigned int *counter;
  double *r, *zz, *p, *q;  // level-0 CG blocks (FP64)
  float2 *p2;               // p as FP32 pairs when the outer product runs in double-float, else nullptr

  void cycle(int lv, const int *done) {
    cudaStream_t s = st;
    Level &L = h->lev[lv];
    const DCsr &A = L.A;
    const int n = A.n;
    const double bt = sizeof(T), bp = sizeof(TP);
    const int64_t nk = (int64_t)n * k;
    if (lv == h->nlevels - 1) {
      ProfScope ps(s, AMG_K_COARSE, 8.0 * (double)n * n + 2.0 * bt * nk, lv);
      const int th = std::min(1024, std::max(32, (int)((nk + 31) / 32 * 32)));
      k_bcoarse<T><<<1, th, 2 * sizeof(double) * nk, s>>>(n, k, h->Linv, wk->y[lv].p, wk->z[lv].p, done);
      AMG_CHECK_LAUNCH();
      return;
    }
    const amg_params &prm = h->prm;
    T *y = wk->y[lv].p, *sv = wk->s[lv].p, *r = wk->r[lv].p, *w = wk->w[lv].p;
    const double abytes = (4.0 + bt) * (double)A.nnz + 4.0 * (n + 1);
    for (int it = 1; it < prm.nu1; ++it) {
      ProfScope ps(s, AMG_K_SOLVE_OTHER, abytes + 4.0 * bt * nk, lv);
      launch_b<K>(n, k, A, BJacobi<T>{k, bv<K, T>(A), wdv<T>(L), y, sv, w, done}, s);
      std::swap(sv, w);
    }
    {
      ProfScope ps(s, AMG_K_SMOOTH_RESID, abytes + 3.0 * bt * nk, lv);
      launch_b<K>(n, k, A, BResid<T>{k, bv<K, T>(A), sv, y, r, done}, s);
    }
    Level &C = h->lev[lv + 1];
    const int nc = C.A.n;
    const bool c_last = lv + 1 == h->nlevels - 1;
    {
      ProfScope ps(s, AMG_K_RESTRICT, (4.0 + bp) * (double)L.R.nnz + 4.0 * (nc + 1) + bt * nk + 3.0 * bt * nc * k, lv);
      launch_b<K>(nc, k, L.R,
                  BRestrict<T, TP>{k, bv<K, TP>(L.R), r, c_last ? nullptr : wdv<T>(C), wk->y[lv + 1].p,
                                   c_last ? nullptr : wk->s[lv + 1].p, c_last ? -1 : (prm.nu1 > 0 ? 1 : 0), done},
                  s);
    }
    cycle(lv + 1, done);
    {
      ProfScope ps(s, AMG_K_PROLONG, (4.0 + bp) * (double)L.P.nnz + 4.0 * (n + 1) + 2.0 * bt * nk + bt * nc * k, lv);
      launch_b<K>(n, k, L.P, BProlong<T, TP>{k, bv<K, TP>(L.P), sv, wk->z[lv + 1].p, r, done}, s);
    }
    if (lv == 0) return;
    T *t = r;
    if (prm.nu2 == 0) {
      k_bcopy<T><<<grid_for(nk), TPB, 0, s>>>(nk, t, wk->z[lv].p);
      AMG_CHECK_LAUNCH();
      return;
    }
    for (int it = 0; it < prm.nu2; ++it) {
      const bool lastp = it == prm.nu2 - 1;
      T *dst = lastp ? wk->z[lv].p : (t == r ? w : r);
      ProfScope ps(s, lastp ? AMG_K_SMOOTH_POST : AMG_K_SOLVE_OTHER, abytes + 4.0 * bt * nk, lv);
      launch_b<K>(n, k, A, BJacobi<T>{k, bv<K, T>(A), wdv<T>(L), y, t, dst, done}, s);
      t = dst;
    }
  }

  void vcycle(int mode, int flexible, const int *done) {
    cudaStream_t s = st;
    Level &L0 = h->lev[0];
    const DCsr &A = L0.A;
    const int n = A.n;
    const int64_t nk = (int64_t)n * k;
    const T *y = wk->y[0].p;
    const T *t;
    bool sweep = true;
    if (h->nlevels == 1) {
      cycle(0, done);
      t = wk->z[0].p;
      sweep = false;
    } else {
      cycle(0, done);
      T *tt = wk->r[0].p, *w = wk->w[0].p;
      for (int it = 0; it + 1 < h->prm.nu2; ++it) {
        launch_b<K>(n, k, A, BJacobi<T>{k, bv<K, T>(A), wdv<T>(L0), y, tt, w, done}, s);
        std::swap(tt, w);
      }
      t = tt;
      sweep = h->prm.nu2 > 0;
    }
    ProfScope ps(s, AMG_K_SMOOTH_POST, (sweep ? 12.0 * A.nnz : 0.0) + 40.0 * nk, 0);
    if (sweep)
      launch_b<K>(n, k, A, BPost0<K, T, true>{k, bv<K, T>(A), wdv<T>(L0), y, t, zz, r, q, p, p2, mode, flexible, sc,
                                                done, partials, counter}, s);
    else
      launch_b<K>(n, k, A, BPost0<K, T, false>{k, bv<K, T>(A), wdv<T>(L0), y, t, zz, r, q, p, p2, mode, flexible, sc,
                                                 done, partials, counter}, s);
  }
};

// The double-float outer product is used in the FP32 modes when level 0 has
// its sliced-ELLPACK copy and the batch is 8 or 16 wide (narrower batches are
// bound by memory, where FP64 costs nothing extra); its FP32 pairs of A are
// built on first use and kept with the hierarchy.
template <int K, typename T>
bool use_df(amg_hierarchy *h) {
  const DCsr &A = h->lev[0].A;
  // below 8 columns the FP64 product is not bound by FP64 arithmetic
  return std::is_same<T, float>::value && K >= 8 && bsell<K>(A) && A.sell.v != nullptr;
}

// Built once per hierarchy, under its mutex, on the hierarchy's own stream
// (where its allocator orders the memory); the caller's stream `s` then waits
// for the build's event, so every user reads a finished copy.
void ensure_df(amg_hierarchy *h, cudaStream_t s) {
  DCsr &A = h->lev[0].A;
  std::lock_guard<std::mutex> lock(h->df_mu);
  cudaStream_t hs = h->mem.stream;
  if (!A.sell.vdf) {
    if (!h->df_ev) AMG_CUDA(cudaEventCreateWithFlags(&h->df_ev, cudaEventDisableTiming));
    float2 *vdf = h->mem.get_n<float2>(std::max<int64_t>(A.sell.nent, 1));
    k_split_df<<<grid_for(A.sell.nent), TPB, 0, hs>>>(A.sell.nent, A.sell.v, vdf);
    AMG_CHECK_LAUNCH();
    AMG_CUDA(cudaEventRecord(h->df_ev, hs));
    A.sell.vdf = vdf;
  }
  if (s != hs) AMG_CUDA(cudaStreamWaitEvent(s, h->df_ev, 0));
}

// q = A p and the alpha bookkeeping: double-float when p2 is set, FP64 otherwise.
template <int K>
void launch_outer(int n, int k, const DCsr &A, const BSpmvDot<K> &op, const float2 *p2, cudaStream_t s) {
  if constexpr (K <= 16) {
    if (p2) {
      const int grid = std::max(1, std::min(ceil_div(A.sell.nslices, TPB / 32), MAX_GRID));
      const bool vec = k == K && (reinterpret_cast<uintptr_t>(p2) & 15) == 0;
      k_bsell_df<K><<<grid, TPB, 0, s>>>(n, k, vec, A.sell.nslices, A.sell.off, A.sell.col, A.sell.perm, A.sell.vdf,
                                         p2, op);
      AMG_CHECK_LAUNCH();
      return;
    }
  }
  launch_b<K>(n, k, A, op, s);
}

template <int K, typename T, typename TP>
int batch_impl(amg_hierarchy *h, int k, const double *B, double *X, double rtol, int maxit, int *iters, int *status,
               double *hist_out, int hist_cap) {
  Mem &m = h->mem;
  cudaStream_t s = m.stream;
  const Level &L0 = h->lev[0];
  const DCsr &A = L0.A;
  const int n = A.n;
  const int64_t nk = (int64_t)n * k;
  const bool fp64 = std::is_same<T, double>::value;
  BWork<T> wk;
  for (int lv = 0; lv < h->nlevels; ++lv) {
    const size_t cnt = (size_t)h->lev[lv].A.n * k;
    wk.y.emplace_back(m, cnt);
    wk.z.emplace_back(m, cnt);
    const bool work = lv < h->nlevels - 1 || lv == 0;
    wk.s.emplace_back(m, work ? cnt : 1);
    wk.r.emplace_back(m, work ? cnt : 1);
    wk.w.emplace_back(m, work ? cnt : 1);
  }
  Buf<double> r(m, nk), zz(m, nk), p(m, nk), q(m, nk);
  const bool df = use_df<K, T>(h);
  Buf<float2> p2;
  if (df) {
    ensure_df(h, s);
    p2 = Buf<float2>(m, nk);
  }
  Buf<BScal> scb(m, 1);
  Buf<double> partials(m, (size_t)MAX_GRID * 3 * KMAX);
  Buf<unsigned int> counter(m, 1);
  Buf<double> hist(m, (size_t)(maxit + 1) * k);
  AMG_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned int), s));
  BScal init{};
  init.maxit = maxit;
  init.k = k;
  AMG_CUDA(cudaMemcpyAsync(scb.p, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  *h->h_done = 0;
  const int *done = &scb.p->all_done;
  // FP64: the V-cycle input y0 is the CG residual block itself
  T *y0 = fp64 ? reinterpret_cast<T *>(r.p) : wk.y[0].p;
  if (fp64) {
    wk.y[0].reset();
    wk.y[0].p = y0;  // alias, not owned
    wk.y[0].m = nullptr;
  }
  T *s0 = wk.s[0].p;
  const bool pre = h->prm.nu1 > 0;
  Batch<K, T, TP> bt{h, s, k, &wk, scb.p, partials.p, counter.p, r.p, zz.p, p.p, q.p, p2.p};
  {
    ProfScope ps(s, AMG_K_SOLVE_OTHER, 12.0 * A.nnz + 40.0 * nk, 0);
    launch_b<K>(n, k, A, BInit<K, T>{k, bv<K, double>(A), X, B, r.p, wdv<T>(L0), y0, s0, !fp64, pre, rtol, scb.p, hist.p, maxit + 1,
                                     partials.p, counter.p}, s);
  }
  const int flexible = fp64 ? 0 : 1;
  bt.vcycle(BPOST_FIRST, flexible, done);
  for (int it = 1; it <= maxit; ++it) {
    {
      ProfScope ps(s, AMG_K_SPMV_DOT, 12.0 * A.nnz + 4.0 * (n + 1) + 24.0 * nk, 0);
      launch_outer<K>(n, k, A, BSpmvDot<K>{k, bv<K, double>(A), p.p, q.p, scb.p, partials.p, counter.p}, p2.p, s);
    }
    {
      ProfScope ps(s, AMG_K_PCG_UPDATE, (48.0 + 3.0 * sizeof(T)) * nk, 0);
      launch_bupdate<K, T>(n, k, X, r.p, p.p, q.p, wdv<T>(L0), y0, s0, !fp64, pre, scb.p, hist.p, maxit + 1,
                           h->d_done, partials.p, counter.p, s);
    }
    bt.vcycle(BPOST_ITER, flexible, done);
    {
      ProfScope ps(s, AMG_K_DIRECTION, 24.0 * nk, 0);
      launch_bdirection<K>(n, k, zz.p, p.p, p2.p, scb.p, s);
    }
    AMG_CUDA(cudaEventRecord(h->iter_ev[it & 1], s));
    if (it > 1) {
      AMG_CUDA(cudaEventSynchronize(h->iter_ev[(it - 1) & 1]));
      if (*(volatile int *)h->h_done) break;
    }
  }
  BScal out{};
  AMG_CUDA(cudaMemcpyAsync(&out, scb.p, sizeof(out), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  prof_collect(s);
  int worst = AMG_OK;
  for (int j = 0; j < k; ++j) {
    if (iters) iters[j] = out.iters[j];
    if (status) status[j] = out.status[j];
    if (out.status[j] != AMG_OK && worst == AMG_OK) worst = out.status[j];
    if (!out.done[j] && worst == AMG_OK) worst = AMG_ERR_NO_CONVERGENCE;
  }
  if (hist_out && hist_cap > 0) {
    const int rows = std::min(hist_cap, maxit + 1);
    AMG_CUDA(cudaMemcpy(hist_out, hist.p, sizeof(double) * (size_t)rows * k, cudaMemcpyDeviceToHost));
  }
  return worst;
}

template <typename T, typename TP>
int batch_dispatch(amg_hierarchy *h, int k, const double *B, double *X, double rtol, int maxit, int *iters,
                   int *status, double *hist, int hist_cap) {
  if (k <= 1) return batch_impl<1, T, TP>(h, k, B, X, rtol, maxit, iters, status, hist, hist_cap);
  if (k <= 2) return batch_impl<2, T, TP>(h, k, B, X, rtol, maxit, iters, status, hist, hist_cap);
  if (k <= 4) return batch_impl<4, T, TP>(h, k, B, X, rtol, maxit, iters, status, hist, hist_cap);
  if (k <= 8) return batch_impl<8, T, TP>(h, k, B, X, rtol, maxit, iters, status, hist, hist_cap);
  if (k <= 16) return batch_impl<16, T, TP>(h, k, B, X, rtol, maxit, iters, status, hist, hist_cap);
  return batch_impl<32, T, TP>(h, k, B, X, rtol, maxit, iters, status, hist, hist_cap);
}


// ------------------------------------------------------------------ slots --
// Continuous batching: a resident n x K block on one hierarchy whose columns
// ("slots") are admitted, stepped and retired independently.

// Column j of an n x K block: x = 0, r = b, p = 0; tol_j = rtol ||b||.
__global__ void __launch_bounds__(TPB) k_admit(int n, int K, int j, unsigned int ticket, const double *__restrict__ b,
                                               double *__restrict__ x, double *__restrict__ r, double *__restrict__ p,
                                               float2 *__restrict__ p2, double rtol, BScal *sc, double *partials,
                                               unsigned int *counter) {
  __shared__ double red[TPB / 32];
  __shared__ bool last;
  double v = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    const size_t o = (size_t)i * K + j;
    x[o] = 0.0;
    r[o] = bi;
    p[o] = 0.0;
    if (p2) p2[o] = make_float2(0.f, 0.f);
    v = fma(bi, bi, v);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < TPB / 32; ++w) t += red[w];
    partials[blockIdx.x * 3 * KMAX] = t;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double tot[1][KMAX];
  grid_totals<1>(partials, gridDim.x, 1, tot);
  if (threadIdx.x != 0) return;
  const double bb = tot[0][0];
  sc->bb[j] = bb;
  sc->ticket[j] = ticket;
  sc->tol[j] = rtol * sqrt(bb);
  sc->iters[j] = 0;
  sc->status[j] = AMG_OK;
  sc->done[j] = bb == 0.0 ? 1 : 0;
  sc->first[j] = bb == 0.0 ? 0 : 1;
  sc->alpha[j] = sc->beta[j] = 0.0;
  sc->rho[j] = 1.0;
  int all = 1;
  for (int c = 0; c < sc->k; ++c) all &= sc->done[c];
  sc->all_done = all;
  *counter = 0u;
}

// Frees slot j (frozen, counted as done).
__global__ void k_release(int j, BScal *sc) {
  sc->done[j] = 1;
  sc->first[j] = 0;
  int all = 1;
  for (int c = 0; c < sc->k; ++c) all &= sc->done[c];
  sc->all_done = all;
}

__global__ void k_take_column(int n, int K, int j, const double *__restrict__ X, double *__restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = X[(size_t)i * K + j];
}

template <int KP, typename T, typename TP>
struct SlotsImpl : SlotsBase {
  amg_hierarchy *h;
  Mem mem;
  int K, maxit;
  double rtol;
  BWork<T> wk;
  Buf<double> X, r, zz, p, q, partials;
  Buf<float2> p2;  // p as FP32 pairs (double-float outer product), when used
  Buf<BScal> scb;
  Buf<unsigned int> counter;
  BScal *host = nullptr;  // pinned copy for poll
  std::vector<int> busy;
  std::vector<unsigned int> ticket;  // admission number of each slot's current request
  unsigned int admitted = 0;
  cudaGraphExec_t exec = nullptr;
  long long per_step = 0;  // kernels in one step
  // snapshots of the per-column state taken at the end of each step (pinned ring)
  static constexpr int kRing = 8;
  BScal *ring = nullptr;
  cudaEvent_t ring_ev[kRing] = {};
  long long issued = 0, completed = 0;

  SlotsImpl(amg_hierarchy *hh, int cap, double rt, int mi, cudaStream_t s) : h(hh), K(cap), maxit(mi), rtol(rt) {
    mem.alloc = h->mem.alloc;
    mem.callbacks = h->mem.callbacks;
    mem.stream = s;
    const int n = h->lev[0].A.n;
    const size_t nk = (size_t)n * K;
    for (int lv = 0; lv < h->nlevels; ++lv) {
      const size_t cnt = (size_t)h->lev[lv].A.n * K;
      const bool work = lv < h->nlevels - 1 || lv == 0;
      wk.y.emplace_back(mem, (lv == 0 && std::is_same<T, double>::value) ? 1 : cnt);
      wk.z.emplace_back(mem, cnt);
      wk.s.emplace_back(mem, work ? cnt : 1);
      wk.r.emplace_back(mem, work ? cnt : 1);
      wk.w.emplace_back(mem, work ? cnt : 1);
    }
    X = Buf<double>(mem, nk);
    r = Buf<double>(mem, nk);
    zz = Buf<double>(mem, nk);
    p = Buf<double>(mem, nk);
    q = Buf<double>(mem, nk);
    partials = Buf<double>(mem, (size_t)MAX_GRID * 3 * KMAX);
    scb = Buf<BScal>(mem, 1);
    counter = Buf<unsigned int>(mem, 1);
    if (use_df<KP, T>(h)) {
      ensure_df(h, s);
      p2 = Buf<float2>(mem, nk);
      AMG_CUDA(cudaMemsetAsync(p2.p, 0, sizeof(float2) * nk, s));
    }
    if (std::is_same<T, double>::value) {  // FP64: the V-cycle input is the CG residual block
      wk.y[0].reset();
      wk.y[0].p = reinterpret_cast<T *>(r.p);
      wk.y[0].m = nullptr;
    }
    AMG_CUDA(cudaMemsetAsync(X.p, 0, sizeof(double) * nk, s));
    AMG_CUDA(cudaMemsetAsync(p.p, 0, sizeof(double) * nk, s));
    AMG_CUDA(cudaMemsetAsync(r.p, 0, sizeof(double) * nk, s));
    AMG_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned int), s));
    BScal init{};
    init.maxit = maxit;
    init.k = K;
    for (int j = 0; j < K; ++j) init.done[j] = 1;
    init.all_done = 1;
    AMG_CUDA(cudaMemcpyAsync(scb.p, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    AMG_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&host), sizeof(BScal), cudaHostAllocDefault));
    AMG_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&ring), sizeof(BScal) * kRing, cudaHostAllocDefault));
    for (int e = 0; e < kRing; ++e) AMG_CUDA(cudaEventCreateWithFlags(&ring_ev[e], cudaEventDisableTiming));
    AMG_CUDA(cudaStreamSynchronize(s));
    busy.assign(K, 0);
    ticket.assign(K, 0);
  }
  ~SlotsImpl() override {
    cudaStreamSynchronize(mem.stream);
    if (exec) cudaGraphExecDestroy(exec);
    if (host) cudaFreeHost(host);
    if (ring) cudaFreeHost(ring);
    for (int e = 0; e < kRing; ++e)
      if (ring_ev[e]) cudaEventDestroy(ring_ev[e]);
    // Bufs return their memory through mem; free_all catches anything left
  }
  void admit(int j, const double *b) override {
    const int n = h->lev[0].A.n;
    ticket[j] = ++admitted;
    k_admit<<<grid_for(n), TPB, 0, mem.stream>>>(n, K, j, ticket[j], b, X.p, r.p, p.p, p2.p, rtol, scb.p,
                                                 partials.p, counter.p);
    AMG_CHECK_LAUNCH();
    busy[j] = 1;
  }
  // One PCG iteration of every running column.  Without profiling the
  // launches are captured once into a CUDA graph and replayed (the launch
  // sequence never changes: masks live in device memory).
  void step() override {
    if (issued - completed >= kRing) {  // every snapshot slot is in flight: wait for the oldest
      AMG_CUDA(cudaEventSynchronize(ring_ev[completed % kRing]));
      ++completed;
    }
    run_step();
    const int e = (int)(issued % kRing);
    AMG_CUDA(cudaMemcpyAsync(ring + e, scb.p, sizeof(BScal), cudaMemcpyDeviceToHost, mem.stream));
    AMG_CUDA(cudaEventRecord(ring_ev[e], mem.stream));
    ++issued;
  }
  // Per-slot states from the newest finished step, without waiting.
  void query(int *state, int *iters, long long *done_steps, long long *issued_steps) override {
    while (completed < issued && cudaEventQuery(ring_ev[completed % kRing]) == cudaSuccess) ++completed;
    const BScal *snap = completed > 0 ? ring + (completed - 1) % kRing : nullptr;
    report(snap, state, iters);
    if (done_steps) *done_steps = completed;
    if (issued_steps) *issued_steps = issued;
  }
  void wait() override {
    if (completed < issued) {
      AMG_CUDA(cudaEventSynchronize(ring_ev[completed % kRing]));
      ++completed;
    }
  }
  // A slot whose request was admitted after the snapshot was taken reads as running.
  void report(const BScal *snap, int *state, int *iters) {
    for (int j = 0; j < K; ++j) {
      int stt = 0, it = 0;
      if (busy[j]) {
        if (snap && snap->ticket[j] == ticket[j]) {
          stt = !snap->done[j] ? 1 : (snap->status[j] == AMG_OK ? 2 : snap->status[j]);
          it = snap->iters[j];
        } else {
          stt = 1;
        }
      }
      if (state) state[j] = stt;
      if (iters) iters[j] = it;
    }
  }
  void run_step() {
    if (prof_records_solve() || mem.stream == nullptr) {  // the legacy default stream cannot be captured
      issue_step();
      return;
    }
    if (!exec) {
      cudaGraph_t g = nullptr;
      const long long before = g_launches.load();
      AMG_CUDA(cudaStreamBeginCapture(mem.stream, cudaStreamCaptureModeThreadLocal));
      try {
        issue_step();
      } catch (...) {
        cudaStreamEndCapture(mem.stream, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      AMG_CUDA(cudaStreamEndCapture(mem.stream, &g));
      per_step = g_launches.load() - before;
      const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      AMG_CUDA(e);
      g_launches.fetch_sub(per_step);
    }
    AMG_CUDA(cudaGraphLaunch(exec, mem.stream));
    g_launches.fetch_add(per_step);
  }
  void issue_step() {
    cudaStream_t s = mem.stream;
    const Level &L0 = h->lev[0];
    const DCsr &A = L0.A;
    const int n = A.n;
    const int64_t nk = (int64_t)n * K;
    const bool fp64 = std::is_same<T, double>::value;
    const int *done = &scb.p->all_done;
    T *y0 = fp64 ? reinterpret_cast<T *>(r.p) : wk.y[0].p;
    Batch<KP, T, TP> bt{h, s, K, &wk, scb.p, partials.p, counter.p, r.p, zz.p, p.p, q.p, p2.p};
    {
      ProfScope ps(s, AMG_K_SPMV_DOT, 12.0 * A.nnz + 4.0 * (n + 1) + 24.0 * nk, 0);
      launch_outer<KP>(n, K, A, BSpmvDot<KP>{K, bv<KP, double>(A), p.p, q.p, scb.p, partials.p, counter.p}, p2.p,
                       s);
    }
    {
      ProfScope ps(s, AMG_K_PCG_UPDATE, (48.0 + 3.0 * sizeof(T)) * nk, 0);
      launch_bupdate<KP, T>(n, K, X.p, r.p, p.p, q.p, wdv<T>(L0), y0, wk.s[0].p, !fp64, h->prm.nu1 > 0, scb.p,
                            nullptr, 0, nullptr, partials.p, counter.p, s);
    }
    bt.vcycle(BPOST_ITER, fp64 ? 0 : 1, done);
    {
      ProfScope ps(s, AMG_K_DIRECTION, 24.0 * nk, 0);
      launch_bdirection<KP>(n, K, zz.p, p.p, p2.p, scb.p, s);
    }
  }
  void poll(int *state, int *iters) override {
    AMG_CUDA(cudaMemcpyAsync(host, scb.p, sizeof(BScal), cudaMemcpyDeviceToHost, mem.stream));
    AMG_CUDA(cudaStreamSynchronize(mem.stream));
    prof_collect(mem.stream);  // event-timed launches of the steps (profiling on)
    completed = issued;
    report(host, state, iters);
  }
  void retire(int j, double *x) override {
    const int n = h->lev[0].A.n;
    if (x) {
      k_take_column<<<grid_for(n), TPB, 0, mem.stream>>>(n, K, j, X.p, x);
      AMG_CHECK_LAUNCH();
    }
    k_release<<<1, 1, 0, mem.stream>>>(j, scb.p);
    AMG_CHECK_LAUNCH();
    busy[j] = 0;
  }
};

template <typename T, typename TP>
SlotsBase *make_slots_t(amg_hierarchy *h, int K, double rtol, int maxit, cudaStream_t s) {
  if (K <= 1) return new SlotsImpl<1, T, TP>(h, K, rtol, maxit, s);
  if (K <= 2) return new SlotsImpl<2, T, TP>(h, K, rtol, maxit, s);
  if (K <= 4) return new SlotsImpl<4, T, TP>(h, K, rtol, maxit, s);
  if (K <= 8) return new SlotsImpl<8, T, TP>(h, K, rtol, maxit, s);
  if (K <= 16) return new SlotsImpl<16, T, TP>(h, K, rtol, maxit, s);
  return new SlotsImpl<32, T, TP>(h, K, rtol, maxit, s);
}

}  // namespace

int pcg_solve_batch(amg_hierarchy *h, int k, const double *B, double *X, double rtol, int maxit, int *iters,
                    int *status, double *hist, int hist_cap) {
  if (h->prm.smoother != AMG_SMOOTH_JACOBI) {
    set_error("multi-RHS solves support the Jacobi smoother only");
    throw Status{AMG_ERR_UNSUPPORTED};
  }
  if (h->nlevels > 0) {
    const int nL = h->nL;
    if ((size_t)2 * sizeof(double) * nL * k > 200 * 1024) {
      set_error("last level of %d rows too large for a %d-column batch", nL, k);
      throw Status{AMG_ERR_UNSUPPORTED};
    }
    static std::atomic<unsigned long long> attr_d{0}, attr_f{0};
    ensure_smem_attr(k_bcoarse<double>, 200 * 1024, attr_d);
    ensure_smem_attr(k_bcoarse<float>, 200 * 1024, attr_f);
  }
  switch (h->prm.precision) {
    case AMG_PREC_FP64: return batch_dispatch<double, double>(h, k, B, X, rtol, maxit, iters, status, hist, hist_cap);
    case AMG_PREC_FP32: return batch_dispatch<float, float>(h, k, B, X, rtol, maxit, iters, status, hist, hist_cap);
    default: return batch_dispatch<float, __nv_bfloat16>(h, k, B, X, rtol, maxit, iters, status, hist, hist_cap);
  }
}

}  // namespace amg

namespace amg {

SlotsBase *make_slots(amg_hierarchy *h, int K, double rtol, int maxit, cudaStream_t s) {
  if (h->prm.smoother != AMG_SMOOTH_JACOBI) {
    set_error("continuous batching supports the Jacobi smoother only");
    throw Status{AMG_ERR_UNSUPPORTED};
  }
  if ((size_t)2 * sizeof(double) * h->nL * K > 200 * 1024) {
    set_error("last level of %d rows too large for %d slots", h->nL, K);
    throw Status{AMG_ERR_UNSUPPORTED};
  }
  static std::atomic<unsigned long long> attr_d{0}, attr_f{0};
  ensure_smem_attr(k_bcoarse<double>, 200 * 1024, attr_d);
  ensure_smem_attr(k_bcoarse<float>, 200 * 1024, attr_f);
  switch (h->prm.precision) {
    case AMG_PREC_FP64: return make_slots_t<double, double>(h, K, rtol, maxit, s);
    case AMG_PREC_FP32: return make_slots_t<float, float>(h, K, rtol, maxit, s);
    default: return make_slots_t<float, __nv_bfloat16>(h, K, rtol, maxit, s);
  }
}

void slots_admit(SlotsBase *b, int j, const double *rhs) { b->admit(j, rhs); }
void slots_step(SlotsBase *b) { b->step(); }
void slots_poll(SlotsBase *b, int *state, int *iters) { b->poll(state, iters); }
void slots_query(SlotsBase *b, int *state, int *iters, long long *done, long long *issued) {
  b->query(state, iters, done, issued);
}
void slots_wait(SlotsBase *b) { b->wait(); }
void slots_retire(SlotsBase *b, int j, double *x) { b->retire(j, x); }
void slots_delete(SlotsBase *b) { delete b; }

}  // namespace amg

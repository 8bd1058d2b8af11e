// solve.cu -- the solve phase: PCG (Sec. 3.1 solver, stopping rule of Sec. 4)
// preconditioned by one V-cycle (Algorithm 2) per iteration.
//
// V-cycle on level k < L with damped Jacobi (S = I - omega D^-1 A, Eq.
// smoother) and zero initial guess; wd_k = omega / diag(A_k):
//   s_k = wd_k .* y_k                 written by whichever kernel produced y_k
//   r_k = y_k - A_k s_k               k_smooth_resid
//   y_{k+1} = R_k r_k, s_{k+1}        k_restrict
//   z_{k+1} = V-cycle(y_{k+1})        recursion; z_L = L^-T L^-1 y_L (k_coarse_solve)
//   t_k = s_k + P_k z_{k+1}           k_prolong  (prolongation + correction)
//   z_k = t_k + wd_k .* (y_k - A_k t_k)   k_smooth_post (level 0: fused with the CG dots)
// nu1 > 1 or nu2 > 1 adds plain Jacobi sweeps (k_jacobi); nu = 0 drops them.
//
// Every kernel is HBM-bound sparse or vector work: thread-per-row CSR with
// one FMA per nonzero (FP64 throughput on this part is ~1.2 TFLOP/s, so the
// FP64 kernels spend exactly one DFMA per stored entry), grid-stride loops
// over a grid sized in multiples of the SM count, and dot products reduced
// per block with warp shuffles and finished by the last block to arrive
// (one grid-level reduction, deterministic order).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr int TPB = 256;
constexpr int MAX_GRID = kNumSMs * 8;

template <typename T>
__device__ __forceinline__ T ld(const T *p) {
  return __ldg(p);
}
__device__ __forceinline__ float tof(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float tof(float v) { return v; }
__device__ __forceinline__ double tof(double v) { return v; }

template <typename TP, typename T>
__device__ __forceinline__ T cvt(TP v) {
  return static_cast<T>(tof(v));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduces up to three partial sums, writes them to partials[3*block+c]
// and returns true in every thread of the last block to finish, whose
// out[c] then holds the grid totals (summed in block order).
template <int NV>
__device__ bool grid_reduce(double (&v)[NV], double *partials, unsigned int *counter, double (&out)[NV]) {
  __shared__ double red[NV][TPB / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    double s = warp_sum(v[c]);
    if (lane == 0) red[c][w] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double s = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[c][k];
      partials[3 * blockIdx.x + c] = s;
    }
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
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
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    double s = warp_sum(acc[c]);
    __syncthreads();
    if (lane == 0) red[c][w] = s;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[c][k];
    out[c] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

#define GRID_STRIDE(i, n) for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)

// r = b - A x;  (b, b), (r, r);  V-cycle input y0 / s0.  Sets the tolerance and
// marks the solve done when ||r_0|| < rtol ||b|| (or b = 0).
template <typename T>
__global__ void __launch_bounds__(TPB) k_init(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                              const double *__restrict__ a, const double *__restrict__ b,
                                              const double *__restrict__ x, double *__restrict__ r,
                                              const T *__restrict__ wd, T *__restrict__ y0, T *__restrict__ s0,
                                              bool write_y, bool pre, double rtol, PcgScalars *sc, double *hist,
                                              double *partials, unsigned int *counter) {
  double v[2] = {0.0, 0.0};
  GRID_STRIDE(i, n) {
    double acc = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) acc = fma(ld(a + p), ld(x + ci[p]), acc);
    const double bi = b[i], ri = bi - acc;
    r[i] = ri;
    v[0] = fma(bi, bi, v[0]);
    v[1] = fma(ri, ri, v[1]);
    const T yi = static_cast<T>(ri);
    if (write_y) y0[i] = yi;
    s0[i] = pre ? wd[i] * yi : T(0);
  }
  double tot[2];
  if (grid_reduce<2>(v, partials, counter, tot) && threadIdx.x == 0) {
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

// q = A p;  alpha = rho / (p, q);  breakdown when (p, q) <= 0 or NaN.
__global__ void __launch_bounds__(TPB) k_spmv_dot(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                  const double *__restrict__ a, const double *__restrict__ p,
                                                  double *__restrict__ q, PcgScalars *sc, double *partials,
                                                  unsigned int *counter) {
  if (sc->done) return;
  double v[1] = {0.0};
  GRID_STRIDE(i, n) {
    double acc = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) acc = fma(ld(a + k), ld(p + ci[k]), acc);
    q[i] = acc;
    v[0] = fma(p[i], acc, v[0]);
  }
  double tot[1];
  if (grid_reduce<1>(v, partials, counter, tot) && threadIdx.x == 0) {
    sc->pq = tot[0];
    if (!(tot[0] > 0.0)) {
      sc->status = AMG_ERR_BREAKDOWN;
      sc->done = 1;
    } else {
      sc->alpha = sc->rho / tot[0];
    }
  }
}

// x += alpha p;  r -= alpha q;  ||r||;  convergence test;  V-cycle input.
template <typename T>
__global__ void __launch_bounds__(TPB) k_pcg_update(int n, double *__restrict__ x, double *__restrict__ r,
                                                    const double *__restrict__ p, const double *__restrict__ q,
                                                    const T *__restrict__ wd, T *__restrict__ y0,
                                                    T *__restrict__ s0, bool write_y, bool pre, PcgScalars *sc,
                                                    double *hist, int hist_cap, int *host_done,
                                                    double *partials, unsigned int *counter) {
  if (sc->done) return;
  const double alpha = sc->alpha;
  double v[1] = {0.0};
  GRID_STRIDE(i, n) {
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

// r = y - A s
template <typename T>
__global__ void __launch_bounds__(TPB) k_smooth_resid(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                      const T *__restrict__ a, const T *__restrict__ y,
                                                      const T *__restrict__ s, T *__restrict__ r,
                                                      const int *__restrict__ done) {
  if (*done) return;
  GRID_STRIDE(i, n) {
    T acc = y[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p) acc = fma(-ld(a + p), ld(s + ci[p]), acc);
    r[i] = acc;
  }
}

// y_c = R r;  s_c = wd_c .* y_c (or 0)
template <typename T, typename TP>
__global__ void __launch_bounds__(TPB) k_restrict(int nc, const int *__restrict__ rp, const int *__restrict__ ci,
                                                  const TP *__restrict__ rv, const T *__restrict__ r,
                                                  T *__restrict__ yc, const T *__restrict__ wdc, T *__restrict__ sc_,
                                                  int pre, const int *__restrict__ done) {
  if (*done) return;
  GRID_STRIDE(I, nc) {
    T acc = T(0);
    for (int p = rp[I]; p < rp[I + 1]; ++p) acc = fma(cvt<TP, T>(rv[p]), ld(r + ci[p]), acc);
    yc[I] = acc;
    if (pre >= 0) sc_[I] = pre ? wdc[I] * acc : T(0);
  }
}

// t = s + P z_c
template <typename T, typename TP>
__global__ void __launch_bounds__(TPB) k_prolong(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                 const TP *__restrict__ pv, const T *__restrict__ s,
                                                 const T *__restrict__ zc, T *__restrict__ t,
                                                 const int *__restrict__ done) {
  if (*done) return;
  GRID_STRIDE(i, n) {
    T acc = s[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p) acc = fma(cvt<TP, T>(pv[p]), ld(zc + ci[p]), acc);
    t[i] = acc;
  }
}

// z = t + wd .* (y - A t)   (one damped Jacobi step from t)
template <typename T>
__global__ void __launch_bounds__(TPB) k_jacobi(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                const T *__restrict__ a, const T *__restrict__ wd,
                                                const T *__restrict__ y, const T *__restrict__ t,
                                                T *__restrict__ z, const int *__restrict__ done) {
  if (*done) return;
  GRID_STRIDE(i, n) {
    T acc = y[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p) acc = fma(-ld(a + p), ld(t + ci[p]), acc);
    z[i] = fma(wd[i], acc, t[i]);
  }
}

enum Post0Mode { POST_APPLY = 0, POST_FIRST = 1, POST_ITER = 2 };

// Level-0 post-smoothing fused with the CG bookkeeping:
//   z = t + wd .* (y - A t)  (SWEEP) or z = t, written in FP64;
//   APPLY: nothing else; FIRST: rho = (r, z), p = z;
//   ITER:  beta = (z, r) / rho (standard) or -alpha (z, q) / rho (flexible:
//          (z_{k+1}, r_{k+1} - r_k) with r_{k+1} - r_k = -alpha q_k), rho = (r, z).
template <typename T, bool SWEEP>
__global__ void __launch_bounds__(TPB) k_post0(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                               const T *__restrict__ a, const T *__restrict__ wd,
                                               const T *__restrict__ y, const T *__restrict__ t,
                                               double *__restrict__ z, const double *__restrict__ r,
                                               const double *__restrict__ q, double *__restrict__ p, int mode,
                                               int flexible, PcgScalars *sc, const int *__restrict__ done,
                                               double *partials, unsigned int *counter) {
  if (*done) return;
  double v[2] = {0.0, 0.0};
  GRID_STRIDE(i, n) {
    T zi = t[i];
    if (SWEEP) {
      T acc = y[i];
      for (int k = rp[i]; k < rp[i + 1]; ++k) acc = fma(-ld(a + k), ld(t + ci[k]), acc);
      zi = fma(wd[i], acc, zi);
    }
    const double zd = static_cast<double>(zi);
    z[i] = zd;
    if (mode != POST_APPLY) {
      v[0] = fma(r[i], zd, v[0]);
      if (mode == POST_FIRST) p[i] = zd;
      else if (flexible) v[1] = fma(zd, q[i], v[1]);
    }
  }
  if (mode == POST_APPLY) return;
  double tot[2];
  if (grid_reduce<2>(v, partials, counter, tot) && threadIdx.x == 0) {
    sc->rz = tot[0];
    sc->zq = tot[1];
    if (mode == POST_ITER) sc->beta = flexible ? -sc->alpha * tot[1] / sc->rho : tot[0] / sc->rho;
    sc->rho = tot[0];
  }
}

// p = z + beta p
__global__ void __launch_bounds__(TPB) k_direction(int n, const double *__restrict__ z, double *__restrict__ p,
                                                   const PcgScalars *sc) {
  if (sc->done) return;
  const double beta = sc->beta;
  GRID_STRIDE(i, n) p[i] = fma(beta, p[i], z[i]);
}

// z = L^-T L^-1 y on the last level (dense Cholesky factor, one block).
template <typename T>
__global__ void k_coarse_solve(int n, const double *__restrict__ L, const T *__restrict__ y, T *__restrict__ z,
                               const int *__restrict__ done) {
  if (*done) return;
  extern __shared__ double w[];
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = static_cast<double>(y[i]);
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) w[j] = w[j] / L[(size_t)j * n + j];
    __syncthreads();
    const double wj = w[j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) w[i] = fma(-L[(size_t)i * n + j], wj, w[i]);
    __syncthreads();
  }
  for (int j = n - 1; j >= 0; --j) {
    if (threadIdx.x == 0) w[j] = w[j] / L[(size_t)j * n + j];
    __syncthreads();
    const double wj = w[j];
    for (int i = threadIdx.x; i < j; i += blockDim.x) w[i] = fma(-L[(size_t)j * n + i], wj, w[i]);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] = static_cast<T>(w[i]);
}

// y = A x (FP64), for amg_spmv
__global__ void __launch_bounds__(TPB) k_spmv64(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                const double *__restrict__ a, const double *__restrict__ x,
                                                double *__restrict__ y) {
  GRID_STRIDE(i, n) {
    double acc = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) acc = fma(ld(a + p), ld(x + ci[p]), acc);
    y[i] = acc;
  }
}

// V-cycle input from an FP64 vector: y = (T) src, s = wd .* y or 0
template <typename T>
__global__ void k_load_y0(int n, const double *__restrict__ src, const T *__restrict__ wd, T *__restrict__ y,
                          T *__restrict__ s, bool write_y, bool pre) {
  GRID_STRIDE(i, n) {
    const T yi = static_cast<T>(src[i]);
    if (write_y) y[i] = yi;
    s[i] = pre ? wd[i] * yi : T(0);
  }
}

template <typename T>
__global__ void k_copy(int n, const T *__restrict__ a, T *__restrict__ b) {
  GRID_STRIDE(i, n) b[i] = a[i];
}

// wd = omega / a_ii
__global__ void k_make_wd(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                          const double *__restrict__ a, double omega, double *__restrict__ wd,
                          float *__restrict__ wd32) {
  GRID_STRIDE(i, n) {
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

inline int grid_for(int64_t n) { return std::max(1, std::min<int>(ceil_div(n, TPB), MAX_GRID)); }

// ---------------------------------------------------------------- V-cycle --
template <typename T>
struct VTypes;
template <>
struct VTypes<double> {
  static const double *A(const DCsr &m) { return m.v; }
  static const double *wd(const Level &l) { return l.wd; }
};
template <>
struct VTypes<float> {
  static const float *A(const DCsr &m) { return m.v32; }
  static const float *wd(const Level &l) { return l.wd32; }
};

template <typename T>
inline T *vec(void *p) {
  return static_cast<T *>(p);
}

struct CycleCtx {
  const int *done;   // device flag: when set, every kernel returns at once
  int mode;          // Post0Mode
  int flexible;
};

template <typename T, typename TP>
const TP *pr_vals(const DCsr &m);
template <>
const double *pr_vals<double, double>(const DCsr &m) { return m.v; }
template <>
const float *pr_vals<float, float>(const DCsr &m) { return m.v32; }
template <>
const __nv_bfloat16 *pr_vals<float, __nv_bfloat16>(const DCsr &m) { return m.v16; }

constexpr double idx_bytes = 4.0;

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
    ProfScope ps(h->mem.stream, AMG_K_COARSE, 8.0 * (double)n * n + 2.0 * bt * n);
    const int th = std::min(1024, std::max(32, (n + 31) / 32 * 32));
    k_coarse_solve<T><<<1, th, sizeof(double) * n, s>>>(n, h->L, vec<T>(L.y), vec<T>(L.z), cc.done);
    AMG_CHECK_LAUNCH();
    return;
  }
  const amg_params &prm = h->prm;
  const T *a = VTypes<T>::A(A);
  const T *wd = VTypes<T>::wd(L);
  T *y = vec<T>(L.y), *sv = vec<T>(L.s), *r = vec<T>(L.r), *w = vec<T>(L.w);
  const double abytes = (idx_bytes + bt) * (double)A.nnz + 4.0 * (n + 1);
  // extra pre-smoothing sweeps (nu1 > 1): s <- s + wd (y - A s)
  for (int it = 1; it < prm.nu1; ++it) {
    ProfScope ps(h->mem.stream, AMG_K_SOLVE_OTHER, abytes + 4.0 * bt * n);
    k_jacobi<T><<<grid_for(n), TPB, 0, s>>>(n, A.rp, A.ci, a, wd, y, sv, w, cc.done);
    AMG_CHECK_LAUNCH();
    std::swap(sv, w);
  }
  {
    ProfScope ps(h->mem.stream, AMG_K_SMOOTH_RESID, abytes + 3.0 * bt * n);
    k_smooth_resid<T><<<grid_for(n), TPB, 0, s>>>(n, A.rp, A.ci, a, y, sv, r, cc.done);
    AMG_CHECK_LAUNCH();
  }
  Level &C = h->lev[k + 1];
  const int nc = C.A.n;
  const bool c_last = (k + 1 == h->nlevels - 1);
  {
    const DCsr &R = L.R;
    ProfScope ps(h->mem.stream, AMG_K_RESTRICT, (idx_bytes + bp) * (double)R.nnz + 4.0 * (nc + 1) + bt * n + bt * nc +
                                        (c_last ? 0.0 : 2.0 * bt * nc));
    k_restrict<T, TP><<<grid_for(nc), TPB, 0, s>>>(nc, R.rp, R.ci, pr_vals<T, TP>(R), r, vec<T>(C.y),
                                                   c_last ? nullptr : VTypes<T>::wd(C), vec<T>(C.s),
                                                   c_last ? -1 : (prm.nu1 > 0 ? 1 : 0), cc.done);
    AMG_CHECK_LAUNCH();
  }
  cycle_level<T, TP>(h, k + 1, cc);
  {
    const DCsr &P = L.P;
    ProfScope ps(h->mem.stream, AMG_K_PROLONG, (idx_bytes + bp) * (double)P.nnz + 4.0 * (n + 1) + 2.0 * bt * n + bt * nc);
    k_prolong<T, TP><<<grid_for(n), TPB, 0, s>>>(n, P.rp, P.ci, pr_vals<T, TP>(P), sv, vec<T>(C.z), r, cc.done);
    AMG_CHECK_LAUNCH();
  }
  if (k == 0) return;  // level 0's post-smoothing is fused with the CG bookkeeping
  // post-smoothing: nu2 sweeps from t (in r)
  T *t = r;
  if (prm.nu2 == 0) {
    ProfScope ps(h->mem.stream, AMG_K_SOLVE_OTHER, 2.0 * bt * n);
    k_copy<T><<<grid_for(n), TPB, 0, s>>>(n, t, vec<T>(L.z));
    AMG_CHECK_LAUNCH();
    return;
  }
  for (int it = 0; it < prm.nu2; ++it) {
    T *dst = (it == prm.nu2 - 1) ? vec<T>(L.z) : (t == r ? w : r);
    ProfScope ps(h->mem.stream, it == prm.nu2 - 1 ? AMG_K_SMOOTH_POST : AMG_K_SOLVE_OTHER, abytes + 4.0 * bt * n);
    k_jacobi<T><<<grid_for(n), TPB, 0, s>>>(n, A.rp, A.ci, a, wd, y, t, dst, cc.done);
    AMG_CHECK_LAUNCH();
    t = dst;
  }
}

// Whole V-cycle from level-0 input (y0, s0 in place) to z (FP64) with the
// level-0 CG bookkeeping of `cc.mode`.
template <typename T, typename TP>
void vcycle(amg_hierarchy *h, double *z, const CycleCtx &cc) {
  cudaStream_t s = h->mem.stream;
  Level &L0 = h->lev[0];
  const int n = L0.A.n;
  const double bt = sizeof(T);
  const T *y = vec<T>(L0.y);
  const T *t;
  bool sweep = true;
  if (h->nlevels == 1) {
    ProfScope ps(h->mem.stream, AMG_K_COARSE, 8.0 * (double)n * n + 2.0 * bt * n);
    const int th = std::min(1024, std::max(32, (n + 31) / 32 * 32));
    k_coarse_solve<T><<<1, th, sizeof(double) * n, s>>>(n, h->L, y, vec<T>(L0.z), cc.done);
    AMG_CHECK_LAUNCH();
    t = vec<T>(L0.z);
    sweep = false;
  } else {
    cycle_level<T, TP>(h, 0, cc);
    T *tt = vec<T>(L0.r), *w = vec<T>(L0.w);
    const T *a = VTypes<T>::A(L0.A);
    const T *wd = VTypes<T>::wd(L0);
    const double abytes = (idx_bytes + bt) * (double)L0.A.nnz + 4.0 * (n + 1);
    for (int it = 0; it + 1 < h->prm.nu2; ++it) {  // all but the last post sweep
      ProfScope ps(h->mem.stream, AMG_K_SOLVE_OTHER, abytes + 4.0 * bt * n);
      k_jacobi<T><<<grid_for(n), TPB, 0, s>>>(n, L0.A.rp, L0.A.ci, a, wd, y, tt, w, cc.done);
      AMG_CHECK_LAUNCH();
      std::swap(tt, w);
    }
    t = tt;
    sweep = h->prm.nu2 > 0;
  }
  const T *a = VTypes<T>::A(L0.A);
  const T *wd = VTypes<T>::wd(L0);
  double bytes = 8.0 * n + bt * n;  // z (FP64) write, t read
  if (sweep) bytes += (idx_bytes + bt) * (double)L0.A.nnz + 4.0 * (n + 1) + 2.0 * bt * n;
  if (cc.mode != POST_APPLY) bytes += 8.0 * n + (cc.mode == POST_FIRST ? 8.0 * n : (cc.flexible ? 8.0 * n : 0.0));
  ProfScope ps(h->mem.stream, AMG_K_SMOOTH_POST, bytes);
  if (sweep)
    k_post0<T, true><<<grid_for(n), TPB, 0, s>>>(n, L0.A.rp, L0.A.ci, a, wd, y, t, z, h->r, h->q, h->p, cc.mode,
                                                 cc.flexible, h->sc, cc.done, h->partials, h->counter);
  else
    k_post0<T, false><<<grid_for(n), TPB, 0, s>>>(n, L0.A.rp, L0.A.ci, a, wd, y, t, z, h->r, h->q, h->p, cc.mode,
                                                  cc.flexible, h->sc, cc.done, h->partials, h->counter);
  AMG_CHECK_LAUNCH();
}

template <typename T>
void load_y0(amg_hierarchy *h, const double *src) {
  Level &L0 = h->lev[0];
  const int n = L0.A.n;
  const bool write_y = !std::is_same<T, double>::value || L0.y != (void *)src;
  k_load_y0<T><<<grid_for(n), TPB, 0, h->mem.stream>>>(n, src, VTypes<T>::wd(L0), vec<T>(L0.y), vec<T>(L0.s),
                                                        write_y, h->prm.nu1 > 0);
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
  // y0 aliases r in FP64 mode
  T *y0 = vec<T>(L0.y);
  {
    ProfScope ps(h->mem.stream, AMG_K_SOLVE_OTHER, (12.0) * A.nnz + 4.0 * (n + 1) + 8.0 * 3 * n + (fp64 ? 0 : bt * n) + 2 * bt * n);
    k_init<T><<<grid_for(n), TPB, 0, s>>>(n, A.rp, A.ci, A.v, b, x, h->r, VTypes<T>::wd(L0), y0, vec<T>(L0.s),
                                          !fp64, h->prm.nu1 > 0, rtol, h->sc, h->hist, h->partials, h->counter);
    AMG_CHECK_LAUNCH();
  }
  CycleCtx cc{done, POST_FIRST, flexible};
  vcycle<T, TP>(h, h->z, cc);
  cc.mode = POST_ITER;
  const double spmv_bytes = 12.0 * A.nnz + 4.0 * (n + 1) + 16.0 * n;
  const double upd_bytes = 48.0 + 2.0 * bt + (fp64 ? 0.0 : bt);
  int launched = 0;
  for (int it = 1; it <= maxit; ++it) {
    {
      ProfScope ps(h->mem.stream, AMG_K_SPMV_DOT, spmv_bytes);
      k_spmv_dot<<<grid_for(n), TPB, 0, s>>>(n, A.rp, A.ci, A.v, h->p, h->q, h->sc, h->partials, h->counter);
      AMG_CHECK_LAUNCH();
    }
    {
      ProfScope ps(h->mem.stream, AMG_K_PCG_UPDATE, upd_bytes * n);
      k_pcg_update<T><<<grid_for(n), TPB, 0, s>>>(n, x, h->r, h->p, h->q, VTypes<T>::wd(L0), y0, vec<T>(L0.s), !fp64,
                                                  h->prm.nu1 > 0, h->sc, h->hist, h->hist_cap, h->d_done,
                                                  h->partials, h->counter);
      AMG_CHECK_LAUNCH();
    }
    vcycle<T, TP>(h, h->z, cc);
    {
      ProfScope ps(h->mem.stream, AMG_K_DIRECTION, 24.0 * n);
      k_direction<<<grid_for(n), TPB, 0, s>>>(n, h->z, h->p, h->sc);
      AMG_CHECK_LAUNCH();
    }
    AMG_CUDA(cudaEventRecord(h->iter_ev[it & 1], s));
    ++launched;
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
size_t alloc_vectors(amg_hierarchy *h) {
  size_t bytes = 0;
  for (int k = 0; k < h->nlevels; ++k) {
    Level &L = h->lev[k];
    const int n = L.A.n;
    auto get = [&](size_t cnt) {
      bytes += cnt * sizeof(T);
      return static_cast<void *>(h->mem.get_n<T>(cnt));
    };
    if (k == 0 && std::is_same<T, double>::value) L.y = h->r;  // FP64: V-cycle input is the CG residual
    else L.y = get(n);
    L.z = get(n);
    if (k < h->nlevels - 1 || k == 0) {
      L.s = get(n);
      L.r = get(n);
      L.w = get(n);
    }
  }
  return bytes;
}

}  // namespace

void prepare_solve(amg_hierarchy *h) {
  Mem &m = h->mem;
  cudaStream_t s = m.stream;
  const int prec = h->prm.precision;
  const int n0 = h->lev[0].A.n;
  // omega / diag, FP32 copies of the hierarchy
  for (int k = 0; k < h->nlevels; ++k) {
    Level &L = h->lev[k];
    const int n = L.A.n;
    L.wd = m.get_n<double>(n);
    h->bytes += 8 * (size_t)n;
    if (prec != AMG_PREC_FP64) {
      L.wd32 = m.get_n<float>(n);
      h->bytes += 4 * (size_t)n;
    }
    {
      ProfScope ps(s, AMG_K_SETUP_OTHER, 4.0 * (n + 1) + 12.0 * L.A.nnz + 12.0 * n);
      k_make_wd<<<grid_for(n), TPB, 0, s>>>(n, L.A.rp, L.A.ci, L.A.v, h->prm.omega, L.wd, L.wd32);
      AMG_CHECK_LAUNCH();
    }
    if (prec != AMG_PREC_FP64) {
      L.A.v32 = m.get_n<float>(std::max<int64_t>(L.A.nnz, 1));
      h->bytes += 4 * (size_t)L.A.nnz;
      k_to_f32<<<grid_for(L.A.nnz), TPB, 0, s>>>(L.A.nnz, L.A.v, L.A.v32);
      AMG_CHECK_LAUNCH();
      if (k < h->nlevels - 1) {
        for (DCsr *M : {&L.P, &L.R}) {
          if (prec == AMG_PREC_FP32) {
            M->v32 = m.get_n<float>(std::max<int64_t>(M->nnz, 1));
            h->bytes += 4 * (size_t)M->nnz;
            k_to_f32<<<grid_for(M->nnz), TPB, 0, s>>>(M->nnz, M->v, M->v32);
          } else {
            M->v16 = m.get_n<__nv_bfloat16>(std::max<int64_t>(M->nnz, 1));
            h->bytes += 2 * (size_t)M->nnz;
            k_to_bf16<<<grid_for(M->nnz), TPB, 0, s>>>(M->nnz, M->v, M->v16);
          }
          AMG_CHECK_LAUNCH();
        }
      }
    }
  }
  // CG vectors (FP64) and scalars
  h->r = m.get_n<double>(n0);
  h->z = m.get_n<double>(n0);
  h->p = m.get_n<double>(n0);
  h->q = m.get_n<double>(n0);
  h->bytes += 32 * (size_t)n0;
  h->sc = m.get_n<PcgScalars>(1);
  h->d_zero = m.get_n<int>(1);
  AMG_CUDA(cudaMemsetAsync(h->d_zero, 0, sizeof(int), s));
  h->partials = m.get_n<double>(3 * MAX_GRID);
  h->counter = m.get_n<unsigned int>(1);
  AMG_CUDA(cudaMemsetAsync(h->counter, 0, sizeof(unsigned int), s));
  h->bytes += (prec == AMG_PREC_FP64) ? alloc_vectors<double>(h) : alloc_vectors<float>(h);
  AMG_CUDA(cudaHostAlloc(reinterpret_cast<void **>(&h->h_done), sizeof(int), cudaHostAllocMapped));
  *h->h_done = 0;
  AMG_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void **>(&h->d_done), h->h_done, 0));
  AMG_CUDA(cudaEventCreateWithFlags(&h->iter_ev[0], cudaEventDisableTiming));
  AMG_CUDA(cudaEventCreateWithFlags(&h->iter_ev[1], cudaEventDisableTiming));
}

void release_solve(amg_hierarchy *h) {
  if (h->h_done) cudaFreeHost(h->h_done);
  h->h_done = nullptr;
  for (auto &e : h->iter_ev)
    if (e) cudaEventDestroy(e);
}

int pcg_solve(amg_hierarchy *h, const double *b, double *x, double rtol, int maxit, int *iters, double *hist,
              int hist_cap) {
  switch (h->prm.precision) {
    case AMG_PREC_FP64: return pcg_impl<double, double>(h, b, x, rtol, maxit, iters, hist, hist_cap);
    case AMG_PREC_FP32: return pcg_impl<float, float>(h, b, x, rtol, maxit, iters, hist, hist_cap);
    default: return pcg_impl<float, __nv_bfloat16>(h, b, x, rtol, maxit, iters, hist, hist_cap);
  }
}

void vcycle_apply(amg_hierarchy *h, const double *y, double *z) {
  switch (h->prm.precision) {
    case AMG_PREC_FP64: vcycle_apply_impl<double, double>(h, y, z); break;
    case AMG_PREC_FP32: vcycle_apply_impl<float, float>(h, y, z); break;
    default: vcycle_apply_impl<float, __nv_bfloat16>(h, y, z); break;
  }
  prof_collect(h->mem.stream);
}

void spmv_level(amg_hierarchy *h, int level, const double *x, double *y) {
  const DCsr &A = h->lev[level].A;
  ProfScope ps(h->mem.stream, AMG_K_SOLVE_OTHER, 12.0 * A.nnz + 4.0 * (A.n + 1) + 16.0 * A.n);
  k_spmv64<<<grid_for(A.n), TPB, 0, h->mem.stream>>>(A.n, A.rp, A.ci, A.v, x, y);
  AMG_CHECK_LAUNCH();
}

}  // namespace amg

// fsai.cu -- set-up of the factored sparse approximate inverse smoother
// (Sec. 2.1, Eq. smo: M^-1 = G^T G with G lower triangular, applied in the
// smoother S = I - omega M^-1 A of Eq. smoother as two sparse products).
//
// The paper's aFSAI grows G's pattern adaptively (a cited method it does not
// describe); this library takes the static pattern of the lower triangle of
// A_k (Kolotilina & Yeremin).  Row i of G, on P_i = { j <= i : a_ij stored }
// (ascending, ending at the diagonal), is the solution of
// A[P_i, P_i] g = e_last scaled to (G A G^T)_ii = 1.  With the Cholesky
// factor A[P_i, P_i] = L L^T that scaled solution is g = L^-T e_last, so each
// row costs one dense Cholesky of its principal submatrix and one triangular
// solve; rows are binned by m:
//   m <= 8: a thread per row, the submatrix in registers (the 7-point
//   operators' finest levels: 4 entries);
//   m <= 16 / m <= 32: 8 / 16 lanes per row, the submatrix in a per-row slice
//   of shared memory, factored right-looking by the row's lanes;
//   m <= 64 / longer: a block of 64 / 256 threads per row, the submatrix a
//   packed lower triangle in shared memory (a warp per row in global scratch
//   when it does not fit).
// Each pivot takes one reciprocal square root, kept on the diagonal of the
// factor, in place of a square root and a division (FP64 square roots and
// divisions are instruction sequences on GB300's narrow FP64 pipe).
// G^T is stored too (a CSR transpose), its values scaled by omega, so that a
// smoothing step is u = G w, s += (omega G^T) u.
#include <cuda_runtime.h>

#include <algorithm>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr int TPB = 256;

// cnt[i] = number of stored entries of row i with column <= i; flags[0] when
// the last of them is not the diagonal.  *mmax receives the largest count.
__global__ void k_fsai_count(int n, const int *__restrict__ rp, const int *__restrict__ ci, int *__restrict__ cnt,
                             int *mmax, int *flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = rp[i], e = rp[i + 1];
  int lo = b, hi = e;  // first entry with column > i
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ci[mid] <= i) lo = mid + 1;
    else hi = mid;
  }
  const int m = lo - b;
  cnt[i] = m;
  if (m == 0 || ci[lo - 1] != i) flags[0] = 1;
  atomicMax(mmax, m);
}

// Thread per row, rows of at most MM lower entries, the submatrix in
// registers; rows (may be null: rows 0..nrows-1) lists the rows to take.
// flags[1]: a non-positive pivot.
template <int MM>
__global__ void __launch_bounds__(TPB) k_fsai_rows(int nrows, const int *__restrict__ rows,
                                                   const int *__restrict__ rp, const int *__restrict__ ci,
                                                   const double *__restrict__ a, const int *__restrict__ grp,
                                                   int *__restrict__ gci, double *__restrict__ gv, int *flags) {
  const int r0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (r0 >= nrows) return;
  const int i = rows ? rows[r0] : r0;
  const int b = rp[i], o = grp[i], m = grp[i + 1] - o;
  int P[MM];
  double M[MM][MM];
#pragma unroll
  for (int r = 0; r < MM; ++r) P[r] = r < m ? ci[b + r] : 0;
#pragma unroll
  for (int r = 0; r < MM; ++r) {
    if (r >= m) break;
    const int row = P[r], rb = rp[row];
    // the lower part of row P[r] holds every P[c] <= P[r] that A couples to it
    int q = rb;
#pragma unroll
    for (int c = 0; c <= r; ++c) {
      const int want = P[c];
      while (ci[q] < want) ++q;  // ascending walk: P is ascending and P[r] is in row P[r]
      M[r][c] = ci[q] == want ? a[q] : 0.0;
    }
  }
  bool ok = true;
#pragma unroll
  for (int j = 0; j < MM; ++j) {
    if (j >= m) break;
    double d = M[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= M[j][k] * M[j][k];
    ok = ok && d > 0.0;
    const double inv = rsqrt(d > 0.0 ? d : 1.0);  // 1 / l_jj, kept on the diagonal
    M[j][j] = inv;
#pragma unroll
    for (int r = j + 1; r < MM; ++r) {
      if (r >= m) break;
      double s = M[r][j];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= M[r][k] * M[j][k];
      M[r][j] = s * inv;
    }
  }
  if (!ok) flags[1] = 1;
  double g[MM];
#pragma unroll
  for (int k = MM - 1; k >= 0; --k) {
    if (k >= m) continue;
    double s = k == m - 1 ? 1.0 : 0.0;
#pragma unroll
    for (int l = k + 1; l < MM; ++l)
      if (l < m) s -= M[l][k] * g[l];
    g[k] = s * M[k][k];
  }
#pragma unroll
  for (int r = 0; r < MM; ++r)
    if (r < m) {
      gci[o + r] = P[r];
      gv[o + r] = g[r];
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Warp per row, for rows too long for k_fsai_block's shared memory.  Each
// warp has a slice of ld * ld + 2 ld doubles (the submatrix, g, and P_i as
// ints) in global scratch (warp w at w * slice; warps beyond nw have no slice
// and return).  Rows are visited with stride nw.
//   gather: the lower parts of the rows P_i[r] are walked as one flattened
//     sequence (lane u takes entry u, found by a shuffle search over the
//     prefix of the parts' lengths); an entry of column l lands at
//     M[r][c] with P_i[c] = l (binary search in P_i);
//   factor: left-looking Cholesky (global scratch is read far more than
//     written), one reciprocal square root per pivot;
//   solve: L^T g = e_last backwards by columns (no warp sums).
__global__ void __launch_bounds__(TPB) k_fsai_warp(int n, const int *__restrict__ rows, const int *__restrict__ rp,
                                                   const int *__restrict__ ci,
                                                   const double *__restrict__ a, const int *__restrict__ grp,
                                                   int *__restrict__ gci, double *__restrict__ gv, double *scratch,
                                                   int ld, int nw, int *flags) {
  const int lane = threadIdx.x & 31;
  const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (w >= nw) return;
  const size_t slice = (size_t)ld * ld + 2 * (size_t)ld;
  double *M = scratch + slice * w;
  double *g = M + (size_t)ld * ld;
  int *P = reinterpret_cast<int *>(g + ld);
  for (int r0 = w; r0 < n; r0 += nw) {
    const int i = rows ? rows[r0] : r0;
    const int b = rp[i], o = grp[i], m = grp[i + 1] - o;
    for (int t = lane; t < m; t += 32) P[t] = ci[b + t];
    for (int t = lane; t < m * m; t += 32) M[(size_t)(t / m) * ld + (t % m)] = 0.0;
    __syncwarp();
    for (int r0 = 0; r0 < m; r0 += 32) {
      const int r = r0 + lane;
      int rs = 0, len = 0;
      if (r < m) {  // the lower part of row P[r]: columns <= P[r], ending at its diagonal
        const int row = P[r];
        rs = rp[row];
        int lo = rs, hi = rp[row + 1];
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (ci[mid] <= row) lo = mid + 1;
          else hi = mid;
        }
        len = lo - rs;
      }
      int incl = len;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
      }
      const int excl = incl - len;
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      for (int u0 = 0; u0 < total; u0 += 32) {
        const int u = u0 + lane;
        int src = 0;
#pragma unroll
        for (int step = 16; step; step >>= 1) {
          const int ex = __shfl_sync(0xffffffffu, excl, src + step);
          if (ex <= u) src += step;
        }
        const int srs = __shfl_sync(0xffffffffu, rs, src), sex = __shfl_sync(0xffffffffu, excl, src);
        if (u < total) {
          const int q = srs + u - sex;
          const int l = ci[q];
          int lo = 0, hi = r0 + src;  // P[c] = l with c <= r
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (P[mid] < l) lo = mid + 1;
            else hi = mid;
          }
          if (P[lo] == l) M[(size_t)(r0 + src) * ld + lo] = a[q];
        }
      }
    }
    __syncwarp();
    bool ok = true;
    for (int j = 0; j < m; ++j) {  // left-looking; 1 / l_jj kept on the diagonal
      const double *Mj = M + (size_t)j * ld;
      double d = 0.0;
      for (int k = lane; k < j; k += 32) d += Mj[k] * Mj[k];
      d = Mj[j] - warp_sum(d);
      ok = ok && d > 0.0;
      const double inv = rsqrt(d > 0.0 ? d : 1.0);
      for (int r = j + 1 + lane; r < m; r += 32) {
        double *Mr = M + (size_t)r * ld;
        double sum = Mr[j];
        for (int k = 0; k < j; ++k) sum -= Mr[k] * Mj[k];
        Mr[j] = sum * inv;
      }
      __syncwarp();
      if (lane == 0) M[(size_t)j * ld + j] = inv;
      __syncwarp();
    }
    if (!ok && lane == 0) flags[1] = 1;
    // L^T g = e_last, backwards by columns: once g_k = rhs_k / l_kk is known,
    // rhs_l -= l_kl g_k for every l < k (the lanes split the l)
    for (int t = lane; t < m; t += 32) g[t] = t == m - 1 ? 1.0 : 0.0;
    __syncwarp();
    for (int k = m - 1; k >= 0; --k) {
      const double gk = g[k] * M[(size_t)k * ld + k];
      __syncwarp();
      const double *Mk = M + (size_t)k * ld;
      for (int l = lane; l < k; l += 32) g[l] -= Mk[l] * gk;
      if (lane == 0) g[k] = gk;
      __syncwarp();
    }
    for (int r = lane; r < m; r += 32) {
      gci[o + r] = P[r];
      gv[o + r] = g[r];
    }
    __syncwarp();
  }
}

// Doubles per row slice of k_fsai_group: the submatrix (LD x LD), g (LD),
// then P_i as ints; an odd count, so that the slices of one warp start on
// different banks.
template <int LD>
__host__ __device__ constexpr int group_slice() {
  return (LD * LD + LD + (LD + 1) / 2) | 1;
}

// G lanes per row (32 / G rows per warp) for rows of at most LD lower
// entries.  Each row has a slice of group_slice<LD>() doubles in shared
// memory: the lanes gather the rows of A[P_i, P_i] (each lane walks rows r,
// r + G, ... of P_i; gathering the rows as one flat list of entries over the
// lanes measured slower), factor it right-looking with the trailing
// triangle's (r, c) pairs spread over the row's lanes, one reciprocal square
// root per pivot, and solve L^T g = e_last by columns.  Several short rows per warp
// keep its lanes busy (a warp per row leaves most idle on rows of ~10
// entries) while the per-row slices stay small enough for many warps per SM.
// The rows of a warp step through the factor together (up to the warp's
// longest row), so its __syncwarp()s are reached by every lane.
template <int G, int LD>
__global__ void __launch_bounds__(TPB) k_fsai_group(int nrows, const int *__restrict__ rows,
                                                    const int *__restrict__ rp, const int *__restrict__ ci,
                                                    const double *__restrict__ a, const int *__restrict__ grp,
                                                    int *__restrict__ gci, double *__restrict__ gv, int *flags) {
  constexpr int RPW = 32 / G;
  constexpr int SLICE = group_slice<LD>();
  extern __shared__ __align__(16) double fsai_gsmem[];
  const int lane = threadIdx.x & 31, sub = lane & (G - 1);
  double *M = fsai_gsmem + (size_t)(threadIdx.x / G) * SLICE;
  double *g = M + LD * LD;
  int *P = reinterpret_cast<int *>(g + LD);
  const int wg = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
  bool ok = true;
  for (int base = wg * RPW; base < nrows; base += nwarps * RPW) {  // warp-uniform
    const int r0 = base + lane / G;
    int b = 0, o = 0, m = 0;
    if (r0 < nrows) {
      const int i = rows[r0];
      b = rp[i];
      o = grp[i];
      m = grp[i + 1] - o;
    }
    const int mw = (int)__reduce_max_sync(0xffffffffu, (unsigned)m);
    for (int t = sub; t < m; t += G) P[t] = ci[b + t];
    for (int t = sub; t < m * LD; t += G) M[t] = 0.0;
    __syncwarp();
    for (int r = sub; r < m; r += G) {  // row P[r]: its columns P[c] (c <= r) are <= P[r]
      const int row = P[r];
      for (int q = rp[row], qe = rp[row + 1]; q < qe; ++q) {
        const int l = ci[q];
        if (l > row) break;
        int lo = 0, hi = r;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (P[mid] < l) lo = mid + 1;
          else hi = mid;
        }
        if (P[lo] == l) M[r * LD + lo] = a[q];
      }
    }
    __syncwarp();
    for (int j = 0; j < mw; ++j) {
      const bool act = j < m;
      double inv = 0.0;
      if (act) {
        const double d = M[j * LD + j];
        ok = ok && d > 0.0;
        inv = rsqrt(d > 0.0 ? d : 1.0);  // 1 / l_jj, kept on the diagonal
      }
      __syncwarp();
      if (act) {
        for (int r = j + 1 + sub; r < m; r += G) M[r * LD + j] *= inv;
        if (sub == 0) M[j * LD + j] = inv;
      }
      __syncwarp();
      if (act) {  // pair t = r'(r'+1)/2 + c' of the trailing triangle, r' = r - j - 1
        const int sz = m - j - 1, npair = sz * (sz + 1) / 2;
        int rr = 0, cc = sub;
        while (cc > rr) {
          cc -= rr + 1;
          ++rr;
        }
        for (int t = sub; t < npair; t += G) {
          const int r = j + 1 + rr, c = j + 1 + cc;
          M[r * LD + c] -= M[r * LD + j] * M[c * LD + j];
          cc += G;
          while (cc > rr) {
            cc -= rr + 1;
            ++rr;
          }
        }
      }
      __syncwarp();
    }
    for (int t = sub; t < m; t += G) g[t] = t == m - 1 ? 1.0 : 0.0;
    __syncwarp();
    for (int k = mw - 1; k >= 0; --k) {  // L^T g = e_last by columns
      const bool act = k < m;
      const double gk = act ? g[k] * M[k * LD + k] : 0.0;
      __syncwarp();
      if (act) {
        for (int l = sub; l < k; l += G) g[l] -= M[k * LD + l] * gk;
        if (sub == 0) g[k] = gk;
      }
      __syncwarp();
    }
    for (int r = sub; r < m; r += G) {
      gci[o + r] = P[r];
      gv[o + r] = g[r];
    }
    __syncwarp();
  }
  if (!ok) flags[1] = 1;
}

// A block per row for rows of more than 32 lower entries (ld = the longest
// such row of the level).  The submatrix is kept as a packed lower triangle,
// M(r, c) at r (r + 1) / 2 + c, followed by g (ld doubles) and P_i (ld ints),
// in shared memory: ld = 123 then takes 62 KB, three rows per SM, where an
// ld x ld slice per warp left one warp per SM.  The block's threads gather
// the rows of A[P_i, P_i] (a thread per row of P_i), factor it right-looking
// -- each column's pivot as
// one reciprocal square root, the trailing triangle's (r, c) pairs spread over
// all threads -- and solve L^T g = e_last by columns.
__device__ __forceinline__ int tri(int r, int c) { return r * (r + 1) / 2 + c; }

__global__ void __launch_bounds__(TPB) k_fsai_block(int nrows, const int *__restrict__ rows,
                                                    const int *__restrict__ rp, const int *__restrict__ ci,
                                                    const double *__restrict__ a, const int *__restrict__ grp,
                                                    int *__restrict__ gci, double *__restrict__ gv, int ld,
                                                    int *flags) {
  extern __shared__ __align__(16) double fsai_bsmem[];
  double *M = fsai_bsmem;
  double *g = M + (size_t)ld * (ld + 1) / 2;
  int *P = reinterpret_cast<int *>(g + ld);
  const int t = threadIdx.x, nt = blockDim.x;
  bool ok = true;
  for (int r0 = blockIdx.x; r0 < nrows; r0 += gridDim.x) {
    const int i = rows[r0];
    const int b = rp[i], o = grp[i], m = grp[i + 1] - o;
    for (int e = t; e < m; e += nt) P[e] = ci[b + e];
    for (int e = t; e < m * (m + 1) / 2; e += nt) M[e] = 0.0;
    __syncthreads();
    for (int r = t; r < m; r += nt) {  // row P[r]: its columns P[c] (c <= r) are <= P[r]
      const int row = P[r];
      for (int q = rp[row], qe = rp[row + 1]; q < qe; ++q) {
        const int l = ci[q];
        if (l > row) break;
        int lo = 0, hi = r;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (P[mid] < l) lo = mid + 1;
          else hi = mid;
        }
        if (P[lo] == l) M[tri(r, lo)] = a[q];
      }
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
      const double d = M[tri(j, j)];
      ok = ok && d > 0.0;
      const double inv = rsqrt(d > 0.0 ? d : 1.0);  // 1 / l_jj
      for (int r = j + 1 + t; r < m; r += nt) M[tri(r, j)] *= inv;
      __syncthreads();
      // trailing triangle rows and columns j+1..m-1: pair u = r'(r'+1)/2 + c'
      const int sz = m - j - 1, npair = sz * (sz + 1) / 2;
      int rr = 0, cc = t;
      while (cc > rr) {
        cc -= rr + 1;
        ++rr;
      }
      for (int u = t; u < npair; u += nt) {
        const int r = j + 1 + rr, c = j + 1 + cc;
        M[tri(r, c)] -= M[tri(r, j)] * M[tri(c, j)];
        cc += nt;
        while (cc > rr) {
          cc -= rr + 1;
          ++rr;
        }
      }
      if (t == 0) M[tri(j, j)] = inv;  // no thread reads the pivot in this phase
      __syncthreads();
    }
    for (int e = t; e < m; e += nt) g[e] = e == m - 1 ? 1.0 : 0.0;
    __syncthreads();
    for (int k = m - 1; k >= 0; --k) {  // L^T g = e_last by columns
      const double gk = g[k] * M[tri(k, k)];
      __syncthreads();
      for (int l = t; l < k; l += nt) g[l] -= M[tri(k, l)] * gk;
      if (t == 0) g[k] = gk;
      __syncthreads();
    }
    for (int e = t; e < m; e += nt) {
      gci[o + e] = P[e];
      gv[o + e] = g[e];
    }
    __syncthreads();
  }
  if (!ok) flags[1] = 1;
}

// shared memory of k_fsai_block for rows of at most ld entries, and the
// most a block may take (the opt-in limit per block)
constexpr int kBlockSmemMax = 227 * 1024;
size_t block_smem_bytes(int ld) {
  return ((size_t)ld * (ld + 1) / 2 + (size_t)ld) * sizeof(double) + (size_t)ld * sizeof(int);
}

template <int G, int LD>
constexpr size_t group_slice_bytes() {
  return (size_t)group_slice<LD>() * sizeof(double);
}

// Rows binned by their lower-entry count m: bin 0 m <= 8, 1 m <= 16,
// 2 m <= 32, 3 m <= 64, 4 longer; list b at lists + b * n, its count in
// counts[b].  Tiles of the block append with one atomic per bin.
constexpr int kFsaiBins = 5;
__global__ void k_fsai_bin(int n, const int *__restrict__ grp, int *__restrict__ lists, int *counts) {
  __shared__ int c[kFsaiBins], base[kFsaiBins];
  if (threadIdx.x < kFsaiBins) c[threadIdx.x] = 0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int bin = -1, pos = 0;
  if (i < n) {
    const int m = grp[i + 1] - grp[i];
    bin = m <= 8 ? 0 : m <= 16 ? 1 : m <= 32 ? 2 : m <= 64 ? 3 : 4;
    pos = atomicAdd(&c[bin], 1);
  }
  __syncthreads();
  if (threadIdx.x < kFsaiBins) base[threadIdx.x] = c[threadIdx.x] ? atomicAdd(&counts[threadIdx.x], c[threadIdx.x]) : 0;
  __syncthreads();
  if (bin >= 0) lists[(size_t)bin * n + base[bin] + pos] = i;
}

__global__ void k_scale(int64_t n, double f, double *__restrict__ v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= f;
}

// Rows of a list with at most LD lower entries, G lanes each, blocks of tpb
// threads (tpb / G row slices of shared memory per block).
template <int G, int LD>
void launch_group(const int *rows, int nrows, int tpb, const DCsr &A, DCsr &G_, int *flags, cudaStream_t s) {
  const size_t smem = (size_t)(tpb / G) * group_slice_bytes<G, LD>();
  static std::atomic<unsigned long long> attr{0};
  ensure_smem_attr(k_fsai_group<G, LD>, (int)smem, attr);
  const int rows_per_block = tpb / G;
  const int blocks = std::max(1, std::min(ceil_div(nrows, rows_per_block), kNumSMs * 16));
  k_fsai_group<G, LD><<<blocks, tpb, smem, s>>>(nrows, rows, A.rp, A.ci, A.v, G_.rp, G_.ci, G_.v, flags);
  AMG_CHECK_LAUNCH();
}

}  // namespace

void build_fsai(amg_hierarchy *h, int k) {
  Mem &m = h->mem;
  cudaStream_t s = m.stream;
  Level &L = h->lev[k];
  const DCsr &A = L.A;
  const int n = A.n;
  DCsr &G = L.G;
  Buf<int> cnt(m, (size_t)n + 1), meta(m, 4);
  AMG_CUDA(cudaMemsetAsync(meta.p, 0, 4 * sizeof(int), s));
  {
    ProfScope ps(s, AMG_K_FSAI, 4.0 * (n + 1) + 4.0 * A.nnz + 4.0 * n, k);
    k_fsai_count<<<ceil_div(n, TPB), TPB, 0, s>>>(n, A.rp, A.ci, cnt.p, meta.p + 2, meta.p);
    AMG_CHECK_LAUNCH();
  }
  G.n = G.ncols = n;
  G.rp = m.get_n<int>((size_t)n + 1);
  G.nnz = scan_counts(m, cnt.p, G.rp, n);  // synchronises: meta is current too
  int hm[4];
  AMG_CUDA(cudaMemcpyAsync(hm, meta.p, sizeof(hm), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  if (hm[0]) {
    set_error("FSAI: a row of A_%d lacks its diagonal", k);
    throw Status{AMG_ERR_INVALID_ARG};
  }
  const int mmax = hm[2];
  G.ci = m.get_n<int>(std::max<int64_t>(G.nnz, 1));
  G.v = m.get_n<double>(std::max<int64_t>(G.nnz, 1));
  {
    // bytes: A's lower rows gathered (once per use, ~m per row), G written
    ProfScope ps(s, AMG_K_FSAI, 4.0 * (n + 1) + 12.0 * (double)A.nnz + 4.0 * (n + 1) + 12.0 * (double)G.nnz, k);
    if (mmax <= 4) {
      k_fsai_rows<4><<<ceil_div(n, TPB), TPB, 0, s>>>(n, nullptr, A.rp, A.ci, A.v, G.rp, G.ci, G.v, meta.p);
    } else if (mmax <= 8) {
      k_fsai_rows<8><<<ceil_div(n, TPB), TPB, 0, s>>>(n, nullptr, A.rp, A.ci, A.v, G.rp, G.ci, G.v, meta.p);
    } else {
      // rows binned by m: registers (m <= 8), 8 lanes per row (m <= 16),
      // 16 lanes per row (m <= 32), a block of 64 threads per row (m <= 64),
      // a block of 256 (longer; a warp per row in global scratch when the
      // packed triangle does not fit in shared memory)
      Buf<int> lists(m, kFsaiBins * (size_t)n), cnts(m, kFsaiBins);
      AMG_CUDA(cudaMemsetAsync(cnts.p, 0, kFsaiBins * sizeof(int), s));
      k_fsai_bin<<<ceil_div(n, TPB), TPB, 0, s>>>(n, G.rp, lists.p, cnts.p);
      AMG_CHECK_LAUNCH();
      int hn[kFsaiBins];
      AMG_CUDA(cudaMemcpyAsync(hn, cnts.p, sizeof(hn), cudaMemcpyDeviceToHost, s));
      AMG_CUDA(cudaStreamSynchronize(s));
      auto list = [&](int b) { return lists.p + (size_t)b * n; };
      if (hn[0] > 0) {
        k_fsai_rows<8><<<ceil_div(hn[0], TPB), TPB, 0, s>>>(hn[0], list(0), A.rp, A.ci, A.v, G.rp, G.ci, G.v,
                                                            meta.p);
        AMG_CHECK_LAUNCH();
      }
      if (hn[1] > 0) launch_group<8, 16>(list(1), hn[1], TPB, A, G, meta.p, s);
      if (hn[2] > 0) launch_group<16, 32>(list(2), hn[2], TPB / 2, A, G, meta.p, s);
      static std::atomic<unsigned long long> attr{0};
      ensure_smem_attr(k_fsai_block, kBlockSmemMax, attr);
      if (hn[3] > 0) {
        const int ld = std::min(mmax, 64);
        const int blocks = std::max(1, std::min(hn[3], kNumSMs * 32));
        k_fsai_block<<<blocks, 64, block_smem_bytes(ld), s>>>(hn[3], list(3), A.rp, A.ci, A.v, G.rp, G.ci, G.v, ld,
                                                              meta.p);
        AMG_CHECK_LAUNCH();
      }
      const int nbig = hn[4];
      const int *llarge = list(4);
      if (nbig > 0) {
        const size_t bsm = block_smem_bytes(mmax);
        if (bsm <= (size_t)kBlockSmemMax) {  // a block per row, packed triangle in shared memory
          const int blocks = std::max(1, std::min(nbig, kNumSMs * 8));
          k_fsai_block<<<blocks, TPB, bsm, s>>>(nbig, llarge, A.rp, A.ci, A.v, G.rp, G.ci, G.v, mmax, meta.p);
        } else {  // a warp per row, the submatrix in a global scratch slice
          // slice per warp: ld * ld + 2 ld doubles (P_i's ints fit in the last ld)
          const size_t slice = ((size_t)mmax * mmax + 2 * (size_t)mmax) * sizeof(double);
          const int64_t cap_warps = std::max<int64_t>(1, ((int64_t)256 << 20) / (int64_t)slice);
          const int warps = (int)std::min<int64_t>({(int64_t)nbig, (int64_t)kNumSMs * 16, cap_warps});
          Buf<double> scr(m, slice / sizeof(double) * (size_t)warps);
          k_fsai_warp<<<ceil_div((int64_t)warps * 32, TPB), TPB, 0, s>>>(nbig, llarge, A.rp, A.ci, A.v, G.rp, G.ci,
                                                                        G.v, scr.p, mmax, warps, meta.p);
        }
      }
    }
    AMG_CHECK_LAUNCH();
  }
  AMG_CUDA(cudaMemcpyAsync(hm, meta.p, sizeof(hm), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  if (hm[1]) {
    set_error("FSAI: a principal submatrix of A_%d is not positive definite", k);
    throw Status{AMG_ERR_NOT_SPD};
  }
  csr_transpose(m, G, n, L.GT);
  {
    ProfScope ps(s, AMG_K_FSAI, 16.0 * (double)L.GT.nnz, k);
    k_scale<<<std::max(1, std::min(ceil_div(L.GT.nnz, TPB), kNumSMs * 8)), TPB, 0, s>>>(L.GT.nnz, h->prm.omega,
                                                                                        L.GT.v);
    AMG_CHECK_LAUNCH();
  }
}

}  // namespace amg

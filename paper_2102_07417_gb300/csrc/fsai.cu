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
// solve:
//   rows of at most 4 or 8 lower entries: a thread per row, the submatrix in
//   registers (the 7-point operators' finest levels: 4 entries);
//   longer rows: a warp per row, the submatrix in a per-warp slice of shared
//   memory (global scratch when a slice does not fit), factored right-looking
//   by the lanes.
// G^T is stored too (a CSR transpose), its values scaled by omega, so that a
// smoothing step is u = G w, s += (omega G^T) u.
#include <cuda_runtime.h>

#include <algorithm>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr int TPB = 256;
constexpr int kThreadRows = 16;  // longest lower row taken by the thread-per-row kernel

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

// Thread per row, rows of at most MM lower entries.  flags[1]: a non-positive pivot.
template <int MM>
__global__ void __launch_bounds__(TPB) k_fsai_rows(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                   const double *__restrict__ a, const int *__restrict__ grp,
                                                   int *__restrict__ gci, double *__restrict__ gv, int *flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
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
    const double l = sqrt(d > 0.0 ? d : 1.0);
    M[j][j] = l;
#pragma unroll
    for (int r = j + 1; r < MM; ++r) {
      if (r >= m) break;
      double s = M[r][j];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= M[r][k] * M[j][k];
      M[r][j] = s / l;
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
    g[k] = s / M[k][k];
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

// Warp per row.  Each warp has a slice of ld * ld + 2 ld doubles (the
// submatrix, g, and P_i as ints) -- in shared memory when SMEM (the block's
// dynamic shared memory, warp w at w * slice), else in global scratch (warp w
// at w * slice; warps beyond nw have no slice and return).  Rows are visited
// with stride nw.
//   gather: the lower parts of the rows P_i[r] are walked as one flattened
//     sequence (lane u takes entry u, found by a shuffle search over the
//     prefix of the parts' lengths); an entry of column l lands at
//     M[r][c] with P_i[c] = l (binary search in P_i);
//   factor: right-looking Cholesky, column j scaled by the lanes, then the
//     trailing lower triangle updated with independent multiply-adds;
//   solve: L^T g = e_last backwards, one warp sum per component.
template <bool SMEM>
__global__ void __launch_bounds__(TPB) k_fsai_warp(int n, const int *__restrict__ rows, const int *__restrict__ rp,
                                                   const int *__restrict__ ci,
                                                   const double *__restrict__ a, const int *__restrict__ grp,
                                                   int *__restrict__ gci, double *__restrict__ gv, double *scratch,
                                                   int ld, int nw, int *flags) {
  extern __shared__ __align__(16) double fsai_smem[];
  const int lane = threadIdx.x & 31;
  const int wb = threadIdx.x >> 5;
  const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (w >= nw) return;
  const size_t slice = (size_t)ld * ld + 2 * (size_t)ld;
  double *M = SMEM ? fsai_smem + slice * wb : scratch + slice * w;
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
    if (SMEM) {  // right-looking: independent updates of the trailing triangle
      for (int j = 0; j < m; ++j) {
        const double d = M[(size_t)j * ld + j];
        ok = ok && d > 0.0;
        const double l = sqrt(d > 0.0 ? d : 1.0), inv = 1.0 / l;
        __syncwarp();
        for (int r = j + 1 + lane; r < m; r += 32) M[(size_t)r * ld + j] *= inv;
        if (lane == 0) M[(size_t)j * ld + j] = l;
        __syncwarp();
        for (int r = j + 1 + lane; r < m; r += 32) {  // trailing update of row r: columns j+1..r
          double *Mr = M + (size_t)r * ld;
          const double lrj = Mr[j];
          for (int c = j + 1; c <= r; ++c) Mr[c] -= lrj * M[(size_t)c * ld + j];
        }
        __syncwarp();
      }
    } else {  // left-looking: global scratch is read far more than written
      for (int j = 0; j < m; ++j) {
        const double *Mj = M + (size_t)j * ld;
        double d = 0.0;
        for (int k = lane; k < j; k += 32) d += Mj[k] * Mj[k];
        d = Mj[j] - warp_sum(d);
        ok = ok && d > 0.0;
        const double l = sqrt(d > 0.0 ? d : 1.0), inv = 1.0 / l;
        for (int r = j + 1 + lane; r < m; r += 32) {
          double *Mr = M + (size_t)r * ld;
          double sum = Mr[j];
          for (int k = 0; k < j; ++k) sum -= Mr[k] * Mj[k];
          Mr[j] = sum * inv;
        }
        __syncwarp();
        if (lane == 0) M[(size_t)j * ld + j] = l;
        __syncwarp();
      }
    }
    if (!ok && lane == 0) flags[1] = 1;
    // L^T g = e_last, backwards: g_k = (e_k - sum_{l > k} L_lk g_l) / L_kk
    for (int k = m - 1; k >= 0; --k) {
      double s = 0.0;
      for (int l = k + 1 + lane; l < m; l += 32) s += M[(size_t)l * ld + k] * g[l];
      s = warp_sum(s);
      if (lane == 0) g[k] = ((k == m - 1 ? 1.0 : 0.0) - s) / M[(size_t)k * ld + k];
      __syncwarp();
    }
    for (int r = lane; r < m; r += 32) {
      gci[o + r] = P[r];
      gv[o + r] = g[r];
    }
    __syncwarp();
  }
}

// Thread per row for rows of at most ld lower entries: the submatrix in the
// thread's slice of shared memory, interleaved across the block's threads
// (element e of thread t at e * NT + t, so a warp's accesses hit distinct
// banks).  Every FP64 operation of the factor and the solve is then done by
// all lanes of a warp at once: GB300 issues FP64 per warp at a small fraction
// of the FP32 rate, so a factor spread over the lanes of one row (the warp
// kernel) spends most of its FP64 issue slots on idle lanes.  rows (may be
// null: all rows) lists the rows to take.
__global__ void k_fsai_thread(int n, const int *__restrict__ rows, int nrows, const int *__restrict__ rp,
                              const int *__restrict__ ci, const double *__restrict__ a, const int *__restrict__ grp,
                              int *__restrict__ gci, double *__restrict__ gv, int ld, int *flags) {
  extern __shared__ __align__(16) double fsai_tsmem[];
  const int NT = blockDim.x, t = threadIdx.x;
  double *M = fsai_tsmem;              // M[(r * ld + c) * NT + t]
  double *g = fsai_tsmem + (size_t)ld * ld * NT;  // g[k * NT + t]
  for (int r0 = blockIdx.x * NT + t; r0 < nrows; r0 += gridDim.x * NT) {
    const int i = rows ? rows[r0] : r0;
    const int b = rp[i], o = grp[i], m = grp[i + 1] - o;
    const int *P = ci + b;  // the row's lower part, ascending, ending at i
    for (int r = 0; r < m; ++r) {
      // row P[r] and P[0..r] are both ascending: one merge walk
      const int row = P[r];
      int q = rp[row], c = 0;
      while (c <= r) {
        const int col = ci[q];
        if (col == P[c]) {
          M[(size_t)(r * ld + c) * NT + t] = a[q];
          ++c;
          ++q;
        } else if (col < P[c]) {
          ++q;
        } else {
          M[(size_t)(r * ld + c) * NT + t] = 0.0;
          ++c;
        }
      }
    }
    bool ok = true;
    for (int j = 0; j < m; ++j) {  // left-looking Cholesky, one multiply by 1/l_jj per entry
      double d = M[(size_t)(j * ld + j) * NT + t];
      for (int k = 0; k < j; ++k) {
        const double v = M[(size_t)(j * ld + k) * NT + t];
        d -= v * v;
      }
      ok = ok && d > 0.0;
      const double l = sqrt(d > 0.0 ? d : 1.0), inv = 1.0 / l;
      M[(size_t)(j * ld + j) * NT + t] = l;
      for (int r = j + 1; r < m; ++r) {
        double s = M[(size_t)(r * ld + j) * NT + t];
        for (int k = 0; k < j; ++k) s -= M[(size_t)(r * ld + k) * NT + t] * M[(size_t)(j * ld + k) * NT + t];
        M[(size_t)(r * ld + j) * NT + t] = s * inv;
      }
    }
    if (!ok) flags[1] = 1;
    for (int k = m - 1; k >= 0; --k) {  // L^T g = e_last
      double s = k == m - 1 ? 1.0 : 0.0;
      for (int l = k + 1; l < m; ++l) s -= M[(size_t)(l * ld + k) * NT + t] * g[(size_t)l * NT + t];
      g[(size_t)k * NT + t] = s / M[(size_t)(k * ld + k) * NT + t];
    }
    for (int r = 0; r < m; ++r) {
      gci[o + r] = P[r];
      gv[o + r] = g[(size_t)r * NT + t];
    }
  }
}

// Rows of at most lim lower entries to list s, the others to list l (counts in
// ns, nl); tiles of the block append with one atomic each.
__global__ void k_fsai_split(int n, const int *__restrict__ grp, int lim, int *__restrict__ ls, int *ns,
                             int *__restrict__ ll, int *nl) {
  __shared__ int cs, cl, bs, bl;
  if (threadIdx.x == 0) cs = cl = 0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < n;
  const bool small = live && grp[i + 1] - grp[i] <= lim;
  int ps = -1, pl = -1;
  if (live && small) ps = atomicAdd(&cs, 1);
  if (live && !small) pl = atomicAdd(&cl, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    bs = cs ? atomicAdd(ns, cs) : 0;
    bl = cl ? atomicAdd(nl, cl) : 0;
  }
  __syncthreads();
  if (ps >= 0) ls[bs + ps] = i;
  if (pl >= 0) ll[bl + pl] = i;
}

__global__ void k_scale(int64_t n, double f, double *__restrict__ v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= f;
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
    auto launch_thread = [&](const int *rows, int nrows, int ld) {
      const size_t per = ((size_t)ld * ld + ld) * sizeof(double);  // per thread
      const int nt = (int)std::max<size_t>(32, std::min<size_t>(256, (200 * 1024 / per) / 32 * 32));
      static std::atomic<unsigned long long> attr{0};
      ensure_smem_attr(k_fsai_thread, 200 * 1024, attr);
      const int blocks = std::max(1, std::min(ceil_div(nrows, nt), kNumSMs * 8));
      k_fsai_thread<<<blocks, nt, per * nt, s>>>(n, rows, nrows, A.rp, A.ci, A.v, G.rp, G.ci, G.v, ld, meta.p);
      AMG_CHECK_LAUNCH();
    };
    if (mmax <= 4) {
      k_fsai_rows<4><<<ceil_div(n, TPB), TPB, 0, s>>>(n, A.rp, A.ci, A.v, G.rp, G.ci, G.v, meta.p);
    } else if (mmax <= 8) {
      k_fsai_rows<8><<<ceil_div(n, TPB), TPB, 0, s>>>(n, A.rp, A.ci, A.v, G.rp, G.ci, G.v, meta.p);
    } else if (mmax <= kThreadRows) {
      launch_thread(nullptr, n, mmax);
    } else {
      // rows of at most kThreadRows lower entries by the thread kernel, the
      // others by the warp kernel
      Buf<int> lsmall(m, n), llarge(m, n), nsl(m, 2);
      AMG_CUDA(cudaMemsetAsync(nsl.p, 0, 2 * sizeof(int), s));
      k_fsai_split<<<ceil_div(n, TPB), TPB, 0, s>>>(n, G.rp, kThreadRows, lsmall.p, nsl.p, llarge.p, nsl.p + 1);
      AMG_CHECK_LAUNCH();
      int hn[2];
      AMG_CUDA(cudaMemcpyAsync(hn, nsl.p, sizeof(hn), cudaMemcpyDeviceToHost, s));
      AMG_CUDA(cudaStreamSynchronize(s));
      if (hn[0] > 0) launch_thread(lsmall.p, hn[0], kThreadRows);
      const int nbig = hn[1];
      // slice per warp: ld * ld + 2 ld doubles (P_i's ints fit in the last ld)
      const size_t slice = ((size_t)mmax * mmax + 2 * (size_t)mmax) * sizeof(double);
      const int wpb = (int)std::min<size_t>(8, (size_t)(200 * 1024) / slice);
      if (wpb >= 1) {  // shared memory
        static std::atomic<unsigned long long> attr{0};
        ensure_smem_attr(k_fsai_warp<true>, 200 * 1024, attr);
        const int blocks = std::max(1, std::min(ceil_div(nbig, wpb), kNumSMs * 32));
        k_fsai_warp<true><<<blocks, wpb * 32, slice * wpb, s>>>(nbig, llarge.p, A.rp, A.ci, A.v, G.rp, G.ci, G.v,
                                                                 nullptr, mmax, blocks * wpb, meta.p);
      } else {  // global scratch
        const int64_t cap_warps = std::max<int64_t>(1, ((int64_t)256 << 20) / (int64_t)slice);
        const int warps = (int)std::min<int64_t>({(int64_t)std::max(nbig, 1), (int64_t)kNumSMs * 16, cap_warps});
        Buf<double> scr(m, slice / sizeof(double) * (size_t)warps);
        k_fsai_warp<false><<<ceil_div((int64_t)warps * 32, TPB), TPB, 0, s>>>(nbig, llarge.p, A.rp, A.ci, A.v,
                                                                             G.rp, G.ci, G.v, scr.p, mmax, warps,
                                                                             meta.p);
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

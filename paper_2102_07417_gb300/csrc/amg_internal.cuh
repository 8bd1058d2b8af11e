// Internal declarations of libamg (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "amg.h"

namespace amg {

constexpr int kMaxLevels = 40;
constexpr int kMaxDense = 4096;  // largest last level factorised densely
constexpr int kNumSMs = 152;     // GB300; grids below are multiples of this

void set_error(const char *fmt, ...);

// Thrown internally, converted to a status code at the C boundary.
struct Status {
  int code;
};

#define AMG_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      ::amg::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      throw ::amg::Status{AMG_ERR_CUDA};                                                     \
    }                                                                                        \
  } while (0)

// Raises `fn`'s dynamic shared-memory limit to `bytes` on the current device,
// once per device (bit d of `done` records device d).  Setting the attribute
// is idempotent, so two host threads racing on a device's first call both
// set it harmlessly; devices beyond 63 set it on every call.
template <typename F>
void ensure_smem_attr(F *fn, int bytes, std::atomic<unsigned long long> &done) {
  int dev = 0;
  AMG_CUDA(cudaGetDevice(&dev));
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return;
  AMG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.fetch_or(bit, std::memory_order_acq_rel);
}

extern std::atomic<long long> g_launches;
#define AMG_CHECK_LAUNCH()                                    \
  do {                                                        \
    ::amg::g_launches.fetch_add(1, std::memory_order_relaxed); \
    AMG_CUDA(cudaGetLastError());                             \
  } while (0)

// Device memory through the caller's allocator (or cudaMallocAsync).
struct Mem {
  amg_allocator alloc{};
  bool callbacks = false;
  cudaStream_t stream = nullptr;
  size_t live_bytes = 0;
  std::unordered_map<void *, size_t> live;  // every allocation not yet returned

  void *get(size_t bytes);   // throws Status{AMG_ERR_OOM} on failure
  void put(void *p, size_t bytes);
  void free_all();
  template <typename T>
  T *get_n(size_t n) {
    return static_cast<T *>(get(n * sizeof(T)));
  }
};

// A device buffer owned by a Mem, freed on destruction (used for temporaries).
template <typename T>
struct Buf {
  Mem *m = nullptr;
  T *p = nullptr;
  size_t n = 0;
  Buf() = default;
  Buf(Mem &mem, size_t count) : m(&mem), p(mem.get_n<T>(count)), n(count) {}
  Buf(const Buf &) = delete;
  Buf &operator=(const Buf &) = delete;
  Buf(Buf &&o) noexcept : m(o.m), p(o.p), n(o.n) { o.p = nullptr; }
  Buf &operator=(Buf &&o) noexcept {
    reset();
    m = o.m; p = o.p; n = o.n; o.p = nullptr;
    return *this;
  }
  ~Buf() { reset(); }
  void reset() {
    if (p && m) m->put(p, n * sizeof(T));
    p = nullptr;
    n = 0;
  }
  T *release() {
    T *q = p;
    p = nullptr;
    return q;
  }
};

// Row-to-lane mapping of the solve kernels: G lanes per row, transposed or vector form.
struct RowMap {
  int g = 1;
  bool tr = true;
};

// Sliced-ELLPACK copy of a CSR matrix for the solve kernels: slices of 32
// rows stored column-major (entry k of the slice's lane l at off[s] + 32 k + l),
// padded with value 0 at a column the row already uses; rows optionally permuted (sorted by length, longest
// first, within windows of 256 rows) so that a slice's rows have similar
// lengths and a warp issues one FMA per stored entry, not per padded one.
struct Sell {
  int nslices = 0;
  int64_t nent = 0;
  int *off = nullptr;             // [nslices + 1] entry offsets (multiples of 32)
  int *col = nullptr;             // [nent]
  double *v = nullptr;            // [nent] FP64 values (when needed)
  float *v32 = nullptr;           // FP32 values (FP32 modes)
  __nv_bfloat16 *v16 = nullptr;   // BF16 values (P and R in the BF16 ablation)
  float2 *vdf = nullptr;          // FP64 values as FP32 pairs hi + lo (level-0 A, batched FP32 modes)
  int *perm = nullptr;            // [n] row held by each slot; nullptr = identity
};

// CSR matrix on the device (int32 indices).  Value arrays for each storage type.
struct DCsr {
  int n = 0, ncols = 0;
  int64_t nnz = 0;
  int *rp = nullptr, *ci = nullptr;
  double *v = nullptr;           // FP64 master copy
  float *v32 = nullptr;          // FP32 copy (FP32 modes)
  __nv_bfloat16 *v16 = nullptr;  // BF16 copy (P and R in the BF16 ablation)
  RowMap map;    // solve kernels in the V-cycle precision
  RowMap map64;  // FP64 products with this matrix
  bool use_sell = false;  // solve kernels read `sell` instead of the CSR arrays
  Sell sell;
};

// Scalars of one PCG solve, resident on the device.
struct PcgScalars {
  double rho;     // (r_k, z_k)
  double alpha;   // rho / (p, q)
  double beta;
  double rr;      // (r, r)
  double bb;      // (b, b)
  double tol;     // rtol * ||b||
  double pq, rz, zq;
  int iters;
  int done;       // 1: converged or failed; every kernel of later iterations returns at once
  int status;     // AMG_OK, AMG_ERR_BREAKDOWN
  int maxit;
};

struct Level {
  DCsr A, P, R;   // P, R empty on the last level
  DCsr G, GT;     // FSAI smoother: G and omega G^T (empty with the Jacobi smoother and on the last level)
  int8_t *cf = nullptr;    // C/F of this level (export), nullptr on the last level
  double *wd = nullptr;    // omega / a_ii (FP64)
  float *wd32 = nullptr;   // omega / a_ii (FP32)
  // V-cycle work vectors (type per precision mode; only one set is allocated)
  void *y = nullptr, *s = nullptr, *r = nullptr, *z = nullptr, *w = nullptr;
};

// Process-wide per-launch event timing (amg_profile_enable), per kernel class
// and hierarchy level (index kMaxLevels: launches that belong to no level).
struct Profile {
  bool on = false;
  int only_kind = -1, only_level = -1;  // amg_profile_filter
  std::vector<cudaEvent_t> ev;  // pool of events, two per recorded launch
  std::vector<int> kind;        // kernel class * (kMaxLevels + 1) + level slot of each pair
  std::vector<double> bytes;    // algorithmic bytes of each recorded pair
  size_t used = 0;
  int64_t launches[AMG_K_COUNT][kMaxLevels + 1] = {};
  double ms[AMG_K_COUNT][kMaxLevels + 1] = {};
  double total_bytes[AMG_K_COUNT][kMaxLevels + 1] = {};
};
extern Profile g_prof;

// True when launches of kernel class `kind` would record events: graphs are
// captured only when none of their kernels would (events inside a captured
// graph would not time its replays).
inline bool prof_records(int kind) {
  return g_prof.on && (g_prof.only_kind < 0 || g_prof.only_kind == kind);
}
// Whether any solve-phase kernel class (AMG_K_SPMV_DOT .. AMG_K_SOLVE_OTHER)
// would record events.
inline bool prof_records_solve() {
  for (int k = AMG_K_SPMV_DOT; k <= AMG_K_SOLVE_OTHER; ++k)
    if (prof_records(k)) return true;
  return false;
}

// Brackets one kernel launch with two events when profiling is on.
struct ProfScope {
  size_t slot = (size_t)-1;
  cudaStream_t stream;
  ProfScope(cudaStream_t s, int kind, double bytes, int level = -1);
  ~ProfScope();
};
// Folds recorded event pairs into the totals; synchronises `s` first.
void prof_collect(cudaStream_t s);

}  // namespace amg

struct amg_hierarchy {
  amg::Mem mem;
  amg_params prm{};
  int nlevels = 0;
  amg::Level lev[amg::kMaxLevels];
  double *L = nullptr;     // dense Cholesky factor of the last level (row-major, lower)
  double *Linv = nullptr;  // its inverse (row-major, lower)
  int nL = 0;
  // PCG vectors (level 0, FP64)
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  amg::PcgScalars *sc = nullptr;   // device scalars
  double *hist = nullptr;          // device residual history
  int hist_cap = 0;
  double *partials = nullptr;      // per-block reduction partials (3 per block)
  unsigned int *counter = nullptr; // last-block tickets
  int *d_zero = nullptr;           // a device int that stays 0 ("never done")
  int *h_done = nullptr;           // mapped pinned host flag (written by the device)
  int *d_done = nullptr;           // its device alias
  cudaEvent_t iter_ev[2] = {nullptr, nullptr};
  // one PCG iteration captured as a CUDA graph (replayed on the solve's stream);
  // valid for the x and history buffers it was captured with
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t iter_exec = nullptr;
  const void *iter_x = nullptr, *iter_hist = nullptr;
  long long iter_launches = 0;
  // amg_vcycle_apply's kernels, captured for one (y, z) pair and replayed
  cudaGraphExec_t vc_exec = nullptr;
  const void *vc_y = nullptr, *vc_z = nullptr;
  long long vc_launches = 0;
  // dense operator of the V-cycle from level dense_level down (solve.cu), n x n
  // FP64 row-major with n = lev[dense_level].A.n; dense_level = -1: none
  int dense_level = -1;
  double *dense_op = nullptr;
  // double-float (FP32 pair) copy of level 0's sliced-ELLPACK values, built on
  // first use by a batched FP32-mode solve or slots object; df_mu serialises
  // its construction across host threads, df_ev marks its completion on the
  // hierarchy's stream (other streams wait on it before reading the copy)
  std::mutex df_mu;
  cudaEvent_t df_ev = nullptr;
  size_t bytes = 0;
};

namespace amg {

// set-up (setup.cu)
void build_hierarchy(amg_hierarchy *h, const amg_csr &A);
// solve (solve.cu)
void prepare_solve(amg_hierarchy *h);
int pcg_solve(amg_hierarchy *h, const double *b, double *x, double rtol, int maxit, int *iters, double *hist,
              int hist_cap);
void vcycle_apply(amg_hierarchy *h, const double *y, double *z);
// continuous batching slots (batch.cu): one resident n x K CG block whose
// columns are admitted, stepped and retired independently
struct SlotsBase {
  virtual ~SlotsBase() = default;
  virtual void admit(int j, const double *b) = 0;
  virtual void step() = 0;
  virtual void poll(int *state, int *iters) = 0;
  virtual void query(int *state, int *iters, long long *done, long long *issued) = 0;
  virtual void wait() = 0;
  virtual void retire(int j, double *x) = 0;
};
SlotsBase *make_slots(amg_hierarchy *h, int K, double rtol, int maxit, cudaStream_t s);
void slots_admit(SlotsBase *b, int j, const double *rhs);
void slots_step(SlotsBase *b);
void slots_poll(SlotsBase *b, int *state, int *iters);
void slots_query(SlotsBase *b, int *state, int *iters, long long *done, long long *issued);
void slots_wait(SlotsBase *b);
void slots_retire(SlotsBase *b, int j, double *x);
void slots_delete(SlotsBase *b);
// batched right-hand sides (batch.cu)
int pcg_solve_batch(amg_hierarchy *h, int k, const double *B, double *X, double rtol, int maxit, int *iters,
                    int *status, double *hist, int hist_cap);
void spmv_level(amg_hierarchy *h, int level, const double *x, double *y);
void release_solve(amg_hierarchy *h);

// FSAI factor G of level k and omega G^T (fsai.cu)
void build_fsai(amg_hierarchy *h, int k);
// R = P^T with rows sorted (setup.cu)
void csr_transpose(Mem &m, const DCsr &P, int ncols, DCsr &R);

// C = X Y with the canonical summation order (spgemm.cu); flags: device error
// flags; level: hierarchy level for the profiler.
void spgemm(Mem &m, int *flags, const DCsr &X, const DCsr &Y, int ncols, DCsr &C, int level);

// device-wide exclusive scan of n int32 counts into out[0..n] (out[n] = total); returns total
int64_t scan_counts(Mem &mem, const int *in, int *out, int n);
// the same scan without the read-back: *total_dev (device) receives the total
void scan_counts_async(Mem &mem, const int *in, int *out, int n, long long *total_dev);
// fails (AMG_ERR_UNSUPPORTED) on totals that do not fit int32 offsets
void check_scan_total(long long total);

inline int ceil_div(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }

}  // namespace amg

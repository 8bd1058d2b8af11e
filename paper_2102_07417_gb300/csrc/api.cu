// api.cu -- the C ABI of libamg (declared in include/amg.h): argument
// checks, allocation, error translation; the work is in setup.cu / solve.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstring>

#include "amg_internal.cuh"

namespace amg {

static thread_local char g_err[512] = "";
std::atomic<long long> g_launches{0};
Profile g_prof;

ProfScope::ProfScope(cudaStream_t s, int kind, double bytes, int level) : stream(s) {
  Profile &pr = g_prof;
  if (!pr.on) return;
  if (pr.only_kind >= 0 && (kind != pr.only_kind || (pr.only_level >= 0 && level != pr.only_level))) return;
  if (pr.used * 2 + 2 > pr.ev.size()) {
    const size_t add = std::max<size_t>(2048, pr.ev.size());
    for (size_t t = 0; t < add; ++t) {
      cudaEvent_t e;
      AMG_CUDA(cudaEventCreate(&e));
      pr.ev.push_back(e);
    }
  }
  slot = pr.used++;
  if (pr.kind.size() < pr.used) {
    pr.kind.resize(pr.used);
    pr.bytes.resize(pr.used);
  }
  pr.kind[slot] = kind * (kMaxLevels + 1) + ((level >= 0 && level < kMaxLevels) ? level : kMaxLevels);
  pr.bytes[slot] = bytes;
  AMG_CUDA(cudaEventRecord(pr.ev[2 * slot], s));
}

ProfScope::~ProfScope() {
  if (slot != (size_t)-1) cudaEventRecord(g_prof.ev[2 * slot + 1], stream);
}

void prof_collect(cudaStream_t s) {
  Profile &pr = g_prof;
  if (!pr.used) return;
  AMG_CUDA(cudaStreamSynchronize(s));
  for (size_t k = 0; k < pr.used; ++k) {
    float ms = 0.f;
    AMG_CUDA(cudaEventSynchronize(pr.ev[2 * k + 1]));
    AMG_CUDA(cudaEventElapsedTime(&ms, pr.ev[2 * k], pr.ev[2 * k + 1]));
    const int kind = pr.kind[k] / (kMaxLevels + 1), lvl = pr.kind[k] % (kMaxLevels + 1);
    pr.launches[kind][lvl] += 1;
    pr.ms[kind][lvl] += ms;
    pr.total_bytes[kind][lvl] += pr.bytes[k];
  }
  pr.used = 0;
}

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void *Mem::get(size_t bytes) {
  if (bytes == 0) bytes = 1;
  void *p = nullptr;
  if (callbacks) {
    p = alloc.alloc(bytes, stream, alloc.ctx);
  } else {
    if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  if (!p) {
    set_error("device allocation of %zu bytes failed", bytes);
    throw Status{AMG_ERR_OOM};
  }
  live[p] = bytes;
  live_bytes += bytes;
  return p;
}

void Mem::put(void *p, size_t) {
  if (!p) return;
  auto it = live.find(p);
  if (it == live.end()) return;
  const size_t bytes = it->second;
  live.erase(it);
  live_bytes -= bytes;
  if (callbacks) alloc.free(p, bytes, stream, alloc.ctx);
  else cudaFreeAsync(p, stream);
}

void Mem::free_all() {
  for (auto &kv : live) {
    if (callbacks) alloc.free(kv.first, kv.second, stream, alloc.ctx);
    else cudaFreeAsync(kv.first, stream);
  }
  live.clear();
  live_bytes = 0;
}

}  // namespace amg

using amg::Status;

#define AMG_GUARD_BEGIN try {
#define AMG_GUARD_END                 \
  }                                   \
  catch (const Status &st) {          \
    return st.code;                   \
  }                                   \
  catch (...) {                       \
    amg::set_error("internal error"); \
    return AMG_ERR_CUDA;              \
  }

static int bad(const char *msg) {
  amg::set_error("%s", msg);
  return AMG_ERR_INVALID_ARG;
}

extern "C" {

int amg_params_default(amg_params *p) {
  if (!p) return bad("params is NULL");
  p->theta = 0.25;
  p->seed = 0;
  p->max_coarse = 64;
  p->max_levels = 25;
  p->omega = 2.0 / 3.0;
  p->nu1 = 1;
  p->nu2 = 1;
  p->precision = AMG_PREC_FP64;
  p->block_size = 1;
  p->smoother = AMG_SMOOTH_JACOBI;
  p->interp = AMG_INTERP_DIRECT;
  return AMG_OK;
}

static int check_params(const amg_params &p) {
  if (!(p.theta > 0.0 && p.theta <= 1.0)) return bad("theta must be in (0, 1]");
  if (p.max_coarse < 1) return bad("max_coarse must be >= 1");
  if (p.max_levels < 1 || p.max_levels > amg::kMaxLevels) return bad("max_levels must be in 1..40");
  if (!(p.omega > 0.0 && p.omega < 2.0)) return bad("omega must be in (0, 2)");
  if (p.nu1 < 0 || p.nu1 > 8 || p.nu2 < 0 || p.nu2 > 8) return bad("nu1, nu2 must be in 0..8");
  if (p.precision < AMG_PREC_FP64 || p.precision > AMG_PREC_FP32_BF16PR) return bad("unknown precision mode");
  if (p.block_size < 1 || p.block_size > 8) return bad("block_size must be in 1..8");
  if (p.smoother != AMG_SMOOTH_JACOBI && p.smoother != AMG_SMOOTH_FSAI) return bad("unknown smoother");
  if (p.interp != AMG_INTERP_DIRECT && p.interp != AMG_INTERP_EXT) return bad("unknown interpolation");
  if (p.interp == AMG_INTERP_EXT && p.block_size != 1) return bad("extended+i interpolation needs block_size 1");
  return AMG_OK;
}

void amg_free(amg_hierarchy *h) {
  if (!h) return;
  amg::release_solve(h);
  h->mem.free_all();
  delete h;
}

int amg_setup(const amg_csr *A, const amg_params *params, const amg_allocator *alloc, void *stream,
              amg_hierarchy **out) {
  if (!out) return bad("out is NULL");
  *out = nullptr;
  if (!A || !A->rowptr || (A->nnz > 0 && (!A->colidx || !A->val))) return bad("A or its arrays are NULL");
  if (A->n < 1 || A->nnz < A->n) return bad("n must be >= 1 and every row needs its diagonal");
  amg_params prm;
  if (params) prm = *params;
  else amg_params_default(&prm);
  int st = check_params(prm);
  if (st) return st;
  if (A->n % prm.block_size) return bad("n must be a multiple of block_size");
  if (alloc && ((alloc->alloc == nullptr) != (alloc->free == nullptr))) return bad("allocator needs both alloc and free");
  amg_hierarchy *h = new amg_hierarchy();
  h->prm = prm;
  h->mem.stream = static_cast<cudaStream_t>(stream);
  if (alloc && alloc->alloc) {
    h->mem.alloc = *alloc;
    h->mem.callbacks = true;
  }
  try {
    amg::build_hierarchy(h, *A);
    amg::prepare_solve(h);
    AMG_CUDA(cudaStreamSynchronize(h->mem.stream));
    amg::prof_collect(h->mem.stream);
  } catch (const Status &e) {
    cudaStreamSynchronize(h->mem.stream);
    amg_free(h);
    return e.code;
  } catch (...) {
    amg::set_error("internal error in set-up");
    amg_free(h);
    return AMG_ERR_CUDA;
  }
  h->bytes = h->mem.live_bytes;
  *out = h;
  return AMG_OK;
}

int amg_pcg_solve(amg_hierarchy *h, const double *b, double *x, double rtol, int32_t maxit, void *stream,
                  int32_t *iters, double *res_hist, int32_t hist_cap) {
  if (!h || !b || !x) return bad("NULL argument");
  if (!(rtol > 0.0) || maxit < 1) return bad("rtol must be > 0 and maxit >= 1");
  if (res_hist && hist_cap < 0) return bad("hist_cap < 0");
  AMG_GUARD_BEGIN
  h->mem.stream = static_cast<cudaStream_t>(stream);
  int it = 0;
  const int st = amg::pcg_solve(h, b, x, rtol, maxit, &it, res_hist, res_hist ? hist_cap : 0);
  if (iters) *iters = it;
  return st;
  AMG_GUARD_END
}

int amg_pcg_solve_batch(amg_hierarchy *h, int32_t k, const double *B, double *X, double rtol, int32_t maxit,
                        void *stream, int32_t *iters, int32_t *status, double *res_hist, int32_t hist_cap) {
  if (!h || !B || !X) return bad("NULL argument");
  if (k < 1 || k > 32) return bad("k must be in 1..32");
  if (!(rtol > 0.0) || maxit < 1) return bad("rtol must be > 0 and maxit >= 1");
  if (res_hist && hist_cap < 0) return bad("hist_cap < 0");
  AMG_GUARD_BEGIN
  h->mem.stream = static_cast<cudaStream_t>(stream);
  return amg::pcg_solve_batch(h, k, B, X, rtol, maxit, iters, status, res_hist, res_hist ? hist_cap : 0);
  AMG_GUARD_END
}

struct amg_slots {
  amg_hierarchy *h;
  amg::SlotsBase *impl;
  int32_t capacity;
};

int amg_slots_create(amg_hierarchy *h, int32_t capacity, double rtol, int32_t maxit, void *stream, amg_slots **out) {
  if (!out) return bad("NULL argument");
  *out = nullptr;
  if (!h) return bad("NULL argument");
  if (capacity < 1 || capacity > 32) return bad("capacity must be in 1..32");
  if (!(rtol > 0.0) || maxit < 1) return bad("rtol must be > 0 and maxit >= 1");
  AMG_GUARD_BEGIN
  amg_slots *s = new amg_slots{h, nullptr, capacity};
  try {
    s->impl = amg::make_slots(h, capacity, rtol, maxit, static_cast<cudaStream_t>(stream));
  } catch (...) {
    delete s;
    throw;
  }
  *out = s;
  return AMG_OK;
  AMG_GUARD_END
}

int amg_slots_admit(amg_slots *s, int32_t slot, const double *b) {
  if (!s || !b) return bad("NULL argument");
  if (slot < 0 || slot >= s->capacity) return bad("slot out of range");
  AMG_GUARD_BEGIN
  amg::slots_admit(s->impl, slot, b);
  return AMG_OK;
  AMG_GUARD_END
}

int amg_slots_step(amg_slots *s) {
  if (!s) return bad("NULL argument");
  AMG_GUARD_BEGIN
  amg::slots_step(s->impl);
  return AMG_OK;
  AMG_GUARD_END
}

int amg_slots_poll(amg_slots *s, int32_t *state, int32_t *iters) {
  if (!s) return bad("NULL argument");
  AMG_GUARD_BEGIN
  amg::slots_poll(s->impl, state, iters);
  return AMG_OK;
  AMG_GUARD_END
}

int amg_slots_query(amg_slots *s, int32_t *state, int32_t *iters, int64_t *steps_done, int64_t *steps_issued) {
  if (!s) return bad("NULL argument");
  AMG_GUARD_BEGIN
  long long d = 0, i = 0;
  amg::slots_query(s->impl, state, iters, &d, &i);
  if (steps_done) *steps_done = d;
  if (steps_issued) *steps_issued = i;
  return AMG_OK;
  AMG_GUARD_END
}

int amg_slots_wait(amg_slots *s) {
  if (!s) return bad("NULL argument");
  AMG_GUARD_BEGIN
  amg::slots_wait(s->impl);
  return AMG_OK;
  AMG_GUARD_END
}

int amg_slots_retire(amg_slots *s, int32_t slot, double *x) {
  if (!s) return bad("NULL argument");
  if (slot < 0 || slot >= s->capacity) return bad("slot out of range");
  AMG_GUARD_BEGIN
  amg::slots_retire(s->impl, slot, x);
  return AMG_OK;
  AMG_GUARD_END
}

void amg_slots_free(amg_slots *s) {
  if (!s) return;
  try {
    amg::slots_delete(s->impl);
  } catch (...) {
  }
  delete s;
}

int amg_vcycle_apply(amg_hierarchy *h, const double *y, double *z, void *stream) {
  if (!h || !y || !z) return bad("NULL argument");
  AMG_GUARD_BEGIN
  h->mem.stream = static_cast<cudaStream_t>(stream);
  amg::vcycle_apply(h, y, z);
  return AMG_OK;
  AMG_GUARD_END
}

int amg_spmv(amg_hierarchy *h, int32_t level, const double *x, double *y, void *stream) {
  if (!h || !x || !y) return bad("NULL argument");
  if (level < 0 || level >= h->nlevels) return bad("level out of range");
  AMG_GUARD_BEGIN
  h->mem.stream = static_cast<cudaStream_t>(stream);
  amg::spmv_level(h, level, x, y);
  amg::prof_collect(h->mem.stream);
  return AMG_OK;
  AMG_GUARD_END
}

int amg_solve(const amg_csr *A, const double *b, double *x, const amg_params *params, double rtol, int32_t maxit,
              const amg_allocator *alloc, void *stream, amg_result *res) {
  if (!A || !b || !x) return bad("NULL argument");
  if (!(rtol > 0.0) || maxit < 1) return bad("rtol must be > 0 and maxit >= 1");
  using clk = std::chrono::steady_clock;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const auto t0 = clk::now();
  amg_hierarchy *h = nullptr;
  int st = amg_setup(A, params, alloc, stream, &h);
  if (st) return st;
  const auto t1 = clk::now();
  AMG_GUARD_BEGIN
  const int n = A->n;
  const double *bd = b;
  double *xd = x;
  if (!A->on_device) {
    bd = h->mem.get_n<double>(n);
    xd = h->mem.get_n<double>(n);
    AMG_CUDA(cudaMemcpyAsync(const_cast<double *>(bd), b, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    AMG_CUDA(cudaMemcpyAsync(xd, x, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  }
  int it = 0;
  st = amg::pcg_solve(h, bd, xd, rtol, maxit, &it, nullptr, 0);
  double rr = 0.0;
  AMG_CUDA(cudaMemcpyAsync(&rr, &h->sc->rr, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (!A->on_device) AMG_CUDA(cudaMemcpyAsync(x, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  const auto t2 = clk::now();
  if (res) {
    res->iters = it;
    res->nlevels = h->nlevels;
    res->final_residual = std::sqrt(rr);
    res->setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    res->solve_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
  }
  amg_free(h);
  return st;
  }
  catch (const Status &e) {
    amg_free(h);
    return e.code;
  }
  catch (...) {
    amg_free(h);
    amg::set_error("internal error");
    return AMG_ERR_CUDA;
  }
}

int amg_hierarchy_info(const amg_hierarchy *h, int32_t *nlevels, int32_t cap, int64_t *n_k, int64_t *nnz_k,
                       int64_t *nnzP_k, double *cgd, double *cop) {
  if (!h) return bad("NULL hierarchy");
  if (nlevels) *nlevels = h->nlevels;
  double sn = 0, sz = 0;
  for (int k = 0; k < h->nlevels; ++k) {
    const amg::Level &L = h->lev[k];
    sn += L.A.n;
    sz += (double)L.A.nnz;
    if (k < cap) {
      if (n_k) n_k[k] = L.A.n;
      if (nnz_k) nnz_k[k] = L.A.nnz;
      if (nnzP_k) nnzP_k[k] = (k < h->nlevels - 1) ? L.P.nnz : 0;
    }
  }
  if (cgd) *cgd = sn / h->lev[0].A.n;
  if (cop) *cop = sz / (double)h->lev[0].A.nnz;
  return AMG_OK;
}

int amg_hierarchy_export(const amg_hierarchy *h, int32_t level, int8_t *cf, int32_t *A_rowptr, int32_t *A_col,
                         double *A_val, int32_t *P_rowptr, int32_t *P_col, double *P_val) {
  if (!h) return bad("NULL hierarchy");
  if (level < 0 || level >= h->nlevels) return bad("level out of range");
  AMG_GUARD_BEGIN
  cudaStream_t s = h->mem.stream;
  const amg::Level &L = h->lev[level];
  const int n = L.A.n;
  const bool last = level == h->nlevels - 1;
  auto d2h = [&](void *dst, const void *src, size_t bytes) {
    if (dst && src && bytes) AMG_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
  };
  if (cf) {
    if (last || !L.cf) std::memset(cf, 0, n);
    else d2h(cf, L.cf, n);
  }
  d2h(A_rowptr, L.A.rp, sizeof(int) * ((size_t)n + 1));
  d2h(A_col, L.A.ci, sizeof(int) * (size_t)L.A.nnz);
  d2h(A_val, L.A.v, sizeof(double) * (size_t)L.A.nnz);
  if (!last) {
    d2h(P_rowptr, L.P.rp, sizeof(int) * ((size_t)n + 1));
    d2h(P_col, L.P.ci, sizeof(int) * (size_t)L.P.nnz);
    d2h(P_val, L.P.v, sizeof(double) * (size_t)L.P.nnz);
  }
  AMG_CUDA(cudaStreamSynchronize(s));
  return AMG_OK;
  AMG_GUARD_END
}

int amg_hierarchy_export_fsai(const amg_hierarchy *h, int32_t level, int64_t *nnz, int32_t *G_rowptr,
                              int32_t *G_col, double *G_val) {
  if (!h) return bad("NULL hierarchy");
  if (level < 0 || level >= h->nlevels) return bad("level out of range");
  AMG_GUARD_BEGIN
  const amg::DCsr &G = h->lev[level].G;
  if (nnz) *nnz = G.rp ? G.nnz : 0;
  if (!G.rp) return AMG_OK;
  cudaStream_t s = h->mem.stream;
  auto d2h = [&](void *dst, const void *src, size_t bytes) {
    if (dst && src && bytes) AMG_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
  };
  d2h(G_rowptr, G.rp, sizeof(int) * ((size_t)G.n + 1));
  d2h(G_col, G.ci, sizeof(int) * (size_t)G.nnz);
  d2h(G_val, G.v, sizeof(double) * (size_t)G.nnz);
  AMG_CUDA(cudaStreamSynchronize(s));
  return AMG_OK;
  AMG_GUARD_END
}

size_t amg_hierarchy_bytes(const amg_hierarchy *h) { return h ? h->mem.live_bytes : 0; }

int amg_profile_enable(int32_t on) {
  amg::Profile &pr = amg::g_prof;
  pr.on = on != 0;
  if (on) {
    for (int k = 0; k < AMG_K_COUNT; ++k)
      for (int l = 0; l <= amg::kMaxLevels; ++l) {
        pr.launches[k][l] = 0;
        pr.ms[k][l] = 0.0;
        pr.total_bytes[k][l] = 0.0;
      }
    pr.used = 0;
  }
  return AMG_OK;
}

int amg_profile_filter(int32_t kernel, int32_t level) {
  if (kernel < -1 || kernel >= AMG_K_COUNT) return bad("kernel class out of range");
  if (level < -1 || level >= amg::kMaxLevels) return bad("level out of range");
  amg::g_prof.only_kind = kernel;
  amg::g_prof.only_level = level;
  return AMG_OK;
}

int amg_profile_read(int32_t kernel, int32_t level, int64_t *launches, double *ms, double *bytes) {
  if (kernel < 0 || kernel >= AMG_K_COUNT) return bad("kernel class out of range");
  if (level < -1 || level >= amg::kMaxLevels) return bad("level out of range");
  const amg::Profile &pr = amg::g_prof;
  int64_t n = 0;
  double t = 0.0, b = 0.0;
  for (int l = 0; l <= amg::kMaxLevels; ++l) {
    if (level >= 0 && l != level) continue;
    n += pr.launches[kernel][l];
    t += pr.ms[kernel][l];
    b += pr.total_bytes[kernel][l];
  }
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (bytes) *bytes = b;
  return AMG_OK;
}

int64_t amg_launch_count(void) { return amg::g_launches.load(); }

const char *amg_status_string(int status) {
  switch (status) {
    case AMG_OK: return "ok";
    case AMG_ERR_INVALID_ARG: return "invalid argument";
    case AMG_ERR_NOT_SPD: return "matrix is not symmetric positive definite";
    case AMG_ERR_BREAKDOWN: return "CG breakdown";
    case AMG_ERR_NO_CONVERGENCE: return "no convergence within maxit";
    case AMG_ERR_SETUP: return "coarsening failed";
    case AMG_ERR_OOM: return "out of device memory";
    case AMG_ERR_CUDA: return "CUDA error";
    case AMG_ERR_TIMEOUT: return "device wait timed out";
    case AMG_ERR_UNSUPPORTED: return "unsupported size or option";
    default: return "unknown status";
  }
}

const char *amg_last_error(void) { return amg::g_err; }

}  // extern "C"

// noalloc.cu -- amg_spmv_dot_noalloc: q = A p and (p, q) in one pass without
// allocating any device memory.
//
// This is the fused sparse matrix-vector product + dot product of the PCG
// loop (the same arithmetic as the solver's own kernel), packaged for callers
// that cannot allocate device memory at the point where they need it.  Its
// only scratch -- one partial sum per thread block and a ticket counter that
// tells the last block to finish the sum -- lives in the file-scope array
// below, which the CUDA runtime places in device memory when the library's
// module is loaded, once per device, and which stays there until the process
// exits.  The array is shared by every call on a device, so calls that
// overlap on the GPU (e.g. on two streams at once) race on it and must be
// serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "amg_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kRowsPerBlock = 8192;  // 32 rows per thread
constexpr int kMaxBlocks = 2048;     // partial-sum slots in the scratch array
constexpr long long kMaxRows = (long long)kRowsPerBlock * kMaxBlocks;  // 16,777,216 rows
constexpr size_t kTicketOffset = kMaxBlocks * sizeof(double);
constexpr size_t kScratchBytes = kTicketOffset + 256;  // 16 KiB of partials + the ticket
constexpr int kMaxDevices = 64;

// The scratch: [0, kTicketOffset) block partial sums (doubles), then the
// ticket counter (unsigned int).  A name in host code only stands for the
// symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__global__ void __launch_bounds__(kThreads) k_spmv_dot_noalloc(int n, const int *__restrict__ rp,
                                                               const int *__restrict__ ci,
                                                               const double *__restrict__ a,
                                                               const double *__restrict__ p, double *__restrict__ q,
                                                               double *__restrict__ pq, unsigned char *scratch) {
  double *partial = reinterpret_cast<double *>(scratch);
  unsigned int *ticket = reinterpret_cast<unsigned int *>(scratch + kTicketOffset);
  __shared__ double red[kThreads / 32];
  __shared__ bool last;
  const int row0 = blockIdx.x * kRowsPerBlock;
  const int row1 = min(n, row0 + kRowsPerBlock);
  double v = 0.0;
  for (int i = row0 + threadIdx.x; i < row1; i += blockDim.x) {
    double acc = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) acc = fma(__ldg(a + k), __ldg(p + ci[k]), acc);
    q[i] = acc;
    v = fma(p[i], acc, v);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) s += red[k];
    partial[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(&partial[b]);
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __syncthreads();
  if (lane == 0) red[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += red[k];
    *pq = t;
    *ticket = 0u;
  }
}

std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context id the address belongs to (0: unknown)

// Id of the calling thread's current CUDA context (0 when none is current or
// the driver does not report it).  The driver entry points are looked up
// through the runtime, so the library keeps no link-time dependency on the
// driver library.
unsigned long long current_context_id() {
  typedef int (*get_current_t)(void **);
  typedef int (*get_id_t)(void *, unsigned long long *);
  static get_current_t get_current = nullptr;
  static get_id_t get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr, *g = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<get_current_t>(f);
      get_id = reinterpret_cast<get_id_t>(g);
    }
  });
  if (!get_current || !get_id) return 0;
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on the current device, looked up on the
// first call on each device and again whenever the device's context has
// changed since (a cudaDeviceReset unloads the module, and the address found
// before it is no longer valid); when the context id cannot be read, it is
// looked up on every call.
int scratch_on_current_device(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    amg::set_error("cudaGetDevice failed: %s", cudaGetErrorString(e));
    return AMG_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    amg::set_error("device ordinal %d beyond the %d devices this entry point tracks", dev, kMaxDevices);
    return AMG_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_ptr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      amg::set_error("cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
      return AMG_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char *>(ptr);
    g_scratch_ctx[dev] = current_context_id();  // the lookup made the context current if it was not
  }
  *out = g_scratch_ptr[dev];
  return AMG_OK;
}

}  // namespace

extern "C" int amg_spmv_dot_noalloc(int32_t n, int32_t nnz, const int32_t *rowptr, const int32_t *colidx,
                                    const double *val, const double *p, double *q, double *pq, void *stream) {
  if (!rowptr || !p || !q || !pq || (nnz > 0 && (!colidx || !val))) {
    amg::set_error("amg_spmv_dot_noalloc: NULL argument");
    return AMG_ERR_INVALID_ARG;
  }
  if (n < 1 || nnz < 0) {
    amg::set_error("amg_spmv_dot_noalloc: n must be >= 1 and nnz >= 0");
    return AMG_ERR_INVALID_ARG;
  }
  if ((long long)n > kMaxRows) {
    amg::set_error("amg_spmv_dot_noalloc: n = %d exceeds the limit of %lld rows set by its fixed scratch array",
                   n, kMaxRows);
    return AMG_ERR_UNSUPPORTED;
  }
  unsigned char *scratch = nullptr;
  int st = scratch_on_current_device(&scratch);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(scratch + kTicketOffset, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) {
    amg::set_error("amg_spmv_dot_noalloc: clearing the ticket failed: %s", cudaGetErrorString(e));
    return AMG_ERR_CUDA;
  }
  const int blocks = (int)((n + (long long)kRowsPerBlock - 1) / kRowsPerBlock);
  k_spmv_dot_noalloc<<<blocks, kThreads, 0, s>>>(n, rowptr, colidx, val, p, q, pq, scratch);
  amg::g_launches.fetch_add(1, std::memory_order_relaxed);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    amg::set_error("amg_spmv_dot_noalloc: launch failed: %s", cudaGetErrorString(e));
    return AMG_ERR_CUDA;
  }
  return AMG_OK;
}

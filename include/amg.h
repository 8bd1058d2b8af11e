/*
 * amg.h -- C ABI of libamg: classical-AMG-preconditioned conjugate gradients
 * on one GB300 GPU (method of Isotton, Frigo, Spiezia & Janna, "Chronos: a
 * general purpose classical AMG solver for High Performance Computing",
 * arXiv 2102.07417).
 *
 * Problem statement (Sec. 1, Eq. linSys): solve A x = b for a sparse
 * symmetric positive definite A.  The preconditioner is one V-cycle
 * (Algorithm 2) over a classical AMG hierarchy built by Algorithm 1; the
 * Krylov solver is PCG with x0 given (zero in every benchmark) and the
 * stopping rule ||r_k||_2 < rtol * ||b||_2 on the recursively updated
 * residual (Sec. 4).  The solver interface mirrors the paper's LinSolver
 * (Sec. 3.1): a preconditioner, the system, a right-hand side and an
 * optional initial solution.
 *
 * Conventions shared by every entry point:
 *   - Return value: AMG_OK (0) or a negative AMG_ERR_* code;
 *     amg_status_string() names it and amg_last_error() gives detail.
 *   - Streams are passed as `void *` holding a cudaStream_t (NULL = the
 *     legacy default stream).  Work is enqueued on that stream.
 *   - Indices are int32 (4-byte local numbering, Sec. 3.2); values FP64.
 *   - The caller owns every buffer it passes; the library copies what it
 *     keeps.  The hierarchy owns its device memory until amg_free().
 *   - Device pointers must point to memory of the current CUDA device.
 *   - A hierarchy is not thread-safe: one host thread drives it at a time.
 */
#ifndef AMG_H
#define AMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ */
/* Status codes                                                         */
/* ------------------------------------------------------------------ */
#define AMG_OK 0
#define AMG_ERR_INVALID_ARG (-1)    /* malformed CSR, bad parameter, NULL pointer */
#define AMG_ERR_NOT_SPD (-2)        /* non-positive diagonal or Cholesky pivot */
#define AMG_ERR_BREAKDOWN (-3)      /* CG breakdown: (p, A p) <= 0 or NaN */
#define AMG_ERR_NO_CONVERGENCE (-4) /* maxit reached; x holds the last iterate */
#define AMG_ERR_SETUP (-5)          /* coarsening stalled above the dense-solve limit */
#define AMG_ERR_OOM (-6)            /* allocation failed (allocator returned NULL) */
#define AMG_ERR_CUDA (-7)           /* a CUDA runtime call failed */
#define AMG_ERR_TIMEOUT (-8)        /* a bounded device-side wait ran out */
#define AMG_ERR_UNSUPPORTED (-9)    /* size beyond a documented limit */

/* Smoothers of the V-cycle: S = I - omega M^-1 A (Eq. smoother). */
#define AMG_SMOOTH_JACOBI 0 /* M = D, damped Jacobi */
#define AMG_SMOOTH_FSAI 1   /* M^-1 = G^T G, G lower triangular (Eq. smo), static pattern lower(A_k) */

/* Interpolation of the set-up (Sec. 2.3). */
#define AMG_INTERP_DIRECT 0 /* direct (distance-one) interpolation */
#define AMG_INTERP_EXT 1    /* extended+i (distance two): interpolatory set C_i^S plus the strong C
                             * neighbours of i's strong F neighbours; scalar problems only */

/* Precision modes of the solve phase (the set-up is always FP64). */
#define AMG_PREC_FP64 0        /* hierarchy and V-cycle in FP64 */
#define AMG_PREC_FP32 1        /* hierarchy stored and V-cycle run in FP32, outer PCG FP64, flexible beta */
#define AMG_PREC_FP32_BF16PR 2 /* as FP32, with P and R stored in BF16 (FP32 accumulation) */

/* Opaque hierarchy (Algorithm 1's levels A_k, P_k, R_k = P_k^T, D_k, L). */
typedef struct amg_hierarchy amg_hierarchy;

/* Optional device allocator (e.g. a PyTorch caching allocator).
 * alloc(bytes, stream, ctx) returns device memory usable in stream order on
 * `stream`, or NULL on failure; free(ptr, bytes, stream, ctx) releases it.
 * A NULL allocator pointer, or NULL alloc/free members, selects
 * cudaMallocAsync / cudaFreeAsync on the call's stream. */
typedef void *(*amg_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*amg_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
typedef struct {
  amg_alloc_fn alloc;
  amg_free_fn free;
  void *ctx;
} amg_allocator;

/* Square sparse matrix in CSR (Sec. 3.2 CSRMAT).  rowptr[n+1] starting at
 * 0; colidx[nnz] strictly ascending within each row and in [0, n); val[nnz],
 * every value finite (a NaN or an infinity gives AMG_ERR_INVALID_ARG).
 * The pattern must be structurally symmetric and every row must hold a
 * positive diagonal entry.  on_device = 1: the three arrays are device
 * pointers; 0: host pointers. */
typedef struct {
  int32_t n;
  int32_t nnz;
  const int32_t *rowptr;
  const int32_t *colidx;
  const double *val;
  int32_t on_device;
} amg_csr;

/* Set-up and cycle parameters (Sec. 2; Algorithm 1 and 2). */
typedef struct {
  double theta;       /* strength threshold of the classical measure (Eq. cla filter), (0, 1]; 0.25 */
  uint64_t seed;      /* seed of the counter-based SplitMix64 stream of the PMIS measures; 0 */
  int32_t max_coarse; /* a level with at most this many rows is factorised densely; 64 */
  int32_t max_levels; /* hard cap on the number of levels, 1..40; 25 */
  double omega;       /* Jacobi damping of the smoother S = I - omega D^-1 A (Eq. smoother); 2/3 */
  int32_t nu1, nu2;   /* pre- and post-smoothing steps (Eq. twoGridOp), 0..8 each; 1, 1 */
  int32_t precision;  /* AMG_PREC_*; AMG_PREC_FP64 */
  int32_t block_size; /* unknowns per node, 1..8; 1.  bs > 1 (systems such as elasticity): the
                       * unknowns are node-major (unknown i is component i % bs of node i / bs),
                       * every coupled node pair must be stored as a full bs x bs block
                       * (explicit zeros allowed; else AMG_ERR_INVALID_ARG) and n % bs == 0.
                       * Strength is nodal: s_IJ = ||A_IJ||_F / sqrt(||A_II||_F ||A_JJ||_F)
                       * (the block form of Eq. sco), J strong for I iff s_IJ >= theta *
                       * max_{K != I} s_IK; PMIS runs on the node graph; every unknown takes its
                       * node's C/F label; interpolation is unknown-wise (direct interpolation
                       * over the same-component couplings only). */
  int32_t smoother;   /* AMG_SMOOTH_*; AMG_SMOOTH_JACOBI.  AMG_SMOOTH_FSAI: the factored sparse
                       * approximate inverse M^-1 = G^T G of Sec. 2.1 with G on the static pattern
                       * of the lower triangle of each A_k (the paper's aFSAI chooses the pattern
                       * adaptively); row i of G solves A[P_i, P_i] g = e_i on P_i = {j <= i :
                       * a_ij stored}, scaled to (G A G^T)_ii = 1.  A smoothing step costs one
                       * product with A, G and G^T.  omega must keep omega rho(G^T G A) < 2
                       * (rho ~ 1.37 on 3-D Poisson: omega = 1 is a good choice).  Single
                       * right-hand-side solves and V-cycles only: amg_pcg_solve_batch and
                       * amg_slots_create return AMG_ERR_UNSUPPORTED on such a hierarchy. */
  int32_t interp;     /* AMG_INTERP_*; AMG_INTERP_DIRECT.  AMG_INTERP_EXT: the extended+i weights of
                       * Sec. 2.3, w_ij = -(a_ij + sum_{k in F_i^S} a_ik abar_kj / d_k) / at_ii with
                       * d_k = sum of abar_kl over l in Chat_i u {i}, evaluated in a fixed order so the
                       * hierarchy is reproducible bit for bit; needs block_size = 1
                       * (AMG_ERR_INVALID_ARG otherwise); a zero modified diagonal at_ii gives
                       * AMG_ERR_SETUP; a row with more interpolatory candidates than the per-warp
                       * shared-memory set holds (~6000) gives AMG_ERR_UNSUPPORTED. */
} amg_params;

/* Fills *p with the defaults above.  Returns AMG_ERR_INVALID_ARG if p is NULL. */
int amg_params_default(amg_params *p);

/* Algorithm 1 (AMG_SetUp), recursively on the GPU: strength of connection
 * (Eq. cla, read as Ruge-Stueben), PMIS C/F splitting (Sec. 2.2), direct
 * interpolation P = [W; I] (Eq. prolOperator), R = P^T and the Galerkin
 * product A_{k+1} = R (A_k P) (Eq. AcDef) as a GPU SpGEMM whose summation
 * order is canonical (the hierarchy is reproducible bit for bit), until a
 * level has at most max_coarse rows, coarsening stalls (n_{k+1} = 0 or
 * n_{k+1} > 0.9 n_k), or max_levels is reached; the last level is factorised
 * by a dense Cholesky A_L = L L^T (at most 4096 rows, else AMG_ERR_SETUP).
 * A is copied; the caller may free it on return.  `alloc` may be NULL.
 * Synchronises `stream` (coarse sizes are needed on the host).
 * On error *out is NULL and nothing is leaked. */
int amg_setup(const amg_csr *A, const amg_params *params, const amg_allocator *alloc, void *stream,
              amg_hierarchy **out);

/* PCG preconditioned by one V-cycle (Algorithm 2) per iteration.
 * b, x: device arrays of n doubles; x holds x0 on entry and the solution
 * (or the last iterate) on return.  Stops when ||r_k||_2 < rtol ||b||_2
 * (recursive residual, Sec. 4) or after maxit iterations.  In the FP32
 * precision modes the flexible (Polak-Ribiere) beta is used.
 * iters (may be NULL) receives the iteration count; res_hist (host, may be
 * NULL) receives ||r_k||_2 for k = 0..min(iters, hist_cap-1).
 * Returns when the solve has finished (the stream is synchronised).
 * AMG_ERR_NO_CONVERGENCE / AMG_ERR_BREAKDOWN leave the last iterate in x. */
int amg_pcg_solve(amg_hierarchy *h, const double *b, double *x, double rtol, int32_t maxit, void *stream,
                  int32_t *iters, double *res_hist, int32_t hist_cap);

/* PCG on k right-hand sides at once (Sec. 3.1: dense blocks stored row-wise
 * for multiple right-hand sides).  B, X: device arrays of n x k doubles,
 * row-major (entry (i, j) at i * k + j), 1 <= k <= 32; X holds the initial
 * guesses on entry and the solutions on return.  Every column runs its own CG
 * recurrence (its own alpha, beta, rho and stopping test ||r_j|| < rtol
 * ||b_j||) while sharing each sparse product and V-cycle with the others (one
 * SpMM per product); a converged column is frozen while the rest continue.
 * iters[k], status[k] (host, may be NULL) receive each column's iteration
 * count and status; res_hist (host, may be NULL) receives ||r_j|| after
 * iteration t at res_hist[t * k + j] for t < hist_cap.  Returns AMG_OK when
 * every column converged, else the first column error met.  Synchronises.
 * The last level must satisfy 16 * n_L * k <= 200 KiB (AMG_ERR_UNSUPPORTED). */
int amg_pcg_solve_batch(amg_hierarchy *h, int32_t k, const double *B, double *X, double rtol, int32_t maxit,
                        void *stream, int32_t *iters, int32_t *status, double *res_hist, int32_t hist_cap);

/* Continuous batching (Sec. 3.1's row-wise dense blocks, used as a resident
 * batch whose columns change while it runs).  A slots object holds an n x
 * capacity block of CG vectors on hierarchy h (1 <= capacity <= 32, the last
 * level bounded as for amg_pcg_solve_batch) and runs on `stream`; every call
 * below is stream-ordered on it.  Each column ("slot") is one request:
 *   amg_slots_admit  starts PCG on slot `slot` with x0 = 0 and right-hand side
 *                    b (device, n doubles; read before the call's work ends,
 *                    i.e. the caller keeps b alive until the next poll);
 *   amg_slots_step   runs one PCG iteration of every running slot (one SpMM,
 *                    one update, one V-cycle, one direction update shared by
 *                    all of them).  A slot admitted since the last step uses
 *                    it to form z = M r and p = z (alpha = beta = 0), the same
 *                    arithmetic as the first step of amg_pcg_solve_batch.
 *                    Converged and free slots are frozen;
 *   amg_slots_poll   synchronises the stream and reports per slot (host
 *                    arrays of capacity, either may be NULL): state 0 free,
 *                    1 running, 2 converged (||r_j|| < rtol ||b_j||), or a
 *                    negative status (AMG_ERR_NO_CONVERGENCE after maxit
 *                    iterations, AMG_ERR_BREAKDOWN); iters = CG iterations;
 *   amg_slots_query  the same report without waiting, from the newest step
 *                    that has finished on the device (a snapshot of the state
 *                    is copied to pinned host memory at the end of every
 *                    step); a slot admitted after that step reads as running.
 *                    steps_done / steps_issued (may be NULL) count the steps
 *                    finished and launched, so a caller can keep a bounded
 *                    number in flight;
 *   amg_slots_wait   blocks until the oldest step still in flight finishes
 *                    (returns at once when none is);
 *   amg_slots_retire copies the slot's x into `x` (device, n doubles; NULL
 *                    discards it) and frees the slot;
 *   amg_slots_free   waits for the stream and releases the object (before
 *                    amg_free(h)).
 * Memory comes from h's allocator.  A slots object must be driven from one
 * host thread; several objects on different streams may share h (the
 * hierarchy is read only).  AMG_ERR_UNSUPPORTED if the last level is too
 * large for `capacity` columns. */
typedef struct amg_slots amg_slots;
int amg_slots_create(amg_hierarchy *h, int32_t capacity, double rtol, int32_t maxit, void *stream, amg_slots **out);
int amg_slots_admit(amg_slots *s, int32_t slot, const double *b);
int amg_slots_step(amg_slots *s);
int amg_slots_poll(amg_slots *s, int32_t *state, int32_t *iters);
int amg_slots_query(amg_slots *s, int32_t *state, int32_t *iters, int64_t *steps_done, int64_t *steps_issued);
int amg_slots_wait(amg_slots *s);
int amg_slots_retire(amg_slots *s, int32_t slot, double *x);
void amg_slots_free(amg_slots *s);

/* One application of the preconditioner z = B y (Algorithm 2 on level 0):
 * y, z device arrays of n doubles (FP64 in and out in every precision mode). */
int amg_vcycle_apply(amg_hierarchy *h, const double *y, double *z, void *stream);

/* y = A_k x with the FP64 copy of level k's operator; x, y device arrays of n_k doubles. */
int amg_spmv(amg_hierarchy *h, int32_t level, const double *x, double *y, void *stream);

/* q = A p and (p, q) in one pass, allocating no device memory.  The paper
 * has no counterpart: this is a library convenience around the CG loop's
 * fused SpMV + dot product.
 *
 * Some callers cannot call cudaMalloc at the point where they need this
 * product: a process whose device memory is already handed out to another
 * allocator (a framework's caching pool sized to nearly all of HBM), a
 * latency-critical loop that must not risk the device-wide synchronisation
 * cudaMalloc/cudaFree can cause, or code that must not fail with "out of
 * memory" halfway through an iteration.  This entry point takes every input
 * and output from the caller and keeps its only scratch (per-block partial
 * sums and a ticket counter, 16 KiB + 256 B) in a fixed array inside the
 * library that each device holds from the moment the library's device code is
 * loaded until the process exits.
 *
 * A as CSR (rowptr[n+1], colidx[nnz], val[nnz]) and p[n], q[n], pq[1] are
 * device pointers on the current device; q receives A p and *pq receives
 * (p, A p), both FP64, stream-ordered on `stream` (nothing is synchronised).
 * q and pq must not overlap each other, p or A's arrays (the kernel reads p
 * and A through the read-only path while it writes q).
 * Limit: n <= 16,777,216 rows (the scratch holds 2048 block partials of 8192
 * rows each); larger n returns AMG_ERR_UNSUPPORTED before any GPU work.
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The address is kept per device and context: after a cudaDeviceReset the
 * next call on that device looks it up again (again outside any capture).
 * Every call on a device shares the scratch array and it keeps the previous
 * call's contents; the ticket is cleared at the start of each call, but calls
 * that overlap on the GPU (e.g. on two streams at once) race on it and give
 * wrong results: serialise them. */
int amg_spmv_dot_noalloc(int32_t n, int32_t nnz, const int32_t *rowptr, const int32_t *colidx, const double *val,
                         const double *p, double *q, double *pq, void *stream);

/* Result of a one-call solve. */
typedef struct {
  int32_t iters;
  int32_t nlevels;
  double final_residual; /* ||r||_2 of the recursive residual at exit */
  double setup_ms;       /* T_p: amg_setup wall time (ms), host-measured */
  double solve_ms;       /* T_s: amg_pcg_solve wall time (ms), host-measured */
} amg_result;

/* Set-up + solve + free in one call (T_t = T_p + T_s, Sec. 4).  A, b, x are
 * host or device according to A->on_device (b and x follow A).  x holds x0 on
 * entry.  Host buffers are copied to and from the device inside the call. */
int amg_solve(const amg_csr *A, const double *b, double *x, const amg_params *params, double rtol,
              int32_t maxit, const amg_allocator *alloc, void *stream, amg_result *res);

/* Hierarchy sizes.  cap = capacity of the per-level arrays (any may be NULL):
 * n_k[k] rows of A_k, nnz_k[k] nonzeros of A_k, nnzP_k[k] nonzeros of P_k
 * (0 on the last level).  cgd = sum n_k / n_0 and cop = sum nnz_k / nnz_0
 * (grid and operator complexities, Sec. 4). */
int amg_hierarchy_info(const amg_hierarchy *h, int32_t *nlevels, int32_t cap, int64_t *n_k, int64_t *nnz_k,
                       int64_t *nnzP_k, double *cgd, double *cop);

/* Copies level k of the FP64 hierarchy to host arrays (any may be NULL):
 * cf[n_k] (1 = C, 0 = F; all zero on the last level), A_k as CSR
 * (A_rowptr[n_k+1], A_col[nnz_k], A_val[nnz_k]) and P_k as CSR
 * (P_rowptr[n_k+1], P_col[nnzP_k], P_val[nnzP_k]; ignored on the last level).
 * Synchronises the hierarchy's stream. */
int amg_hierarchy_export(const amg_hierarchy *h, int32_t level, int8_t *cf, int32_t *A_rowptr, int32_t *A_col,
                         double *A_val, int32_t *P_rowptr, int32_t *P_col, double *P_val);

/* FSAI factor of level k (smoother AMG_SMOOTH_FSAI, k < nlevels - 1): *nnz (may be
 * NULL) receives nnz(G_k); G_rowptr[n_k + 1], G_col[nnz], G_val[nnz] (host, any may be
 * NULL) receive G_k as CSR (rows ascending, each ending at its diagonal).  *nnz = 0 and
 * nothing is copied on the last level or with the Jacobi smoother.  Synchronises the
 * hierarchy's stream. */
int amg_hierarchy_export_fsai(const amg_hierarchy *h, int32_t level, int64_t *nnz, int32_t *G_rowptr,
                              int32_t *G_col, double *G_val);

/* Device bytes held by the hierarchy (for admission by free HBM). */
size_t amg_hierarchy_bytes(const amg_hierarchy *h);

/* Releases the hierarchy (stream-ordered on the stream given to amg_setup). NULL is a no-op. */
void amg_free(amg_hierarchy *h);

/* Per-kernel timing with CUDA events on each launch's stream (process-wide,
 * not thread-safe).  amg_profile_enable(1) clears the totals and starts
 * recording every libamg kernel launch; amg_profile_enable(0) stops.
 * amg_profile_read(kernel, level, &launches, &ms, &bytes) returns, for kernel
 * class `kernel` (AMG_K_*) on hierarchy level `level` (-1: all levels and
 * launches that belong to none), the number of launches, their summed
 * event-timed duration and the algorithmic bytes they move (int32 indices,
 * values and vectors counted once per launch; the accounting behind the
 * roofline).  Totals include every call that has returned. */
#define AMG_K_SPMV_DOT 0      /* PCG: q = A p and (p, q) */
#define AMG_K_PCG_UPDATE 1    /* PCG: x += alpha p, r -= alpha q, ||r||, smoother input */
#define AMG_K_SMOOTH_RESID 2  /* V-cycle: r_k = y_k - A_k s_k (pre-smoothed residual) */
#define AMG_K_RESTRICT 3      /* V-cycle: y_{k+1} = R_k r_k */
#define AMG_K_PROLONG 4       /* V-cycle: t_k = s_k + P_k z_{k+1} */
#define AMG_K_SMOOTH_POST 5   /* V-cycle: z_k = t_k + omega D^-1 (y_k - A_k t_k) */
#define AMG_K_COARSE 6        /* V-cycle: z_L = L^-T L^-1 y_L */
#define AMG_K_DIRECTION 7     /* PCG: p = z + beta p */
#define AMG_K_SOLVE_OTHER 8   /* initial residual, extra sweeps, copies, level SpMV */
#define AMG_K_STRENGTH 9      /* set-up: validation, strength, PMIS measures */
#define AMG_K_PMIS 10         /* set-up: PMIS rounds and C/F output */
#define AMG_K_INTERP 11       /* set-up: direct interpolation */
#define AMG_K_TRANSPOSE 12    /* set-up: R = P^T */
#define AMG_K_SPGEMM 13       /* set-up: Galerkin SpGEMM (A P, then R (A P)) */
#define AMG_K_SETUP_OTHER 14  /* set-up: scans, dense factor, casts, diagonal */
#define AMG_K_SMOOTH_FSAI 15  /* V-cycle, FSAI smoother: u = G w and s += omega G^T u */
#define AMG_K_FSAI 16         /* set-up: FSAI factor G and omega G^T */
#define AMG_K_COUNT 17
int amg_profile_enable(int32_t on);
/* Restricts recording to launches of kernel class `kernel` on level `level`
 * (-1: any level); kernel = -1 records every launch again (the default).
 * Recording one class keeps the event overhead out of the other launches. */
int amg_profile_filter(int32_t kernel, int32_t level);
int amg_profile_read(int32_t kernel, int32_t level, int64_t *launches, double *ms, double *bytes);

/* Number of libamg kernel launches in this process so far. */
int64_t amg_launch_count(void);

/* Static strings; never NULL. */
const char *amg_status_string(int status);
const char *amg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AMG_H */

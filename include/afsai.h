/*
 * afsai.h - C ABI of the GB300 (sm_103a) adaptive FSAI preconditioner and
 * aFSAI-preconditioned conjugate gradient library (libafsai.so).
 *
 * Method: Isotton, Janna, Bernaschi, "A GPU-accelerated Adaptive FSAI
 * preconditioner for Massively Parallel Simulations" (arXiv 2010.14175),
 * Section 2 (set-up), Section 3 (kernels: Kaporin gradient, systems gather,
 * batched Cholesky, miniwarp SpMV) and Section 5.2 (PCG to an 8-order
 * residual reduction).
 *
 * Conventions shared by every entry point:
 *   - Plain C types only; no exceptions cross the boundary.  Every call
 *     returns an afsai_status; on failure a thread-local message is available
 *     from afsai_last_error().
 *   - "device pointer" = memory of the current CUDA device (cudaMalloc,
 *     cudaMallocAsync or a framework allocator).  "host pointer" = CPU
 *     memory (pinned memory makes the host<->device copies faster).
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it; calls that must read a result on the host
 *     (status, counts, iteration numbers) synchronise that stream.
 *   - The caller owns every buffer it passes.  The library owns what it
 *     returns through an opaque handle until the matching destroy call.
 *   - Matrices are CSR with int32 row pointers and column indices, 0-based,
 *     columns strictly increasing within each row, full symmetric storage
 *     (both triangles), diagonal present and positive.  The set-up assumes
 *     A is symmetric positive definite and reads the lower part of row r
 *     for A[r, j], j <= r, and row r for a_jr by symmetry.
 */
#ifndef AFSAI_H
#define AFSAI_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AFSAI_API __attribute__((visibility("default")))
#else
#define AFSAI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AFSAI_OK = 0,
    AFSAI_EINVAL = 1,   /* invalid argument or malformed CSR */
    AFSAI_ENOMEM = 2,   /* device or host allocation failed */
    AFSAI_ENOTSPD = 3,  /* a non-positive pivot in a row system (A not SPD) */
    AFSAI_ENOCONV = 4,  /* PCG did not reach rtol within maxit iterations */
    AFSAI_ECUDA = 5,    /* a CUDA runtime call failed */
    AFSAI_ETIMEOUT = 6, /* a bounded device-side wait ran out */
    AFSAI_EAGAIN = 7,   /* result not ready yet (serving) */
    AFSAI_EBUSY = 8,    /* no free slot or memory (serving admission) */
    AFSAI_ENOTSUP = 9   /* parameters beyond what this build supports */
} afsai_status;

/* A sparse matrix in CSR.  rowptr: n+1 entries, col/val: nnz entries.
 * Whether the pointers are host or device memory is stated per call. */
typedef struct {
    int32_t n;
    int64_t nnz;
    const int32_t* rowptr;
    const int32_t* col;
    const double* val;
} afsai_csr;

/* Parameters of the adaptive set-up (Section 2, "three user-specified
 * parameters": k_max, s, epsilon).
 *   kiter      number of pattern enlargement steps per row (k_max), >= 0;
 *              a row holds at most 1 + kiter*s entries (<= 128 here).
 *   s          entries added per step, >= 1.
 *   eps        tolerance of the Kaporin-number reduction test, >= 0.
 *   exit_mode  0: stop a row after step k when
 *                 (psi_{k-1} - psi_k) < eps * psi_{k-1}   (default reading
 *                 of "relative tolerance on the Kaporin number reduction");
 *              1: the printed test psi_k / psi_0 <= eps (Eq. "exit_crit").
 *   g_prec     storage and arithmetic of G and G^T in the application:
 *              0 fp64, 1 fp32, 2 bf16 (fp32 accumulation for 1 and 2).
 *   chol_prec  0: FP64 Cholesky of every row system (bit-exact with the
 *              plain FP64 definition); 1: FP32 Cholesky followed by one
 *              FP64 iterative-refinement step.  The Kaporin gradient and the
 *              selection stay FP64 in both.
 *   block_rows, block_power
 *              locality bound of the distributed set-up (Section 4, "aFSAI
 *              set-up on a distributed memory computer"): with
 *              block_rows > 0 the rows are cut into stripes of block_rows
 *              consecutive rows (the last may be shorter), Ahat is the
 *              stripe adjacency of A (Ahat_IJ = 1 iff block (I, J) holds a
 *              nonzero) and a row of stripe I only takes candidates from
 *              stripes J with (Ahat^block_power)_IJ = 1, so that the stripe
 *              graph of G lies in the lower part of Ahat^block_power.
 *              block_rows = 0: no bound (block_power is then ignored);
 *              block_power in [0, 64], 0 keeps every row inside its own
 *              stripe; at most 8192 stripes (else AFSAI_ENOTSUP).  Single
 *              system set-ups only (the batched and served forms return
 *              AFSAI_ENOTSUP for block_rows != 0). */
typedef struct {
    int32_t kiter;
    int32_t s;
    double eps;
    int32_t exit_mode;
    int32_t g_prec;
    int32_t chol_prec;
    int32_t block_rows;
    int32_t block_power;
} afsai_params;

/* Opaque preconditioner: G (lower triangular, CSR, sorted columns), its
 * explicitly stored transpose G^T, and per-row set-up results, all in
 * device memory owned by the library. */
typedef struct afsai_precond afsai_precond;

typedef struct {
    int32_t n;          /* rows */
    int64_t nnz_G;      /* entries of G (= entries of G^T) */
    int32_t max_row;    /* longest row of G */
    int32_t g_prec;     /* as in afsai_params */
    int32_t n_retry;    /* rows whose candidate table overflowed shared
                           memory and were redone with a larger table */
    double setup_ms;    /* device time of the whole set-up (CUDA events) */
    double kernel_ms;   /* device time of the fused pattern-search kernel */
} afsai_info;

typedef struct {
    int32_t iters;       /* PCG iterations performed */
    int32_t converged;   /* 1 if both ||r_k|| and ||b - A x_k|| reached rtol ||b|| */
    double relres_rec;   /* recursive ||r_k|| / ||b|| at exit */
    double relres_true;  /* ||b - A x|| / ||b|| recomputed at exit */
    double solve_ms;     /* device time of the solve (CUDA events) */
    double kernel_ms[5]; /* pcg_solve with a preconditioner: device time of each
                            kernel of one iteration (q = A p with p.q; the x, r
                            update with r.r; t = G r; z = G^T t with r.z; the
                            p update), from CUDA events around the first
                            iteration of the first graph launch; else 0 */
} pcg_info;

/* Builds the aFSAI preconditioner of A (Section 2): for every row i, grow
 * the pattern P_i from {i} by the s candidates j < i of largest Kaporin
 * gradient |(A g_i)_j| (Eq. "grapsi"), solve A[P_i,P_i] g_i = e_m by
 * Cholesky (Eq. "DensSys"), stop after kiter steps or on the exit test
 * (Eq. "exit_crit"), and scale G[i,P_i] = g_i / sqrt(g_i,m) so that
 * diag(G A G^T) = I (Eq. "diagScal").  Then builds G^T, and sliced
 * (SELL-32) copies of G and G^T for the one-lane-per-row SpMV engines
 * (about twice the memory of G and G^T; skipped, without error, when the
 * device has no room for them).  The first successful set-up on a device
 * also loads the 8 MiB device array of afsai_apply_static there (once per
 * device, held until the process exits).
 *   A       device pointers; must stay valid during the call only.
 *   params  host pointer.
 *   out     receives a new handle (free with afsai_destroy).
 * Synchronises `stream`.  Errors: EINVAL (bad parameters or CSR: n <= 0,
 * rowptr not monotone or rowptr[0] != 0 or rowptr[n] != nnz, a column out
 * of range or not strictly increasing, a missing or non-positive diagonal),
 * ENOTSUP (1 + kiter*s > 128), ENOTSPD (a non-positive pivot; the handle is
 * not created), ENOMEM, ECUDA. */
AFSAI_API afsai_status afsai_setup(const afsai_csr* A, const afsai_params* params, void* stream, afsai_precond** out);

/* z = G^T (G r), the preconditioner application M^{-1} r (Eq. "prec"), as
 * two SpMVs (G, then the stored G^T; Section 3 "miniwarp" SpMV), on the CSR
 * or the sliced copies, whichever engine the autotuner chose.
 * r, z: device vectors of n doubles (must not overlap).  Asynchronous. */
AFSAI_API afsai_status afsai_apply(const afsai_precond* M, const double* r, double* z, void* stream);

/* Same result as afsai_apply, for callers that cannot allocate device
 * memory: code whose device memory is owned by another allocator (a
 * framework's caching allocator that has reserved the free memory), and
 * code on a latency-critical path where cudaMalloc / cudaFree may
 * synchronise the device.  The paper has no counterpart; this is a service
 * entry point of the library.
 *   - Allocates nothing: the intermediate G r is kept in a fixed device
 *     array of 2^20 doubles (8 MiB).  n > 2^20 returns AFSAI_EINVAL.
 *   - The array is loaded into a device's memory when the library's
 *     module that holds it is first used on that device (CUDA loads
 *     modules lazily); afsai_setup does that, so after a successful
 *     afsai_setup on a device the array is in place and stays until the
 *     process exits or the device is reset.  If the set-up could not load
 *     it (no device memory left at that moment), the first
 *     afsai_apply_static on that device tries again and returns
 *     AFSAI_ENOMEM if it still cannot; if that first attempt happens
 *     during a stream capture, it returns AFSAI_EINVAL instead (loading is
 *     not allowed during a capture).
 *   - The array's device address is cached per device: after
 *     cudaDeviceReset every handle of this library is invalid, and so is
 *     that cached address; calls after a reset are not supported.
 *   - M must belong to the current device (else AFSAI_EINVAL).
 *   - All calls share the array and it keeps the last call's contents;
 *     calls that overlap on the GPU (different streams, no ordering) race
 *     on it and give wrong results.  Calls on one stream are safe.
 *   - The SpMV engines are the ones already chosen for this matrix shape
 *     by afsai_apply / pcg_solve, else a default; nothing is timed.
 * r, z: device vectors of n doubles (must not overlap).  Asynchronous. */
AFSAI_API afsai_status afsai_apply_static(const afsai_precond* M, const double* r, double* z, void* stream);

/* y = A x (CSR SpMV, FP64).  A, x, y device pointers.  Asynchronous. */
AFSAI_API afsai_status afsai_spmv(const afsai_csr* A, const double* x, double* y, void* stream);

/* Preconditioned conjugate gradients for A x = b with M^{-1} = G^T G
 * (M = NULL gives unpreconditioned CG).  x (device, n doubles) is the
 * initial guess on entry and the solution on exit; b device.  Stops when
 * the recursive residual satisfies ||r_k||_2 <= rtol ||b||_2 (Section 5.2:
 * 8 orders of reduction for rtol = 1e-8) or after maxit iterations.  The
 * iteration runs on the device (CUDA graphs); the host only polls a flag.
 * When the SpMV engine of A is a sliced one (or not chosen yet), the solve
 * builds a sliced copy of A for its own use (about the memory of A, freed
 * before it returns; without room for it the CSR engines serve).
 * Synchronises `stream`.  info (host, may be NULL) receives the outcome.
 * Returns OK, ENOCONV (maxit reached), EINVAL, ENOMEM, ECUDA. */
AFSAI_API afsai_status pcg_solve(const afsai_csr* A, const afsai_precond* M, const double* b, double* x, double rtol,
                       int32_t maxit, void* stream, pcg_info* info);

/* Outcome of a batched solve (host struct). */
typedef struct {
    int32_t nsys;          /* systems in the batch */
    int32_t converged;     /* systems that reached rtol */
    int32_t max_iters;     /* largest PCG iteration count of the batch */
    int32_t graph_launches;/* graph launches of the PCG loop */
    int64_t total_rows;    /* sum of n */
    int64_t nnz_G;         /* sum of the entries of the G factors */
    double setup_ms;       /* device time of the packed set-up */
    double solve_ms;       /* device time of the batched PCG */
} afsai_batch_info;

/* Solves nsys independent SPD systems A_k x_k = b_k with aFSAI-PCG in one
 * batch (Section 2 set-up, Section 5.2 stopping rule): one fused set-up
 * launch over the rows of all systems (packed block-diagonally, so each
 * G_k equals the G of system k alone), then graph-captured PCG iterations
 * that advance every unconverged system per launch; each system keeps its
 * own alpha, beta and convergence test, and its result does not depend on
 * the other systems of the batch.
 *   A       host array of nsys CSR descriptors with DEVICE pointers.
 *   params  one parameter set for all systems (host).
 *   b, x    host arrays of nsys DEVICE pointers; x_k is the initial guess
 *           on entry and the solution on exit.
 *   info    host array of nsys pcg_info (may be NULL); binfo may be NULL.
 * Synchronises `stream`.  Returns OK, ENOCONV (some system reached maxit),
 * EINVAL (bad arguments or parameters, checked before any device work),
 * ENOTSPD, ENOTSUP (1 + kiter*s > 128, or the locality bound, which applies
 * to single-system set-ups only), ENOMEM, ECUDA. */
AFSAI_API afsai_status afsai_batch_solve(int32_t nsys, const afsai_csr* A, const afsai_params* params,
                                         const double* const* b, double* const* x, double rtol, int32_t maxit,
                                         void* stream, pcg_info* info, afsai_batch_info* binfo);

/* ---- Solve server (continuous batching; no counterpart in the paper, which
 * solves one system at a time).  Registered matrices stay on the device;
 * the set-up of a matrix runs at its first request and its G is reused.
 * Requests (1..k right-hand sides each) are admitted in arrival order as
 * slots and device memory (the budget covers matrices, preconditioners and
 * vectors) free up; every server step advances all running systems by a
 * few PCG iterations in one graph launch, whatever their sizes; finished
 * systems leave and free their slot.  A system's result does not depend on
 * which other systems were running with it. */
typedef struct afsai_server afsai_server;

typedef struct {
    int32_t nrhs;            /* right-hand sides of the request */
    int32_t max_iters;       /* largest PCG iteration count among them */
    int32_t converged;       /* 1 if all reached their rtol */
    int32_t pad;
    double max_relres_true;  /* largest ||b - A x|| / ||b|| */
    double queue_ms;         /* submit -> admission */
    double setup_ms;         /* set-up time paid by this request (0 if G was reused) */
    double latency_ms;       /* submit -> completion */
} serve_result;

typedef struct {
    int64_t requests_submitted, requests_done, solves, steps;
    int64_t peak_mem_bytes, mem_used_bytes, queued, running;
} serve_stats;

/* Starts a server thread on the current device.  mem_budget_bytes bounds
 * the device memory of matrices + preconditioners + vectors; max_slots
 * bounds the systems on the GPU at once; params applies to every matrix
 * (checked here as by afsai_setup: EINVAL or ENOTSUP; the locality bound
 * block_rows > 0 is ENOTSUP); iters_per_step = PCG iterations per server
 * step (<= 0: 4).  Errors: EINVAL (NULL out or params, max_slots <= 0, a
 * zero budget, maxit <= 0, bad parameters), ENOTSUP, ENOMEM, ECUDA. */
AFSAI_API afsai_status serve_create(size_t mem_budget_bytes, int32_t max_slots, const afsai_params* params,
                                    int32_t maxit, int32_t iters_per_step, afsai_server** out);
/* Copies A (host or device CSR) to the device; *matrix_id names it in
 * later requests.  EBUSY if it does not fit the budget. */
AFSAI_API afsai_status serve_register(afsai_server* S, const afsai_csr* A, int32_t* matrix_id);
/* Queues a request: b = n * nrhs HOST doubles (right-hand side k at offset
 * k n), copied before return.  Returns at once with a ticket. */
AFSAI_API afsai_status serve_submit(afsai_server* S, int32_t matrix_id, const double* b, int32_t nrhs, double rtol,
                                    int64_t* ticket);
/* AFSAI_EAGAIN while the request runs; then copies x (n * nrhs HOST
 * doubles), per-rhs info (nrhs entries) and the summary (each may be NULL)
 * and releases the ticket.  ENOCONV if a right-hand side hit maxit. */
AFSAI_API afsai_status serve_poll(afsai_server* S, int64_t ticket, double* x, pcg_info* info, serve_result* res);
AFSAI_API afsai_status serve_get_stats(afsai_server* S, serve_stats* out);
/* Stops the server thread and frees everything (pending requests are dropped). */
AFSAI_API void serve_destroy(afsai_server* S);

/* End-to-end solve from HOST buffers: copies A and b to the device, builds
 * the preconditioner, runs PCG from x = 0 and copies x back (x_host: n
 * doubles).  Device memory is allocated and freed inside the call.
 * setup_info and info may be NULL.  Synchronises `stream`. */
AFSAI_API afsai_status afsai_solve_host(const afsai_csr* A_host, const afsai_params* params, const double* b_host,
                              double* x_host, double rtol, int32_t maxit, void* stream, afsai_info* setup_info,
                              pcg_info* info);

/* Sizes and timings of a preconditioner (host struct). */
AFSAI_API afsai_status afsai_get_info(const afsai_precond* M, afsai_info* info);

/* Copies G or G^T to HOST buffers: rowptr n+1, col nnz_G, val nnz_G
 * (converted to double whatever g_prec is).  Any pointer may be NULL to
 * skip it.  Synchronous. */
AFSAI_API afsai_status afsai_export_G(const afsai_precond* M, int32_t* rowptr, int32_t* col, double* val);
AFSAI_API afsai_status afsai_export_Gt(const afsai_precond* M, int32_t* rowptr, int32_t* col, double* val);

/* Copies per-row set-up results to HOST buffers of n entries: psi (final
 * Kaporin row measure psi_i = 1 / g_i,m, Eq. "kap_min") and the number of
 * enlargement steps performed.  Either pointer may be NULL. */
AFSAI_API afsai_status afsai_export_rows(const afsai_precond* M, double* psi, int32_t* steps);

AFSAI_API void afsai_destroy(afsai_precond* M);

/* Message of the last failure on the calling thread ("" if none). */
AFSAI_API const char* afsai_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (kernels inside CUDA graph launches included). */
AFSAI_API int64_t afsai_kernel_launches(void);

/* Device memory pool of the library (no counterpart in the paper).  Every
 * device allocation of the library (set-up temporaries, G and G^T, PCG
 * vectors, batch and server tables) comes from a stream-ordered memory
 * pool that the library creates on each device at first use; memory freed
 * by the library stays in that pool for its next call instead of being
 * returned to the device (the environment variable AFSAI_POOL=0 makes the
 * library use the device's default pool instead).
 * afsai_trim_pool returns the unused memory of the current device's pool
 * to the device (cudaMemPoolTrimTo); memory of live handles stays.
 * afsai_pool_stats writes the bytes in use and the bytes reserved by the
 * current device's pool (either pointer may be NULL, not both; 0 and 0
 * without a pool).  Both return AFSAI_OK, AFSAI_EINVAL or AFSAI_ECUDA. */
AFSAI_API afsai_status afsai_trim_pool(void);
AFSAI_API afsai_status afsai_pool_stats(int64_t* used_bytes, int64_t* reserved_bytes);

/* Library version string. */
AFSAI_API const char* afsai_version(void);

/* Diagnostic: the CSR SpMV engine chosen (timed once per matrix shape) for
 * role 0 (A), 1 (G) or 2 (G^T) of an n x n matrix with nnz entries and value
 * type vtype (0 fp64, 1 fp32, 2 bf16) on the calling thread's device, or 0
 * if none was chosen yet.  Engines: 1, 2, 4, 8 = that many lanes per row,
 * strided; 3, 6 = grouped lanes; 101, 102 = staged tiles with 1 or 2
 * threads per row.  The environment variable AFSAI_SPMV_MODES="a,g,gt" (or
 * AFSAI_SPMV_MODE for all roles) pins the engines instead of timing them,
 * e.g. to profile the engines a timed run chose. */
AFSAI_API int32_t afsai_spmv_engine(int32_t role, int32_t n, int64_t nnz, int32_t vtype);

/* Self-check of the library's own FP64 arithmetic (no counterpart in the
 * paper).  The lane-per-row dense solves of the FP64 set-up compute their
 * square roots and divisions on the integer pipes (GB300 runs FP64 at 1/64
 * of the FP32 rate) and must give the IEEE round-to-nearest results bit for
 * bit.  This call draws n operand sets on the device from a counter-based
 * generator seeded by `seed` (random and structured significands, normal
 * and extreme exponents, near-exact quotients, zero numerators, squares and
 * their neighbours), compares every result with the hardware IEEE
 * operation and writes the mismatch counts to mismatches[0] (divisions) and
 * mismatches[1] (square roots), a host array of two entries.  Synchronous
 * on `stream`.  Returns AFSAI_EINVAL for n < 0 or mismatches == NULL. */
AFSAI_API afsai_status afsai_check_arith(int64_t n, uint64_t seed, int64_t* mismatches, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* AFSAI_H */

/*
 * aar.h -- C ABI of the GB300 (sm_103a) Alternating Anderson-Richardson (AAR) solver.
 *
 * The method (Suryanarayana, Pratapa, Pask, arXiv:1606.08740, Sec. 2) solves A x = b (Eq. 1)
 * with the fixed-point iteration x_{k+1} = x_k + B_k f_k (Eq. 2), where
 *   f_k = M^{-1} (b - A x_k), M = diag(A) (Jacobi; Eq. 6, AAJ in Sec. 2),
 *   B_k = omega I                                          if (k+1) mod p != 0 (Richardson),
 *   B_k = beta I - (X_k + beta F_k) pinv(F_k^T F_k) F_k^T  if (k+1) mod p == 0 (Anderson, Eq. 3),
 * and X_k, F_k hold the last min(k, m) differences of iterates and residuals (Eq. 4, 5).
 * The relative residual ||b - A x_k|| / ||b|| is evaluated only at Anderson steps (Sec. 2), and
 * the Gram matrix is inverted as a Moore-Penrose pseudoinverse (Sec. 3.2), eigenvalues at or
 * below m * 2^-52 * lambda_max treated as zero.
 *
 * Conventions for every call:
 *  - Every function returns an aar_status; nothing throws across the ABI.
 *  - Vectors are FP64, length N = nx*ny*nz (stencil, index (z*ny + y)*nx + x, interior points
 *    only, zero Dirichlet ghosts) or n (CSR).
 *  - Pointers marked "device" must be device memory of the handle's device. Pointers marked
 *    "device or host" may be either (host memory is staged through the handle's buffers).
 *  - A handle is used by one host thread at a time. All work is enqueued on the handle's
 *    stream; calls that return results synchronise that stream before returning.
 *  - The handle owns its workspace (history ring, partial sums, solver state). Caller arrays
 *    given to a create call (CSR arrays, dinv) are borrowed until the handle is destroyed.
 *
 * Environment variables read by the library (none is needed; each selects an alternative that
 * does the same work, or a diagnostic):
 *  - AAR_DEBUG: print the CUDA error behind an AAR_ERR_CUDA status, a failed step of building
 *    the solve graph, and where a bounded device wait gave up (AAR_ERR_TIMEOUT).
 *  - AAR_WAIT_TIMEOUT_S: seconds a host wait for the handle's stream may take before the call
 *    returns an error (default 1800); the device-side step limit bounds the work itself.
 *  - AAR_HOST_LOOP: run the solve loop's ticks from a host loop instead of the CUDA graph with a
 *    device-side loop (same kernels, same results; for profilers that cannot see kernels in
 *    graphs with conditional nodes).
 *  - AAR_SWEEP_VARIANT: FP32 sweep tiling of a Jacobi stencil solve (an index of the tile-shape
 *    variants, used when valid for the grid; the autotuner's hint takes precedence).
 *  - AAR_ZSWEEP_REG=1, AAR_ZGRAM_REG=1 (complex solves, aar_complex.h): the register-fed FP32
 *    sweep and Gram kernels instead of the shared-memory-staged and bulk-copy-fed ones.
 */
#ifndef AAR_H
#define AAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AAR_OK = 0,
    AAR_NOT_CONVERGED = 1,     /* max_iter (or the refinement cap) reached; x holds the last iterate */
    AAR_ERR_INVALID_ARG = -1,  /* a size, pointer or parameter outside its documented range */
    AAR_ERR_OOM = -2,          /* device allocation failed or exceeded the configured budget */
    AAR_ERR_CUDA = -3,         /* a CUDA runtime call failed (context may be unusable) */
    AAR_ERR_BREAKDOWN = -4,    /* non-finite residual or extrapolation coefficients */
    AAR_ERR_TIMEOUT = -5,      /* the device-side step limit was exhausted */
    AAR_ERR_UNSUPPORTED = -6,  /* combination not supported by this build */
    AAR_ERR_COMM = -7          /* a communication callback of a domain-decomposed solve failed */
} aar_status;

enum { AAR_FP64 = 0,   /* plain method: all vectors and arithmetic in FP64 */
       AAR_MIXED = 1   /* FP32 AAR inner solves inside FP64 iterative refinement */ };

#define AAR_MAX_M 16
#define AAR_MAX_RADIUS 6
/* aar_params.flags: AAR_MIXED starts every inner solve from an empty Anderson history (plain
 * iterative refinement) instead of continuing the one of the previous inner solve. */
#define AAR_FLAG_RESTART_HISTORY 1

typedef struct aar_ctx* aar_handle;
typedef struct aar_batch_ctx* aar_batch;
typedef struct aar_server_ctx* aar_server;

/* Constant-coefficient finite-difference operator A = -(1/h^2)(Dxx + Dyy + Dzz) + shift I,
 * with (D u)_i = sum_{k=-r..r} w[|k|] u_{i+k} along each axis (Sec. 3.2/3.3 discretise the
 * Helmholtz and Poisson equations this way; shift = 0 is Poisson). radius r in [1, 6];
 * w[0..r] are the 1-D second-derivative weights for unit spacing; shift >= 0; h > 0.
 * periodic = 0: neighbours outside the grid are zero (zero Dirichlet ghosts); periodic = 1:
 * every axis wraps (index i + k taken modulo the axis length), the periodic cells of the
 * paper's Sec. 3.2/3.3 runs. Periodic Poisson (shift = 0) is singular: b must have zero mean,
 * and from x0 = 0 the solve returns the zero-mean solution. */
typedef struct {
    int32_t nx, ny, nz, radius;
    double w[AAR_MAX_RADIUS + 1];
    double h, shift;
    /* Tile hints (0 = automatic): tile_variant = 1 + sweep variant id, tile_zc = z depth of a
     * tile (for the paired-FP32 TMA sweep, variant 4: the length in planes of the equal segments
     * its columns are cut into; automatic = one segment per resident CTA). Set by
     * aar_tune_stencil / the autotuner; they change speed, never results' meaning (a system's
     * reduction order follows its own tiles only). */
    int32_t tile_variant, tile_zc;
    int32_t periodic;  /* 0 or 1, see above; other values are invalid */
    /* Preconditioner M (Eq. 6): 0 or 1 = Jacobi, M = diag(A); 2 = block Jacobi with 2 x 2 x 2
     * boxes (the block Jacobi of Sec. 3.2/3.3, each block solved exactly): M = the diagonal
     * blocks of A for the tiling of the grid by 2 x 2 x 2 boxes. A box holds the centre weight
     * and the distance-1 couplings inside it, so every block is d I + c1 Q3 (Q3 the cube graph)
     * and M^{-1} is applied in the cube's Walsh-Hadamard basis. Needs even sides, a periodic side
     * of at least radius + 2 and no dinv array; batches and servers may mix block-Jacobi and
     * Jacobi systems. */
    int32_t block;
} aar_stencil_desc;

/* General sparse operator in CSR, int32 indices, FP64 values (device pointers, borrowed).
 * Every row must hold a nonzero diagonal entry when dinv is derived. */
typedef struct {
    int32_t n;
    int64_t nnz;
    const int32_t* row_ptr; /* device, n+1 entries, row_ptr[0] = 0, row_ptr[n] = nnz */
    const int32_t* col_idx; /* device, nnz entries in [0, n) */
    const double* val;      /* device, nnz entries */
} aar_csr_desc;

/* Solver parameters (Eq. 2-3 and the refinement loop). */
typedef struct {
    double omega;       /* Richardson relaxation (paper default 0.6) */
    double beta;        /* Anderson relaxation (paper default 0.6) */
    int32_t m;          /* history length, 0..AAR_MAX_M (paper default 9) */
    int32_t p;          /* Anderson period, >= 1 (paper default 8) */
    double tol;         /* stop when ||b - A x|| / ||b|| <= tol (FP64 residual), tol >= 0 */
    int64_t max_iter;   /* cap on iterations (all inner iterations for AAR_MIXED), >= 0 */
    double inner_tol;   /* AAR_MIXED: relative residual target of each FP32 inner solve */
    int32_t max_refine; /* AAR_MIXED: cap on outer FP64 refinements */
    int32_t flags;      /* 0 or AAR_FLAG_RESTART_HISTORY; other bits are invalid */
    /* Watchdog on the device-side solve loop, in device steps (each step advances every
     * unfinished system by one iteration or one refinement step): 0 = derived from max_iter and
     * max_refine, so that max_iter is always reached first; > 0 = stop after about this many
     * steps (checked between groups of steps, when no kernel of the loop is running), every
     * unfinished system then ending with AAR_ERR_TIMEOUT and x holding its last certified
     * iterate (or zeros). A batch takes the largest limit of its systems. Negative is invalid. */
    int64_t step_limit;
} aar_params;

typedef struct {
    int64_t iterations;    /* updates performed (AAR_MIXED: summed over inner solves) */
    int32_t anderson_steps;
    int32_t refinements;   /* AAR_MIXED: FP32 inner solves run (one per refinement step) */
    double rel_residual;   /* last FP64 ||b - A x|| / ||b|| measured (NaN if none) */
    int32_t status;        /* repeats the returned aar_status */
    int32_t last_rank;     /* kept rank of the last pseudoinverse */
    int64_t ticks;         /* device steps run (each advances every unfinished system once) */
    int64_t launches;      /* kernels launched by the solve, early-exiting ones included */
    int32_t eigen_steps;   /* Anderson steps whose m x m solve used the eigen-decomposition
                              (AAR_FP64: when the LDL^T solve could not certify
                              cond(G) < 2^42 / m, i.e. pinv(G) = G^-1; AAR_MIXED: when an LDL^T
                              pivot was tiny) */
    int32_t reserved;
} aar_info;

/* Fill *p with the paper's defaults {omega, beta, m, p} = {0.6, 0.6, 9, 8} (Sec. 2), tol 1e-8,
 * max_iter 100000, inner_tol 0.1, max_refine 30, flags 0, step_limit 0. (AAR_MIXED keeps the Anderson history
 * across refinements, so a loose inner target costs no restart and keeps the FP32 inner solves
 * away from their rounding floor.) */
aar_status aar_default_params(aar_params* p);

/* Create a solver for a stencil operator. dinv: NULL derives the Jacobi scaling 1/diag(A)
 * = 1/(-3 w[0]/h^2 + shift); otherwise a device array of N FP64 values used as M^{-1}
 * (Eq. 6), borrowed. precision: AAR_FP64 or AAR_MIXED. stream: a cudaStream_t (NULL = the
 * legacy default stream). Returns AAR_ERR_INVALID_ARG for sizes <= 0, radius outside [1, 6],
 * h <= 0, shift < 0 or a non-positive diagonal. */
aar_status aar_create_stencil(const aar_stencil_desc* desc, const double* dinv, int32_t precision,
                              void* stream, aar_handle* out);

/* Create a solver for a CSR operator (Sec. 3.1's general sparse systems). dinv: NULL extracts
 * 1/diag(A) on the device (AAR_ERR_INVALID_ARG if a diagonal entry is zero or missing), or a
 * device array of n FP64 values, borrowed. */
aar_status aar_create_csr(const aar_csr_desc* desc, const double* dinv, int32_t precision,
                          void* stream, aar_handle* out);

/* Solve A x = b. b: device or host, N values. x0: device or host, N values, or NULL for zeros.
 * x: device or host, N values (may alias x0); on AAR_OK it holds the first Anderson-step
 * iterate whose FP64 relative residual is <= tol; on AAR_NOT_CONVERGED the last iterate.
 * info may be NULL. ||b|| == 0 returns x = 0 and AAR_OK after 0 iterations.
 * AAR_ERR_INVALID_ARG: m outside [0, AAR_MAX_M], p < 1, tol < 0, max_iter < 0, omega or beta
 * not finite, inner_tol outside (0, 1), max_refine < 1, unknown flags, or NULL b / x. */
aar_status aar_solve(aar_handle h, const double* b, const double* x0, double* x,
                     const aar_params* params, aar_info* info);

/* y = A x in FP64 (device pointers, N values each; y must not alias x). */
aar_status aar_apply(aar_handle h, const double* x, double* y);

/* *rel = ||b - A x||_2 / ||b||_2 in FP64 (device pointers). */
aar_status aar_rel_residual(aar_handle h, const double* b, const double* x, double* rel);

/* Allocation-free form of aar_rel_residual, for callers that must not allocate device memory
 * during a call: code inside a latency-critical loop where cudaMalloc's implicit device
 * synchronisation is not acceptable, or a process whose device memory is budgeted in full up
 * front. The paper has no counterpart; this is an interface convenience. It computes the same
 * *rel = ||b - A x||_2 / ||b||_2 in FP64 (summed in a different order, so the two agree to
 * rounding), with the operator applied inside the norm kernel. Its only scratch is a file-scope
 * device array of 16392 doubles (128 KB) that every device which loads the library holds until
 * the process exits; the call allocates nothing and frees nothing.
 *  - Size limit: N <= 67,108,864 unknowns (8192 blocks of 8192 points); larger operators get
 *    AAR_ERR_INVALID_ARG.
 *  - Call it with the handle's device current (the device that was current when the handle was
 *    created); with another device current it returns AAR_ERR_INVALID_ARG, since each device
 *    holds its own copy of the array.
 *  - The first call on a device looks up the array's device address (once per device, with that
 *    device current); make that first call before any stream capture.
 *  - All calls share the array and it keeps the last call's partial sums and result. Calls that
 *    overlap on the GPU (different streams or handles at once) race on it and must be ordered by
 *    the caller.
 * b, x: device pointers, N values; rel: host pointer. Synchronises the handle's stream. */
aar_status aar_rel_residual_noalloc(aar_handle h, const double* b, const double* x, double* rel);

aar_status aar_destroy(aar_handle h);

/* Kernels of the solve loop that aar_profile_kernel can time. */
enum { AAR_K_SWEEP = 0,          /* Richardson step: f_k and x_{k+1} (Eq. 2, 3, 6) */
       AAR_K_SWEEP_ANDERSON = 1, /* Anderson step pass 1: f_k and ||b - A x_k||^2 partial sums */
       AAR_K_GRAM = 2,           /* F^T F and F^T f partial sums over a full history (Eq. 3) */
       AAR_K_UPDATE = 3,         /* x_{k+1} = x_k + beta f_k - (X + beta F) gamma (Eq. 3) */
       AAR_K_RESID64 = 4,        /* AAR_MIXED: FP64 residual b - A x of the refinement loop */
       AAR_K_FINALIZE = 5,       /* Anderson-step finalize: partial sums, r_k, pinv solve (one CTA) */
       AAR_K_BLOCK = 6 };        /* block Jacobi (block = 2): f = M^{-1} res and the Richardson update */

/* Time one kernel of the solve loop in isolation: launch it `launches` times on the handle's
 * stream, in the tile layout and grid aar_solve uses, with the history and parameters left by
 * the last aar_solve on this handle (which must have run), bracketed by CUDA events; *ms is the
 * mean time per launch. The solver state is left undefined until the next aar_solve.
 * AAR_ERR_INVALID_ARG: no previous solve, launches < 1, unknown kernel; AAR_ERR_UNSUPPORTED:
 * the kernel does not occur with these parameters (p = 1 has no Richardson step; FP64 solves
 * have no refinement residual; AAR_K_BLOCK needs block = 2). */
aar_status aar_profile_kernel(aar_handle h, int32_t kernel, int32_t launches, float* ms);

/* Measurement primitive (no operation of the paper): the device's FP64 instruction rate, the
 * denominator of the roofline of the FP64 stencil sweeps (about 6 r + 4 FP64 instructions per
 * point against 32 bytes, so bound by the FP64 pipe on this part). op = 0 times DFMA, op = 1
 * DADD: every thread of a grid that fills each SM runs 8 independent dependency chains, timed
 * with CUDA events on `stream` (a cudaStream_t, NULL = legacy default stream) after a warm-up
 * launch. *instr_per_s = thread-level FP64 instructions per second (one DFMA = 2 flops) of the
 * current device. AAR_ERR_INVALID_ARG for another op or a NULL output. */
aar_status aar_measure_fp64_rate(void* stream, int32_t op, double* instr_per_s);

/* Autotuner primitive: time the sweep of one grid shape under every tile variant and z depth
 * valid for `precision` (a short solve with history length m sets up the state, then each
 * candidate's Richardson sweep is timed with CUDA events), and return the fastest as tile
 * hints (*tile_variant, *tile_zc, in aar_stencil_desc's encoding) and its time per sweep.
 * desc's own tile hints are ignored. Allocates and frees a temporary solver. */
aar_status aar_tune_stencil(const aar_stencil_desc* desc, int32_t precision, int32_t m, void* stream,
                            int32_t* tile_variant, int32_t* tile_zc, float* ms);

/* Static description of a status code. Never NULL. */
const char* aar_status_string(aar_status s);

/* ---- Batched solves: many independent stencil systems advanced together ------------------
 * All systems share radius and precision; sizes, weights, h and shift may differ. Each step of
 * the solve advances every unfinished system by one iteration (its own Richardson or Anderson
 * step, or its own refinement step), in launches shared by the whole batch. A system's
 * arithmetic and reduction order depend only on its own size, so its result does not depend on
 * which other systems share the batch. */
aar_status aar_batch_create(const aar_stencil_desc* descs, int32_t nsys, int32_t precision,
                            void* stream, aar_batch* out);

/* b[i], x[i]: device pointers of system i (x0 = 0 for every system). params: nsys entries,
 * or one entry applied to all when params_stride == 0. infos: nsys entries (may be NULL). */
aar_status aar_batch_solve(aar_batch bt, const double* const* b, double* const* x,
                           const aar_params* params, int32_t params_stride, aar_info* infos);

aar_status aar_batch_destroy(aar_batch bt);

/* ---- Serving: continuous batching of stencil solves ------------------------------------------
 * Repeated Poisson/Helmholtz solves are the workload the paper's introduction motivates. A
 * server keeps every admitted solve's state on the device (history ring, iterate, right-hand
 * side, phase) and advances all of them together with the batched kernels. Between scheduling
 * rounds it retires finished solves and admits waiting requests in arrival order while their
 * device footprint fits the budget and a slot is free; requests that arrive while others run
 * join at the next round, and the others continue where they were. A solve's arithmetic and
 * reduction order depend only on its own size, so its result is the same alone and in any mix.
 * All systems of a server share radius and precision. */

/* budget_bytes: device memory the admitted solves may hold together (footprint of one request:
 * 2 max(m+1, 2) N words of history + N FP64 right-hand side [+ N FP64 iterate + N FP32 inner
 * right-hand side for AAR_MIXED], N padded to 64). max_active: slots in [1, 65536]. The slots'
 * memory comes from a stream-ordered pool the server owns, which keeps up to budget_bytes of what
 * retired solves freed for later admissions; aar_server_destroy releases it. AAR_ERR_CUDA if the
 * pool cannot be created. */
aar_status aar_server_create(int32_t radius, int32_t precision, int64_t budget_bytes, int32_t max_active,
                             void* stream, aar_server* out);

/* Queue one solve. b (host, N values) is read when the request is admitted; x (host, N values)
 * receives the solution when it completes; both stay caller-owned and must live until then.
 * x0 = 0. AAR_ERR_OOM if the request alone exceeds the budget. *request_id identifies it. */
aar_status aar_server_submit(aar_server sv, const aar_stencil_desc* desc, const double* b, double* x,
                             const aar_params* params, int64_t* request_id);

/* One scheduling round: admit, advance every resident solve by `ticks` iterations (or
 * refinement steps), retire finished ones (their x is written and their info queued for
 * aar_server_poll). When every resident solve has the same Anderson period p >= 2, `ticks` is
 * rounded to a whole number (at least one) of bodies of p ticks: p - 1 sweeps alone, then one
 * tick of every kernel, as in aar_solve. Reports the resident and waiting counts and the bytes in
 * use. */
aar_status aar_server_run(aar_server sv, int32_t ticks, int32_t* n_active, int32_t* n_waiting,
                          int64_t* bytes_in_use);

/* Completed requests since the last poll, oldest first: up to cap (id, info) pairs; *n = count. */
aar_status aar_server_poll(aar_server sv, int64_t* ids, aar_info* infos, int32_t cap, int32_t* n);

aar_status aar_server_destroy(aar_server sv);

#ifdef __cplusplus
}
#endif

#endif /* AAR_H */

/*
 * aar_dd.h -- domain-decomposed AAR: one stencil system split over ranks (one GPU each).
 *
 * The paper's parallel runs (Sec. 3.2, 3.3) decompose the grid into subdomains, one per process:
 * every sweep needs the neighbouring subdomains' boundary values (a halo exchange of the r
 * planes the stencil reaches), and every Anderson step needs one global reduction, in which the
 * residual norm and F^T F, F^T f travel together (Sec. 3.2: one MPI_Allreduce per Anderson
 * step). Everything else of Eq. 2-6 is local to a subdomain.
 *
 * Here the grid nx x ny x nz is cut into slabs of whole z-planes: a rank owns planes
 * [z_lo, z_hi) and holds its vectors as slabs of nx * ny * (z_hi - z_lo) values (plane-major,
 * index ((z - z_lo) * ny + y) * nx + x). The library runs the iteration on the rank's GPU with
 * the single-GPU kernels (plain FP64 arithmetic, Jacobi M = diag(A)); the caller supplies the
 * communication as two callbacks, so any transport works (NCCL through torch.distributed, MPI,
 * or copies between slabs held by one process). Each rank calls aar_dd_solve with its own slab;
 * the calls proceed in lockstep through the callbacks, and every rank returns the same status,
 * iteration count and residual. For the same global problem the iterates equal those of the
 * single-GPU FP64 solve to rounding (the sums are taken in another order).
 *
 * Conventions as in aar.h: every call returns an aar_status; b and x are device pointers of the
 * handle's device; a handle is used by one host thread at a time.
 */
#ifndef AAR_DD_H
#define AAR_DD_H

#include <stdint.h>

#include "aar.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aar_dd_ctx* aar_dd_handle;

/* Halo exchange of the current iterate x_k (once per sweep). send_lo / send_hi: the rank's
 * lowest / highest r planes (count = r nx ny doubles each, device); recv_lo / recv_hi: the
 * ghost planes below / above the slab, which must receive the highest r planes of the rank
 * below (z_lo - r .. z_lo - 1) and the lowest r planes of the rank above (z_hi .. z_hi + r - 1).
 * Where the grid has no neighbour (zero Dirichlet ends of a non-periodic grid) the callback
 * leaves that ghost buffer untouched (it holds zeros); on a periodic grid the lowest and highest
 * ranks are neighbours (a single rank is its own neighbour). stream: the handle's cudaStream_t;
 * x_k is complete once the work queued on it before the call is, and the sweep that reads the
 * ghosts is queued on it after the call returns, so the callback orders its copies with that
 * stream (or synchronises it). Returns 0 on success; anything else ends the solve with
 * AAR_ERR_COMM. */
typedef int32_t (*aar_halo_fn)(void* ctx, const double* send_lo, const double* send_hi, double* recv_lo,
                               double* recv_hi, int64_t count, void* stream);

/* Sum buf[0 .. count-1] (device, FP64) over all ranks in place, every rank receiving the same
 * values (the one reduction of an Anderson step: ||b - A x_k||^2, the upper triangle of F^T F
 * and F^T f_k; and ||b||^2 once at the start). Ordered with `stream` as the halo exchange is.
 * Returns 0 on success; anything else ends the solve with AAR_ERR_COMM. */
typedef int32_t (*aar_allreduce_fn)(void* ctx, double* buf, int32_t count, void* stream);

typedef struct {
    void* ctx; /* passed back to both callbacks */
    aar_halo_fn halo;
    aar_allreduce_fn allreduce;
} aar_comm;

/* Create the handle of the slab [z_lo, z_hi) of the grid `global` (aar_stencil_desc: radius
 * 1..6, zero Dirichlet or periodic boundaries, Jacobi; tile hints ignored). The slab holds at
 * least `radius` planes, so that its ghost planes come from one neighbour each. The handle owns
 * its history ring and two ghost buffers of r nx ny doubles. stream: a cudaStream_t (NULL =
 * legacy default stream). AAR_ERR_INVALID_ARG for an invalid descriptor, z_lo < 0, z_hi > nz,
 * z_hi - z_lo < radius, or block Jacobi (block = 2). */
aar_status aar_dd_create(const aar_stencil_desc* global, int32_t z_lo, int32_t z_hi, void* stream,
                         aar_dd_handle* out);

/* Solve the global A x = b from x_0 = 0 with the plain FP64 method (Eq. 2-6): b, x are this
 * rank's slabs (device, nx ny (z_hi - z_lo) values each). Per iteration: the halo callback,
 * the fused sweep; at an Anderson step also the Gram pass, one allreduce callback of
 * 1 + c(c+1)/2 + c doubles, the pseudoinverse solve (identical on every rank, since the
 * reduced values are) and the update. params as for aar_solve (inner_tol, max_refine and flags
 * are not used; step_limit caps the iterations like max_iter). On AAR_OK x holds the first
 * Anderson iterate whose global relative residual is <= tol; on AAR_NOT_CONVERGED the last
 * iterate. AAR_ERR_COMM if a callback failed (the other ranks then fail in their own
 * callbacks); AAR_ERR_INVALID_ARG for NULL or host b / x, invalid params or a comm without
 * both callbacks. Synchronises the handle's stream before returning. */
aar_status aar_dd_solve(aar_dd_handle h, const double* b, double* x, const aar_params* params,
                        const aar_comm* comm, aar_info* info);

aar_status aar_dd_destroy(aar_dd_handle h);

#ifdef __cplusplus
}
#endif

#endif /* AAR_DD_H */

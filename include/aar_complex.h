/*
 * aar_complex.h -- C ABI of the complex-valued AAR solver (GB300, sm_103a).
 *
 * Sec. 2 of arXiv:1606.08740 states the method over the complex numbers: A, x, b (Eq. 1),
 * omega and beta complex, and the superscript T of Eq. 3 the conjugate transpose, so that
 *   x_{k+1} = x_k + omega f_k                                 if (k+1) mod p != 0,
 *   x_{k+1} = x_k + beta f_k - (X_k + beta F_k) pinv(F_k^H F_k) F_k^H f_k   otherwise,
 * with f_k = M^{-1} (b - A x_k) (Eq. 6) and X_k, F_k the last min(k, m) differences of iterates
 * and residuals (Eq. 4, 5). The operator is the one of the OF-DFT kernel-potential equation
 * (Eq. 7, Sec. 3.2):
 *   A = scale * (-(1/h^2)(Dxx + Dyy + Dzz)) + q I,
 * (D u)_i = sum_{k=-r..r} w[|k|] u_{i+k} along each axis, q = Q complex, scale = 1/(4 pi) in Eq. 7,
 * periodic in every axis (periodic = 1) or with zero Dirichlet ghosts (periodic = 0). M = D is
 * the stencil's centre coefficient, scale * (-3 w[0] / h^2) + q (Jacobi; the appendix runs of
 * Sec. 3.2). r_k = ||b - A x_k|| / ||b|| is evaluated only at Anderson steps. The Hermitian Gram
 * matrix is inverted as a Moore-Penrose pseudoinverse through its real symmetric 2c x 2c form
 * [[Re G, -Im G], [Im G, Re G]] (same eigenvalues, each twice), eigenvalues at or below
 * c * 2^-52 * lambda_max dropped.
 *
 * The mixed form (AAR_MIXED) runs FP32 AAR inner solves inside FP64 iterative refinement (see
 * aar_zcreate_stencil); it is not in the paper.
 *
 * Conventions (as in aar.h): every function returns an aar_status; vectors hold N = nx*ny*nz
 * complex values as interleaved (real, imaginary) FP64 pairs -- the layout of C99 double complex,
 * numpy complex128 and torch.complex128 -- at index (z*ny + y)*nx + x, 2N doubles in all.
 * "device" pointers are device memory of the handle's device; "device or host" pointers may be
 * either. A handle is used by one host thread at a time; its work runs on its stream and calls
 * that return results synchronise that stream. The handle owns its workspace.
 */
#ifndef AAR_COMPLEX_H
#define AAR_COMPLEX_H

#include <stdint.h>

#include "aar.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aar_zctx* aar_zhandle;

/* Complex stencil operator of Eq. 7 (see above). radius in [1, 6]; h > 0; scale > 0; q finite;
 * periodic 0 or 1; the centre coefficient scale * (-3 w[0] / h^2) + q must be nonzero.
 * block: the preconditioner M of Eq. 6. 0 or 1 = Jacobi (M = the centre coefficient); 2 = block
 * Jacobi with 2 x 2 x 2 boxes (the block Jacobi of Sec. 3.2's Helmholtz runs, each block solved
 * exactly): M = the diagonal blocks of A for the tiling of the grid by 2 x 2 x 2 boxes. Every block
 * is d I + c1 Q3 (d the complex centre coefficient, c1 = -scale w[1] / h^2, Q3 the cube graph),
 * applied in the cube's Walsh-Hadamard basis. Needs even sides, periodic sides of at least
 * radius + 2 and nonzero block eigenvalues d + c1 (3 - 2t), t = 0..3. */
typedef struct {
    int32_t nx, ny, nz, radius;
    double w[AAR_MAX_RADIUS + 1];
    double h, scale;
    double q_re, q_im;
    int32_t periodic;
    int32_t block;
} aar_zstencil_desc;

/* Solver parameters of Eq. 2-3 over C. */
typedef struct {
    double omega_re, omega_im; /* Richardson relaxation (paper default 0.6) */
    double beta_re, beta_im;   /* Anderson relaxation (paper default 0.6) */
    int32_t m;                 /* history length, 0..AAR_MAX_M (paper default 9) */
    int32_t p;                 /* Anderson period, >= 1 (paper default 8) */
    double tol;                /* stop when ||b - A x|| / ||b|| <= tol, tol >= 0 */
    int64_t max_iter;          /* cap on iterations (AAR_MIXED: inner iterations summed), >= 0 */
    double inner_tol;          /* AAR_MIXED: relative residual target of each FP32 inner solve, (0, 1) */
    int32_t max_refine;        /* AAR_MIXED: cap on FP64 refinements, >= 1 */
    int32_t reserved;          /* 0 */
} aar_zparams;

/* Defaults: omega = beta = 0.6, m = 9, p = 8 (Sec. 3), tol 1e-6 (the tolerance of the paper's
 * Helmholtz runs, Sec. 3.2), max_iter 100000, inner_tol 1e-3, max_refine 30. */
aar_status aar_zdefault_params(aar_zparams* p);

/* Create a solver for a complex stencil operator. precision: AAR_FP64 (all vectors and
 * arithmetic in FP64) or AAR_MIXED (FP32 AAR inner solves of A d = r inside FP64 iterative
 * refinement: r = b - A x in FP64, each inner solve from d = 0 with an empty history until its
 * relative residual is <= max(inner_tol, tol ||b|| / (2 ||r||)) at an Anderson step or has not
 * dropped 10% over 12 Anderson steps, then x += d in FP64; the solve ends when the FP64
 * ||b - A x|| / ||b|| <= tol). stream: a cudaStream_t (NULL = the legacy default stream).
 * AAR_ERR_INVALID_ARG for an invalid descriptor or precision. */
aar_status aar_zcreate_stencil(const aar_zstencil_desc* desc, int32_t precision, void* stream, aar_zhandle* out);

/* Solve A x = b. b: device or host, 2N doubles. x0: device or host, 2N doubles, or NULL for zeros.
 * x: device or host, 2N doubles (may alias x0). AAR_FP64: on AAR_OK x holds the first
 * Anderson-step iterate whose relative residual is <= tol, on AAR_NOT_CONVERGED the iterate
 * x_{max_iter}, on AAR_ERR_BREAKDOWN the iterate whose residual or extrapolation was not finite.
 * AAR_MIXED: x holds the FP64 iterate after the last refinement (AAR_OK once its FP64 residual is
 * <= tol). ||b|| == 0 returns x = 0 and AAR_OK after 0 iterations. info may be NULL (iterations,
 * anderson_steps and eigen_steps summed over inner solves; eigen_steps = Anderson steps whose
 * 2c x 2c solve needed the eigen-decomposition; rel_residual: the last r_k (AAR_FP64) or FP64
 * refinement residual (AAR_MIXED); ticks = iterations). AAR_ERR_INVALID_ARG: m outside
 * [0, AAR_MAX_M], p < 1, tol < 0, max_iter < 0, omega or beta not finite, inner_tol outside
 * (0, 1), max_refine < 1, NULL b or x. */
aar_status aar_zsolve(aar_zhandle h, const double* b, const double* x0, double* x, const aar_zparams* params,
                      aar_info* info);

/* y = A x (device pointers, 2N doubles each; y must not alias x). */
aar_status aar_zapply(aar_zhandle h, const double* x, double* y);

/* *rel = ||b - A x||_2 / ||b||_2 (device pointers; rel: host). */
aar_status aar_zrel_residual(aar_zhandle h, const double* b, const double* x, double* rel);

/* Time one kernel of the last aar_zsolve on this handle, as aar_profile_kernel does (kernel ids
 * AAR_K_SWEEP, AAR_K_SWEEP_ANDERSON, AAR_K_GRAM, AAR_K_UPDATE, AAR_K_FINALIZE, AAR_K_RESID64
 * for AAR_MIXED, and AAR_K_BLOCK for block = 2: the box solve with the Richardson update); the FP32 kernels of its last inner solve for AAR_MIXED; the Gram and the update
 * take the history length of the last Anderson step). *ms: mean per launch. Kernel outputs that
 * would overwrite the history go to scratch vectors. AAR_ERR_INVALID_ARG: no previous solve with
 * an Anderson step, launches < 1, unknown kernel; AAR_ERR_UNSUPPORTED: p = 1 for AAR_K_SWEEP,
 * AAR_K_RESID64 for AAR_FP64, AAR_K_GRAM with an empty history. */
aar_status aar_zprofile_kernel(aar_zhandle h, int32_t kernel, int32_t launches, float* ms);

aar_status aar_zdestroy(aar_zhandle h);

#ifdef __cplusplus
}
#endif

#endif /* AAR_COMPLEX_H */

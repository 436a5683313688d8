/*
 * aar_oracle.c -- plain, slow, FP64 CPU oracle of the Alternating Anderson-Richardson (AAR)
 * method (Suryanarayana, Pratapa, Pask, arXiv:1606.08740, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's CPU
 * baseline load this file. The CUDA solver never links, calls or includes it, and it shares
 * no code with the CUDA solver.
 *
 * Everything is IEEE FP64, compiled with -O2 -ffp-contract=off, sequential, with dot products
 * summed in index order. Each function cites the equation it follows.
 *
 * Readings of the paper that the paper leaves open (all listed in the design notes):
 *  - iteration index k starts at 0; the Anderson branch is taken when (k+1) mod p == 0 (Eq. 3);
 *  - the convergence check uses r_k = ||b - A x_k|| / ||b|| of the iterate x_k *before*
 *    extrapolation, evaluated only at Anderson steps (Sec. 2: one reduction gives r and F^T F);
 *  - the history at step k holds the last c = min(k, m) consecutive differences (Eq. 4, 5);
 *    columns with j < 0 are omitted (the footnote to Eq. 5);
 *  - (F^T F)^{-1} is the Moore-Penrose pseudoinverse (Sec. 3.2), eigenvalues
 *    lambda_i <= c * 2^-52 * lambda_max are dropped;
 *  - ||b|| == 0 returns x = 0 after 0 iterations;
 *  - complex systems (orz_*): the same loop over C, with F^H (conjugate transpose) in Eq. 3,
 *    inner products <a, b> = sum conj(a_i) b_i, complex omega and beta, and the pseudoinverse of
 *    the Hermitian Gram matrix taken through its real symmetric 2c x 2c form with the same
 *    eigenvalue cut c * 2^-52 * lambda_max.
 *
 * Parity status of each function (pins live in the CPU test suite):
 *  orc_op_apply, orc_op_diag, orc_sym_eig, orc_pinv_solve, orc_aar_solve: pinned;
 *  orc_block_apply, orc_aar_solve_block: pinned;
 *  orz_op_apply, orz_op_diag, orz_pinv_solve, orz_aar_solve: pinned;
 *  orz_block_apply, orz_aar_solve_block: pinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_RADIUS 6
#define ORC_MAX_M 64

enum { ORC_OK = 0, ORC_NOT_CONVERGED = 1, ORC_ERR_INVALID_ARG = -1, ORC_ERR_OOM = -2,
       ORC_ERR_BREAKDOWN = -4 };

/* Operator: kind 0 = constant-coefficient stencil (-lap_h + shift), kind 1 = CSR.
 * Stencil: (D2 u)_i = sum_{k=-r..r} w[|k|] u_{i+k} per axis, A = -(1/h^2) (D2x + D2y + D2z)
 * + shift I. Boundary: periodic == 0 reads every neighbour outside the interior as zero (zero
 * Dirichlet ghosts); periodic == 1 wraps every axis (index i+k taken modulo the axis length, as
 * in the periodic cells of the paper's Sec. 3.2/3.3 runs). Layout x fastest: index
 * (z*ny + y)*nx + x. */
typedef struct {
    int32_t kind;
    int32_t nx, ny, nz, radius;
    int32_t periodic;
    double w[ORC_MAX_RADIUS + 1];
    double h, shift;
    int32_t n;
    int64_t nnz;
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const double* val;
} orc_op;

typedef struct {
    int64_t iterations;
    int32_t anderson_steps;
    int32_t status;
    double rel_residual;
} orc_info;

/* Per-Anderson-step record: k, r_k, c, kept rank, and ||f_k - F gamma|| (the minimised
 * preconditioned residual of Sec. 2). Arrays of length cap, filled up to *count. */
typedef struct {
    int64_t cap;
    int64_t count;
    int64_t* k;
    double* r;
    int32_t* c;
    int32_t* rank;
    double* fmin;
} orc_trace;

int64_t orc_op_size(const orc_op* A) {
    if (A->kind == 0) return (int64_t)A->nx * A->ny * A->nz;
    return A->n;
}

static int64_t wrap(int64_t j, int64_t n) {
    int64_t q = j % n;
    return q < 0 ? q + n : q;
}

static double stencil_at(const orc_op* A, const double* x, int64_t ix, int64_t iy, int64_t iz) {
    /* (-1/h^2) * sum over axes of sum_{k=-r..r} w[|k|] x(neighbour) + shift * x(centre); a
     * neighbour outside the interior is zero (Dirichlet ghosts) or, for a periodic operator, the
     * point at its index modulo the axis length. */
    const int64_t nx = A->nx, ny = A->ny, nz = A->nz;
    const int r = A->radius;
    double lap = 0.0;
    for (int axis = 0; axis < 3; ++axis) {
        for (int k = -r; k <= r; ++k) {
            int64_t jx = ix, jy = iy, jz = iz;
            if (axis == 0) jx += k;
            else if (axis == 1) jy += k;
            else jz += k;
            if (A->periodic) {
                jx = wrap(jx, nx);
                jy = wrap(jy, ny);
                jz = wrap(jz, nz);
            } else if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) {
                continue;
            }
            double wk = A->w[k < 0 ? -k : k];
            lap += wk * x[(jz * ny + jy) * nx + jx];
        }
    }
    double xc = x[(iz * ny + iy) * nx + ix];
    return -lap / (A->h * A->h) + A->shift * xc;
}

/* y = A x (the operator of Eq. 1). */
void orc_op_apply(const orc_op* A, const double* x, double* y) {
    if (A->kind == 0) {
        for (int64_t iz = 0; iz < A->nz; ++iz)
            for (int64_t iy = 0; iy < A->ny; ++iy)
                for (int64_t ix = 0; ix < A->nx; ++ix)
                    y[(iz * A->ny + iy) * A->nx + ix] = stencil_at(A, x, ix, iy, iz);
    } else {
        for (int64_t i = 0; i < A->n; ++i) {
            double s = 0.0;
            for (int64_t e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e) s += A->val[e] * x[A->col_idx[e]];
            y[i] = s;
        }
    }
}

/* One entry (A x)_i, for sampled checks on grids too large to sweep here. */
double orc_op_apply_at(const orc_op* A, const double* x, int64_t i) {
    if (A->kind == 0) {
        int64_t ix = i % A->nx, iy = (i / A->nx) % A->ny, iz = i / ((int64_t)A->nx * A->ny);
        return stencil_at(A, x, ix, iy, iz);
    }
    double s = 0.0;
    for (int64_t e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e) s += A->val[e] * x[A->col_idx[e]];
    return s;
}

/* d = diag(A): the Jacobi preconditioner M = D of Sec. 2 (AAJ, M^{-1} = D^{-1}). */
void orc_op_diag(const orc_op* A, double* d) {
    if (A->kind == 0) {
        double dd = -3.0 * A->w[0] / (A->h * A->h) + A->shift;
        int64_t n = orc_op_size(A);
        for (int64_t i = 0; i < n; ++i) d[i] = dd;
    } else {
        for (int64_t i = 0; i < A->n; ++i) {
            d[i] = 0.0;
            for (int64_t e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e)
                if (A->col_idx[e] == i) d[i] += A->val[e];
        }
    }
}

/* Symmetric eigendecomposition S = V diag(lam) V^T by the cyclic Jacobi method: sweep over all
 * off-diagonal pairs (p, q) in row order and annihilate S_pq with a plane rotation. An entry
 * with |S_pq| <= 2^-52 sqrt(|S_pp S_qq|) is negligible at working precision: it is set to zero
 * and not rotated. The method stops after a sweep that rotated nothing (at most 100 sweeps).
 * S, V are c x c row-major; lam has c entries. Returns the number of sweeps used. */
int orc_sym_eig(int c, const double* S_in, double* lam, double* V) {
    double* S = (double*)malloc(sizeof(double) * (size_t)c * c + 1);
    memcpy(S, S_in, sizeof(double) * (size_t)c * c);
    for (int i = 0; i < c; ++i)
        for (int j = 0; j < c; ++j) V[i * c + j] = (i == j) ? 1.0 : 0.0;
    const double eps = ldexp(1.0, -52);
    int sweep = 0;
    for (; sweep < 100; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < c - 1; ++p) {
            for (int q = p + 1; q < c; ++q) {
                double apq = S[p * c + q];
                if (apq == 0.0) continue;
                double app = S[p * c + p], aqq = S[q * c + q];
                if (fabs(apq) <= eps * sqrt(fabs(app * aqq))) {
                    S[p * c + q] = 0.0;
                    S[q * c + p] = 0.0;
                    continue;
                }
                ++rotated;
                /* choose t = tan(theta) so that the rotated (p, q) entry vanishes:
                 * cot(2 theta) = (aqq - app) / (2 apq), smaller root of t^2 + 2 cot t - 1 = 0 */
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double cs = 1.0 / sqrt(t * t + 1.0);
                double sn = t * cs;
                /* S <- J^T S J with J the rotation in the (p, q) plane */
                for (int k = 0; k < c; ++k) {
                    double skp = S[k * c + p], skq = S[k * c + q];
                    S[k * c + p] = cs * skp - sn * skq;
                    S[k * c + q] = sn * skp + cs * skq;
                }
                for (int k = 0; k < c; ++k) {
                    double spk = S[p * c + k], sqk = S[q * c + k];
                    S[p * c + k] = cs * spk - sn * sqk;
                    S[q * c + k] = sn * spk + cs * sqk;
                }
                for (int k = 0; k < c; ++k) {
                    double vkp = V[k * c + p], vkq = V[k * c + q];
                    V[k * c + p] = cs * vkp - sn * vkq;
                    V[k * c + q] = sn * vkp + cs * vkq;
                }
            }
        }
        if (!rotated) break;
    }
    for (int i = 0; i < c; ++i) lam[i] = S[i * c + i];
    free(S);
    return sweep;
}

/* gamma = pinv(G) g with G symmetric positive semidefinite c x c (the (F^T F)^{-1} F^T f of
 * Eq. 3, taken as a Moore-Penrose pseudoinverse, Sec. 3.2). Eigenvalues lambda_i <= tau with
 * tau = c * 2^-52 * lambda_max are treated as zero. Writes the kept rank. */
int orc_pinv_solve(int c, const double* G, const double* g, double* gamma, int* rank) {
    if (c <= 0) {
        if (rank) *rank = 0;
        return ORC_OK;
    }
    double* lam = (double*)malloc(sizeof(double) * (size_t)c);
    double* V = (double*)malloc(sizeof(double) * (size_t)c * c);
    orc_sym_eig(c, G, lam, V);
    double lmax = 0.0;
    for (int i = 0; i < c; ++i)
        if (lam[i] > lmax) lmax = lam[i];
    double tau = (double)c * ldexp(1.0, -52) * lmax;
    int kept = 0;
    for (int i = 0; i < c; ++i) gamma[i] = 0.0;
    for (int j = 0; j < c; ++j) {
        if (!(lam[j] > tau) || lmax <= 0.0) continue;
        ++kept;
        double vg = 0.0; /* v_j . g */
        for (int i = 0; i < c; ++i) vg += V[i * c + j] * g[i];
        double coef = vg / lam[j];
        for (int i = 0; i < c; ++i) gamma[i] += V[i * c + j] * coef;
    }
    if (rank) *rank = kept;
    free(lam);
    free(V);
    return ORC_OK;
}

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Entry A_ij of a stencil operator: the sum of the taps of row i that land on column j (wrapped
 * for a periodic operator, so that taps wrapping onto the same point add up), plus shift on the
 * diagonal. i, j are grid indices (z*ny + y)*nx + x. */
static double stencil_entry(const orc_op* A, int64_t i, int64_t j) {
    const int64_t nx = A->nx, ny = A->ny, nz = A->nz;
    const int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
    const int r = A->radius;
    double v = (i == j) ? A->shift : 0.0;
    for (int axis = 0; axis < 3; ++axis) {
        for (int k = -r; k <= r; ++k) {
            int64_t jx = ix, jy = iy, jz = iz;
            if (axis == 0) jx += k;
            else if (axis == 1) jy += k;
            else jz += k;
            if (A->periodic) {
                jx = wrap(jx, nx);
                jy = wrap(jy, ny);
                jz = wrap(jz, nz);
            } else if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) {
                continue;
            }
            if ((jz * ny + jy) * nx + jx == j) v += -A->w[k < 0 ? -k : k] / (A->h * A->h);
        }
    }
    return v;
}

/* Solve the dense c x c system G y = g in place (G row-major, destroyed; y returned in g) by
 * Gaussian elimination with partial pivoting. Returns -1 on an exactly zero pivot. */
static int dense_solve(int c, double* G, double* g) {
    for (int k = 0; k < c; ++k) {
        int piv = k;
        for (int i = k + 1; i < c; ++i)
            if (fabs(G[i * c + k]) > fabs(G[piv * c + k])) piv = i;
        if (G[piv * c + k] == 0.0) return -1;
        if (piv != k) {
            for (int j = 0; j < c; ++j) {
                double t = G[k * c + j];
                G[k * c + j] = G[piv * c + j];
                G[piv * c + j] = t;
            }
            double t = g[k];
            g[k] = g[piv];
            g[piv] = t;
        }
        for (int i = k + 1; i < c; ++i) {
            double l = G[i * c + k] / G[k * c + k];
            for (int j = k; j < c; ++j) G[i * c + j] -= l * G[k * c + j];
            g[i] -= l * g[k];
        }
    }
    for (int k = c - 1; k >= 0; --k) {
        double s = g[k];
        for (int j = k + 1; j < c; ++j) s -= G[k * c + j] * g[j];
        g[k] = s / G[k * c + k];
    }
    return 0;
}

/* Block-Jacobi preconditioner (the block Jacobi of Sec. 3.2/3.3, with exact block solves in
 * place of ILU(0)): M = the diagonal blocks of A for the tiling of the grid by bs x bs x bs boxes
 * (box (X, Y, Z) holds the points with x / bs = X, y / bs = Y, z / bs = Z), f = M^{-1} r, each
 * block's system B f_B = r_B solved by Gaussian elimination with partial pivoting, B read entry
 * by entry from the operator. Stencil operators whose sides are multiples of bs. Returns
 * ORC_ERR_INVALID_ARG otherwise, ORC_ERR_BREAKDOWN on a singular block. */
int orc_block_apply(const orc_op* A, int bs, const double* r, double* f) {
    if (A->kind != 0 || bs < 1 || A->nx % bs || A->ny % bs || A->nz % bs) return ORC_ERR_INVALID_ARG;
    const int64_t nx = A->nx, ny = A->ny;
    const int c = bs * bs * bs;
    double* B = (double*)malloc(sizeof(double) * (size_t)c * c);
    double* v = (double*)malloc(sizeof(double) * (size_t)c);
    int64_t* id = (int64_t*)malloc(sizeof(int64_t) * (size_t)c);
    if (!B || !v || !id) {
        free(B); free(v); free(id);
        return ORC_ERR_OOM;
    }
    int st = ORC_OK;
    for (int64_t Z = 0; Z < A->nz; Z += bs)
        for (int64_t Y = 0; Y < ny; Y += bs)
            for (int64_t X = 0; X < nx; X += bs) {
                int t = 0;
                for (int dz = 0; dz < bs; ++dz)
                    for (int dy = 0; dy < bs; ++dy)
                        for (int dx = 0; dx < bs; ++dx) id[t++] = ((Z + dz) * ny + (Y + dy)) * nx + (X + dx);
                for (int a = 0; a < c; ++a) {
                    for (int bcol = 0; bcol < c; ++bcol) B[a * c + bcol] = stencil_entry(A, id[a], id[bcol]);
                    v[a] = r[id[a]];
                }
                if (dense_solve(c, B, v) != 0) st = ORC_ERR_BREAKDOWN;
                for (int a = 0; a < c; ++a) f[id[a]] = v[a];
            }
    free(B); free(v); free(id);
    return st;
}

/*
 * AAR solve of A x = b (Eq. 1) with left Jacobi preconditioning M^{-1} = diag(dinv) (Eq. 6):
 *   f_k     = M^{-1} (b - A x_k)                                        (Eq. 6)
 *   history: X_k, F_k = last c = min(k, m) differences of x and f       (Eq. 4, 5)
 *   x_{k+1} = x_k + omega f_k                      if (k+1) mod p != 0  (Eq. 2, 3 Richardson)
 *   x_{k+1} = x_k + beta f_k - (X_k + beta F_k) gamma,
 *             gamma = pinv(F_k^T F_k) F_k^T f_k    if (k+1) mod p == 0  (Eq. 2, 3 Anderson)
 * r_k = ||b - A x_k|| / ||b|| is evaluated only at Anderson steps; the solve stops there when
 * r_k <= tol and returns x_k (Sec. 2). After max_iter updates it returns x_{max_iter}.
 * dinv may be NULL (then 1/diag(A)). x0 may be NULL (zeros). trace may be NULL.
 */
static int aar_solve_impl(const orc_op* A, const double* dinv_in, int block, const double* b, const double* x0,
                          double* x_out, double omega, double beta, int m, int p, double tol,
                          int64_t max_iter, orc_info* info, orc_trace* trace) {
    const int64_t n = orc_op_size(A);
    if (n <= 0 || p < 1 || m < 0 || m > ORC_MAX_M || tol < 0.0 || max_iter < 0 || !b || !x_out)
        return ORC_ERR_INVALID_ARG;
    if (block > 1 && (dinv_in || A->kind != 0 || A->nx % block || A->ny % block || A->nz % block))
        return ORC_ERR_INVALID_ARG;
    info->iterations = 0;
    info->anderson_steps = 0;
    info->status = ORC_OK;
    info->rel_residual = 0.0;
    if (trace) trace->count = 0;

    double nb = sqrt(dot(n, b, b));
    if (nb == 0.0) {
        for (int64_t i = 0; i < n; ++i) x_out[i] = 0.0;
        return ORC_OK;
    }
    double* dinv = (double*)malloc(sizeof(double) * (size_t)n);
    double* x = (double*)malloc(sizeof(double) * (size_t)n);
    double* x_prev = (double*)malloc(sizeof(double) * (size_t)n);
    double* x_next = (double*)malloc(sizeof(double) * (size_t)n);
    double* res = (double*)malloc(sizeof(double) * (size_t)n);
    double* f = (double*)malloc(sizeof(double) * (size_t)n);
    double* f_prev = (double*)malloc(sizeof(double) * (size_t)n);
    double* Ax = (double*)malloc(sizeof(double) * (size_t)n);
    size_t hist_cols = m > 0 ? (size_t)m : 1;
    double* DX = (double*)malloc(sizeof(double) * (size_t)n * hist_cols); /* FIFO, oldest first */
    double* DF = (double*)malloc(sizeof(double) * (size_t)n * hist_cols);
    double G[ORC_MAX_M * ORC_MAX_M], g[ORC_MAX_M], gamma[ORC_MAX_M];
    if (!dinv || !x || !x_prev || !x_next || !res || !f || !f_prev || !Ax || !DX || !DF) {
        free(dinv); free(x); free(x_prev); free(x_next); free(res); free(f); free(f_prev);
        free(Ax); free(DX); free(DF);
        return ORC_ERR_OOM;
    }
    if (dinv_in) {
        memcpy(dinv, dinv_in, sizeof(double) * (size_t)n);
    } else {
        orc_op_diag(A, dinv);
        for (int64_t i = 0; i < n; ++i) dinv[i] = 1.0 / dinv[i];
    }
    for (int64_t i = 0; i < n; ++i) x[i] = x0 ? x0[i] : 0.0;

    int hist = 0; /* number of stored columns, <= m */
    int64_t k = 0;
    int status = ORC_NOT_CONVERGED;
    double r_last = NAN;
    int32_t anderson = 0;
    if (max_iter == 0) {
        memcpy(x_out, x, sizeof(double) * (size_t)n);
        info->status = ORC_NOT_CONVERGED;
        info->rel_residual = r_last;
        goto done;
    }
    for (;;) {
        /* Eq. 6: res = b - A x_k ; f_k = M^{-1} res (Jacobi, or block Jacobi for block > 1) */
        orc_op_apply(A, x, Ax);
        for (int64_t i = 0; i < n; ++i) {
            res[i] = b[i] - Ax[i];
            f[i] = dinv[i] * res[i];
        }
        if (block > 1 && orc_block_apply(A, block, res, f) != ORC_OK) {
            status = ORC_ERR_BREAKDOWN;
            memcpy(x_out, x, sizeof(double) * (size_t)n);
            break;
        }
        /* Eq. 4, 5: append (x_k - x_{k-1}, f_k - f_{k-1}), keep the newest m */
        if (k >= 1 && m >= 1) {
            if (hist == m) {
                memmove(DX, DX + n, sizeof(double) * (size_t)n * (size_t)(m - 1));
                memmove(DF, DF + n, sizeof(double) * (size_t)n * (size_t)(m - 1));
                --hist;
            }
            double* dx = DX + (size_t)hist * n;
            double* df = DF + (size_t)hist * n;
            for (int64_t i = 0; i < n; ++i) {
                dx[i] = x[i] - x_prev[i];
                df[i] = f[i] - f_prev[i];
            }
            ++hist;
        }
        if ((k + 1) % p != 0) {
            /* Eq. 3, Richardson branch: B_k = omega I */
            for (int64_t i = 0; i < n; ++i) x_next[i] = x[i] + omega * f[i];
        } else {
            /* Eq. 3, Anderson branch; r_k from the same residual (Sec. 2, Sec. 3.2) */
            double r = sqrt(dot(n, res, res)) / nb;
            r_last = r;
            ++anderson;
            if (!isfinite(r)) {
                status = ORC_ERR_BREAKDOWN;
                memcpy(x_out, x, sizeof(double) * (size_t)n);
                break;
            }
            int c = hist;
            int rank = 0;
            if (r <= tol) {
                if (trace && trace->count < trace->cap) {
                    int64_t t = trace->count++;
                    trace->k[t] = k; trace->r[t] = r; trace->c[t] = c; trace->rank[t] = -1;
                    trace->fmin[t] = NAN;
                }
                status = ORC_OK;
                memcpy(x_out, x, sizeof(double) * (size_t)n);
                break;
            }
            for (int a = 0; a < c; ++a) {
                for (int bcol = 0; bcol < c; ++bcol)
                    G[a * c + bcol] = dot(n, DF + (size_t)a * n, DF + (size_t)bcol * n);
                g[a] = dot(n, DF + (size_t)a * n, f);
            }
            orc_pinv_solve(c, G, g, gamma, &rank);
            int ok = 1;
            for (int a = 0; a < c; ++a) ok = ok && isfinite(gamma[a]);
            if (!ok) {
                status = ORC_ERR_BREAKDOWN;
                memcpy(x_out, x, sizeof(double) * (size_t)n);
                break;
            }
            double fmin2 = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                double corr = 0.0; /* sum_a gamma_a (dX_a + beta dF_a) */
                double fg = f[i];  /* (f_k - F gamma)_i */
                for (int a = 0; a < c; ++a) {
                    corr += gamma[a] * (DX[(size_t)a * n + i] + beta * DF[(size_t)a * n + i]);
                    fg -= gamma[a] * DF[(size_t)a * n + i];
                }
                x_next[i] = x[i] + beta * f[i] - corr;
                fmin2 += fg * fg;
            }
            if (trace && trace->count < trace->cap) {
                int64_t t = trace->count++;
                trace->k[t] = k; trace->r[t] = r; trace->c[t] = c; trace->rank[t] = rank;
                trace->fmin[t] = sqrt(fmin2);
            }
        }
        /* advance: x_{k-1} <- x_k, f_{k-1} <- f_k, x_k <- x_{k+1} */
        double* tmp = x_prev; x_prev = x; x = x_next; x_next = tmp;
        tmp = f_prev; f_prev = f; f = tmp;
        ++k;
        if (k >= max_iter) {
            status = ORC_NOT_CONVERGED;
            memcpy(x_out, x, sizeof(double) * (size_t)n);
            break;
        }
    }
    info->iterations = k;
    info->anderson_steps = anderson;
    info->status = status;
    info->rel_residual = r_last;
done:
    free(dinv); free(x); free(x_prev); free(x_next); free(res); free(f); free(f_prev);
    free(Ax); free(DX); free(DF);
    return info->status;
}

int orc_aar_solve(const orc_op* A, const double* dinv_in, const double* b, const double* x0,
                  double* x_out, double omega, double beta, int m, int p, double tol,
                  int64_t max_iter, orc_info* info, orc_trace* trace) {
    return aar_solve_impl(A, dinv_in, 0, b, x0, x_out, omega, beta, m, p, tol, max_iter, info, trace);
}

/* The same solve with the block-Jacobi preconditioner of orc_block_apply (block >= 2) in place of
 * the Jacobi M of Eq. 6 (block <= 1: Jacobi). */
int orc_aar_solve_block(const orc_op* A, int block, const double* b, const double* x0, double* x_out,
                        double omega, double beta, int m, int p, double tol, int64_t max_iter,
                        orc_info* info, orc_trace* trace) {
    return aar_solve_impl(A, NULL, block, b, x0, x_out, omega, beta, m, p, tol, max_iter, info, trace);
}

/* ||b - A x||_2 / ||b||_2 in FP64: the true relative residual used to certify any solution. */
double orc_rel_residual(const orc_op* A, const double* b, const double* x) {
    int64_t n = orc_op_size(A);
    double* Ax = (double*)malloc(sizeof(double) * (size_t)n);
    if (!Ax) return NAN;
    orc_op_apply(A, x, Ax);
    double s = 0.0, nb = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double ri = b[i] - Ax[i];
        s += ri * ri;
        nb += b[i] * b[i];
    }
    free(Ax);
    return sqrt(s) / sqrt(nb);
}

/* ======================================================================================
 * Complex-valued AAR (Sec. 2 states Eq. 1-6 over C: A, x, b, omega and beta complex, and the
 * superscript T in Eq. 3 is the conjugate transpose), with the operator of the OF-DFT Helmholtz
 * equation of Eq. 7. Vectors are arrays of C99 double complex (real and imaginary parts
 * interleaved, the layout of numpy complex128).
 * ====================================================================================== */
#include <complex.h>

typedef double complex zc;

/* Stencil operator of Eq. 7: A = scale * (-(1/h^2)(D2x + D2y + D2z)) + Q I with real weights
 * w[0..r] (D2 as in orc_op) and complex Q = q_re + i q_im; scale = 1/(4 pi) in Eq. 7. periodic as
 * in orc_op (Eq. 7's cells are periodic). */
typedef struct {
    int32_t nx, ny, nz, radius;
    int32_t periodic, pad;
    double w[ORC_MAX_RADIUS + 1];
    double h, scale;
    double q_re, q_im;
} orz_op;

int64_t orz_op_size(const orz_op* A) { return (int64_t)A->nx * A->ny * A->nz; }

static zc zstencil_at(const orz_op* A, const zc* x, int64_t ix, int64_t iy, int64_t iz) {
    const int64_t nx = A->nx, ny = A->ny, nz = A->nz;
    const int r = A->radius;
    zc lap = 0.0;
    for (int axis = 0; axis < 3; ++axis) {
        for (int k = -r; k <= r; ++k) {
            int64_t jx = ix, jy = iy, jz = iz;
            if (axis == 0) jx += k;
            else if (axis == 1) jy += k;
            else jz += k;
            if (A->periodic) {
                jx = wrap(jx, nx);
                jy = wrap(jy, ny);
                jz = wrap(jz, nz);
            } else if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) {
                continue;
            }
            lap += A->w[k < 0 ? -k : k] * x[(jz * ny + jy) * nx + jx];
        }
    }
    const zc q = A->q_re + A->q_im * I;
    return A->scale * (-lap / (A->h * A->h)) + q * x[(iz * ny + iy) * nx + ix];
}

/* y = A x (Eq. 1 with the operator of Eq. 7). */
void orz_op_apply(const orz_op* A, const zc* x, zc* y) {
    for (int64_t iz = 0; iz < A->nz; ++iz)
        for (int64_t iy = 0; iy < A->ny; ++iy)
            for (int64_t ix = 0; ix < A->nx; ++ix) y[(iz * A->ny + iy) * A->nx + ix] = zstencil_at(A, x, ix, iy, iz);
}

/* One entry (A x)_i, into *out. */
void orz_op_apply_at(const orz_op* A, const zc* x, int64_t i, zc* out) {
    int64_t ix = i % A->nx, iy = (i / A->nx) % A->ny, iz = i / ((int64_t)A->nx * A->ny);
    *out = zstencil_at(A, x, ix, iy, iz);
}

/* diag(A), the same complex value at every point: the Jacobi M = D (Eq. 6). */
static zc zdiag(const orz_op* A) {
    return A->scale * (-3.0 * A->w[0] / (A->h * A->h)) + (A->q_re + A->q_im * I);
}

void orz_op_diag(const orz_op* A, zc* out) { *out = zdiag(A); }

/* Entry A_ij of the operator of Eq. 7: scale * (-(1/h^2)) times the sum of the taps of row i that
 * land on column j (wrapped taps of a periodic operator adding up), plus Q on the diagonal. */
static zc zstencil_entry(const orz_op* A, int64_t i, int64_t j) {
    const int64_t nx = A->nx, ny = A->ny, nz = A->nz;
    const int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
    const int r = A->radius;
    double lap = 0.0;
    for (int axis = 0; axis < 3; ++axis) {
        for (int k = -r; k <= r; ++k) {
            int64_t jx = ix, jy = iy, jz = iz;
            if (axis == 0) jx += k;
            else if (axis == 1) jy += k;
            else jz += k;
            if (A->periodic) {
                jx = wrap(jx, nx);
                jy = wrap(jy, ny);
                jz = wrap(jz, nz);
            } else if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) {
                continue;
            }
            if ((jz * ny + jy) * nx + jx == j) lap += A->w[k < 0 ? -k : k];
        }
    }
    zc v = A->scale * (-lap / (A->h * A->h));
    if (i == j) v += A->q_re + A->q_im * I;
    return v;
}

/* Solve the dense complex c x c system G y = g in place (G row-major, destroyed; y returned in g)
 * by Gaussian elimination with partial pivoting on the modulus. Returns -1 on a zero pivot. */
static int zdense_solve(int c, zc* G, zc* g) {
    for (int k = 0; k < c; ++k) {
        int piv = k;
        for (int i = k + 1; i < c; ++i)
            if (cabs(G[i * c + k]) > cabs(G[piv * c + k])) piv = i;
        if (G[piv * c + k] == 0.0) return -1;
        if (piv != k) {
            for (int j = 0; j < c; ++j) {
                zc t = G[k * c + j];
                G[k * c + j] = G[piv * c + j];
                G[piv * c + j] = t;
            }
            zc t = g[k];
            g[k] = g[piv];
            g[piv] = t;
        }
        for (int i = k + 1; i < c; ++i) {
            zc l = G[i * c + k] / G[k * c + k];
            for (int j = k; j < c; ++j) G[i * c + j] -= l * G[k * c + j];
            g[i] -= l * g[k];
        }
    }
    for (int k = c - 1; k >= 0; --k) {
        zc s = g[k];
        for (int j = k + 1; j < c; ++j) s -= G[k * c + j] * g[j];
        g[k] = s / G[k * c + k];
    }
    return 0;
}

/* Block-Jacobi preconditioner for the operator of Eq. 7 (the block Jacobi of Sec. 3.2's
 * Helmholtz runs, with exact block solves): M = the diagonal blocks of A for the tiling of the
 * grid by bs x bs x bs boxes, f = M^{-1} r, each block's complex system solved by Gaussian
 * elimination, the block read entry by entry from the operator. Sides must be multiples of bs.
 * Returns ORC_ERR_INVALID_ARG otherwise, ORC_ERR_BREAKDOWN on a singular block. */
int orz_block_apply(const orz_op* A, int bs, const zc* r, zc* f) {
    if (bs < 1 || A->nx % bs || A->ny % bs || A->nz % bs) return ORC_ERR_INVALID_ARG;
    const int64_t nx = A->nx, ny = A->ny;
    const int c = bs * bs * bs;
    zc* B = (zc*)malloc(sizeof(zc) * (size_t)c * c);
    zc* v = (zc*)malloc(sizeof(zc) * (size_t)c);
    int64_t* id = (int64_t*)malloc(sizeof(int64_t) * (size_t)c);
    if (!B || !v || !id) {
        free(B); free(v); free(id);
        return ORC_ERR_OOM;
    }
    int st = ORC_OK;
    for (int64_t Z = 0; Z < A->nz; Z += bs)
        for (int64_t Y = 0; Y < ny; Y += bs)
            for (int64_t X = 0; X < nx; X += bs) {
                int t = 0;
                for (int dz = 0; dz < bs; ++dz)
                    for (int dy = 0; dy < bs; ++dy)
                        for (int dx = 0; dx < bs; ++dx) id[t++] = ((Z + dz) * ny + (Y + dy)) * nx + (X + dx);
                for (int a = 0; a < c; ++a) {
                    for (int bcol = 0; bcol < c; ++bcol) B[a * c + bcol] = zstencil_entry(A, id[a], id[bcol]);
                    v[a] = r[id[a]];
                }
                if (zdense_solve(c, B, v) != 0) st = ORC_ERR_BREAKDOWN;
                for (int a = 0; a < c; ++a) f[id[a]] = v[a];
            }
    free(B); free(v); free(id);
    return st;
}

/* gamma = pinv(G) g with G Hermitian positive semidefinite c x c (row-major): the
 * (F^H F)^{-1} F^H f of Eq. 3 as a Moore-Penrose pseudoinverse (Sec. 3.2). G acts on
 * (Re gamma, Im gamma) as the real symmetric 2c x 2c matrix [[Re G, -Im G], [Im G, Re G]], whose
 * eigenvalues are those of G, each twice; its pseudoinverse is that of G in the same form. It is
 * decomposed by orc_sym_eig, eigenvalues <= c * 2^-52 * lambda_max dropped as in the real case.
 * *rank = kept eigenvalues of the 2c x 2c form / 2. */
int orz_pinv_solve(int c, const zc* G, const zc* g, zc* gamma, int* rank) {
    if (c <= 0) {
        if (rank) *rank = 0;
        return ORC_OK;
    }
    const int c2 = 2 * c;
    double* S = (double*)malloc(sizeof(double) * (size_t)c2 * c2);
    double* V = (double*)malloc(sizeof(double) * (size_t)c2 * c2);
    double* lam = (double*)malloc(sizeof(double) * (size_t)c2);
    double* rhs = (double*)malloc(sizeof(double) * (size_t)c2);
    double* sol = (double*)malloc(sizeof(double) * (size_t)c2);
    if (!S || !V || !lam || !rhs || !sol) {
        free(S); free(V); free(lam); free(rhs); free(sol);
        return ORC_ERR_OOM;
    }
    for (int a = 0; a < c; ++a) {
        for (int b = 0; b < c; ++b) {
            const double gr = creal(G[a * c + b]), gi = cimag(G[a * c + b]);
            S[a * c2 + b] = gr;
            S[a * c2 + c + b] = -gi;
            S[(c + a) * c2 + b] = gi;
            S[(c + a) * c2 + c + b] = gr;
        }
        rhs[a] = creal(g[a]);
        rhs[c + a] = cimag(g[a]);
    }
    orc_sym_eig(c2, S, lam, V);
    double lmax = 0.0;
    for (int i = 0; i < c2; ++i)
        if (lam[i] > lmax) lmax = lam[i];
    const double tau = (double)c * ldexp(1.0, -52) * lmax;
    int kept = 0;
    for (int i = 0; i < c2; ++i) sol[i] = 0.0;
    for (int j = 0; j < c2; ++j) {
        if (!(lam[j] > tau) || lmax <= 0.0) continue;
        ++kept;
        double vg = 0.0;
        for (int i = 0; i < c2; ++i) vg += V[i * c2 + j] * rhs[i];
        const double coef = vg / lam[j];
        for (int i = 0; i < c2; ++i) sol[i] += V[i * c2 + j] * coef;
    }
    for (int a = 0; a < c; ++a) gamma[a] = sol[a] + sol[c + a] * I;
    if (rank) *rank = kept / 2;
    free(S); free(V); free(lam); free(rhs); free(sol);
    return ORC_OK;
}

/* <a, b> = sum_i conj(a_i) b_i in index order (the conjugate transpose of Eq. 3). */
static zc zdot(int64_t n, const zc* a, const zc* b) {
    zc s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    return s;
}

static double znorm(int64_t n, const zc* a) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return sqrt(s);
}

/*
 * Complex AAR solve of A x = b, step for step the loop of orc_aar_solve over C:
 *   f_k = D^{-1} (b - A x_k), D = diag(A)                               (Eq. 6)
 *   X_k, F_k: last c = min(k, m) differences of x and f                 (Eq. 4, 5)
 *   x_{k+1} = x_k + omega f_k                           (k+1) mod p != 0 (Eq. 2, 3)
 *   x_{k+1} = x_k + beta f_k - (X_k + beta F_k) gamma,
 *             gamma = pinv(F_k^H F_k) F_k^H f_k        (k+1) mod p == 0 (Eq. 2, 3)
 * with omega, beta complex; r_k = ||b - A x_k|| / ||b|| at Anderson steps only (Sec. 2).
 * x0 may be NULL (zeros); trace may be NULL (fmin = ||f_k - F_k gamma||).
 */
static int orz_aar_solve_impl(const orz_op* A, int block, const zc* b, const zc* x0, zc* x_out, double omega_re,
                              double omega_im, double beta_re, double beta_im, int m, int p, double tol,
                              int64_t max_iter, orc_info* info, orc_trace* trace) {
    const int64_t n = orz_op_size(A);
    if (n <= 0 || p < 1 || m < 0 || m > ORC_MAX_M || tol < 0.0 || max_iter < 0 || !b || !x_out)
        return ORC_ERR_INVALID_ARG;
    if (block >= 2 && (A->nx % block || A->ny % block || A->nz % block)) return ORC_ERR_INVALID_ARG;
    const zc omega = omega_re + omega_im * I, beta = beta_re + beta_im * I;
    info->iterations = 0;
    info->anderson_steps = 0;
    info->status = ORC_OK;
    info->rel_residual = 0.0;
    if (trace) trace->count = 0;
    const double nb = znorm(n, b);
    if (nb == 0.0) {
        for (int64_t i = 0; i < n; ++i) x_out[i] = 0.0;
        return ORC_OK;
    }
    const zc dinv = 1.0 / zdiag(A);
    zc* x = (zc*)malloc(sizeof(zc) * (size_t)n);
    zc* x_prev = (zc*)malloc(sizeof(zc) * (size_t)n);
    zc* x_next = (zc*)malloc(sizeof(zc) * (size_t)n);
    zc* res = (zc*)malloc(sizeof(zc) * (size_t)n);
    zc* f = (zc*)malloc(sizeof(zc) * (size_t)n);
    zc* f_prev = (zc*)malloc(sizeof(zc) * (size_t)n);
    zc* Ax = (zc*)malloc(sizeof(zc) * (size_t)n);
    const size_t hist_cols = m > 0 ? (size_t)m : 1;
    zc* DX = (zc*)malloc(sizeof(zc) * (size_t)n * hist_cols);
    zc* DF = (zc*)malloc(sizeof(zc) * (size_t)n * hist_cols);
    zc* G = (zc*)malloc(sizeof(zc) * hist_cols * hist_cols);
    zc* g = (zc*)malloc(sizeof(zc) * hist_cols);
    zc* gamma = (zc*)malloc(sizeof(zc) * hist_cols);
    if (!x || !x_prev || !x_next || !res || !f || !f_prev || !Ax || !DX || !DF || !G || !g || !gamma) {
        free(x); free(x_prev); free(x_next); free(res); free(f); free(f_prev); free(Ax);
        free(DX); free(DF); free(G); free(g); free(gamma);
        return ORC_ERR_OOM;
    }
    for (int64_t i = 0; i < n; ++i) x[i] = x0 ? x0[i] : 0.0;
    int hist = 0;
    int64_t k = 0;
    int status = ORC_NOT_CONVERGED;
    double r_last = NAN;
    int32_t anderson = 0;
    if (max_iter == 0) {
        memcpy(x_out, x, sizeof(zc) * (size_t)n);
        goto finish;
    }
    for (;;) {
        orz_op_apply(A, x, Ax); /* Eq. 6 */
        for (int64_t i = 0; i < n; ++i) {
            res[i] = b[i] - Ax[i];
            f[i] = dinv * res[i];
        }
        if (block >= 2 && orz_block_apply(A, block, res, f) != ORC_OK) { /* f = M^{-1} res, block Jacobi */
            status = ORC_ERR_BREAKDOWN;
            memcpy(x_out, x, sizeof(zc) * (size_t)n);
            break;
        }
        if (k >= 1 && m >= 1) { /* Eq. 4, 5 */
            if (hist == m) {
                memmove(DX, DX + n, sizeof(zc) * (size_t)n * (size_t)(m - 1));
                memmove(DF, DF + n, sizeof(zc) * (size_t)n * (size_t)(m - 1));
                --hist;
            }
            zc* dx = DX + (size_t)hist * n;
            zc* df = DF + (size_t)hist * n;
            for (int64_t i = 0; i < n; ++i) {
                dx[i] = x[i] - x_prev[i];
                df[i] = f[i] - f_prev[i];
            }
            ++hist;
        }
        if ((k + 1) % p != 0) {
            for (int64_t i = 0; i < n; ++i) x_next[i] = x[i] + omega * f[i]; /* Eq. 3, Richardson */
        } else {
            const double r = znorm(n, res) / nb; /* Sec. 2 */
            r_last = r;
            ++anderson;
            if (!isfinite(r)) {
                status = ORC_ERR_BREAKDOWN;
                memcpy(x_out, x, sizeof(zc) * (size_t)n);
                break;
            }
            const int c = hist;
            int rank = 0;
            if (r <= tol) {
                if (trace && trace->count < trace->cap) {
                    int64_t t = trace->count++;
                    trace->k[t] = k; trace->r[t] = r; trace->c[t] = c; trace->rank[t] = -1;
                    trace->fmin[t] = NAN;
                }
                status = ORC_OK;
                memcpy(x_out, x, sizeof(zc) * (size_t)n);
                break;
            }
            for (int a = 0; a < c; ++a) { /* Eq. 3: F^H F and F^H f */
                for (int bcol = 0; bcol < c; ++bcol) G[a * c + bcol] = zdot(n, DF + (size_t)a * n, DF + (size_t)bcol * n);
                g[a] = zdot(n, DF + (size_t)a * n, f);
            }
            orz_pinv_solve(c, G, g, gamma, &rank);
            int ok = 1;
            for (int a = 0; a < c; ++a) ok = ok && isfinite(creal(gamma[a])) && isfinite(cimag(gamma[a]));
            if (!ok) {
                status = ORC_ERR_BREAKDOWN;
                memcpy(x_out, x, sizeof(zc) * (size_t)n);
                break;
            }
            double fmin2 = 0.0;
            for (int64_t i = 0; i < n; ++i) { /* Eq. 3, Anderson */
                zc corr = 0.0, fg = f[i];
                for (int a = 0; a < c; ++a) {
                    corr += gamma[a] * (DX[(size_t)a * n + i] + beta * DF[(size_t)a * n + i]);
                    fg -= gamma[a] * DF[(size_t)a * n + i];
                }
                x_next[i] = x[i] + beta * f[i] - corr;
                fmin2 += creal(fg) * creal(fg) + cimag(fg) * cimag(fg);
            }
            if (trace && trace->count < trace->cap) {
                int64_t t = trace->count++;
                trace->k[t] = k; trace->r[t] = r; trace->c[t] = c; trace->rank[t] = rank;
                trace->fmin[t] = sqrt(fmin2);
            }
        }
        zc* tmp = x_prev; x_prev = x; x = x_next; x_next = tmp;
        tmp = f_prev; f_prev = f; f = tmp;
        ++k;
        if (k >= max_iter) {
            status = ORC_NOT_CONVERGED;
            memcpy(x_out, x, sizeof(zc) * (size_t)n);
            break;
        }
    }
finish:
    info->iterations = k;
    info->anderson_steps = anderson;
    info->status = status;
    info->rel_residual = r_last;
    free(x); free(x_prev); free(x_next); free(res); free(f); free(f_prev); free(Ax);
    free(DX); free(DF); free(G); free(g); free(gamma);
    return info->status;
}

int orz_aar_solve(const orz_op* A, const zc* b, const zc* x0, zc* x_out, double omega_re, double omega_im,
                  double beta_re, double beta_im, int m, int p, double tol, int64_t max_iter, orc_info* info,
                  orc_trace* trace) {
    return orz_aar_solve_impl(A, 0, b, x0, x_out, omega_re, omega_im, beta_re, beta_im, m, p, tol, max_iter, info,
                              trace);
}

/* The same loop with f_k = M^{-1} (b - A x_k) for the block-Jacobi M of orz_block_apply with boxes
 * of block^3 points (block >= 2; sides multiples of block). */
int orz_aar_solve_block(const orz_op* A, int block, const zc* b, const zc* x0, zc* x_out, double omega_re,
                        double omega_im, double beta_re, double beta_im, int m, int p, double tol, int64_t max_iter,
                        orc_info* info, orc_trace* trace) {
    if (block < 2) return ORC_ERR_INVALID_ARG;
    return orz_aar_solve_impl(A, block, b, x0, x_out, omega_re, omega_im, beta_re, beta_im, m, p, tol, max_iter,
                              info, trace);
}

/* ||b - A x||_2 / ||b||_2 in FP64 for the complex operator. */
double orz_rel_residual(const orz_op* A, const zc* b, const zc* x) {
    const int64_t n = orz_op_size(A);
    zc* r = (zc*)malloc(sizeof(zc) * (size_t)n);
    if (!r) return NAN;
    orz_op_apply(A, x, r);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    const double v = znorm(n, r) / znorm(n, b);
    free(r);
    return v;
}

// aar_complex.cu -- complex-valued AAR (Sec. 2 over C; the OF-DFT operator of Eq. 7), FP64.
//
// Five kernels make up the solve loop, all on the handle's stream:
//   k_zstencil<R, MODE>  the sweep: f_k = D^{-1}(b - A x_k) (Eq. 6) fused with the Richardson
//                        update x_{k+1} = x_k + omega f_k (Eq. 2, 3), or at an Anderson step with
//                        the ||b - A x_k||^2 partial sums (Sec. 2); also A x and ||b - A x||^2;
//   k_zgram              F^H F and F^H f_k (Eq. 3) from the raw residual ring, one pass;
//   k_zfinalize          one CTA: fixed-order sums, r_k, the pseudoinverse solve of the
//                        Hermitian Gram system through its real 2c x 2c form, the update's
//                        coefficients;
//   k_zupdate            x_{k+1} = x_k + beta f_k - (X + beta F) gamma (Eq. 3);
//   k_znorm              ||b||^2 partial sums.
// On this part FP64 runs at 1/64 of the FP32 rate, so the sweep, the Gram pass and the update
// are bound by FP64 instruction issue rather than by HBM; the kernels are written to issue as
// few FP64 instructions per point as the arithmetic allows (neighbour sums first, one multiply by
// each real stencil weight, complex products as two FMAs per component). Vectors are interleaved
// complex (double2); the history is a ring of raw iterates x_j and residuals f_j, the
// differences of Eq. 4, 5 being formed inside the Gram pass and folded into the update's
// coefficients.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <new>

#include "aar.h"
#include "aar_complex.h"
#include "aar_linalg.cuh"

namespace aar {
namespace {

constexpr int ZMAXM = AAR_MAX_M;
constexpr int ZLD = 2 * ZMAXM;  // leading dimension of the real 2c x 2c form (2c <= 32)
constexpr int ZMAXE = ZMAXM * (ZMAXM + 1) / 2 + ZMAXM;  // Gram entries (F^H F upper triangle + F^H f)
constexpr int GRAM_CH = 128;  // points per Gram chunk

enum { ZM_RICH = 0, ZM_AND = 1, ZM_APPLY = 2, ZM_RESID = 3 };
enum { ZS_RUN = 0, ZS_CONV = 1, ZS_BREAK = 2 };

// Operator of Eq. 7: (A x)_i = d x_i + sum_{k=1..r} ck[k] * (sum of the 6 neighbours at distance k),
// d = scale * (-3 w0 / h^2) + q, ck[k] = -scale * w[k] / h^2.
struct ZOp {
    int nx, ny, nz, radius, periodic;
    int64_t n;
    double ck[AAR_MAX_RADIUS + 1];
    double2 d, dinv;
};

struct ZState {
    double nb, r;
    int status, c, rank, kept2, eig;  // eig: the last Anderson step's solve took the eigen path
    double2 ax[ZMAXM + 1], af[ZMAXM + 1];  // x_{k+1} = x_k + beta f_k - sum_j (ax_j x_{k-c+j} + af_j f_{k-c+j})
};

struct ZCols {
    const double2* p[ZMAXM + 1];  // x or f of iterates k - c .. k
};

__device__ __forceinline__ int wrap_axis(int j, int n) {
    int q = j % n;
    return q < 0 ? q + n : q;
}

template <int NW>
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < NW; ++w) s += red[w];
    return s;  // thread 0
}

// ------------------------------------------------------------------------------- the sweep
// Block (32, 8) over an x-y tile, marching z over [z0, z0 + zc). Neighbour indices are wrapped
// (periodic) or flagged out of range (zero Dirichlet ghosts) once per thread and plane.
template <int R, int MODE>
__global__ void __launch_bounds__(256) k_zstencil(ZOp op, const double2* __restrict__ x, const double2* __restrict__ b,
                                                  double2* __restrict__ f, double2* __restrict__ xn,
                                                  double* __restrict__ part, double2 omega, int zc) {
    __shared__ double red[8];
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 8 + threadIdx.y;
    const int z0 = blockIdx.z * zc, z1 = min(op.nz, z0 + zc);
    const int nx = op.nx, ny = op.ny, nz = op.nz;
    const int64_t plane = (int64_t)nx * ny;
    double s2 = 0.0;
    if (ix < nx && iy < ny) {
        int xo[2 * R + 1];      // x of neighbour ix + k - R, or -1 outside the grid
        int64_t yo[2 * R + 1];  // row offset of neighbour iy + k - R, or -1
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) {
            const int jx = ix + k - R, jy = iy + k - R;
            if (op.periodic) {
                xo[k] = wrap_axis(jx, nx);
                yo[k] = (int64_t)wrap_axis(jy, ny) * nx;
            } else {
                xo[k] = (jx >= 0 && jx < nx) ? jx : -1;
                yo[k] = (jy >= 0 && jy < ny) ? (int64_t)jy * nx : -1;
            }
        }
        const int64_t row = (int64_t)iy * nx;
        for (int z = z0; z < z1; ++z) {
            int64_t zo[2 * R + 1];
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k) {
                const int jz = z + k - R;
                if (op.periodic) zo[k] = (int64_t)wrap_axis(jz, nz) * plane;
                else zo[k] = (jz >= 0 && jz < nz) ? (int64_t)jz * plane : -1;
            }
            const int64_t pz = (int64_t)z * plane;
            const int64_t c = pz + row + ix;
            const double2 xc = __ldg(x + c);
            double lr = 0.0, li = 0.0;
#pragma unroll
            for (int k = 1; k <= R; ++k) {
                double sr = 0.0, si = 0.0;
                const int km = R - k, kp = R + k;
                const int64_t nb6[6] = {xo[km] >= 0 ? pz + row + xo[km] : -1, xo[kp] >= 0 ? pz + row + xo[kp] : -1,
                                        yo[km] >= 0 ? pz + yo[km] + ix : -1, yo[kp] >= 0 ? pz + yo[kp] + ix : -1,
                                        zo[km] >= 0 ? zo[km] + row + ix : -1, zo[kp] >= 0 ? zo[kp] + row + ix : -1};
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    if (nb6[q] >= 0) {
                        const double2 v = __ldg(x + nb6[q]);
                        sr += v.x;
                        si += v.y;
                    }
                }
                if (k == 1) {
                    lr = op.ck[1] * sr;
                    li = op.ck[1] * si;
                } else {
                    lr = fma(op.ck[k], sr, lr);
                    li = fma(op.ck[k], si, li);
                }
            }
            // (A x)_c = d x_c + lap
            double axr = fma(op.d.x, xc.x, lr);
            axr = fma(-op.d.y, xc.y, axr);
            double axi = fma(op.d.x, xc.y, li);
            axi = fma(op.d.y, xc.x, axi);
            if (MODE == ZM_APPLY) {
                f[c] = make_double2(axr, axi);
                continue;
            }
            const double2 bv = __ldg(b + c);
            const double rr = bv.x - axr, ri = bv.y - axi;
            if (MODE == ZM_RESID) {
                s2 = fma(rr, rr, fma(ri, ri, s2));
                continue;
            }
            // f = D^{-1} res (Eq. 6)
            const double fr = fma(op.dinv.x, rr, -op.dinv.y * ri);
            const double fi = fma(op.dinv.x, ri, op.dinv.y * rr);
            f[c] = make_double2(fr, fi);
            if (MODE == ZM_AND) {
                s2 = fma(rr, rr, fma(ri, ri, s2));
            } else {
                // x_{k+1} = x_k + omega f_k (Eq. 2, 3)
                const double xr = fma(omega.x, fr, fma(-omega.y, fi, xc.x));
                const double xi = fma(omega.x, fi, fma(omega.y, fr, xc.y));
                xn[c] = make_double2(xr, xi);
            }
        }
    }
    if (MODE == ZM_AND || MODE == ZM_RESID) {
        const double t = block_sum<8>(s2, red);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            part[((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
    }
}

// ----------------------------------------------------------------------------- ||b||^2
__global__ void __launch_bounds__(256) k_znorm(const double2* __restrict__ b, int64_t n, double* __restrict__ part) {
    __shared__ double red[8];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const double2 v = b[i];
        s = fma(v.x, v.x, fma(v.y, v.y, s));
    }
    const double t = block_sum<8>(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// -------------------------------------------------------------------------------- Gram
// Per CTA: chunks of GRAM_CH points of f_{k-c} .. f_k staged in shared memory, differenced in
// place (column a <- f_{k-c+a+1} - f_{k-c+a}, the columns of F_k in Eq. 5; column c keeps f_k),
// then each Gram entry (the upper triangle of F^H F and F^H f_k) is accumulated by 256 / E
// threads over strided points. Partial sums per CTA, combined in a fixed order by the finalize.
__global__ void __launch_bounds__(256) k_zgram(ZCols cols, int c, int64_t n, double* __restrict__ part) {
    __shared__ double2 sd[(ZMAXM + 1) * GRAM_CH];
    __shared__ unsigned char ea[ZMAXE], eb[ZMAXE];
    __shared__ double2 red[256];
    const int tid = threadIdx.x;
    const int E = c * (c + 1) / 2 + c;
    if (tid == 0) {
        int e = 0;
        for (int a = 0; a < c; ++a)
            for (int bb = a; bb < c; ++bb) {
                ea[e] = (unsigned char)a;
                eb[e] = (unsigned char)bb;
                ++e;
            }
        for (int a = 0; a < c; ++a) {
            ea[e] = (unsigned char)a;
            eb[e] = (unsigned char)c;
            ++e;
        }
    }
    __syncthreads();
    const int T = 256 / E;
    const int e = tid / T, sub = tid - e * T;
    const bool act = e < E;
    const int ca = act ? ea[e] : 0, cb = act ? eb[e] : 0;
    double accr = 0.0, acci = 0.0;
    const int64_t nch = (n + GRAM_CH - 1) / GRAM_CH;
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        const int64_t base = ch * GRAM_CH;
        __syncthreads();  // the previous chunk's products are done
        for (int idx = tid; idx < (c + 1) * GRAM_CH; idx += 256) {
            const int col = idx / GRAM_CH, pt = idx - col * GRAM_CH;
            const int64_t i = base + pt;
            sd[idx] = i < n ? cols.p[col][i] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        if (tid < GRAM_CH) {
            for (int a = 0; a < c; ++a) {
                const double2 u = sd[a * GRAM_CH + tid], v = sd[(a + 1) * GRAM_CH + tid];
                sd[a * GRAM_CH + tid] = make_double2(v.x - u.x, v.y - u.y);
            }
        }
        __syncthreads();
        if (act) {
            const double2* U = sd + ca * GRAM_CH;
            const double2* V = sd + cb * GRAM_CH;
            for (int pt = sub; pt < GRAM_CH; pt += T) {
                const double2 u = U[pt], v = V[pt];
                // conj(u) v
                accr = fma(u.x, v.x, accr);
                accr = fma(u.y, v.y, accr);
                acci = fma(u.x, v.y, acci);
                acci = fma(-u.y, v.x, acci);
            }
        }
    }
    red[tid] = make_double2(accr, acci);
    __syncthreads();
    if (tid < E) {
        double sr = 0.0, si = 0.0;
        for (int s = 0; s < T; ++s) {
            sr += red[tid * T + s].x;
            si += red[tid * T + s].y;
        }
        part[(int64_t)blockIdx.x * 2 * E + 2 * tid] = sr;
        part[(int64_t)blockIdx.x * 2 * E + 2 * tid + 1] = si;
    }
}

// ---------------------------------------------------------------------------- finalize
// mode 0: ||b|| from the k_znorm partials; mode 1: an Anderson step (r_k, convergence, gamma and
// the update's coefficients); mode 2: ||b - A x|| / ||b|| from the ZM_RESID and k_znorm partials
// (into r).
__global__ void __launch_bounds__(256) k_zfinalize(ZState* st, const double* __restrict__ part_r, int nr,
                                                   const double* __restrict__ part_g, int ng,
                                                   const double* __restrict__ part_b, int nbp, int c, double tol,
                                                   double2 beta, int mode) {
    __shared__ double red[8];
    __shared__ double gs[2 * ZMAXE];
    __shared__ double Sm[ZLD * ZLD], Vm[ZLD * ZLD], Wm[ZLD * ZLD], Xm[ZLD * ZLD];
    __shared__ double rhs[ZLD], coef[ZLD], sol2[ZLD], dinvp[ZLD], trinv[ZLD], rot[4];
    __shared__ int s_go, s_ok, s_cert, s_kept;
    const int tid = threadIdx.x;
    double s = 0.0;
    for (int i = tid; i < nr; i += 256) s += part_r[i];
    const double tot = block_sum<8>(s, red);
    if (mode == 0) {
        if (tid == 0) {
            st->nb = sqrt(tot);
            st->r = nan("");
            st->status = ZS_RUN;
            st->rank = 0;
            st->c = 0;
            st->eig = 0;
        }
        return;
    }
    if (mode == 2) {
        double sb = 0.0;
        for (int i = tid; i < nbp; i += 256) sb += part_b[i];
        const double totb = block_sum<8>(sb, red);
        if (tid == 0) st->r = sqrt(tot) / sqrt(totb);
        return;
    }
    if (tid == 0) {
        const double r = sqrt(tot) / st->nb;
        st->r = r;
        st->c = c;
        int go = 0;
        if (!isfinite(r)) st->status = ZS_BREAK;
        else if (r <= tol) st->status = ZS_CONV;
        else go = 1;
        if (go && c == 0) {
            st->ax[0] = make_double2(0.0, 0.0);
            st->af[0] = make_double2(0.0, 0.0);
            st->rank = 0;
            st->kept2 = 0;
            st->eig = 0;
            go = 0;
        }
        s_go = go;
    }
    __syncthreads();
    if (!s_go) return;
    // fixed-order sums of the Gram partials: entry t over the CTAs of the Gram pass
    const int E = c * (c + 1) / 2 + c;
    for (int t = tid; t < 2 * E; t += 256) {
        double v = 0.0;
        for (int blk = 0; blk < ng; ++blk) v += part_g[(int64_t)blk * 2 * E + t];
        gs[t] = v;
    }
    __syncthreads();
    // real 2c x 2c form [[Re G, -Im G], [Im G, Re G]] and right-hand side [Re g; Im g]
    const int c2 = 2 * c;
    if (tid == 0) {
        int e = 0;
        for (int a = 0; a < c; ++a)
            for (int bb = a; bb < c; ++bb) {
                const double gr = gs[2 * e], gi = gs[2 * e + 1];  // G_ab = <dF_a, dF_b>, G_ba = conj(G_ab)
                Sm[a * ZLD + bb] = gr;
                Sm[bb * ZLD + a] = gr;
                Sm[(c + a) * ZLD + c + bb] = gr;
                Sm[(c + bb) * ZLD + c + a] = gr;
                Sm[a * ZLD + c + bb] = -gi;
                Sm[(c + bb) * ZLD + a] = -gi;
                Sm[(c + a) * ZLD + bb] = gi;
                Sm[bb * ZLD + c + a] = gi;
                ++e;
            }
        for (int a = 0; a < c; ++a) {
            rhs[a] = gs[2 * e];
            rhs[c + a] = gs[2 * e + 1];
            ++e;
        }
    }
    __syncthreads();
    // (1) LDL^T of a copy of the 2c x 2c form (lower triangle), all threads, with the certificate
    //     lambda_max / lambda_min <= trace(S) trace(S^-1) < 2^42 / c: every eigenvalue then lies
    //     2^10 above the pseudoinverse's cut c 2^-52 lambda_max, so pinv(S) = S^-1 and gamma is
    //     the plain solve. S^-1 = L^-T D^-1 L^-1 with L^-1 formed explicitly (Xm).
    for (int t = tid; t < c2 * c2; t += 256) {
        const int i = t / c2, j = t - (t / c2) * c2;
        Wm[i * ZLD + j] = Sm[i * ZLD + j];
        Xm[i * ZLD + j] = (i == j) ? 1.0 : 0.0;
    }
    if (tid == 0) s_ok = 1;
    __syncthreads();
    for (int k = 0; k < c2; ++k) {
        if (tid == 0) {
            const double dk = Wm[k * ZLD + k];
            const bool good = dk > 0.0 && isfinite(dk);
            if (!good) s_ok = 0;
            dinvp[k] = good ? recip_nr(dk) : 0.0;
        }
        __syncthreads();
        if (!s_ok) break;  // the flag is read after the barrier by every thread
        const int mm = c2 - k - 1;
        const double dik = dinvp[k];
        for (int t = tid; t < mm * mm; t += 256) {
            const int i = k + 1 + t / mm, j = k + 1 + t % mm;
            if (j <= i) Wm[i * ZLD + j] = fma(-Wm[i * ZLD + k] * dik, Wm[j * ZLD + k], Wm[i * ZLD + j]);
        }
        __syncthreads();
        for (int i = k + 1 + tid; i < c2; i += 256) Wm[i * ZLD + k] *= dik;
        __syncthreads();
    }
    if (s_ok) {
        // L^-1 by columns: row k of Xm is final at step k; rows r > k take - L_rk * X_k
        for (int k = 0; k < c2 - 1; ++k) {
            const int mm = c2 - k - 1;
            for (int t = tid; t < mm * (k + 1); t += 256) {
                const int r = k + 1 + t / (k + 1), i = t - (t / (k + 1)) * (k + 1);
                Xm[r * ZLD + i] = fma(-Wm[r * ZLD + k], Xm[k * ZLD + i], Xm[r * ZLD + i]);
            }
            __syncthreads();
        }
        if (tid < c2) {
            double q = 0.0, y = 0.0;
            for (int i = 0; i <= tid; ++i) {
                q = fma(Xm[tid * ZLD + i], Xm[tid * ZLD + i], q);
                y = fma(Xm[tid * ZLD + i], rhs[i], y);
            }
            trinv[tid] = q * dinvp[tid];  // row tid's share of trace(S^-1)
            coef[tid] = y * dinvp[tid];   // D^-1 L^-1 rhs
        }
        __syncthreads();
        if (tid == 0) {
            double t1 = 0.0, t2 = 0.0;
            for (int k = 0; k < c2; ++k) {
                t1 += Sm[k * ZLD + k];
                t2 += trinv[k];
            }
            const double prod = t1 * t2 * (double)c;
            s_cert = isfinite(prod) && prod < ldexp(1.0, 42);
        }
        __syncthreads();
        if (s_cert && tid < c2) {
            double g = 0.0;  // (L^-T z)_tid
            for (int k = tid; k < c2; ++k) g = fma(Xm[k * ZLD + tid], coef[k], g);
            sol2[tid] = g;
        }
    } else if (tid == 0) {
        s_cert = 0;
    }
    __syncthreads();
    // (2) otherwise the pseudoinverse through the eigen-decomposition (warp 0)
    if (!s_cert && tid < 32) {
        warp_sym_eig<ZLD>(c2, Sm, Vm, rot);
        const int lane = tid;
        double lmax = 0.0;
        for (int i = 0; i < c2; ++i) lmax = fmax(lmax, Sm[i * ZLD + i]);
        const double tau = (double)c * ldexp(1.0, -52) * lmax;
        if (lane < c2) {
            const double lam = Sm[lane * ZLD + lane];
            double cf = 0.0;
            if (lam > tau && lmax > 0.0) {
                double vg = 0.0;
                for (int i = 0; i < c2; ++i) vg += Vm[i * ZLD + lane] * rhs[i];
                cf = vg / lam;
            }
            coef[lane] = cf;
        }
        __syncwarp();
        double sl = 0.0;
        if (lane < c2)
            for (int j = 0; j < c2; ++j) sl += Vm[lane * ZLD + j] * coef[j];
        if (lane < c2) sol2[lane] = sl;
        int kept = 0;
        for (int j = 0; j < c2; ++j) kept += (Sm[j * ZLD + j] > tau && lmax > 0.0) ? 1 : 0;
        if (lane == 0) s_kept = kept;
    }
    __syncthreads();
    if (tid == 0) {
        const int kept = s_cert ? c2 : s_kept;
        bool ok = true;
        for (int i = 0; i < c2; ++i) ok = ok && isfinite(sol2[i]);
        if (!ok) {
            st->status = ZS_BREAK;
        } else {
            // gamma = sol2[0..c) + i sol2[c..2c); coefficient of x_{k-c+j}: gamma_{j-1} - gamma_j
            // (gamma_{-1} = gamma_c = 0)
            for (int j = 0; j <= c; ++j) {
                const double ar = (j > 0 ? sol2[j - 1] : 0.0) - (j < c ? sol2[j] : 0.0);
                const double ai = (j > 0 ? sol2[c + j - 1] : 0.0) - (j < c ? sol2[c + j] : 0.0);
                st->ax[j] = make_double2(ar, ai);
                st->af[j] = make_double2(beta.x * ar - beta.y * ai, beta.x * ai + beta.y * ar);
            }
            st->rank = kept / 2;
            st->kept2 = kept;
            st->eig = s_cert ? 0 : 1;
        }
    }
}

// ------------------------------------------------------------------------------ update
// x_{k+1} = x_k + beta f_k - sum_{j=0..c} (ax_j x_{k-c+j} + af_j f_{k-c+j}) (Eq. 3 with the
// differences of Eq. 4, 5 expanded). xout may be the slot of x_{k-c}: each element is read
// before it is written, by the same thread.
__global__ void __launch_bounds__(256) k_zupdate(const ZState* st, ZCols xs, ZCols fs, int c, double2* xout,
                                                 double2 beta, int64_t n, int force) {
    __shared__ double2 ax[ZMAXM + 1], af[ZMAXM + 1];
    __shared__ int run;
    if (threadIdx.x == 0) run = force || st->status == ZS_RUN;
    if (threadIdx.x <= c) {
        ax[threadIdx.x] = st->ax[threadIdx.x];
        af[threadIdx.x] = st->af[threadIdx.x];
    }
    __syncthreads();
    if (!run) return;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const double2 xk = xs.p[c][i], fk = fs.p[c][i];
        double vr = fma(beta.x, fk.x, fma(-beta.y, fk.y, xk.x));
        double vi = fma(beta.x, fk.y, fma(beta.y, fk.x, xk.y));
        for (int j = 0; j <= c; ++j) {
            const double2 xj = xs.p[j][i], fj = fs.p[j][i];
            const double2 a = ax[j], g = af[j];
            vr = fma(-a.x, xj.x, vr);
            vr = fma(a.y, xj.y, vr);
            vi = fma(-a.x, xj.y, vi);
            vi = fma(-a.y, xj.x, vi);
            vr = fma(-g.x, fj.x, vr);
            vr = fma(g.y, fj.y, vr);
            vi = fma(-g.x, fj.y, vi);
            vi = fma(-g.y, fj.x, vi);
        }
        xout[i] = make_double2(vr, vi);
    }
}

// ------------------------------------------------------------------------------- host
template <int R>
cudaError_t launch_zstencil_r(int mode, dim3 grid, cudaStream_t s, const ZOp& op, const double2* x,
                              const double2* b, double2* f, double2* xn, double* part, double2 om, int zc) {
    const dim3 blk(32, 8);
    switch (mode) {
        case ZM_RICH: k_zstencil<R, ZM_RICH><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc); break;
        case ZM_AND: k_zstencil<R, ZM_AND><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc); break;
        case ZM_APPLY: k_zstencil<R, ZM_APPLY><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc); break;
        default: k_zstencil<R, ZM_RESID><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_zstencil(int mode, dim3 grid, cudaStream_t s, const ZOp& op, const double2* x, const double2* b,
                            double2* f, double2* xn, double* part, double2 om, int zc) {
    switch (op.radius) {
        case 1: return launch_zstencil_r<1>(mode, grid, s, op, x, b, f, xn, part, om, zc);
        case 2: return launch_zstencil_r<2>(mode, grid, s, op, x, b, f, xn, part, om, zc);
        case 3: return launch_zstencil_r<3>(mode, grid, s, op, x, b, f, xn, part, om, zc);
        case 4: return launch_zstencil_r<4>(mode, grid, s, op, x, b, f, xn, part, om, zc);
        case 5: return launch_zstencil_r<5>(mode, grid, s, op, x, b, f, xn, part, om, zc);
        case 6: return launch_zstencil_r<6>(mode, grid, s, op, x, b, f, xn, part, om, zc);
        default: return cudaErrorInvalidValue;
    }
}

bool zis_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

aar_status zfail(cudaError_t e) {
    if (getenv("AAR_DEBUG")) fprintf(stderr, "aar (complex): CUDA error %d: %s\n", (int)e, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return AAR_ERR_OOM;
    }
    return AAR_ERR_CUDA;
}

#define ZCHECK(call)                                \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return zfail(e_);    \
    } while (0)

bool finite2(double a, double b) { return isfinite(a) && isfinite(b); }

}  // namespace
}  // namespace aar

using namespace aar;

struct aar_zctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    ZOp op{};
    int sms = 1;
    int64_t n = 0, ld = 0;  // ld: ring slot stride in complex values
    int sx_cap = 0, sf_cap = 0;
    double2* X = nullptr;
    double2* F = nullptr;
    double2* bstage = nullptr;
    double2* tmp = nullptr;  // scratch vector (residual checks)
    double* part_r = nullptr;
    double* part_b = nullptr;
    double* part_g = nullptr;
    ZState* d_st = nullptr;
    ZState* h_st = nullptr;
    dim3 sgrid;
    int zc = 16, nr = 0, nvec = 0, ngram = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // the last solve, for aar_zprofile_kernel
    bool solved = false;
    int64_t last_k = -1;
    int last_c = 0, last_sx = 2, last_sf = 1;
    aar_zparams last_p{};
    const double2* last_b = nullptr;
};

namespace {

aar_status zvalid_desc(const aar_zstencil_desc* d) {
    if (!d || d->nx <= 0 || d->ny <= 0 || d->nz <= 0 || d->radius < 1 || d->radius > AAR_MAX_RADIUS)
        return AAR_ERR_INVALID_ARG;
    if (!(d->h > 0.0) || !isfinite(d->h) || !(d->scale > 0.0) || !isfinite(d->scale)) return AAR_ERR_INVALID_ARG;
    if (!finite2(d->q_re, d->q_im) || (d->periodic != 0 && d->periodic != 1)) return AAR_ERR_INVALID_ARG;
    if ((int64_t)d->nx * d->ny >= ((int64_t)1 << 31)) return AAR_ERR_INVALID_ARG;
    for (int k = 0; k <= d->radius; ++k)
        if (!isfinite(d->w[k])) return AAR_ERR_INVALID_ARG;
    return AAR_OK;
}

bool zvalid_params(const aar_zparams* p) {
    return p && p->m >= 0 && p->m <= AAR_MAX_M && p->p >= 1 && p->tol >= 0.0 && isfinite(p->tol) &&
           p->max_iter >= 0 && finite2(p->omega_re, p->omega_im) && finite2(p->beta_re, p->beta_im);
}

double2 d2(double a, double b) { return make_double2(a, b); }

const double2* slot(const aar_zctx* h, const double2* base, int64_t k, int ns) {
    return base + (k % ns) * h->ld;
}

// Ring capacity for history length m: X holds x_{k-m} .. x_{k+1} (m + 1 slots, at least 2, as
// x_{k+1} takes the slot of x_{k-m}); F holds f_{k-m} .. f_k.
aar_status zensure(aar_zctx* h, int m) {
    const int sx = std::max(m + 1, 2), sf = std::max(m + 1, 1);
    if (sx > h->sx_cap) {
        cudaFree(h->X);
        h->X = nullptr;
        h->sx_cap = 0;
        ZCHECK(cudaMalloc(&h->X, sizeof(double2) * h->ld * sx));
        h->sx_cap = sx;
    }
    if (sf > h->sf_cap) {
        cudaFree(h->F);
        h->F = nullptr;
        h->sf_cap = 0;
        ZCHECK(cudaMalloc(&h->F, sizeof(double2) * h->ld * sf));
        h->sf_cap = sf;
    }
    return AAR_OK;
}

cudaError_t zgram(aar_zctx* h, int64_t k, int c, int sf) {
    ZCols cols{};
    for (int j = 0; j <= c; ++j) cols.p[j] = slot(h, h->F, k - c + j, sf);
    k_zgram<<<h->ngram, 256, 0, h->stream>>>(cols, c, h->n, h->part_g);
    return cudaGetLastError();
}

cudaError_t zupdate(aar_zctx* h, int64_t k, int c, int sx, int sf, double2 beta, double2* xout, int force) {
    ZCols xs{}, fs{};
    for (int j = 0; j <= c; ++j) {
        xs.p[j] = slot(h, h->X, k - c + j, sx);
        fs.p[j] = slot(h, h->F, k - c + j, sf);
    }
    k_zupdate<<<h->nvec, 256, 0, h->stream>>>(h->d_st, xs, fs, c, xout, beta, h->n, force);
    return cudaGetLastError();
}

cudaError_t zfinalize(aar_zctx* h, int nr_used, int c, double tol, double2 beta, int mode) {
    k_zfinalize<<<1, 256, 0, h->stream>>>(h->d_st, h->part_r, nr_used, h->part_g, h->ngram, h->part_b, h->nvec, c,
                                          tol, beta, mode);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

aar_status aar_zdefault_params(aar_zparams* p) {
    if (!p) return AAR_ERR_INVALID_ARG;
    p->omega_re = 0.6;
    p->omega_im = 0.0;
    p->beta_re = 0.6;
    p->beta_im = 0.0;
    p->m = 9;
    p->p = 8;
    p->tol = 1e-6;
    p->max_iter = 100000;
    return AAR_OK;
}

aar_status aar_zcreate_stencil(const aar_zstencil_desc* desc, int32_t precision, void* stream, aar_zhandle* out) {
    if (!out) return AAR_ERR_INVALID_ARG;
    *out = nullptr;
    const aar_status vs = zvalid_desc(desc);
    if (vs != AAR_OK) return vs;
    if (precision == AAR_MIXED) return AAR_ERR_UNSUPPORTED;
    if (precision != AAR_FP64) return AAR_ERR_INVALID_ARG;
    const double ih2 = 1.0 / (desc->h * desc->h);
    const std::complex<double> dd(desc->scale * (-3.0 * desc->w[0] * ih2) + desc->q_re, desc->q_im);
    if (dd == std::complex<double>(0.0, 0.0)) return AAR_ERR_INVALID_ARG;
    const std::complex<double> di = 1.0 / dd;
    if (!finite2(di.real(), di.imag())) return AAR_ERR_INVALID_ARG;

    aar_zctx* h = new (std::nothrow) aar_zctx();
    if (!h) return AAR_ERR_OOM;
    h->stream = (cudaStream_t)stream;
    ZOp& op = h->op;
    op.nx = desc->nx;
    op.ny = desc->ny;
    op.nz = desc->nz;
    op.radius = desc->radius;
    op.periodic = desc->periodic;
    op.n = (int64_t)desc->nx * desc->ny * desc->nz;
    for (int k = 0; k <= AAR_MAX_RADIUS; ++k) op.ck[k] = k <= desc->radius ? -desc->scale * desc->w[k] * ih2 : 0.0;
    op.d = d2(dd.real(), dd.imag());
    op.dinv = d2(di.real(), di.imag());
    h->n = op.n;
    h->ld = (op.n + 31) / 32 * 32;
    aar_status st = AAR_OK;
    auto fail = [&](aar_status s) {
        aar_zdestroy(h);
        return s;
    };
    if (cudaGetDevice(&h->dev) != cudaSuccess) return fail(AAR_ERR_CUDA);
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->dev);
    if (h->sms < 1) h->sms = 1;
    // z depth per CTA: up to 16 planes, fewer when the x-y tiles alone leave the SMs short of
    // about four CTAs each (small grids such as the 48^3 cell of Sec. 3.2)
    {
        const int64_t cols = (int64_t)((op.nx + 31) / 32) * ((op.ny + 7) / 8);
        const int64_t want = 4LL * h->sms;
        h->zc = (int)std::max<int64_t>(1, std::min<int64_t>(16, cols * op.nz / want));
    }
    h->sgrid = dim3((unsigned)((op.nx + 31) / 32), (unsigned)((op.ny + 7) / 8), (unsigned)((op.nz + h->zc - 1) / h->zc));
    if (h->sgrid.y > 65535u || h->sgrid.z > 65535u) return fail(AAR_ERR_INVALID_ARG);
    h->nr = (int)(h->sgrid.x * h->sgrid.y * h->sgrid.z);
    h->nvec = (int)std::max<int64_t>(1, std::min<int64_t>((op.n + 255) / 256, 8LL * h->sms));
    h->ngram = (int)std::max<int64_t>(1, std::min<int64_t>((op.n + GRAM_CH - 1) / GRAM_CH, 2LL * h->sms));
    if (cudaMalloc(&h->part_r, sizeof(double) * h->nr) != cudaSuccess ||
        cudaMalloc(&h->part_b, sizeof(double) * h->nvec) != cudaSuccess ||
        cudaMalloc(&h->part_g, sizeof(double) * 2 * ZMAXE * h->ngram) != cudaSuccess ||
        cudaMalloc(&h->d_st, sizeof(ZState)) != cudaSuccess ||
        cudaMallocHost(&h->h_st, sizeof(ZState)) != cudaSuccess ||
        cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
        cudaGetLastError();
        return fail(AAR_ERR_OOM);
    }
    (void)st;
    *out = h;
    return AAR_OK;
}

aar_status aar_zsolve(aar_zhandle h, const double* b, const double* x0, double* x, const aar_zparams* params,
                      aar_info* info) {
    if (info) {
        memset(info, 0, sizeof(*info));
        info->rel_residual = NAN;
    }
    if (!h || !b || !x || !zvalid_params(params)) {
        if (info) info->status = AAR_ERR_INVALID_ARG;
        return AAR_ERR_INVALID_ARG;
    }
    const aar_zparams P = *params;
    aar_status st = zensure(h, P.m);
    if (st != AAR_OK) return st;
    const int sx = std::max(P.m + 1, 2), sf = std::max(P.m + 1, 1);
    cudaStream_t s = h->stream;
    const int64_t n = h->n;
    int64_t launches = 0;
    // right-hand side: device pointer used in place, host memory staged
    const double2* bd = nullptr;
    if (zis_device_ptr(b)) {
        bd = reinterpret_cast<const double2*>(b);
    } else {
        if (!h->bstage) ZCHECK(cudaMalloc(&h->bstage, sizeof(double2) * h->ld));
        ZCHECK(cudaMemcpyAsync(h->bstage, b, sizeof(double2) * n, cudaMemcpyHostToDevice, s));
        bd = h->bstage;
    }
    const double2 omega = d2(P.omega_re, P.omega_im), beta = d2(P.beta_re, P.beta_im);
    // ||b||
    k_znorm<<<h->nvec, 256, 0, s>>>(bd, n, h->part_b);
    ZCHECK(cudaGetLastError());
    k_zfinalize<<<1, 256, 0, s>>>(h->d_st, h->part_b, h->nvec, h->part_g, 0, h->part_b, h->nvec, 0, P.tol, beta, 0);
    ZCHECK(cudaGetLastError());
    launches += 2;
    ZCHECK(cudaMemcpyAsync(h->h_st, h->d_st, sizeof(ZState), cudaMemcpyDeviceToHost, s));
    ZCHECK(cudaStreamSynchronize(s));
    const double nb = h->h_st->nb;
    h->solved = false;
    if (!isfinite(nb)) {
        if (info) info->status = AAR_ERR_BREAKDOWN;
        return AAR_ERR_BREAKDOWN;
    }
    if (nb == 0.0) {
        if (zis_device_ptr(x)) ZCHECK(cudaMemsetAsync(x, 0, sizeof(double2) * n, s));
        else memset(x, 0, sizeof(double2) * n);
        ZCHECK(cudaStreamSynchronize(s));
        if (info) {
            info->status = AAR_OK;
            info->rel_residual = 0.0;
            info->launches = launches;
        }
        return AAR_OK;
    }
    // x_0
    double2* X0 = h->X;
    if (x0) ZCHECK(cudaMemcpyAsync(X0, x0, sizeof(double2) * n, cudaMemcpyDefault, s));
    else ZCHECK(cudaMemsetAsync(X0, 0, sizeof(double2) * n, s));

    int64_t k = 0, k_final = 0;
    int status = AAR_NOT_CONVERGED, anderson = 0, eig = 0, rank = 0, last_c = 0;
    double r_last = NAN;
    int64_t last_and = -1;
    if (P.max_iter == 0) {
        k_final = 0;
    } else {
        for (;;) {
            const double2* xk = slot(h, h->X, k, sx);
            double2* fk = const_cast<double2*>(slot(h, h->F, k, sf));
            if ((k + 1) % P.p != 0) {
                double2* xn = const_cast<double2*>(slot(h, h->X, k + 1, sx));
                ZCHECK(launch_zstencil(ZM_RICH, h->sgrid, s, h->op, xk, bd, fk, xn, nullptr, omega, h->zc));
                ++launches;
            } else {
                const int c = (int)std::min<int64_t>(k, P.m);
                ZCHECK(launch_zstencil(ZM_AND, h->sgrid, s, h->op, xk, bd, fk, nullptr, h->part_r, omega, h->zc));
                ++launches;
                if (c > 0) {
                    ZCHECK(zgram(h, k, c, sf));
                    ++launches;
                }
                ZCHECK(zfinalize(h, h->nr, c, P.tol, beta, 1));
                ZCHECK(zupdate(h, k, c, sx, sf, beta, const_cast<double2*>(slot(h, h->X, k + 1, sx)), 0));
                launches += 2;
                ZCHECK(cudaMemcpyAsync(h->h_st, h->d_st, sizeof(ZState), cudaMemcpyDeviceToHost, s));
                ZCHECK(cudaStreamSynchronize(s));
                ++anderson;
                last_and = k;
                last_c = c;
                const ZState& R = *h->h_st;
                r_last = R.r;
                if (R.status == ZS_CONV) {
                    status = AAR_OK;
                    k_final = k;
                    break;
                }
                if (R.status == ZS_BREAK) {
                    status = AAR_ERR_BREAKDOWN;
                    k_final = k;
                    break;
                }
                if (c > 0 && R.eig) ++eig;
                rank = R.rank;
            }
            ++k;
            if (k >= P.max_iter) {
                status = AAR_NOT_CONVERGED;
                k_final = k;
                break;
            }
        }
    }
    ZCHECK(cudaMemcpyAsync(x, slot(h, h->X, k_final, sx), sizeof(double2) * n, cudaMemcpyDefault, s));
    ZCHECK(cudaStreamSynchronize(s));
    h->solved = last_and >= 0;
    h->last_k = last_and;
    h->last_c = last_c;
    h->last_sx = sx;
    h->last_sf = sf;
    h->last_p = P;
    h->last_b = bd;
    if (info) {
        info->iterations = k_final;
        info->anderson_steps = anderson;
        info->refinements = 0;
        info->rel_residual = r_last;
        info->status = status;
        info->last_rank = rank;
        info->ticks = k_final;
        info->launches = launches;
        info->eigen_steps = eig;
    }
    return (aar_status)status;
}

aar_status aar_zapply(aar_zhandle h, const double* x, double* y) {
    if (!h || !x || !y || x == y) return AAR_ERR_INVALID_ARG;
    if (!zis_device_ptr(x) || !zis_device_ptr(y)) return AAR_ERR_INVALID_ARG;
    ZCHECK(launch_zstencil(ZM_APPLY, h->sgrid, h->stream, h->op, reinterpret_cast<const double2*>(x), nullptr,
                           reinterpret_cast<double2*>(y), nullptr, nullptr, d2(0, 0), h->zc));
    ZCHECK(cudaStreamSynchronize(h->stream));
    return AAR_OK;
}

aar_status aar_zrel_residual(aar_zhandle h, const double* b, const double* x, double* rel) {
    if (!h || !b || !x || !rel) return AAR_ERR_INVALID_ARG;
    if (!zis_device_ptr(b) || !zis_device_ptr(x)) return AAR_ERR_INVALID_ARG;
    cudaStream_t s = h->stream;
    const double2* bd = reinterpret_cast<const double2*>(b);
    ZCHECK(launch_zstencil(ZM_RESID, h->sgrid, s, h->op, reinterpret_cast<const double2*>(x), bd, nullptr, nullptr,
                           h->part_r, d2(0, 0), h->zc));
    k_znorm<<<h->nvec, 256, 0, s>>>(bd, h->n, h->part_b);
    ZCHECK(cudaGetLastError());
    ZCHECK(zfinalize(h, h->nr, 0, 0.0, d2(0, 0), 2));
    ZCHECK(cudaMemcpyAsync(h->h_st, h->d_st, sizeof(ZState), cudaMemcpyDeviceToHost, s));
    ZCHECK(cudaStreamSynchronize(s));
    *rel = h->h_st->r;  // the ring and the update's coefficients are untouched
    return AAR_OK;
}

aar_status aar_zprofile_kernel(aar_zhandle h, int32_t kernel, int32_t launches, float* ms) {
    if (!h || !ms || launches < 1 || !h->solved) return AAR_ERR_INVALID_ARG;
    const aar_zparams& P = h->last_p;
    const int64_t k = h->last_k;
    const int c = h->last_c, sx = h->last_sx, sf = h->last_sf;
    const double2 omega = d2(P.omega_re, P.omega_im), beta = d2(P.beta_re, P.beta_im);
    cudaStream_t s = h->stream;
    if (kernel == AAR_K_SWEEP && P.p == 1) return AAR_ERR_UNSUPPORTED;
    if (kernel < AAR_K_SWEEP || kernel > AAR_K_FINALIZE || kernel == AAR_K_RESID64) return AAR_ERR_INVALID_ARG;
    if (kernel == AAR_K_GRAM && c == 0) return AAR_ERR_UNSUPPORTED;
    const double2* xk = slot(h, h->X, k, sx);
    double2* fk = const_cast<double2*>(slot(h, h->F, k, sf));
    // x_{k+1} of the timed sweep or update goes to a scratch vector, so the history of step k
    // stays intact (the sweeps rewrite f_k with the same values)
    if (!h->tmp) ZCHECK(cudaMalloc(&h->tmp, sizeof(double2) * h->ld));
    double2* xn = h->tmp;
    auto one = [&]() -> cudaError_t {
        switch (kernel) {
            case AAR_K_SWEEP: return launch_zstencil(ZM_RICH, h->sgrid, s, h->op, xk, h->last_b, fk, xn, nullptr, omega, h->zc);
            case AAR_K_SWEEP_ANDERSON:
                return launch_zstencil(ZM_AND, h->sgrid, s, h->op, xk, h->last_b, fk, nullptr, h->part_r, omega, h->zc);
            case AAR_K_GRAM: return zgram(h, k, c, sf);
            case AAR_K_UPDATE: return zupdate(h, k, c, sx, sf, beta, xn, 1);
            default: return zfinalize(h, h->nr, c, 0.0, beta, 1);
        }
    };
    ZCHECK(one());  // warm-up
    ZCHECK(cudaEventRecord(h->ev0, s));
    for (int i = 0; i < launches; ++i) ZCHECK(one());
    ZCHECK(cudaEventRecord(h->ev1, s));
    ZCHECK(cudaEventSynchronize(h->ev1));
    float t = 0.f;
    ZCHECK(cudaEventElapsedTime(&t, h->ev0, h->ev1));
    *ms = t / launches;
    return AAR_OK;
}

aar_status aar_zdestroy(aar_zhandle h) {
    if (!h) return AAR_ERR_INVALID_ARG;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    cudaFree(h->X);
    cudaFree(h->F);
    cudaFree(h->bstage);
    cudaFree(h->tmp);
    cudaFree(h->part_r);
    cudaFree(h->part_b);
    cudaFree(h->part_g);
    cudaFree(h->d_st);
    if (h->h_st) cudaFreeHost(h->h_st);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    cudaGetLastError();
    delete h;
    return AAR_OK;
}

}  // extern "C"

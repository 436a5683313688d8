// aar_complex.cu -- complex-valued AAR (Sec. 2 over C; the OF-DFT operator of Eq. 7).
//
// Kernels of the solve loop, all on the handle's stream:
//   k_zstencil<T, R, MODE>  the sweep: f_k = D^{-1}(b - A x_k) (Eq. 6) fused with the Richardson
//                           update x_{k+1} = x_k + omega f_k (Eq. 2, 3), or at an Anderson step with
//                           the ||b - A x_k||^2 partial sums (Sec. 2); also A x, ||b - A x||^2 and
//                           (mixed form) the FP64 residual handed to the FP32 inner solve;
//   k_zsweep_sm<R, MODE>    the FP32 sweep of the mixed form's inner solves: in-plane tiles staged
//                           in shared memory, the z column in a register queue turned by renaming
//                           (k_zstencil<float, ...> with AAR_ZSWEEP_REG=1);
//   k_zgram<T, NJ>          F^H F and F^H f_k (Eq. 3) from the raw residual ring, one pass
//                           (FP32: k_zgram_bulk<C>, fed by bulk copies; k_zgram_reg<C> with
//                           AAR_ZGRAM_REG=1);
//   k_zfinalize             one CTA: fixed-order sums, r_k, the pseudoinverse solve of the
//                           Hermitian Gram system through its real 2c x 2c form, the update's
//                           coefficients;
//   k_zupdate<T>            x_{k+1} = x_k + beta f_k - (X + beta F) gamma (Eq. 3); FP32: Richardson
//                           differences taken as omega f_i, so fewer x columns are read;
//   k_znorm, k_zadd         ||b||^2 partial sums; x64 += d (mixed form).
// T = double is the plain method. T = float is the mixed form's inner solve: FP32 AAR on
// A d = r inside FP64 iterative refinement (r = b - A x in FP64, x += d in FP64), the Anderson
// history restarted at every refinement. On this part FP64 runs at 1/64 of the FP32 rate: the
// FP64 kernels are bound by FP64 instruction issue and written to issue as few FP64
// instructions per point as the arithmetic allows (neighbour sums first, one multiply by each
// real stencil weight, complex products as two FMAs per component); the FP32 sweep and update
// are bound by HBM (the FP32 sweep also by instruction issue and the load/store pipe). Vectors are
// interleaved complex (double2 / float2); the history is a ring of raw iterates x_j and residuals
// f_j, the differences of Eq. 4, 5 being formed inside the Gram pass and folded into the update's
// coefficients.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <new>
#include <utility>

#include "aar.h"
#include "aar_fp64.cuh"
#include "aar_complex.h"
#include "aar_linalg.cuh"
#include "aar_mbar.cuh"

namespace aar {
namespace {

constexpr int ZMAXM = AAR_MAX_M;
constexpr int ZLD = 2 * ZMAXM;  // leading dimension of the real 2c x 2c form (2c <= 32)
constexpr int ZMAXE = ZMAXM * (ZMAXM + 1) / 2 + ZMAXM;  // Gram entries (F^H F upper triangle + F^H f)
constexpr int GRAM_CH = 128;  // points per Gram chunk
constexpr int GRAM_OCC_MAX = 8;  // Gram partial-sum slots per SM

// sweep modes; ZM_BRES / ZM_BRES_AND: the block-Jacobi sweep of a Richardson / Anderson step,
// writing b - A x_k into f (and at an Anderson step its norm) for k_zblock
enum { ZM_RICH = 0, ZM_AND = 1, ZM_APPLY = 2, ZM_RESID = 3, ZM_RESOUT = 4, ZM_BRES = 5, ZM_BRES_AND = 6 };
enum { ZS_RUN = 0, ZS_CONV = 1, ZS_BREAK = 2 };

// Operator of Eq. 7: (A x)_i = d x_i + sum_{k=1..r} ck[k] * (sum of the 6 neighbours at distance k),
// d = scale * (-3 w0 / h^2) + q, ck[k] = -scale * w[k] / h^2.
struct ZOp {
    int nx, ny, nz, radius, periodic;
    int64_t n;
    double ck[AAR_MAX_RADIUS + 1];
    double2 d, dinv;
    // block Jacobi with 2 x 2 x 2 boxes (blk = 1): M^{-1} = H diag(mu_|s|) H, mu_t = 1 / (8 lambda_t),
    // lambda_t = d + ck[1] (3 - 2t) (complex); the sweep then writes b - A x into f, k_zblock scales it
    int blk;
    double2 mu[4];
};

struct ZState {
    double nb, r;
    int status, c, rank, kept2, eig;  // eig: the last Anderson step's solve took the eigen path
    int err[4];  // a bounded wait in a bulk-fed kernel gave up (err[0] != 0): where, parity, barrier
    double2 ax[ZMAXM + 1], af[ZMAXM + 1];  // x_{k+1} = x_k + beta f_k - sum_j (ax_j x_{k-c+j} + af_j f_{k-c+j})
    double2 gam[ZMAXM];                     // gamma of the last Anderson step (the FP32 update's compressed form)
};

template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
    using type = double2;
};
template <>
struct Vec2<float> {
    using type = float2;
};
template <typename T>
using V2 = typename Vec2<T>::type;

template <typename T>
__host__ __device__ __forceinline__ V2<T> mk2(T a, T b) {
    V2<T> v;
    v.x = a;
    v.y = b;
    return v;
}

// Component-wise complex-pair arithmetic: the two FP32 lanes of a float2 in one paired
// instruction (sm_100 family), plain scalar operations for FP64. Each component is rounded as the
// scalar operation would round it.
// the sweep's neighbour sums: FP64 additions as FMAs with a unit multiplier (aar_fp64.cuh)
__device__ __forceinline__ float2 uadd2(float2 a, float2 b, float) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 uadd2(double2 a, double2 b, double one) {
    return make_double2(fma(a.x, one, b.x), fma(a.y, one, b.y));
}
__device__ __forceinline__ float2 scl2(float c, float2 a) { return __fmul2_rn(make_float2(c, c), a); }
__device__ __forceinline__ double2 scl2(double c, double2 a) { return make_double2(c * a.x, c * a.y); }
__device__ __forceinline__ float2 fma2(float c, float2 a, float2 acc) { return __ffma2_rn(make_float2(c, c), a, acc); }
__device__ __forceinline__ double2 fma2(double c, double2 a, double2 acc) {
    return make_double2(fma(c, a.x, acc.x), fma(c, a.y, acc.y));
}

template <typename T>
struct ZCols {
    const V2<T>* p[ZMAXM + 1];  // x or f of iterates k - c .. k
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
// (periodic) or flagged out of range (zero Dirichlet ghosts) once per thread and plane. The
// squared-residual sums of a thread (at most 16 points) are kept in T and reduced in FP64.
template <typename T, int R, int MODE>
__global__ void __launch_bounds__(256) k_zstencil(ZOp op, const V2<T>* __restrict__ x, const V2<T>* __restrict__ b,
                                                  V2<T>* __restrict__ f, V2<T>* __restrict__ xn,
                                                  double* __restrict__ part, double2 omega_d, int zc,
                                                  float2* __restrict__ rout) {
    __shared__ double red[8];
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 8 + threadIdx.y;
    const int z0 = blockIdx.z * zc, z1 = min(op.nz, z0 + zc);
    const int nx = op.nx, ny = op.ny, nz = op.nz;
    const int64_t plane = (int64_t)nx * ny;
    const T dr = (T)op.d.x, di = (T)op.d.y, vr = (T)op.dinv.x, vi = (T)op.dinv.y;
    const T omr = (T)omega_d.x, omi = (T)omega_d.y;
    const T one = sizeof(T) == 8 ? (T)unit_one() : T(1);
    T s2 = 0;
    if (ix < nx && iy < ny) {
        // in-plane offsets of the x and y neighbours at -R .. R (index k + R), -1 outside the grid;
        // a plane holds fewer than 2^31 points, so in-plane offsets are 32-bit
        const int oc = iy * nx + ix;
        int ox[2 * R + 1], oy[2 * R + 1];
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) {
            const int jx = ix + k - R, jy = iy + k - R;
            if (op.periodic) {
                ox[k] = iy * nx + wrap_axis(jx, nx);
                oy[k] = wrap_axis(jy, ny) * nx + ix;
            } else {
                ox[k] = (jx >= 0 && jx < nx) ? iy * nx + jx : -1;
                oy[k] = (jy >= 0 && jy < ny) ? jy * nx + ix : -1;
            }
        }
        // z column x(ix, iy, z - R .. z + R) in registers (zero outside a Dirichlet grid), and the
        // plane index of z + R, advanced one plane per step: each step loads one new z value
        V2<T> q[2 * R + 1];
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) {
            const int jz = z0 + k - R;
            const int zi = op.periodic ? wrap_axis(jz, nz) : ((jz >= 0 && jz < nz) ? jz : -1);
            q[k] = zi >= 0 ? __ldg(x + (int64_t)zi * plane + oc) : mk2<T>(0, 0);
        }
        // the next plane's new z value and right-hand side are loaded one step ahead
        auto zval = [&](int jz) -> V2<T> {
            const int zi = op.periodic ? (jz >= nz ? wrap_axis(jz, nz) : jz) : (jz < nz ? jz : -1);
            return zi >= 0 ? __ldg(x + (int64_t)zi * plane + oc) : mk2<T>(0, 0);
        };
        const bool need_b = MODE != ZM_APPLY;
        T ckt[R + 1];  // the weights in T, converted once (an FP64 -> FP32 conversion uses the FP64 pipe)
#pragma unroll
        for (int k = 0; k <= R; ++k) ckt[k] = (T)op.ck[k];
        V2<T> qn = mk2<T>(0, 0);  // x(z + 1 + R), loaded at step z for step z + 1
        V2<T> bn = need_b ? __ldg(b + (int64_t)z0 * plane + oc) : mk2<T>(0, 0);  // b(z)
        for (int z = z0; z < z1; ++z) {
            if (z > z0) {
#pragma unroll
                for (int k = 0; k < 2 * R; ++k) q[k] = q[k + 1];
                q[2 * R] = qn;
            }
            const V2<T> bv = bn;
            if (z + 1 < z1) {
                qn = zval(z + 1 + R);
                if (need_b) bn = __ldg(b + (int64_t)(z + 1) * plane + oc);
            }
            const int64_t pz = (int64_t)z * plane;
            const V2<T>* xp = x + pz;
            const int64_t c = pz + oc;
            const V2<T> xc = q[R];
            // x and y neighbours of every ring first (independent loads), then the sums
            V2<T> nb[4 * R];
#pragma unroll
            for (int k = 1; k <= R; ++k) {
                const int km = R - k, kp = R + k;
                nb[4 * (k - 1) + 0] = ox[km] >= 0 ? __ldg(xp + ox[km]) : mk2<T>(0, 0);
                nb[4 * (k - 1) + 1] = ox[kp] >= 0 ? __ldg(xp + ox[kp]) : mk2<T>(0, 0);
                nb[4 * (k - 1) + 2] = oy[km] >= 0 ? __ldg(xp + oy[km]) : mk2<T>(0, 0);
                nb[4 * (k - 1) + 3] = oy[kp] >= 0 ? __ldg(xp + oy[kp]) : mk2<T>(0, 0);
            }
            V2<T> lap = mk2<T>(0, 0);
#pragma unroll
            for (int k = 1; k <= R; ++k) {
                // the six neighbours at distance k: x - k, x + k, y - k, y + k, z - k, z + k
                V2<T> sk = uadd2(nb[4 * (k - 1) + 0], nb[4 * (k - 1) + 1], one);
                sk = uadd2(sk, nb[4 * (k - 1) + 2], one);
                sk = uadd2(sk, nb[4 * (k - 1) + 3], one);
                sk = uadd2(sk, q[R - k], one);
                sk = uadd2(sk, q[R + k], one);
                lap = (k == 1) ? scl2(ckt[k], sk) : fma2(ckt[k], sk, lap);
            }
            const T lr = lap.x, li = lap.y;
            // (A x)_c = d x_c + lap
            T axr = fma(dr, xc.x, lr);
            axr = fma(-di, xc.y, axr);
            T axi = fma(dr, xc.y, li);
            axi = fma(di, xc.x, axi);
            if (MODE == ZM_APPLY) {
                f[c] = mk2<T>(axr, axi);
                continue;
            }
            const T rr = bv.x - axr, ri = bv.y - axi;
            if (MODE == ZM_RESID || MODE == ZM_RESOUT) {
                if (MODE == ZM_RESOUT) rout[c] = make_float2((float)rr, (float)ri);
                s2 = fma(rr, rr, fma(ri, ri, s2));
                continue;
            }
            if (MODE == ZM_BRES || MODE == ZM_BRES_AND) {  // block Jacobi: k_zblock applies M^{-1}
                f[c] = mk2<T>(rr, ri);
                if (MODE == ZM_BRES_AND) s2 = fma(rr, rr, fma(ri, ri, s2));
                continue;
            }
            // f = D^{-1} res (Eq. 6)
            const T fr = fma(vr, rr, -vi * ri);
            const T fi = fma(vr, ri, vi * rr);
            f[c] = mk2<T>(fr, fi);
            if (MODE == ZM_AND) {
                s2 = fma(rr, rr, fma(ri, ri, s2));
            } else {
                // x_{k+1} = x_k + omega f_k (Eq. 2, 3)
                const T xr = fma(omr, fr, fma(-omi, fi, xc.x));
                const T xi = fma(omr, fi, fma(omi, fr, xc.y));
                xn[c] = mk2<T>(xr, xi);
            }
        }
    }
    if (MODE == ZM_AND || MODE == ZM_RESID || MODE == ZM_RESOUT || MODE == ZM_BRES_AND) {
        const double t = block_sum<8>((double)s2, red);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            part[((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
    }
}

// FP32 sweep of the mixed form's inner solves (modes ZM_RICH, ZM_AND, ZM_BRES, ZM_BRES_AND) with
// each plane's 32 x 8 tile and its in-plane halo staged in shared memory: 8-byte cp.async copies
// (wrapped indices on a periodic grid; zeros outside a Dirichlet grid), two planes ahead in a
// ring of three buffers, one CTA barrier per plane. The z column of a thread stays in registers
// as in k_zstencil, and the sums are formed in the same order, so the results are the same bit
// for bit; the x and y neighbours come from shared memory instead of 4r scattered global loads
// per point, on which the register-fed form waited (long-scoreboard stalls).
template <int R, int MODE>
__global__ void __launch_bounds__(256) k_zsweep_sm(ZOp op, const float2* __restrict__ x, const float2* __restrict__ b,
                                                   float2* __restrict__ f, float2* __restrict__ xn,
                                                   double* __restrict__ part, double2 omega_d, int zc) {
    constexpr int TX = 32, TY = 8, SW = TX + 2 * R, SH = TY + 2 * R, CELLS = SW * SH;
    constexpr int NC = (CELLS + 255) / 256, NBUF = 3;
    __shared__ __align__(16) float2 pl[NBUF][CELLS];
    __shared__ double red[8];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int ix = x0 + tx, iy = y0 + ty;
    const int z0 = blockIdx.z * zc, z1 = min(op.nz, z0 + zc);
    const int nx = op.nx, ny = op.ny, nz = op.nz;
    const int64_t plane = (int64_t)nx * ny;
    const float dr = (float)op.d.x, di = (float)op.d.y, vr = (float)op.dinv.x, vi = (float)op.dinv.y;
    const float omr = (float)omega_d.x, omi = (float)omega_d.y;
    const bool active = ix < nx && iy < ny;
    // this thread's cells of the staged box: in-plane offsets; -1 outside a Dirichlet grid
    int cg[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int cell = tid + 256 * c;
        const int row = cell / SW, col = cell - (cell / SW) * SW;
        const int gx = x0 - R + col, gy = y0 - R + row;
        if (op.periodic) cg[c] = wrap_axis(gy, ny) * nx + wrap_axis(gx, nx);
        else cg[c] = (gx >= 0 && gx < nx && gy >= 0 && gy < ny) ? gy * nx + gx : -1;
    }
    // plane z into buffer buf, as one cp.async group per thread (committed even when empty)
    auto fill = [&](int z, int buf) {
        if (z < z1) {
            const float2* src = x + (int64_t)z * plane;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int cell = tid + 256 * c;
                if (cell < CELLS) {
                    if (cg[c] >= 0) cp_async8(smem_u32(&pl[buf][cell]), src + cg[c]);
                    else pl[buf][cell] = make_float2(0.f, 0.f);
                }
            }
        }
        cp_async_commit();
    };
    fill(z0, 0);
    fill(z0 + 1, 1);
    const int oc = active ? iy * nx + ix : 0;
    const int cc = (R + ty) * SW + (R + tx);  // this thread's point in a staged plane
    float2 q[2 * R + 1];  // z column x(ix, iy, z - R .. z + R), zero outside a Dirichlet grid
    float2 qn = make_float2(0.f, 0.f), bn = make_float2(0.f, 0.f);
    if (active) {
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) {
            const int jz = z0 + k - R;
            const int zi = op.periodic ? wrap_axis(jz, nz) : ((jz >= 0 && jz < nz) ? jz : -1);
            q[k] = zi >= 0 ? __ldg(x + (int64_t)zi * plane + oc) : make_float2(0.f, 0.f);
        }
        bn = __ldg(b + (int64_t)z0 * plane + oc);
    }
    auto zval = [&](int jz) -> float2 {
        const int zi = op.periodic ? (jz >= nz ? wrap_axis(jz, nz) : jz) : (jz < nz ? jz : -1);
        return zi >= 0 ? __ldg(x + (int64_t)zi * plane + oc) : make_float2(0.f, 0.f);
    };
    // the weights in FP32, converted once (a conversion from FP64 runs on the FP64 pipe)
    float ckf[R + 1];
#pragma unroll
    for (int k = 0; k <= R; ++k) ckf[k] = (float)op.ck[k];
    float s2 = 0.f;
    // The march is unrolled by the queue length Q = 2R + 1: plane z + d sits in q[(u + R + d) mod
    // Q] at step z = zb + u (zb - z0 a multiple of Q), so the queue turns by renaming registers
    // instead of moving 2R values every plane; the plane that enters at step z (z + R, loaded one
    // step ahead) takes the slot of the one that left (z - R - 1).
    constexpr int Q = 2 * R + 1;
    int buf = 0;  // staged buffer of plane z: (z - z0) mod NBUF
#pragma unroll 1
    for (int zb = z0; zb < z1; zb += Q) {
#pragma unroll
        for (int u = 0; u < Q; ++u) {
            const int z = zb + u;
            if (z >= z1) break;  // uniform across the CTA
            cp_async_wait_prior();  // plane z has landed (only plane z + 1 may still be in flight)
            __syncthreads();        // ... for every thread; and every thread is done with plane z - 1
            fill(z + 2, buf == 0 ? NBUF - 1 : buf - 1);  // into the buffer of plane z - 1
            if (active) {
                if (u > 0 || zb > z0) q[(u + Q - 1) % Q] = qn;
                const float2 bv = bn;
                if (z + 1 < z1) {
                    qn = zval(z + 1 + R);
                    bn = __ldg(b + (int64_t)(z + 1) * plane + oc);
                }
                const float2* P = pl[buf];
                const float2 xc = q[(u + R) % Q];
                float2 lap = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                    // the six neighbours at distance k, in k_zstencil's order
                    float2 sk = uadd2(P[cc - k], P[cc + k], 1.f);
                    sk = uadd2(sk, P[cc - k * SW], 1.f);
                    sk = uadd2(sk, P[cc + k * SW], 1.f);
                    sk = uadd2(sk, q[(u + R - k) % Q], 1.f);
                    sk = uadd2(sk, q[(u + R + k) % Q], 1.f);
                    lap = (k == 1) ? scl2(ckf[k], sk) : fma2(ckf[k], sk, lap);
                }
                const int64_t c = (int64_t)z * plane + oc;
                float axr = fmaf(dr, xc.x, lap.x);
                axr = fmaf(-di, xc.y, axr);
                float axi = fmaf(dr, xc.y, lap.y);
                axi = fmaf(di, xc.x, axi);
                const float rr = bv.x - axr, ri = bv.y - axi;
                if constexpr (MODE == ZM_BRES || MODE == ZM_BRES_AND) {  // block Jacobi: k_zblock applies M^{-1}
                    f[c] = make_float2(rr, ri);
                    if constexpr (MODE == ZM_BRES_AND) s2 = fmaf(rr, rr, fmaf(ri, ri, s2));
                } else {
                    const float fr = fmaf(vr, rr, -vi * ri);
                    const float fi = fmaf(vr, ri, vi * rr);
                    f[c] = make_float2(fr, fi);
                    if constexpr (MODE == ZM_AND) {
                        s2 = fmaf(rr, rr, fmaf(ri, ri, s2));
                    } else {
                        const float xr = fmaf(omr, fr, fmaf(-omi, fi, xc.x));
                        const float xi = fmaf(omr, fi, fmaf(omi, fr, xc.y));
                        xn[c] = make_float2(xr, xi);
                    }
                }
            }
            buf = buf == NBUF - 1 ? 0 : buf + 1;
        }
    }
    cp_async_wait_all();  // the empty trailing groups
    if constexpr (MODE == ZM_AND || MODE == ZM_BRES_AND) {
        const double t = block_sum<8>((double)s2, red);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            part[((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
    }
}

// ------------------------------------------------------------------ block Jacobi (2 x 2 x 2)
// The block Jacobi of Sec. 3.2's Helmholtz runs with exact block solves, on boxes of 2 x 2 x 2
// points: a box holds a point's three distance-1 partners and no other tap of the stencil (sides
// even; periodic sides at least r + 2), so every block of Eq. 7's operator is d I + c1 Q3, with d
// the complex centre coefficient, c1 = ck[1] the real distance-1 coefficient and Q3 the cube
// graph. Q3's eigenvectors are the 8-point Walsh-Hadamard vectors (eigenvalue 3 - 2|s| for the
// sign pattern s), so M^{-1} = H diag(mu_|s|) H with mu_t = 1 / (8 (d + c1 (3 - 2t))): the real
// transform H applied to the real and imaginary parts alike, three butterfly stages, one complex
// scaling, three stages. One thread per box: f <- M^{-1} f (the sweep wrote b - A x_k into f) and,
// at a Richardson step, x_{k+1} = x_k + omega f (Eq. 2, 3).
template <typename T>
__device__ __forceinline__ void zfwht8(V2<T> (&v)[8]) {
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1)
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (!(q & bit)) {
                const V2<T> a = v[q], b = v[q | bit];
                v[q] = mk2<T>(a.x + b.x, a.y + b.y);
                v[q | bit] = mk2<T>(a.x - b.x, a.y - b.y);
            }
}

template <typename T>
__global__ void __launch_bounds__(256) k_zblock(ZOp op, V2<T>* __restrict__ f, const V2<T>* __restrict__ x,
                                                V2<T>* __restrict__ xn, double2 omega_d, int rich) {
    const int bx = op.nx / 2, by = op.ny / 2;
    const int64_t nbox = (int64_t)bx * by * (op.nz / 2);
    const int64_t plane = (int64_t)op.nx * op.ny;
    T mr[4], mi[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        mr[t] = (T)op.mu[t].x;
        mi[t] = (T)op.mu[t].y;
    }
    const T omr = (T)omega_d.x, omi = (T)omega_d.y;
    for (int64_t bi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; bi < nbox; bi += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(bi % bx);
        const int64_t t2 = bi / bx;
        const int Y = (int)(t2 % by), Z = (int)(t2 / by);
        const int64_t base = (int64_t)(2 * Z) * plane + (int64_t)(2 * Y) * op.nx + 2 * X;
        int64_t idx[8];
        V2<T> v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {  // q = dx + 2 dy + 4 dz
            idx[q] = base + ((q >> 2) & 1) * plane + ((q >> 1) & 1) * op.nx + (q & 1);
            v[q] = f[idx[q]];
        }
        zfwht8<T>(v);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int t = __popc(q);
            const V2<T> a = v[q];
            v[q] = mk2<T>(fma(mr[t], a.x, -mi[t] * a.y), fma(mr[t], a.y, mi[t] * a.x));
        }
        zfwht8<T>(v);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            f[idx[q]] = v[q];
            if (rich) {
                const V2<T> xc = x[idx[q]];
                xn[idx[q]] = mk2<T>(fma(omr, v[q].x, fma(-omi, v[q].y, xc.x)), fma(omr, v[q].y, fma(omi, v[q].x, xc.y)));
            }
        }
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
// place (column a <- f_{k-c+a+1} - f_{k-c+a}, the columns of F_k in Eq. 5; column c keeps f_k).
// Warp w accumulates the Gram entries e = w, w + 8, ... (the upper triangle of F^H F, then
// F^H f_k) over all points of the chunk, lane l over points l, l + 32, ... so that a warp's
// shared-memory reads are contiguous. FP64: one accumulator per entry and lane. FP32: each
// chunk's sum is folded into a compensated (TwoSum) pair, so that the CTA's sum over many chunks
// keeps FP32 accuracy. Lanes are combined in FP64 by a fixed shuffle tree; partial sums per CTA
// are combined in a fixed order by the finalize.
constexpr int GRAM_PF = ((ZMAXM + 1) * GRAM_CH + 255) / 256;  // chunk elements each thread loads

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (v - bp);
    hi = s;
}

// NJ >= ceil(E / 8) entries per warp (a template parameter, so that the accumulators stay in
// registers and the CTA's register footprint follows the history length). The next chunk's
// loads are issued into registers before the current chunk's products.
template <typename T, int NJ>
__global__ void __launch_bounds__(256) k_zgram(ZCols<T> cols, int c, int64_t n, double* __restrict__ part) {
    __shared__ __align__(16) unsigned char sdraw[(ZMAXM + 1) * GRAM_CH * sizeof(V2<T>)];
    __shared__ unsigned char ea[ZMAXE], eb[ZMAXE];
    V2<T>* sd = reinterpret_cast<V2<T>*>(sdraw);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
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
    T hr[NJ], hi_[NJ], lr[NJ], li[NJ];  // lr, li: compensation terms (FP32 only)
#pragma unroll
    for (int j = 0; j < NJ; ++j) hr[j] = hi_[j] = lr[j] = li[j] = 0;
    const int64_t nch = (n + GRAM_CH - 1) / GRAM_CH;
    const int NL = (c + 1) * GRAM_CH;
    V2<T> pf[GRAM_PF];
    auto fetch = [&](int64_t ch) {
        const int64_t base = ch * GRAM_CH;
#pragma unroll
        for (int r = 0; r < GRAM_PF; ++r) {
            const int idx = tid + 256 * r;
            if (idx < NL) {
                const int col = idx / GRAM_CH, pt = idx - col * GRAM_CH;
                const int64_t i = base + pt;
                pf[r] = i < n ? cols.p[col][i] : mk2<T>(0, 0);
            }
        }
    };
    if (blockIdx.x < nch) fetch(blockIdx.x);
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        __syncthreads();  // the previous chunk's products are done
#pragma unroll
        for (int r = 0; r < GRAM_PF; ++r) {
            const int idx = tid + 256 * r;
            if (idx < NL) sd[idx] = pf[r];
        }
        if (ch + gridDim.x < nch) fetch(ch + gridDim.x);
        __syncthreads();
        if (tid < GRAM_CH) {
            for (int a = 0; a < c; ++a) {
                const V2<T> u = sd[a * GRAM_CH + tid], v = sd[(a + 1) * GRAM_CH + tid];
                sd[a * GRAM_CH + tid] = mk2<T>(v.x - u.x, v.y - u.y);
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const int e = w + 8 * j;
            if (e < E) {
                const V2<T>* U = sd + ea[e] * GRAM_CH;
                const V2<T>* V = sd + eb[e] * GRAM_CH;
                if constexpr (sizeof(T) == 8) {
#pragma unroll
                    for (int q = 0; q < GRAM_CH / 32; ++q) {
                        const V2<T> u = U[lane + 32 * q], v = V[lane + 32 * q];
                        // conj(u) v
                        hr[j] = fma(u.x, v.x, hr[j]);
                        hr[j] = fma(u.y, v.y, hr[j]);
                        hi_[j] = fma(u.x, v.y, hi_[j]);
                        hi_[j] = fma(-u.y, v.x, hi_[j]);
                    }
                } else {
                    T cr = 0, ci = 0;
#pragma unroll
                    for (int q = 0; q < GRAM_CH / 32; ++q) {
                        const V2<T> u = U[lane + 32 * q], v = V[lane + 32 * q];
                        cr = fma(u.x, v.x, cr);
                        cr = fma(u.y, v.y, cr);
                        ci = fma(u.x, v.y, ci);
                        ci = fma(-u.y, v.x, ci);
                    }
                    two_sum_acc(hr[j], lr[j], cr);
                    two_sum_acc(hi_[j], li[j], ci);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int e = w + 8 * j;
        if (e < E) {  // uniform within the warp
            double vr = (double)hr[j] + (double)lr[j], vi = (double)hi_[j] + (double)li[j];
            for (int o = 16; o > 0; o >>= 1) {
                vr += __shfl_down_sync(0xffffffffu, vr, o);
                vi += __shfl_down_sync(0xffffffffu, vi, o);
            }
            if (lane == 0) {
                part[(int64_t)blockIdx.x * 2 * E + 2 * e] = vr;
                part[(int64_t)blockIdx.x * 2 * E + 2 * e + 1] = vi;
            }
        }
    }
}

// FP32 Gram with the operands in registers (the mixed form's inner solves). A CTA is two groups
// of four warps; a group takes 32-point chunks, lane l point l of the chunk, and every warp of
// the group loads the chunk's c + 1 residual values (the other three warps' loads hit L1), forms
// the c differences in registers, and accumulates the Gram entries e = WQ, WQ + 4, ... (WQ = its
// place in the group). C = c and WQ are template parameters, so every operand and accumulator
// index is a compile-time constant and nothing is staged in shared memory. A lane sums its
// points in FP32; lanes are combined in FP32 by a fixed shuffle tree, warps and groups in FP64
// in a fixed order (an FP64 shuffle tree costs 64 times as much issue time on this part).
constexpr int ZGRAM_REG_MAXC = 12;  // longer histories take the shared-memory Gram
__host__ __device__ constexpr int gram_entries(int C) { return C * (C + 1) / 2 + C; }
__host__ __device__ constexpr int gram_ea(int C, int e) {  // row of entry e
    int a = 0, rem = e;
    while (a < C && rem >= C - a) {
        rem -= C - a;
        ++a;
    }
    return a < C ? a : e - C * (C + 1) / 2;
}
__host__ __device__ constexpr int gram_eb(int C, int e) {  // column of entry e (C: the f_k column)
    int a = 0, rem = e;
    while (a < C && rem >= C - a) {
        rem -= C - a;
        ++a;
    }
    return a < C ? a + rem : C;
}

// one Gram entry E of the chunk's point: (a, b) fixed at compile time
template <int C, int E>
__device__ __forceinline__ void zgram_one(const float2 (&col)[C + 1], float& ar, float& ai) {
    constexpr int a = gram_ea(C, E), b = gram_eb(C, E);
    const float2 u = col[a], v = col[b];
    ar = fmaf(u.x, v.x, ar);
    ar = fmaf(u.y, v.y, ar);
    ai = fmaf(u.x, v.y, ai);
    ai = fmaf(-u.y, v.x, ai);
}

template <int C, int WQ, int NJ, int... J>
__device__ __forceinline__ void zgram_entries(const float2 (&col)[C + 1], float (&ar)[NJ], float (&ai)[NJ],
                                              std::integer_sequence<int, J...>) {
    (zgram_one<C, WQ + 4 * J>(col, ar[J], ai[J]), ...);
}

template <int C, int WQ>
__device__ __forceinline__ void zgram_reg_warp(ZCols<float> cols, int64_t n, int64_t ch0, int64_t chstep,
                                               int lane, double* outr, double* outi) {
    constexpr int E = gram_entries(C);
    constexpr int NJ = (E - WQ + 3) / 4;  // entries WQ, WQ + 4, ... below E
    if constexpr (NJ > 0) {
        float ar[NJ], ai[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) ar[j] = ai[j] = 0.f;
        const int64_t nch = (n + 31) / 32;
        for (int64_t ch = ch0; ch < nch; ch += chstep) {
            const int64_t i = ch * 32 + lane;
            float2 col[C + 1];
#pragma unroll
            for (int j = 0; j <= C; ++j) col[j] = i < n ? __ldg(cols.p[j] + i) : make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < C; ++a) col[a] = make_float2(col[a + 1].x - col[a].x, col[a + 1].y - col[a].y);
            zgram_entries<C, WQ>(col, ar, ai, std::make_integer_sequence<int, NJ>{});
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {  // lanes combined in FP32 (a warp tree), warps in FP64
            float vr = ar[j], vi = ai[j];
            for (int o = 16; o > 0; o >>= 1) {
                vr += __shfl_down_sync(0xffffffffu, vr, o);
                vi += __shfl_down_sync(0xffffffffu, vi, o);
            }
            if (lane == 0) {
                outr[WQ + 4 * j] = (double)vr;
                outi[WQ + 4 * j] = (double)vi;
            }
        }
    }
}

template <int C>
__global__ void __launch_bounds__(256) k_zgram_reg(ZCols<float> cols, int64_t n, double* __restrict__ part) {
    constexpr int E = gram_entries(C);
    __shared__ double gr[2][E], gi[2][E];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, grp = w >> 2, wq = w & 3;
    const int64_t ch0 = (int64_t)blockIdx.x * 2 + grp, chstep = (int64_t)gridDim.x * 2;
    switch (wq) {  // warp-uniform
        case 0: zgram_reg_warp<C, 0>(cols, n, ch0, chstep, lane, gr[grp], gi[grp]); break;
        case 1: zgram_reg_warp<C, 1>(cols, n, ch0, chstep, lane, gr[grp], gi[grp]); break;
        case 2: zgram_reg_warp<C, 2>(cols, n, ch0, chstep, lane, gr[grp], gi[grp]); break;
        default: zgram_reg_warp<C, 3>(cols, n, ch0, chstep, lane, gr[grp], gi[grp]); break;
    }
    __syncthreads();
    for (int e = tid; e < E; e += 256) {
        part[(int64_t)blockIdx.x * 2 * E + 2 * e] = gr[0][e] + gr[1][e];
        part[(int64_t)blockIdx.x * 2 * E + 2 * e + 1] = gi[0][e] + gi[1][e];
    }
}

// FP32 Gram fed by 1-D bulk copies (the mixed form's inner solves, c <= ZGRAM_REG_MAXC). The
// lanes of warp 0 copy a chunk of 256 to 512 points of each of the c + 1 residual columns into a
// shared-memory stage with cp.async.bulk, completing the stage's mbarrier, three stages deep, so a
// CTA keeps (c + 1) chunks of 8-byte values per stage in flight without holding them in registers.
// Copies start 16-byte aligned (ring slots start on 256-byte boundaries and chunks are 2 to 4 KB); a
// ragged last chunk is rounded up to an even point count, inside the slot's padding. G groups of
// 256 / G threads share every chunk: group g takes the Gram entries g, g + G, ... (their (a, b)
// compile-time constants), each thread the points t, t + 256 / G, ... of the chunk. A thread sums
// its points in FP32; lanes are combined in FP32 by a fixed shuffle tree, warps and groups in FP64
// in a fixed order.
template <int C>
__host__ __device__ constexpr int zb_groups() { return C <= 9 ? 2 : 4; }
template <int C>
__host__ __device__ constexpr int zb_njmax() { return (gram_entries(C) + zb_groups<C>() - 1) / zb_groups<C>(); }
// points per chunk: 512 (4 KB per column, 4 points per thread between barriers) where three
// stages of c + 1 columns still let two CTAs share an SM; 384 for c = 9 (3 per thread); 256 for
// c > 9 (4 groups: again 4 points per thread)
template <int C>
__host__ __device__ constexpr int zb_ch() { return C <= 8 ? 512 : C == 9 ? 384 : 256; }
constexpr int ZB_STAGES = 3;
template <int C>
constexpr size_t zgram_bulk_smem() { return (size_t)ZB_STAGES * (C + 1) * zb_ch<C>() * sizeof(float2) + 1024; }

template <int C, int G, int GQ, int NJ, int... J>
__device__ __forceinline__ void zgram_group_entries(const float2 (&col)[C + 1], float (&ar)[NJ], float (&ai)[NJ],
                                                    std::integer_sequence<int, J...>) {
    (zgram_one<C, GQ + G * J>(col, ar[J], ai[J]), ...);
}

// The chunk pipeline of one group; false when a bounded wait gave up somewhere in the CTA (every
// thread then returns, thread 0 after the copies still in flight have landed). A thread whose wait
// gave up skips its later waits; warp 0 issues only while none of its lanes gave up, and the
// CTA-wide vote runs once, after the last chunk, so the per-chunk barrier is a plain one.
template <int C, int GQ>
__device__ __forceinline__ bool zgram_bulk_run(const ZCols<float>& cols, int64_t n, float2* sm, uint64_t* bars,
                                               int* err, double (*red)[2 * zb_njmax<C>()], int tid) {
    constexpr int E = gram_entries(C), G = zb_groups<C>(), TG = 256 / G, NSTG = ZB_STAGES, ZB_CH = zb_ch<C>();
    constexpr int NJ = (E - GQ + G - 1) / G;  // entries GQ, GQ + G, ... below E
    const int lane = tid & 31, warp = tid >> 5, tq = tid % TG;
    const int64_t nch = (n + ZB_CH - 1) / ZB_CH, b0 = blockIdx.x, gs = gridDim.x;
    const int mine = b0 < nch ? (int)((nch - 1 - b0) / gs + 1) : 0;  // this CTA's chunks b0, b0 + gs, ...
    auto cstart = [&](int q) { return (b0 + (int64_t)q * gs) * ZB_CH; };
    auto clen = [&](int q) {
        const int64_t r = n - cstart(q);
        return (int)(r < ZB_CH ? r : ZB_CH);
    };
    uint32_t hi = 0;
    bool abort = false;
    auto issue = [&](int q) {  // the lanes of warp 0: lane j copies column j
        const uint32_t bar = smem_u32(&bars[q % NSTG]);
        const uint32_t bytes = (uint32_t)((clen(q) + 1) & ~1) * (uint32_t)sizeof(float2);
        if (lane == 0) mbar_expect_tx(bar, bytes * (uint32_t)(C + 1));
        float2* st = sm + (size_t)(q % NSTG) * (C + 1) * ZB_CH;
        if (lane <= C) bulk_g2s(smem_u32(st + lane * ZB_CH), cols.p[lane] + cstart(q), bytes, bar);
        hi = (uint32_t)q + 1;
    };
    if (warp == 0 && !__any_sync(0xffffffffu, abort))
        for (int q = 0; q < NSTG && q < mine; ++q) issue(q);
    float ar[NJ], ai[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) ar[j] = ai[j] = 0.f;
#pragma unroll 1
    for (int q = 0; q < mine; ++q) {
        mbar_wait(smem_u32(&bars[q % NSTG]), (uint32_t)(q / NSTG) & 1u, err, abort, q);
        const float2* st = sm + (size_t)(q % NSTG) * (C + 1) * ZB_CH;
        const int len = clen(q);
#pragma unroll 1
        for (int p = tq; p < len; p += TG) {
            float2 col[C + 1];
#pragma unroll
            for (int j = 0; j <= C; ++j) col[j] = st[j * ZB_CH + p];
#pragma unroll
            for (int a = 0; a < C; ++a) col[a] = make_float2(col[a + 1].x - col[a].x, col[a + 1].y - col[a].y);
            zgram_group_entries<C, G, GQ>(col, ar, ai, std::make_integer_sequence<int, NJ>{});
        }
        __syncthreads();  // chunk q is consumed: its stage takes chunk q + NSTG
        if (warp == 0 && q + NSTG < mine && !__any_sync(0xffffffffu, abort)) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(q + NSTG);
        }
    }
    if (__syncthreads_or(abort)) {
        if (tid == 0) mbar_drain(bars, NSTG, 0, hi);
        return false;
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) {  // lanes combined in FP32 (a warp tree), warps in FP64
        float vr = ar[j], vi = ai[j];
        for (int o = 16; o > 0; o >>= 1) {
            vr += __shfl_down_sync(0xffffffffu, vr, o);
            vi += __shfl_down_sync(0xffffffffu, vi, o);
        }
        if (lane == 0) {
            red[warp][2 * j] = (double)vr;
            red[warp][2 * j + 1] = (double)vi;
        }
    }
    return true;
}

template <int C>
__global__ void __launch_bounds__(256, 2) k_zgram_bulk(ZCols<float> cols, int64_t n, double* __restrict__ part,
                                                    int* err) {
    constexpr int E = gram_entries(C), G = zb_groups<C>(), NWG = 8 / G, NSTG = ZB_STAGES;
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[NSTG];
    __shared__ double red[8][2 * zb_njmax<C>()];
    float2* sm = reinterpret_cast<float2*>(smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u));
    const int tid = threadIdx.x, grp = (tid >> 5) / NWG;
    if (tid == 0) {
        for (int q = 0; q < NSTG; ++q) mbar_init(smem_u32(&bars[q]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    bool ok;
    if (grp == 0) ok = zgram_bulk_run<C, 0>(cols, n, sm, bars, err, red, tid);
    else if (grp == 1) ok = zgram_bulk_run<C, 1>(cols, n, sm, bars, err, red, tid);
    else if constexpr (G > 2) {
        if (grp == 2) ok = zgram_bulk_run<C, 2>(cols, n, sm, bars, err, red, tid);
        else ok = zgram_bulk_run<C, G - 1>(cols, n, sm, bars, err, red, tid);
    }
    if (!ok) return;  // the same for every thread (decided by a CTA-wide vote)
    __syncthreads();
    for (int e = tid; e < E; e += 256) {
        const int g = e % G, j = e / G;
        double vr = 0.0, vi = 0.0;
        for (int w = g * NWG; w < (g + 1) * NWG; ++w) {
            vr += red[w][2 * j];
            vi += red[w][2 * j + 1];
        }
        part[(int64_t)blockIdx.x * 2 * E + 2 * e] = vr;
        part[(int64_t)blockIdx.x * 2 * E + 2 * e + 1] = vi;
    }
}

// ---------------------------------------------------------------------------- finalize
// ldl_solve_warp (certified) for the real 2c x 2c form, 2c in {2, 4, ..., 2 ZLDL_MAXC}; longer
// histories take the eigen-decomposition (the unrolled solves of 2c > 24 would mostly add compile
// time)
constexpr int ZLDL_MAXC = 12;
template <int... Ks>
__device__ __forceinline__ bool zldl_dispatch(int c2, const double* Sm, const double* rhs, double* Vm, int lane,
                                              double& z, std::integer_sequence<int, Ks...>) {
    bool ok = false;
    ((c2 == 2 * (Ks + 1) ? (ok = ldl_solve_warp<2 * (Ks + 1), ZLD, true>(Sm, rhs, Vm, lane, z, (double)(Ks + 1)), 0)
                         : 0),
     ...);
    return ok;
}

// mode 0: ||b|| from the k_znorm partials; mode 1: an Anderson step (r_k, convergence, gamma and
// the update's coefficients); mode 2: ||b - A x|| / ||b|| from the ZM_RESID and k_znorm partials
// (into r).
__global__ void __launch_bounds__(256) k_zfinalize(ZState* st, const double* __restrict__ part_r, int nr,
                                                   const double* __restrict__ part_g, int ng,
                                                   const double* __restrict__ part_b, int nbp, int c, double tol,
                                                   double2 beta, int mode) {
    __shared__ double red[8];
    __shared__ double gs[2 * ZMAXE];
    __shared__ double gpart[256 > 2 * ZMAXE ? 256 : 2 * ZMAXE];  // G * 2E <= max(256, 2E)
    __shared__ double Sm[ZLD * ZLD], Vm[ZLD * ZLD];
    __shared__ double rhs[ZLD], coef[ZLD], sol2[ZLD];
    __shared__ int s_go, s_cert, s_kept;
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
    // fixed-order sums of the Gram partials: entry t over the CTAs of the Gram pass. The 256
    // threads form G groups of 2E (G = 256 / 2E, at most 8); group g adds the CTAs of its
    // contiguous range in order, eight loads in flight at a time, and the G group sums are added
    // in group order (shorter dependent FP64 chains: an FP64 add takes about 64 cycles here).
    const int E = c * (c + 1) / 2 + c;
    {
        const int G = max(1, min(8, 256 / (2 * E)));
        const int per = (ng + G - 1) / G;
        for (int idx = tid; idx < G * 2 * E; idx += 256) {
            const int g = idx / (2 * E), t = idx - g * (2 * E);
            const int b0 = g * per, b1 = min(ng, b0 + per);
            double v = 0.0;
            int blk = b0;
            for (; blk + 8 <= b1; blk += 8) {
                double w[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) w[u] = part_g[(int64_t)(blk + u) * 2 * E + t];
#pragma unroll
                for (int u = 0; u < 8; ++u) v += w[u];
            }
            for (; blk < b1; ++blk) v += part_g[(int64_t)blk * 2 * E + t];
            gpart[g * 2 * E + t] = v;
        }
        __syncthreads();
        for (int t = tid; t < 2 * E; t += 256) {
            double v = gpart[t];
            for (int q = 1; q < G; ++q) v += gpart[q * 2 * E + t];
            gs[t] = v;
        }
    }
    __syncthreads();
    // real 2c x 2c form [[Re G, -Im G], [Im G, Re G]] and right-hand side [Re g; Im g], one
    // Gram entry per thread
    const int c2 = 2 * c;
    for (int e = tid; e < E; e += 256) {
        const double gr = gs[2 * e], gi = gs[2 * e + 1];
        if (e < c * (c + 1) / 2) {  // G_ab (a <= bb) = <dF_a, dF_b>, G_ba = conj(G_ab)
            int a = 0, rem = e;
            while (rem >= c - a) {
                rem -= c - a;
                ++a;
            }
            const int bb = a + rem;
            Sm[a * ZLD + bb] = gr;
            Sm[bb * ZLD + a] = gr;
            Sm[(c + a) * ZLD + c + bb] = gr;
            Sm[(c + bb) * ZLD + c + a] = gr;
            Sm[a * ZLD + c + bb] = -gi;
            Sm[(c + bb) * ZLD + a] = -gi;
            Sm[(c + a) * ZLD + bb] = gi;
            Sm[bb * ZLD + c + a] = gi;
        } else {
            const int a = e - c * (c + 1) / 2;
            rhs[a] = gr;
            rhs[c + a] = gi;
        }
    }
    __syncthreads();
    // (1) the certified LDL^T solve on warp 0 (ldl_solve_warp): trace(S) trace(S^-1) c < 2^42
    //     bounds lambda_max / lambda_min, so every eigenvalue lies 2^10 above the pseudoinverse's
    //     cut and pinv(S) = S^-1: gamma is the plain solve.
    if (tid < 32) {
        double z = 0.0;
        const bool ok = zldl_dispatch(c2, Sm, rhs, Vm, tid, z, std::make_integer_sequence<int, ZLDL_MAXC>{});
        if (ok && tid < c2) sol2[tid] = z;
        if (tid == 0) s_cert = ok ? 1 : 0;
    }
    __syncthreads();
    // (2) otherwise the pseudoinverse through the eigen-decomposition (all 8 warps), then warp 0
    if (!s_cert) cta_sym_eig<ZLD, 8>(c2, Sm, Vm);  // all 8 warps: one item per thread up to 2c = 22
    if (!s_cert && tid < 32) {
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
    // the update's coefficients, one column per thread: gamma = sol2[0..c) + i sol2[c..2c); the
    // coefficient of x_{k-c+j} is gamma_{j-1} - gamma_j (gamma_{-1} = gamma_c = 0)
    if (tid < 32) {
        const bool fin = __all_sync(0xffffffffu, tid >= c2 || finite_bits(sol2[tid]));
        if (fin && tid <= c) {
            const int j = tid;
            const double ar = (j > 0 ? sol2[j - 1] : 0.0) - (j < c ? sol2[j] : 0.0);
            const double ai = (j > 0 ? sol2[c + j - 1] : 0.0) - (j < c ? sol2[c + j] : 0.0);
            st->ax[j] = make_double2(ar, ai);
            st->af[j] = make_double2(beta.x * ar - beta.y * ai, beta.x * ai + beta.y * ar);
            if (j < c) st->gam[j] = make_double2(sol2[j], sol2[c + j]);
        }
        if (tid == 0) {
            if (!fin) {
                st->status = ZS_BREAK;
            } else {
                const int kept = s_cert ? c2 : s_kept;
                st->rank = kept / 2;
                st->kept2 = kept;
                st->eig = s_cert ? 0 : 1;
            }
        }
    }
}

// ------------------------------------------------------------------------------ update
// x_{k+1} = x_k + beta f_k - sum_{j=0..c} (ax_j x_{k-c+j} + af_j f_{k-c+j}) (Eq. 3 with the
// differences of Eq. 4, 5 expanded). xout may be the slot of x_{k-c}: each element is read
// before it is written, by the same thread.
// FP32 (the mixed form's inner solves): the x part sum_j ax_j x_j equals sum_i gamma_i (x_{i+1} -
// x_i) over the window's differences (ax_j = gamma_{j-1} - gamma_j), and a difference made by a
// Richardson step (step s = k - c + i with (s + 1) mod p != 0) is omega f_i, so it moves into the
// coefficient of f_i; only the differences made by Anderson steps keep their two x columns. An x
// column whose coefficient is then zero is not read: about c + 4 columns instead of 2c + 2. The
// FP64 form keeps the literal expansion (the oracle's arithmetic).
template <typename T>
__global__ void __launch_bounds__(256) k_zupdate(const ZState* st, ZCols<T> xs, ZCols<T> fs, int c, V2<T>* xout,
                                                 double2 beta_d, int64_t n, int force, int64_t k, int p,
                                                 double2 omega_d) {
    __shared__ V2<T> ax[ZMAXM + 1], af[ZMAXM + 1];
    __shared__ int xuse[ZMAXM + 1];
    __shared__ int run;
    if (threadIdx.x == 0) run = force || st->status == ZS_RUN;
    if (threadIdx.x <= c) {
        const int j = threadIdx.x;
        double2 cx = st->ax[j], cf = st->af[j];
        if constexpr (sizeof(T) == 4) {
            cx = make_double2(0.0, 0.0);
            auto made_by_anderson = [&](int i) { return (k - c + i + 1) % p == 0; };  // difference i
            if (j > 0 && made_by_anderson(j - 1)) {  // + gamma_{j-1} x_j
                cx.x += st->gam[j - 1].x;
                cx.y += st->gam[j - 1].y;
            }
            if (j < c) {
                const double2 g = st->gam[j];
                if (made_by_anderson(j)) {  // - gamma_j x_j
                    cx.x -= g.x;
                    cx.y -= g.y;
                } else {  // gamma_j omega f_j
                    cf.x += g.x * omega_d.x - g.y * omega_d.y;
                    cf.y += g.x * omega_d.y + g.y * omega_d.x;
                }
            }
        }
        ax[j] = mk2<T>((T)cx.x, (T)cx.y);
        af[j] = mk2<T>((T)cf.x, (T)cf.y);
        xuse[j] = (cx.x != 0.0 || cx.y != 0.0) ? 1 : 0;
    }
    __syncthreads();
    if (!run) return;
    const T br = (T)beta_d.x, bi = (T)beta_d.y;
    auto axpy = [](V2<T> a, V2<T> v, T& vr, T& vi) {  // (vr, vi) -= a v
        vr = fma(-a.x, v.x, vr);
        vr = fma(a.y, v.y, vr);
        vi = fma(-a.x, v.y, vi);
        vi = fma(-a.y, v.x, vi);
    };
    if constexpr (sizeof(T) == 4) {
        // the x columns in use as a compact list, so that both column loops are free of branches
        __shared__ const V2<T>* xp[ZMAXM + 1];
        __shared__ V2<T> xa[ZMAXM + 1];
        __shared__ int nxu;
        if (threadIdx.x == 0) {
            int u = 0;
            for (int j = 0; j <= c; ++j)
                if (xuse[j]) {
                    xp[u] = xs.p[j];
                    xa[u] = ax[j];
                    ++u;
                }
            nxu = u;
        }
        __syncthreads();
        for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
            const V2<T> xk = xs.p[c][i], fk = fs.p[c][i];
            T vr = fma(br, fk.x, fma(-bi, fk.y, xk.x));
            T vi = fma(br, fk.y, fma(bi, fk.x, xk.y));
            for (int u = 0; u < nxu; ++u) axpy(xa[u], xp[u][i], vr, vi);
            for (int j = 0; j <= c; ++j) axpy(af[j], fs.p[j][i], vr, vi);
            xout[i] = mk2<T>(vr, vi);
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
            const V2<T> xk = xs.p[c][i], fk = fs.p[c][i];
            T vr = fma(br, fk.x, fma(-bi, fk.y, xk.x));
            T vi = fma(br, fk.y, fma(bi, fk.x, xk.y));
            for (int j = 0; j <= c; ++j) {
                axpy(ax[j], xs.p[j][i], vr, vi);
                axpy(af[j], fs.p[j][i], vr, vi);
            }
            xout[i] = mk2<T>(vr, vi);
        }
    }
}

// Mixed form: x64 += d (the FP32 inner solution), in FP64.
__global__ void __launch_bounds__(256) k_zadd(double2* __restrict__ x64, const float2* __restrict__ d, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
        const float2 v = d[i];
        double2 xv = x64[i];
        xv.x += (double)v.x;
        xv.y += (double)v.y;
        x64[i] = xv;
    }
}

// ------------------------------------------------------------------------------- host
// AAR_ZSWEEP_REG=1 selects the register-fed FP32 sweep (k_zstencil) instead of the staged one
bool zsweep_use_reg() {
    static const int v = [] {
        const char* e = getenv("AAR_ZSWEEP_REG");
        return (e && e[0] == '1') ? 1 : 0;
    }();
    return v != 0;
}

template <typename T, int R>
cudaError_t launch_zstencil_r(int mode, dim3 grid, cudaStream_t s, const ZOp& op, const V2<T>* x, const V2<T>* b,
                              V2<T>* f, V2<T>* xn, double* part, double2 om, int zc, float2* rout) {
    const dim3 blk(32, 8);
    if constexpr (sizeof(T) == 4) {
        // the FP32 sweeps of the inner solves: planes staged in shared memory (k_zsweep_sm), unless
        // AAR_ZSWEEP_REG=1 selects the register-fed kernel; same grid, same results
        if (!zsweep_use_reg()) {
            switch (mode) {
                case ZM_RICH: k_zsweep_sm<R, ZM_RICH><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc); return cudaGetLastError();
                case ZM_AND: k_zsweep_sm<R, ZM_AND><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc); return cudaGetLastError();
                case ZM_BRES: k_zsweep_sm<R, ZM_BRES><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc); return cudaGetLastError();
                case ZM_BRES_AND:
                    k_zsweep_sm<R, ZM_BRES_AND><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc);
                    return cudaGetLastError();
                default: break;
            }
        }
    }
    switch (mode) {
        case ZM_RICH: k_zstencil<T, R, ZM_RICH><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc, rout); break;
        case ZM_AND: k_zstencil<T, R, ZM_AND><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc, rout); break;
        case ZM_APPLY: k_zstencil<T, R, ZM_APPLY><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc, rout); break;
        case ZM_RESID: k_zstencil<T, R, ZM_RESID><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc, rout); break;
        case ZM_BRES: k_zstencil<T, R, ZM_BRES><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc, rout); break;
        case ZM_BRES_AND:
            k_zstencil<T, R, ZM_BRES_AND><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc, rout);
            break;
        default:
            if constexpr (sizeof(T) == 8) {
                k_zstencil<T, R, ZM_RESOUT><<<grid, blk, 0, s>>>(op, x, b, f, xn, part, om, zc, rout);
                break;
            } else {
                return cudaErrorInvalidValue;
            }
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zstencil(int mode, dim3 grid, cudaStream_t s, const ZOp& op, const V2<T>* x, const V2<T>* b,
                            V2<T>* f, V2<T>* xn, double* part, double2 om, int zc, float2* rout = nullptr) {
    switch (op.radius) {
        case 1: return launch_zstencil_r<T, 1>(mode, grid, s, op, x, b, f, xn, part, om, zc, rout);
        case 2: return launch_zstencil_r<T, 2>(mode, grid, s, op, x, b, f, xn, part, om, zc, rout);
        case 3: return launch_zstencil_r<T, 3>(mode, grid, s, op, x, b, f, xn, part, om, zc, rout);
        case 4: return launch_zstencil_r<T, 4>(mode, grid, s, op, x, b, f, xn, part, om, zc, rout);
        case 5: return launch_zstencil_r<T, 5>(mode, grid, s, op, x, b, f, xn, part, om, zc, rout);
        case 6: return launch_zstencil_r<T, 6>(mode, grid, s, op, x, b, f, xn, part, om, zc, rout);
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
    int sms = 1, fp32 = 0;
    int64_t n = 0, ld = 0;  // ld: ring slot stride in complex values
    int sx_cap = 0, sf_cap = 0;
    double2* X = nullptr;  // FP64 rings (plain method)
    double2* F = nullptr;
    float2* X32 = nullptr;  // FP32 rings (mixed form's inner solves)
    float2* F32 = nullptr;
    float2* rhs32 = nullptr;  // mixed: FP32 inner right-hand side r = b - A x
    double2* x64 = nullptr;   // mixed: FP64 iterate
    double2* bstage = nullptr;
    double2* tmp = nullptr;  // scratch output of profiled kernels
    float2* tmp32 = nullptr;
    double* part_r = nullptr;
    double* part_b = nullptr;
    double* part_g = nullptr;
    ZState* d_st = nullptr;
    ZState* h_st = nullptr;
    dim3 sgrid;
    int zc = 16, nr = 0, nvec = 0, ngram = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // the last solve (its last inner solve for the mixed form), for aar_zprofile_kernel
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
    // block Jacobi with 2 x 2 x 2 boxes: even sides; a periodic side of at least r + 2 points, so
    // that no tap other than the distance-1 ones wraps into a box
    if (d->block != 0 && d->block != 1 && d->block != 2) return AAR_ERR_INVALID_ARG;
    if (d->block == 2) {
        if (d->nx % 2 || d->ny % 2 || d->nz % 2) return AAR_ERR_INVALID_ARG;
        if (d->periodic && (d->nx < d->radius + 2 || d->ny < d->radius + 2 || d->nz < d->radius + 2))
            return AAR_ERR_INVALID_ARG;
        const double ih2 = 1.0 / (d->h * d->h);
        const std::complex<double> dd(d->scale * (-3.0 * d->w[0] * ih2) + d->q_re, d->q_im);
        for (int t = 0; t < 4; ++t) {  // the block's eigenvalues must be nonzero
            const std::complex<double> lam = dd + (-d->scale * d->w[1] * ih2) * (3.0 - 2.0 * t);
            const std::complex<double> mu = 1.0 / (8.0 * lam);
            if (lam == std::complex<double>(0.0, 0.0) || !finite2(mu.real(), mu.imag())) return AAR_ERR_INVALID_ARG;
        }
    }
    return AAR_OK;
}

bool zvalid_params(const aar_zparams* p) {
    return p && p->m >= 0 && p->m <= AAR_MAX_M && p->p >= 1 && p->tol >= 0.0 && isfinite(p->tol) &&
           p->max_iter >= 0 && finite2(p->omega_re, p->omega_im) && finite2(p->beta_re, p->beta_im) &&
           p->inner_tol > 0.0 && p->inner_tol < 1.0 && p->max_refine >= 1;
}

double2 d2(double a, double b) { return make_double2(a, b); }

template <typename VT>
VT* zslot(VT* base, int64_t k, int ns, int64_t ld) {
    return base + (k % ns) * ld;
}

template <typename T>
V2<T>* ring_x(aar_zctx* h);
template <>
double2* ring_x<double>(aar_zctx* h) { return h->X; }
template <>
float2* ring_x<float>(aar_zctx* h) { return h->X32; }
template <typename T>
V2<T>* ring_f(aar_zctx* h);
template <>
double2* ring_f<double>(aar_zctx* h) { return h->F; }
template <>
float2* ring_f<float>(aar_zctx* h) { return h->F32; }

// Ring capacity for history length m: X holds x_{k-m} .. x_{k+1} (m + 1 slots, at least 2, as
// x_{k+1} takes the slot of x_{k-m}); F holds f_{k-m} .. f_k. The mixed form keeps FP32 rings,
// the FP32 inner right-hand side and the FP64 iterate.
aar_status zensure(aar_zctx* h, int m) {
    const int sx = std::max(m + 1, 2), sf = std::max(m + 1, 1);
    const size_t es = h->fp32 ? sizeof(float2) : sizeof(double2);
    void** px = h->fp32 ? reinterpret_cast<void**>(&h->X32) : reinterpret_cast<void**>(&h->X);
    void** pf = h->fp32 ? reinterpret_cast<void**>(&h->F32) : reinterpret_cast<void**>(&h->F);
    if (sx > h->sx_cap) {
        cudaFree(*px);
        *px = nullptr;
        h->sx_cap = 0;
        ZCHECK(cudaMalloc(px, es * h->ld * sx));
        h->sx_cap = sx;
    }
    if (sf > h->sf_cap) {
        cudaFree(*pf);
        *pf = nullptr;
        h->sf_cap = 0;
        ZCHECK(cudaMalloc(pf, es * h->ld * sf));
        h->sf_cap = sf;
    }
    if (h->fp32 && !h->x64) {
        ZCHECK(cudaMalloc(&h->x64, sizeof(double2) * h->ld));
        ZCHECK(cudaMalloc(&h->rhs32, sizeof(float2) * h->ld));
    }
    return AAR_OK;
}

template <typename T>
cudaError_t launch_zblock(aar_zctx* h, V2<T>* f, const V2<T>* x, V2<T>* xn, double2 omega, int rich) {
    const int64_t nbox = h->op.n / 8;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nbox + 255) / 256, 8LL * h->sms));
    k_zblock<T><<<grid, 256, 0, h->stream>>>(h->op, f, x, xn, omega, rich);
    return cudaGetLastError();
}

// Device address of the handle's error words (ZState::err), for the kernels' bounded waits.
int* zerr_ptr(aar_zctx* h) { return reinterpret_cast<int*>(reinterpret_cast<char*>(h->d_st) + offsetof(ZState, err)); }

// One Gram variant: its grid is one wave of resident CTAs (at most the chunk count), so that
// every CTA takes the same number of chunks; *ng receives the grid (the partial-sum count).
// Gram grid: every resident CTA slot (at most GRAM_OCC_MAX per SM), but for the FP32 passes at
// least GRAM_MIN_CH chunks per CTA, so that small systems leave the finalize few per-CTA partial
// sums to add (it adds them in FP64, at 1/64 of the FP32 rate) and each CTA's copy pipeline has
// chunks to overlap. The FP64 pass is bound by the FP64 pipe and takes every slot.
constexpr int GRAM_MIN_CH = 4;
int gram_grid(int64_t nch, int occ, int sms, int min_ch = GRAM_MIN_CH) {
    const int64_t want = (nch + min_ch - 1) / min_ch;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, std::min(occ, GRAM_OCC_MAX) * (int64_t)sms));
}

template <typename T, int NJ>
cudaError_t zgram_nj(aar_zctx* h, const ZCols<T>& cols, int c, int* ng) {
    static int occ = 0;
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_zgram<T, NJ>, 256, 0) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
    }
    const int64_t nch = (h->n + GRAM_CH - 1) / GRAM_CH;
    *ng = gram_grid(nch, occ, h->sms, sizeof(T) == 8 ? 1 : GRAM_MIN_CH);
    k_zgram<T, NJ><<<*ng, 256, 0, h->stream>>>(cols, c, h->n, h->part_g);
    return cudaGetLastError();
}

template <int C>
cudaError_t zgram_bulk_c(aar_zctx* h, const ZCols<float>& cols, int* ng) {
    static int occ = 0;
    constexpr size_t bytes = zgram_bulk_smem<C>();
    if (occ == 0) {
        if (cudaFuncSetAttribute(k_zgram_bulk<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_zgram_bulk<C>, 256, bytes) != cudaSuccess ||
            occ < 1) {
            cudaGetLastError();
            return cudaErrorInvalidConfiguration;
        }
    }
    const int64_t nch = (h->n + zb_ch<C>() - 1) / zb_ch<C>();
    *ng = gram_grid(nch, occ, h->sms);
    k_zgram_bulk<C><<<*ng, 256, bytes, h->stream>>>(cols, h->n, h->part_g, zerr_ptr(h));
    return cudaGetLastError();
}

// AAR_ZGRAM_REG=1 selects the register-fed FP32 Gram (k_zgram_reg) instead of the bulk-fed one
bool zgram_use_reg() {
    static const int v = [] {
        const char* e = getenv("AAR_ZGRAM_REG");
        return (e && e[0] == '1') ? 1 : 0;
    }();
    return v != 0;
}

cudaError_t zgram_bulk(aar_zctx* h, const ZCols<float>& cols, int c, int* ng) {
    switch (c) {
        case 1: return zgram_bulk_c<1>(h, cols, ng);
        case 2: return zgram_bulk_c<2>(h, cols, ng);
        case 3: return zgram_bulk_c<3>(h, cols, ng);
        case 4: return zgram_bulk_c<4>(h, cols, ng);
        case 5: return zgram_bulk_c<5>(h, cols, ng);
        case 6: return zgram_bulk_c<6>(h, cols, ng);
        case 7: return zgram_bulk_c<7>(h, cols, ng);
        case 8: return zgram_bulk_c<8>(h, cols, ng);
        case 9: return zgram_bulk_c<9>(h, cols, ng);
        case 10: return zgram_bulk_c<10>(h, cols, ng);
        case 11: return zgram_bulk_c<11>(h, cols, ng);
        default: return zgram_bulk_c<12>(h, cols, ng);
    }
}

template <int C>
cudaError_t zgram_reg_c(aar_zctx* h, const ZCols<float>& cols, int* ng) {
    static int occ = 0;
    if (occ == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_zgram_reg<C>, 256, 0) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
    }
    const int64_t nch = (h->n + 63) / 64;  // 64 points per CTA step (two groups of 32)
    *ng = gram_grid(nch, occ, h->sms);
    k_zgram_reg<C><<<*ng, 256, 0, h->stream>>>(cols, h->n, h->part_g);
    return cudaGetLastError();
}

cudaError_t zgram_reg(aar_zctx* h, const ZCols<float>& cols, int c, int* ng) {
    switch (c) {
        case 1: return zgram_reg_c<1>(h, cols, ng);
        case 2: return zgram_reg_c<2>(h, cols, ng);
        case 3: return zgram_reg_c<3>(h, cols, ng);
        case 4: return zgram_reg_c<4>(h, cols, ng);
        case 5: return zgram_reg_c<5>(h, cols, ng);
        case 6: return zgram_reg_c<6>(h, cols, ng);
        case 7: return zgram_reg_c<7>(h, cols, ng);
        case 8: return zgram_reg_c<8>(h, cols, ng);
        case 9: return zgram_reg_c<9>(h, cols, ng);
        case 10: return zgram_reg_c<10>(h, cols, ng);
        case 11: return zgram_reg_c<11>(h, cols, ng);
        default: return zgram_reg_c<12>(h, cols, ng);
    }
}

template <typename T>
cudaError_t zgram(aar_zctx* h, int64_t k, int c, int sf) {
    ZCols<T> cols{};
    for (int j = 0; j <= c; ++j) cols.p[j] = zslot(ring_f<T>(h), k - c + j, sf, h->ld);
    if constexpr (sizeof(T) == 4) {
        if (c <= ZGRAM_REG_MAXC) return zgram_use_reg() ? zgram_reg(h, cols, c, &h->ngram) : zgram_bulk(h, cols, c, &h->ngram);
    }
    const int E = c * (c + 1) / 2 + c;
    int* ng = &h->ngram;
    if (E <= 16) return zgram_nj<T, 2>(h, cols, c, ng);
    if (E <= 32) return zgram_nj<T, 4>(h, cols, c, ng);
    if (E <= 56) return zgram_nj<T, 7>(h, cols, c, ng);
    if (E <= 96) return zgram_nj<T, 12>(h, cols, c, ng);
    return zgram_nj<T, (ZMAXE + 7) / 8>(h, cols, c, ng);
}

template <typename T>
cudaError_t zupdate(aar_zctx* h, int64_t k, int c, int sx, int sf, double2 beta, V2<T>* xout, int force, int p,
                    double2 omega) {
    ZCols<T> xs{}, fs{};
    for (int j = 0; j <= c; ++j) {
        xs.p[j] = zslot(ring_x<T>(h), k - c + j, sx, h->ld);
        fs.p[j] = zslot(ring_f<T>(h), k - c + j, sf, h->ld);
    }
    k_zupdate<T><<<h->nvec, 256, 0, h->stream>>>(h->d_st, xs, fs, c, xout, beta, h->n, force, k, p, omega);
    return cudaGetLastError();
}

cudaError_t zfinalize(aar_zctx* h, const double* part, int nr_used, int c, double tol, double2 beta, int mode) {
    k_zfinalize<<<1, 256, 0, h->stream>>>(h->d_st, part, nr_used, h->part_g, h->ngram, h->part_b, h->nvec, c, tol,
                                          beta, mode);
    return cudaGetLastError();
}

enum { RUN_CONV = 0, RUN_CAP = 1, RUN_BREAK = 2, RUN_STALL = 3 };

struct RunResult {
    int status = RUN_CAP;
    int64_t k_final = 0;  // iterations performed; the result is iterate k_final of the ring
    int anderson = 0, eig = 0, rank = 0, last_c = 0;
    int64_t last_and = -1, launches = 0;
    double r_last = NAN;
};

// AAR iterations k = 0, 1, ... on A u = rhs from the iterate already in slot 0 of the T ring, until
// the first Anderson step with ||rhs - A u_k|| / st.nb <= tol_rel (st.nb set by the caller), kmax
// iterations, a breakdown, or (stall > 0) an Anderson step whose residual is not 10% below the
// one `stall` Anderson steps earlier (the FP32 rounding floor of an inner solve). One host
// synchronisation per Anderson step reads the finalize's outcome.
template <typename T>
aar_status run_aar(aar_zctx* h, const V2<T>* rhs, const aar_zparams& P, double tol_rel, int64_t kmax, int stall,
                   RunResult& R) {
    const int sx = std::max(P.m + 1, 2), sf = std::max(P.m + 1, 1);
    cudaStream_t s = h->stream;
    const double2 omega = d2(P.omega_re, P.omega_im), beta = d2(P.beta_re, P.beta_im);
    V2<T>* X = ring_x<T>(h);
    V2<T>* F = ring_f<T>(h);
    R = RunResult{};
    double hist[64];  // residuals of the last Anderson steps (circular)
    if (kmax <= 0) return AAR_OK;
    int64_t k = 0;
    for (;;) {
        const V2<T>* xk = zslot(X, k, sx, h->ld);
        V2<T>* fk = zslot(F, k, sf, h->ld);
        if ((k + 1) % P.p != 0) {
            ZCHECK(launch_zstencil<T>(h->op.blk ? ZM_BRES : ZM_RICH, h->sgrid, s, h->op, xk, rhs, fk,
                                      zslot(X, k + 1, sx, h->ld), nullptr, omega, h->zc));
            ++R.launches;
            if (h->op.blk) {
                ZCHECK(launch_zblock<T>(h, fk, xk, zslot(X, k + 1, sx, h->ld), omega, 1));
                ++R.launches;
            }
        } else {
            const int c = (int)std::min<int64_t>(k, P.m);
            ZCHECK(launch_zstencil<T>(h->op.blk ? ZM_BRES_AND : ZM_AND, h->sgrid, s, h->op, xk, rhs, fk, nullptr,
                                      h->part_r, omega, h->zc));
            ++R.launches;
            if (h->op.blk) {
                ZCHECK(launch_zblock<T>(h, fk, xk, nullptr, omega, 0));
                ++R.launches;
            }
            if (c > 0) {
                ZCHECK(zgram<T>(h, k, c, sf));
                ++R.launches;
            }
            ZCHECK(zfinalize(h, h->part_r, h->nr, c, tol_rel, beta, 1));
            ZCHECK(zupdate<T>(h, k, c, sx, sf, beta, zslot(X, k + 1, sx, h->ld), 0, P.p, omega));
            R.launches += 2;
            ZCHECK(cudaMemcpyAsync(h->h_st, h->d_st, sizeof(ZState), cudaMemcpyDeviceToHost, s));
            ZCHECK(cudaStreamSynchronize(s));
            const ZState& S = *h->h_st;
            if (S.err[0]) return AAR_ERR_TIMEOUT;  // a bounded wait gave up: results are not trustworthy
            hist[R.anderson % 64] = S.r;
            ++R.anderson;
            R.last_and = k;
            R.last_c = c;
            R.r_last = S.r;
            if (S.status == ZS_CONV) {
                R.status = RUN_CONV;
                R.k_final = k;
                return AAR_OK;
            }
            if (S.status == ZS_BREAK) {
                R.status = RUN_BREAK;
                R.k_final = k;
                return AAR_OK;
            }
            if (c > 0 && S.eig) ++R.eig;
            R.rank = S.rank;
            if (stall > 0 && R.anderson > stall && S.r > 0.9 * hist[(R.anderson - 1 - stall) % 64]) {
                R.status = RUN_STALL;
                R.k_final = k;
                return AAR_OK;
            }
        }
        ++k;
        if (k >= kmax) {
            R.status = RUN_CAP;
            R.k_final = k;
            return AAR_OK;
        }
    }
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
    p->inner_tol = 1e-3;
    p->max_refine = 30;
    p->reserved = 0;
    return AAR_OK;
}

aar_status aar_zcreate_stencil(const aar_zstencil_desc* desc, int32_t precision, void* stream, aar_zhandle* out) {
    if (!out) return AAR_ERR_INVALID_ARG;
    *out = nullptr;
    const aar_status vs = zvalid_desc(desc);
    if (vs != AAR_OK) return vs;
    if (precision != AAR_FP64 && precision != AAR_MIXED) return AAR_ERR_INVALID_ARG;
    const double ih2 = 1.0 / (desc->h * desc->h);
    const std::complex<double> dd(desc->scale * (-3.0 * desc->w[0] * ih2) + desc->q_re, desc->q_im);
    if (dd == std::complex<double>(0.0, 0.0)) return AAR_ERR_INVALID_ARG;
    const std::complex<double> di = 1.0 / dd;
    if (!finite2(di.real(), di.imag())) return AAR_ERR_INVALID_ARG;

    aar_zctx* h = new (std::nothrow) aar_zctx();
    if (!h) return AAR_ERR_OOM;
    h->stream = (cudaStream_t)stream;
    h->fp32 = precision == AAR_MIXED;
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
    if (desc->block == 2) {
        op.blk = 1;
        for (int t = 0; t < 4; ++t) {
            const std::complex<double> lam = dd + op.ck[1] * (3.0 - 2.0 * t);
            const std::complex<double> mu = 1.0 / (8.0 * lam);
            op.mu[t] = d2(mu.real(), mu.imag());
        }
    }
    h->n = op.n;
    h->ld = (op.n + 31) / 32 * 32;
    auto fail = [&](aar_status st) {
        aar_zdestroy(h);
        return st;
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
    h->ngram = 1;  // set by each Gram launch (its grid)
    if (cudaMalloc(&h->part_r, sizeof(double) * h->nr) != cudaSuccess ||
        cudaMalloc(&h->part_b, sizeof(double) * h->nvec) != cudaSuccess ||
        cudaMalloc(&h->part_g, sizeof(double) * 2 * ZMAXE * GRAM_OCC_MAX * h->sms) != cudaSuccess ||
        cudaMalloc(&h->d_st, sizeof(ZState)) != cudaSuccess ||
        cudaMallocHost(&h->h_st, sizeof(ZState)) != cudaSuccess ||
        cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
        cudaGetLastError();
        return fail(AAR_ERR_OOM);
    }
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
    ZCHECK(cudaMemsetAsync(zerr_ptr(h), 0, sizeof(int) * 4, h->stream));
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
    const double2 beta = d2(P.beta_re, P.beta_im);
    // ||b||
    k_znorm<<<h->nvec, 256, 0, s>>>(bd, n, h->part_b);
    ZCHECK(cudaGetLastError());
    ZCHECK(zfinalize(h, h->part_b, h->nvec, 0, P.tol, beta, 0));
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
    RunResult R;
    int status = AAR_NOT_CONVERGED, refinements = 0, anderson = 0, eig = 0, rank = 0;
    int64_t its = 0;
    double r_last = NAN;
    const void* result = nullptr;
    if (!h->fp32) {
        // plain method: AAR in FP64 on A x = b from x_0
        double2* X0 = h->X;
        if (x0) ZCHECK(cudaMemcpyAsync(X0, x0, sizeof(double2) * n, cudaMemcpyDefault, s));
        else ZCHECK(cudaMemsetAsync(X0, 0, sizeof(double2) * n, s));
        st = run_aar<double>(h, bd, P, P.tol, P.max_iter, 0, R);
        if (st != AAR_OK) return st;
        launches += R.launches;
        its = R.k_final;
        anderson = R.anderson;
        eig = R.eig;
        rank = R.rank;
        r_last = R.r_last;
        status = R.status == RUN_CONV ? AAR_OK : R.status == RUN_BREAK ? AAR_ERR_BREAKDOWN : AAR_NOT_CONVERGED;
        result = zslot(h->X, R.k_final, sx, h->ld);
        h->solved = R.last_and >= 0;
    } else {
        // mixed form: r = b - A x in FP64, FP32 AAR on A d = r to max(inner_tol, tol ||b|| / (2 ||r||)),
        // x += d in FP64, until ||b - A x|| / ||b|| <= tol
        if (x0) ZCHECK(cudaMemcpyAsync(h->x64, x0, sizeof(double2) * n, cudaMemcpyDefault, s));
        else ZCHECK(cudaMemsetAsync(h->x64, 0, sizeof(double2) * n, s));
        for (;;) {
            ZCHECK(launch_zstencil<double>(ZM_RESOUT, h->sgrid, s, h->op, h->x64, bd, nullptr, nullptr, h->part_r,
                                           d2(0, 0), h->zc, h->rhs32));
            ZCHECK(zfinalize(h, h->part_r, h->nr, 0, 0.0, beta, 0));  // st.nb = ||r||
            launches += 2;
            ZCHECK(cudaMemcpyAsync(h->h_st, h->d_st, sizeof(ZState), cudaMemcpyDeviceToHost, s));
            ZCHECK(cudaStreamSynchronize(s));
            const double rr = h->h_st->nb / nb;
            r_last = rr;
            if (!isfinite(rr)) {
                status = AAR_ERR_BREAKDOWN;
                break;
            }
            if (rr <= P.tol) {
                status = AAR_OK;
                break;
            }
            if (refinements >= P.max_refine || its >= P.max_iter) {
                status = AAR_NOT_CONVERGED;
                break;
            }
            const double tin = std::max(P.inner_tol, 0.5 * P.tol / rr);
            ZCHECK(cudaMemsetAsync(h->X32, 0, sizeof(float2) * n, s));
            RunResult Ri;
            st = run_aar<float>(h, h->rhs32, P, tin, P.max_iter - its, 12, Ri);
            if (st != AAR_OK) return st;
            launches += Ri.launches;
            its += Ri.k_final;
            anderson += Ri.anderson;
            eig += Ri.eig;
            rank = Ri.rank;
            if (Ri.last_and >= 0) {
                R = Ri;
                h->solved = true;
            }
            if (Ri.status == RUN_BREAK || Ri.k_final == 0) {
                status = Ri.status == RUN_BREAK ? AAR_ERR_BREAKDOWN : AAR_NOT_CONVERGED;
                break;
            }
            k_zadd<<<h->nvec, 256, 0, s>>>(h->x64, zslot(h->X32, Ri.k_final, sx, h->ld), n);
            ZCHECK(cudaGetLastError());
            ++launches;
            ++refinements;
        }
        result = h->x64;
    }
    ZCHECK(cudaMemcpyAsync(x, result, sizeof(double2) * n, cudaMemcpyDefault, s));
    ZCHECK(cudaStreamSynchronize(s));
    h->last_k = R.last_and;
    h->last_c = R.last_c;
    h->last_sx = sx;
    h->last_sf = sf;
    h->last_p = P;
    h->last_b = bd;
    if (info) {
        info->iterations = its;
        info->anderson_steps = anderson;
        info->refinements = refinements;
        info->rel_residual = r_last;
        info->status = status;
        info->last_rank = rank;
        info->ticks = its;
        info->launches = launches;
        info->eigen_steps = eig;
    }
    return (aar_status)status;
}

aar_status aar_zapply(aar_zhandle h, const double* x, double* y) {
    if (!h || !x || !y || x == y) return AAR_ERR_INVALID_ARG;
    if (!zis_device_ptr(x) || !zis_device_ptr(y)) return AAR_ERR_INVALID_ARG;
    ZCHECK(launch_zstencil<double>(ZM_APPLY, h->sgrid, h->stream, h->op, reinterpret_cast<const double2*>(x), nullptr,
                                   reinterpret_cast<double2*>(y), nullptr, nullptr, d2(0, 0), h->zc));
    ZCHECK(cudaStreamSynchronize(h->stream));
    return AAR_OK;
}

aar_status aar_zrel_residual(aar_zhandle h, const double* b, const double* x, double* rel) {
    if (!h || !b || !x || !rel) return AAR_ERR_INVALID_ARG;
    if (!zis_device_ptr(b) || !zis_device_ptr(x)) return AAR_ERR_INVALID_ARG;
    cudaStream_t s = h->stream;
    const double2* bd = reinterpret_cast<const double2*>(b);
    ZCHECK(launch_zstencil<double>(ZM_RESID, h->sgrid, s, h->op, reinterpret_cast<const double2*>(x), bd, nullptr,
                                   nullptr, h->part_r, d2(0, 0), h->zc));
    k_znorm<<<h->nvec, 256, 0, s>>>(bd, h->n, h->part_b);
    ZCHECK(cudaGetLastError());
    ZCHECK(zfinalize(h, h->part_r, h->nr, 0, 0.0, d2(0, 0), 2));
    ZCHECK(cudaMemcpyAsync(h->h_st, h->d_st, sizeof(ZState), cudaMemcpyDeviceToHost, s));
    ZCHECK(cudaStreamSynchronize(s));
    *rel = h->h_st->r;  // the ring and the update's coefficients are untouched
    return AAR_OK;
}

}  // extern "C"

namespace {

template <typename T>
aar_status zprofile(aar_zhandle h, int32_t kernel, int32_t launches, float* ms) {
    const aar_zparams& P = h->last_p;
    const int64_t k = h->last_k;
    const int c = h->last_c, sx = h->last_sx, sf = h->last_sf;
    const double2 omega = d2(P.omega_re, P.omega_im), beta = d2(P.beta_re, P.beta_im);
    cudaStream_t s = h->stream;
    if (kernel == AAR_K_SWEEP && P.p == 1) return AAR_ERR_UNSUPPORTED;
    if (kernel < AAR_K_SWEEP || kernel > AAR_K_BLOCK) return AAR_ERR_INVALID_ARG;
    if (kernel == AAR_K_BLOCK && !h->op.blk) return AAR_ERR_UNSUPPORTED;
    if (kernel == AAR_K_RESID64 && !h->fp32) return AAR_ERR_UNSUPPORTED;
    if (kernel == AAR_K_GRAM && c == 0) return AAR_ERR_UNSUPPORTED;
    V2<T>* X = ring_x<T>(h);
    V2<T>* F = ring_f<T>(h);
    const V2<T>* xk = zslot(X, k, sx, h->ld);
    V2<T>* fk = zslot(F, k, sf, h->ld);
    const V2<T>* rhs = nullptr;
    if constexpr (sizeof(T) == 8) rhs = h->last_b;
    else rhs = h->rhs32;
    // x_{k+1} of the timed sweep or update goes to a scratch vector, so the history of step k
    // stays intact (the sweeps rewrite f_k with the same values)
    V2<T>* xn = nullptr;
    if constexpr (sizeof(T) == 8) {
        if (!h->tmp) ZCHECK(cudaMalloc(&h->tmp, sizeof(double2) * h->ld));
        xn = h->tmp;
    } else {
        if (!h->tmp32) ZCHECK(cudaMalloc(&h->tmp32, sizeof(float2) * h->ld));
        xn = h->tmp32;
    }
    auto one = [&]() -> cudaError_t {
        switch (kernel) {
            case AAR_K_SWEEP:
                return launch_zstencil<T>(h->op.blk ? ZM_BRES : ZM_RICH, h->sgrid, s, h->op, xk, rhs, fk, xn, nullptr,
                                          omega, h->zc);
            case AAR_K_SWEEP_ANDERSON:
                return launch_zstencil<T>(h->op.blk ? ZM_BRES_AND : ZM_AND, h->sgrid, s, h->op, xk, rhs, fk, nullptr,
                                          h->part_r, omega, h->zc);
            case AAR_K_GRAM: return zgram<T>(h, k, c, sf);
            case AAR_K_UPDATE: return zupdate<T>(h, k, c, sx, sf, beta, xn, 1, P.p, omega);
            case AAR_K_RESID64:
                // the refinement's FP64 residual; its FP32 output goes to a scratch vector
                if (!h->tmp32) {
                    cudaError_t e = cudaMalloc(&h->tmp32, sizeof(float2) * h->ld);
                    if (e != cudaSuccess) return e;
                }
                return launch_zstencil<double>(ZM_RESOUT, h->sgrid, s, h->op, h->x64, h->last_b, nullptr, nullptr,
                                               h->part_r, d2(0, 0), h->zc, h->tmp32);
            case AAR_K_BLOCK: return launch_zblock<T>(h, fk, xk, xn, omega, 1);
            default: return zfinalize(h, h->part_r, h->nr, c, 0.0, beta, 1);
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

}  // namespace

extern "C" {

aar_status aar_zprofile_kernel(aar_zhandle h, int32_t kernel, int32_t launches, float* ms) {
    if (!h || !ms || launches < 1 || !h->solved) return AAR_ERR_INVALID_ARG;
    return h->fp32 ? zprofile<float>(h, kernel, launches, ms) : zprofile<double>(h, kernel, launches, ms);
}

aar_status aar_zdestroy(aar_zhandle h) {
    if (!h) return AAR_ERR_INVALID_ARG;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    cudaFree(h->X);
    cudaFree(h->F);
    cudaFree(h->X32);
    cudaFree(h->F32);
    cudaFree(h->rhs32);
    cudaFree(h->x64);
    cudaFree(h->bstage);
    cudaFree(h->tmp);
    cudaFree(h->tmp32);
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

// aar_linalg.cuh -- small dense linear algebra run by one to four warps inside the finalize kernels
// (the m x m, or 2m x 2m for complex systems, pseudoinverse solve of Eq. 3).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <utility>

namespace aar {

// 1/d for a positive normal d: the hardware's approximate FP64 reciprocal refined by two
// Newton-Raphson steps (x <- x + x (1 - d x)), each of which doubles the number of correct bits.
__device__ __forceinline__ double recip_nr(double d) {
    double x;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
    double e = fma(-d, x, 1.0);
    x = fma(x, e, x);
    e = fma(-d, x, 1.0);
    return fma(x, e, x);
}

// 1/sqrt(x) for a positive normal x: the hardware's approximate FP64 reciprocal square root refined
// by two Newton-Raphson steps y <- y (3/2 - (x/2) y^2), each of which doubles the correct bits.
__device__ __forceinline__ double rsqrt_nr(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double h = 0.5 * x;
    y = y * fma(-h * y, y, 1.5);
    return y * fma(-h * y, y, 1.5);
}

// Jacobi eigendecomposition S = V diag(lam) V^T of a c x c symmetric matrix held in shared memory
// (leading dimension LD, c <= 32); on return the diagonal of S holds lam. Every
// sweep visits each off-diagonal pair (p, q) once, in the round-robin order of the parallel
// Jacobi method: round t pairs the indices (plus one dummy when c is odd) so that no index occurs
// twice, and its n/2 plane rotations, which commute, are computed by n/2 lanes at once and
// applied together. An entry with |S_pq| <= 2^-52 sqrt(|S_pp S_qq|) is negligible at working
// precision and is zeroed instead of rotated; the method stops after a sweep that rotated nothing
// (at most 100 sweeps). The rotation annihilating S_pq: with d = S_qq - S_pp and e = 2 S_pq,
// t = tan(theta) = sign(d) e / (|d| + sqrt(d^2 + e^2)) (the smaller root of t^2 + 2 (d/e) t - 1,
// scaled so that d and e enter without a division), cos = 1/sqrt(1 + t^2), sin = t cos.
// FP64 is slow on this part, so the square roots and the one reciprocal are Newton-refined
// hardware approximations (rsqrt_nr, recip_nr) rather than correctly rounded operations.
// Run by the first 32 NW threads of a 1-D CTA (NW warps; barrier 1 among them): warp 0 computes
// each round's rotations and all NW warps apply them (the FP64 pipe of one SM sub-partition was
// the bottleneck of a one-warp solver). Every entry is updated by the same operations in the same
// order as in a one-warp solver, so the result does not depend on NW.
template <int LD, int NW>
__device__ void cta_sym_eig(int c, double* Sm, double* Vm) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int NT = 32 * NW;
    __shared__ int rp[16], rq[16], s_rot[2];
    __shared__ double rc[16], rs[16];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto bar = [] { asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory"); };
    for (int r = tid; r < c; r += NT)
        for (int q = 0; q < c; ++q) Vm[r * LD + q] = (r == q) ? 1.0 : 0.0;
    bar();
    if (c < 2) return;
    const int n = c + (c & 1), np = n / 2;  // indices incl. the dummy (= c when c is odd); pairs
    const double eps2 = ldexp(1.0, -104);
    int par = 0;  // flag word of the round: alternates every round, across sweeps too
    for (int sweep = 0; sweep < 100; ++sweep) {
        bool rotated = false;  // identical in every thread
        for (int t = 0; t < n - 1; ++t, par ^= 1) {
            if (warp == 0) {
                // lane i < np: the rotation of pair i of round t (position 0 fixed, 1 .. n-1 cycled)
                int p = 0, q = -1;
                double cs = 1.0, sn = 0.0;
                if (lane < np) {
                    const int a = lane == 0 ? 0 : 1 + (lane - 1 + t) % (n - 1);
                    const int b = 1 + (n - 2 - lane + t) % (n - 1);
                    p = min(a, b);
                    const int qq = max(a, b);
                    if (qq < c) {
                        const double apq = Sm[p * LD + qq];
                        // the tests below compare bit patterns (integer instructions; an FP64
                        // compare-and-select is about 230 cycles on this part): apq != 0, and
                        // apq^2 <= eps2 |app aqq| for the non-negative operands (a NaN bound
                        // compares false, as in FP64)
                        if ((__double_as_longlong(apq) << 1) != 0) {
                            const double app = Sm[p * LD + p], aqq = Sm[qq * LD + qq];
                            const long long lhs = __double_as_longlong(apq * apq);
                            const long long rhs = __double_as_longlong(eps2 * fabs(app * aqq));
                            if (lhs <= rhs && rhs <= 0x7ff0000000000000LL) {
                                Sm[p * LD + qq] = 0.0;
                                Sm[qq * LD + p] = 0.0;
                            } else {
                                // t is invariant under a common positive scale of d and e: scale by
                                // about 1/max(|d|, |e|) so that the squares neither overflow nor
                                // underflow
                                const double d0 = aqq - app, e0 = 2.0 * apq;
                                double inv;
                                asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(inv) : "d"(fmax(fabs(d0), fabs(e0))));
                                const double d = d0 * inv, e = e0 * inv;
                                const double x = fma(d, d, e * e);
                                const double den = fabs(d) + x * rsqrt_nr(x);
                                // sign(d) with d = -0 counted as non-negative, from the bits
                                const long long db = __double_as_longlong(d);
                                const bool dneg = db < 0 && (db << 1) != 0;
                                const double tt = (dneg ? -e : e) * recip_nr(den);
                                cs = rsqrt_nr(fma(tt, tt, 1.0));
                                sn = tt * cs;
                                q = qq;
                            }
                        }
                    }
                    rp[lane] = p;
                    rq[lane] = q;
                    rc[lane] = cs;
                    rs[lane] = sn;
                }
                const bool any = __any_sync(FULL, q >= 0);
                if (lane == 0) s_rot[par] = any ? 1 : 0;
            }
            bar();  // the rotations and the zeroed negligible entries are visible to every thread
            // the flag alternates between two words: warp 0 writes this word again two rounds on,
            // after every thread has passed the next round's barrier (so has read it)
            const bool any = s_rot[par] != 0;
            if (!any) continue;
            rotated = true;
            // S <- S J: columns p_i, q_i of every row (disjoint pairs: no two items share an entry)
            for (int it = tid; it < c * np; it += NT) {
                const int i = it / c, r = it - i * c;
                const int pi = rp[i], qi = rq[i];
                if (qi >= 0) {
                    const double ci = rc[i], si = rs[i];
                    const double skp = Sm[r * LD + pi], skq = Sm[r * LD + qi];
                    Sm[r * LD + pi] = ci * skp - si * skq;
                    Sm[r * LD + qi] = si * skp + ci * skq;
                }
            }
            bar();
            // S <- J^T S (rows p_i, q_i) and V <- V J
            for (int it = tid; it < c * np; it += NT) {
                const int i = it / c, r = it - i * c;
                const int pi = rp[i], qi = rq[i];
                if (qi >= 0) {
                    const double ci = rc[i], si = rs[i];
                    const double spk = Sm[pi * LD + r], sqk = Sm[qi * LD + r];
                    Sm[pi * LD + r] = ci * spk - si * sqk;
                    Sm[qi * LD + r] = si * spk + ci * sqk;
                    const double vkp = Vm[r * LD + pi], vkq = Vm[r * LD + qi];
                    Vm[r * LD + pi] = ci * vkp - si * vkq;
                    Vm[r * LD + qi] = si * vkp + ci * vkq;
                }
            }
            bar();
        }
        if (!rotated) break;
    }
}

// FP64 comparisons and divisions are slow on this part (a dependent compare-and-select takes
// about 230 cycles, a division about 560, against 65 for a multiply-add), so the factorisation
// below compares non-negative doubles through their bit patterns (ordered like the values) and
// divides by multiplying with a Newton-refined reciprocal.
__device__ __forceinline__ bool finite_bits(double v) {
    return (__double_as_longlong(v) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

// gamma = G^{-1} g for the c x c Gram system (G in Sm with leading dimension LD, g in gv) by an
// LDL^T factorisation on the 32 lanes of one warp, compiled for each c (no predicated-off
// columns): lane i keeps row i of the remaining matrix, then of L, in registers; L also goes to
// Vm for the back substitution. False when a pivot is not above c 2^-52 max_i G_ii (the rank
// test of the pseudoinverse) or the result is not finite: the caller then takes the
// eigen-decomposition.
// CERT (the plain FP64 form): also false unless trace(G) trace(G^-1) ncut < 2^42. The condition
// number is at most trace(G) trace(G^-1), so every eigenvalue then lies at least 2^10 above the
// pseudoinverse's cut ncut 2^-52 lambda_max: pinv(G) g = G^-1 g, and the solve gives the
// eigen-decomposition's gamma up to rounding. trace(G^-1) = sum_k ||row k of L^-1||^2 / d_k;
// lane j forms column j of L^-1 by forward substitution.
// ncut: the n of the pseudoinverse's cut n 2^-52 lambda_max (C for a real c x c system; c for the
// real 2c x 2c form of a complex one).
template <int C, int LD, bool CERT>
__device__ bool ldl_solve_warp(const double* Sm, const double* gv, double* Vm, int lane, double& z, double ncut) {
    static_assert(C <= 32 && C <= LD, "one row per lane");
    constexpr unsigned FULL = 0xffffffffu;
    double a[C];
#pragma unroll
    for (int q = 0; q < C; ++q) a[q] = lane < C ? Sm[lane * LD + q] : 0.0;
    // max_i G_ii through the bit patterns (non-negative finite diagonals; any other fails)
    const double di = lane < C ? Sm[lane * LD + lane] : 0.0;
    const long long db = __double_as_longlong(di);
    bool ok = __all_sync(FULL, lane >= C || (db >= 0 && finite_bits(di)));
    long long gb = lane < C ? db : 0;
    for (int o = 16; o > 0; o >>= 1) {
        const long long v = __shfl_xor_sync(FULL, gb, o);
        gb = v > gb ? v : gb;
    }
    ok = ok && gb > 0;
    const double piv_min = ncut * ldexp(1.0, -52) * __longlong_as_double(gb);
    const long long pb = __double_as_longlong(piv_min);
    double dinv = 1.0;  // lane j: 1 / d_j
#pragma unroll
    for (int j = 0; j < C; ++j) {
        if (!ok) break;  // uniform across the warp
        const double dj = __shfl_sync(FULL, a[j], j);
        if (!(__double_as_longlong(dj) > pb)) {  // dj <= piv_min (or negative)
            ok = false;
            break;
        }
        const double inv = recip_nr(dj);
        if (lane == j) dinv = inv;
        const bool below = lane > j && lane < C;
        const double lij = below ? a[j] * inv : 0.0;
        const double t = below ? -a[j] : 0.0;  // -(G_ij after j eliminations)
#pragma unroll
        for (int q = j + 1; q < C; ++q) {
            const double lqj = __shfl_sync(FULL, lij, q);
            if (lane >= q && lane < C) a[q] = fma(t, lqj, a[q]);
        }
        if (below) a[j] = lij;
    }
    z = 0.0;
    if (!ok) return false;
#pragma unroll
    for (int q = 0; q < C; ++q)
        if (q < lane && lane < C) Vm[lane * LD + q] = a[q];
    __syncwarp();
    double y = lane < C ? gv[lane] : 0.0;
#pragma unroll
    for (int j = 0; j < C; ++j) {  // L y = g
        const double yj = __shfl_sync(FULL, y, j);
        if (lane > j && lane < C) y = fma(-a[j], yj, y);
    }
    z = lane < C ? y * dinv : 0.0;  // D w = y
#pragma unroll
    for (int j = C - 1; j >= 0; --j) {  // L^T gamma = w
        const double zj = __shfl_sync(FULL, z, j);
        if (lane < j) z = fma(-Vm[j * LD + lane], zj, z);
    }
    if (!__all_sync(FULL, lane >= C || finite_bits(z))) return false;
    if constexpr (CERT) {
        double y[C];  // column `lane` of L^-1 (rows below the lane's own start at zero)
#pragma unroll
        for (int i = 0; i < C; ++i) {
            y[i] = i == lane ? 1.0 : 0.0;
#pragma unroll
            for (int q = 0; q < i; ++q) y[i] = fma(-Vm[i * LD + q], y[q], y[i]);
        }
        double tr = 0.0;  // this column's share of trace(G^-1)
#pragma unroll
        for (int i = 0; i < C; ++i) tr = fma(y[i] * y[i], __shfl_sync(FULL, dinv, i), tr);
        double tg = lane < C ? di : 0.0;
        if (lane >= C) tr = 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            tr += __shfl_xor_sync(FULL, tr, o);
            tg += __shfl_xor_sync(FULL, tg, o);
        }
        const double prod = tr * tg * ncut;
        return finite_bits(prod) && prod < ldexp(1.0, 42);
    }
    return true;
}

// ldl_solve_warp for a runtime size c in {Cs + 1}
template <int LD, bool CERT, int... Cs>
__device__ __forceinline__ bool ldl_solve_dispatch(int c, const double* Sm, const double* gv, double* Vm, int lane,
                                                   double& z, std::integer_sequence<int, Cs...>) {
    bool ok = false;
    ((c == Cs + 1 ? (ok = ldl_solve_warp<Cs + 1, LD, CERT>(Sm, gv, Vm, lane, z, (double)(Cs + 1)), 0) : 0), ...);
    return ok;
}

}  // namespace aar

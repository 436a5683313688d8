// aar_linalg.cuh -- small dense linear algebra run by one warp inside the finalize kernels
// (the m x m, or 2m x 2m for complex systems, pseudoinverse solve of Eq. 3).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

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
// (leading dimension LD, c <= 32), run by one warp; on return the diagonal of S holds lam. Every
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
template <int LD>
__device__ void warp_sym_eig(int c, double* Sm, double* Vm) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (int r = lane; r < c; r += 32)
        for (int q = 0; q < c; ++q) Vm[r * LD + q] = (r == q) ? 1.0 : 0.0;
    __syncwarp();
    if (c < 2) return;
    const int n = c + (c & 1), np = n / 2;  // indices incl. the dummy (= c when c is odd); pairs
    const int nu = (c * np + 31) / 32;      // update items (row, pair) per lane
    const double eps2 = ldexp(1.0, -104);
    for (int sweep = 0; sweep < 100; ++sweep) {
        bool rotated = false;  // identical in every lane
        for (int t = 0; t < n - 1; ++t) {
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
                    if (apq != 0.0) {
                        const double app = Sm[p * LD + p], aqq = Sm[qq * LD + qq];
                        if (apq * apq <= eps2 * fabs(app * aqq)) {
                            Sm[p * LD + qq] = 0.0;
                            Sm[qq * LD + p] = 0.0;
                        } else {
                            // t is invariant under a common positive scale of d and e: scale by
                            // about 1/max(|d|, |e|) so that the squares neither overflow nor underflow
                            const double d0 = aqq - app, e0 = 2.0 * apq;
                            double inv;
                            asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(inv) : "d"(fmax(fabs(d0), fabs(e0))));
                            const double d = d0 * inv, e = e0 * inv;
                            const double x = fma(d, d, e * e);
                            const double den = fabs(d) + x * rsqrt_nr(x);
                            const double tt = (d >= 0.0 ? e : -e) * recip_nr(den);
                            cs = rsqrt_nr(fma(tt, tt, 1.0));
                            sn = tt * cs;
                            q = qq;
                        }
                    }
                }
            }
            if (!__any_sync(FULL, q >= 0)) {
                __syncwarp();
                continue;
            }
            rotated = true;
            __syncwarp();  // the zeroed negligible entries are visible to every lane
            // S <- S J: columns p_i, q_i of every row (disjoint pairs: no two items share an entry)
            for (int u = 0; u < nu; ++u) {
                const int it = lane + 32 * u, i = it < c * np ? it / c : 0, r = it - i * c;
                const int pi = __shfl_sync(FULL, p, i), qi = __shfl_sync(FULL, q, i);
                const double ci = __shfl_sync(FULL, cs, i), si = __shfl_sync(FULL, sn, i);
                if (it < c * np && qi >= 0) {
                    const double skp = Sm[r * LD + pi], skq = Sm[r * LD + qi];
                    Sm[r * LD + pi] = ci * skp - si * skq;
                    Sm[r * LD + qi] = si * skp + ci * skq;
                }
            }
            __syncwarp();
            // S <- J^T S (rows p_i, q_i) and V <- V J
            for (int u = 0; u < nu; ++u) {
                const int it = lane + 32 * u, i = it < c * np ? it / c : 0, r = it - i * c;
                const int pi = __shfl_sync(FULL, p, i), qi = __shfl_sync(FULL, q, i);
                const double ci = __shfl_sync(FULL, cs, i), si = __shfl_sync(FULL, sn, i);
                if (it < c * np && qi >= 0) {
                    const double spk = Sm[pi * LD + r], sqk = Sm[qi * LD + r];
                    Sm[pi * LD + r] = ci * spk - si * sqk;
                    Sm[qi * LD + r] = si * spk + ci * sqk;
                    const double vkp = Vm[r * LD + pi], vkq = Vm[r * LD + qi];
                    Vm[r * LD + pi] = ci * vkp - si * vkq;
                    Vm[r * LD + qi] = si * vkp + ci * vkq;
                }
            }
            __syncwarp();
        }
        if (!rotated) break;
    }
}

}  // namespace aar

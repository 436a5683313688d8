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

// Cyclic Jacobi eigendecomposition S = V diag(lam) V^T of a c x c symmetric matrix held in
// shared memory (leading dimension LD, c <= 32), run by one warp. Row-order sweeps over the pairs
// (p, q); an entry with |S_pq| <= 2^-52 sqrt(|S_pp S_qq|) is negligible at working precision and
// is zeroed instead of rotated; the method stops after a sweep that rotated nothing (at most 100
// sweeps). Lane 0 computes each rotation (FP64 division and square roots are slow on this part,
// so they run on one lane) and publishes it in rot[]; lane r then updates row/column r.
template <int LD>
__device__ void warp_sym_eig(int c, double* Sm, double* Vm, double* rot) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < c; ++r)
        if (lane == r)
            for (int q = 0; q < c; ++q) Vm[r * LD + q] = (r == q) ? 1.0 : 0.0;
    __syncwarp();
    const double eps = ldexp(1.0, -52);
    for (int sweep = 0; sweep < 100; ++sweep) {
        int rotated = 0;  // identical in every lane (derived from rot[2])
        for (int p = 0; p < c - 1; ++p) {
            for (int q = p + 1; q < c; ++q) {
                if (lane == 0) {
                    const double apq = Sm[p * LD + q];
                    double cs = 1.0, sn = 0.0, act = 0.0;
                    if (apq != 0.0) {
                        const double app = Sm[p * LD + p], aqq = Sm[q * LD + q];
                        if (fabs(apq) <= eps * sqrt(fabs(app * aqq))) {
                            Sm[p * LD + q] = 0.0;
                            Sm[q * LD + p] = 0.0;
                        } else {
                            const double theta = (aqq - app) / (2.0 * apq);
                            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                            cs = 1.0 / sqrt(t * t + 1.0);
                            sn = t * cs;
                            act = 1.0;
                        }
                    }
                    rot[0] = cs;
                    rot[1] = sn;
                    rot[2] = act;
                }
                __syncwarp();
                const double cs = rot[0], sn = rot[1];
                const bool act = rot[2] != 0.0;
                __syncwarp();
                if (!act) continue;  // uniform: every lane read the same flag
                ++rotated;
                if (lane < c) {  // columns p, q
                    const double skp = Sm[lane * LD + p], skq = Sm[lane * LD + q];
                    Sm[lane * LD + p] = cs * skp - sn * skq;
                    Sm[lane * LD + q] = sn * skp + cs * skq;
                }
                __syncwarp();
                if (lane < c) {  // rows p, q
                    const double spk = Sm[p * LD + lane], sqk = Sm[q * LD + lane];
                    Sm[p * LD + lane] = cs * spk - sn * sqk;
                    Sm[q * LD + lane] = sn * spk + cs * sqk;
                    const double vkp = Vm[lane * LD + p], vkq = Vm[lane * LD + q];
                    Vm[lane * LD + p] = cs * vkp - sn * vkq;
                    Vm[lane * LD + q] = sn * vkp + cs * vkq;
                }
                __syncwarp();
            }
        }
        if (!rotated) break;
    }
}

}  // namespace aar

// aar_stencil.cuh -- fused finite-difference sweep kernels (radius 1..6, FP32 or FP64).
//
// One kernel template serves three modes over a list of 32 x TY x ZC tiles:
//   SM_SWEEP : f_k = M^{-1}(b - A x_k) (Eq. 6), written to the F ring; at a Richardson step
//              also x_{k+1} = x_k + omega f_k (Eq. 2-3, B_k = omega I) into the X ring; at an
//              Anderson step instead the tile's partial sum of ||b - A x_k||^2 (the residual
//              that Sec. 2 checks only at Anderson steps).
//   SM_RESID : FP64 r = b - A x (the refinement residual of the mixed-precision form), written
//              as FP32 for the next inner solve, plus the tile's partial sum of ||r||^2.
//   SM_APPLY : y = A x in FP64.
// Each CTA marches its tile along z. A thread owns one x column and PY consecutive y rows; it
// keeps its own column's 2R+1 values in a register queue (the z neighbours), writes the centre
// plane into a double-buffered shared-memory plane with an R-wide halo (the x and y
// neighbours), and prefetches the next plane's halo and queue values into registers while the
// current plane is computed. Points outside the grid read as zero (zero Dirichlet ghosts).
#pragma once

#include "aar_engine.cuh"
#include "aar_fp64.cuh"
#include "aar_stencil_tma.cuh"

namespace aar {

template <typename T>
__device__ __forceinline__ T ldg_t(const T* p) { return __ldg(p); }

template <typename T, int R, int BY, int PY, int MODE>
__global__ void __launch_bounds__(32 * BY)
k_stencil(EngineView ev, const OpTile* __restrict__ tiles, int ntiles, int j, const double* __restrict__ xin,
          double* __restrict__ yout) {
    AAR_COUNT_LAUNCH(ev);
    constexpr int TX = 32, TY = BY * PY, SW = TX + 2 * R, SH = TY + 2 * R, Q = 2 * R + 1;
    constexpr int NT = 32 * BY;
    constexpr int NH = 2 * R * SW + 2 * TY * R;  // halo cells of one plane
    constexpr int HR = (NH + NT - 1) / NT;       // halo cells per thread
    constexpr int NCOL = PY + 2 * R;             // column values a thread reads per plane
    __shared__ T pl[2][SH * SW];
    __shared__ double red[BY];

    const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const OpTile tile = tiles[t];
        const SysDesc& S = ev.sys[tile.sys];
        const SysState& st = ev.st[tile.sys];

        const T* x = nullptr;
        const T* rhs = nullptr;
        T* fout = nullptr;
        T* xnext = nullptr;
        T* xzero = nullptr;
        float* r32 = nullptr;
        double* y = nullptr;
        bool anderson = false, zero_x = false;
        if constexpr (MODE == SM_SWEEP) {
            if (st.phase != PH_INNER || !tick_sweeps(st, S.p, j)) continue;
            const int64_t k = tick_step(st, S.p, j);
            anderson = ((k + 1) % S.p) == 0;
            zero_x = S.mixed && k == st.k_zero;
            x = ring_ptr<T>(S.X, k, S);
            fout = ring_ptr<T>(S.F, k, S);
            xnext = ring_ptr<T>(S.X, k + 1, S);
            if constexpr (sizeof(T) == 4) rhs = reinterpret_cast<const T*>(S.rhs32);
            else rhs = reinterpret_cast<const T*>(S.b64);
            if (zero_x) xzero = const_cast<T*>(x);
        } else if constexpr (MODE == SM_RESID) {
            if (st.phase != PH_RESID) continue;
            x = reinterpret_cast<const T*>(S.x64);
            rhs = reinterpret_cast<const T*>(S.b64);
            r32 = S.rhs32;
        } else {
            x = reinterpret_cast<const T*>(xin);
            y = yout;
        }
        const bool want_sum = (MODE == SM_RESID) || (MODE == SM_SWEEP && anderson);

        const int nx = S.nx, ny = S.ny, nz = S.nz;
        const int64_t pstride = (int64_t)nx * ny;
        const int x0 = tile.x0, y0 = tile.y0, z0 = tile.z0, z1 = tile.z1;
        const T cd = Coef<T>::cdiag(S);
        T co[R + 1];
#pragma unroll
        for (int kk = 1; kk <= R; ++kk) co[kk] = Coef<T>::coff(S, kk);
        const T dinv_s = Coef<T>::dinv(S);
        const double* dvec = S.dinv_vec;
        const float* dvec32 = S.dinv_vec32;
        const T omega = (T)S.omega;
        const bool blk = S.block == 2;

        // periodic grids (every axis wraps): neighbour indices are taken modulo the axis length
        const bool per = S.periodic != 0;
        auto wrapi = [](int jj, int nn) {
            const int qq = jj % nn;
            return qq < 0 ? qq + nn : qq;
        };
        // halo cells this thread loads: shared-memory index and in-plane global offset
        int h_s[HR], h_g[HR];
#pragma unroll
        for (int i = 0; i < HR; ++i) {
            const int h = tid + i * NT;
            h_s[i] = -1;
            h_g[i] = -1;
            if (h < NH) {
                int row, col;
                if (h < 2 * R * SW) {
                    const int r = h / SW;
                    col = h - r * SW;
                    row = r < R ? r : r + TY;
                } else {
                    const int h2 = h - 2 * R * SW;
                    const int side = h2 / (TY * R);
                    const int rem = h2 - side * (TY * R);
                    row = R + rem / R;
                    col = rem % R + (side ? R + TX : 0);
                }
                h_s[i] = row * SW + col;
                const int gx = x0 - R + col, gy = y0 - R + row;
                if (per) h_g[i] = wrapi(gy, ny) * nx + wrapi(gx, nx);
                else if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) h_g[i] = gy * nx + gx;
            }
        }
        // own points (computed and stored when own >= 0); ldo: the in-plane offset whose value
        // fills the point's place in the shared plane (for a tile point past the grid edge of a
        // periodic grid, the wrapped point, which the edge points read as a neighbour)
        const int gx = x0 + lane;
        int own[PY], ldo[PY];
#pragma unroll
        for (int i = 0; i < PY; ++i) {
            const int gy = y0 + ty * PY + i;
            own[i] = (gx < nx && gy < ny) ? gy * nx + gx : -1;
            ldo[i] = per ? wrapi(gy, ny) * nx + wrapi(gx, nx) : own[i];
        }

        // slab of a domain-decomposed grid (FP64): z neighbours beyond the slab come from the r
        // ghost planes exchanged with the neighbouring ranks
        const double* glo = sizeof(T) == 8 ? S.ghost_lo : nullptr;
        const double* ghi = S.ghost_hi;
        auto ldx = [&](int z, int off) -> T {
            if (zero_x || off < 0) return T(0);
            if (z < 0 || z >= nz) {  // beyond the grid (or the slab)
                if constexpr (sizeof(T) == 8) {
                    if (glo)
                        return z < 0 ? ldg_t(glo + (int64_t)(z + R) * pstride + off)
                                     : ldg_t(ghi + (int64_t)(z - nz) * pstride + off);
                }
                if (!per) return T(0);
                z = wrapi(z, nz);
            }
            return ldg_t(x + (int64_t)z * pstride + off);
        };

        // register queue: q[i][d] holds plane z - R + d of the current step z; qn / rvn / hv hold
        // the values of the next plane, loaded one step ahead
        T q[PY][Q], qn[PY], rvn[PY];
#pragma unroll
        for (int i = 0; i < PY; ++i) {
#pragma unroll
            for (int d = -R; d < R; ++d) q[i][d + R] = ldx(z0 + d, ldo[i]);
            q[i][2 * R] = T(0);
            qn[i] = ldx(z0 + R, ldo[i]);
            rvn[i] = T(0);
            if constexpr (MODE != SM_APPLY) {
                if (own[i] >= 0 && z0 < z1) rvn[i] = ldg_t(rhs + (int64_t)z0 * pstride + own[i]);
            }
        }
        T hv[HR];
#pragma unroll
        for (int i = 0; i < HR; ++i) hv[i] = ldx(z0, h_g[i]);

        T ssum = T(0);
        const T one = sizeof(T) == 8 ? (T)unit_one() : T(1);  // FP64 sums as FMAs (aar_fp64.cuh)
        __syncthreads();  // previous tile's last plane reads are done

        // one z step per iteration, not unrolled (small loop body for the instruction cache)
#pragma unroll 1
        for (int z = z0; z < z1; ++z) {
            T rv[PY];
#pragma unroll
            for (int i = 0; i < PY; ++i) {
                q[i][2 * R] = qn[i];  // plane z + R joins the queue
                rv[i] = rvn[i];
            }
            T* P = pl[(z - z0) & 1];
#pragma unroll
            for (int i = 0; i < PY; ++i) P[(R + ty * PY + i) * SW + R + lane] = q[i][R];
#pragma unroll
            for (int i = 0; i < HR; ++i)
                if (h_s[i] >= 0) P[h_s[i]] = hv[i];
            __syncthreads();
            // prefetch the next plane while this one is computed
            if (z + 1 < z1) {
#pragma unroll
                for (int i = 0; i < HR; ++i) hv[i] = ldx(z + 1, h_g[i]);
#pragma unroll
                for (int i = 0; i < PY; ++i) {
                    qn[i] = ldx(z + 1 + R, ldo[i]);
                    if constexpr (MODE != SM_APPLY)
                        rvn[i] = own[i] >= 0 ? ldg_t(rhs + (int64_t)(z + 1) * pstride + own[i]) : T(0);
                }
            }
            T col[NCOL];
#pragma unroll
            for (int r = 0; r < NCOL; ++r) col[r] = P[(ty * PY + r) * SW + R + lane];
#pragma unroll
            for (int i = 0; i < PY; ++i) {
                const T c = q[i][R];
                const T* row = P + (R + ty * PY + i) * SW + R + lane;
                T acc = cd * c;
#pragma unroll
                for (int kk = 1; kk <= R; ++kk) {
                    const T s = uadd(uadd(uadd(q[i][R - kk], q[i][R + kk], one),
                                          uadd(col[i + R - kk], col[i + R + kk], one), one),
                                     uadd(row[-kk], row[kk], one), one);
                    acc = fma(co[kk], s, acc);
                }
                if (own[i] >= 0) {
                    const int64_t gi = (int64_t)z * pstride + own[i];
                    if constexpr (MODE == SM_SWEEP) {
                        const T res = rv[i] - acc;
                        if (blk) {
                            // block Jacobi: the residual itself; k_block_apply scales and updates
                            fout[gi] = res;
                            if (anderson) ssum = fma(res, res, ssum);
                        } else {
                            T dv = dinv_s;
                            if (dvec) {
                                if constexpr (sizeof(T) == 4) dv = __ldg(dvec32 + gi);
                                else dv = __ldg(dvec + gi);
                            }
                            const T f = dv * res;
                            fout[gi] = f;
                            if (anderson) ssum = fma(res, res, ssum);
                            else xnext[gi] = fma(omega, f, c);
                        }
                        if (zero_x) xzero[gi] = T(0);
                    } else if constexpr (MODE == SM_RESID) {
                        const T r = rv[i] - acc;
                        r32[gi] = (float)r;
                        ssum = fma(r, r, ssum);
                    } else {
                        y[gi] = (double)acc;
                    }
                }
#pragma unroll
                for (int d = 0; d < 2 * R; ++d) q[i][d] = q[i][d + 1];
            }
        }
        if (want_sum) {
            const double tot = block_sum<BY>((double)ssum, red);
            if (tid == 0) ev.part_s[(MODE == SM_RESID ? S.opd0 : S.op0) + tile.local] = tot;
        }
    }
}

template <typename T, int R, int BY, int PY, int MODE>
inline cudaError_t launch_one(const OpLaunch& L, const EngineView& ev, int j, const double* xin, double* yout,
                              cudaStream_t s) {
    if (L.ntiles <= 0) return cudaSuccess;
    dim3 block(32, BY);
    k_stencil<T, R, BY, PY, MODE><<<L.grid, block, 0, s>>>(ev, L.tiles, L.ntiles, j, xin, yout);
    return cudaGetLastError();
}

template <typename T, int R, int BY, int PY, int MODE>
inline int occ_one() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stencil<T, R, BY, PY, MODE>, 32 * BY, 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

// Tile-shape variants: FP32 {0: 32x32 (8 warps, 4 rows/thread), 1: 32x8 (4 warps, 2 rows),
//                             2: TMA 32x32, 3: TMA 32x16, 4: TMA 64x16 paired FP32 (nx % 4 == 0 only),
//                             5: the paired sweep of 4 on a periodic grid (cp.async fills, radius <= 4),
//                             6, 7: 4 and 5 with block Jacobi (2 x 2 x 2 boxes) fused},
//                      FP64 {0: 32x16 (8 warps, 2 rows/thread), 1: 32x8 (4 warps, 2 rows)}.
#define AAR_STENCIL_RADIUS_IMPL(RR)                                                                          \
    cudaError_t launch_stencil_r##RR(int fp32, int mode, const OpLaunch& L, const EngineView& ev, int j,       \
                                     const double* xin, double* yout, cudaStream_t s) {                       \
        if (mode == SM_SWEEP && fp32) {                                                                        \
            if (L.variant == 2) return launch_tma<RR, 4, 3>(L, ev, j, s);                                      \
            if (L.variant == 3) return launch_tma<RR, 2, 3>(L, ev, j, s);                                      \
            if (L.variant == 4) return launch_tma2<RR, 2, 3, 2, 2, false>(L, ev, j, s);                       \
            if (L.variant == 5) return launch_tma2_per<RR>(L, ev, j, s);                                        \
            if (L.variant == 6) return launch_tma2<RR, 2, 3, 2, 2, false, true>(L, ev, j, s);                   \
            if (L.variant == 7) return launch_tma2_per<RR, true>(L, ev, j, s);                                  \
            if (L.variant == 0) return launch_one<float, RR, 8, 4, SM_SWEEP>(L, ev, j, xin, yout, s);          \
            return launch_one<float, RR, 4, 2, SM_SWEEP>(L, ev, j, xin, yout, s);                              \
        }                                                                                                      \
        if (mode == SM_SWEEP) {                                                                                \
            if (L.variant == 0) return launch_one<double, RR, 8, 2, SM_SWEEP>(L, ev, j, xin, yout, s);         \
            return launch_one<double, RR, 4, 2, SM_SWEEP>(L, ev, j, xin, yout, s);                             \
        }                                                                                                      \
        if (mode == SM_RESID) {                                                                                \
            if (L.variant == 0) return launch_one<double, RR, 8, 2, SM_RESID>(L, ev, j, xin, yout, s);         \
            return launch_one<double, RR, 4, 2, SM_RESID>(L, ev, j, xin, yout, s);                             \
        }                                                                                                      \
        if (L.variant == 0) return launch_one<double, RR, 8, 2, SM_APPLY>(L, ev, j, xin, yout, s);             \
        return launch_one<double, RR, 4, 2, SM_APPLY>(L, ev, j, xin, yout, s);                                 \
    }                                                                                                          \
    int occupancy_r##RR(int fp32, int mode, int variant) {                                                     \
        if (mode == SM_SWEEP && fp32) {                                                                        \
            if (variant == 2) return occ_tma<RR, 4, 3>();                                                      \
            if (variant == 3) return occ_tma<RR, 2, 3>();                                                      \
            if (variant == 4) return occ_tma2<RR, 2, 3, 2, 2, false>();                                       \
            if (variant == 5) return occ_tma2_per<RR>();                                                        \
            if (variant == 6) return occ_tma2<RR, 2, 3, 2, 2, false, true>();                                   \
            if (variant == 7) return occ_tma2_per<RR, true>();                                                  \
            return variant == 0 ? occ_one<float, RR, 8, 4, SM_SWEEP>() : occ_one<float, RR, 4, 2, SM_SWEEP>(); \
        }                                                                                                      \
        if (mode == SM_SWEEP)                                                                                  \
            return variant == 0 ? occ_one<double, RR, 8, 2, SM_SWEEP>() : occ_one<double, RR, 4, 2, SM_SWEEP>(); \
        if (mode == SM_RESID)                                                                                  \
            return variant == 0 ? occ_one<double, RR, 8, 2, SM_RESID>() : occ_one<double, RR, 4, 2, SM_RESID>(); \
        return variant == 0 ? occ_one<double, RR, 8, 2, SM_APPLY>() : occ_one<double, RR, 4, 2, SM_APPLY>();   \
    }

}  // namespace aar

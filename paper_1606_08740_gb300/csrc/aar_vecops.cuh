// aar_vecops.cuh -- vector access helpers and the plain-load Anderson update shared by the
// register-fed and bulk-fed vector passes.
#pragma once

#include "aar_engine.cuh"
#include "aar_fp64.cuh"

namespace aar {

template <typename T> struct Vec2;
template <> struct Vec2<float> {
    using V = float4;
    static constexpr int W = 4;
    static __device__ __forceinline__ void load(const float* p, float* o) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ void store(float* p, const float* o) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <> struct Vec2<double> {
    using V = double2;
    static constexpr int W = 2;
    static __device__ __forceinline__ void load(const double* p, double* o) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = v.x; o[1] = v.y;
    }
    static __device__ __forceinline__ void store(double* p, const double* o) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    }
};

template <typename T> struct GramVec;  // two-element loads (float2 / double2) of the literal update
template <> struct GramVec<float> {
    static constexpr int W = 2;
    static __device__ __forceinline__ void load(const float* p, float* o) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        o[0] = v.x; o[1] = v.y;
    }
};
template <> struct GramVec<double> {
    static constexpr int W = 2;
    static __device__ __forceinline__ void load(const double* p, double* o) { Vec2<double>::load(p, o); }
};

// Literal Anderson update (Eq. 3) and the mixed form's x64 += d for one vec tile, from plain loads.
template <typename T, int CMAX>
__device__ void update_plain_tile(const SysDesc& S, const SysState& st, const VecTile& tile) {
    constexpr int W = 2;  // 2 elements per access (float2 / double2), few registers
    const int tid = threadIdx.x;
    if (st.upd == UPD_ANDERSON) {
        const int64_t k = st.upd_k;
        const int c = st.upd_c;
        T gam[CMAX];
#pragma unroll
        for (int a = 0; a < CMAX; ++a) gam[a] = (a < c) ? (T)st.gamma[a] : T(0);
        const T beta = (T)S.beta;
        const T* xc[CMAX + 1];
        const T* fc[CMAX + 1];
#pragma unroll
        for (int a = 0; a <= CMAX; ++a) {
            const int64_t kk = k - c + (a <= c ? a : c);
            xc[a] = ring_ptr<T>(S.X, kk, S);
            fc[a] = ring_ptr<T>(S.F, kk, S);
        }
        // window column (a: iterate k-c+1+a) whose upper end is the split iterate, if any
        const int as = (sizeof(T) == 4 && st.split_k >= 0) ? (int)(st.split_k - (k - c + 1)) : -1;
        const T* xo = reinterpret_cast<const T*>(S.xold);
        const T* fo = reinterpret_cast<const T*>(S.fold);
        T* xn = ring_ptr<T>(S.X, k + 1, S);
        const T* xk = ring_ptr<T>(S.X, k, S);
        const T* fk = ring_ptr<T>(S.F, k, S);
        const T one = sizeof(T) == 8 ? (T)unit_one() : T(1);  // FP64 differences as FMAs (aar_fp64.cuh)
        for (int64_t i = tile.start + (int64_t)tid * W; i < tile.end; i += 256 * W) {
            T xv[W], fv[W], corr[W], out[W];
            GramVec<T>::load(xk + i, xv);
            GramVec<T>::load(fk + i, fv);
#pragma unroll
            for (int w = 0; w < W; ++w) corr[w] = T(0);
            T xprev[W], fprev[W];
            GramVec<T>::load(xc[0] + i, xprev);
            GramVec<T>::load(fc[0] + i, fprev);
#pragma unroll
            for (int a = 0; a < CMAX; ++a) {
                if (a < c) {
                    T xa[W], fa[W], xu[W], fu[W];
                    GramVec<T>::load(xc[a + 1] + i, xa);
                    GramVec<T>::load(fc[a + 1] + i, fa);
                    if (a == as) {
                        GramVec<T>::load(xo + i, xu);
                        GramVec<T>::load(fo + i, fu);
                    } else {
#pragma unroll
                        for (int w = 0; w < W; ++w) {
                            xu[w] = xa[w];
                            fu[w] = fa[w];
                        }
                    }
#pragma unroll
                    for (int w = 0; w < W; ++w) {
                        const T dx = usub(xu[w], xprev[w], one);
                        const T df = usub(fu[w], fprev[w], one);
                        corr[w] = fma(gam[a], fma(beta, df, dx), corr[w]);
                        xprev[w] = xa[w];
                        fprev[w] = fa[w];
                    }
                }
            }
#pragma unroll
            for (int w = 0; w < W; ++w) out[w] = usub(fma(beta, fv[w], xv[w]), corr[w], one);
            if constexpr (sizeof(T) == 4) *reinterpret_cast<float2*>(xn + i) = make_float2(out[0], out[1]);
            else Vec2<T>::store(xn + i, out);
        }
    } else if (st.upd == UPD_ADD_D) {
        // mixed precision: x64 += d, d = the FP32 inner iterate x_{upd_k}. When the next inner
        // solve keeps the history, x_{upd_k} and f_{upd_k} are also saved to xold / fold: the
        // restart overwrites them, and the difference column that straddles it still needs them.
        const float* d = ring_ptr<float>(S.X, st.upd_k, S);
        const float* fk = ring_ptr<float>(S.F, st.upd_k, S);
        const bool save = st.keep != 0;
        const int64_t end = tile.end < S.n ? tile.end : S.n;
        for (int64_t i = tile.start + (int64_t)tid * 4; i < end; i += 1024) {
            if (i + 4 <= end) {
                const float4 dv = __ldg(reinterpret_cast<const float4*>(d + i));
                double2* xp = reinterpret_cast<double2*>(S.x64 + i);
                double2 lo = xp[0], hi = xp[1];
                lo.x += (double)dv.x;
                lo.y += (double)dv.y;
                hi.x += (double)dv.z;
                hi.y += (double)dv.w;
                xp[0] = lo;
                xp[1] = hi;
                if (save) {
                    *reinterpret_cast<float4*>(S.xold + i) = dv;
                    *reinterpret_cast<float4*>(S.fold + i) = __ldg(reinterpret_cast<const float4*>(fk + i));
                }
            } else {
                for (int64_t q = i; q < end; ++q) {
                    S.x64[q] += (double)d[q];
                    if (save) {
                        S.xold[q] = d[q];
                        S.fold[q] = fk[q];
                    }
                }
            }
        }
    }
}

}  // namespace aar

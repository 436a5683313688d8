// aar_block.cu -- block Jacobi with 2 x 2 x 2 boxes (the block Jacobi of Sec. 3.2/3.3, each
// block solved exactly) for the stencil operators.
//
// M is the block-diagonal part of A for the tiling of the grid by 2 x 2 x 2 boxes. Inside a box a
// point's only neighbours are its three partners at distance 1 (one along each axis), so every
// block is the same 8 x 8 matrix B = d I + c1 Q3, d the centre coefficient and c1 the distance-1
// weight, Q3 the adjacency of the cube graph. The Walsh-Hadamard vectors h_s(a) = (-1)^{|s & a|}
// (a = dx + 2 dy + 4 dz) diagonalise it: B h_s = (d + c1 (3 - 2 |s|)) h_s. Hence
//   M^{-1} r = H diag(1 / (8 lambda_s)) H r,
// three butterfly stages, one scaling by mu_|s| = 1 / (8 lambda_|s|), three butterfly stages.
//
// The sweep of a block-Jacobi system writes the residual b - A x_k into the F slot; this kernel
// replaces it by f_k = M^{-1}(b - A x_k) (Eq. 6 with the block M) and, at a Richardson step,
// writes x_{k+1} = x_k + omega f_k (Eq. 2, 3). One thread per box: two float2 / double2 loads per
// plane pair and row (the box's two x points are adjacent), coalesced across the warp.
#include <cuda_runtime.h>

#include "aar_engine.cuh"

namespace aar {
namespace {

template <typename T>
struct BVec;
template <>
struct BVec<float> {
    using type = float2;
};
template <>
struct BVec<double> {
    using type = double2;
};

template <typename T>
__device__ __forceinline__ T bl_mu(const SysDesc& S, int t) {
    if constexpr (sizeof(T) == 4) return S.bl_mu_f[t];
    else return S.bl_mu[t];
}

// in-place Walsh-Hadamard transform of v[a], a = dx + 2 dy + 4 dz (unnormalised)
template <typename T>
__device__ __forceinline__ void fwht8(T (&v)[8]) {
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1) {
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            if (a & bit) continue;
            const T u = v[a], w = v[a | bit];
            v[a] = u + w;
            v[a | bit] = u - w;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_block_apply(EngineView ev, int j) {
    using V = typename BVec<T>::type;
    AAR_COUNT_LAUNCH(ev);
    for (int sidx = 0; sidx < ev.nsys; ++sidx) {
        const SysDesc& S = ev.sys[sidx];
        const SysState& st = ev.st[sidx];
        if (S.block != 2 || st.phase != PH_INNER) continue;  // 3: boxes applied inside the sweep
        if (!tick_sweeps(st, S.p, j)) continue;
        const int64_t k = tick_step(st, S.p, j);
        const bool anderson = ((k + 1) % S.p) == 0;
        T* f = ring_ptr<T>(S.F, k, S);
        const T* xk = ring_ptr<T>(S.X, k, S);
        T* xn = ring_ptr<T>(S.X, k + 1, S);
        const int nx = S.nx, bx = S.nx / 2, by = S.ny / 2, bz = S.nz / 2;
        const int64_t ps = (int64_t)S.nx * S.ny;
        const int64_t nbox = (int64_t)bx * by * bz;
        T mu[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) mu[t] = bl_mu<T>(S, t);
        const T omega = (T)S.omega;
        for (int64_t bi = (int64_t)blockIdx.x * 256 + threadIdx.x; bi < nbox; bi += (int64_t)gridDim.x * 256) {
            const int X = (int)(bi % bx);
            const int64_t rest = bi / bx;
            const int Y = (int)(rest % by), Z = (int)(rest / by);
            const int64_t base = (int64_t)(2 * Z) * ps + (int64_t)(2 * Y) * nx + 2 * X;
            T v[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // q = dy + 2 dz
                const int64_t o = base + (q >> 1) * ps + (q & 1) * nx;
                const V w = *reinterpret_cast<const V*>(f + o);
                v[2 * q] = w.x;
                v[2 * q + 1] = w.y;
            }
            fwht8(v);
#pragma unroll
            for (int a = 0; a < 8; ++a) v[a] *= mu[__popc(a)];
            fwht8(v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t o = base + (q >> 1) * ps + (q & 1) * nx;
                V w;
                w.x = v[2 * q];
                w.y = v[2 * q + 1];
                *reinterpret_cast<V*>(f + o) = w;
                if (!anderson) {
                    const V xv = *reinterpret_cast<const V*>(xk + o);
                    V nv;
                    nv.x = fma(omega, w.x, xv.x);
                    nv.y = fma(omega, w.y, xv.y);
                    *reinterpret_cast<V*>(xn + o) = nv;
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_block_apply(int fp32, const EngineView& ev, int j, int grid, cudaStream_t s) {
    if (fp32) k_block_apply<float><<<grid, 256, 0, s>>>(ev, j);
    else k_block_apply<double><<<grid, 256, 0, s>>>(ev, j);
    return cudaGetLastError();
}

}  // namespace aar

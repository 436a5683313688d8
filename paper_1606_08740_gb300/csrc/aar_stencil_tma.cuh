// aar_stencil_tma.cuh -- TMA-fed FP32 Richardson/Anderson sweep (Eq. 2, 3, 6) for grids whose x
// extent is a multiple of 4 (16-byte rows, the tensor-map stride rule).
//
// Each CTA marches a 32 x TY x ZC tile along z. One elected thread streams whole x-y planes of
// x_k (tile plus an R-wide halo, the x start rounded down to a 16-byte boundary) into a ring of
// NS shared-memory stages with cp.async.bulk.tensor (3-D tiled TMA); out-of-grid cells arrive
// as zeros, which are exactly the Dirichlet ghosts. Each stage has an mbarrier that the copy
// completes (complete_tx); consumers wait on it with a bounded try_wait. A thread keeps its own
// column's 2R+1 values in a register queue (the z neighbours), fed from the stage of plane z+R,
// and reads x/y neighbours from the stage of plane z. The loads in flight live in shared memory,
// not registers, so D planes of prefetch cost no registers.
#pragma once

#include <cuda.h>

#include <type_traits>

#include "aar_engine.cuh"
#include "aar_mbar.cuh"

namespace aar {

template <int R>
struct TmaGeom {
    static constexpr int RA = (R + 3) / 4 * 4;  // halo width rounded up to 16 bytes
    static constexpr int BX = 32 + 2 * RA;      // box x extent
};

template <int R, int PY>
__host__ __device__ constexpr int tma_stage_floats() { return TmaGeom<R>::BX * (8 * PY + 2 * R); }

template <int R, int PY, int D>
__host__ __device__ constexpr int tma_stages() { return R + 1 + D; }

// stage bytes are rounded up to 128 (the TMA shared-memory destination alignment); 1024 bytes of
// slack let the kernel align the stage base itself
template <int R, int PY>
__host__ __device__ constexpr int tma_stage_stride() { return (tma_stage_floats<R, PY>() * 4 + 127) / 128 * 128; }

template <int R, int PY, int D>
__host__ __device__ constexpr size_t tma_smem_bytes() {
    return (size_t)tma_stages<R, PY, D>() * tma_stage_stride<R, PY>() + 1024;
}

template <int R, int PY, int D>
__global__ void __launch_bounds__(256, 2)
k_sweep_tma(EngineView ev, const OpTile* __restrict__ tiles, int ntiles, int j, const CUtensorMap* __restrict__ maps) {
    AAR_COUNT_LAUNCH(ev);
    constexpr int BY = 8, TY = BY * PY, RA = TmaGeom<R>::RA, BX = TmaGeom<R>::BX, Q = 2 * R + 1;
    static_assert(TY <= 256 && BX <= 256, "TMA box extents are at most 256");
    constexpr int NS = tma_stages<R, PY, D>();
    constexpr uint32_t BYTES = tma_stage_floats<R, PY>() * 4;  // one box
    constexpr int STAGE = tma_stage_stride<R, PY>() / 4;      // stage stride in floats
    constexpr int NCOL = PY + 2 * R;
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[NS];
    __shared__ double red[BY];
    // stage ring base aligned to 1024 bytes whatever the dynamic region's placement
    float* sm = reinterpret_cast<float*>(smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u));
    bool abort = false;

    const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    uint32_t seq = 0;  // planes issued by this CTA before the current tile
    uint32_t hi = 0;   // thread 0: planes issued so far (index of the last one + 1)

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const OpTile tile = tiles[t];
        const SysDesc& S = ev.sys[tile.sys];
        const SysState& st = ev.st[tile.sys];
        if (st.phase != PH_INNER || !tick_sweeps(st, S.p, j)) continue;
        const int64_t k = tick_step(st, S.p, j);
        const bool anderson = ((k + 1) % S.p) == 0;
        const bool zero_x = S.mixed && k == st.k_zero;
        float* xk = ring_ptr<float>(S.X, k, S);
        float* fout = ring_ptr<float>(S.F, k, S);
        float* xnext = ring_ptr<float>(S.X, k + 1, S);
        const float* rhs = S.rhs32;
        const CUtensorMap* map = maps + S.map0 + ring_slot(k, S.nslots);

        const int nx = S.nx, ny = S.ny;
        const int64_t pstride = (int64_t)nx * ny;
        const int x0 = tile.x0, y0 = tile.y0, z0 = tile.z0, z1 = tile.z1;
        const float cd = S.cdiag_f;
        float co[R + 1];
#pragma unroll
        for (int kk = 1; kk <= R; ++kk) co[kk] = S.coff_f[kk];
        const float dinv_s = S.dinv_f;
        const float* dvec32 = S.dinv_vec32;
        const float omega = (float)S.omega;
        const int gx = x0 + lane;
        int own[PY];
#pragma unroll
        for (int i = 0; i < PY; ++i) {
            const int gy = y0 + ty * PY + i;
            own[i] = (gx < nx && gy < ny) ? gy * nx + gx : -1;
        }
        float ssum = 0.f;

        if (zero_x) {
            // x_k = 0 (first step of an inner solve): f_k = M^{-1} rhs, x_{k+1} = omega f_k, and
            // slot k is cleared
            for (int z = z0; z < z1; ++z) {
#pragma unroll
                for (int i = 0; i < PY; ++i) {
                    if (own[i] < 0) continue;
                    const int64_t gi = (int64_t)z * pstride + own[i];
                    const float res = __ldg(rhs + gi);
                    const float f = (dvec32 ? __ldg(dvec32 + gi) : dinv_s) * res;
                    fout[gi] = f;
                    xk[gi] = 0.f;
                    if (anderson) ssum = fmaf(res, res, ssum);
                    else xnext[gi] = omega * f;
                }
            }
        } else {
            const int NP = (z1 - z0) + 2 * R;  // planes z0-R .. z1+R-1
            auto issue = [&](int i) {
                const uint32_t g = seq + (uint32_t)i;
                const int s = (int)(g % NS);
                const uint32_t bar = smem_u32(&bars[s]);
                mbar_expect_tx(bar, BYTES);
                tma_load_3d(smem_u32(sm + s * STAGE), map, x0 - RA, y0 - R, z0 - R + i, bar);
                hi = g + 1;
            };
            auto wait = [&](int i) {
                const uint32_t g = seq + (uint32_t)i;
                mbar_wait(smem_u32(&bars[g % NS]), (g / NS) & 1u, ev.err, abort, i);
            };
            auto stage = [&](int i) -> const float* { return sm + ((seq + (uint32_t)i) % NS) * STAGE; };

            if (tid == 0 && !abort)
                for (int i = 0; i < NS && i < NP; ++i) issue(i);

            // register queue: q[p][d] holds plane z - R + d of the current step z.
            // Planes 0..R-1 only feed the queue: each one's stage is handed back (plane i + NS) as soon
            // as every thread has read it, so the prologue never needs more than NS stages at once.
            float q[PY][Q];
#pragma unroll
            for (int i = 0; i < 2 * R; ++i) {
                wait(i);
                const float* P = stage(i);
#pragma unroll
                for (int p = 0; p < PY; ++p) q[p][i] = P[(R + ty * PY + p) * BX + RA + lane];
                if (i < R) {
                    __syncthreads();
                    if (tid == 0 && i + NS < NP && !abort) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue(i + NS);
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < PY; ++p) q[p][2 * R] = 0.f;
            float rvn[PY];
#pragma unroll
            for (int p = 0; p < PY; ++p) rvn[p] = own[p] >= 0 ? __ldg(rhs + (int64_t)z0 * pstride + own[p]) : 0.f;

            // one z step per iteration, not unrolled: the queue shifts by one slot per step, which
            // keeps the loop body small enough for the instruction cache
#pragma unroll 1
            for (int z = z0; z < z1; ++z) {
                const int iz = z - z0 + R;  // plane z (x/y neighbours)
                float rv[PY];
#pragma unroll
                for (int p = 0; p < PY; ++p) rv[p] = rvn[p];
                if (z + 1 < z1) {
#pragma unroll
                    for (int p = 0; p < PY; ++p)
                        rvn[p] = own[p] >= 0 ? __ldg(rhs + (int64_t)(z + 1) * pstride + own[p]) : 0.f;
                }
                wait(iz + R);  // plane z + R joins the queue
                {
                    const float* F = stage(iz + R);
#pragma unroll
                    for (int p = 0; p < PY; ++p) q[p][2 * R] = F[(R + ty * PY + p) * BX + RA + lane];
                }
                const float* P = stage(iz);
                float col[NCOL];
#pragma unroll
                for (int r = 0; r < NCOL; ++r) col[r] = P[(ty * PY + r) * BX + RA + lane];
#pragma unroll
                for (int p = 0; p < PY; ++p) {
                    const float c = q[p][R];
                    const float* row = P + (R + ty * PY + p) * BX + RA + lane;
                    float acc = cd * c;
#pragma unroll
                    for (int kk = 1; kk <= R; ++kk) {
                        const float s = ((q[p][R - kk] + q[p][R + kk]) + (col[p + R - kk] + col[p + R + kk])) +
                                        (row[-kk] + row[kk]);
                        acc = fmaf(co[kk], s, acc);
                    }
                    if (own[p] >= 0) {
                        const int64_t gi = (int64_t)z * pstride + own[p];
                        const float res = rv[p] - acc;
                        const float f = (dvec32 ? __ldg(dvec32 + gi) : dinv_s) * res;
                        fout[gi] = f;
                        if (anderson) ssum = fmaf(res, res, ssum);
                        else xnext[gi] = fmaf(omega, f, c);
                    }
#pragma unroll
                    for (int d = 0; d < 2 * R; ++d) q[p][d] = q[p][d + 1];
                }
                __syncthreads();  // plane z is consumed: its stage takes plane iz + NS
                if (tid == 0 && iz + NS < NP && !abort) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue(iz + NS);
                }
            }
            seq += (uint32_t)NP;
            // a wait that gave up anywhere in the CTA ends the kernel here (the control kernel then
            // stops the solve), once the copies still in flight have landed
            if (__syncthreads_or(abort)) {
                if (tid == 0) mbar_drain(bars, NS, seq - (uint32_t)NP, hi);
                return;
            }
        }
        if (anderson) {
            // warp sums in FP32, the 8 warp sums in FP64 in warp order
            float v = ssum;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[ty] = (double)v;
            __syncthreads();
            if (tid == 0) {
                double tot = 0.0;
                for (int w = 0; w < BY; ++w) tot += red[w];
                ev.part_s[S.op0 + tile.local] = tot;
            }
        }
        __syncthreads();
    }
}

template <int R, int PY, int D>
inline cudaError_t launch_tma(const OpLaunch& L, const EngineView& ev, int j, cudaStream_t s) {
    if (L.ntiles <= 0) return cudaSuccess;
    constexpr size_t bytes = tma_smem_bytes<R, PY, D>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep_tma<R, PY, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_sweep_tma<R, PY, D><<<L.grid, dim3(32, 8), bytes, s>>>(ev, L.tiles, L.ntiles, j,
                                                             reinterpret_cast<const CUtensorMap*>(L.maps));
    return cudaGetLastError();
}

template <int R, int PY, int D>
inline int occ_tma() {
    constexpr size_t bytes = tma_smem_bytes<R, PY, D>();
    if (cudaFuncSetAttribute(k_sweep_tma<R, PY, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_tma<R, PY, D>, 256, bytes) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

// ---------------------------------------------------------------------------------------------
// Two x points per thread: 64 x TY x ZC tiles, every stencil sum formed on float2 pairs with the
// paired FP32 instructions (__fadd2_rn / __ffma2_rn / __fmul2_rn), shared-memory reads and global
// stores 8 bytes wide. Component for component the arithmetic is the scalar kernels' (same
// operands, same order, one rounding per add and per fused multiply-add). The z queue holds 2R+U
// planes and is shifted once every U steps.
template <int R>
struct Tma2Geom {
    static constexpr int RA = (R + 3) / 4 * 4;
    static constexpr int BX = 64 + 2 * RA;
    static constexpr int RE = (R + 1) / 2 * 2;  // x reach rounded up to a float2 boundary
};

template <int R, int PY>
__host__ __device__ constexpr int tma2_stage_stride() {
    return (Tma2Geom<R>::BX * (8 * PY + 2 * R) * 4 + 127) / 128 * 128;
}

// Right-hand-side ring of the TMA-fed paired sweep: NB2 stages of one 64 x TY plane box of b each
// (no halo), filled by TMA like the x planes, so that b reaches the threads through shared memory
// instead of per-thread global loads.
constexpr int NB2 = 4;
template <int PY>
__host__ __device__ constexpr int tma2_bstage_bytes() { return 64 * 8 * PY * 4; }

template <int R, int PY, int D, bool PER = false>
__host__ __device__ constexpr size_t tma2_smem_bytes() {
    // + 128 bytes of slack for aligning the ring base to the TMA destination alignment
    return (size_t)(R + 1 + D) * tma2_stage_stride<R, PY>() + (PER ? 0 : NB2 * tma2_bstage_bytes<PY>()) + 128;
}

// Block Jacobi with 2 x 2 x 2 boxes on a thread's own box: r[q] holds the residual pair (x, x + 1)
// of row dy and plane dz, q = dy + 2 dz; on return r[q] = M^{-1} r in the same places. M^{-1} =
// H diag(mu_|s|) H with H the 8-point Walsh-Hadamard transform (butterflies over x inside a pair,
// over y and z between pairs) and mu_t = 1 / (8 (cdiag + coff[1] (3 - 2t))).
__device__ __forceinline__ void block2_apply(float2 (&r)[4], const float (&mu)[4]) {
    const float2 mone = make_float2(-1.f, -1.f);
    auto fwht = [&](float2 (&v)[4]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = make_float2(v[q].x + v[q].y, v[q].x - v[q].y);
        const float2 b0 = __fadd2_rn(v[0], v[1]), b1 = __ffma2_rn(mone, v[1], v[0]);
        const float2 b2 = __fadd2_rn(v[2], v[3]), b3 = __ffma2_rn(mone, v[3], v[2]);
        v[0] = __fadd2_rn(b0, b2);
        v[2] = __ffma2_rn(mone, b2, b0);
        v[1] = __fadd2_rn(b1, b3);
        v[3] = __ffma2_rn(mone, b3, b1);
    };
    fwht(r);
    // r[q] now holds the Walsh index (sx, sy, sz) = (lane of the pair, q & 1, q >> 1)
    r[0] = __fmul2_rn(r[0], make_float2(mu[0], mu[1]));
    r[1] = __fmul2_rn(r[1], make_float2(mu[1], mu[2]));
    r[2] = __fmul2_rn(r[2], make_float2(mu[1], mu[2]));
    r[3] = __fmul2_rn(r[3], make_float2(mu[2], mu[3]));
    fwht(r);
}

// PER: periodic grid. The TMA box reads zero outside the grid and cannot wrap, so each plane stage
// is filled with 4-byte cp.async copies from wrapped indices by all threads instead; a thread waits
// for its copies before the CTA barrier that precedes a plane's first read (planes issued at one
// barrier are read after the next one).
// BLK: block Jacobi with 2 x 2 x 2 boxes fused into the sweep (PY = 2; pieces start and end on even
// planes): a thread owns the box of its two x points and two rows over every pair of planes, keeps
// the first plane's residuals in registers and, after the second, writes f = M^{-1} res and the
// Richardson update for both planes.
template <int R, int PY, int D, int U, int RB, bool PER, bool BLK>
__global__ void __launch_bounds__(256, 2)
k_sweep_tma2(EngineView ev, const OpTile* __restrict__ tiles, int ntiles, int j, const CUtensorMap* __restrict__ maps) {
    AAR_COUNT_LAUNCH(ev);
    constexpr int BY = 8, TY = BY * PY, RA = Tma2Geom<R>::RA, BX = Tma2Geom<R>::BX, RE = Tma2Geom<R>::RE;
    constexpr int NS = R + 1 + D;
    constexpr uint32_t BYTES = BX * (TY + 2 * R) * 4;
    constexpr int STAGE = tma2_stage_stride<R, PY>() / 4;
    constexpr int NCOL = PY + 2 * R;
    constexpr int QL = 2 * R + U;
    constexpr int NW = RE + 1;  // float2 words of an x row segment
    static_assert(TY + 2 * R <= 256 && BX <= 256, "TMA box extents are at most 256");
    constexpr int B = RB;  // planes between CTA barriers (stage refills in groups of B)
    constexpr int SH = TY + 2 * R;
    constexpr int NC = (BX * SH + 255) / 256;  // PER: plane cells copied by each thread
    static_assert(U % B == 0 && D >= B - 1, "stage refill groups");
    static_assert(!BLK || (PY == 2 && U % 2 == 0), "block Jacobi pairs rows and planes");
    constexpr uint32_t BBYTES = tma2_bstage_bytes<PY>();  // one right-hand-side box (64 x TY floats)
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[NS];
    __shared__ __align__(8) uint64_t bbars[NB2];
    __shared__ double red[BY];
    float* sm = reinterpret_cast<float*>(smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u));
    float* bsm = sm + NS * STAGE;  // right-hand-side ring (TMA-fed variants)
    bool abort = false;

    const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&bars[s]), 1);
        for (int s = 0; s < NB2; ++s) mbar_init(smem_u32(&bbars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    uint32_t seq = 0;   // planes issued by this CTA before the current piece
    uint32_t hi = 0;    // thread 0 (TMA-fed variants): planes issued so far (last index + 1)
    uint32_t bseq = 0;  // right-hand-side planes issued before the current piece
    uint32_t bhi = 0;   // thread 0: right-hand-side planes issued so far

    // A tile is a segment [z0, z1) of the system's linear (column, plane) index u = col * nz + z,
    // columns being the 64 x TY boxes of the x-y plane in row-major order. Segments of one system
    // are of equal length, so every CTA of a single-system launch does the same work; a segment
    // runs through one or two columns (pieces), each a z-march with its own plane pipeline.
    // The z-march is specialised on whether the step is an Anderson step, whether M^{-1} is a
    // vector, and whether the column touches the grid edge, so the per-point work carries no
    // branches; offsets within a vector are 32-bit (n < 2^31 for this variant).
    using BT = std::true_type;
    using BF = std::false_type;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const OpTile tile = tiles[t];
        const SysDesc& S = ev.sys[tile.sys];
        const SysState& st = ev.st[tile.sys];
        if (st.phase != PH_INNER || !tick_sweeps(st, S.p, j)) continue;
        const int64_t k = tick_step(st, S.p, j);
        const bool anderson = ((k + 1) % S.p) == 0;
        const bool zero_x = S.mixed && k == st.k_zero;
        float* xk = ring_ptr<float>(S.X, k, S);
        float* fout = ring_ptr<float>(S.F, k, S);
        float* xnext = ring_ptr<float>(S.X, k + 1, S);
        const float* rhs = S.rhs32;
        const CUtensorMap* map = PER ? nullptr : maps + S.map0 + ring_slot(k, S.nslots);
        const CUtensorMap* bmap = PER ? nullptr : maps + S.map0 + S.nslots;  // rhs32

        const int nx = S.nx, ny = S.ny, nz = S.nz;
        const int txn = (nx + 63) / 64;
        const uint32_t ps = (uint32_t)nx * (uint32_t)ny;
        const float2 cd = make_float2(S.cdiag_f, S.cdiag_f);
        float2 co[R + 1];
#pragma unroll
        for (int kk = 1; kk <= R; ++kk) co[kk] = make_float2(S.coff_f[kk], S.coff_f[kk]);
        const float2 dinv_s = make_float2(S.dinv_f, S.dinv_f);
        const float* dvec32 = S.dinv_vec32;
        float bmu[4];  // block Jacobi scalings (BLK only)
#pragma unroll
        for (int t = 0; t < 4; ++t) bmu[t] = BLK ? S.bl_mu_f[t] : 0.f;
        const float2 omega = make_float2((float)S.omega, (float)S.omega);
        const float2 mone = make_float2(-1.f, -1.f);
        float2 ssum = make_float2(0.f, 0.f);
        auto ld2 = [](const float* p) { return *reinterpret_cast<const float2*>(p); };
        auto ldg2 = [](const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); };
        auto st2 = [](float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; };

        for (int u = tile.z0; u < tile.z1;) {
            const int colx = u / nz;
            const int z0 = u - colx * nz;
            const int z1 = min(nz, z0 + (tile.z1 - u));
            u += z1 - z0;
            const int x0 = (colx % txn) * 64, y0 = (colx / txn) * TY;
            const int gx = x0 + 2 * lane;  // this thread's points: gx, gx + 1 (nx is a multiple of 4)
            const bool edge = x0 + 64 > nx || y0 + TY > ny;
            int own[PY];
#pragma unroll
            for (int i = 0; i < PY; ++i) {
                const int gy = y0 + ty * PY + i;
                own[i] = (gx < nx && gy < ny) ? gy * nx + gx : -1;
            }

            if (BLK && zero_x) {
                // x_k = 0 with block Jacobi: the residual is rhs; boxes of two planes at a time
                for (int z = z0; z + 1 < z1; z += 2) {
                    if (own[0] < 0) continue;  // both rows of a box lie inside or outside the grid
                    float2 rr[4];
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq)
                        rr[qq] = ldg2(rhs + (uint32_t)(z + (qq >> 1)) * ps + (uint32_t)own[qq & 1]);
                    if (anderson) {
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) ssum = __ffma2_rn(rr[qq], rr[qq], ssum);
                    }
                    block2_apply(rr, bmu);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        const uint32_t gi = (uint32_t)(z + (qq >> 1)) * ps + (uint32_t)own[qq & 1];
                        st2(fout + gi, rr[qq]);
                        st2(xk + gi, make_float2(0.f, 0.f));
                        if (!anderson) st2(xnext + gi, __fmul2_rn(omega, rr[qq]));
                    }
                }
                continue;
            }
            if (zero_x) {
                // x_k = 0 (first step of an inner solve): f_k = M^{-1} rhs, x_{k+1} = omega f_k, and
                // slot k is cleared
                for (int z = z0; z < z1; ++z) {
#pragma unroll
                    for (int i = 0; i < PY; ++i) {
                        if (own[i] < 0) continue;
                        const uint32_t gi = (uint32_t)z * ps + (uint32_t)own[i];
                        const float2 res = ldg2(rhs + gi);
                        const float2 f = __fmul2_rn(dvec32 ? ldg2(dvec32 + gi) : dinv_s, res);
                        st2(fout + gi, f);
                        st2(xk + gi, make_float2(0.f, 0.f));
                        if (anderson) ssum = __ffma2_rn(res, res, ssum);
                        else st2(xnext + gi, __fmul2_rn(omega, f));
                    }
                }
                continue;
            }
            // Planes 0 .. NP-1 of the piece (plane i is z0 - R + i), NS stages deep; the stage of
            // plane i is refilled with plane i + NS once every thread has passed the step that
            // last reads plane i (a CTA barrier per step).
            const int NP = (z1 - z0) + 2 * R;
            // PER: wrapped in-plane offsets of this thread's cells of the stage box (cell = row BX + col)
            int cgo[PER ? NC : 1];
            if constexpr (PER) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int cell = tid + 256 * c, row = cell / BX, col = cell - row * BX;
                    cgo[c] = wrap_index(y0 - R + row, ny) * nx + wrap_index(x0 - RA + col, nx);
                }
            }
            auto issue = [&](int i) {
                const uint32_t g = seq + (uint32_t)i;
                const int s = (int)(g % NS);
                if constexpr (PER) {
                    float* st = sm + s * STAGE;
                    const float* src = xk + (size_t)wrap_index(z0 - R + i, S.nz) * ps;
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        if (tid + 256 * c < BX * SH) cp_async4(smem_u32(st + tid + 256 * c), src + cgo[c]);
                    cp_async_commit();
                } else {
                    const uint32_t bar = smem_u32(&bars[s]);
                    mbar_expect_tx(bar, BYTES);
                    tma_load_3d(smem_u32(sm + s * STAGE), map, x0 - RA, y0 - R, z0 - R + i, bar);
                    hi = g + 1;
                }
            };
            auto wait = [&](int i) {
                if constexpr (!PER) {
                    const uint32_t g = seq + (uint32_t)i;
                    const uint32_t bar = smem_u32(&bars[g % NS]);
                    if (!mbar_try_wait(bar, (g / NS) & 1u)) mbar_wait(bar, (g / NS) & 1u, ev.err, abort, i);
                }
            };
            auto stage = [&](int i) -> const float* { return sm + ((seq + (uint32_t)i) % NS) * STAGE; };
            const int own_off = RA + 2 * lane;
            // right-hand side of step sn (plane z0 + sn) in ring stage (bseq + sn) mod NB2
            const int len = z1 - z0;
            auto issue_b = [&](int sn) {
                const uint32_t g = bseq + (uint32_t)sn;
                const uint32_t bar = smem_u32(&bbars[g % NB2]);
                mbar_expect_tx(bar, BBYTES);
                tma_load_3d(smem_u32(bsm + (g % NB2) * (BBYTES / 4)), bmap, x0, y0, z0 + sn, bar);
                bhi = g + 1;
            };
            auto wait_b = [&](int sn) {
                const uint32_t g = bseq + (uint32_t)sn;
                const uint32_t bar = smem_u32(&bbars[g % NB2]);
                if (!mbar_try_wait(bar, (g / NB2) & 1u)) mbar_wait(bar, (g / NB2) & 1u, ev.err, abort, 1 << 20);
            };
            auto bstage = [&](int sn) -> const float* { return bsm + ((bseq + (uint32_t)sn) % NB2) * (BBYTES / 4); };

            if (PER || (tid == 0 && !abort))
                for (int i = 0; i < NS && i < NP; ++i) issue(i);
            if (!PER && tid == 0 && !abort)
                for (int sn = 0; sn < NB2 && sn < len; ++sn) issue_b(sn);
            if constexpr (PER) {
                cp_async_wait_all();
                __syncthreads();
            }

            // q[p][d] holds plane zb - R + d, zb the first plane of the current group of U steps
            float2 q[PY][QL];
#pragma unroll
            for (int i = 0; i < 2 * R; ++i) {
                wait(i);
                const float* P = stage(i);
#pragma unroll
                for (int p = 0; p < PY; ++p) q[p][i] = ld2(P + (R + ty * PY + p) * BX + own_off);
                if (i < R) {
                    if constexpr (PER) cp_async_wait_all();
                    __syncthreads();
                    if constexpr (PER) {
                        if (i + NS < NP) issue(i + NS);
                    } else if (tid == 0 && i + NS < NP && !abort) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue(i + NS);
                    }
                }
            }
            if constexpr (PER) {
                cp_async_wait_all();
                __syncthreads();
            }

            auto march = [&](auto AND_c, auto DV_c, auto EDGE_c) {
                constexpr bool AND = decltype(AND_c)::value, DV = decltype(DV_c)::value, EDGE = decltype(EDGE_c)::value;
                // 32-bit offset of this thread's first point in plane z (row p adds p nx); rows with
                // own[p] < 0 (edges only) are never touched
                uint32_t off = (uint32_t)z0 * ps + (uint32_t)((y0 + ty * PY) * nx + gx);
                // PER: right-hand side fetched two planes ahead by the threads (the last planes
                // re-read the piece's last); TMA-fed variants: from the right-hand-side ring
                float2 rvn[PY], rvn2[PY];
                if constexpr (PER) {
                    const uint32_t d1 = z0 + 1 < z1 ? ps : 0u;
#pragma unroll
                    for (int p = 0; p < PY; ++p) {
                        rvn[p] = (!EDGE || own[p] >= 0) ? ldg2(rhs + off + p * nx) : make_float2(0.f, 0.f);
                        rvn2[p] = (!EDGE || own[p] >= 0) ? ldg2(rhs + off + d1 + p * nx) : make_float2(0.f, 0.f);
                    }
                }
                float2 rprev[PY];  // BLK: residuals of the box's first plane
                // one z step; uu is the step's place in its group of U (a constant once unrolled)
                auto step = [&](int z, int uu) {
                    const int iz = z - z0 + R;
                    float2 rv[PY];
                    if constexpr (PER) {
#pragma unroll
                        for (int p = 0; p < PY; ++p) {
                            rv[p] = rvn[p];
                            rvn[p] = rvn2[p];
                        }
                        const uint32_t d2 = z + 2 < z1 ? 2u * ps : (z + 1 < z1 ? ps : 0u);
#pragma unroll
                        for (int p = 0; p < PY; ++p)
                            rvn2[p] = (!EDGE || own[p] >= 0) ? ldg2(rhs + off + d2 + p * nx) : make_float2(0.f, 0.f);
                    } else {
                        wait_b(z - z0);
                        const float* Bp = bstage(z - z0);
#pragma unroll
                        for (int p = 0; p < PY; ++p) rv[p] = ld2(Bp + (ty * PY + p) * 64 + 2 * lane);
                    }
                    // ring position of the incoming plane iz + R (one division per step): its
                    // stage and phase parity; the current plane iz sits R stages behind it
                    const uint32_t g_in = seq + (uint32_t)(iz + R), q_in = g_in / NS;
                    const uint32_t s_in = g_in - q_in * NS, par_in = q_in & 1u;
                    if constexpr (!PER) {  // plane iz + R has landed
                        const uint32_t bar = smem_u32(&bars[s_in]);
                        if (!mbar_try_wait(bar, par_in)) mbar_wait(bar, par_in, ev.err, abort, iz + R);
                    }
                    {
                        const float* F = sm + s_in * STAGE;
#pragma unroll
                        for (int p = 0; p < PY; ++p) q[p][uu + 2 * R] = ld2(F + (R + ty * PY + p) * BX + own_off);
                    }
                    const uint32_t s_cur = s_in >= (uint32_t)R ? s_in - R : s_in + (NS - R);
                    const float* P = sm + s_cur * STAGE;
                    float2 col[NCOL];
#pragma unroll
                    for (int r = 0; r < NCOL; ++r) col[r] = ld2(P + (ty * PY + r) * BX + own_off);
#pragma unroll
                    for (int p = 0; p < PY; ++p) {
                        const float* row = P + (R + ty * PY + p) * BX + own_off;
                        float2 w[NW];  // row elements -RE .. RE+1 around this thread's pair
#pragma unroll
                        for (int m = 0; m < NW; ++m) w[m] = ld2(row - RE + 2 * m);
                        const float2 c = q[p][uu + R];
                        float2 acc = __fmul2_rn(cd, c);
#pragma unroll
                        for (int kk = 1; kk <= R; ++kk) {
                            // x neighbours at distance kk of the pair: aligned words for even kk; for
                            // odd kk each point's two neighbours sit in different words, so the two
                            // sums are formed as scalars straight into the pair
                            float2 xs;
                            if (kk % 2 == 0) {
                                xs = __fadd2_rn(w[(RE - kk) / 2], w[(RE + kk) / 2]);
                            } else {
                                xs.x = w[(RE - kk - 1) / 2].y + w[(RE + kk - 1) / 2].y;
                                xs.y = w[(RE - kk + 1) / 2].x + w[(RE + kk + 1) / 2].x;
                            }
                            const float2 sv = __fadd2_rn(__fadd2_rn(__fadd2_rn(q[p][uu + R - kk], q[p][uu + R + kk]),
                                                                    __fadd2_rn(col[p + R - kk], col[p + R + kk])),
                                                         xs);
                            acc = __ffma2_rn(co[kk], sv, acc);
                        }
                        if constexpr (BLK) {
                            const float2 res = __ffma2_rn(mone, acc, rv[p]);  // rv - acc, one rounding
                            if ((!EDGE || own[p] >= 0) && AND) ssum = __ffma2_rn(res, res, ssum);
                            if (uu % 2 == 0) rprev[p] = res;
                            else rv[p] = res;  // the box's second plane (rv is not read again)
                        } else if (!EDGE || own[p] >= 0) {
                            const uint32_t o = off + p * nx;
                            const float2 res = __ffma2_rn(mone, acc, rv[p]);  // rv - acc, one rounding
                            const float2 f = __fmul2_rn(DV ? ldg2(dvec32 + o) : dinv_s, res);
                            st2(fout + o, f);
                            if constexpr (AND) ssum = __ffma2_rn(res, res, ssum);
                            else st2(xnext + o, __ffma2_rn(omega, f, c));
                        }
                    }
                    if constexpr (BLK) {
                        if (uu % 2 == 1 && (!EDGE || own[0] >= 0)) {
                            // the box of planes z - 1, z is complete: f = M^{-1} res for both planes
                            float2 rr[4] = {rprev[0], rprev[1], rv[0], rv[1]};
                            block2_apply(rr, bmu);
#pragma unroll
                            for (int qq = 0; qq < 4; ++qq) {
                                const int p = qq & 1, dz = qq >> 1;
                                const uint32_t o = off - (dz ? 0u : ps) + p * nx;
                                st2(fout + o, rr[qq]);
                                if constexpr (!AND) st2(xnext + o, __ffma2_rn(omega, rr[qq], q[p][uu - 1 + dz + R]));
                            }
                        }
                    }
                    off += ps;
                    // a CTA barrier after every B-th plane (B divides U): the stages of the last B
                    // planes are then free and take the planes NS further on. Planes skipped at a
                    // piece's last, incomplete group are not needed by the piece.
                    if (uu % B == B - 1) {
                        if constexpr (PER) cp_async_wait_all();  // planes read after this barrier
                        __syncthreads();
                        if constexpr (PER) {
#pragma unroll
                            for (int qq = B - 1; qq >= 0; --qq)
                                if (iz - qq + NS < NP) issue(iz - qq + NS);
                        } else if (tid == 0 && !abort) {
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll
                            for (int qq = B - 1; qq >= 0; --qq)
                                if (iz - qq + NS < NP) issue(iz - qq + NS);
                            // the right-hand-side stages of the last B steps take the steps NB2
                            // further on
                            const int sn = z - z0;
#pragma unroll
                            for (int qq = B - 1; qq >= 0; --qq)
                                if (sn - qq + NB2 < len) issue_b(sn - qq + NB2);
                        }
                    }
                };
                int zb = z0;
#pragma unroll 1
                for (; zb + U <= z1; zb += U) {
#pragma unroll
                    for (int uu = 0; uu < U; ++uu) step(zb + uu, uu);
#pragma unroll
                    for (int p = 0; p < PY; ++p)
#pragma unroll
                        for (int d = 0; d < 2 * R; ++d) q[p][d] = q[p][d + U];
                }
                if (zb < z1) {
#pragma unroll
                    for (int uu = 0; uu < U - 1; ++uu)
                        if (zb + uu < z1) step(zb + uu, uu);
                }
            };
            const bool dv = dvec32 != nullptr;
            if (anderson) {
                if (dv) {
                    if (edge) march(BT{}, BT{}, BT{});
                    else march(BT{}, BT{}, BF{});
                } else {
                    if (edge) march(BT{}, BF{}, BT{});
                    else march(BT{}, BF{}, BF{});
                }
            } else {
                if (dv) {
                    if (edge) march(BF{}, BT{}, BT{});
                    else march(BF{}, BT{}, BF{});
                } else {
                    if (edge) march(BF{}, BF{}, BT{});
                    else march(BF{}, BF{}, BF{});
                }
            }
            seq += (uint32_t)NP;
            bseq += (uint32_t)len;
            if constexpr (PER) cp_async_wait_all();
            // every read of this piece's stages is done before the next issue. A wait that gave up
            // anywhere in the CTA (TMA-fed variants; the others have no bounded waits) ends the
            // kernel here, once the copies still in flight have landed; the control kernel then
            // stops the solve with AAR_ERR_TIMEOUT.
            if (__syncthreads_or(abort)) {
                if (!PER && tid == 0) {
                    mbar_drain(bars, NS, seq - (uint32_t)NP, hi);
                    mbar_drain(bbars, NB2, bseq - (uint32_t)len, bhi);
                }
                return;
            }
        }
        if (anderson) {
            float v = ssum.x + ssum.y;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[ty] = (double)v;
            __syncthreads();
            if (tid == 0) {
                double tot = 0.0;
                for (int w = 0; w < BY; ++w) tot += red[w];
                ev.part_s[S.op0 + tile.local] = tot;
            }
        }
        __syncthreads();
    }
}

template <int R, int PY, int D, int U, int RB, bool PER, bool BLK = false>
inline cudaError_t launch_tma2(const OpLaunch& L, const EngineView& ev, int j, cudaStream_t s) {
    if (L.ntiles <= 0) return cudaSuccess;
    constexpr size_t bytes = tma2_smem_bytes<R, PY, D, PER>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep_tma2<R, PY, D, U, RB, PER, BLK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_sweep_tma2<R, PY, D, U, RB, PER, BLK><<<L.grid, dim3(32, 8), bytes, s>>>(ev, L.tiles, L.ntiles, j,
                                                                 reinterpret_cast<const CUtensorMap*>(L.maps));
    return cudaGetLastError();
}

template <int R, int PY, int D, int U, int RB, bool PER, bool BLK = false>
inline int occ_tma2() {
    constexpr size_t bytes = tma2_smem_bytes<R, PY, D, PER>();
    if (cudaFuncSetAttribute(k_sweep_tma2<R, PY, D, U, RB, PER, BLK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_tma2<R, PY, D, U, RB, PER, BLK>, 256, bytes) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

// Periodic paired sweep (plane stages filled by cp.async from wrapped indices), radius <= 4;
// BLK: with the fused block-Jacobi boxes
template <int R, bool BLK = false>
inline cudaError_t launch_tma2_per(const OpLaunch& L, const EngineView& ev, int j, cudaStream_t s) {
    if constexpr (R <= 4) return launch_tma2<R, 2, 3, 2, 2, true, BLK>(L, ev, j, s);
    else return cudaErrorInvalidValue;
}
template <int R, bool BLK = false>
inline int occ_tma2_per() {
    if constexpr (R <= 4) return occ_tma2<R, 2, 3, 2, 2, true, BLK>();
    else return 1;
}

}  // namespace aar

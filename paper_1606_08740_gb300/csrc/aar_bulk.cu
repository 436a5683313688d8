// aar_bulk.cu -- FP32 Anderson-step passes fed by 1-D bulk TMA copies (cp.async.bulk).
//
// The Gram pass (Eq. 3: F^T F and F^T f, c+1 residual columns) and the compressed update of the
// mixed-precision inner solves read 8 to 12 streams at once. In the register-fed kernels the
// bytes in flight per SM were capped by registers (their ncu long-scoreboard stalls dominated);
// here one elected thread copies a 512-element chunk of every stream into a shared-memory stage
// with cp.async.bulk, completing an mbarrier, three stages deep, and the CTA computes from shared
// memory. Per system the tile split, each thread's element order and the reduction order are
// fixed, so results depend only on the system.
#include <cuda.h>

#include "aar_engine.cuh"
#include "aar_mbar.cuh"
#include "aar_vecops.cuh"

namespace aar {

constexpr int BULK_CH = 512;     // elements per stream per chunk
constexpr int GRAM_STAGES = 4;   // Gram pass: 4 stages, freed two at a time (one CTA barrier per 2 chunks)
constexpr int GRAM_RB = 2;
constexpr int UPD_STAGES = 3;    // update pass: 3 stages, a CTA barrier per chunk

// Streams of one chunk: stage layout [stream][BULK_CH] floats.
struct BulkStreams {
    const float* p[MAXM + 3 + 2 * NAMAX];
    int ns;
};

template <int NSMAX, int NST>
struct BulkPipe {
    float* sm;           // NST * NSMAX * BULK_CH floats
    uint64_t* bars;      // NST barriers
    uint32_t seq;        // chunks issued before this tile
    uint32_t hi;         // warp 0: chunks issued so far (index of the last one + 1)
    bool abort;          // a wait of this thread gave up

    __device__ float* stage(uint32_t g) { return sm + (size_t)(g % NST) * NSMAX * BULK_CH; }

    // Called by the 32 lanes of warp 0: lane 0 posts the chunk's bytes on the stage's barrier,
    // lane s copies stream s (the copies of a chunk are issued in parallel, not one by one).
    __device__ void issue(uint32_t g, const BulkStreams& S, int64_t off, int len, int lane) {
        const uint32_t bar = smem_u32(&bars[g % NST]);
        const uint32_t bytes = (uint32_t)len * 4u;
        if (lane == 0) mbar_expect_tx(bar, bytes * (uint32_t)S.ns);
        float* st = stage(g);
        for (int s = lane; s < S.ns; s += 32) bulk_g2s(smem_u32(st + s * BULK_CH), S.p[s] + off, bytes, bar);
        hi = g + 1;
    }

    // Abort protocol. A thread whose wait gave up skips its later waits and computes on whatever
    // its stages hold (the solve ends with AAR_ERR_TIMEOUT, its results unused); the per-chunk CTA
    // barrier stays a plain __syncthreads, so the chunk loop carries no vote. Warp 0 issues only
    // while none of its lanes gave up (a warp-wide vote of the issuing warp alone): it waited for
    // every chunk it consumed, so a stage it refills holds no copy in flight. The CTA-wide vote runs
    // once per tile, after its last chunk (tile_end); on a wait that gave up anywhere, every thread
    // leaves the kernel and thread 0 first waits, bounded, for the copies still in flight. Each
    // thread gives up at most once, so a CTA whose copies stopped ends within one wait limit per
    // thread.
    __device__ bool may_issue() { return !__any_sync(0xffffffffu, abort); }

    __device__ bool tile_end(int tid) {
        if (!__syncthreads_or(abort)) return false;
        if (tid == 0) mbar_drain(bars, NST, 0u, hi);
        return true;
    }

    __device__ void wait(uint32_t g, int* err, int where) {
        mbar_wait(smem_u32(&bars[g % NST]), (g / NST) & 1u, err, abort, where);
    }
};

// ------------------------------------------------------------------------------------ Gram

template <int CMAX>
__global__ void __launch_bounds__(256, CMAX <= 8 ? 2 : 1) k_gram_bulk(EngineView ev, const VecTile* __restrict__ tiles, int ntiles,
                                                   int j) {
    AAR_COUNT_LAUNCH(ev);
    constexpr int NG = CMAX * (CMAX + 1) / 2 + CMAX;
    constexpr int NSMAX = CMAX + 2;  // f_k .. f_{k-c}, and fold for a split column
    constexpr bool PAIRED = CMAX <= 8;
    constexpr int NST = GRAM_STAGES, RB = GRAM_RB;
    static_assert(NST > RB && RB >= 1, "stage refill groups");
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[NST];
    __shared__ double red[8][NG];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    BulkPipe<NSMAX, NST> P;
    P.sm = reinterpret_cast<float*>(smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u));
    P.bars = bars;
    P.seq = 0;
    P.hi = 0;
    P.abort = false;
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const VecTile tile = tiles[t];
        const SysDesc& S = ev.sys[tile.sys];
        const SysState& st = ev.st[tile.sys];
        if (st.phase != PH_INNER) continue;
        const int64_t k = tick_step(st, S.p, j);
        if (k >= st.kcap || ((k + 1) % S.p) != 0) continue;
        const int c = (int)(k < S.m ? k : S.m);
        if (c == 0) continue;
        BulkStreams B;
        B.ns = c + 1;
        for (int a = 0; a <= c; ++a) B.p[a] = ring_ptr<float>(S.F, k - a, S);  // newest first
        // difference column a (f_{k-a} - f_{k-a-1}) whose upper end is the split iterate reads
        // that iterate's residual as it was before the restart (fold)
        int as = -1;
        if (st.split_k >= 0 && k >= st.split_k && k - st.split_k < c) {
            as = (int)(k - st.split_k);
            B.p[B.ns++] = S.fold;
        }
        const int64_t len_all = tile.end - tile.start;
        const int nch = (int)((len_all + BULK_CH - 1) / BULK_CH);
        auto chunk_len = [&](int q) { const int64_t r = len_all - (int64_t)q * BULK_CH; return (int)(r < BULK_CH ? r : BULK_CH); };
        if (warp == 0 && P.may_issue())
            for (int q = 0; q < NST && q < nch; ++q)
                P.issue(P.seq + q, B, tile.start + (int64_t)q * BULK_CH, chunk_len(q), lane);
        // PAIRED (short histories): each thread takes two neighbouring elements at a time and keeps
        // a pair of sums per entry (paired FP32 arithmetic, half the instructions), folded at the end
        float G[NG];
        float2 G2[PAIRED ? NG : 1];
#pragma unroll
        for (int e = 0; e < NG; ++e) G[e] = 0.f;
#pragma unroll
        for (int e = 0; e < (PAIRED ? NG : 1); ++e) G2[e] = make_float2(0.f, 0.f);
        const float2 mone = make_float2(-1.f, -1.f);
        // FULL: the window holds CMAX columns and none is split (the common case once the history
        // is full), compiled without the per-column selects of the general form
        auto run = [&](auto FULL_c) {
            constexpr bool FULL = decltype(FULL_c)::value;
#pragma unroll 1
            for (int q = 0; q < nch; ++q) {
                const uint32_t g = P.seq + q;
                P.wait(g, ev.err, q);
                const float* sm = P.stage(g);
                const int len = chunk_len(q);
                if constexpr (PAIRED) {
                    for (int e = 2 * tid; e < len; e += 512) {  // len is a multiple of 8
                        float2 v[CMAX + 1];
#pragma unroll
                        for (int a = 0; a <= CMAX; ++a)
                            v[a] = (FULL || a <= c) ? *reinterpret_cast<const float2*>(sm + a * BULK_CH + e)
                                                    : make_float2(0.f, 0.f);
                        float2 df[CMAX];
                        if constexpr (FULL) {
#pragma unroll
                            for (int a = 0; a < CMAX; ++a) df[a] = __ffma2_rn(mone, v[a + 1], v[a]);
                        } else {
                            const float2 vold = as >= 0 ? *reinterpret_cast<const float2*>(sm + (c + 1) * BULK_CH + e)
                                                        : make_float2(0.f, 0.f);
#pragma unroll
                            for (int a = 0; a < CMAX; ++a)
                                df[a] = (a < c) ? __ffma2_rn(mone, v[a + 1], a == as ? vold : v[a]) : make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int a = 0; a < CMAX; ++a) {
                            if (FULL || a < c) {
#pragma unroll
                                for (int b = 0; b <= a; ++b)
                                    G2[a * (a + 1) / 2 + b] = __ffma2_rn(df[a], df[b], G2[a * (a + 1) / 2 + b]);
                                G2[CMAX * (CMAX + 1) / 2 + a] = __ffma2_rn(df[a], v[0], G2[CMAX * (CMAX + 1) / 2 + a]);
                            }
                        }
                    }
                } else {
                    for (int e = tid; e < len; e += 256) {
                        float v[CMAX + 1];
#pragma unroll
                        for (int a = 0; a <= CMAX; ++a) v[a] = (FULL || a <= c) ? sm[a * BULK_CH + e] : 0.f;
                        float df[CMAX];
                        if constexpr (FULL) {
#pragma unroll
                            for (int a = 0; a < CMAX; ++a) df[a] = v[a] - v[a + 1];
                        } else {
                            const float vold = as >= 0 ? sm[(c + 1) * BULK_CH + e] : 0.f;
#pragma unroll
                            for (int a = 0; a < CMAX; ++a) df[a] = (a < c) ? (a == as ? vold : v[a]) - v[a + 1] : 0.f;
                        }
#pragma unroll
                        for (int a = 0; a < CMAX; ++a) {
                            if (FULL || a < c) {
#pragma unroll
                                for (int b = 0; b <= a; ++b)
                                    G[a * (a + 1) / 2 + b] = fmaf(df[a], df[b], G[a * (a + 1) / 2 + b]);
                                G[CMAX * (CMAX + 1) / 2 + a] = fmaf(df[a], v[0], G[CMAX * (CMAX + 1) / 2 + a]);
                            }
                        }
                    }
                }
                // a CTA barrier after every RB-th chunk: the stages of chunks q-RB+1 .. q then take
                // the chunks NST further on (the tile's last, incomplete group needs no refill; the
                // vote after the loop is its barrier)
                if (q % RB == RB - 1) {
                    __syncthreads();
                    if (warp == 0 && q + 1 - RB + NST < nch && P.may_issue()) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll
                        for (int qq = RB - 1; qq >= 0; --qq) {
                            const int qi = q - qq + NST;
                            if (qi < nch) P.issue(P.seq + qi, B, tile.start + (int64_t)qi * BULK_CH, chunk_len(qi), lane);
                        }
                    }
                }
            }
        };
        if (c == CMAX && as < 0) run(std::true_type{});
        else run(std::false_type{});
        P.seq += (uint32_t)nch;
        if (P.tile_end(tid)) return;
        if constexpr (PAIRED) {
#pragma unroll
            for (int e = 0; e < NG; ++e) G[e] = G2[e].x + G2[e].y;
        }
        // warp trees in FP32, the 8 warp sums in FP64 in warp order
#pragma unroll
        for (int e = 0; e < NG; ++e) {
            float v = G[e];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][e] = (double)v;
        }
        __syncthreads();
        // the tile's partial sums, as double-float pairs in the FP64 slots (the finalize adds them
        // with FP32 instructions)
        DF* out = reinterpret_cast<DF*>(ev.part_g + (int64_t)(S.vec0 + tile.local) * GSTRIDE);
        const int nlow = c * (c + 1) / 2;
        for (int e = tid; e < NG; e += 256) {
            double s = 0.0;
            for (int w = 0; w < 8; ++w) s += red[w][e];
            if (e < CMAX * (CMAX + 1) / 2) {
                if (e < nlow) out[e] = df_from_double(s);
            } else {
                const int a = e - CMAX * (CMAX + 1) / 2;
                if (a < c) out[nlow + a] = df_from_double(s);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------- update

// Compressed Anderson update of the FP32 inner solves (UPD_ANDERSON_C):
// x_{k+1} = x_k + sum_b alpha[b] f_{k-c+b} + sum_q ag[q] (x_{aj[q]-1} - x_{aj[q]})
//           [+ alpha_old fold],
// where x_{aj} is read from xold when aj is the split iterate. The other update kinds of a tick
// (x64 += d, and the literal form when more than NAMAX columns came from Anderson steps) run from
// plain loads (update_plain_tile).
template <int CMAX>
__global__ void __launch_bounds__(256, 2) k_update_bulk(EngineView ev, const VecTile* __restrict__ tiles, int ntiles) {
    AAR_COUNT_LAUNCH(ev);
    constexpr int NSMAX = CMAX + 3 + 2 * NAMAX;
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[UPD_STAGES];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    BulkPipe<NSMAX, UPD_STAGES> P;
    P.sm = reinterpret_cast<float*>(smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u));
    P.bars = bars;
    P.seq = 0;
    P.hi = 0;
    P.abort = false;
    if (tid == 0) {
        for (int s = 0; s < UPD_STAGES; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const VecTile tile = tiles[t];
        const SysDesc& S = ev.sys[tile.sys];
        const SysState& st = ev.st[tile.sys];
        if (st.upd == UPD_ADD_D || st.upd == UPD_ANDERSON) {
            update_plain_tile<float, CMAX>(S, st, tile);
            continue;
        }
        if (st.upd != UPD_ANDERSON_C) continue;
        const int64_t k = st.upd_k;
        const int c = st.upd_c, na = st.na;
        // streams: x_k, f_{k-c..k}, then (x_{aj-1}, x_{aj}) pairs
        BulkStreams B;
        B.p[0] = ring_ptr<float>(S.X, k, S);
        for (int b = 0; b <= c; ++b) B.p[1 + b] = ring_ptr<float>(S.F, k - c + b, S);
        for (int q = 0; q < na; ++q) {
            B.p[c + 2 + 2 * q] = ring_ptr<float>(S.X, st.aj[q] - 1, S);
            B.p[c + 3 + 2 * q] = st.aj[q] == st.split_k ? S.xold : ring_ptr<float>(S.X, st.aj[q], S);
        }
        B.ns = c + 2 + 2 * na;
        const bool use_old = st.alpha_old != 0.0;
        const float a_old = (float)st.alpha_old;
        if (use_old) B.p[B.ns++] = S.fold;
        const int s_old = c + 2 + 2 * na;
        float al[CMAX + 1], ag[NAMAX];
#pragma unroll
        for (int b = 0; b <= CMAX; ++b) al[b] = b <= c ? (float)st.alpha[b] : 0.f;
#pragma unroll
        for (int q = 0; q < NAMAX; ++q) ag[q] = q < na ? (float)st.ag[q] : 0.f;
        float* xn = ring_ptr<float>(S.X, k + 1, S);
        const int64_t len_all = tile.end - tile.start;
        const int nch = (int)((len_all + BULK_CH - 1) / BULK_CH);
        auto chunk_len = [&](int q) { const int64_t r = len_all - (int64_t)q * BULK_CH; return (int)(r < BULK_CH ? r : BULK_CH); };
        if (warp == 0 && P.may_issue())
            for (int q = 0; q < UPD_STAGES && q < nch; ++q)
                P.issue(P.seq + q, B, tile.start + (int64_t)q * BULK_CH, chunk_len(q), lane);
        for (int q = 0; q < nch; ++q) {
            const uint32_t g = P.seq + q;
            P.wait(g, ev.err, q);
            const float* sm = P.stage(g);
            const int len = chunk_len(q);
            const int64_t base = tile.start + (int64_t)q * BULK_CH;
            for (int e = 2 * tid; e < len; e += 512) {
                float2 out = *reinterpret_cast<const float2*>(sm + e);
#pragma unroll
                for (int b = 0; b <= CMAX; ++b) {
                    if (b <= c) {
                        const float2 f = *reinterpret_cast<const float2*>(sm + (1 + b) * BULK_CH + e);
                        out.x = fmaf(al[b], f.x, out.x);
                        out.y = fmaf(al[b], f.y, out.y);
                    }
                }
#pragma unroll
                for (int qq = 0; qq < NAMAX; ++qq) {
                    if (qq < na) {
                        const float2 va = *reinterpret_cast<const float2*>(sm + (c + 2 + 2 * qq) * BULK_CH + e);
                        const float2 vb = *reinterpret_cast<const float2*>(sm + (c + 3 + 2 * qq) * BULK_CH + e);
                        out.x = fmaf(ag[qq], va.x - vb.x, out.x);
                        out.y = fmaf(ag[qq], va.y - vb.y, out.y);
                    }
                }
                if (use_old) {
                    const float2 fo = *reinterpret_cast<const float2*>(sm + s_old * BULK_CH + e);
                    out.x = fmaf(a_old, fo.x, out.x);
                    out.y = fmaf(a_old, fo.y, out.y);
                }
                *reinterpret_cast<float2*>(xn + base + e) = out;
            }
            __syncthreads();  // chunk q is consumed: its stage takes chunk q + UPD_STAGES
            if (warp == 0 && q + UPD_STAGES < nch && P.may_issue()) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                P.issue(g + UPD_STAGES, B, tile.start + (int64_t)(q + UPD_STAGES) * BULK_CH, chunk_len(q + UPD_STAGES),
                        lane);
            }
        }
        P.seq += (uint32_t)nch;
        if (P.tile_end(tid)) return;
    }
}

template <int CMAX>
static size_t gram_bulk_smem() { return (size_t)GRAM_STAGES * (CMAX + 2) * BULK_CH * 4 + 1024; }
template <int CMAX>
static size_t update_bulk_smem() { return (size_t)UPD_STAGES * (CMAX + 3 + 2 * NAMAX) * BULK_CH * 4 + 1024; }

template <int CMAX>
static cudaError_t gram_bulk_c(const VecTile* tiles, int ntiles, int grid, const EngineView& ev, int j, cudaStream_t s) {
    static bool attr = false;
    const size_t bytes = gram_bulk_smem<CMAX>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gram_bulk<CMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_gram_bulk<CMAX><<<grid, 256, bytes, s>>>(ev, tiles, ntiles, j);
    return cudaGetLastError();
}

template <int CMAX>
static cudaError_t update_bulk_c(const VecTile* tiles, int ntiles, int grid, const EngineView& ev, cudaStream_t s) {
    static bool attr = false;
    const size_t bytes = update_bulk_smem<CMAX>();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_update_bulk<CMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_update_bulk<CMAX><<<grid, 256, bytes, s>>>(ev, tiles, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_gram_bulk(int cmax, const VecTile* tiles, int ntiles, int grid, const EngineView& ev, int j,
                             cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if (cmax <= 4) return gram_bulk_c<4>(tiles, ntiles, grid, ev, j, s);
    if (cmax <= 7) return gram_bulk_c<7>(tiles, ntiles, grid, ev, j, s);
    if (cmax <= 8) return gram_bulk_c<8>(tiles, ntiles, grid, ev, j, s);
    if (cmax <= 10) return gram_bulk_c<10>(tiles, ntiles, grid, ev, j, s);
    if (cmax <= 12) return gram_bulk_c<12>(tiles, ntiles, grid, ev, j, s);
    return gram_bulk_c<16>(tiles, ntiles, grid, ev, j, s);
}

cudaError_t launch_update_bulk(int cmax, const VecTile* tiles, int ntiles, int grid, const EngineView& ev,
                               cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if (cmax <= 4) return update_bulk_c<4>(tiles, ntiles, grid, ev, s);
    if (cmax <= 7) return update_bulk_c<7>(tiles, ntiles, grid, ev, s);
    if (cmax <= 8) return update_bulk_c<8>(tiles, ntiles, grid, ev, s);
    if (cmax <= 10) return update_bulk_c<10>(tiles, ntiles, grid, ev, s);
    if (cmax <= 12) return update_bulk_c<12>(tiles, ntiles, grid, ev, s);
    return update_bulk_c<16>(tiles, ntiles, grid, ev, s);
}

}  // namespace aar

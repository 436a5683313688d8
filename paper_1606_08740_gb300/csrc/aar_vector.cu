// aar_vector.cu -- Anderson-step kernels (Gram pass, finalize, update), CSR sweeps and the
// small control kernels of the AAR engine.
//
//  k_gram     : per vec tile, partial sums of G = F_k^T F_k and g = F_k^T f_k (Eq. 3) with the
//               difference columns of Eq. 5 formed on the fly from the raw residual ring.
//  k_finalize : one CTA per system. Sums the partial sums in tile order, evaluates
//               r_k = ||b - A x_k|| / ||b|| (checked only at Anderson steps, Sec. 2), and
//               solves gamma = pinv(G) g (Moore-Penrose, Sec. 3.2) with a one-warp cyclic
//               Jacobi eigensolver; drives the per-system phase machine.
//  k_update   : x_{k+1} = x_k + beta f_k - (X_k + beta F_k) gamma (Eq. 3, Anderson branch).
//  k_gram and k_update serve the FP64 form; the FP32 inner solves of the mixed form use the
//  bulk-copy-fed passes of aar_bulk.cu.
//  k_csr      : CSR variant of the fused sweep / FP64 residual / FP64 apply.
#include <math.h>
#include <stdlib.h>

#include <utility>

#include "aar_engine.cuh"
#include "aar_linalg.cuh"
#include "aar_vecops.cuh"

namespace aar {

// ------------------------------------------------------------------------------ Gram pass

__host__ __device__ constexpr int ngram(int c) { return c * (c + 1) / 2 + c; }

// Gram entries are stored row-major lower triangle: (a, b) with b <= a -> a(a+1)/2 + b, then g_a.
// Entry E of a history of CMAX columns: its row a and column b (b = CMAX: the f_k column of g).
__host__ __device__ constexpr int gram_row(int E, int C) {
    if (E >= C * (C + 1) / 2) return E - C * (C + 1) / 2;
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= E) ++a;
    return a;
}
__host__ __device__ constexpr int gram_col(int E, int C) {
    return E >= C * (C + 1) / 2 ? C : E - gram_row(E, C) * (gram_row(E, C) + 1) / 2;
}

constexpr int G64_CH = 256;  // points per chunk of the FP64 Gram pass

template <int CMAX, int E>
__device__ __forceinline__ void gram64_one(const double (*sd)[G64_CH], int p, double& g) {
    constexpr int a = gram_row(E, CMAX), b = gram_col(E, CMAX);
    g = fma(sd[a][p], sd[b][p], g);
}

template <int CMAX, int W, int NJ, int... J>
__device__ __forceinline__ void gram64_entries(const double (*sd)[G64_CH], int p, double* G,
                                               std::integer_sequence<int, J...>) {
    (gram64_one<CMAX, W + 8 * J>(sd, p, G[J]), ...);
}

// warp W: the entries W, W + 8, ... over the chunk's points lane, lane + 32, ...
template <int CMAX, int W>
__device__ __forceinline__ void gram64_chunk(const double (*sd)[G64_CH], int lane, double* G) {
    constexpr int NJ = (ngram(CMAX) - W + 7) / 8;
    if constexpr (NJ > 0) {
#pragma unroll 2
        for (int p = lane; p < G64_CH; p += 32)
            gram64_entries<CMAX, W, NJ>(sd, p, G, std::make_integer_sequence<int, NJ>{});
    }
}

// FP64 Gram pass of the plain FP64 form (Eq. 3: F^T F and F^T f_k). Chunks of 256 points: every
// thread loads one point's c + 1 residual values (the next chunk's while the current one is
// being summed), forms the c differences once and stores them with f_k in shared memory; warp w
// then accumulates the Gram entries w, w + 8, ... (their (a, b) compile-time constants, one
// multiply-add per entry and point), lane l over the points l, l + 32, ... Each entry belongs to
// one warp, whose lanes combine by a fixed shuffle tree. (A per-thread copy of every entry, as in
// the FP32 pass, made the FP64 cross-lane trees of all 8 warps cost more than the sums.)
template <int CMAX>
__global__ void __launch_bounds__(256) k_gram(EngineView ev, const VecTile* __restrict__ tiles, int ntiles, int j) {
    AAR_COUNT_LAUNCH(ev);
    constexpr int NG = ngram(CMAX), NJM = (NG + 7) / 8;
    __shared__ double sd[CMAX + 1][G64_CH];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const VecTile tile = tiles[t];
        const SysDesc& S = ev.sys[tile.sys];
        const SysState& st = ev.st[tile.sys];
        if (st.phase != PH_INNER) continue;
        const int64_t k = tick_step(st, S.p, j);
        if (k >= st.kcap || ((k + 1) % S.p) != 0) continue;
        const int c = (int)(k < S.m ? k : S.m);
        if (c == 0) continue;
        // columns newest first: fcol[a] = f_{k-a}, difference column a' = fcol[a'] - fcol[a'+1]
        // (= column c-1-a' of F_k in Eq. 5's oldest-first order; the finalize maps it back)
        const double* fcol[CMAX + 1];
#pragma unroll
        for (int a = 0; a <= CMAX; ++a) fcol[a] = ring_ptr<double>(S.F, k - (a <= c ? a : c), S);
        double G[NJM];
#pragma unroll
        for (int e = 0; e < NJM; ++e) G[e] = 0.0;
        const int64_t len = tile.end - tile.start;
        const int nch = (int)((len + G64_CH - 1) / G64_CH);
        double v[CMAX + 1];  // this thread's point of the next chunk
        auto load = [&](int q) {
            const int64_t i = tile.start + (int64_t)q * G64_CH + tid;
            const bool in = i < tile.end;
#pragma unroll
            for (int a = 0; a <= CMAX; ++a) v[a] = (a <= c && in) ? fcol[a][i] : 0.0;
        };
        load(0);
        const double one = unit_one();  // differences as FMAs (aar_fp64.cuh)
        for (int q = 0; q < nch; ++q) {
#pragma unroll
            for (int a = 0; a < CMAX; ++a) sd[a][tid] = a < c ? usub(v[a], v[a + 1], one) : 0.0;
            sd[CMAX][tid] = v[0];
            __syncthreads();
            if (q + 1 < nch) load(q + 1);
            switch (warp) {  // warp-uniform
                case 0: gram64_chunk<CMAX, 0>(sd, lane, G); break;
                case 1: gram64_chunk<CMAX, 1>(sd, lane, G); break;
                case 2: gram64_chunk<CMAX, 2>(sd, lane, G); break;
                case 3: gram64_chunk<CMAX, 3>(sd, lane, G); break;
                case 4: gram64_chunk<CMAX, 4>(sd, lane, G); break;
                case 5: gram64_chunk<CMAX, 5>(sd, lane, G); break;
                case 6: gram64_chunk<CMAX, 6>(sd, lane, G); break;
                default: gram64_chunk<CMAX, 7>(sd, lane, G); break;
            }
            __syncthreads();
        }
        double* out = ev.part_g + (int64_t)(S.vec0 + tile.local) * GSTRIDE;
        const int nlow = c * (c + 1) / 2;
#pragma unroll
        for (int jj = 0; jj < NJM; ++jj) {
            const int e = warp + 8 * jj;
            if (e >= NG) break;  // warp-uniform
            double g = G[jj];
            for (int o = 16; o > 0; o >>= 1) g += __shfl_down_sync(0xffffffffu, g, o);
            if (lane == 0) {
                // compact to the c-sized layout: lower triangle of c, then g
                if (e < CMAX * (CMAX + 1) / 2) {
                    if (e < nlow) out[e] = g;
                } else {
                    const int a = e - CMAX * (CMAX + 1) / 2;
                    if (a < c) out[nlow + a] = g;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------- update pass

template <typename T, int CMAX>
__global__ void __launch_bounds__(256, 2) k_update(EngineView ev, const VecTile* __restrict__ tiles, int ntiles) {
    AAR_COUNT_LAUNCH(ev);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const VecTile tile = tiles[t];
        const SysDesc& S = ev.sys[tile.sys];
        const SysState& st = ev.st[tile.sys];
        if (st.upd == UPD_ANDERSON) update_plain_tile<T, CMAX>(S, st, tile);
    }
}

// ------------------------------------------------------------------------------ ||b||^2

__global__ void __launch_bounds__(256) k_norm_b(EngineView ev, const VecTile* __restrict__ tiles, int ntiles) {
    AAR_COUNT_LAUNCH(ev);
    __shared__ double red[8];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const VecTile tile = tiles[t];
        const SysDesc& S = ev.sys[tile.sys];
        if (ev.st[tile.sys].phase != PH_INIT) continue;
        double s = 0.0;
        const int64_t end = tile.end < S.n ? tile.end : S.n;
        for (int64_t i = tile.start + threadIdx.x; i < end; i += 256) {
            const double b = S.b64[i];
            s = fma(b, b, s);
        }
        const double tot = block_sum<8>(s, red);
        if (threadIdx.x == 0) ev.part_g[(int64_t)(S.vec0 + tile.local) * GSTRIDE] = tot;
    }
}

// ------------------------------------------------------------------------------- finalize

__device__ double cta_sum_strided(const double* base, int64_t stride, int count, double* red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) s += base[(int64_t)i * stride];
    return block_sum<8>(s, red);  // thread 0 only
}

__device__ inline bool finite_d(double v) { return isfinite(v); }

// Mixed form: the inner solve that ended at iterate k_end hands its solution to the outer loop.
// at_anderson: it stopped at an Anderson step with its history intact, so the next inner solve
// can continue from that history instead of starting from an empty one.
__device__ void end_inner(const SysDesc& S, SysState& st, int64_t k_end, bool update_pending,
                          bool at_anderson = false) {
    st.iters_total += k_end - st.k_start;
    if (!S.mixed) {
        st.phase = PH_DONE;
        st.status = AAR_NOT_CONVERGED;
        st.k_final = k_end;
        return;
    }
    // the history is kept when the stop came at an Anderson step with nothing pending, and no
    // column of the window that the restart keeps straddles an earlier restart (one split
    // column at a time)
    const int64_t c_end = k_end < S.m ? k_end : S.m;
    st.keep = (!S.restart_history && at_anderson && !update_pending && k_end >= 1 &&
               st.split_k < k_end - c_end + 1) ? 1 : 0;
    st.hist_k = k_end;
    if (update_pending) {
        st.phase = PH_ADD;
        st.add_k = k_end;
    } else {
        st.upd = UPD_ADD_D;
        st.upd_k = k_end;
        st.phase = PH_RESID;
    }
}

struct FinShared {
    double Sm[MAXM * MAXM], Vm[MAXM * MAXM], gv[MAXM], lam[MAXM], vg[MAXM];
    double red[8];
    double gred[8 * GSTRIDE];  // per-warp Gram sums (FP64, or double-float pairs in the mixed form)
    int s_go;
};

// Record the Anderson update of step k with c columns (gamma already in st.gamma). For the FP32
// inner solves a difference column x_j - x_{j-1} whose step j-1 was a Richardson step equals
// omega f_{j-1} (Eq. 3), so (X + beta F) gamma folds into coefficients of the c+1 residual
// columns and only the columns produced by Anderson steps read iterates. A split column (see
// SysState::split_k) takes its upper end from xold / fold: its f term gets its own coefficient
// alpha_old, and x_{j-1} - x_j of an Anderson-produced split column reads xold (update pass).
__device__ void finish_anderson(const SysDesc& S, SysState& st, int64_t k, int c) {
    st.upd = UPD_ANDERSON;
    st.upd_k = k;
    st.upd_c = c;
    st.k0 = k + 1;
    if (S.mixed) {
        for (int b = 0; b <= c; ++b) st.alpha[b] = 0.0;
        st.alpha[c] = S.beta;
        st.alpha_old = 0.0;
        int na = 0;
        bool ok = true;
        for (int a = 0; a < c; ++a) {
            const int64_t jj = k - c + 1 + a;
            const double g = st.gamma[a];
            if (jj == st.split_k) st.alpha_old -= g * S.beta;
            else st.alpha[a + 1] -= g * S.beta;
            if (jj % S.p != 0) {
                st.alpha[a] -= g * (S.omega - S.beta);
            } else {
                st.alpha[a] += g * S.beta;
                if (na < NAMAX) {
                    st.aj[na] = jj;
                    st.ag[na] = g;
                    ++na;
                } else {
                    ok = false;
                }
            }
        }
        st.na = na;
        if (ok) st.upd = UPD_ANDERSON_C;
    }
    if (st.k0 >= st.kcap) end_inner(S, st, st.k0, true);
}

// finish_anderson for the FP32 inner solves, by the 32 lanes of warp 0: lane a handles window
// column a (iterate k - c + 1 + a, gamma_a = g) and coefficient alpha[a]; each alpha term is
// formed in the order the single-thread form applies it.
__device__ void finish_anderson_warp(const SysDesc& S, SysState& st, int64_t k, int c, int lane, double g) {
    constexpr unsigned FULL = 0xffffffffu;
    const int64_t jj = k - c + 1 + lane;
    const bool col = lane < c;
    // step jj-1 was an Anderson step: jj = 0 (mod p); k + 1 = 0 (mod p) at an Anderson step, so
    // jj = lane - c (mod p), in 32-bit arithmetic
    const int rj = (lane - c) % S.p;
    const bool isA = col && rj == 0;
    const bool split = col && jj == st.split_k;
    const double gprev = __shfl_up_sync(FULL, g, 1);
    const bool split_prev = __shfl_up_sync(FULL, split ? 1 : 0, 1) != 0;
    if (lane <= c) {
        double t = lane == c ? S.beta : 0.0;
        if (lane >= 1 && !split_prev) t -= gprev * S.beta;
        if (lane < c) t = isA ? t + g * S.beta : t - g * (S.omega - S.beta);
        st.alpha[lane] = t;
    }
    const unsigned smask = __ballot_sync(FULL, split);
    const double gs = __shfl_sync(FULL, g, smask ? __ffs(smask) - 1 : 0);
    const unsigned amask = __ballot_sync(FULL, isA);
    const int rank = __popc(amask & ((1u << lane) - 1u));
    if (isA && rank < NAMAX) {
        st.aj[rank] = jj;
        st.ag[rank] = g;
    }
    __syncwarp();
    if (lane == 0) {
        const int total = __popc(amask);
        st.alpha_old = smask ? 0.0 - gs * S.beta : 0.0;
        st.na = total < NAMAX ? total : NAMAX;
        st.upd = total <= NAMAX ? UPD_ANDERSON_C : UPD_ANDERSON;
        st.upd_k = k;
        st.upd_c = c;
        st.k0 = k + 1;
        st.last_rank = c;
        if (st.k0 >= st.kcap) end_inner(S, st, st.k0, true);
    }
}

// Warp w of the finalize adds the Gram partial sums of tiles w, w+8, w+16, ... in that order,
// lane l the entries l, l+32, ... (EPLR of them) of each; a tile's entries are contiguous, so
// every load is coalesced. U = 32 / EPLR tiles of the warp are loaded before they are added, so
// that a partial sum written by the Gram pass (often in the other die's L2) costs one round trip
// per U tiles, not per tile.
template <int EPLR, typename T, typename Add>
__device__ __forceinline__ void sum_tile_rows(const T* gb, int nvec, int ng, int warp, int lane, T (&acc)[EPLR],
                                              Add add) {
    constexpr int U = 32 / EPLR;
    for (int t0 = warp; t0 < nvec; t0 += 8 * U) {
        T v[U][EPLR];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const T* row = gb + (int64_t)min(t0 + 8 * u, nvec - 1) * GSTRIDE;  // in bounds
#pragma unroll
            for (int q = 0; q < EPLR; ++q) v[u][q] = (t0 + 8 * u < nvec && lane + 32 * q < ng) ? row[lane + 32 * q] : T{};
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int q = 0; q < EPLR; ++q)
                if (t0 + 8 * u < nvec && lane + 32 * q < ng) acc[q] = add(acc[q], v[u][q]);
    }
}

// The warp sums of sum_tile_rows into red[warp * GSTRIDE + e], for the EPLR that ng needs.
template <typename T, typename Add, int... Es>
__device__ __forceinline__ void sum_tiles_to(const T* gb, int nvec, int ng, int warp, int lane, T* red, Add add,
                                             std::integer_sequence<int, Es...>) {
    const int eplr = (ng + 31) / 32;
    (
        [&] {
            constexpr int E = Es + 1;
            if (eplr != E) return;
            T acc[E];
#pragma unroll
            for (int q = 0; q < E; ++q) acc[q] = T{};
            sum_tile_rows<E>(gb, nvec, ng, warp, lane, acc, add);
#pragma unroll
            for (int q = 0; q < E; ++q)
                if (lane + 32 * q < ng) red[warp * GSTRIDE + lane + 32 * q] = acc[q];
        }(),
        ...);
}

// S and st are the CTA's shared-memory copies of the system's descriptor and state (k_finalize
// copies them in and the state back out); ev supplies the partial sums.
__device__ void finalize_sys(EngineView ev, const SysDesc& S, SysState& st, int j, double pinv_eps_mixed,
                             FinShared& sh) {
    double* Sm = sh.Sm;
    double* Vm = sh.Vm;
    double* gv = sh.gv;
    double* lam = sh.lam;
    double* vg = sh.vg;
    double* red = sh.red;
    int& s_go = sh.s_go;
    const int tid = threadIdx.x;
    // every thread takes its branch decisions from values read before any thread writes state
    const int phase = st.phase;
    const int64_t kcap = st.kcap;
    const int64_t kt = tick_step(st, S.p, j);  // this tick's step (past the body's Richardson-only ticks)
    __syncthreads();
    // the update of the previous tick has run: clear it for every system, finished ones included
    if (tid == 0) st.upd = UPD_NONE;
    if (phase == PH_DONE) return;

    if (phase == PH_INIT) {
        const double s = cta_sum_strided(ev.part_g + (int64_t)S.vec0 * GSTRIDE, GSTRIDE, S.nvec, red);
        if (tid == 0) {
            const double nb = sqrt(s);
            st.nb = nb;
            st.r_last = nan("");
            if (!finite_d(nb)) {
                st.phase = PH_DONE;
                st.status = AAR_ERR_BREAKDOWN;
                st.k_final = 0;
            } else if (nb == 0.0) {
                st.phase = PH_DONE;
                st.status = AAR_OK;
                st.k_final = -1;
                st.r_last = 0.0;
            } else if (S.mixed) {
                st.phase = PH_RESID;
            } else {
                st.phase = PH_INNER;
                st.k0 = 0;
                st.kcap = S.max_iter;
                st.nrhs = nb;
            }
        }
        return;
    }
    if (phase == PH_ADD) {
        if (tid == 0) {
            st.upd = UPD_ADD_D;
            st.upd_k = st.add_k;
            st.phase = PH_RESID;
        }
        return;
    }
    if (phase == PH_RESID) {
        const double s = cta_sum_strided(ev.part_s + S.opd0, 1, S.nopd, red);
        if (tid == 0) {
            const double nr = sqrt(s);
            const double R = nr / st.nb;
            st.r_last = R;
            if (!finite_d(R)) {
                st.phase = PH_DONE;
                st.status = AAR_ERR_BREAKDOWN;
            } else if (R <= S.tol) {
                st.phase = PH_DONE;
                st.status = AAR_OK;
            } else if (st.iters_total >= S.max_iter || st.refinements >= S.max_refine) {
                st.phase = PH_DONE;
                st.status = AAR_NOT_CONVERGED;
            } else {
                st.phase = PH_INNER;
                if (st.keep) {
                    // continue on the new right-hand side with the history kept: step hist_k is
                    // re-run as an Anderson step from x = 0 (its earlier x and f were saved to
                    // xold / fold by the x64 += d pass)
                    const int64_t k = st.hist_k;
                    st.k0 = k;
                    st.k_start = k;
                    st.k_zero = k;
                    st.split_k = k;
                    st.kcap = k + (S.max_iter - st.iters_total);
                } else {
                    st.k0 = 0;
                    st.k_start = 0;
                    st.k_zero = 0;
                    st.split_k = -1;
                    st.kcap = S.max_iter - st.iters_total;
                }
                st.keep = 0;
                st.nrhs = nr;
                st.refinements += 1;
                st.n_rin = 0;
            }
        }
        return;
    }
    // PH_INNER
    const int64_t k = kt;
    if (k >= kcap) {
        if (tid == 0) end_inner(S, st, kcap, false);
        return;
    }
    const bool anderson = ((k + 1) % S.p) == 0;
    if (!anderson) {
        if (tid == 0) {
            st.k0 = k + 1;
            if (st.k0 >= st.kcap) end_inner(S, st, st.k0, false);
        }
        return;
    }
    const int c = (int)(k < S.m ? k : S.m);
    const double s = cta_sum_strided(ev.part_s + S.op0, 1, S.nop, red);
    if (tid == 0) {
        const double rin = sqrt(s) / st.nrhs;
        st.anderson += 1;
        st.r_inner = rin;
        int go = 1;
        if (!finite_d(rin)) {
            st.phase = PH_DONE;
            st.status = AAR_ERR_BREAKDOWN;
            st.k_final = k;
            st.iters_total += k - st.k_start;
            go = 0;
        } else if (!S.mixed) {
            st.r_last = rin;
            if (rin <= S.tol) {
                st.phase = PH_DONE;
                st.status = AAR_OK;
                st.k_final = k;
                st.iters_total += k - st.k_start;
                go = 0;
            }
        } else {
            double target = 0.5 * S.tol * st.nb / st.nrhs;
            if (target < S.inner_tol) target = S.inner_tol;
            bool stop = rin <= target;
            // stagnation at the FP32 floor: less than a 10% decrease over the last STAG_WINDOW
            // Anderson steps of this inner solve
            if (st.n_rin >= STAG_WINDOW && rin >= 0.9 * st.rin_hist[st.n_rin % STAG_WINDOW]) stop = true;
            st.rin_hist[st.n_rin % STAG_WINDOW] = rin;
            st.n_rin += 1;
            if (stop) {
                end_inner(S, st, k, false, true);
                go = 0;
            }
        }
        s_go = go;
    }
    __syncthreads();
    if (!s_go) return;
    // Gram sums: warp w adds the tiles w, w+8, ... in turn (sum_tile_rows), then entry e of the 8
    // warp sums in warp order. The order is fixed by the system's tiles alone.
    const int ng = ngram(c), nlow = c * (c + 1) / 2;
    const int warp = tid >> 5, lane = tid & 31;
    // entry e of the Gram pass (newest column first) into G and g (oldest column first)
    auto place = [&](int e, double v) {
        if (e < nlow) {
            int a = 0;
            while ((a + 1) * (a + 2) / 2 <= e) ++a;
            const int b = e - a * (a + 1) / 2;
            const int ra = c - 1 - a, rb = c - 1 - b;
            Sm[ra * MAXM + rb] = v;
            Sm[rb * MAXM + ra] = v;
        } else {
            gv[c - 1 - (e - nlow)] = v;
        }
    };
    constexpr auto EPLS = std::make_integer_sequence<int, (GSTRIDE + 31) / 32>{};
    if (S.mixed) {
        // double-float partials added with FP32 instructions
        const DF* gb = reinterpret_cast<const DF*>(ev.part_g + (int64_t)S.vec0 * GSTRIDE);
        DF* wred = reinterpret_cast<DF*>(sh.gred);
        sum_tiles_to(gb, S.nvec, ng, warp, lane, wred, [](DF a, DF b) { return df_add(a, b); }, EPLS);
        __syncthreads();
        for (int e = tid; e < ng; e += blockDim.x) {
            DF v = wred[e];
            for (int w = 1; w < 8; ++w) v = df_add(v, wred[w * GSTRIDE + e]);
            place(e, df_to_double(v));
        }
    } else {
        const double* gb = ev.part_g + (int64_t)S.vec0 * GSTRIDE;
        sum_tiles_to(gb, S.nvec, ng, warp, lane, sh.gred, [](double a, double b) { return a + b; }, EPLS);
        __syncthreads();
        for (int e = tid; e < ng; e += blockDim.x) {
            double v = sh.gred[e];
            for (int w = 1; w < 8; ++w) v += sh.gred[w * GSTRIDE + e];
            place(e, v);
        }
    }
    __syncthreads();
    if (S.mixed) {
        // FP32 inner solve: gamma from the normal equations G gamma = g by an LDL^T factorisation
        // (about c^3/6 FP64 operations instead of a Jacobi eigensolve, whose FP64 cost dominates
        // the Anderson step on this part). It equals pinv(G) g whenever every pivot clears the
        // rank threshold; otherwise the eigen-decomposition below decides the kept rank. Warp 0
        // factorises right-looking with one row per lane (lane i keeps row i of the remaining
        // matrix, then of L, in registers); L also goes to Vm for the back substitution.
        if (warp == 0) {
            double z = 0.0;
            const bool ok = ldl_solve_dispatch<MAXM, false>(c, Sm, gv, Vm, lane, z, std::make_integer_sequence<int, MAXM>{});
            if (lane == 0) s_go = ok ? 2 : 1;  // 2: solved by LDL^T, 1: eigen-decomposition below
            if (ok) {
                if (lane < c) {
                    st.gamma[lane] = z;
                    vg[lane] = z;
                }
                finish_anderson_warp(S, st, k, c, lane, z);
            }
        }
        __syncthreads();
        if (s_go == 2) return;
    } else {
        // plain FP64 form: the certified LDL^T solve (pinv(G) = G^-1 proven), else the eigen
        // pseudoinverse below
        if (warp == 0) {
            double z = 0.0;
            const bool ok = ldl_solve_dispatch<MAXM, true>(c, Sm, gv, Vm, lane, z, std::make_integer_sequence<int, MAXM>{});
            if (lane == 0) s_go = ok ? 2 : 1;
            if (ok) {
                if (lane < c) st.gamma[lane] = z;
                __syncwarp();
                if (lane == 0) {
                    st.last_rank = c;
                    finish_anderson(S, st, k, c);
                }
            }
        }
        __syncthreads();
        if (s_go == 2) return;
    }
    if (warp < 4) cta_sym_eig<MAXM, 4>(c, Sm, Vm);  // warps 0-3; ends with a barrier among them
    if (warp == 0) {
        const double pinv_eps = S.mixed ? pinv_eps_mixed : ldexp(1.0, -52);
        if (lane == 0) st.n_eig += 1;
        if (lane < c) lam[lane] = Sm[lane * MAXM + lane];
        __syncwarp();
        double lmax = 0.0;
        for (int i = 0; i < c; ++i) lmax = fmax(lmax, lam[i]);
        const double tau = (double)c * pinv_eps * lmax;
        if (lane < c) {  // v_j . g for column j = lane
            double acc = 0.0;
            for (int i = 0; i < c; ++i) acc += Vm[i * MAXM + lane] * gv[i];
            vg[lane] = acc;
        }
        __syncwarp();
        if (lane < c) {
            double gam = 0.0;
            for (int jj = 0; jj < c; ++jj)
                if (lam[jj] > tau && lmax > 0.0) gam += Vm[lane * MAXM + jj] * (vg[jj] / lam[jj]);
            st.gamma[lane] = gam;
        }
        int kept = 0;
        bool fin = true;
        for (int jj = 0; jj < c; ++jj) kept += (lam[jj] > tau && lmax > 0.0) ? 1 : 0;
        __syncwarp();
        if (lane == 0) {
            for (int a = 0; a < c; ++a) fin = fin && finite_d(st.gamma[a]);
            st.last_rank = kept;
            if (!fin) {
                st.phase = PH_DONE;
                st.status = AAR_ERR_BREAKDOWN;
                st.k_final = k;
                st.iters_total += k - st.k_start;
            } else {
                finish_anderson(S, st, k, c);
            }
        }
    }
}

// One CTA per system. When the tick runs inside the solve graph, the last CTA to finish (found
// with a fenced counter) also sets the conditions of the graph's IF nodes: whether the next
// tick needs the FP64 residual pass or the Gram pass, and whether this tick's update pass runs.
__global__ void __launch_bounds__(256) k_finalize(EngineView ev, int j, double pinv_eps_mixed, FinConds fc) {
    AAR_COUNT_LAUNCH(ev);
    __shared__ FinShared sh;
    __shared__ int last, f_resid, f_gram, f_upd;
    // the system's descriptor and state in shared memory: the finalize's many scattered field
    // reads (several inside one-thread sections) would otherwise each be a global round trip
    __shared__ __align__(16) SysDesc s_desc;
    __shared__ __align__(16) SysState s_st;
    static_assert(sizeof(SysDesc) % 8 == 0 && sizeof(SysState) % 8 == 0, "copied as 8-byte words");
    const int sys = blockIdx.x;
    const int tid = threadIdx.x;
    if (sys < ev.nsys) {
        const uint64_t* gd = reinterpret_cast<const uint64_t*>(&ev.sys[sys]);
        uint64_t* gs = reinterpret_cast<uint64_t*>(&ev.st[sys]);
        uint64_t* ld = reinterpret_cast<uint64_t*>(&s_desc);
        uint64_t* ls = reinterpret_cast<uint64_t*>(&s_st);
        for (int i = tid; i < (int)(sizeof(SysDesc) / 8); i += blockDim.x) ld[i] = gd[i];
        for (int i = tid; i < (int)(sizeof(SysState) / 8); i += blockDim.x) ls[i] = gs[i];
        __syncthreads();
        finalize_sys(ev, s_desc, s_st, j, pinv_eps_mixed, sh);
        __syncthreads();
        for (int i = tid; i < (int)(sizeof(SysState) / 8); i += blockDim.x) gs[i] = ls[i];
    }
    if (!fc.use) return;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(fc.counter, 1) == (int)gridDim.x - 1;
        f_resid = f_gram = f_upd = 0;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int s = tid; s < ev.nsys; s += blockDim.x) {
        const volatile SysState& st = ev.st[s];
        const int ph = st.phase;
        if (st.upd != UPD_NONE) f_upd = 1;
        if (ph == PH_RESID) f_resid = 1;
        if (ph == PH_INNER) {
            const int64_t k = st.k0;  // the next tick's step
            if (k < st.kcap && ((k + 1) % ev.sys[s].p) == 0) f_gram = 1;
        }
    }
    __syncthreads();
    if (tid == 0) {
        cudaGraphSetConditional(fc.h_resid, f_resid ? 1u : 0u);
        cudaGraphSetConditional(fc.h_gram, f_gram ? 1u : 0u);
        cudaGraphSetConditional(fc.h_upd, f_upd ? 1u : 0u);
        *fc.counter = 0;
    }
}

// ------------------------------------------------------------------------------ control

__global__ void k_control(EngineView ev, int* ctrl, cudaGraphConditionalHandle h, int ticks, int use_handle) {
    AAR_COUNT_LAUNCH(ev);
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < ev.nsys; s += blockDim.x)
        if (ev.st[s].phase != PH_DONE) any = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        ctrl[0] += ticks;
        int cont = any;
        if (cont && (ctrl[0] >= ctrl[1] || ctrl[3] != 0)) {
            for (int s = 0; s < ev.nsys; ++s) {
                SysState& st = ev.st[s];
                if (st.phase != PH_DONE) {
                    st.phase = PH_DONE;
                    st.status = AAR_ERR_TIMEOUT;
                    st.k_final = st.k0;
                }
            }
            cont = 0;
        }
        ctrl[2] = cont;
        if (use_handle) cudaGraphSetConditional(h, cont ? 1u : 0u);
    }
}

// Sets IF conditions to 1 at the start of a solve-graph body pass (handles without a default).
__global__ void k_set_conds(cudaGraphConditionalHandle h0, cudaGraphConditionalHandle h1, cudaGraphConditionalHandle h2) {
    cudaGraphSetConditional(h0, 1u);
    cudaGraphSetConditional(h1, 1u);
    cudaGraphSetConditional(h2, 1u);
}

cudaError_t launch_set_conds(const cudaGraphConditionalHandle* h, int n, cudaStream_t s) {
    if (n != 3) return cudaErrorInvalidValue;
    k_set_conds<<<1, 1, 0, s>>>(h[0], h[1], h[2]);
    return cudaGetLastError();
}

// -------------------------------------------------------------------------------- CSR

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_csr(EngineView ev, const OpTile* __restrict__ tiles, int ntiles, int j,
                                             const double* __restrict__ xin, double* __restrict__ yout) {
    AAR_COUNT_LAUNCH(ev);
    __shared__ double red[8];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const OpTile tile = tiles[t];
        const SysDesc& S = ev.sys[tile.sys];
        const SysState& st = ev.st[tile.sys];
        const T* x = nullptr;
        const T* rhs = nullptr;
        T* fout = nullptr;
        T* xnext = nullptr;
        T* xzero = nullptr;
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
        } else {
            x = reinterpret_cast<const T*>(xin);
        }
        const bool want_sum = (MODE == SM_RESID) || (MODE == SM_SWEEP && anderson);
        const T omega = (T)S.omega;
        T ssum = T(0);
        for (int row = tile.x0 + threadIdx.x; row < tile.y0; row += blockDim.x) {
            const int e0 = __ldg(S.row_ptr + row), e1 = __ldg(S.row_ptr + row + 1);
            T acc = T(0);
            if (!zero_x) {
                for (int e = e0; e < e1; ++e) {
                    T a;
                    if constexpr (sizeof(T) == 4) a = __ldg(S.val32 + e);
                    else a = __ldg(S.val + e);
                    acc = fma(a, __ldg(x + __ldg(S.col_idx + e)), acc);
                }
            }
            if constexpr (MODE == SM_SWEEP) {
                const T res = __ldg(rhs + row) - acc;
                T dv;
                if constexpr (sizeof(T) == 4) dv = __ldg(S.dinv_vec32 + row);
                else dv = __ldg(S.dinv_vec + row);
                const T f = dv * res;
                fout[row] = f;
                const T xc = zero_x ? T(0) : __ldg(x + row);
                if (anderson) ssum = fma(res, res, ssum);
                else xnext[row] = fma(omega, f, xc);
                if (zero_x) xzero[row] = T(0);
            } else if constexpr (MODE == SM_RESID) {
                const T r = __ldg(rhs + row) - acc;
                S.rhs32[row] = (float)r;
                ssum = fma(r, r, ssum);
            } else {
                yout[row] = (double)acc;
            }
        }
        if (want_sum) {
            const double tot = block_sum<8>((double)ssum, red);
            if (threadIdx.x == 0) ev.part_s[(MODE == SM_RESID ? S.opd0 : S.op0) + tile.local] = tot;
        }
    }
}

// Diagonal extraction (Jacobi M = D) plus a structural check of the CSR arrays: row_ptr must be
// non-decreasing within [0, nnz] and every column index must lie in [0, n); any violation sets
// *bad and the entries of that row are not followed.
__global__ void k_csr_diag(int n, const int* __restrict__ row_ptr, const int* __restrict__ col_idx,
                           const double* __restrict__ val, double* dinv, float* dinv32, float* val32, int64_t nnz,
                           int* bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n; row += stride) {
        const int e0 = row_ptr[row], e1 = row_ptr[row + 1];
        if (e0 < 0 || e1 < e0 || e1 > nnz || (row == 0 && e0 != 0) || (row == n - 1 && e1 != nnz)) {
            atomicExch(bad, 1);
            continue;
        }
        double d = 0.0;
        for (int e = e0; e < e1; ++e) {
            const int c = col_idx[e];
            if (c < 0 || c >= n) atomicExch(bad, 1);
            if (c == row) d += val[e];
        }
        if (dinv) {
            if (d == 0.0 || !isfinite(d)) atomicExch(bad, 1);
            dinv[row] = 1.0 / d;
            if (dinv32) dinv32[row] = (float)(1.0 / d);
        }
    }
    if (val32)
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += stride) val32[e] = (float)val[e];
}

__global__ void k_to_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = (float)src[i];
}

__global__ void __launch_bounds__(256) k_dot_partials(const double* __restrict__ a, const double* __restrict__ b,
                                                      int64_t n, double* partials) {
    __shared__ double red[8];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t s0 = blockIdx.x * per, s1 = s0 + per < n ? s0 + per : n;
    double s = 0.0;
    for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) s = fma(a[i], b[i], s);
    const double tot = block_sum<8>(s, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// ||b - y|| / ||b|| for the public residual check: per-block partial sums, then one block
// combines them in block order.
__global__ void __launch_bounds__(256) k_resid_norm(const double* __restrict__ b, const double* __restrict__ y,
                                                    int64_t n, double* parts) {
    __shared__ double red[8];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t s0 = blockIdx.x * per, s1 = s0 + per < n ? s0 + per : n;
    double rr = 0.0, bb = 0.0;
    for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
        const double r = b[i] - y[i];
        rr = fma(r, r, rr);
        bb = fma(b[i], b[i], bb);
    }
    const double t0 = block_sum<8>(rr, red);
    const double t1 = block_sum<8>(bb, red);
    if (threadIdx.x == 0) {
        parts[2 * blockIdx.x] = t0;
        parts[2 * blockIdx.x + 1] = t1;
    }
}

__global__ void __launch_bounds__(256) k_resid_norm_final(const double* __restrict__ parts, int np, double* out) {
    __shared__ double red[8];
    double rr = 0.0, bb = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        rr += parts[2 * i];
        bb += parts[2 * i + 1];
    }
    const double t0 = block_sum<8>(rr, red);
    const double t1 = block_sum<8>(bb, red);
    if (threadIdx.x == 0) out[0] = sqrt(t0) / sqrt(t1);
}

cudaError_t launch_resid_norm(const double* b, const double* y, int64_t n, double* parts, int np, double* out,
                              cudaStream_t s) {
    k_resid_norm<<<np, 256, 0, s>>>(b, y, n, parts);
    k_resid_norm_final<<<1, 256, 0, s>>>(parts, np, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ launches

template <int CMAX>
static cudaError_t gram_c(const VecTile* tiles, int ntiles, int grid, const EngineView& ev, int j, cudaStream_t s) {
    k_gram<CMAX><<<grid, 256, 0, s>>>(ev, tiles, ntiles, j);
    return cudaGetLastError();
}

cudaError_t launch_gram(int cmax, const VecTile* tiles, int ntiles, int grid, const EngineView& ev, int j,
                        cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if (cmax <= 4) return gram_c<4>(tiles, ntiles, grid, ev, j, s);
    if (cmax <= 7) return gram_c<7>(tiles, ntiles, grid, ev, j, s);
    if (cmax <= 8) return gram_c<8>(tiles, ntiles, grid, ev, j, s);
    if (cmax <= 10) return gram_c<10>(tiles, ntiles, grid, ev, j, s);
    if (cmax <= 12) return gram_c<12>(tiles, ntiles, grid, ev, j, s);
    return gram_c<16>(tiles, ntiles, grid, ev, j, s);
}

template <int CMAX>
static cudaError_t update_c(const VecTile* tiles, int ntiles, int grid, const EngineView& ev, cudaStream_t s) {
    k_update<double, CMAX><<<grid, 256, 0, s>>>(ev, tiles, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_update(int cmax, const VecTile* tiles, int ntiles, int grid, const EngineView& ev, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    if (cmax <= 4) return update_c<4>(tiles, ntiles, grid, ev, s);
    if (cmax <= 7) return update_c<7>(tiles, ntiles, grid, ev, s);
    if (cmax <= 8) return update_c<8>(tiles, ntiles, grid, ev, s);
    if (cmax <= 10) return update_c<10>(tiles, ntiles, grid, ev, s);
    if (cmax <= 12) return update_c<12>(tiles, ntiles, grid, ev, s);
    return update_c<16>(tiles, ntiles, grid, ev, s);
}

cudaError_t launch_norm_b(const VecTile* tiles, int ntiles, int grid, const EngineView& ev, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    k_norm_b<<<grid, 256, 0, s>>>(ev, tiles, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const EngineView& ev, int j, cudaStream_t s, FinConds fc) {
    k_finalize<<<ev.nsys, 256, 0, s>>>(ev, j, ldexp(1.0, -52), fc);
    return cudaGetLastError();
}

cudaError_t launch_control(const EngineView& ev, int* ctrl, cudaGraphConditionalHandle h, int ticks,
                           cudaStream_t s) {
    k_control<<<1, 256, 0, s>>>(ev, ctrl, h, ticks, h != 0 ? 1 : 0);
    return cudaGetLastError();
}

// ------------------------------------------------------------ domain decomposition

// One CTA: warp w folds the entries w, w + 8, ... of system 0's tile partials, lanes striding
// the tiles, then a fixed warp tree (the finalize's own order of summation).
__global__ void __launch_bounds__(256) k_dd_pack(EngineView ev, int mode, int c, double* __restrict__ packed) {
    const SysDesc& S = ev.sys[0];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ne = mode == 0 ? 1 : 1 + ngram(c);
    for (int e = warp; e < ne; e += 8) {
        double v = 0.0;
        if (mode == 0) {
            for (int t = lane; t < S.nvec; t += 32) v += ev.part_g[(int64_t)(S.vec0 + t) * GSTRIDE];
        } else if (e == 0) {
            for (int t = lane; t < S.nop; t += 32) v += ev.part_s[S.op0 + t];
        } else {
            for (int t = lane; t < S.nvec; t += 32) v += ev.part_g[(int64_t)(S.vec0 + t) * GSTRIDE + (e - 1)];
        }
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) packed[e] = v;
    }
}

__global__ void __launch_bounds__(256) k_dd_unpack(EngineView ev, int mode, int c, const double* __restrict__ packed) {
    const SysDesc& S = ev.sys[0];
    const int ng = mode == 0 ? 1 : ngram(c);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)S.nvec * ng;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(i / ng), e = (int)(i - (int64_t)t * ng);
        ev.part_g[(int64_t)(S.vec0 + t) * GSTRIDE + e] = t == 0 ? packed[mode == 0 ? 0 : 1 + e] : 0.0;
    }
    if (mode == 1)
        for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < S.nop; t += (int64_t)gridDim.x * blockDim.x)
            ev.part_s[S.op0 + t] = t == 0 ? packed[0] : 0.0;
}

cudaError_t launch_dd_pack(const EngineView& ev, int mode, int c, double* packed, cudaStream_t s) {
    k_dd_pack<<<1, 256, 0, s>>>(ev, mode, c, packed);
    return cudaGetLastError();
}

cudaError_t launch_dd_unpack(const EngineView& ev, int mode, int c, const double* packed, cudaStream_t s) {
    k_dd_unpack<<<64, 256, 0, s>>>(ev, mode, c, packed);
    return cudaGetLastError();
}

cudaError_t launch_csr(int fp32, int mode, const OpLaunch& L, const EngineView& ev, int j, const double* xin,
                       double* yout, cudaStream_t s) {
    if (L.ntiles <= 0) return cudaSuccess;
    if (mode == SM_SWEEP && fp32) k_csr<float, SM_SWEEP><<<L.grid, 256, 0, s>>>(ev, L.tiles, L.ntiles, j, xin, yout);
    else if (mode == SM_SWEEP) k_csr<double, SM_SWEEP><<<L.grid, 256, 0, s>>>(ev, L.tiles, L.ntiles, j, xin, yout);
    else if (mode == SM_RESID) k_csr<double, SM_RESID><<<L.grid, 256, 0, s>>>(ev, L.tiles, L.ntiles, j, xin, yout);
    else k_csr<double, SM_APPLY><<<L.grid, 256, 0, s>>>(ev, L.tiles, L.ntiles, j, xin, yout);
    return cudaGetLastError();
}

cudaError_t launch_csr_diag(int n, const int* row_ptr, const int* col_idx, const double* val, double* dinv,
                            float* dinv32, float* val32, int64_t nnz, int* bad, cudaStream_t s) {
    k_csr_diag<<<1024, 256, 0, s>>>(n, row_ptr, col_idx, val, dinv, dinv32, val32, nnz, bad);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t s) {
    k_to_f32<<<1024, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_dot_partials(const double* a, const double* b, int64_t n, double* partials, int nparts,
                                cudaStream_t s) {
    k_dot_partials<<<nparts, 256, 0, s>>>(a, b, n, partials);
    return cudaGetLastError();
}

}  // namespace aar

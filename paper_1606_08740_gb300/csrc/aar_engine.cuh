// aar_engine.cuh -- internal data layout and device helpers of the GB300 AAR engine.
//
// One engine advances a batch of independent systems (a single solve is a batch of one).
// Every system owns, in HBM:
//   X ring : nslots = max(m+1, 2) iterate slots x_{k-m..k}   (Eq. 4 is formed from these)
//   F ring : nslots residual slots f_{k-m..k}                  (Eq. 5 is formed from these)
//   slot(k) = k mod nslots; slot length ld (padded to 64 elements, padding stays zero)
// plus, for the mixed-precision form, an FP64 iterate x64 and an FP32 right-hand side rhs32.
// Work is described by two tile lists shared by the whole batch:
//   op tiles  : 32 x TY x ZC boxes of a stencil grid, or row ranges of a CSR matrix
//   vec tiles : contiguous index ranges, used by the Gram and update passes
// Each tile owns one slot of partial sums, and a system's partial sums are always combined in
// tile order, so a system's reduction order depends only on its own size.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "aar.h"

namespace aar {

constexpr int MAXM = AAR_MAX_M;
constexpr int MAXR = AAR_MAX_RADIUS;
constexpr int GSTRIDE = MAXM * (MAXM + 1) / 2 + MAXM;  // Gram partial slot: c(c+1)/2 + c entries
constexpr int VEC_ALIGN = 8;                          // vec tile starts are multiples of this
constexpr int PAD = 64;                               // vector length padding (elements)
constexpr int STAG_WINDOW = 12;                       // inner stagnation window (Anderson steps)

enum Phase : int { PH_INIT = 0, PH_INNER = 1, PH_RESID = 2, PH_ADD = 3, PH_DONE = 4 };
enum Upd : int { UPD_NONE = 0, UPD_ANDERSON = 1, UPD_ADD_D = 2, UPD_ANDERSON_C = 3 };
constexpr int NAMAX = 4;  // Anderson-produced difference columns the compressed update handles

struct OpTile {
    int sys;    // system index
    int local;  // tile index within the system (partial-sum slot = SysDesc::op0 + local)
    int x0, y0; // stencil: tile origin; CSR: row range [x0, y0)
    int z0, z1; // stencil: z range
};

struct VecTile {
    int sys;
    int local;
    int64_t start, end;  // [start, end), start % VEC_ALIGN == 0, end <= padded length
};

struct SysDesc {
    int64_t n;
    int nx, ny, nz, is_csr;
    int periodic;  // stencil: 1 = every axis wraps, 0 = zero Dirichlet ghosts
    int radius;    // stencil radius r (0 for CSR)
    int block;     // 2: block Jacobi with 2 x 2 x 2 boxes (the sweep writes b - A x_k, k_block_apply
                   // applies M^{-1} and the Richardson update); else Jacobi
    double bl_mu[4];  // block Jacobi: 1 / (8 lambda_t), lambda_t = cdiag + coff[1] (3 - 2t), t = 0..3
    float bl_mu_f[4];
    // stencil: (A x)_i = cdiag x_i + sum_{k=1..r} coff[k] * (sum of the 6 neighbours at distance k)
    double cdiag, coff[MAXR + 1];
    float cdiag_f, coff_f[MAXR + 1];
    double dinv;            // scalar Jacobi scaling when dinv_vec == nullptr
    float dinv_f;
    const double* dinv_vec; // per-point M^{-1} (FP64) or nullptr
    const float* dinv_vec32;
    // CSR
    const int* row_ptr;
    const int* col_idx;
    const double* val;
    const float* val32;
    // vectors
    void* X;
    void* F;
    int64_t ld;
    int nslots, mixed;
    const double* b64;  // right-hand side (FP64)
    double* x64;        // mixed: FP64 iterate
    float* rhs32;       // mixed: FP32 inner right-hand side
    float* xold;        // mixed: x and f of the split iterate (the one a refinement restarted at,
    float* fold;        //        as they were before it; see SysState::split_k)
    // tiles / partial slots
    int op0, nop;    // sweep-tile partial slots (precision's own tile shape)
    int opd0, nopd;  // FP64 residual-tile partial slots
    int vec0, nvec;  // vec-tile partial slots
    // parameters
    double omega, beta, tol, inner_tol;
    int m, p, max_refine;
    int restart_history;  // mixed: every inner solve starts from an empty history
    int hint_variant, hint_zc;  // tile hints (0 = automatic)
    int map0;           // first tensor map of this system's X ring (TMA sweep variants)
    int64_t max_iter;
    // slab of a domain-decomposed grid (FP64 sweeps): the z neighbours below plane 0 and above
    // plane nz - 1 are read from these r planes each (exchanged between ranks) instead of being
    // zero or wrapped; nullptr for a whole grid
    const double* ghost_lo;
    const double* ghost_hi;
};

struct SysState {
    int phase, status, upd, last_rank;
    int64_t k0;          // inner iteration index at the current tick (k = tick_step(st, j))
    int64_t kcap;        // inner iteration cap of the current inner solve
    int64_t upd_k;       // iterate index the pending update reads (x_{upd_k}, f_{upd_k})
    int64_t add_k;       // mixed: inner iterate to add once the pending update has run
    int64_t iters_total; // all inner iterations so far
    int64_t k_final;     // FP64: ring index of the returned iterate; -1 = zero vector
    int upd_c, anderson, refinements, n_rin;
    int n_eig;           // Anderson steps whose m x m solve took the eigen-decomposition
    double nb, nrhs, r_last, r_inner;
    double rin_hist[16];  // mixed: inner residuals of the last Anderson steps (circular)
    double gamma[MAXM];
    // compressed Anderson update of the FP32 inner solves (UPD_ANDERSON_C):
    // x_{k+1} = x_k + sum_b alpha[b] f_{k-c+b} + sum_q ag[q] (x_{aj[q]-1} - x_{aj[q]})
    double alpha[MAXM + 1];
    double ag[NAMAX];
    int64_t aj[NAMAX];
    double alpha_old;  // UPD_ANDERSON_C: coefficient of fold (split column inside the window)
    int na, keep;
    // mixed form, history kept across refinements. A refinement that keeps the history restarts
    // the inner iteration at the Anderson step K = hist_k where the previous one stopped, on the
    // new right-hand side, with x_K = 0 (k_zero = K: the sweep treats x_K as zero). Differences
    // between stored columns are independent of the right-hand side (Eq. 4/5), so the older
    // columns stay as stored; only the difference column x_K - x_{K-1}, f_K - f_{K-1} straddles
    // the restart, and it reads x_K, f_K as they were before it from xold / fold
    // (split_k = K; -1 when no column straddles a restart).
    int64_t k_start, hist_k, k_zero, split_k;
};

struct EngineView {
    const SysDesc* sys;
    SysState* st;
    double* part_s;  // [op tiles]
    double* part_g;  // [vec tiles * GSTRIDE]
    int nsys;
    int* err;        // set by a kernel whose bounded wait gave up
    int* nlaunch;    // kernels launched during the current solve (each kernel counts itself once)
};

// Every solve-loop kernel counts its own launch (block 0, thread 0), so kernels skipped by the
// solve graph's IF nodes are not counted.
#define AAR_COUNT_LAUNCH(ev)                                                                  \
    do {                                                                                      \
        if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0 && (ev).nlaunch)          \
            atomicAdd((ev).nlaunch, 1);                                                       \
    } while (0)

__host__ __device__ inline int64_t ring_slot(int64_t k, int nslots) { return k % nslots; }

template <typename T>
__device__ inline T* ring_ptr(void* base, int64_t k, const SysDesc& S) {
    return reinterpret_cast<T*>(base) + ring_slot(k, S.nslots) * S.ld;
}

template <typename T> struct Coef;
template <> struct Coef<double> {
    static __device__ inline double cdiag(const SysDesc& S) { return S.cdiag; }
    static __device__ inline double coff(const SysDesc& S, int k) { return S.coff[k]; }
    static __device__ inline double dinv(const SysDesc& S) { return S.dinv; }
};
template <> struct Coef<float> {
    static __device__ inline float cdiag(const SysDesc& S) { return S.cdiag_f; }
    static __device__ inline float coff(const SysDesc& S, int k) { return S.coff_f[k]; }
    static __device__ inline float dinv(const SysDesc& S) { return S.dinv_f; }
};

// Block-wide FP64 sum with a fixed combination order (warp tree, then warps in index order).
template <int NWARPS>
__device__ inline double block_sum(double v, double* scratch /* >= NWARPS */) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0) {
        for (int w = 0; w < NWARPS; ++w) s += scratch[w];
    }
    return s;  // valid in thread 0 only
}

// Tick index j of a solve-loop launch:
//   j = 0: a full tick: every unfinished system takes its step k0 (Richardson, Anderson or a
//          refinement phase) and the finalize advances its state;
//   j = 1 .. p-1: the j-th Richardson-only tick of a loop body laid out for a common Anderson
//          period p (p - 1 of them, then one TICK_FULL tick): only the sweep runs, a system in an
//          inner solve taking step k0 + j - 1 when steps k0 .. k0 + j - 1 are Richardson steps
//          below its cap; nothing else of its state changes, so no finalize is needed;
//   j = TICK_FULL: the full tick that ends such a body: step k0 + n, n the Richardson steps the
//          system took in the body's Richardson-only ticks (the finalize then sets k0 past them).
constexpr int TICK_FULL = -2;

// Richardson steps a system takes in the Richardson-only ticks of a body that starts at k0: those
// before its next Anderson step (k + 1 = 0 mod p), at most p - 1, and below its cap.
template <typename State>
__host__ __device__ inline int64_t tick_rsteps(const State& st, int p) {
    if (st.phase != PH_INNER || p < 2) return 0;
    int64_t n = (int64_t)(p - 1) - st.k0 % p;
    if (n > st.kcap - st.k0) n = st.kcap - st.k0;
    return n > 0 ? n : 0;
}

template <typename State>
__host__ __device__ inline int64_t tick_step(const State& st, int p, int j) {
    if (j == TICK_FULL) return st.k0 + tick_rsteps(st, p);
    return st.k0 + (j > 0 ? j - 1 : 0);
}

// Whether the sweep of tick j takes a step for a system in an inner solve.
template <typename State>
__host__ __device__ inline bool tick_sweeps(const State& st, int p, int j) {
    if (j > 0) return j - 1 < tick_rsteps(st, p);
    return tick_step(st, p, j) < st.kcap;
}

// Double-float numbers: an unevaluated sum hi + lo of two FP32 values, about 48 significant
// bits. The mixed form's Gram pass stores each tile's partial sums this way and the finalize adds
// them with FP32 instructions (this part's FP32 rate is 64 times its FP64 rate).
struct DF {
    float hi, lo;
};

__device__ inline DF df_from_double(double v) {
    const float hi = (float)v;
    return DF{hi, (float)(v - (double)hi)};
}

// a + b: Knuth's TwoSum of the high parts, the low parts added to its error term, and the result
// renormalised with Dekker's Fast2Sum.
__device__ inline DF df_add(DF a, DF b) {
    const float s = a.hi + b.hi;
    const float v = s - a.hi;
    const float e = (a.hi - (s - v)) + (b.hi - v);
    const float t = e + (a.lo + b.lo);
    const float hi = s + t;
    return DF{hi, t - (hi - s)};
}

__device__ inline double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

// ---- launch entry points implemented in the .cu files (host side) --------------------------
struct OpLaunch {
    const OpTile* tiles;
    int ntiles;
    int grid;
    int variant;  // tile-shape variant
    const void* maps = nullptr;  // CUtensorMap array (TMA variants)
};

// stencil kernels (aar_stencil_r*.cu)
enum StencilMode : int { SM_SWEEP = 0, SM_RESID = 1, SM_APPLY = 2 };
cudaError_t launch_stencil(int radius, int fp32, int mode, const OpLaunch& L, const EngineView& ev, int j,
                           const double* xin, double* yout, cudaStream_t s);
int stencil_variant_ty(int fp32, int variant);            // tile height of a variant
int stencil_variant_threads(int fp32, int variant);       // threads per CTA
int stencil_tma_box_x(int radius, int variant);           // TMA box x extent
int stencil_variant_tx(int fp32, int variant);            // tile width of a variant
int stencil_occupancy(int radius, int fp32, int mode, int variant);  // resident CTAs per SM
// block Jacobi (SysDesc::block == 2): f = M^{-1} res over the 2 x 2 x 2 boxes of every system in
// an inner phase at tick j, then x_{k+1} = x_k + omega f at a Richardson step (aar_block.cu)
cudaError_t launch_block_apply(int fp32, const EngineView& ev, int j, int grid, cudaStream_t s);

// vector/CSR/control kernels (aar_vector.cu)
cudaError_t launch_csr(int fp32, int mode, const OpLaunch& L, const EngineView& ev, int j, const double* xin,
                       double* yout, cudaStream_t s);
// register-fed Gram / literal update of the FP64 form
cudaError_t launch_gram(int cmax, const VecTile* tiles, int ntiles, int grid, const EngineView& ev, int j,
                        cudaStream_t s);
cudaError_t launch_update(int cmax, const VecTile* tiles, int ntiles, int grid, const EngineView& ev, cudaStream_t s);
// bulk-TMA-fed Gram / update of the FP32 inner solves (aar_bulk.cu)
cudaError_t launch_gram_bulk(int cmax, const VecTile* tiles, int ntiles, int grid, const EngineView& ev, int j,
                             cudaStream_t s);
cudaError_t launch_update_bulk(int cmax, const VecTile* tiles, int ntiles, int grid, const EngineView& ev,
                               cudaStream_t s);
cudaError_t launch_norm_b(const VecTile* tiles, int ntiles, int grid, const EngineView& ev, cudaStream_t s);
// Domain decomposition: fold system 0's tile partial sums into one packed vector (mode 0: ||b||^2;
// mode 1: ||b - A x_k||^2 and the c(c+1)/2 + c Gram entries), and after the sum over ranks write
// the packed values back as the first tile's partials (the other tiles' zeroed).
cudaError_t launch_dd_pack(const EngineView& ev, int mode, int c, double* packed, cudaStream_t s);
cudaError_t launch_dd_unpack(const EngineView& ev, int mode, int c, const double* packed, cudaStream_t s);
// IF-node conditions a finalize sets when it runs inside the solve graph (use = 0 elsewhere)
struct FinConds {
    int use;
    int* counter;  // device counter, zero between launches
    cudaGraphConditionalHandle h_resid, h_gram, h_upd;
};
cudaError_t launch_finalize(const EngineView& ev, int j, cudaStream_t s, FinConds fc = FinConds{0, nullptr, 0, 0, 0});
cudaError_t launch_set_conds(const cudaGraphConditionalHandle* h, int n, cudaStream_t s);
cudaError_t launch_control(const EngineView& ev, int* ctrl, cudaGraphConditionalHandle h, int ticks,
                           cudaStream_t s);
cudaError_t launch_csr_diag(int n, const int* row_ptr, const int* col_idx, const double* val, double* dinv,
                            float* dinv32, float* val32, int64_t nnz, int* bad, cudaStream_t s);
cudaError_t launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t s);
cudaError_t launch_resid_norm(const double* b, const double* y, int64_t n, double* parts, int np, double* out,
                              cudaStream_t s);
cudaError_t launch_dot_partials(const double* a, const double* b, int64_t n, double* partials, int nparts,
                                cudaStream_t s);

}  // namespace aar

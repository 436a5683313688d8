// aar_api.cu -- host side of the AAR engine and the C ABI declared in include/aar.h.
//
// An Engine advances nsys independent systems. It owns the device tables (system descriptors,
// per-system state, tile lists, partial-sum slots) and each system's history ring. A solve is:
//   1. copy parameters and the initial state to the device, place x0 in the ring (or x64),
//   2. ||b||^2 partial sums + finalize (PH_INIT),
//   3. a CUDA graph whose single conditional WHILE node repeats a body of ticks plus a control
//      kernel; a full tick = [FP64 residual (mixed)] -> sweep -> Gram -> finalize -> update,
//      each kernel covering every system whose phase asks for it. When every system has the
//      same Anderson period p >= 2 the body is p - 1 Richardson-only ticks (sweep -> finalize)
//      and one full tick, so the passes that only Anderson steps and refinements need are not
//      launched for the steps in between; otherwise the body is TICKS full ticks. The control
//      kernel ends the loop once every system is done or the step limit is reached,
//   4. copy the returned iterate out and read the per-system state back.
// If conditional graph nodes are unavailable the same body runs from a host loop instead.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <thread>
#include <deque>
#include <mutex>
#include <new>
#include <vector>

#include "aar.h"
#include "aar_dd.h"
#include "aar_engine.cuh"

using namespace aar;

namespace {

constexpr int TICKS = 8;           // ticks per WHILE-body iteration

struct Group {  // op tiles launched together with one kernel variant
    int variant;
    int offset, count, grid;
};

#define AAR_CHECK(call)                               \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return fail_cuda(e_);  \
    } while (0)

aar_status fail_cuda(cudaError_t e) {
    if (getenv("AAR_DEBUG")) fprintf(stderr, "aar: CUDA error %d: %s\n", (int)e, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return AAR_ERR_OOM;
    }
    if (e == cudaErrorLaunchTimeout) return AAR_ERR_TIMEOUT;
    return AAR_ERR_CUDA;
}

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Wait for the stream, giving up after AAR_WAIT_TIMEOUT_S seconds (default 1800) so that a
// caller is never blocked forever; the device-side step limit bounds the work itself.
cudaError_t wait_stream(cudaStream_t s) {
    double limit = 1800.0;
    if (const char* v = getenv("AAR_WAIT_TIMEOUT_S")) limit = atof(v);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(s);
        if (e != cudaErrorNotReady) return e;
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (dt > limit) return cudaErrorLaunchTimeout;
        std::this_thread::sleep_for(std::chrono::microseconds(dt < 0.01 ? 5 : 200));
    }
}

int cmax_for(int m) { return m <= 4 ? 4 : m <= 7 ? 7 : m <= 8 ? 8 : m <= 10 ? 10 : m <= 12 ? 12 : 16; }

struct Engine {
    int nsys = 0, fp32 = 0, radius = 0, is_csr = 0, sms = 1;
    int device = -1;  // ordinal of the device that was current when the engine was set up
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream used for graph capture
    std::vector<SysDesc> sys;
    std::vector<OpTile> sweep_tiles, dtiles;
    std::vector<VecTile> vtiles;
    std::vector<Group> sweep_groups, dgroups;
    SysDesc* d_sys = nullptr;
    SysState* d_st = nullptr;
    SysState* h_st = nullptr;  // pinned
    OpTile* d_sweep_tiles = nullptr;
    OpTile* d_dtiles = nullptr;
    VecTile* d_vtiles = nullptr;
    double* d_part_s = nullptr;
    double* d_part_g = nullptr;
    int* d_ctrl = nullptr;
    int* h_ctrl = nullptr;  // pinned
    int vec_grid = 1;
    // memory
    std::vector<int> slots_alloc;  // per system: slots currently allocated
    void* d_pool = nullptr;        // rings (+ x64, rhs32, xold, fold) of all systems
    size_t pool_bytes = 0;
    double* d_bstage = nullptr;    // single-system host-b staging
    // TMA tensor maps of the FP32 X rings (one per slot of each system on a TMA variant)
    std::vector<int> sweep_variant;
    std::vector<char> active;  // server engines: systems currently admitted (empty = all)
    size_t cap_sweep = 0, cap_dtiles = 0, cap_vtiles = 0, cap_part_s = 0, cap_part_g = 0;
    CUtensorMap* d_maps = nullptr;
    // CSR-owned extras
    double* d_dinv_own = nullptr;
    float* d_dinv32 = nullptr;
    float* d_val32 = nullptr;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_cmax = -1;
    bool graph_failed = false;
    int graph_mode = -1;       // solve-graph variant in use (-1: not built yet)
    int graph_period = -1;     // Anderson period the graph body is laid out for (0: full ticks)
    cudaStream_t cap_stream2 = nullptr;  // captures IF-node bodies
    bool solved = false;       // a solve has staged parameters and rings
    int last_cmax = 4;
    int64_t last_ticks = 0;    // ticks run by the last solve
    int64_t last_launches = 0; // kernels the last solve launched (counted on the device)

    EngineView view() const { return EngineView{d_sys, d_st, d_part_s, d_part_g, nsys, d_ctrl + 3, d_ctrl + 8}; }

    ~Engine() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaFree(d_sys);
        cudaFree(d_st);
        cudaFreeHost(h_st);
        cudaFree(d_sweep_tiles);
        cudaFree(d_dtiles);
        cudaFree(d_vtiles);
        cudaFree(d_part_s);
        cudaFree(d_part_g);
        cudaFree(d_ctrl);
        cudaFreeHost(h_ctrl);
        cudaFree(d_pool);
        cudaFree(d_bstage);
        cudaFree(d_dinv_own);
        cudaFree(d_dinv32);
        cudaFree(d_val32);
        cudaFree(d_maps);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (cap_stream2) cudaStreamDestroy(cap_stream2);
    }
};

// --------------------------------------------------------------------------- tile building

// z-chunk depth of a stencil tile: deep enough that the 2r-plane prologue is amortised, shallow
// enough to give the grid several CTAs per SM. A grid too small to fill the device with such
// tiles (a few x-y tiles, each marching z plane after plane) is latency-bound: its chunks are
// halved, down to r planes, until there is a tile per SM.
int choose_zc(int nz, int radius, int64_t xy_tiles, int sms) {
    int zc = 32;
    if (nz <= 48) zc = nz;
    // grow while there are plenty of tiles
    while (zc < nz && xy_tiles * ((nz + zc - 1) / zc) > (int64_t)sms * 16) zc *= 2;
    if (zc < 4 * radius && nz > zc) zc = std::min(nz, 4 * radius);
    while (zc > radius && zc > 1 && xy_tiles * ((nz + zc - 1) / zc) < (int64_t)sms) zc = (zc + 1) / 2;
    return std::max(1, std::min(zc, nz));
}

void build_stencil_tiles(int sys, const SysDesc& S, int tx, int ty, int radius, int sms, std::vector<OpTile>& out,
                         int* count) {
    const int tx_n = (S.nx + tx - 1) / tx, ty_n = (S.ny + ty - 1) / ty;
    const int zc = S.hint_zc > 0 ? std::min(S.hint_zc, S.nz) : choose_zc(S.nz, radius, (int64_t)tx_n * ty_n, sms);
    const int nzc = (S.nz + zc - 1) / zc;
    int local = 0;
    for (int yt = 0; yt < ty_n; ++yt)
        for (int xt = 0; xt < tx_n; ++xt)
            for (int zt = 0; zt < nzc; ++zt) {
                OpTile t;
                t.sys = sys;
                t.local = local++;
                t.x0 = xt * tx;
                t.y0 = yt * ty;
                t.z0 = zt * zc;
                t.z1 = std::min(S.nz, (zt + 1) * zc);
                out.push_back(t);
            }
    *count = local;
}

// Segments for the paired-FP32 TMA sweep: the system's linear (column, plane) index space
// u = col * nz + z (columns: the tx x ty boxes in row-major order) cut into nseg equal ranges
// [z0, z1), so that a single system's CTAs all get the same work whatever the grid shape. nseg is
// the sweep's resident CTA count (slots), unless that makes segments shorter than max(16, 4r)
// planes; a tile_zc hint asks for segments of about that many planes instead. The split depends
// only on the system and the device.
void build_segment_tiles(int sys, const SysDesc& S, int tx, int ty, int radius, int slots, std::vector<OpTile>& out,
                         int* count) {
    const int64_t cols = (int64_t)((S.nx + tx - 1) / tx) * ((S.ny + ty - 1) / ty);
    const int64_t U = cols * S.nz;
    const int64_t lmin = std::max(16, 4 * radius);
    int64_t nseg = S.hint_zc > 0 ? (U + S.hint_zc - 1) / S.hint_zc : std::min<int64_t>(slots, U / lmin);
    nseg = std::max<int64_t>(1, std::min<int64_t>(nseg, U));
    // block Jacobi pairs planes: segment ends on even planes (nz is even, so an even index u is an
    // even plane); segments left empty by the rounding are dropped
    const int64_t al = S.block >= 2 ? 2 : 1;
    int local = 0;
    for (int64_t i = 0; i < nseg; ++i) {
        OpTile t;
        t.sys = sys;
        t.x0 = t.y0 = 0;
        t.z0 = (int)(i * U / nseg / al * al);
        t.z1 = (int)(i + 1 == nseg ? U : (i + 1) * U / nseg / al * al);
        if (t.z1 <= t.z0) continue;
        t.local = local++;
        out.push_back(t);
    }
    *count = local;
}

void build_csr_tiles(int sys, int64_t n, std::vector<OpTile>& out, int* count) {
    const int rows = 2048;
    int local = 0;
    for (int64_t r = 0; r < n; r += rows) {
        OpTile t;
        t.sys = sys;
        t.local = local++;
        t.x0 = (int)r;
        t.y0 = (int)std::min<int64_t>(n, r + rows);
        t.z0 = t.z1 = 0;
        out.push_back(t);
    }
    *count = local;
}

// Vec tiles of one system: at most 2 per SM (so the Gram partial sums stay few and the finalize
// combines them quickly), at least min_pts points each (2048 for the bandwidth-bound FP32 passes;
// 256 for FP64, whose Gram and update passes are bound by the FP64 pipe, so that a small system
// still spreads over the device); boundaries on 64-element multiples. The split depends only on
// the system size, the precision and the device, never on the rest of the batch.
// Smallest vector tile of an FP32 system (the bulk-copy Gram and update passes restart their copy
// pipeline at every tile, so small systems of a batch get few, long tiles). A system's tiles
// depend on its own size only.
constexpr int64_t VEC_MIN_FP32 = 8192;

void build_vec_tiles(int sys, int64_t n, int sms, int64_t min_pts, std::vector<VecTile>& out, int* count) {
    const int64_t end_all = round_up(n, 8);
    const int64_t ntile = std::max<int64_t>(1, std::min<int64_t>((n + min_pts - 1) / min_pts, 2 * (int64_t)sms));
    const int64_t chunk = round_up((end_all + ntile - 1) / ntile, 64);
    int local = 0;
    for (int64_t s = 0; s < end_all; s += chunk) {
        VecTile t;
        t.sys = sys;
        t.local = local++;
        t.start = s;
        t.end = std::min(end_all, s + chunk);
        out.push_back(t);
    }
    *count = local;
}

// Variant choice for the op kernels (tile shape) from the system size only. FP32 sweeps of grids
// with 16-byte rows (nx % 4 == 0) use the TMA-fed kernel, or on a periodic grid of radius <= 4
// its cp.async-fed form (variant 5). AAR_SWEEP_VARIANT forces a variant for FP32 sweeps where it
// is valid (used by the tile autotuner).
bool variant_valid(const SysDesc& S, int fp32, int v) {
    if (v < 0 || v > 7) return false;
    if (!fp32) return v <= 1;
    if (v >= 4 && S.n >= ((int64_t)1 << 31)) return false;  // 32-bit offsets
    // block Jacobi: the register-fed sweep writes b - A x (k_block_apply follows), or the paired
    // sweep with the boxes fused (6: zero ghosts, 7: periodic, radius <= 4)
    if (S.block >= 2) {
        if (v == 6) return !S.periodic && !S.is_csr && S.nx % 4 == 0;
        if (v == 7) return S.periodic && !S.is_csr && S.nx % 4 == 0 && S.radius <= 4;
        return v <= 1;
    }
    if (v >= 6) return false;
    if (v == 5) return S.periodic && !S.is_csr && S.nx % 4 == 0 && S.radius <= 4;
    if (S.periodic) return v <= 1;  // the TMA box reads zero ghosts, never wraps
    return v <= 1 || S.nx % 4 == 0;
}

int choose_variant(const SysDesc& S, int fp32) {
    const int64_t side = std::max(S.nx, S.ny);
    if (S.hint_variant > 0 && variant_valid(S, fp32, S.hint_variant - 1)) return S.hint_variant - 1;
    if (fp32 && !S.is_csr && S.block >= 2) {
        if (side >= 64 && variant_valid(S, fp32, 6)) return 6;
        if (side >= 64 && variant_valid(S, fp32, 7)) return 7;
    } else if (fp32 && !S.is_csr) {
        if (const char* v = getenv("AAR_SWEEP_VARIANT")) {
            const int f = atoi(v);
            if (variant_valid(S, fp32, f)) return f;
        }
        if (S.periodic) {
            if (side >= 64 && variant_valid(S, fp32, 5)) return 5;
        } else if (S.nx % 4 == 0) {
            return side >= 64 ? 4 : 3;
        }
    }
    return side >= 48 ? 0 : 1;
}

int grid_for(int ntiles, int occ, int sms) {
    const int64_t cap = (int64_t)occ * sms;
    return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, cap));
}

template <typename T>
cudaError_t upload(T** dptr, const std::vector<T>& v) {
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc(dptr, sizeof(T) * v.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

// Tiles, groups, partial-slot bases and grids of the active systems (all systems unless the
// engine is a server's, whose membership changes between scheduling rounds).
void build_tiles(Engine& E) {
    E.sweep_tiles.clear();
    E.dtiles.clear();
    E.vtiles.clear();
    E.sweep_groups.clear();
    E.dgroups.clear();
    E.sweep_variant.assign(E.nsys, 0);
    auto active = [&](int s) { return E.active.empty() || E.active[s]; };
    for (int pass = 0; pass < 2; ++pass) {
        const int fp = pass == 0 ? E.fp32 : 0;
        auto& tiles = pass == 0 ? E.sweep_tiles : E.dtiles;
        auto& groups = pass == 0 ? E.sweep_groups : E.dgroups;
        for (int v = 0; v < 8; ++v) {
            Group g{v, (int)tiles.size(), 0, 1};
            for (int s = 0; s < E.nsys; ++s) {
                if (!active(s)) continue;
                SysDesc& S = E.sys[s];
                int cnt = 0;
                if (E.is_csr) {
                    if (v != 0) continue;
                    build_csr_tiles(s, S.n, tiles, &cnt);
                } else {
                    if (choose_variant(S, fp) != v) continue;
                    if (pass == 0) {
                        E.sweep_variant[s] = v;
                        // block Jacobi: 3 marks a system whose sweep (variants 6, 7) applies the
                        // boxes itself, so that k_block_apply (which takes block == 2 only) leaves
                        // it alone; 2 a system whose register sweep writes b - A x for k_block_apply
                        if (S.block >= 2) S.block = v >= 6 ? 3 : 2;
                    }
                    if (fp && v >= 4)
                        build_segment_tiles(s, S, stencil_variant_tx(fp, v), stencil_variant_ty(fp, v), E.radius,
                                            stencil_occupancy(E.radius, 1, SM_SWEEP, v) * E.sms, tiles, &cnt);
                    else
                        build_stencil_tiles(s, S, stencil_variant_tx(fp, v), stencil_variant_ty(fp, v), E.radius,
                                            E.sms, tiles, &cnt);
                }
                if (pass == 0) S.nop = cnt;
                else S.nopd = cnt;
            }
            g.count = (int)tiles.size() - g.offset;
            if (g.count > 0) groups.push_back(g);
        }
    }
    // partial-slot bases: each system's tiles are contiguous in its group
    std::vector<int> first_sweep(E.nsys, -1), first_d(E.nsys, -1);
    for (size_t i = 0; i < E.sweep_tiles.size(); ++i)
        if (first_sweep[E.sweep_tiles[i].sys] < 0) first_sweep[E.sweep_tiles[i].sys] = (int)i;
    for (size_t i = 0; i < E.dtiles.size(); ++i)
        if (first_d[E.dtiles[i].sys] < 0) first_d[E.dtiles[i].sys] = (int)i;
    const int nsweep = (int)E.sweep_tiles.size();
    int nvec_total = 0;
    for (int s = 0; s < E.nsys; ++s) {
        SysDesc& S = E.sys[s];
        if (!active(s)) {
            S.op0 = S.opd0 = S.vec0 = 0;
            S.nop = S.nopd = S.nvec = 0;
            continue;
        }
        S.op0 = first_sweep[s];
        S.opd0 = nsweep + first_d[s];
        int cnt = 0;
        S.vec0 = nvec_total;
        build_vec_tiles(s, S.n, E.sms, E.fp32 ? VEC_MIN_FP32 : 256, E.vtiles, &cnt);
        S.nvec = cnt;
        nvec_total += cnt;
    }
    for (auto* gl : {&E.sweep_groups, &E.dgroups}) {
        const bool sweep = gl == &E.sweep_groups;
        for (auto& g : *gl) {
            int occ = 8;
            if (!E.is_csr)
                occ = stencil_occupancy(E.radius, sweep ? E.fp32 : 0, sweep ? SM_SWEEP : SM_RESID, g.variant);
            g.grid = grid_for(g.count, occ, E.sms);
        }
    }
    E.vec_grid = grid_for((int)E.vtiles.size(), 2, E.sms);
}

// Device copies of the tile lists and partial-sum slots, grown when the lists outgrow them.
template <typename T>
cudaError_t upload_grow(T** dptr, size_t* cap, const std::vector<T>& v, cudaStream_t s) {
    if (v.size() > *cap || !*dptr) {
        cudaFree(*dptr);
        *dptr = nullptr;
        const size_t n = std::max<size_t>(v.size() + v.size() / 2, 64);
        cudaError_t e = cudaMalloc(dptr, sizeof(T) * n);
        if (e != cudaSuccess) return e;
        *cap = n;
    }
    if (v.empty()) return cudaSuccess;
    return cudaMemcpyAsync(*dptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s);
}

aar_status upload_tiles(Engine& E) {
    AAR_CHECK(upload_grow(&E.d_sweep_tiles, &E.cap_sweep, E.sweep_tiles, E.stream));
    AAR_CHECK(upload_grow(&E.d_dtiles, &E.cap_dtiles, E.dtiles, E.stream));
    AAR_CHECK(upload_grow(&E.d_vtiles, &E.cap_vtiles, E.vtiles, E.stream));
    const size_t ns = E.sweep_tiles.size() + E.dtiles.size() + 1, ng = (size_t)GSTRIDE * (E.vtiles.size() + 1);
    if (ns > E.cap_part_s) {
        cudaFree(E.d_part_s);
        E.d_part_s = nullptr;
        E.cap_part_s = ns + ns / 2;
        AAR_CHECK(cudaMalloc(&E.d_part_s, sizeof(double) * E.cap_part_s));
    }
    if (ng > E.cap_part_g) {
        cudaFree(E.d_part_g);
        E.d_part_g = nullptr;
        E.cap_part_g = ng + ng / 2;
        AAR_CHECK(cudaMalloc(&E.d_part_g, sizeof(double) * E.cap_part_g));
    }
    return AAR_OK;
}

aar_status alloc_tables(Engine& E) {
    int dev = 0;
    AAR_CHECK(cudaGetDevice(&dev));
    AAR_CHECK(cudaDeviceGetAttribute(&E.sms, cudaDevAttrMultiProcessorCount, dev));
    AAR_CHECK(cudaMalloc(&E.d_sys, sizeof(SysDesc) * E.nsys));
    AAR_CHECK(cudaMalloc(&E.d_st, sizeof(SysState) * E.nsys));
    AAR_CHECK(cudaMallocHost(&E.h_st, sizeof(SysState) * E.nsys));
    AAR_CHECK(cudaMalloc(&E.d_ctrl, sizeof(int) * 16));
    AAR_CHECK(cudaMallocHost(&E.h_ctrl, sizeof(int) * 16));
    AAR_CHECK(cudaMemset(E.d_ctrl, 0, sizeof(int) * 16));
    AAR_CHECK(cudaStreamCreateWithFlags(&E.cap_stream, cudaStreamNonBlocking));
    AAR_CHECK(cudaStreamCreateWithFlags(&E.cap_stream2, cudaStreamNonBlocking));
    E.slots_alloc.assign(E.nsys, 0);
    return AAR_OK;
}

// Build tiles, groups and device tables once the SysDesc geometry is filled in.
aar_status engine_setup(Engine& E) {
    AAR_CHECK(cudaGetDevice(&E.device));
    aar_status st = alloc_tables(E);
    if (st != AAR_OK) return st;
    build_tiles(E);
    st = upload_tiles(E);
    if (st != AAR_OK) return st;
    AAR_CHECK(cudaStreamSynchronize(E.stream));
    return AAR_OK;
}

using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
        cudaGetLastError();
    }
    return fn;
}

// One 3-D tensor map per X-ring slot of every system on a TMA sweep variant: dims (nx, ny, nz),
// box (32 + 2 * roundup4(r), TY + 2r, 1), zero fill outside the grid (the Dirichlet ghosts); then
// one for the FP32 inner right-hand side rhs32 (index nslots), box (64, TY, 1), which the paired
// sweep streams through its right-hand-side ring.
aar_status build_maps(Engine& E) {
    std::vector<CUtensorMap> maps;
    for (int s = 0; s < E.nsys; ++s) {
        SysDesc& S = E.sys[s];
        const int v = E.sweep_variant[s];
        S.map0 = 0;
        if (!E.fp32 || E.is_csr || v < 2 || v == 5 || v == 7) continue;  // 5 and 7 fill their stages themselves
        if (!E.active.empty() && !E.active[s]) continue;
        EncodeFn enc = encode_fn();
        if (!enc) return AAR_ERR_UNSUPPORTED;
        S.map0 = (int)maps.size();
        for (int k = 0; k < S.nslots; ++k) {
            CUtensorMap m;
            const cuuint64_t dims[3] = {(cuuint64_t)S.nx, (cuuint64_t)S.ny, (cuuint64_t)S.nz};
            const cuuint64_t strides[2] = {(cuuint64_t)S.nx * 4, (cuuint64_t)S.nx * S.ny * 4};
            const cuuint32_t box[3] = {(cuuint32_t)stencil_tma_box_x(E.radius, v),
                                       (cuuint32_t)(stencil_variant_ty(1, v) + 2 * E.radius), 1};
            const cuuint32_t estr[3] = {1, 1, 1};
            void* base = reinterpret_cast<float*>(S.X) + (size_t)k * S.ld;
            CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return AAR_ERR_UNSUPPORTED;
            maps.push_back(m);
        }
        {
            CUtensorMap m;
            const cuuint64_t dims[3] = {(cuuint64_t)S.nx, (cuuint64_t)S.ny, (cuuint64_t)S.nz};
            const cuuint64_t strides[2] = {(cuuint64_t)S.nx * 4, (cuuint64_t)S.nx * S.ny * 4};
            const cuuint32_t box[3] = {64u, (cuuint32_t)stencil_variant_ty(1, v), 1};
            const cuuint32_t estr[3] = {1, 1, 1};
            CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, S.rhs32, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return AAR_ERR_UNSUPPORTED;
            maps.push_back(m);
        }
    }
    if (maps.empty()) return AAR_OK;
    if (E.d_maps) {
        cudaFree(E.d_maps);
        E.d_maps = nullptr;
    }
    AAR_CHECK(cudaMalloc(&E.d_maps, sizeof(CUtensorMap) * maps.size()));
    AAR_CHECK(cudaMemcpy(E.d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
    return AAR_OK;
}

// (Re)allocate the rings so that system s holds nslots[s] slots; zero everything.
aar_status engine_alloc(Engine& E, const std::vector<int>& nslots) {
    bool ok = true;
    for (int s = 0; s < E.nsys; ++s) ok = ok && E.slots_alloc[s] >= nslots[s];
    if (ok && E.d_pool) return AAR_OK;
    const size_t w = E.fp32 ? 4 : 8;
    size_t total = 0;
    std::vector<size_t> off(E.nsys);
    for (int s = 0; s < E.nsys; ++s) {
        const SysDesc& S = E.sys[s];
        off[s] = total;
        total += 2 * (size_t)nslots[s] * S.ld * w;
        if (E.fp32) total += (size_t)S.ld * 8 + 3 * (size_t)S.ld * 4;  // x64, rhs32, xold, fold
        total = (size_t)round_up((int64_t)total, 256);
    }
    if (E.d_pool) {
        AAR_CHECK(cudaStreamSynchronize(E.stream));
        cudaFree(E.d_pool);
        E.d_pool = nullptr;
    }
    AAR_CHECK(cudaMalloc(&E.d_pool, total));
    AAR_CHECK(cudaMemsetAsync(E.d_pool, 0, total, E.stream));
    E.pool_bytes = total;
    for (int s = 0; s < E.nsys; ++s) {
        SysDesc& S = E.sys[s];
        char* base = reinterpret_cast<char*>(E.d_pool) + off[s];
        S.nslots = nslots[s];
        S.X = base;
        S.F = base + (size_t)nslots[s] * S.ld * w;
        if (E.fp32) {
            S.x64 = reinterpret_cast<double*>(base + 2 * (size_t)nslots[s] * S.ld * w);
            S.rhs32 = reinterpret_cast<float*>(reinterpret_cast<char*>(S.x64) + (size_t)S.ld * 8);
            S.xold = S.rhs32 + S.ld;
            S.fold = S.xold + S.ld;
        } else {
            S.x64 = nullptr;
            S.rhs32 = S.xold = S.fold = nullptr;
        }
        E.slots_alloc[s] = nslots[s];
    }
    return build_maps(E);
}

cudaError_t launch_resid_groups(Engine& E, cudaStream_t s) {
    if (!E.fp32) return cudaSuccess;
    const EngineView ev = E.view();
    for (const Group& g : E.dgroups) {
        OpLaunch L{E.d_dtiles + g.offset, g.count, g.grid, g.variant};
        cudaError_t e = E.is_csr ? launch_csr(0, SM_RESID, L, ev, 0, nullptr, nullptr, s)
                                 : launch_stencil(E.radius, 0, SM_RESID, L, ev, 0, nullptr, nullptr, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Block Jacobi after a register-fed sweep: whether any active system needs the k_block_apply pass
// (block Jacobi on a sweep variant that does not fuse it), and its grid: one CTA per 256 boxes of
// the largest such system, at most 8 per SM (the kernel takes the systems one after another).
int block_grid(const Engine& E) {
    int64_t nbox = 0;
    for (int s = 0; s < E.nsys; ++s) {
        if (!E.active.empty() && !E.active[s]) continue;
        const SysDesc& S = E.sys[s];
        if (S.block != 2 || E.is_csr) continue;  // 3: the sweep applies the boxes itself
        nbox = std::max<int64_t>(nbox, (int64_t)(S.nx / 2) * (S.ny / 2) * (S.nz / 2));
    }
    if (nbox == 0) return 0;
    return (int)std::max<int64_t>(1, std::min<int64_t>((nbox + 255) / 256, 8LL * E.sms));
}

cudaError_t launch_sweep_groups(Engine& E, cudaStream_t s, int j = 0) {
    const EngineView ev = E.view();
    for (const Group& g : E.sweep_groups) {
        OpLaunch L{E.d_sweep_tiles + g.offset, g.count, g.grid, g.variant, E.d_maps};
        cudaError_t e = E.is_csr ? launch_csr(E.fp32, SM_SWEEP, L, ev, j, nullptr, nullptr, s)
                                 : launch_stencil(E.radius, E.fp32, SM_SWEEP, L, ev, j, nullptr, nullptr, s);
        if (e != cudaSuccess) return e;
    }
    // block Jacobi: M^{-1} and the Richardson update after the sweep, for the systems whose sweep
    // variant does not fuse them (the paired sweeps 6, 7 do)
    if (!E.is_csr) {
        const int grid = block_grid(E);
        if (grid > 0) return launch_block_apply(E.fp32, ev, j, grid, s);
    }
    return cudaSuccess;
}

// The Anderson-step streams: bulk-TMA-fed passes for the FP32 inner solves, register-fed
// passes for the FP64 form (whose arithmetic, not bandwidth, bounds them).
cudaError_t launch_gram_any(Engine& E, int cmax, int j, cudaStream_t s) {
    const int nv = (int)E.vtiles.size();
    if (E.fp32) return launch_gram_bulk(cmax, E.d_vtiles, nv, E.vec_grid, E.view(), j, s);
    return launch_gram(cmax, E.d_vtiles, nv, E.vec_grid, E.view(), j, s);
}

cudaError_t launch_update_any(Engine& E, int cmax, cudaStream_t s) {
    const int nv = (int)E.vtiles.size();
    if (E.fp32) return launch_update_bulk(cmax, E.d_vtiles, nv, E.vec_grid, E.view(), s);
    return launch_update(cmax, E.d_vtiles, nv, E.vec_grid, E.view(), s);
}

// One full tick (j = 0, or TICK_FULL at the end of a body with Richardson-only ticks): every
// system advances by one step of its own phase machine. Launched directly (host loop, profiling)
// every kernel runs and the ones with nothing to do exit at once.
cudaError_t launch_tick(Engine& E, int cmax, cudaStream_t s, int j = 0) {
    const EngineView ev = E.view();
    cudaError_t e;
    if ((e = launch_resid_groups(E, s)) != cudaSuccess) return e;
    if ((e = launch_sweep_groups(E, s, j)) != cudaSuccess) return e;
    if ((e = launch_gram_any(E, cmax, j, s)) != cudaSuccess) return e;
    if ((e = launch_finalize(ev, j, s)) != cudaSuccess) return e;
    return launch_update_any(E, cmax, s);
}

// Richardson-only tick jr (1 .. p-1) of a body: the sweep alone, each system in an inner solve
// taking step k0 + jr - 1 when it is a Richardson step (see tick_step); no state changes.
cudaError_t launch_tick_r(Engine& E, int jr, cudaStream_t s) { return launch_sweep_groups(E, s, jr); }

// The Anderson period every active system shares (>= 2), else 0: the layout of the graph body.
int common_period(const Engine& E) {
    int p = 0;
    for (int s = 0; s < E.nsys; ++s) {
        if (!E.active.empty() && !E.active[s]) continue;
        if (p == 0) p = E.sys[s].p;
        else if (E.sys[s].p != p) return 0;
    }
    return p >= 2 ? p : 0;
}

bool debug_on() { return getenv("AAR_DEBUG") != nullptr; }

cudaError_t dbg(cudaError_t e, const char* what) {
    if (e != cudaSuccess && debug_on()) fprintf(stderr, "aar: %s failed: %s\n", what, cudaGetErrorString(e));
    return e;
}

// The WHILE body is assembled segment by segment: plain kernels are captured into it with an
// explicit dependency set (cudaStreamBeginCaptureToGraph), and each IF node is added between two
// captures, never while a capture into the body is active.
struct BodyBuilder {
    Engine& E;
    cudaGraph_t body;
    std::vector<cudaGraphNode_t> leaves;  // current dependency set of the next node

    template <typename Fn>
    cudaError_t capture(Fn fn) {
        cudaError_t e = dbg(cudaStreamBeginCaptureToGraph(E.cap_stream, body, leaves.empty() ? nullptr : leaves.data(),
                                                          nullptr, leaves.size(), cudaStreamCaptureModeRelaxed),
                            "cudaStreamBeginCaptureToGraph(segment)");
        if (e != cudaSuccess) return e;
        const cudaError_t e1 = dbg(fn(E.cap_stream), "segment launch");
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        const cudaError_t e3 = dbg(cudaStreamGetCaptureInfo(E.cap_stream, &cs, nullptr, nullptr, &deps, nullptr, &nd),
                                   "cudaStreamGetCaptureInfo");
        std::vector<cudaGraphNode_t> next;
        if (e3 == cudaSuccess && deps) next.assign(deps, deps + nd);
        cudaGraph_t tmp = nullptr;
        const cudaError_t e2 = dbg(cudaStreamEndCapture(E.cap_stream, &tmp), "cudaStreamEndCapture(segment)");
        if (e1 != cudaSuccess) return e1;
        if (e3 != cudaSuccess) return e3;
        if (e2 != cudaSuccess) return e2;
        leaves.swap(next);
        return cudaSuccess;
    }

    template <typename Fn>
    cudaError_t if_node(cudaGraphConditionalHandle h, Fn fn) {
        cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeIf;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        cudaError_t e = dbg(cudaGraphAddNode(&node, body, leaves.empty() ? nullptr : leaves.data(), nullptr,
                                             leaves.size(), &p),
                            "cudaGraphAddNode(IF)");
        if (e != cudaSuccess) return e;
        e = dbg(cudaStreamBeginCaptureToGraph(E.cap_stream, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed),
                "cudaStreamBeginCaptureToGraph(IF body)");
        if (e != cudaSuccess) return e;
        const cudaError_t e1 = dbg(fn(E.cap_stream), "IF body launch");
        cudaGraph_t tmp = nullptr;
        const cudaError_t e2 = dbg(cudaStreamEndCapture(E.cap_stream, &tmp), "cudaStreamEndCapture(IF body)");
        if (e1 != cudaSuccess) return e1;
        if (e2 != cudaSuccess) return e2;
        leaves.assign(1, node);
        return cudaSuccess;
    }
};

// One tick inside the solve graph: the FP64 residual, Gram and update passes sit in IF nodes
// whose conditions the finalize of the previous (resp. same) tick sets, so a Richardson tick
// launches only the sweep and the finalize.
cudaError_t build_tick_if(BodyBuilder& B, int cmax, const cudaGraphConditionalHandle* h) {
    Engine& E = B.E;
    const EngineView ev = E.view();
    const int nv = (int)E.vtiles.size();
    cudaError_t e;
    if (E.fp32 && (e = B.if_node(h[0], [&](cudaStream_t s) { return launch_resid_groups(E, s); })) != cudaSuccess)
        return e;
    if ((e = B.capture([&](cudaStream_t s) { return launch_sweep_groups(E, s); })) != cudaSuccess) return e;
    if ((e = B.if_node(h[1], [&](cudaStream_t s) { return launch_gram_any(E, cmax, 0, s); })) != cudaSuccess)
        return e;
    FinConds fc{1, E.d_ctrl + 7, h[0], h[1], h[2]};
    if ((e = B.capture([&](cudaStream_t s) { return launch_finalize(ev, 0, s, fc); })) != cudaSuccess) return e;
    return B.if_node(h[2], [&](cudaStream_t s) { return launch_update_any(E, cmax, s); });
}

// Solve-graph variants: 0 = plain ticks; 1..3 = IF-gated ticks with the IF handles created on
// the top-level graph with a default of 1 (1), on the WHILE body without a default plus a
// prelude kernel that sets them to 1 at the start of every body pass (2), or on the top-level
// graph the same way (3). The first variant the runtime accepts is kept.
aar_status build_graph(Engine& E, int cmax, int mode) {
    const int period = mode == 0 ? common_period(E) : 0;
    if (E.exec && E.graph_cmax == cmax && E.graph_period == period) return AAR_OK;
    if (E.exec) {
        cudaGraphExecDestroy(E.exec);
        E.exec = nullptr;
    }
    if (E.graph) {
        cudaGraphDestroy(E.graph);
        E.graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h, hif[3] = {0, 0, 0};
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return AAR_ERR_CUDA;
    auto fail = [&]() {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return AAR_ERR_UNSUPPORTED;
    };
    if (dbg(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault), "handle(WHILE)") != cudaSuccess)
        return fail();
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) return fail();
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (mode > 0) {
        cudaGraph_t owner = mode == 2 ? body : g;
        const unsigned flags = mode == 1 ? cudaGraphCondAssignDefault : 0u;
        for (int i = 0; i < 3; ++i)
            if (dbg(cudaGraphConditionalHandleCreate(&hif[i], owner, 1, flags), "handle(IF)") != cudaSuccess)
                return fail();
        BodyBuilder B{E, body, {}};
        cudaError_t err = cudaSuccess;
        if (mode >= 2) err = B.capture([&](cudaStream_t s) { return launch_set_conds(hif, 3, s); });
        for (int t = 0; t < TICKS && err == cudaSuccess; ++t) err = build_tick_if(B, cmax, hif);
        if (err == cudaSuccess)
            err = B.capture([&](cudaStream_t s) { return launch_control(E.view(), E.d_ctrl, h, TICKS, s); });
        if (err != cudaSuccess) return fail();
    } else {
        if (cudaStreamBeginCaptureToGraph(E.cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
            cudaSuccess)
            return fail();
        cudaError_t err = cudaSuccess;
        int nt = 0;
        if (period > 0) {
            // (period - 1) Richardson-only ticks and one full tick, repeated to about TICKS ticks
            const int reps = std::max(1, TICKS / period);
            for (int r = 0; r < reps && err == cudaSuccess; ++r) {
                for (int t = 0; t < period - 1 && err == cudaSuccess; ++t) err = launch_tick_r(E, t + 1, E.cap_stream);
                if (err == cudaSuccess) err = launch_tick(E, cmax, E.cap_stream, TICK_FULL);
            }
            nt = reps * period;
        } else {
            for (int t = 0; t < TICKS && err == cudaSuccess; ++t) err = launch_tick(E, cmax, E.cap_stream);
            nt = TICKS;
        }
        if (err == cudaSuccess) err = launch_control(E.view(), E.d_ctrl, h, nt, E.cap_stream);
        cudaGraph_t captured = nullptr;
        cudaError_t e2 = dbg(cudaStreamEndCapture(E.cap_stream, &captured), "cudaStreamEndCapture(body)");
        if (err != cudaSuccess || e2 != cudaSuccess) return fail();
    }
    cudaGraphExec_t ex = nullptr;
    if (dbg(cudaGraphInstantiate(&ex, g, 0), "cudaGraphInstantiate") != cudaSuccess) return fail();
    E.graph = g;
    E.exec = ex;
    E.graph_cmax = cmax;
    E.graph_mode = mode;
    E.graph_period = period;
    if (debug_on()) fprintf(stderr, "aar: solve graph built, mode %d (0 = plain ticks, >0 = IF-gated)\n", mode);
    return AAR_OK;
}

bool valid_params(const aar_params* p) {
    if (!p) return false;
    if (p->m < 0 || p->m > AAR_MAX_M || p->p < 1 || !(p->tol >= 0.0) || p->max_iter < 0) return false;
    if (!isfinite(p->omega) || !isfinite(p->beta) || !isfinite(p->tol)) return false;
    if (!(p->inner_tol > 0.0 && p->inner_tol < 1.0) || p->max_refine < 1) return false;
    if (p->flags & ~AAR_FLAG_RESTART_HISTORY) return false;
    if (p->step_limit < 0) return false;
    return true;
}

// Run the solve loop for all systems whose descriptors/state have been staged on the device.
aar_status engine_run(Engine& E, int cmax, int64_t step_limit) {
    const EngineView ev = E.view();
    E.h_ctrl[0] = 0;
    E.h_ctrl[1] = (int)std::min<int64_t>(step_limit, 2000000000);
    E.h_ctrl[2] = 1;
    for (int i = 3; i < 16; ++i) E.h_ctrl[i] = 0;
    AAR_CHECK(cudaMemcpyAsync(E.d_ctrl, E.h_ctrl, sizeof(int) * 16, cudaMemcpyHostToDevice, E.stream));
    // INIT: ||b||^2 partial sums, then the finalize turns them into ||b|| and picks the phase
    AAR_CHECK(launch_norm_b(E.d_vtiles, (int)E.vtiles.size(), E.vec_grid, ev, E.stream));
    AAR_CHECK(launch_finalize(ev, 0, E.stream));
    if (getenv("AAR_HOST_LOOP")) E.graph_failed = true;
    if (!E.graph_failed) {
        // IF-gated ticks first; plain graph ticks if conditional IF nodes cannot be built
        aar_status gs = AAR_ERR_UNSUPPORTED;
        if (E.graph_mode > 0 || E.graph_mode < 0)
            for (int mode = (E.graph_mode > 0 ? E.graph_mode : 1); mode <= 3 && gs != AAR_OK; ++mode)
                gs = build_graph(E, cmax, mode);
        if (gs != AAR_OK) gs = build_graph(E, cmax, 0);
        if (gs != AAR_OK) E.graph_failed = true;
    }
    if (!E.graph_failed) {
        AAR_CHECK(cudaGraphLaunch(E.exec, E.stream));
        AAR_CHECK(wait_stream(E.stream));
    } else {
        // host-driven loop: the graph body's ticks, then read the control word
        const int period = common_period(E);
        const int reps = period > 0 ? std::max(1, TICKS / period) : 0;
        const int nt = period > 0 ? reps * period : TICKS;
        for (;;) {
            for (int t = 0; t < nt; ++t) {
                const bool full = period == 0 || t % period == period - 1;
                AAR_CHECK(full ? launch_tick(E, cmax, E.stream, period > 0 ? TICK_FULL : 0)
                               : launch_tick_r(E, t % period + 1, E.stream));
            }
            AAR_CHECK(launch_control(ev, E.d_ctrl, 0, nt, E.stream));
            AAR_CHECK(cudaMemcpyAsync(E.h_ctrl + 2, E.d_ctrl + 2, sizeof(int), cudaMemcpyDeviceToHost, E.stream));
            AAR_CHECK(cudaStreamSynchronize(E.stream));
            if (!E.h_ctrl[2]) break;
        }
    }
    AAR_CHECK(cudaMemcpyAsync(E.h_st, E.d_st, sizeof(SysState) * E.nsys, cudaMemcpyDeviceToHost, E.stream));
    AAR_CHECK(cudaMemcpyAsync(E.h_ctrl, E.d_ctrl, sizeof(int) * 16, cudaMemcpyDeviceToHost, E.stream));
    AAR_CHECK(cudaStreamSynchronize(E.stream));
    E.last_ticks = E.h_ctrl[0];
    E.last_launches = E.h_ctrl[8];
    if (E.h_ctrl[3]) {  // a bounded device wait gave up: results are not trustworthy
        for (int s = 0; s < E.nsys; ++s) E.h_st[s].status = AAR_ERR_TIMEOUT;
        if (getenv("AAR_DEBUG"))
            fprintf(stderr, "aar: device wait gave up: plane %d parity %d barrier 0x%x\n", E.h_ctrl[4], E.h_ctrl[5],
                    (unsigned)E.h_ctrl[6]);
    }
    E.last_cmax = cmax;
    E.solved = true;
    return AAR_OK;
}

void init_state(SysState& st) {
    memset(&st, 0, sizeof(st));
    st.split_k = -1;  // k_zero = 0: x_0 = 0
    st.phase = PH_INIT;
    st.status = AAR_NOT_CONVERGED;
    st.k_final = 0;
    st.r_last = NAN;
}

void set_params(SysDesc& S, const aar_params* p) {
    S.omega = p->omega;
    S.beta = p->beta;
    S.m = p->m;
    S.p = p->p;
    S.tol = p->tol;
    S.max_iter = p->max_iter;
    S.inner_tol = p->inner_tol;
    S.max_refine = p->max_refine;
    S.restart_history = (p->flags & AAR_FLAG_RESTART_HISTORY) ? 1 : 0;
}

int64_t step_limit_for(const aar_params* p, int mixed) {
    // every full tick advances each unfinished system by one iteration or one refinement step; in
    // a periodic body a system may wait up to p - 1 Richardson-only ticks for a full tick at each
    // change of phase or of step alignment (a few per refinement)
    const int64_t wait = p->p >= 2 ? (int64_t)p->p : 0;
    if (p->step_limit > 0) return p->step_limit;  // the caller's own watchdog
    return p->max_iter + (mixed ? (3 + 3 * wait) * ((int64_t)p->max_refine + 2) : 2 * wait) + 4 * TICKS + 16 + wait;
}

void fill_info(const SysState& st, aar_info* info, const Engine& E) {
    if (!info) return;
    info->ticks = E.last_ticks;
    info->launches = E.last_launches;
    info->iterations = st.iters_total;
    info->anderson_steps = st.anderson;
    info->refinements = st.refinements;
    info->rel_residual = st.r_last;
    info->status = st.status;
    info->last_rank = st.last_rank;
    info->eigen_steps = st.n_eig;
    info->reserved = 0;
}

// Stencil geometry and coefficients into a SysDesc; returns false on an invalid descriptor.
bool stencil_desc(const aar_stencil_desc* d, SysDesc& S) {
    if (!d || d->nx <= 0 || d->ny <= 0 || d->nz <= 0 || d->radius < 1 || d->radius > AAR_MAX_RADIUS) return false;
    if (!(d->h > 0.0) || !isfinite(d->h) || !(d->shift >= 0.0) || !isfinite(d->shift)) return false;
    if ((int64_t)d->nx * d->ny >= (int64_t)1 << 31) return false;
    if (d->periodic != 0 && d->periodic != 1) return false;
    for (int k = 0; k <= d->radius; ++k)
        if (!isfinite(d->w[k])) return false;
    memset(&S, 0, sizeof(S));
    S.periodic = d->periodic;
    S.radius = d->radius;
    S.nx = d->nx;
    S.ny = d->ny;
    S.nz = d->nz;
    S.n = (int64_t)d->nx * d->ny * d->nz;
    S.ld = round_up(S.n, PAD);
    const double ih2 = 1.0 / (d->h * d->h);
    S.cdiag = -3.0 * d->w[0] * ih2 + d->shift;
    for (int k = 1; k <= AAR_MAX_RADIUS; ++k) S.coff[k] = k <= d->radius ? -d->w[k] * ih2 : 0.0;
    if (!(S.cdiag > 0.0) || !isfinite(S.cdiag)) return false;
    S.cdiag_f = (float)S.cdiag;
    for (int k = 0; k <= AAR_MAX_RADIUS; ++k) S.coff_f[k] = (float)S.coff[k];
    S.dinv = 1.0 / S.cdiag;
    S.dinv_f = (float)S.dinv;
    // block Jacobi with 2 x 2 x 2 boxes: every block is cdiag I + coff[1] Q3 when a periodic side
    // is at least radius + 2 (no other tap wraps into the box); its eigenvalues
    // cdiag + coff[1] (3 - 2t), t = 0..3, must be nonzero
    if (d->block != 0 && d->block != 1 && d->block != 2) return false;
    S.block = d->block == 2 ? 2 : 0;
    if (S.block == 2) {
        if (d->nx % 2 || d->ny % 2 || d->nz % 2) return false;
        if (d->periodic && (d->nx < d->radius + 2 || d->ny < d->radius + 2 || d->nz < d->radius + 2)) return false;
        for (int t = 0; t < 4; ++t) {
            const double lam = S.cdiag + S.coff[1] * (3.0 - 2.0 * t);
            if (!(lam != 0.0) || !isfinite(lam)) return false;
            S.bl_mu[t] = 1.0 / (8.0 * lam);
            S.bl_mu_f[t] = (float)S.bl_mu[t];
            if (!isfinite(S.bl_mu[t])) return false;
        }
    }
    S.hint_variant = d->tile_variant;
    S.hint_zc = d->tile_zc;
    return true;
}

}  // namespace

// =============================================================================== C ABI

struct aar_ctx {
    Engine E;
    int precision = AAR_FP64;
};

struct aar_batch_ctx {
    Engine E;
    int precision = AAR_FP64;
};

extern "C" {

aar_status aar_default_params(aar_params* p) {
    if (!p) return AAR_ERR_INVALID_ARG;
    memset(p, 0, sizeof(*p));
    p->omega = 0.6;
    p->beta = 0.6;
    p->m = 9;
    p->p = 8;
    p->tol = 1e-8;
    p->max_iter = 100000;
    p->inner_tol = 0.1;
    p->max_refine = 30;
    return AAR_OK;
}

const char* aar_status_string(aar_status s) {
    switch (s) {
        case AAR_OK: return "converged";
        case AAR_NOT_CONVERGED: return "iteration limit reached before the tolerance";
        case AAR_ERR_INVALID_ARG: return "invalid argument";
        case AAR_ERR_OOM: return "device memory allocation failed";
        case AAR_ERR_CUDA: return "CUDA runtime error";
        case AAR_ERR_BREAKDOWN: return "breakdown: non-finite residual or extrapolation coefficients";
        case AAR_ERR_TIMEOUT: return "device step limit exhausted or a bounded device wait gave up";
        case AAR_ERR_UNSUPPORTED: return "unsupported configuration";
        case AAR_ERR_COMM: return "a communication callback failed";
    }
    return "unknown status";
}

aar_status aar_create_stencil(const aar_stencil_desc* desc, const double* dinv, int32_t precision, void* stream,
                              aar_handle* out) {
    if (!out) return AAR_ERR_INVALID_ARG;
    *out = nullptr;
    if (precision != AAR_FP64 && precision != AAR_MIXED) return AAR_ERR_INVALID_ARG;
    SysDesc S;
    if (!stencil_desc(desc, S)) return AAR_ERR_INVALID_ARG;
    if (dinv && !is_device_ptr(dinv)) return AAR_ERR_INVALID_ARG;
    if (dinv && S.block == 2) return AAR_ERR_INVALID_ARG;  // one preconditioner at a time
    aar_ctx* h = new (std::nothrow) aar_ctx;
    if (!h) return AAR_ERR_OOM;
    h->precision = precision;
    Engine& E = h->E;
    E.nsys = 1;
    E.fp32 = precision == AAR_MIXED;
    E.radius = desc->radius;
    E.stream = (cudaStream_t)stream;
    S.mixed = E.fp32;
    E.sys.push_back(S);
    aar_status st = engine_setup(E);
    if (st == AAR_OK && dinv) {
        E.sys[0].dinv_vec = dinv;
        if (E.fp32) {
            if (cudaMalloc(&E.d_dinv32, sizeof(float) * E.sys[0].ld) != cudaSuccess ||
                launch_to_f32(dinv, E.d_dinv32, E.sys[0].n, E.stream) != cudaSuccess)
                st = AAR_ERR_CUDA;
            E.sys[0].dinv_vec32 = E.d_dinv32;
        }
    }
    if (st != AAR_OK) {
        delete h;
        return st;
    }
    *out = h;
    return AAR_OK;
}

aar_status aar_create_csr(const aar_csr_desc* desc, const double* dinv, int32_t precision, void* stream,
                          aar_handle* out) {
    if (!out) return AAR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!desc || desc->n <= 0 || desc->nnz < 0 || !desc->row_ptr || !desc->col_idx || !desc->val)
        return AAR_ERR_INVALID_ARG;
    if (precision != AAR_FP64 && precision != AAR_MIXED) return AAR_ERR_INVALID_ARG;
    if (desc->nnz > INT32_MAX) return AAR_ERR_UNSUPPORTED;
    if (!is_device_ptr(desc->row_ptr) || !is_device_ptr(desc->col_idx) || !is_device_ptr(desc->val))
        return AAR_ERR_INVALID_ARG;
    if (dinv && !is_device_ptr(dinv)) return AAR_ERR_INVALID_ARG;
    aar_ctx* h = new (std::nothrow) aar_ctx;
    if (!h) return AAR_ERR_OOM;
    h->precision = precision;
    Engine& E = h->E;
    E.nsys = 1;
    E.fp32 = precision == AAR_MIXED;
    E.is_csr = 1;
    E.stream = (cudaStream_t)stream;
    SysDesc S;
    memset(&S, 0, sizeof(S));
    S.is_csr = 1;
    S.n = desc->n;
    S.nx = desc->n;
    S.ny = S.nz = 1;
    S.ld = round_up(S.n, PAD);
    S.row_ptr = desc->row_ptr;
    S.col_idx = desc->col_idx;
    S.val = desc->val;
    S.mixed = E.fp32;
    E.sys.push_back(S);
    aar_status st = engine_setup(E);
    int* d_bad = nullptr;
    if (st == AAR_OK) {
        SysDesc& T = E.sys[0];
        bool ok = true;
        if (!dinv) ok = ok && cudaMalloc(&E.d_dinv_own, sizeof(double) * T.ld) == cudaSuccess;
        if (E.fp32) {
            ok = ok && cudaMalloc(&E.d_dinv32, sizeof(float) * T.ld) == cudaSuccess;
            ok = ok && cudaMalloc(&E.d_val32, sizeof(float) * (desc->nnz + 1)) == cudaSuccess;
        }
        ok = ok && cudaMalloc(&d_bad, sizeof(int)) == cudaSuccess;
        ok = ok && cudaMemsetAsync(d_bad, 0, sizeof(int), E.stream) == cudaSuccess;
        if (ok) {
            // the structural check always runs; the diagonal is extracted only when derived
            ok = launch_csr_diag(desc->n, desc->row_ptr, desc->col_idx, desc->val, dinv ? nullptr : E.d_dinv_own,
                                 (dinv || !E.fp32) ? nullptr : E.d_dinv32, E.fp32 ? E.d_val32 : nullptr, desc->nnz,
                                 d_bad, E.stream) == cudaSuccess;
            if (ok && dinv && E.fp32) ok = launch_to_f32(dinv, E.d_dinv32, desc->n, E.stream) == cudaSuccess;
        }
        int bad = 0;
        if (ok) ok = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, E.stream) == cudaSuccess;
        if (ok) ok = cudaStreamSynchronize(E.stream) == cudaSuccess;
        if (!ok) st = AAR_ERR_CUDA;
        else if (bad) st = AAR_ERR_INVALID_ARG;
        T.dinv_vec = dinv ? dinv : E.d_dinv_own;
        T.dinv_vec32 = E.d_dinv32;
        T.val32 = E.d_val32;
    }
    cudaFree(d_bad);
    if (st != AAR_OK) {
        delete h;
        return st;
    }
    *out = h;
    return AAR_OK;
}

aar_status aar_solve(aar_handle h, const double* b, const double* x0, double* x, const aar_params* params,
                     aar_info* info) {
    if (info) {
        memset(info, 0, sizeof(*info));
        info->rel_residual = NAN;
    }
    if (!h || !b || !x || !valid_params(params)) {
        if (info) info->status = AAR_ERR_INVALID_ARG;
        return AAR_ERR_INVALID_ARG;
    }
    Engine& E = h->E;
    SysDesc& S = E.sys[0];
    aar_status st = engine_alloc(E, std::vector<int>{std::max(params->m + 1, 2)});
    if (st != AAR_OK) return st;
    set_params(S, params);
    // right-hand side: device pointer used in place, host memory staged
    if (is_device_ptr(b)) {
        S.b64 = b;
    } else {
        if (!E.d_bstage) AAR_CHECK(cudaMalloc(&E.d_bstage, sizeof(double) * S.ld));
        AAR_CHECK(cudaMemcpyAsync(E.d_bstage, b, sizeof(double) * S.n, cudaMemcpyHostToDevice, E.stream));
        S.b64 = E.d_bstage;
    }
    // initial iterate
    void* xdst = E.fp32 ? (void*)S.x64 : S.X;
    if (x0) AAR_CHECK(cudaMemcpyAsync(xdst, x0, sizeof(double) * S.n, cudaMemcpyDefault, E.stream));
    else AAR_CHECK(cudaMemsetAsync(xdst, 0, sizeof(double) * S.n, E.stream));
    SysState init;
    init_state(init);
    *E.h_st = init;
    AAR_CHECK(cudaMemcpyAsync(E.d_sys, &S, sizeof(SysDesc), cudaMemcpyHostToDevice, E.stream));
    AAR_CHECK(cudaMemcpyAsync(E.d_st, E.h_st, sizeof(SysState), cudaMemcpyHostToDevice, E.stream));
    st = engine_run(E, cmax_for(params->m), step_limit_for(params, E.fp32));
    if (st != AAR_OK) return st;
    const SysState& R = *E.h_st;
    if (R.k_final < 0) {
        if (is_device_ptr(x)) AAR_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * S.n, E.stream));
        else memset(x, 0, sizeof(double) * S.n);
    } else {
        const void* src = E.fp32 ? (const void*)S.x64
                                 : (const void*)((const double*)S.X + ring_slot(R.k_final, S.nslots) * S.ld);
        AAR_CHECK(cudaMemcpyAsync(x, src, sizeof(double) * S.n, cudaMemcpyDefault, E.stream));
    }
    AAR_CHECK(cudaStreamSynchronize(E.stream));
    fill_info(R, info, E);
    return (aar_status)R.status;
}

aar_status aar_apply(aar_handle h, const double* x, double* y) {
    if (!h || !x || !y || x == y) return AAR_ERR_INVALID_ARG;
    Engine& E = h->E;
    if (!is_device_ptr(x) || !is_device_ptr(y)) return AAR_ERR_INVALID_ARG;
    const EngineView ev = E.view();
    AAR_CHECK(cudaMemcpyAsync(E.d_sys, E.sys.data(), sizeof(SysDesc), cudaMemcpyHostToDevice, E.stream));
    for (const Group& g : E.dgroups) {
        OpLaunch L{E.d_dtiles + g.offset, g.count, g.grid, g.variant};
        cudaError_t e = E.is_csr ? launch_csr(0, SM_APPLY, L, ev, 0, x, y, E.stream)
                                 : launch_stencil(E.radius, 0, SM_APPLY, L, ev, 0, x, y, E.stream);
        if (e != cudaSuccess) return fail_cuda(e);
    }
    AAR_CHECK(cudaStreamSynchronize(E.stream));
    return AAR_OK;
}

aar_status aar_rel_residual(aar_handle h, const double* b, const double* x, double* rel) {
    if (!h || !b || !x || !rel) return AAR_ERR_INVALID_ARG;
    Engine& E = h->E;
    const SysDesc& S = E.sys[0];
    if (!is_device_ptr(b) || !is_device_ptr(x)) return AAR_ERR_INVALID_ARG;
    const int np = 512;
    double* y = nullptr;
    double* parts = nullptr;
    if (cudaMalloc(&y, sizeof(double) * S.n) != cudaSuccess ||
        cudaMalloc(&parts, sizeof(double) * (2 * np + 1)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(y);
        cudaFree(parts);
        return AAR_ERR_OOM;
    }
    aar_status st = aar_apply(h, x, y);
    if (st == AAR_OK) {
        if (launch_resid_norm(b, y, S.n, parts, np, parts + 2 * np, E.stream) != cudaSuccess ||
            cudaMemcpyAsync(rel, parts + 2 * np, sizeof(double), cudaMemcpyDeviceToHost, E.stream) != cudaSuccess ||
            cudaStreamSynchronize(E.stream) != cudaSuccess)
            st = AAR_ERR_CUDA;
    }
    cudaFree(y);
    cudaFree(parts);
    return st;
}

aar_status aar_profile_kernel(aar_handle h, int32_t kernel, int32_t launches, float* ms) {
    if (!h || !ms || launches < 1 || kernel < AAR_K_SWEEP || kernel > AAR_K_BLOCK) return AAR_ERR_INVALID_ARG;
    Engine& E = h->E;
    if (!E.solved) return AAR_ERR_INVALID_ARG;
    const SysDesc& S = E.sys[0];
    SysState st;
    init_state(st);
    st.phase = PH_INNER;
    st.kcap = INT64_MAX / 2;
    st.nb = st.nrhs = 1.0;
    // an Anderson step with a full history: smallest k >= max(m, 1) with (k+1) mod p == 0
    int64_t ka = std::max<int64_t>(S.m, 1);
    while ((ka + 1) % S.p != 0) ++ka;
    if (kernel == AAR_K_BLOCK && block_grid(E) == 0) return AAR_ERR_UNSUPPORTED;
    if (kernel == AAR_K_SWEEP || kernel == AAR_K_BLOCK) {
        int64_t k = 1;
        while ((k + 1) % S.p == 0 && k < 4 * (int64_t)S.p) ++k;
        if ((k + 1) % S.p == 0) return AAR_ERR_UNSUPPORTED;
        st.k0 = k;
    } else if (kernel == AAR_K_SWEEP_ANDERSON || kernel == AAR_K_GRAM) {
        st.k0 = ka;
    } else if (kernel == AAR_K_UPDATE) {
        // the form the solve uses: literal (Eq. 3) in FP64, compressed for FP32 inner solves
        st.upd = UPD_ANDERSON;
        st.upd_k = ka;
        st.upd_c = (int)std::min<int64_t>(ka, S.m);
        for (int a = 0; a < MAXM; ++a) st.gamma[a] = 1e-3 * (a + 1);
        if (E.fp32) {
            const int c = st.upd_c;
            for (int b = 0; b <= c; ++b) st.alpha[b] = 1e-3 * (b + 1);
            int na = 0;
            for (int a = 0; a < c; ++a) {
                const int64_t jj = ka - c + 1 + a;
                if (jj % S.p == 0 && na < NAMAX) {
                    st.aj[na] = jj;
                    st.ag[na] = 1e-3;
                    ++na;
                }
            }
            st.na = na;
            st.upd = UPD_ANDERSON_C;
        }
        st.phase = PH_DONE;
    } else if (kernel == AAR_K_FINALIZE) {
        // an Anderson step with a full history that goes on (the residual norm is far above any
        // stopping target), so the launch runs the m x m solve; partial sums from the last solve
        st.k0 = ka;
        st.nb = st.nrhs = 1e-300;
        st.r_last = st.r_inner = 1.0;
        for (int i = 0; i < STAG_WINDOW; ++i) st.rin_hist[i] = 1.0;
    } else {
        if (!E.fp32) return AAR_ERR_UNSUPPORTED;
        st.phase = PH_RESID;
    }
    *E.h_st = st;
    if (kernel == AAR_K_FINALIZE) {
        // the finalize advances the state: re-stage it before every launch, and subtract the cost
        // of the re-staging copies measured alone
        if (E.nsys != 1) return AAR_ERR_UNSUPPORTED;
        // fill the Gram partial sums once from the current history
        AAR_CHECK(cudaMemcpyAsync(E.d_st, E.h_st, sizeof(SysState), cudaMemcpyHostToDevice, E.stream));
        AAR_CHECK(launch_gram_any(E, E.last_cmax, 0, E.stream));
        for (const Group& g : E.sweep_groups) {
            OpLaunch L{E.d_sweep_tiles + g.offset, g.count, g.grid, g.variant, E.d_maps};
            cudaError_t e = E.is_csr ? launch_csr(E.fp32, SM_SWEEP, L, E.view(), 0, nullptr, nullptr, E.stream)
                                     : launch_stencil(E.radius, E.fp32, SM_SWEEP, L, E.view(), 0, nullptr, nullptr,
                                                      E.stream);
            if (e != cudaSuccess) return fail_cuda(e);
        }
        cudaEvent_t a0, a1, b1;
        AAR_CHECK(cudaEventCreate(&a0));
        AAR_CHECK(cudaEventCreate(&a1));
        AAR_CHECK(cudaEventCreate(&b1));
        AAR_CHECK(cudaEventRecord(a0, E.stream));
        for (int i = 0; i < launches; ++i)
            AAR_CHECK(cudaMemcpyAsync(E.d_st, E.h_st, sizeof(SysState), cudaMemcpyHostToDevice, E.stream));
        AAR_CHECK(cudaEventRecord(a1, E.stream));
        for (int i = 0; i < launches; ++i) {
            AAR_CHECK(cudaMemcpyAsync(E.d_st, E.h_st, sizeof(SysState), cudaMemcpyHostToDevice, E.stream));
            AAR_CHECK(launch_finalize(E.view(), 0, E.stream));
        }
        AAR_CHECK(cudaEventRecord(b1, E.stream));
        AAR_CHECK(cudaEventSynchronize(b1));
        float tc = 0.f, tb = 0.f;
        cudaEventElapsedTime(&tc, a0, a1);
        cudaEventElapsedTime(&tb, a1, b1);
        cudaEventDestroy(a0);
        cudaEventDestroy(a1);
        cudaEventDestroy(b1);
        *ms = (tb - tc) / launches;
        return AAR_OK;
    }
    AAR_CHECK(cudaMemcpyAsync(E.d_st, E.h_st, sizeof(SysState), cudaMemcpyHostToDevice, E.stream));
    cudaEvent_t e0, e1;
    AAR_CHECK(cudaEventCreate(&e0));
    AAR_CHECK(cudaEventCreate(&e1));
    const EngineView ev = E.view();
    const int nv = (int)E.vtiles.size();
    cudaError_t err = cudaEventRecord(e0, E.stream);
    for (int i = 0; i < launches && err == cudaSuccess; ++i) {
        if (kernel == AAR_K_SWEEP || kernel == AAR_K_SWEEP_ANDERSON) {
            for (const Group& g : E.sweep_groups) {
                OpLaunch L{E.d_sweep_tiles + g.offset, g.count, g.grid, g.variant, E.d_maps};
                err = E.is_csr ? launch_csr(E.fp32, SM_SWEEP, L, ev, 0, nullptr, nullptr, E.stream)
                               : launch_stencil(E.radius, E.fp32, SM_SWEEP, L, ev, 0, nullptr, nullptr, E.stream);
            }
        } else if (kernel == AAR_K_BLOCK) {
            err = launch_block_apply(E.fp32, ev, 0, block_grid(E), E.stream);
        } else if (kernel == AAR_K_GRAM) {
            err = launch_gram_any(E, E.last_cmax, 0, E.stream);
        } else if (kernel == AAR_K_UPDATE) {
            err = launch_update_any(E, E.last_cmax, E.stream);
        } else {
            for (const Group& g : E.dgroups) {
                OpLaunch L{E.d_dtiles + g.offset, g.count, g.grid, g.variant};
                err = E.is_csr ? launch_csr(0, SM_RESID, L, ev, 0, nullptr, nullptr, E.stream)
                               : launch_stencil(E.radius, 0, SM_RESID, L, ev, 0, nullptr, nullptr, E.stream);
            }
        }
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, E.stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return fail_cuda(err);
    *ms = t / launches;
    return AAR_OK;
}

aar_status aar_tune_stencil(const aar_stencil_desc* desc, int32_t precision, int32_t m, void* stream,
                            int32_t* tile_variant, int32_t* tile_zc, float* ms) {
    if (!desc || !tile_variant || !tile_zc || !ms || m < 0 || m > AAR_MAX_M) return AAR_ERR_INVALID_ARG;
    if (precision != AAR_FP64 && precision != AAR_MIXED) return AAR_ERR_INVALID_ARG;
    SysDesc probe;
    if (!stencil_desc(desc, probe)) return AAR_ERR_INVALID_ARG;
    const int fp32 = precision == AAR_MIXED;
    const int64_t n = probe.n;
    double* b = nullptr;
    double* x = nullptr;
    if (cudaMalloc(&b, sizeof(double) * n) != cudaSuccess || cudaMalloc(&x, sizeof(double) * n) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b);
        cudaFree(x);
        return AAR_ERR_OOM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // a smooth right-hand side: every candidate sees the same data
    aar_status st = AAR_OK;
    if (cudaMemsetAsync(b, 0, sizeof(double) * n, s) != cudaSuccess) st = AAR_ERR_CUDA;
    std::vector<double> one(1, 1.0);
    if (st == AAR_OK && cudaMemcpyAsync(b + n / 2, one.data(), sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = AAR_ERR_CUDA;
    float best = 1e30f;
    int best_v = 0, best_zc = 0;
    // z-chunk depths; for the segmented sweep (variant 4) segment lengths, 0 = one segment per
    // resident CTA
    const int zcs[] = {0, 8, 16, 32, 64, 128};
    for (int v = 0; v <= 7 && st == AAR_OK; ++v) {
        if (!variant_valid(probe, fp32, v) || (fp32 && v == 2)) continue;
        for (int zc : zcs) {
            if (zc == 0 && !(fp32 && v >= 4)) continue;
            if (zc > 2 * probe.nz && zc != 8) continue;
            aar_stencil_desc d = *desc;
            d.tile_variant = v + 1;
            d.tile_zc = zc;
            aar_handle h = nullptr;
            if (aar_create_stencil(&d, nullptr, precision, stream, &h) != AAR_OK) continue;
            aar_params p;
            aar_default_params(&p);
            p.m = m;
            p.p = std::max(2, std::min(6, m));
            p.tol = 0.0;
            p.max_iter = 2 * p.p + 2;
            aar_info info;
            const aar_status ss = aar_solve(h, b, nullptr, x, &p, &info);
            float t = 0.f;
            if ((ss == AAR_OK || ss == AAR_NOT_CONVERGED) && aar_profile_kernel(h, AAR_K_SWEEP, 10, &t) == AAR_OK &&
                t < best) {
                best = t;
                best_v = v;
                best_zc = zc;
            }
            aar_destroy(h);
        }
    }
    cudaFree(b);
    cudaFree(x);
    if (st != AAR_OK) return st;
    if (best >= 1e30f) return AAR_ERR_UNSUPPORTED;
    *tile_variant = best_v + 1;
    *tile_zc = best_zc;
    *ms = best;
    return AAR_OK;
}

aar_status aar_destroy(aar_handle h) {
    if (!h) return AAR_ERR_INVALID_ARG;
    if (h->E.stream) cudaStreamSynchronize(h->E.stream);
    delete h;
    return AAR_OK;
}

// ------------------------------------------------------------------------------- batches

aar_status aar_batch_create(const aar_stencil_desc* descs, int32_t nsys, int32_t precision, void* stream,
                            aar_batch* out) {
    if (!out) return AAR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!descs || nsys <= 0) return AAR_ERR_INVALID_ARG;
    if (precision != AAR_FP64 && precision != AAR_MIXED) return AAR_ERR_INVALID_ARG;
    const int radius = descs[0].radius;
    aar_batch_ctx* bt = new (std::nothrow) aar_batch_ctx;
    if (!bt) return AAR_ERR_OOM;
    bt->precision = precision;
    Engine& E = bt->E;
    E.nsys = nsys;
    E.fp32 = precision == AAR_MIXED;
    E.radius = radius;
    E.stream = (cudaStream_t)stream;
    for (int i = 0; i < nsys; ++i) {
        SysDesc S;
        if (descs[i].radius != radius || !stencil_desc(&descs[i], S)) {
            delete bt;
            return AAR_ERR_INVALID_ARG;
        }
        S.mixed = E.fp32;
        E.sys.push_back(S);
    }
    aar_status st = engine_setup(E);
    if (st != AAR_OK) {
        delete bt;
        return st;
    }
    *out = bt;
    return AAR_OK;
}

aar_status aar_batch_solve(aar_batch bt, const double* const* b, double* const* x, const aar_params* params,
                           int32_t params_stride, aar_info* infos) {
    if (!bt || !b || !x || !params) return AAR_ERR_INVALID_ARG;
    Engine& E = bt->E;
    std::vector<int> slots(E.nsys);
    int mmax = 0;
    int64_t limit = 0;
    for (int i = 0; i < E.nsys; ++i) {
        const aar_params* p = params + (params_stride ? i : 0);
        if (!valid_params(p) || !b[i] || !x[i] || !is_device_ptr(b[i]) || !is_device_ptr(x[i]))
            return AAR_ERR_INVALID_ARG;
        slots[i] = std::max(p->m + 1, 2);
        mmax = std::max(mmax, p->m);
        limit = std::max(limit, step_limit_for(p, E.fp32));
    }
    aar_status st = engine_alloc(E, slots);
    if (st != AAR_OK) return st;
    for (int i = 0; i < E.nsys; ++i) {
        SysDesc& S = E.sys[i];
        set_params(S, params + (params_stride ? i : 0));
        S.b64 = b[i];
        void* xdst = E.fp32 ? (void*)S.x64 : S.X;
        AAR_CHECK(cudaMemsetAsync(xdst, 0, sizeof(double) * S.n, E.stream));
        init_state(E.h_st[i]);
    }
    AAR_CHECK(cudaMemcpyAsync(E.d_sys, E.sys.data(), sizeof(SysDesc) * E.nsys, cudaMemcpyHostToDevice, E.stream));
    AAR_CHECK(cudaMemcpyAsync(E.d_st, E.h_st, sizeof(SysState) * E.nsys, cudaMemcpyHostToDevice, E.stream));
    st = engine_run(E, cmax_for(mmax), limit);
    if (st != AAR_OK) return st;
    aar_status worst = AAR_OK;
    for (int i = 0; i < E.nsys; ++i) {
        const SysDesc& S = E.sys[i];
        const SysState& R = E.h_st[i];
        if (R.k_final < 0) {
            AAR_CHECK(cudaMemsetAsync(x[i], 0, sizeof(double) * S.n, E.stream));
        } else {
            const void* src = E.fp32 ? (const void*)S.x64
                                     : (const void*)((const double*)S.X + ring_slot(R.k_final, S.nslots) * S.ld);
            AAR_CHECK(cudaMemcpyAsync(x[i], src, sizeof(double) * S.n, cudaMemcpyDeviceToDevice, E.stream));
        }
        if (infos) fill_info(R, &infos[i], E);
        if (R.status < 0 && worst >= 0) worst = (aar_status)R.status;
        else if (R.status == AAR_NOT_CONVERGED && worst == AAR_OK) worst = AAR_NOT_CONVERGED;
    }
    AAR_CHECK(cudaStreamSynchronize(E.stream));
    return worst;
}

aar_status aar_batch_destroy(aar_batch bt) {
    if (!bt) return AAR_ERR_INVALID_ARG;
    if (bt->E.stream) cudaStreamSynchronize(bt->E.stream);
    delete bt;
    return AAR_OK;
}

}  // extern "C"

// ====================================================================== allocation-free check
//
// aar_rel_residual_noalloc computes the same quantity as aar_rel_residual without allocating:
// the operator application is fused into the norm kernel, so the only scratch is one pair of
// partial sums per block, kept in a file-scope device array. Callers that must not allocate
// (code inside a latency-critical loop where cudaMalloc's implicit device synchronisation is not
// acceptable, or a process whose device memory is fully budgeted up front) use this form.

namespace {

constexpr int NOALLOC_MAX_PARTIALS = 8192;           // blocks per call
constexpr int64_t NOALLOC_CHUNK = 8192;              // points per block
constexpr int64_t NOALLOC_MAX_N = NOALLOC_MAX_PARTIALS * NOALLOC_CHUNK;  // 67,108,864 unknowns

// 2 partial sums per block plus the result: 128 KB + 64 B, held by every device that loads the
// library until the process exits. Shared by all calls; overlapping calls race on it.
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_MAX_PARTIALS + 8];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {};  // device address of g_noalloc_scratch, per device ordinal

// ||b - A x||^2 and ||b||^2 of one chunk of points, A applied straight from global memory.
__global__ void __launch_bounds__(256) k_resid_norm_fused(const SysDesc S, const double* __restrict__ b,
                                                         const double* __restrict__ x, int radius,
                                                         double* __restrict__ parts) {
    __shared__ double red[8];
    const int64_t s0 = (int64_t)blockIdx.x * NOALLOC_CHUNK;
    const int64_t s1 = s0 + NOALLOC_CHUNK < S.n ? s0 + NOALLOC_CHUNK : S.n;
    double rr = 0.0, bb = 0.0;
    for (int64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
        double ax = 0.0;
        if (S.is_csr) {
            for (int e = S.row_ptr[i]; e < S.row_ptr[i + 1]; ++e) ax = fma(S.val[e], x[S.col_idx[e]], ax);
        } else {
            const int64_t nx = S.nx, ny = S.ny, nz = S.nz, pst = nx * ny;
            const int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / pst;
            ax = S.cdiag * x[i];
            for (int k = 1; k <= radius; ++k) {
                double s = 0.0;
                if (S.periodic) {  // every axis wraps
                    auto wr = [](int64_t j, int64_t n) {
                        const int64_t q = j % n;
                        return q < 0 ? q + n : q;
                    };
                    s += x[(iz * ny + iy) * nx + wr(ix - k, nx)];
                    s += x[(iz * ny + iy) * nx + wr(ix + k, nx)];
                    s += x[(iz * ny + wr(iy - k, ny)) * nx + ix];
                    s += x[(iz * ny + wr(iy + k, ny)) * nx + ix];
                    s += x[(wr(iz - k, nz) * ny + iy) * nx + ix];
                    s += x[(wr(iz + k, nz) * ny + iy) * nx + ix];
                } else {
                    if (ix - k >= 0) s += x[i - k];
                    if (ix + k < nx) s += x[i + k];
                    if (iy - k >= 0) s += x[i - k * nx];
                    if (iy + k < ny) s += x[i + k * nx];
                    if (iz - k >= 0) s += x[i - k * pst];
                    if (iz + k < nz) s += x[i + k * pst];
                }
                ax = fma(S.coff[k], s, ax);
            }
        }
        const double r = b[i] - ax;
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

__global__ void __launch_bounds__(256) k_resid_norm_fused_final(double* parts, int np) {
    __shared__ double red[8];
    double rr = 0.0, bb = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        rr += parts[2 * i];
        bb += parts[2 * i + 1];
    }
    const double t0 = block_sum<8>(rr, red);
    const double t1 = block_sum<8>(bb, red);
    if (threadIdx.x == 0) parts[2 * NOALLOC_MAX_PARTIALS] = sqrt(t0) / sqrt(t1);
}

// Device address of the scratch array on device `dev`, which must be the current device;
// resolved once per device.
aar_status noalloc_scratch(int dev, double** out) {
    if (dev < 0 || dev >= 256) return AAR_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        double* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return AAR_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return AAR_OK;
}

}  // namespace

extern "C" aar_status aar_rel_residual_noalloc(aar_handle h, const double* b, const double* x, double* rel) {
    if (!h || !b || !x || !rel) return AAR_ERR_INVALID_ARG;
    Engine& E = h->E;
    const SysDesc& S = E.sys[0];
    if (S.n > NOALLOC_MAX_N) return AAR_ERR_INVALID_ARG;  // more blocks than the scratch array holds
    if (!is_device_ptr(b) || !is_device_ptr(x)) return AAR_ERR_INVALID_ARG;
    // the handle's stream belongs to the handle's device: the scratch address must be that
    // device's copy of the array, so the call is made with that device current
    int dev = -1;
    AAR_CHECK(cudaGetDevice(&dev));
    if (dev != E.device) return AAR_ERR_INVALID_ARG;
    double* scratch = nullptr;
    aar_status st = noalloc_scratch(dev, &scratch);
    if (st != AAR_OK) return st;
    const int np = (int)((S.n + NOALLOC_CHUNK - 1) / NOALLOC_CHUNK);
    k_resid_norm_fused<<<np, 256, 0, E.stream>>>(S, b, x, E.radius, scratch);
    k_resid_norm_fused_final<<<1, 256, 0, E.stream>>>(scratch, np);
    AAR_CHECK(cudaGetLastError());
    AAR_CHECK(cudaMemcpyAsync(rel, scratch + 2 * NOALLOC_MAX_PARTIALS, sizeof(double), cudaMemcpyDeviceToHost,
                              E.stream));
    AAR_CHECK(cudaStreamSynchronize(E.stream));
    return AAR_OK;
}

// ================================================================================== serving
//
// Continuous batching: every admitted solve keeps its whole state (ring, iterate, right-hand
// side, phase machine) on the device; aar_server_run admits waiting requests in arrival order
// while their footprint fits the budget and a slot is free, advances every resident solve by a
// number of ticks with the batched kernels, then retires the finished ones. Systems enter and
// leave between rounds while the others continue where they were.

namespace {

struct ServerRequest {
    int64_t id;
    aar_stencil_desc desc;
    const double* b;  // host, caller-owned until completion
    double* x;        // host, written at completion
    aar_params prm;
    size_t bytes;
};

struct ServerSlot {
    bool used = false;
    int64_t id = -1;
    void* mem = nullptr;
    size_t bytes = 0;
    double* x = nullptr;
};

size_t request_bytes(const SysDesc& S, int m, int fp32) {
    const size_t w = fp32 ? 4 : 8;
    const size_t nslots = (size_t)std::max(m + 1, 2);
    size_t bytes = 2 * nslots * S.ld * w + (size_t)S.ld * 8;  // rings + b
    if (fp32) bytes += (size_t)S.ld * 8 + 3 * (size_t)S.ld * 4;  // x64, rhs32, xold, fold
    return bytes;
}

}  // namespace

struct aar_server_ctx {
    Engine E;
    int precision = AAR_FP64;
    int64_t budget = 0, used = 0, next_id = 1;
    int max_m = 0;
    std::deque<ServerRequest> waiting;
    std::vector<ServerSlot> slots;
    std::vector<std::pair<int64_t, aar_info>> done;
    bool dirty = false;
    // the slots' memory comes from the server's own stream-ordered pool, which keeps what retired
    // solves free (up to the budget) for the next admissions instead of returning it to the
    // driver at every synchronisation
    cudaMemPool_t pool = nullptr;
};

extern "C" {

aar_status aar_server_create(int32_t radius, int32_t precision, int64_t budget_bytes, int32_t max_active,
                             void* stream, aar_server* out) {
    if (!out) return AAR_ERR_INVALID_ARG;
    *out = nullptr;
    if (radius < 1 || radius > AAR_MAX_RADIUS || budget_bytes <= 0 || max_active < 1 || max_active > 65536)
        return AAR_ERR_INVALID_ARG;
    if (precision != AAR_FP64 && precision != AAR_MIXED) return AAR_ERR_INVALID_ARG;
    aar_server_ctx* sv = new (std::nothrow) aar_server_ctx;
    if (!sv) return AAR_ERR_OOM;
    Engine& E = sv->E;
    E.nsys = max_active;
    E.fp32 = precision == AAR_MIXED;
    E.radius = radius;
    E.stream = (cudaStream_t)stream;
    sv->precision = precision;
    sv->budget = budget_bytes;
    SysDesc empty;
    memset(&empty, 0, sizeof(empty));
    empty.nx = empty.ny = empty.nz = 1;
    empty.n = 1;
    empty.ld = PAD;
    empty.p = 1;
    E.sys.assign(max_active, empty);
    E.active.assign(max_active, 0);
    sv->slots.resize(max_active);
    aar_status st = alloc_tables(E);
    if (st == AAR_OK) {
        int dev = 0;
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        const uint64_t keep = (uint64_t)budget_bytes;
        bool ok = cudaGetDevice(&dev) == cudaSuccess;
        props.location.id = dev;
        ok = ok && cudaMemPoolCreate(&sv->pool, &props) == cudaSuccess;
        ok = ok && cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, (void*)&keep) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            st = AAR_ERR_CUDA;
        }
    }
    if (st == AAR_OK) {
        for (int s = 0; s < max_active; ++s) {
            init_state(E.h_st[s]);
            E.h_st[s].phase = PH_DONE;
        }
        if (cudaMemcpy(E.d_st, E.h_st, sizeof(SysState) * max_active, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(E.d_sys, E.sys.data(), sizeof(SysDesc) * max_active, cudaMemcpyHostToDevice) != cudaSuccess)
            st = AAR_ERR_CUDA;
    }
    if (st != AAR_OK) {
        if (sv->pool) cudaMemPoolDestroy(sv->pool);
        delete sv;
        return st;
    }
    *out = sv;
    return AAR_OK;
}

aar_status aar_server_submit(aar_server sv, const aar_stencil_desc* desc, const double* b, double* x,
                             const aar_params* params, int64_t* request_id) {
    if (!sv || !desc || !b || !x || !request_id || !valid_params(params)) return AAR_ERR_INVALID_ARG;
    if (desc->radius != sv->E.radius) return AAR_ERR_INVALID_ARG;
    SysDesc S;
    if (!stencil_desc(desc, S)) return AAR_ERR_INVALID_ARG;
    ServerRequest r;
    r.id = sv->next_id++;
    r.desc = *desc;
    r.b = b;
    r.x = x;
    r.prm = *params;
    r.bytes = request_bytes(S, params->m, sv->E.fp32);
    if ((int64_t)r.bytes > sv->budget) return AAR_ERR_OOM;
    sv->waiting.push_back(r);
    *request_id = r.id;
    return AAR_OK;
}

aar_status aar_server_run(aar_server sv, int32_t ticks, int32_t* n_active, int32_t* n_waiting,
                          int64_t* bytes_in_use) {
    if (!sv || ticks < 0) return AAR_ERR_INVALID_ARG;
    Engine& E = sv->E;
    const int cap = E.nsys;
    // admit in arrival order while the head fits (no overtaking: first come, first served)
    bool admitted = false;
    while (!sv->waiting.empty()) {
        ServerRequest& r = sv->waiting.front();
        if (sv->used + (int64_t)r.bytes > sv->budget) break;
        int slot = -1;
        for (int s = 0; s < cap; ++s)
            if (!sv->slots[s].used) {
                slot = s;
                break;
            }
        if (slot < 0) break;
        SysDesc S;
        stencil_desc(&r.desc, S);
        S.mixed = E.fp32;
        set_params(S, &r.prm);
        void* mem = nullptr;
        if (cudaMallocFromPoolAsync(&mem, r.bytes, sv->pool, E.stream) != cudaSuccess) {
            cudaGetLastError();
            break;  // retry after something retires
        }
        AAR_CHECK(cudaMemsetAsync(mem, 0, r.bytes, E.stream));
        const size_t w = E.fp32 ? 4 : 8;
        const int nslots = std::max(r.prm.m + 1, 2);
        char* base = reinterpret_cast<char*>(mem);
        S.nslots = nslots;
        S.X = base;
        S.F = base + (size_t)nslots * S.ld * w;
        char* tail = base + 2 * (size_t)nslots * S.ld * w;
        double* b64 = reinterpret_cast<double*>(tail);
        tail += (size_t)S.ld * 8;
        if (E.fp32) {
            S.x64 = reinterpret_cast<double*>(tail);
            S.rhs32 = reinterpret_cast<float*>(tail + (size_t)S.ld * 8);
            S.xold = S.rhs32 + S.ld;
            S.fold = S.xold + S.ld;
        }
        AAR_CHECK(cudaMemcpyAsync(b64, r.b, sizeof(double) * S.n, cudaMemcpyHostToDevice, E.stream));
        S.b64 = b64;
        E.sys[slot] = S;
        E.active[slot] = 1;
        init_state(E.h_st[slot]);
        AAR_CHECK(cudaMemcpyAsync(E.d_st + slot, E.h_st + slot, sizeof(SysState), cudaMemcpyHostToDevice, E.stream));
        ServerSlot& sl = sv->slots[slot];
        sl.used = true;
        sl.id = r.id;
        sl.mem = mem;
        sl.bytes = r.bytes;
        sl.x = r.x;
        sv->used += (int64_t)r.bytes;
        sv->max_m = std::max(sv->max_m, r.prm.m);
        sv->waiting.pop_front();
        admitted = true;
    }
    if (admitted || sv->dirty) {
        build_tiles(E);
        aar_status st = build_maps(E);
        if (st != AAR_OK) return st;
        st = upload_tiles(E);
        if (st != AAR_OK) return st;
        AAR_CHECK(cudaMemcpyAsync(E.d_sys, E.sys.data(), sizeof(SysDesc) * cap, cudaMemcpyHostToDevice, E.stream));
        sv->dirty = false;
    }
    int active = 0;
    for (int s = 0; s < cap; ++s) active += sv->slots[s].used ? 1 : 0;
    if (active > 0) {
        const EngineView ev = E.view();
        const int cmax = cmax_for(sv->max_m);
        const int nv = (int)E.vtiles.size();
        // when every resident solve has the same Anderson period p >= 2, the ticks take the
        // solve graph's layout: p - 1 Richardson-only ticks (the sweep alone) and one full tick,
        // rounded to whole bodies of p ticks; otherwise every tick is a full tick
        const int period = common_period(E);
        const int nt = period > 0 ? std::max(1, (ticks + period / 2) / period) * period : ticks;
        for (int t = 0; t < nt; ++t) {
            if (period > 0 && t % period != period - 1) {
                AAR_CHECK(launch_tick_r(E, t % period + 1, E.stream));
                continue;
            }
            const int j = period > 0 ? TICK_FULL : 0;
            // a full tick of the solve loop plus the norm pass for newly admitted systems
            AAR_CHECK(launch_resid_groups(E, E.stream));
            AAR_CHECK(launch_sweep_groups(E, E.stream, j));
            AAR_CHECK(launch_gram_any(E, cmax, j, E.stream));
            AAR_CHECK(launch_norm_b(E.d_vtiles, nv, E.vec_grid, ev, E.stream));
            AAR_CHECK(launch_finalize(ev, j, E.stream));
            AAR_CHECK(launch_update_any(E, cmax, E.stream));
        }
        // retire finished solves
        AAR_CHECK(cudaMemcpyAsync(E.h_st, E.d_st, sizeof(SysState) * cap, cudaMemcpyDeviceToHost, E.stream));
        AAR_CHECK(cudaStreamSynchronize(E.stream));
        for (int s = 0; s < cap; ++s) {
            ServerSlot& sl = sv->slots[s];
            if (!sl.used || E.h_st[s].phase != PH_DONE) continue;
            const SysDesc& S = E.sys[s];
            const SysState& R = E.h_st[s];
            if (R.k_final < 0) {
                memset(sl.x, 0, sizeof(double) * S.n);
            } else {
                const void* src = E.fp32 ? (const void*)S.x64
                                         : (const void*)((const double*)S.X + ring_slot(R.k_final, S.nslots) * S.ld);
                AAR_CHECK(cudaMemcpyAsync(sl.x, src, sizeof(double) * S.n, cudaMemcpyDeviceToHost, E.stream));
            }
            aar_info info;
            memset(&info, 0, sizeof(info));
            info.iterations = R.iters_total;
            info.anderson_steps = R.anderson;
            info.refinements = R.refinements;
            info.rel_residual = R.r_last;
            info.status = R.status;
            info.last_rank = R.last_rank;
            sv->done.emplace_back(sl.id, info);
            AAR_CHECK(cudaFreeAsync(sl.mem, E.stream));
            sv->used -= (int64_t)sl.bytes;
            sl = ServerSlot();
            E.active[s] = 0;
            sv->dirty = true;
            --active;
        }
        AAR_CHECK(cudaStreamSynchronize(E.stream));
    }
    if (n_active) *n_active = active;
    if (n_waiting) *n_waiting = (int32_t)sv->waiting.size();
    if (bytes_in_use) *bytes_in_use = sv->used;
    return AAR_OK;
}

aar_status aar_server_poll(aar_server sv, int64_t* ids, aar_info* infos, int32_t cap, int32_t* n) {
    if (!sv || !n || cap < 0 || (cap > 0 && (!ids || !infos))) return AAR_ERR_INVALID_ARG;
    const int32_t k = (int32_t)std::min<size_t>((size_t)cap, sv->done.size());
    for (int32_t i = 0; i < k; ++i) {
        ids[i] = sv->done[i].first;
        infos[i] = sv->done[i].second;
    }
    sv->done.erase(sv->done.begin(), sv->done.begin() + k);
    *n = k;
    return AAR_OK;
}

aar_status aar_server_destroy(aar_server sv) {
    if (!sv) return AAR_ERR_INVALID_ARG;
    Engine& E = sv->E;
    if (E.stream) cudaStreamSynchronize(E.stream);
    for (ServerSlot& sl : sv->slots)
        if (sl.used) cudaFreeAsync(sl.mem, E.stream);
    if (E.stream) cudaStreamSynchronize(E.stream);
    if (sv->pool) cudaMemPoolDestroy(sv->pool);
    delete sv;
    return AAR_OK;
}

}  // extern "C"

// ====================================================================== domain decomposition
//
// A rank's slab [z_lo, z_hi) of a stencil grid is an ordinary one-system engine of that many
// planes whose FP64 sweep reads the z neighbours beyond the slab from two ghost buffers (r planes
// each). The iteration runs from the host, one step at a time, because two of its steps need the
// other ranks: before every sweep the caller's halo callback fills the ghost buffers from the
// neighbouring slabs' boundary planes of x_k (Sec. 3.2: ghost regions of a subdomain), and at an
// Anderson step the tile partial sums of ||b - A x_k||^2, F^T F and F^T f_k are folded into one
// packed vector that the caller's allreduce callback sums over ranks (Sec. 3.2: the single
// reduction per Anderson step), then written back as the first tile's partials so that the
// finalize kernel sees the global sums. ||b|| is reduced the same way once at the start. Every
// rank then takes the same decisions and the same gamma.

struct aar_dd_ctx {
    Engine E;
    int32_t z_lo = 0, z_hi = 0;
    double* ghosts = nullptr;  // [2][r nx ny]: below, above (zero where the grid has no neighbour)
    double* packed = nullptr;  // 1 + c(c+1)/2 + c reduced values (MAXM columns at most)
    ~aar_dd_ctx() {
        cudaFree(ghosts);
        cudaFree(packed);
    }
};

extern "C" {

aar_status aar_dd_create(const aar_stencil_desc* global, int32_t z_lo, int32_t z_hi, void* stream,
                         aar_dd_handle* out) {
    if (!out) return AAR_ERR_INVALID_ARG;
    *out = nullptr;
    SysDesc G;
    if (!stencil_desc(global, G)) return AAR_ERR_INVALID_ARG;
    if (G.block == 2) return AAR_ERR_INVALID_ARG;
    if (z_lo < 0 || z_hi > global->nz || z_hi - z_lo < global->radius) return AAR_ERR_INVALID_ARG;
    aar_stencil_desc d = *global;
    d.nz = z_hi - z_lo;
    d.tile_variant = d.tile_zc = 0;
    SysDesc S;
    if (!stencil_desc(&d, S)) return AAR_ERR_INVALID_ARG;
    aar_dd_ctx* h = new (std::nothrow) aar_dd_ctx;
    if (!h) return AAR_ERR_OOM;
    h->z_lo = z_lo;
    h->z_hi = z_hi;
    Engine& E = h->E;
    E.nsys = 1;
    E.fp32 = 0;
    E.radius = d.radius;
    E.stream = (cudaStream_t)stream;
    S.mixed = 0;
    E.sys.push_back(S);
    aar_status st = engine_setup(E);
    const size_t gbytes = sizeof(double) * (size_t)d.radius * d.nx * d.ny;
    if (st == AAR_OK) {
        if (cudaMalloc(&h->ghosts, 2 * gbytes) != cudaSuccess ||
            cudaMalloc(&h->packed, sizeof(double) * (1 + MAXM * (MAXM + 1) / 2 + MAXM)) != cudaSuccess ||
            cudaMemsetAsync(h->ghosts, 0, 2 * gbytes, E.stream) != cudaSuccess ||
            cudaStreamSynchronize(E.stream) != cudaSuccess) {
            cudaGetLastError();
            st = AAR_ERR_OOM;
        }
    }
    if (st != AAR_OK) {
        delete h;
        return st;
    }
    E.sys[0].ghost_lo = h->ghosts;
    E.sys[0].ghost_hi = h->ghosts + (size_t)d.radius * d.nx * d.ny;
    *out = h;
    return AAR_OK;
}

aar_status aar_dd_solve(aar_dd_handle h, const double* b, double* x, const aar_params* params, const aar_comm* comm,
                        aar_info* info) {
    if (info) {
        memset(info, 0, sizeof(*info));
        info->rel_residual = NAN;
    }
    if (!h || !b || !x || !valid_params(params) || !comm || !comm->halo || !comm->allreduce) {
        if (info) info->status = AAR_ERR_INVALID_ARG;
        return AAR_ERR_INVALID_ARG;
    }
    if (!is_device_ptr(b) || !is_device_ptr(x)) {
        if (info) info->status = AAR_ERR_INVALID_ARG;
        return AAR_ERR_INVALID_ARG;
    }
    Engine& E = h->E;
    SysDesc& S = E.sys[0];
    const int m = params->m, p = params->p, R = E.radius;
    aar_status st = engine_alloc(E, std::vector<int>{std::max(m + 1, 2)});
    if (st != AAR_OK) return st;
    set_params(S, params);
    if (params->step_limit > 0) S.max_iter = std::min<int64_t>(S.max_iter, params->step_limit);
    S.b64 = b;
    const int cmax = cmax_for(m);
    const int64_t ps = (int64_t)S.nx * S.ny;
    AAR_CHECK(cudaMemsetAsync(S.X, 0, sizeof(double) * S.n, E.stream));  // x_0 = 0
    SysState init;
    init_state(init);
    *E.h_st = init;
    AAR_CHECK(cudaMemcpyAsync(E.d_sys, &S, sizeof(SysDesc), cudaMemcpyHostToDevice, E.stream));
    AAR_CHECK(cudaMemcpyAsync(E.d_st, E.h_st, sizeof(SysState), cudaMemcpyHostToDevice, E.stream));
    for (int i = 0; i < 16; ++i) E.h_ctrl[i] = 0;
    AAR_CHECK(cudaMemcpyAsync(E.d_ctrl, E.h_ctrl, sizeof(int) * 16, cudaMemcpyHostToDevice, E.stream));
    const EngineView ev = E.view();
    auto read_state = [&]() -> aar_status {
        AAR_CHECK(cudaMemcpyAsync(E.h_st, E.d_st, sizeof(SysState), cudaMemcpyDeviceToHost, E.stream));
        AAR_CHECK(cudaStreamSynchronize(E.stream));
        return AAR_OK;
    };
    int64_t launches = 0;
    auto comm_fail = [&]() {
        cudaStreamSynchronize(E.stream);
        if (info) info->status = AAR_ERR_COMM;
        return AAR_ERR_COMM;
    };
    // ||b||: this slab's partial sums, one sum over ranks, then the finalize's INIT phase
    AAR_CHECK(launch_norm_b(E.d_vtiles, (int)E.vtiles.size(), E.vec_grid, ev, E.stream));
    AAR_CHECK(launch_dd_pack(ev, 0, 0, h->packed, E.stream));
    if (comm->allreduce(comm->ctx, h->packed, 1, E.stream) != 0) return comm_fail();
    AAR_CHECK(launch_dd_unpack(ev, 0, 0, h->packed, E.stream));
    AAR_CHECK(launch_finalize(ev, 0, E.stream));
    launches += 4;
    if ((st = read_state()) != AAR_OK) return st;
    for (int64_t k = 0; E.h_st->phase != PH_DONE; ++k) {
        // ghost planes of x_k from the neighbouring slabs
        double* xk = reinterpret_cast<double*>(S.X) + ring_slot(k, S.nslots) * S.ld;
        if (comm->halo(comm->ctx, xk, xk + (int64_t)(S.nz - R) * ps, const_cast<double*>(S.ghost_lo),
                       const_cast<double*>(S.ghost_hi), (int64_t)R * ps, E.stream) != 0)
            return comm_fail();
        AAR_CHECK(launch_sweep_groups(E, E.stream));
        const bool anderson = ((k + 1) % p) == 0;
        if (anderson) {
            const int c = (int)std::min<int64_t>(k, m);
            AAR_CHECK(launch_gram_any(E, cmax, 0, E.stream));
            AAR_CHECK(launch_dd_pack(ev, 1, c, h->packed, E.stream));
            if (comm->allreduce(comm->ctx, h->packed, 1 + c * (c + 1) / 2 + c, E.stream) != 0) return comm_fail();
            AAR_CHECK(launch_dd_unpack(ev, 1, c, h->packed, E.stream));
            launches += 3;
        }
        AAR_CHECK(launch_finalize(ev, 0, E.stream));
        launches += 2;
        if (anderson) {
            AAR_CHECK(launch_update_any(E, cmax, E.stream));
            ++launches;
        }
        // the state decides at every Anderson step and at the iteration cap
        if (anderson || k + 1 >= S.max_iter)
            if ((st = read_state()) != AAR_OK) return st;
    }
    const SysState& R0 = *E.h_st;
    if (R0.k_final < 0) {
        AAR_CHECK(cudaMemsetAsync(x, 0, sizeof(double) * S.n, E.stream));
    } else {
        const double* src = reinterpret_cast<const double*>(S.X) + ring_slot(R0.k_final, S.nslots) * S.ld;
        AAR_CHECK(cudaMemcpyAsync(x, src, sizeof(double) * S.n, cudaMemcpyDeviceToDevice, E.stream));
    }
    AAR_CHECK(cudaStreamSynchronize(E.stream));
    E.last_ticks = R0.iters_total;
    E.last_launches = launches;
    fill_info(R0, info, E);
    return (aar_status)R0.status;
}

aar_status aar_dd_destroy(aar_dd_handle h) {
    if (!h) return AAR_ERR_INVALID_ARG;
    if (h->E.stream) cudaStreamSynchronize(h->E.stream);
    delete h;
    return AAR_OK;
}

}  // extern "C"

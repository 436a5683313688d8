// aar_mbar.cuh -- shared-memory barriers and asynchronous copies (inline PTX, sm_100 family):
// mbarrier set-up and bounded waits, 3-D tiled TMA loads, 1-D bulk copies and 4-byte cp.async.
// Every wait is bounded: one that gives up records where in err[0..3] and sets the caller's abort
// flag; mbar_drain lets a CTA that gave up wait (bounded again) for its copies still in flight.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace aar {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// 4-byte global -> shared copies (the periodic sweep's plane fills)
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
// 8-byte global -> shared copies (the complex FP32 sweep's plane fills)
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// every committed group of this thread but the most recent one has landed
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ int wrap_index(int j, int n) {
    const int q = j % n;
    return q < 0 ? q + n : q;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after 2^20 polls (each try_wait itself suspends for a bounded time),
// records where it gave up in err[0..3] and sets *abort so the thread skips every later wait.
__device__ __forceinline__ void mbar_wait(uint32_t bar, uint32_t parity, int* err, bool& abort, int where) {
    if (abort) return;
    for (uint32_t it = 0; it < (1u << 20); ++it)
        if (mbar_try_wait(bar, parity)) return;
    abort = true;
    if (atomicCAS(err, 0, 1) == 0) {
        err[1] = where;
        err[2] = (int)parity;
        err[3] = (int)bar;
    }
}

// Ends the pipeline of a CTA in which a wait gave up: waits, bounded again, for the copies that may
// still be landing before the CTA leaves. Planes (chunks) lo .. hi-1 were issued in order on a ring
// of ns stages; only the last ns of them can still be in flight, and each of those is the latest
// copy on its stage, so its phase parity shows whether it has landed. Called by the issuing thread
// after a CTA-wide vote (__syncthreads_or) found a wait that gave up, with no further issue.
__device__ __forceinline__ void mbar_drain(const uint64_t* bars, uint32_t ns, uint32_t lo, uint32_t hi) {
    if (hi <= lo) return;
    for (uint32_t g = (hi - lo > ns ? hi - ns : lo); g < hi; ++g) {
        const uint32_t bar = smem_u32(&bars[g % ns]);
        for (uint32_t it = 0; it < (1u << 22); ++it)
            if (mbar_try_wait(bar, (g / ns) & 1u)) break;
    }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

}  // namespace aar

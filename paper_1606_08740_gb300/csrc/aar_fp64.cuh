// aar_fp64.cuh -- FP64 additions issued as fused multiply-adds.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so the FP64 stencil sweeps, Gram and update passes
// are bound by the FP64 pipe, not by HBM. On this part that pipe retires DFMA at a higher rate than
// DADD (0.63e12 against 0.53e12 instructions/s, independent chains on every SM), and fma(a, 1, b)
// rounds exactly as a + b does: those passes form their sums and differences with uadd / usub,
// which give bitwise the same values as plain additions and subtractions. The unit multiplier is
// read from device memory so that the compiler keeps the multiply-add instead of folding it back
// into an add.
#pragma once

namespace aar {

static __device__ double g_unit_one = 1.0;

// The multiplier: read once per thread, before the loops that use it.
__device__ __forceinline__ double unit_one() { return *reinterpret_cast<const volatile double*>(&g_unit_one); }

// a + b, for FP64 as fma(a, one, b) (one == 1.0), for FP32 as a plain addition.
template <typename T>
__device__ __forceinline__ T uadd(T a, T b, T one) {
    if constexpr (sizeof(T) == 8) return fma(a, one, b);
    else return a + b;
}

// b - a, for FP64 as fma(a, -one, b) (the same single rounding), for FP32 as a plain subtraction.
template <typename T>
__device__ __forceinline__ T usub(T b, T a, T one) {
    if constexpr (sizeof(T) == 8) return fma(a, -one, b);
    else return b - a;
}

}  // namespace aar

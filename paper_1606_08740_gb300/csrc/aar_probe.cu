// aar_probe.cu -- FP64 instruction-rate probe: the denominator of the FP64 sweeps' roofline.
//
// The FP64 stencil sweeps run about 6r + 4 FP64 instructions per point against 32 bytes, so on
// this part they are bound by the FP64 pipe, not by HBM. Their roofline divides the sweep's FP64
// instruction count by the rate this probe measures: every thread runs 8 independent dependency
// chains of DFMA (or DADD) instructions, enough blocks are resident to fill every SM, and the
// launch is timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include "aar.h"

namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_UNROLL = 16;

template <int OP>  // 0: DFMA a = a * m + c; 1: DADD a = a + c
__global__ void __launch_bounds__(256) k_fp64_rate(double m, double c, int iters, double* sink) {
    double a[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int i = 0; i < PROBE_CHAINS; ++i) a[i] = OP == 0 ? fma(a[i], m, c) : a[i] + c;
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += a[i];
    if (s == -1.0) sink[threadIdx.x] = s;  // never true: keeps every chain live
}

}  // namespace

extern "C" aar_status aar_measure_fp64_rate(void* stream, int32_t op, double* instr_per_s) {
    if (!instr_per_s || (op != 0 && op != 1)) return AAR_ERR_INVALID_ARG;
    *instr_per_s = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return AAR_ERR_CUDA;
    const cudaError_t eo = op == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_rate<0>, 256, 0)
                                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_rate<1>, 256, 0);
    if (eo != cudaSuccess || per_sm < 1) return AAR_ERR_CUDA;
    const int grid = sms * per_sm, iters = 400;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return AAR_ERR_CUDA;
    }
    auto launch = [&]() {
        if (op == 0) k_fp64_rate<0><<<grid, 256, 0, s>>>(1.0000001, 1e-9, iters, nullptr);
        else k_fp64_rate<1><<<grid, 256, 0, s>>>(1.0000001, 1e-9, iters, nullptr);
    };
    launch();  // warm-up
    cudaEventRecord(e0, s);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, s);
    float ms = 0.f;
    const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) return AAR_ERR_CUDA;
    const double instr = (double)grid * 256.0 * iters * PROBE_UNROLL * PROBE_CHAINS * reps;
    *instr_per_s = instr / (ms * 1e-3);
    return AAR_OK;
}

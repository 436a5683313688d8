// Radius dispatch of the fused stencil kernels.
#include "aar_engine.cuh"

namespace aar {

#define AAR_DECL(RR)                                                                                   \
    cudaError_t launch_stencil_r##RR(int fp32, int mode, const OpLaunch& L, const EngineView& ev, int j, \
                                     const double* xin, double* yout, cudaStream_t s);                  \
    int occupancy_r##RR(int fp32, int mode, int variant);
AAR_DECL(1)
AAR_DECL(2)
AAR_DECL(3)
AAR_DECL(4)
AAR_DECL(5)
AAR_DECL(6)
#undef AAR_DECL

cudaError_t launch_stencil(int radius, int fp32, int mode, const OpLaunch& L, const EngineView& ev, int j,
                           const double* xin, double* yout, cudaStream_t s) {
    switch (radius) {
        case 1: return launch_stencil_r1(fp32, mode, L, ev, j, xin, yout, s);
        case 2: return launch_stencil_r2(fp32, mode, L, ev, j, xin, yout, s);
        case 3: return launch_stencil_r3(fp32, mode, L, ev, j, xin, yout, s);
        case 4: return launch_stencil_r4(fp32, mode, L, ev, j, xin, yout, s);
        case 5: return launch_stencil_r5(fp32, mode, L, ev, j, xin, yout, s);
        case 6: return launch_stencil_r6(fp32, mode, L, ev, j, xin, yout, s);
        default: return cudaErrorInvalidValue;
    }
}

int stencil_occupancy(int radius, int fp32, int mode, int variant) {
    switch (radius) {
        case 1: return occupancy_r1(fp32, mode, variant);
        case 2: return occupancy_r2(fp32, mode, variant);
        case 3: return occupancy_r3(fp32, mode, variant);
        case 4: return occupancy_r4(fp32, mode, variant);
        case 5: return occupancy_r5(fp32, mode, variant);
        case 6: return occupancy_r6(fp32, mode, variant);
        default: return 1;
    }
}

// Tile heights and CTA sizes of the variants instantiated in aar_stencil.cuh.
int stencil_variant_ty(int fp32, int variant) {
    if (fp32) return variant == 0 ? 32 : variant == 1 ? 8 : variant == 2 ? 32 : 16;
    return variant == 0 ? 16 : 8;
}

int stencil_variant_tx(int fp32, int variant) { return (fp32 && variant >= 4) ? 64 : 32; }

int stencil_variant_threads(int fp32, int variant) { return (variant == 1) ? 128 : 256; }

// x extent of the TMA box of a variant: the 32-wide tile plus the halo rounded up to 16 bytes
int stencil_tma_box_x(int radius, int variant) {
    return (variant == 4 || variant == 6 ? 64 : 32) + 2 * ((radius + 3) / 4 * 4);
}

}  // namespace aar

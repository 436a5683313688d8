// Radius-4 instantiations of the fused stencil kernels (see aar_stencil.cuh).
#include "aar_stencil.cuh"

namespace aar {
AAR_STENCIL_RADIUS_IMPL(4)
}  // namespace aar

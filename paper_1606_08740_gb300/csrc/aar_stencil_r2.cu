// Radius-2 instantiations of the fused stencil kernels (see aar_stencil.cuh).
#include "aar_stencil.cuh"

namespace aar {
AAR_STENCIL_RADIUS_IMPL(2)
}  // namespace aar

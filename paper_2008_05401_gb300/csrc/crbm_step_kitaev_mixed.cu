// Instantiations of the fused kernel for Kitaev / Mixed.
#include "crbm_step.cuh"

namespace crbm {
CRBM_VARIANTS(kKitaev, kMixed)
}  // namespace crbm

// Instantiations of the fused kernel for Kitaev / Mixed, CTAs of 64 threads.
#include "crbm_step.cuh"

namespace crbm {
CRBM_VARIANTS_NT(kKitaev, kMixed, 64)
}  // namespace crbm

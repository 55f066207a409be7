// Instantiations of the fused kernel for Kitaev / FP64, CTAs of 256 threads.
#include "crbm_step.cuh"

namespace crbm {
CRBM_VARIANTS_NT(kKitaev, kFP64, 256)
}  // namespace crbm

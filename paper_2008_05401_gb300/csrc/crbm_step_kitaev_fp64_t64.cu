// Instantiations of the fused kernel for Kitaev / FP64, CTAs of 64 threads.
#include "crbm_step.cuh"

namespace crbm {
CRBM_VARIANTS_NT(kKitaev, kFP64, 64)
}  // namespace crbm

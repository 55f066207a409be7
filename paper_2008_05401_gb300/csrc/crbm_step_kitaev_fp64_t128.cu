// Instantiations of the fused kernel for Kitaev / FP64, CTAs of 128 threads.
#include "crbm_step.cuh"

namespace crbm {
CRBM_VARIANTS_NT(kKitaev, kFP64, 128)
}  // namespace crbm

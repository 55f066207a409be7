// Instantiations of the fused kernel for Kitaev / FP64.
#include "crbm_step.cuh"

namespace crbm {
CRBM_VARIANTS(kKitaev, kFP64)
}  // namespace crbm

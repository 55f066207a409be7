// Instantiations of the fused proposal kernel for Kitaev / FP64, CTAs of 256
// threads holding several chain groups (batches of mixed lattice sizes).
#include "crbm_step.cuh"

namespace crbm {
CRBM_VARIANTS_MULTI(kKitaev, kFP64, 256)
}  // namespace crbm

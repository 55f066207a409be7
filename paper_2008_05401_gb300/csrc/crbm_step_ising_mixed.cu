// Instantiations of the fused kernel for Ising / Mixed.
#include "crbm_step.cuh"

namespace crbm {
CRBM_VARIANTS(kIsing, kMixed)
}  // namespace crbm

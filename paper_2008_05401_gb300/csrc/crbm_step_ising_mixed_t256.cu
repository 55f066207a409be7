// Instantiations of the fused kernel for Ising / Mixed, CTAs of 256 threads.
#include "crbm_step.cuh"

namespace crbm {
CRBM_VARIANTS_NT(kIsing, kMixed, 256)
}  // namespace crbm

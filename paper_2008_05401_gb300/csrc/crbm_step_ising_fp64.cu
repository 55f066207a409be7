// Instantiations of the fused kernel for Ising / FP64.
#include "crbm_step.cuh"

namespace crbm {
CRBM_VARIANTS(kIsing, kFP64)
}  // namespace crbm

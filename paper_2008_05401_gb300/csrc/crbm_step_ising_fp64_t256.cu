// Instantiations of the fused kernel for Ising / FP64, CTAs of 256 threads.
#include "crbm_step.cuh"

namespace crbm {
CRBM_VARIANTS_NT(kIsing, kFP64, 256)
}  // namespace crbm

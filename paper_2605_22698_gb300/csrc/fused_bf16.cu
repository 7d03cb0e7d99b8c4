// Fused BF16 form of the interaction layer (tcgen05 radial MLP).
#include "launchers.cuh"

namespace mlip {

int energy_forces_fused(mlip_model*, const double*, const int*, int64_t, const double*, const uint8_t*, double*,
                        double*, double*, cudaStream_t) {
  set_error("the fused BF16 form is not available in this build");
  return MLIP_ERR_INVALID_ARG;
}

}  // namespace mlip

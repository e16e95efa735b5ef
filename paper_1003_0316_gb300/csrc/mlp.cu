// Learned initialiser of the multipole fit (placeholder until the kernels land).
#include "gw_internal.cuh"

namespace gw {

int mlp_forward(int, const double*, const float*, float*, cudaStream_t) {
  return set_error(GW_EUNSUPPORTED, "MLP forward not built");
}
int mlp_train_step(int, const OmegaArr&, const double*, float*, float*, float*, float*, float, int,
                   float*, cudaStream_t) {
  return set_error(GW_EUNSUPPORTED, "MLP training not built");
}

}  // namespace gw

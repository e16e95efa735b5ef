// a2 tensor-core path (placeholder until the tcgen05 kernel lands).
#include "gw_internal.cuh"

namespace gw {

size_t pol_tc_workspace(int, const int64_t*, const int*, int, int) { return 0; }

int pol_tc(int, const PolQ*, double, int, const OmegaArr&, int precision, void*, size_t,
           cudaStream_t, const DeviceCtx&) {
  return set_error(GW_EUNSUPPORTED, "tensor-core polarization (precision %d) not built", precision);
}

}  // namespace gw

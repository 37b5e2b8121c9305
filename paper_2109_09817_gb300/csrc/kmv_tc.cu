// Tensor-core K-hat V (tcgen05): not built yet; every precision other than
// GP_FP32_PLAIN reports GP_EINVAL through kmv().
#include "gp_internal.cuh"

namespace gp {

bool kmv_tc_supported(const Prep&, int, int) { return false; }

int kmv_tc(gp_ctx* ctx, const Prep&, const Prep&, const float*, int64_t, int,
           float*, int64_t, float, bool, int) {
  return set_err(ctx, GP_EINVAL, "tensor-core product not available");
}

}  // namespace gp

// Relight contraction on the tensor cores (placeholder until the tcgen05 path lands).
#include "common.cuh"
#include "internal.h"

namespace prtgs {

int relight_tc(int64_t, int32_t, const float*, const float*, const float*, int32_t, int32_t, float*, void*,
               cudaStream_t) {
  return PRTGS_ERR_UNSUPPORTED;
}

}  // namespace prtgs

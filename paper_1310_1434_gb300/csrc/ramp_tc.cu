// Ramp filtration on tensor cores: placeholder until the tcgen05 kernel lands.
#include "ramp_tc.h"

namespace air {
air_status ramp_tc_create(air_plan *) {
    return fail(AIR_ERR_INVALID_ARG, "AIR_PREC_BF16X3 is not available in this build");
}
void ramp_tc_destroy(air_plan *) {}
air_status ramp_tc_apply(const air_plan *, const float *, float *, const CgState *, int, cudaStream_t) {
    return fail(AIR_ERR_INVALID_ARG, "AIR_PREC_BF16X3 is not available in this build");
}
}  // namespace air

// Ramp filtration C on the tensor cores (tcgen05, split BF16), AIR_PREC_BF16X3.
#pragma once

#include "host_common.h"

namespace air {
// Allocates the pre-split Toeplitz operand and the split-sinogram buffer.
air_status ramp_tc_create(air_plan *P);
void ramp_tc_destroy(air_plan *P);
// dst = C src for all views of the plan; when respect_stop, does nothing if
// cg->stop is set (the CG of this outer step has ended).
air_status ramp_tc_apply(const air_plan *P, const float *src, float *dst, const CgState *cg,
                         int respect_stop, cudaStream_t st);
// The plan's tensor-core status word (0, or AIR_ERR_TIMEOUT after a bounded
// wait gave up), cleared once read; synchronous.
int ramp_tc_status(const air_plan *P);
// Poll budget of the first pipeline wait of the tensor-core GEMM on the
// current device (negative: the default); the waits that drain a CTA's own
// copies and MMAs before it exits keep the default.  Synchronous.
cudaError_t ramp_tc_set_wait_budget(long long polls);
}  // namespace air

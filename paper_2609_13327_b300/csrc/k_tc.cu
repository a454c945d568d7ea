// Tensor-core left inverse (ZL_MIXED).  Placeholder until the tcgen05 kernel lands:
// tc_prepare reports ZL_ERR_UNSUPPORTED and the plan runs the FP32 CUDA-core passes.
#include "zl_internal.cuh"

namespace zl {

zl_status tc_prepare(zl_plan_s&, cudaStream_t) { return ZL_ERR_UNSUPPORTED; }
void tc_release(zl_plan_s&) {}
cudaError_t forward_tc(const zl_plan_s&, const float*, float*, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace zl

// Fused FP32 OLS kernels for N = 512 (see ols_fp32.cuh).
#include "ols_fp32.cuh"

namespace vbw {
VBW_INSTANTIATE_OLS(512)
}  // namespace vbw

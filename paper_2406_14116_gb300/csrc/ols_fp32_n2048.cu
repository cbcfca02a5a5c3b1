// Fused FP32 OLS kernels for N = 2048 (see ols_fp32.cuh).
#include "ols_fp32.cuh"

namespace vbw {
VBW_INSTANTIATE_OLS(2048)
}  // namespace vbw

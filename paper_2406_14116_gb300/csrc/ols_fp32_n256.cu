// Fused FP32 OLS kernels for N = 256 (see ols_fp32.cuh).
#include "ols_fp32.cuh"

namespace vbw {
VBW_INSTANTIATE_OLS(256)
}  // namespace vbw

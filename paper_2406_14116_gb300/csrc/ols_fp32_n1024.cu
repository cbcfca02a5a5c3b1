// Fused FP32 OLS kernels for N = 1024 (see ols_fp32.cuh).
#include "ols_fp32.cuh"

namespace vbw {
VBW_INSTANTIATE_OLS(1024)
}  // namespace vbw

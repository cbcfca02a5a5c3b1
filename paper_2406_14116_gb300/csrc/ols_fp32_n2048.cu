// Fused FP32 OLS kernels for N = 2048 (see ols_fp32.cuh): the single-warp kernel for any even
// overlap, and the warp-pair kernel (ols_pair.cuh) for overlap N/4.
#include "ols_pair.cuh"

namespace vbw {
VBW_INSTANTIATE_OLS(2048)
template cudaError_t launch_ols_pair_w<4, false>(const OlsArgs&, int, int, cudaStream_t, int*);
template cudaError_t launch_ols_pair_w<4, true>(const OlsArgs&, int, int, cudaStream_t, int*);
template cudaError_t launch_ols_pair_w<8, false>(const OlsArgs&, int, int, cudaStream_t, int*);
template cudaError_t launch_ols_pair_w<8, true>(const OlsArgs&, int, int, cudaStream_t, int*);

cudaError_t launch_export_hr_pair(const float* V, int LV, int k1, float* out, cudaStream_t st)
{
    export_hr_pair_kernel<<<1, 64, 0, st>>>(V, LV, k1, out);
    return cudaGetLastError();
}
}  // namespace vbw

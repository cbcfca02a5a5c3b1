// Mixed-plan persistent OLS kernel (see ols_mixed_kernel in ols_fp32.cuh): one launch over a
// batch whose signals use different N (overlap N/4). MAXN = 1024 covers N = 128..1024; a batch that
// also holds N = 2048 runs that plan in its own single-plan kernel beside it.
#include "ols_fp32.cuh"

namespace vbw {

cudaError_t launch_ols_mixed(const MixedArgs& a, int maxn, int warps, int sms, int max_ctas,
                             cudaStream_t st, int* grid_out)
{
    const size_t smem = (size_t)a.tw_bytes + (size_t)warps * a.warp_bytes;
    if (maxn <= 1024) {
        switch (warps) {
        case 4: return launch_persistent(ols_mixed_kernel<1024, 4>, 4, smem, a.ntiles, sms, max_ctas, st, grid_out, &a);
        case 8: return launch_persistent(ols_mixed_kernel<1024, 8>, 8, smem, a.ntiles, sms, max_ctas, st, grid_out, &a);
        default: return cudaErrorInvalidValue;
        }
    }
    return launch_persistent(ols_mixed_kernel<2048, 4>, 4, smem, a.ntiles, sms, max_ctas, st, grid_out, &a);
}

// Per-warp shared bytes of the largest transform in a mixed launch.
size_t ols_warp_bytes(int N)
{
    switch (N) {
    case 128: return OlsGeom<128>::WARP_BYTES;
    case 256: return OlsGeom<256>::WARP_BYTES;
    case 512: return OlsGeom<512>::WARP_BYTES;
    case 1024: return OlsGeom<1024>::WARP_BYTES;
    case 2048: return OlsGeom<2048>::WARP_BYTES;
    default: return 0;
    }
}

}  // namespace vbw

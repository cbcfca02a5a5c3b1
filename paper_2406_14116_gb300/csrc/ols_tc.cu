// Tensor-core (tcgen05) OLS kernels for N = 256 and 512 (overlap N/4), their per-plan tables, and
// a GEMM test hook that checks the UMMA operand layout against a host GEMM.
#include <atomic>
#include <cuda_runtime.h>

#include <cstdlib>
#include <vector>

#include "ols_tc.cuh"
#include "vbw.h"

namespace vbw {

template <int N, int PREC, bool BATCH>
static cudaError_t launch_tc_w(const OlsArgs& a, int sms, cudaStream_t st)
{
    using G = TcSmem<N, PREC>;
    auto kern = ols_tc_kernel<N, PREC, BATCH>;
    cudaError_t e = ensure_smem_limit((const void*)kern, G::BYTES);
    if (e != cudaSuccess) return e;
    // Resident CTAs per SM, from the SM's shared memory, registers and threads. (The occupancy
    // calculator reports one CTA per SM for this kernel, while four fit and run concurrently:
    // measured 43 -> 127 Gsamples/s for BF16 x3 at N = 256.) VBW_TC_CTAS (1..8) overrides it. At
    // most the TMEM columns of one SM allow: every CTA holds kTcTmemCols. Worked out once per
    // device (the runtime queries cost microseconds per launch).
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    static std::atomic<int> fits[64];
    int per_sm = (dev >= 0 && dev < 64) ? fits[dev].load(std::memory_order_relaxed) : 0;
    if (per_sm == 0) {
        int smem_sm = 0, smem_rsv = 0;
        cudaFuncAttributes fa;
        if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess ||
            (e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess)
            return e;
        per_sm = smem_sm / (int)(G::BYTES + smem_rsv);
        const int regs = ((fa.numRegs + 7) / 8) * 8 * kTcThreads;
        if (regs > 0 && 65536 / regs < per_sm) per_sm = 65536 / regs;
        if (2048 / kTcThreads < per_sm) per_sm = 2048 / kTcThreads;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        if (dev >= 0 && dev < 64) fits[dev].store(per_sm, std::memory_order_relaxed);
    }
    static const int env_ctas = [] {
        const char* v = getenv("VBW_TC_CTAS");
        const int c = v ? atoi(v) : 0;
        return (c >= 1 && c <= 8) ? c : 0;
    }();
    if (env_ctas) per_sm = env_ctas;
    if (per_sm > 512 / kTcTmemCols) per_sm = 512 / kTcTmemCols;
    int64_t grid = (int64_t)per_sm * sms;
    if (grid > a.ntiles) grid = a.ntiles;
    if (grid <= 0) return cudaSuccess;
    kern<<<(int)grid, kTcThreads, G::BYTES, st>>>(a);
    return cudaGetLastError();
}

// prec: 1 = BF16 x3, 2 = FP16 scaled, 3 = BF16 x6
cudaError_t launch_ols_tc(int N, int prec, const OlsArgs& a, int sms, cudaStream_t st)
{
    const bool b = a.jobs != nullptr;
#define VBW_TC_CASE(NN, PP)                                                                     \
    if (N == NN && prec == PP)                                                                  \
        return b ? launch_tc_w<NN, PP, true>(a, sms, st) : launch_tc_w<NN, PP, false>(a, sms, st);
    VBW_TC_CASE(256, kTcBf16x3)
    VBW_TC_CASE(256, kTcFp16s)
    VBW_TC_CASE(256, kTcBf16x6)
    VBW_TC_CASE(512, kTcBf16x3)
    VBW_TC_CASE(512, kTcFp16s)
    VBW_TC_CASE(512, kTcBf16x6)
#undef VBW_TC_CASE
    return cudaErrorInvalidValue;
}

size_t tc_table_bytes(int N, int prec)
{
#define VBW_TC_BYTES(NN, PP) if (N == NN && prec == PP) return TcSmem<NN, PP>::TABLE_BYTES;
    VBW_TC_BYTES(256, kTcBf16x3)
    VBW_TC_BYTES(256, kTcFp16s)
    VBW_TC_BYTES(256, kTcBf16x6)
    VBW_TC_BYTES(512, kTcBf16x3)
    VBW_TC_BYTES(512, kTcFp16s)
    VBW_TC_BYTES(512, kTcBf16x6)
#undef VBW_TC_BYTES
    return 0;
}

cudaError_t build_tc_table(int N, int prec, unsigned char* out, cudaStream_t st)
{
    const int n = (2 * 32) * (2 * 32) + 2 * (2 * 16) * (2 * 16) + 2048;   // covers matrix entries and twiddles
#define VBW_TC_TAB(NN, PP)                                                                      \
    if (N == NN && prec == PP) {                                                                \
        tc_table_kernel<NN, PP><<<(n + 255) / 256, 256, 0, st>>>(out);                          \
        return cudaGetLastError();                                                              \
    }
    VBW_TC_TAB(256, kTcBf16x3)
    VBW_TC_TAB(256, kTcFp16s)
    VBW_TC_TAB(256, kTcBf16x6)
    VBW_TC_TAB(512, kTcBf16x3)
    VBW_TC_TAB(512, kTcFp16s)
    VBW_TC_TAB(512, kTcBf16x6)
#undef VBW_TC_TAB
    return cudaErrorInvalidValue;
}

// ---- GEMM test: D (128 x NN) = A (128 x K) B (K x NN) with one rounding of A and B to 16 bits,
// through the same descriptors, instruction descriptor, TMEM load and waits the OLS kernel uses.
// flags: bit 0 BF16 (else FP16); bit 1 A in MN-major core matrices (as rounds 2 and 4 of the OLS
// kernel take it), else K-major. Both layouts use 128 bytes between core matrices along K and
// K/8 * 128 bytes between them along the rows (the descriptor's leading and stride offsets).
template <bool BF16>
__global__ void __launch_bounds__(128) tc_gemm_test_kernel(const float* A, const float* B, float* D, int K,
                                                             int NN, int flags, int* status)
{
    using H = Half16<BF16>;
    using T16 = typename H::T;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* As = sm;                          // 128 x K
    unsigned char* Bs = sm + 128 * 64 * 2;           // NN x K (B stored K-major: row n = column n of B)
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 128 * 64 * 2 + 64 * 64 * 2);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const bool a_mn = (flags & 2) != 0;
    for (int k = 0; k < K; ++k) {
        const uint32_t off = a_mn ? mn_line_offset(tid & ~7, k, K) + (tid & 7) * 2 : core_offset(tid, k, K);
        *reinterpret_cast<T16*>(As + off) = H::from(A[tid * K + k]);
    }
    if (tid < NN)
        for (int k = 0; k < K; ++k)
            *reinterpret_cast<T16*>(Bs + core_offset(tid, k, K)) = H::from(B[k * NN + tid]);
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(tslot, 64);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        const uint32_t idesc = umma_idesc(BF16, 128, NN) | (a_mn ? (1u << 15) : 0u);
        const uint32_t sbo = (uint32_t)(K / 8) * 128;
        for (int s = 0; s < K / 16; ++s)
            umma_f16(tmem, umma_desc(As + s * 256, 128, sbo), umma_desc(Bs + s * 256, 128, sbo), idesc,
                     s > 0 ? 1u : 0u);
        umma_commit(bar);
    }
    bool ok = mbar_wait_bounded(bar, 0, kWaitLimitCycles);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicOr(status, kStatusWaitTimeout);
        mbar_wait_bounded(bar, 0, kWaitLimitCycles);
    } else {
        tc_fence_after_sync();
        for (int c = 0; c < NN; c += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
            for (int i = 0; i < 32; ++i) D[tid * NN + c + i] = v[i];
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 64);
}

}  // namespace vbw

namespace vbw {
vbw_status set_error(vbw_status st, const char* msg);
}

extern "C" vbw_status vbw_debug_tc_gemm(int flags, int K, int NN, const float* A, const float* B, float* D)
{
    using namespace vbw;
    if ((K != 32 && K != 64) || (NN != 32 && NN != 64) || !A || !B || !D)
        return set_error(VBW_ERR_INVALID_ARG, "K and NN must be 32 or 64; A, B, D non-NULL");
    float *dA = nullptr, *dB = nullptr, *dD = nullptr;
    int* dS = nullptr;
    const size_t smem = 128 * 64 * 2 + 64 * 64 * 2 + 64;
    cudaError_t e = cudaMalloc(&dA, sizeof(float) * 128 * K);
    if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(float) * K * NN);
    if (e == cudaSuccess) e = cudaMalloc(&dD, sizeof(float) * 128 * NN);
    if (e == cudaSuccess) e = cudaMalloc(&dS, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(dA, A, sizeof(float) * 128 * K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, B, sizeof(float) * K * NN, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dS, 0, sizeof(int));
    if (e == cudaSuccess) {
        if (flags & 1) {
            e = cudaFuncSetAttribute(tc_gemm_test_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) tc_gemm_test_kernel<true><<<1, 128, smem>>>(dA, dB, dD, K, NN, flags, dS);
        } else {
            e = cudaFuncSetAttribute(tc_gemm_test_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) tc_gemm_test_kernel<false><<<1, 128, smem>>>(dA, dB, dD, K, NN, flags, dS);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(D, dD, sizeof(float) * 128 * NN, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&st, dS, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(dS);
    if (e != cudaSuccess) return set_error(VBW_ERR_CUDA, cudaGetErrorString(e));
    if (st) return set_error(VBW_ERR_TIMEOUT, "tensor-core GEMM did not complete");
    return set_error(VBW_OK, "");
}

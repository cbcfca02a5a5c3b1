// vbw_filter_static: whole-signal OLS VBW filtering that allocates nothing.
//
// Some callers cannot allocate device memory. A host framework may own every device allocation
// through its own pool. A real-time loop cannot afford cudaMalloc's implicit device
// synchronization and unbounded latency. Code may run where the CUDA allocator must not be
// touched. The usual path needs a plan (its twiddle rows and transition table live in memory
// that vbw_plan allocates). This entry point keeps those tables in
// one fixed array of device memory that is part of the library image. Every GPU that loads the
// library holds that array until the process exits.
//
// The kernels are those of every other path (ols_fp32_kernel, and for N = 2048 with overlap N/4 the
// split kernel of ols_split2048.cu), in their single-job form.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "ols_fp32.cuh"
#include "vbw.h"

// Plan-time table kernels of vbw_api.cu.
__global__ void vbw_twiddle_kernel(float2* tw, int N, int T, int E);
__global__ void vbw_halfphase_kernel(float2* ph, int N);

namespace vbw {
template <int N>
cudaError_t launch_ols_fp32(const OlsArgs& a, int warps, int sms, int max_ctas, cudaStream_t st,
                            int* grid_out);
vbw_status set_error(vbw_status st, const char* msg);   // vbw_last_error() text (vbw_api.cu)
int split2048_choice(int64_t ntiles, int sms);           // vbw_api.cu
int split2048_table_entries();                           // ols_split2048.cu
cudaError_t build_split2048_table(float2* tw, cudaStream_t st);
cudaError_t launch_ols_split2048(const OlsArgs& a, int warps, int sms, int max_ctas, cudaStream_t st,
                                 int* grid_out);
}  // namespace vbw

namespace {

// Layout of the scratch (bytes). Sized for the largest plan the library accepts (N = 2048,
// L_V = N/2 - 2), so every valid request fits.
constexpr size_t kTwOff = 0;           // twiddle rows: at most 32 x 66 float2 = 16896 bytes, then
constexpr size_t kTwCap = 49152;       // for N = 2048, overlap N/4, the split kernel's 26112 bytes
constexpr size_t kVOff = kTwOff + kTwCap;    // transition table, float32: at most 4088 bytes
constexpr size_t kVCap = 8192;
constexpr size_t kScratchBytes = 64 * 1024;      // the whole array: 64 KiB per GPU
constexpr int kMaxLV = 1022;                     // N / 2 - 2 at N = 2048
static_assert(kVOff + kVCap <= kScratchBytes, "scratch layout exceeds the array");
static_assert(sizeof(float) * kMaxLV <= kVCap, "transition table exceeds its share");

static __device__ __align__(256) unsigned char vbw_static_scratch[kScratchBytes];

// The transition table travels to the GPU inside the launch parameters (8 KiB of the 32 KiB a
// launch may carry): no copy from pageable host memory, so the call never waits on the host.
struct StaticV {
    double v[kMaxLV];
};

__global__ void static_round_v_kernel(const StaticV p, int LV, float* Vf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < LV) Vf[i] = (float)p.v[i];
}

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_scratch[kMaxDevices] = {};   // device address of the scratch, per device

// What the scratch of each device holds (the last call's geometry and table), so that a call
// with the same ones enqueues no table kernels.
struct TableKey {
    int N = 0, overlap = 0, LV = 0;
    double V[kMaxLV];
};
TableKey g_key[kMaxDevices];

vbw_status fail_static(vbw_status st, const char* msg) { return vbw::set_error(st, msg); }

// Device address of this device's scratch. The first call on a device looks it up, with the
// device current; later calls reuse it.
vbw_status scratch_address(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail_static(VBW_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, vbw_static_scratch);
        if (e != cudaSuccess || !p) return fail_static(VBW_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        g_scratch[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch[dev];
    return VBW_OK;
}

int layout_T_of(int N) { return vbw::layout_T(N); }

}  // namespace

extern "C" vbw_status vbw_filter_static(int N, int overlap, const double* V, int LV, int band,
                                        const void* in, void* out, int64_t nsamples,
                                        void* cuda_stream)
{
    using namespace vbw;
    if (N < 128 || N > 2048 || (N & (N - 1)))
        return fail_static(VBW_ERR_INVALID_ARG, "N must be a power of two in [128, 2048]");
    if (overlap <= 0 || overlap >= N)
        return fail_static(VBW_ERR_INVALID_ARG, "overlap must be in (0, N)");
    if (LV < 1 || LV > N / 2 - 2) return fail_static(VBW_ERR_INVALID_ARG, "L_V must be in [1, N/2-2]");
    if (!V) return fail_static(VBW_ERR_INVALID_ARG, "transition_samples is NULL");
    if (band < 1 || band > N / 2 - LV - 1) return fail_static(VBW_ERR_BAND_RANGE, "band outside [1, N/2-L_V-1]");
    if (nsamples < 0) return fail_static(VBW_ERR_INVALID_ARG, "nsamples < 0");
    const int T = layout_T_of(N), E = N / T;
    const bool split = (N == 2048 && overlap == N / 4);   // the split kernel's tables follow the rows
    const size_t tw_bytes = sizeof(float2) * ((size_t)T * (E + 2) + ((overlap & 1) ? half_phase_entries(N) : 0) +
                                              (split ? split2048_table_entries() : 0));
    if (tw_bytes > kTwCap || LV > kMaxLV)
        return fail_static(VBW_ERR_INVALID_ARG, "request exceeds the static scratch (64 KiB)");
    if (nsamples == 0) return vbw::set_error(VBW_OK, "");
    if (!in || !out) return fail_static(VBW_ERR_INVALID_ARG, "in/out is NULL");
    if (((uintptr_t)in & 7) || ((uintptr_t)out & 7))
        return fail_static(VBW_ERR_INVALID_ARG, "in/out not 8-byte aligned");
    {
        const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out, n = sizeof(float2) * (uintptr_t)nsamples;
        if (a < b + n && b < a + n) return fail_static(VBW_ERR_INVALID_ARG, "in and out overlap");
    }

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail_static(VBW_ERR_CUDA, "no usable CUDA device");
    unsigned char* scratch = nullptr;
    vbw_status st = scratch_address(dev, &scratch);
    if (st != VBW_OK) return st;
    float2* tw = reinterpret_cast<float2*>(scratch + kTwOff);
    float* Vf = reinterpret_cast<float*>(scratch + kVOff);
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // tables of this call, unless the scratch already holds them (same geometry and table)
    {
        std::lock_guard<std::mutex> lk(g_mu);
        TableKey& k = g_key[dev];
        const bool same = k.N == N && k.overlap == overlap && k.LV == LV &&
                          memcmp(k.V, V, sizeof(double) * (size_t)LV) == 0;
        if (!same) {
            k.N = 0;   // invalid until every table kernel is enqueued
            StaticV pv;
            memcpy(pv.v, V, sizeof(double) * (size_t)LV);
            const int tw_entries = T * (E + 2);
            vbw_twiddle_kernel<<<(tw_entries + 255) / 256, 256, 0, s>>>(tw, N, T, E);
            if (overlap & 1)
                vbw_halfphase_kernel<<<(half_phase_entries(N) + 255) / 256, 256, 0, s>>>(tw + tw_entries, N);
            if (split && build_split2048_table(tw + tw_entries, s) != cudaSuccess)
                return fail_static(VBW_ERR_CUDA, "table kernels failed");
            static_round_v_kernel<<<(LV + 255) / 256, 256, 0, s>>>(pv, LV, Vf);
            if (cudaGetLastError() != cudaSuccess) return fail_static(VBW_ERR_CUDA, "table kernels failed");
            k.N = N;
            k.overlap = overlap;
            k.LV = LV;
            memcpy(k.V, V, sizeof(double) * (size_t)LV);
        }
    }

    OlsArgs a;
    memset(&a, 0, sizeof(a));
    a.job.in = static_cast<const float2*>(in);
    a.job.out = static_cast<float2*>(out);
    a.job.nsamp = nsamples;
    a.job.band0 = band;
    const int64_t M = N - overlap;
    const int64_t nblocks = (nsamples + M - 1) / M;
    const int B = 32 / T;
    a.ntiles = (nblocks + B - 1) / B;
    a.tw = tw;
    a.V = Vf;
    a.overlap = overlap;
    a.LV = LV;
    const int warps = 8;
    int grid = 0;
    cudaError_t e;
    switch (N) {
    case 128: e = launch_ols_fp32<128>(a, warps, sms, 0, s, &grid); break;
    case 256: e = launch_ols_fp32<256>(a, warps, sms, 0, s, &grid); break;
    case 512: e = launch_ols_fp32<512>(a, warps, sms, 0, s, &grid); break;
    case 1024: e = launch_ols_fp32<1024>(a, warps, sms, 0, s, &grid); break;
    default: {
        const int sw = split ? split2048_choice(a.ntiles, sms) : 0;
        e = sw ? launch_ols_split2048(a, sw, sms, 0, s, &grid) : launch_ols_fp32<2048>(a, warps, sms, 0, s, &grid);
        break;
    }
    }
    if (e != cudaSuccess) return fail_static(VBW_ERR_CUDA, "filter launch failed");
    return vbw::set_error(VBW_OK, "");
}

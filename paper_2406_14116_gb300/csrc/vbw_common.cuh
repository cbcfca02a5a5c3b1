// Shared device-side definitions of libvbw: work descriptors, compile-time trigonometry and the
// per-N thread layout of the fused OLS kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

namespace vbw {

// ---------------------------------------------------------------------------------------------
// Compile-time unrolling helper: calls f(std::integral_constant<int, i>) for i = B, B+S, ... < E.
template <int B, int E, int S = 1, class F>
__host__ __device__ __forceinline__ constexpr void static_for(F&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + S, E, S>(f);
    }
}

// ---------------------------------------------------------------------------------------------
// Compile-time cos/sin of 2*pi*p/q for the constant twiddles inside the register DFT codelets.
// The angle is folded into [0, pi/4] with exact integer symmetries (f -> 1-f, 1/2-f, 1/4-f),
// then evaluated with the Maclaurin series in double precision and rounded to float once at the
// point of use. (The run-time twiddle tables are generated on the GPU in FP64 instead.)
struct CosSin {
    double c, s;
};

constexpr double kPi = 3.141592653589793238462643383279502884;

constexpr double maclaurin_cos(double x)
{
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 24; ++i) {
        term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
        sum += term;
    }
    return sum;
}

constexpr double maclaurin_sin(double x)
{
    double term = x, sum = x;
    for (int i = 1; i < 24; ++i) {
        term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
        sum += term;
    }
    return sum;
}

constexpr CosSin cos_sin_2pi(long p, long q)
{
    p %= q;
    if (p < 0) p += q;
    bool neg_s = false, neg_c = false, swap = false;
    if (2 * p > q) { p = q - p; neg_s = true; }             // 1 - f: sin changes sign
    if (4 * p > q) { p = q - 2 * p; q = 2 * q; neg_c = true; }  // 1/2 - f: cos changes sign
    if (8 * p > q) { p = q - 4 * p; q = 4 * q; swap = true; }   // 1/4 - f: sin <-> cos
    const double x = 2.0 * kPi * static_cast<double>(p) / static_cast<double>(q);
    double c = maclaurin_cos(x), s = maclaurin_sin(x);
    if (swap) { const double t = c; c = s; s = t; }
    if (neg_c) c = -c;
    if (neg_s) s = -s;
    return CosSin{c, s};
}

// ---------------------------------------------------------------------------------------------
// Thread layout of the fused FP32 OLS kernel for each N (see ols_fp32.cuh):
//   T threads cooperate on one block, each holding E = N/T samples; N = E * T with T | E.
//   Pass 1 is an E-point register DFT per thread, pass 2 does E/T T-point register DFTs per
//   thread after a shared-memory transpose. 32/T blocks share one warp.
template <int N>
struct Layout;
template <> struct Layout<128>  { static constexpr int E = 16, T = 8;  };
template <> struct Layout<256>  { static constexpr int E = 16, T = 16; };
template <> struct Layout<512>  { static constexpr int E = 32, T = 16; };
template <> struct Layout<1024> { static constexpr int E = 32, T = 32; };
template <> struct Layout<2048> { static constexpr int E = 64, T = 32; };

// Entries (float2) of the half-sample phase table of an odd-overlap plan: exp(-j pi kk / N) for
// kk = 0..N/2, padded to an even count.
__host__ __device__ constexpr int half_phase_entries(int N) { return N / 2 + 2; }

// Host mirror of Layout<N>::T (the twiddle table layout depends on it).
inline int layout_T(int N)
{
    switch (N) {
    case 128: return 8;
    case 256: return 16;
    case 512: return 16;
    case 1024: return 32;
    case 2048: return 32;
    default: return 0;
    }
}

// ---------------------------------------------------------------------------------------------
// Work descriptors.

// One stream segment filtered by a launch. Block m of the job reads x(mM - O .. mM + M - 1) of
// the segment (negative indices come from tail_in, or zeros) and writes y(mM .. mM + M - 1).
struct OlsJob {
    const float2* in;      // device, nsamp samples
    float2* out;           // device, nsamp samples
    const float2* tail_in; // device, O samples preceding in[0]; nullptr = zeros
    float2* tail_out;      // device, receives the last O samples of tail_in ++ in; nullptr = none
    const int32_t* band;   // device, k1 per block; nullptr = band0 (plus inline changes)
    int64_t nsamp;
    int32_t band0;
    int32_t plan;          // index into MixedArgs::plans (mixed launches; 0 otherwise)
};

constexpr int kInlineChanges = 16;

struct OlsArgs {
    const OlsJob* jobs;   // device job array (batch mode); nullptr = single job `job`
    const int2* tiles;    // device: per warp-tile (job index, first block); batch mode only
    int64_t ntiles;       // warp-tiles in this launch
    OlsJob job;           // single-job mode
    int32_t nchg;         // single-job mode: inline band changes (block, band), sorted by block
    int32_t chg_band[kInlineChanges];
    int64_t chg_block[kInlineChanges];
    const float2* tw;     // device twiddle table: row t holds W_N^{t ka}, ka < E, padded to E + 2
    const float* V;       // device transition samples, L_V floats
    int32_t overlap;
    int32_t LV;
    int* status;          // device status word (bit flags, e.g. a bounded wait that gave up) or nullptr
    int64_t wait_limit;   // bound of device-side waits in SM cycles (0 = default, about 2 s)
    int32_t debug;        // test hook, bit 0: the tensor-core kernel issues no MMAs (its waits run out)
    int32_t flags;        // kOlsNoBulk: signals live in host memory, use plain loads and stores only;
                          // kOlsReal: real signals (float32), processed as pairs of blocks
    const unsigned char* tc_tables;   // tensor-core plans: DFT-matrix pieces and twiddles
};

constexpr int kOlsNoBulk = 1;
constexpr int kOlsReal = 2;   // the jobs' signals are real float32: blocks go through in pairs

// One plan of a mixed-plan launch (overlap N/4).
struct MixedPlan {
    const float2* tw;     // device twiddle rows of this plan
    const float* V;       // device transition samples
    int32_t N, LV;
    int32_t tw_off;       // offset of the rows in shared memory (float2 units, 16-byte aligned)
    int32_t tw_len;       // number of float2 entries
};

constexpr int kMaxMixedPlans = 8;

struct MixedArgs {
    const OlsJob* jobs;   // jobs grouped by plan
    const int2* tiles;    // per warp-tile (job index, first block)
    int64_t ntiles;
    MixedPlan plans[kMaxMixedPlans];
    int32_t nplans;
    int32_t tw_bytes;     // shared bytes of all twiddle rows
    int32_t warp_bytes;   // per-warp region (largest N of the launch)
    int32_t flags;        // as OlsArgs::flags
};

// ---------------------------------------------------------------------------------------------
// Launch preparation of the persistent kernels (host). Raising a kernel's dynamic shared-memory
// limit and asking how many CTAs fit per SM are two runtime calls that cost microseconds, most of
// a small launch. Both answers are kept per (device, kernel, block size, shared memory). A
// kernel's limit only ever rises, so a launch prepared earlier with more shared memory stays
// valid. The state belongs to the devices' current contexts, like the plans: a device reset
// invalidates both.
struct LaunchPrep {
    int dev;
    const void* kern;
    int threads;
    size_t smem;
    int per_sm;
};

struct SmemLimit {
    int dev;
    const void* kern;
    size_t smem;
};

inline std::mutex& launch_prep_mutex()
{
    static std::mutex mu;
    return mu;
}

// Raises kern's dynamic shared-memory limit on the current device to at least smem.
inline cudaError_t ensure_smem_limit(const void* kern, size_t smem)
{
    static std::vector<SmemLimit> limits;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(launch_prep_mutex());
    SmemLimit* lim = nullptr;
    for (SmemLimit& l : limits)
        if (l.dev == dev && l.kern == kern) lim = &l;
    if (lim && lim->smem >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (lim) lim->smem = smem;
    else limits.push_back(SmemLimit{dev, kern, smem});
    return cudaSuccess;
}

// CTAs of `threads` threads with `smem` dynamic shared memory that fit per SM, the limit raised.
inline cudaError_t prepared_occupancy(const void* kern, int threads, size_t smem, int* per_sm)
{
    static std::vector<LaunchPrep> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(launch_prep_mutex());
        for (const LaunchPrep& c : cache)
            if (c.dev == dev && c.kern == kern && c.threads == threads && c.smem == smem) {
                *per_sm = c.per_sm;
                return cudaSuccess;
            }
    }
    if ((e = ensure_smem_limit(kern, smem)) != cudaSuccess) return e;
    int n = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(launch_prep_mutex());
    cache.push_back(LaunchPrep{dev, kern, threads, smem, n});
    *per_sm = n;
    return cudaSuccess;
}

}  // namespace vbw

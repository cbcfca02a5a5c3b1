// libvbw host side: the C ABI of include/vbw.h. Plans, streams, batches, validation and launches.
// Every filtering step runs in the CUDA kernels of ols_fp32.cuh; this file only prepares
// descriptors and enqueues work.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "vbw.h"
#include "vbw_common.cuh"
#include "vbw_internal.h"

namespace vbw {
template <int N>
cudaError_t launch_ols_fp32(const OlsArgs& a, int warps, int sms, int max_ctas, cudaStream_t st,
                            int* grid_out);
template <int N>
cudaError_t launch_export_hr(const float* V, int LV, int k1, float* out, cudaStream_t st);
cudaError_t launch_ols_mixed(const MixedArgs& a, int maxn, int warps, int sms, int max_ctas,
                             cudaStream_t st, int* grid_out);
size_t ols_warp_bytes(int N);
cudaError_t launch_ols_tc(int N, int prec, const OlsArgs& a, int sms, cudaStream_t st);
size_t tc_table_bytes(int N, int prec);
cudaError_t build_tc_table(int N, int prec, unsigned char* out, cudaStream_t st);
int split2048_table_entries();
int split2048_choice(int64_t ntiles, int sms);
cudaError_t launch_split2048_export_hr(const float* V, int LV, int k1, float* out, cudaStream_t st);
cudaError_t build_split2048_table(float2* tw, cudaStream_t st);
cudaError_t launch_ols_split2048(const OlsArgs& a, int warps, int sms, int max_ctas, cudaStream_t st,
                                 int* grid_out);
constexpr int kTcTileBlocks = 8;
}  // namespace vbw

using namespace vbw;

// ------------------------------------------------------------------------------------------------
// errors

static thread_local std::string g_last_error;

vbw_status fail(vbw_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define VBW_CUDA(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(VBW_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));        \
    } while (0)

vbw_status ok()
{
    g_last_error.clear();
    return VBW_OK;
}

namespace vbw {
vbw_status set_error(vbw_status st, const char* msg)
{
    g_last_error = msg;
    return st;
}
}  // namespace vbw

extern "C" const char* vbw_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* vbw_version(void) { return "libvbw 0.1 (sm_103a)"; }

// ------------------------------------------------------------------------------------------------
// device-side table generation (FP64 on the GPU, rounded once to FP32)

// tw[n2*(E+2) + ka] = exp(-j 2 pi (n2 ka mod N) / N) for ka < E (pad entries 0): the four-step
// twiddle of the fused kernel, one row per thread n2.
__global__ void vbw_twiddle_kernel(float2* tw, int N, int T, int E)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = E + 2;
    if (idx >= T * row) return;
    const int n2 = idx / row, ka = idx % row;
    if (ka >= E) {
        tw[idx] = make_float2(0.f, 0.f);
        return;
    }
    const long long j = ((long long)n2 * (long long)ka) % N;
    double s, c;
    sincospi(-2.0 * (double)j / (double)N, &s, &c);
    tw[idx] = make_float2((float)c, (float)s);
}

// Half-sample phase of an odd-overlap plan: ph[kk] = exp(-j pi kk / N), kk = 0..N/2, in FP64
// rounded once (the exp(-j 2 pi k_s (O/2) / N) of eq. (FS_Hk_exp) past its whole-sample shift).
__global__ void vbw_halfphase_kernel(float2* ph, int N)
{
    const int kk = blockIdx.x * blockDim.x + threadIdx.x;
    if (kk >= half_phase_entries(N)) return;
    if (kk > N / 2) {
        ph[kk] = make_float2(0.f, 0.f);
        return;
    }
    double s, c;
    sincospi(-(double)kk / (double)N, &s, &c);
    ph[kk] = make_float2((float)c, (float)s);
}

__global__ void vbw_round_table_kernel(const double* Vd, float* Vf, int LV)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < LV) Vf[i] = (float)Vd[i];
}

// ------------------------------------------------------------------------------------------------
// objects


struct vbw_stream_s {
    vbw_plan_s* plan = nullptr;
    cudaStream_t st = nullptr;
    float2* d_tail[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t pos = 0;   // blocks submitted
    int band = 1;      // k1 in effect at block `pos` unless `pending` overrides it
    bool flushed = false;
    std::map<int64_t, int> pending;  // absolute block -> k1
    // host-buffer path (lazily created)
    cudaStream_t cp_in = nullptr, cp_out = nullptr;
    float2* d_stage[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int64_t stage_blocks = 0;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_k[2] = {nullptr, nullptr},
                ev_out[2] = {nullptr, nullptr};
};

struct BatchGroup {
    vbw_plan_s* plan = nullptr;
    OlsJob* d_jobs = nullptr;
    int2* d_tiles = nullptr;
    int64_t ntiles = 0;
    double cost = 0;                // transform work of the group (blocks x N log2 N)
    std::vector<int> sig;           // signal index of each job
    std::vector<int64_t> tile_off;  // first tile of each job (size jobs + 1)
};

struct vbw_batch_s {
    bool real = false;              // float32 signals, blocks in pairs (vbw_batch_create_real)
    std::vector<BatchGroup> groups;
    std::vector<vbw_signal> sigs;
    int32_t* d_bands = nullptr;
    int last_launches = 0;
    // mixed-plan launch over the groups that qualify (overlap N/4, N <= 1024)
    std::vector<int> mixed_groups;
    OlsJob* d_mjobs = nullptr;
    int2* d_mtiles = nullptr;
    MixedArgs margs;
    double mixed_cost = 0;
    int mode = VBW_BATCH_AUTO;
    double split = 0;               // share of the SMs for the mixed launch (0 = by cost)
    cudaStream_t s_side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // zero-copy runs from pinned host memory: job arrays with host addresses (per group, mixed)
    std::vector<OlsJob*> d_zjobs;
    OlsJob* d_zmjobs = nullptr;
    std::vector<const void*> z_in, z_out;   // host pointers the zero-copy arrays hold
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_start = nullptr, ev_h = nullptr, ev_c = nullptr, ev_done = nullptr;
};

// ------------------------------------------------------------------------------------------------
// process-wide tuning (CTA shapes), from vbw_tune_set or a tune cache

static std::mutex g_tune_mu;
static int g_tune_warps[5] = {0, 0, 0, 0, 0};   // N = 128 << i; 0 = default
static int g_tune_ctas[5] = {0, 0, 0, 0, 0};    // resident CTAs per SM cap; 0 = occupancy limit
static int g_wait_limit_debug = 0;               // test hook: tensor-core MMAs not issued, short waits
static int g_full_band_debug = 0;                // test hook: accept k1 = N/2 + 1 (H_R = 1)

static int n_index(int N)
{
    switch (N) {
    case 128: return 0;
    case 256: return 1;
    case 512: return 2;
    case 1024: return 3;
    case 2048: return 4;
    default: return -1;
    }
}

// ------------------------------------------------------------------------------------------------
// validation helpers (pure host logic: no CUDA call before the arguments are known to be valid)

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

vbw_status check_band(const vbw_plan_s* p, int band)
{
    const int kmax = p->N / 2 - p->LV - 1;
    // test hook: k1 = N/2 + 1 puts every bin in the passband (H_R = 1, the full-band identity)
    if (g_full_band_debug && band == p->N / 2 + 1) return VBW_OK;
    if (band < 1 || band > kmax)
        return fail(VBW_ERR_BAND_RANGE, "band k1=%d outside [1, %d] for N=%d, L_V=%d", band, kmax,
                    p->N, p->LV);
    return VBW_OK;
}

// complex64 samples need 8-byte alignment
bool misaligned(const void* p) { return ((uintptr_t)p & 7) != 0; }

static bool ranges_overlap(const void* a, const void* b, size_t bytes)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bytes && y < x + bytes;
}

static int env_int(const char* name, int dflt)
{
    const char* v = getenv(name);
    if (!v || !*v) return dflt;
    return atoi(v);
}

// Warps per CTA for each N: a tuned value (vbw_tune_set / tune cache), else VBW_WARPS (4 or 8),
// else the largest CTA whose register footprint keeps 16 resident warps per SM (N <= 1024) or
// 8 (N = 2048).
static int warps_for(int N)
{
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        const int i = n_index(N);
        if (i >= 0 && (g_tune_warps[i] == 4 || g_tune_warps[i] == 8)) return g_tune_warps[i];
    }
    const int w = env_int("VBW_WARPS", 0);
    if (w == 4 || w == 8) return w;
    // 8-warp CTAs measured fastest for every N on GB300, N = 2048 included (one 8-warp CTA per SM
    // at about 210 registers beat three 4-warp CTAs capped at 168 registers, which spill)
    return 8;
}

static int ctas_cap_for(int N, int sms)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int i = n_index(N);
    return (i >= 0 && g_tune_ctas[i] > 0) ? g_tune_ctas[i] * sms : 0;
}

// N = 2048 with overlap N/4 runs the split kernel (two 1024-point halves, one parked in tensor
// memory; ols_split2048.cu) when it is expected to finish first. A persistent launch lasts about as
// long as its busiest warp: ceil(tiles / warp slots) tiles. The four-step kernel has 8 warps per SM,
// the split kernel 12, and a split-kernel tile takes about 1.35 four-step tile times (its warps
// share an SM twelve ways; the ratio of the two kernels' large-launch throughputs, 195 / 176
// Gsamples/s, gives it). In a sweep of launch sizes (8, 16, 32, 48, 64, 128 and 512 channels of
// 2^16 samples) this estimate picked the faster kernel every time: the four-step kernel below one
// split wave (serving's batches) and just past a wave boundary, the split kernel otherwise and
// for large launches (10% faster at 512 channels).
// VBW_SPLIT2048=0 never runs it, =2 runs it for every size; VBW_SPLIT2048_WARPS picks 8, 12 or 16
// warps per CTA (one CTA per SM).
static bool split2048_enabled() { return env_int("VBW_SPLIT2048", 1) != 0; }

static bool split2048_for(int64_t ntiles, int sms, int warps)
{
    const int mode = env_int("VBW_SPLIT2048", 1);
    if (mode == 2) return true;
    if (mode == 0 || ntiles <= 0 || sms <= 0) return false;
    const int64_t slots4 = (int64_t)sms * 8, slots_s = (int64_t)sms * warps;
    const double t4 = (double)((ntiles + slots4 - 1) / slots4);
    const double ts = 1.35 * (warps / 12.0) * (double)((ntiles + slots_s - 1) / slots_s);
    return ts < t4;
}

static int split2048_warps()
{
    const int w = env_int("VBW_SPLIT2048_WARPS", 0);
    return (w == 8 || w == 12 || w == 16) ? w : 12;
}

// The same choice for callers outside this file (vbw_filter_static): warps per CTA of the split
// kernel, or 0 when the 64 x 32 four-step kernel runs, for a launch of ntiles tiles (ntiles < 0:
// whether the split kernel runs for some size, which decides the H_R export's layout).
int vbw::split2048_choice(int64_t ntiles, int sms)
{
    if (ntiles < 0) return split2048_enabled() ? split2048_warps() : 0;
    return split2048_for(ntiles, sms, split2048_warps()) ? split2048_warps() : 0;
}

static cudaError_t launch_fp32(int N, const OlsArgs& a, int sms, cudaStream_t st, int max_ctas = 0)
{
    int grid = 0;
    const int warps = warps_for(N);
    const int cap = ctas_cap_for(N, sms);
    if (cap > 0 && (max_ctas == 0 || cap < max_ctas)) max_ctas = cap;
    switch (N) {
    case 128: return launch_ols_fp32<128>(a, warps, sms, max_ctas, st, &grid);
    case 256: return launch_ols_fp32<256>(a, warps, sms, max_ctas, st, &grid);
    case 512: return launch_ols_fp32<512>(a, warps, sms, max_ctas, st, &grid);
    case 1024: return launch_ols_fp32<1024>(a, warps, sms, max_ctas, st, &grid);
    case 2048:
        if (a.overlap == 512 && !(a.flags & kOlsReal) && split2048_for(a.ntiles, sms, split2048_warps()))
            return launch_ols_split2048(a, split2048_warps(), sms, max_ctas, st, &grid);
        return launch_ols_fp32<2048>(a, warps, sms, max_ctas, st, &grid);
    default: return cudaErrorInvalidValue;
    }
}

// Kernel arguments common to every launch of plan p.
void fill_plan_args(OlsArgs& a, const vbw_plan_s* p)
{
    a.tw = p->d_tw;
    a.V = p->d_V;
    a.overlap = p->O;
    a.LV = p->LV;
    a.status = p->d_status;
    a.wait_limit = g_wait_limit_debug ? 2000000LL : 0;
    a.debug = g_wait_limit_debug ? 1 : 0;
    a.tc_tables = p->d_tc;
}

// Launch of plan p's kernel: the fused FP32 kernel, or the tensor-core one.
cudaError_t launch_plan(const vbw_plan_s* p, const OlsArgs& a, cudaStream_t st, int max_ctas)
{
    if (p->prec != VBW_PREC_FP32) return launch_ols_tc(p->N, p->prec, a, p->sms, st);
    return launch_fp32(p->N, a, p->sms, st, max_ctas);
}

static int blocks_per_warp(int N) { return 32 / layout_T(N); }

int tile_blocks(const vbw_plan_s* p)
{
    return p->prec == VBW_PREC_FP32 ? blocks_per_warp(p->N) : kTcTileBlocks;
}

// entries of the per-plan twiddle table: T rows of E + 2 (see OlsGeom::TW)
static int twiddle_entries(int N) { return layout_T(N) * (N / layout_T(N) + 2); }

// Entries of a plan's twiddle array: the four-step rows, the half-sample phases of an odd
// overlap, and for N = 2048 with overlap N/4 the split kernel's F2 tables.
static int plan_twiddle_entries(int N, int overlap)
{
    return twiddle_entries(N) + ((overlap & 1) ? half_phase_entries(N) : 0) +
           ((N == 2048 && overlap == N / 4) ? split2048_table_entries() : 0);
}

// ------------------------------------------------------------------------------------------------
// plans

extern "C" vbw_status vbw_plan(int N, int overlap, const double* V, int LV, int precision,
                               vbw_plan_t* out)
{
    if (!out) return fail(VBW_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!is_pow2(N) || N < 128 || N > 2048)
        return fail(VBW_ERR_INVALID_ARG, "N=%d: must be a power of two in [128, 2048]", N);
    if (overlap <= 0 || overlap >= N)
        return fail(VBW_ERR_INVALID_ARG, "overlap=%d: must be in (0, N)", overlap);
    if (LV < 1 || LV > N / 2 - 2)
        return fail(VBW_ERR_INVALID_ARG, "L_V=%d: must be in [1, N/2-2]", LV);
    if (!V) return fail(VBW_ERR_INVALID_ARG, "transition_samples is NULL");
    for (int i = 0; i < LV; ++i)
        if (!std::isfinite(V[i])) return fail(VBW_ERR_INVALID_ARG, "V[%d] is not finite", i);
    if (precision < VBW_PREC_FP32 || precision > VBW_PREC_BF16_SPLIT3)
        return fail(VBW_ERR_INVALID_ARG, "precision %d is not a known precision", precision);
    if (precision != VBW_PREC_FP32 && !((N == 256 || N == 512) && overlap == N / 4))
        return fail(VBW_ERR_UNSUPPORTED, "tensor-core precisions need N in {256, 512} and overlap N/4");

    vbw_plan_s* p = new (std::nothrow) vbw_plan_s();
    if (!p) return fail(VBW_ERR_NOMEM, "host allocation failed");
    p->N = N;
    p->O = overlap;
    p->M = N - overlap;
    p->LV = LV;
    p->prec = precision;
    p->V.assign(V, V + LV);
    vbw_status st = VBW_OK;
    double* d_Vd = nullptr;
    do {
        cudaError_t e;
        if ((e = cudaGetDevice(&p->device)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device)) !=
                cudaSuccess) {
            st = fail(VBW_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
            break;
        }
        const int tw_total = plan_twiddle_entries(N, overlap);
        if (cudaMalloc(&p->d_tw, sizeof(float2) * tw_total) != cudaSuccess ||
            cudaMalloc(&p->d_V, sizeof(float) * LV) != cudaSuccess ||
            cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess ||
            cudaMalloc(&d_Vd, sizeof(double) * LV) != cudaSuccess) {
            cudaGetLastError();
            st = fail(VBW_ERR_NOMEM, "device allocation for the plan failed");
            break;
        }
        if ((e = cudaMemcpy(d_Vd, V, sizeof(double) * LV, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemset(p->d_status, 0, sizeof(int))) != cudaSuccess) {
            st = fail(VBW_ERR_CUDA, "V upload failed: %s", cudaGetErrorString(e));
            break;
        }
        vbw_twiddle_kernel<<<(twiddle_entries(N) + 255) / 256, 256>>>(p->d_tw, N, layout_T(N),
                                                                       N / layout_T(N));
        if (overlap & 1)
            vbw_halfphase_kernel<<<(half_phase_entries(N) + 255) / 256, 256>>>(p->d_tw + twiddle_entries(N), N);
        if (N == 2048 && overlap == N / 4 && (e = build_split2048_table(p->d_tw + twiddle_entries(N), 0)) != cudaSuccess) {
            st = fail(VBW_ERR_CUDA, "split twiddle kernel failed: %s", cudaGetErrorString(e));
            break;
        }
        if (precision != VBW_PREC_FP32) {
            if (cudaMalloc(&p->d_tc, tc_table_bytes(N, precision)) != cudaSuccess) {
                cudaGetLastError();
                st = fail(VBW_ERR_NOMEM, "device allocation for the tensor-core tables failed");
                break;
            }
            if ((e = build_tc_table(N, precision, p->d_tc, 0)) != cudaSuccess) {
                st = fail(VBW_ERR_CUDA, "tensor-core table kernel failed: %s", cudaGetErrorString(e));
                break;
            }
        }
        vbw_round_table_kernel<<<(LV + 255) / 256, 256>>>(d_Vd, p->d_V, LV);
        if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaDeviceSynchronize()) != cudaSuccess) {
            st = fail(VBW_ERR_CUDA, "plan table kernels failed: %s", cudaGetErrorString(e));
            break;
        }
    } while (0);
    if (d_Vd) cudaFree(d_Vd);
    if (st != VBW_OK) {
        if (p->d_tw) cudaFree(p->d_tw);
        if (p->d_V) cudaFree(p->d_V);
        if (p->d_status) cudaFree(p->d_status);
        if (p->d_tc) cudaFree(p->d_tc);
        delete p;
        return st;
    }
    *out = p;
    return ok();
}

extern "C" vbw_status vbw_plan_destroy(vbw_plan_t p)
{
    if (!p) return fail(VBW_ERR_INVALID_ARG, "plan is NULL");
    cudaFree(p->d_tw);
    cudaFree(p->d_V);
    cudaFree(p->d_status);
    cudaFree(p->d_tc);
    delete p;
    return ok();
}

extern "C" vbw_status vbw_plan_status(vbw_plan_t p, int* flags, int clear)
{
    if (!p || !flags) return fail(VBW_ERR_INVALID_ARG, "NULL argument");
    VBW_CUDA(cudaMemcpy(flags, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (clear) VBW_CUDA(cudaMemset(p->d_status, 0, sizeof(int)));
    if (*flags & 1) return fail(VBW_ERR_TIMEOUT, "a bounded device wait gave up (status 0x%x)", *flags);
    return ok();
}

extern "C" vbw_status vbw_tune_set(int N, int warps, int ctas_per_sm)
{
    const int i = n_index(N);
    if (i < 0) return fail(VBW_ERR_INVALID_ARG, "N=%d is not a supported transform size", N);
    if (warps != 0 && warps != 4 && warps != 8)
        return fail(VBW_ERR_INVALID_ARG, "warps=%d: must be 0 (default), 4 or 8", warps);
    if (ctas_per_sm < 0 || ctas_per_sm > 32)
        return fail(VBW_ERR_INVALID_ARG, "ctas_per_sm=%d: must be in [0, 32]", ctas_per_sm);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_warps[i] = warps;
    g_tune_ctas[i] = ctas_per_sm;
    return ok();
}

extern "C" vbw_status vbw_debug_set(int flags)
{
    g_wait_limit_debug = flags & 1;
    g_full_band_debug = (flags >> 1) & 1;
    return ok();
}

extern "C" vbw_status vbw_plan_info(vbw_plan_t p, int* N, int* overlap, int* LV, int* M)
{
    if (!p) return fail(VBW_ERR_INVALID_ARG, "plan is NULL");
    if (N) *N = p->N;
    if (overlap) *overlap = p->O;
    if (LV) *LV = p->LV;
    if (M) *M = p->M;
    return ok();
}

// ------------------------------------------------------------------------------------------------
// streams

extern "C" vbw_status vbw_stream_create(vbw_plan_t p, int band, void* cuda_stream, vbw_stream_t* out)
{
    if (!out) return fail(VBW_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail(VBW_ERR_INVALID_ARG, "plan is NULL");
    vbw_status st = check_band(p, band);
    if (st != VBW_OK) return st;
    vbw_stream_s* s = new (std::nothrow) vbw_stream_s();
    if (!s) return fail(VBW_ERR_NOMEM, "host allocation failed");
    s->plan = p;
    s->st = (cudaStream_t)cuda_stream;
    s->band = band;
    if (cudaMalloc(&s->d_tail[0], sizeof(float2) * p->O) != cudaSuccess ||
        cudaMalloc(&s->d_tail[1], sizeof(float2) * p->O) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->d_tail[0]);
        delete s;
        return fail(VBW_ERR_NOMEM, "device allocation for the stream tail failed");
    }
    cudaError_t e = cudaMemsetAsync(s->d_tail[0], 0, sizeof(float2) * p->O, s->st);
    if (e != cudaSuccess) {
        cudaFree(s->d_tail[0]);
        cudaFree(s->d_tail[1]);
        delete s;
        return fail(VBW_ERR_CUDA, "tail reset failed: %s", cudaGetErrorString(e));
    }
    *out = s;
    return ok();
}

static void free_stage(vbw_stream_s* s)
{
    for (int i = 0; i < 2; ++i) {
        for (int j = 0; j < 2; ++j)
            if (s->d_stage[i][j]) cudaFree(s->d_stage[i][j]), s->d_stage[i][j] = nullptr;
        if (s->ev_in[i]) cudaEventDestroy(s->ev_in[i]), s->ev_in[i] = nullptr;
        if (s->ev_k[i]) cudaEventDestroy(s->ev_k[i]), s->ev_k[i] = nullptr;
        if (s->ev_out[i]) cudaEventDestroy(s->ev_out[i]), s->ev_out[i] = nullptr;
    }
    if (s->cp_in) cudaStreamDestroy(s->cp_in), s->cp_in = nullptr;
    if (s->cp_out) cudaStreamDestroy(s->cp_out), s->cp_out = nullptr;
    s->stage_blocks = 0;
}

extern "C" vbw_status vbw_stream_destroy(vbw_stream_t s)
{
    if (!s) return fail(VBW_ERR_INVALID_ARG, "stream is NULL");
    cudaStreamSynchronize(s->st);
    free_stage(s);
    cudaFree(s->d_tail[0]);
    cudaFree(s->d_tail[1]);
    delete s;
    return ok();
}

extern "C" vbw_status vbw_stream_reset(vbw_stream_t s, int band)
{
    if (!s) return fail(VBW_ERR_INVALID_ARG, "stream is NULL");
    vbw_status st = check_band(s->plan, band);
    if (st != VBW_OK) return st;
    s->cur = 0;
    VBW_CUDA(cudaMemsetAsync(s->d_tail[0], 0, sizeof(float2) * s->plan->O, s->st));
    s->pos = 0;
    s->band = band;
    s->flushed = false;
    s->pending.clear();
    return ok();
}

extern "C" vbw_status vbw_set_bandwidth(vbw_stream_t s, int band)
{
    if (!s) return fail(VBW_ERR_INVALID_ARG, "stream is NULL");
    vbw_status st = check_band(s->plan, band);
    if (st != VBW_OK) return st;
    s->pending[s->pos] = band;
    return ok();
}

extern "C" vbw_status vbw_set_bandwidth_at(vbw_stream_t s, int64_t block, int band)
{
    if (!s) return fail(VBW_ERR_INVALID_ARG, "stream is NULL");
    if (block < s->pos)
        return fail(VBW_ERR_INVALID_ARG, "block %lld is already submitted (position %lld)",
                    (long long)block, (long long)s->pos);
    vbw_status st = check_band(s->plan, band);
    if (st != VBW_OK) return st;
    s->pending[block] = band;
    return ok();
}

extern "C" vbw_status vbw_stream_position(vbw_stream_t s, int64_t* blocks)
{
    if (!s || !blocks) return fail(VBW_ERR_INVALID_ARG, "NULL argument");
    *blocks = s->pos;
    return ok();
}

// Band in effect at the stream's current position (applies and drops pending changes <= pos).
static void settle_band(vbw_stream_s* s)
{
    while (!s->pending.empty() && s->pending.begin()->first <= s->pos) {
        s->band = s->pending.begin()->second;
        s->pending.erase(s->pending.begin());
    }
}

// Enqueues one launch for blocks [pos, pos + nb) of the stream: input `in` holds nsamp samples
// (nsamp = nb*M, or fewer for the final partial block). Inline band changes come from `pending`.
static vbw_status launch_stream_range(vbw_stream_s* s, const float2* in, float2* out, int64_t nb,
                                      int64_t nsamp, bool keep_tail)
{
    vbw_plan_s* p = s->plan;
    settle_band(s);
    OlsArgs a;
    memset(&a, 0, sizeof(a));
    a.job.in = in;
    a.job.out = out;
    a.job.tail_in = s->d_tail[s->cur];
    a.job.tail_out = keep_tail ? s->d_tail[s->cur ^ 1] : nullptr;
    a.job.band = nullptr;
    a.job.nsamp = nsamp;
    a.job.band0 = s->band;
    int nchg = 0;
    for (auto it = s->pending.begin(); it != s->pending.end() && it->first < s->pos + nb; ++it) {
        if (nchg == kInlineChanges) break;
        a.chg_block[nchg] = it->first - s->pos;
        a.chg_band[nchg] = it->second;
        ++nchg;
    }
    a.nchg = nchg;
    const int B = tile_blocks(p);
    a.ntiles = (nb + B - 1) / B;
    fill_plan_args(a, p);
    cudaError_t e = launch_plan(p, a, s->st);
    if (e != cudaSuccess) return fail(VBW_ERR_CUDA, "filter launch failed: %s", cudaGetErrorString(e));
    if (keep_tail) s->cur ^= 1;
    s->pos += nb;
    settle_band(s);
    return VBW_OK;
}

// Splits [pos, pos + nblocks) so that no launch carries more than kInlineChanges band changes.
static vbw_status filter_blocks(vbw_stream_s* s, const float2* in, float2* out, int64_t nblocks)
{
    const int64_t M = s->plan->M;
    int64_t done = 0;
    while (done < nblocks) {
        settle_band(s);
        int64_t nb = nblocks - done;
        int count = 0;
        for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
            if (it->first >= s->pos + nb) break;
            if (++count > kInlineChanges) {
                nb = it->first - s->pos;
                break;
            }
        }
        vbw_status st = launch_stream_range(s, in + done * M, out + done * M, nb, nb * M, true);
        if (st != VBW_OK) return st;
        done += nb;
    }
    return VBW_OK;
}

extern "C" vbw_status vbw_filter(vbw_stream_t s, const void* in, void* out, int64_t nblocks)
{
    if (!s) return fail(VBW_ERR_INVALID_ARG, "stream is NULL");
    if (s->flushed) return fail(VBW_ERR_STATE, "stream was flushed; reset it first");
    if (nblocks < 0) return fail(VBW_ERR_INVALID_ARG, "nblocks < 0");
    if (nblocks == 0) return ok();
    if (!in || !out) return fail(VBW_ERR_INVALID_ARG, "in/out is NULL");
    if (misaligned(in) || misaligned(out)) return fail(VBW_ERR_INVALID_ARG, "in/out not 8-byte aligned");
    const size_t bytes = sizeof(float2) * (size_t)nblocks * s->plan->M;
    if (ranges_overlap(in, out, bytes)) return fail(VBW_ERR_INVALID_ARG, "in and out overlap");
    vbw_status st = filter_blocks(s, (const float2*)in, (float2*)out, nblocks);
    return st == VBW_OK ? ok() : st;
}

extern "C" vbw_status vbw_flush(vbw_stream_t s, const void* in, void* out, int nvalid)
{
    if (!s) return fail(VBW_ERR_INVALID_ARG, "stream is NULL");
    if (s->flushed) return fail(VBW_ERR_STATE, "stream was flushed; reset it first");
    if (nvalid < 0 || nvalid >= s->plan->M)
        return fail(VBW_ERR_INVALID_ARG, "nvalid=%d outside [0, M)", nvalid);
    if (nvalid > 0) {
        if (!in || !out) return fail(VBW_ERR_INVALID_ARG, "in/out is NULL");
        if (misaligned(in) || misaligned(out))
            return fail(VBW_ERR_INVALID_ARG, "in/out not 8-byte aligned");
        if (ranges_overlap(in, out, sizeof(float2) * (size_t)nvalid))
            return fail(VBW_ERR_INVALID_ARG, "in and out overlap");
        vbw_status st = launch_stream_range(s, (const float2*)in, (float2*)out, 1, nvalid, false);
        if (st != VBW_OK) return st;
    }
    s->flushed = true;
    return ok();
}

static vbw_status ensure_stage(vbw_stream_s* s, int64_t blocks)
{
    if (s->stage_blocks >= blocks) return VBW_OK;
    free_stage(s);
    const size_t bytes = sizeof(float2) * (size_t)blocks * s->plan->M;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            if (cudaMalloc(&s->d_stage[i][j], bytes) != cudaSuccess) {
                cudaGetLastError();
                free_stage(s);
                return fail(VBW_ERR_NOMEM, "staging allocation failed");
            }
    for (int i = 0; i < 2; ++i) {
        VBW_CUDA(cudaEventCreateWithFlags(&s->ev_in[i], cudaEventDisableTiming));
        VBW_CUDA(cudaEventCreateWithFlags(&s->ev_k[i], cudaEventDisableTiming));
        VBW_CUDA(cudaEventCreateWithFlags(&s->ev_out[i], cudaEventDisableTiming));
    }
    VBW_CUDA(cudaStreamCreateWithFlags(&s->cp_in, cudaStreamNonBlocking));
    VBW_CUDA(cudaStreamCreateWithFlags(&s->cp_out, cudaStreamNonBlocking));
    s->stage_blocks = blocks;
    return VBW_OK;
}

extern "C" vbw_status vbw_filter_host(vbw_stream_t s, const void* in, void* out, int64_t nblocks)
{
    if (!s) return fail(VBW_ERR_INVALID_ARG, "stream is NULL");
    if (s->flushed) return fail(VBW_ERR_STATE, "stream was flushed; reset it first");
    if (nblocks < 0) return fail(VBW_ERR_INVALID_ARG, "nblocks < 0");
    if (nblocks == 0) return ok();
    if (!in || !out) return fail(VBW_ERR_INVALID_ARG, "in/out is NULL");
    const int64_t M = s->plan->M;
    if (ranges_overlap(in, out, sizeof(float2) * (size_t)nblocks * M))
        return fail(VBW_ERR_INVALID_ARG, "in and out overlap");
    // chunks of about 32 MiB of input
    int64_t chunk = std::max<int64_t>(1, (int64_t(32) << 20) / (int64_t)(sizeof(float2) * M));
    chunk = std::min(chunk, nblocks);
    vbw_status st = ensure_stage(s, chunk);
    if (st != VBW_OK) return st;
    const float2* hin = (const float2*)in;
    float2* hout = (float2*)out;
    int slot = 0;
    bool used[2] = {false, false};
    for (int64_t b0 = 0; b0 < nblocks; b0 += chunk, slot ^= 1) {
        const int64_t nb = std::min(chunk, nblocks - b0);
        const size_t bytes = sizeof(float2) * (size_t)(nb * M);
        if (used[slot]) VBW_CUDA(cudaStreamWaitEvent(s->cp_in, s->ev_out[slot], 0));
        VBW_CUDA(cudaMemcpyAsync(s->d_stage[slot][0], hin + b0 * M, bytes, cudaMemcpyHostToDevice,
                                 s->cp_in));
        VBW_CUDA(cudaEventRecord(s->ev_in[slot], s->cp_in));
        VBW_CUDA(cudaStreamWaitEvent(s->st, s->ev_in[slot], 0));
        st = filter_blocks(s, s->d_stage[slot][0], s->d_stage[slot][1], nb);
        if (st != VBW_OK) return st;
        VBW_CUDA(cudaEventRecord(s->ev_k[slot], s->st));
        VBW_CUDA(cudaStreamWaitEvent(s->cp_out, s->ev_k[slot], 0));
        VBW_CUDA(cudaMemcpyAsync(hout + b0 * M, s->d_stage[slot][1], bytes, cudaMemcpyDeviceToHost,
                                 s->cp_out));
        VBW_CUDA(cudaEventRecord(s->ev_out[slot], s->cp_out));
        used[slot] = true;
    }
    VBW_CUDA(cudaStreamSynchronize(s->cp_out));
    return ok();
}

// ------------------------------------------------------------------------------------------------
// checkpoint / resume

namespace {
struct SavedHeader {
    uint32_t magic, version;
    int32_t N, O, LV, band;
    int64_t pos;
    int32_t flushed, npending;
};
constexpr uint32_t kMagic = 0x56425753u;  // "VBWS"
}  // namespace

extern "C" vbw_status vbw_stream_save(vbw_stream_t s, void* host_buf, size_t* bytes)
{
    if (!s || !bytes) return fail(VBW_ERR_INVALID_ARG, "NULL argument");
    const vbw_plan_s* p = s->plan;
    const size_t need = sizeof(SavedHeader) + s->pending.size() * (sizeof(int64_t) + sizeof(int32_t)) +
                        sizeof(float2) * (size_t)p->O;
    if (!host_buf) {
        *bytes = need;
        return ok();
    }
    if (*bytes < need) return fail(VBW_ERR_INVALID_ARG, "buffer too small (%zu < %zu)", *bytes, need);
    VBW_CUDA(cudaStreamSynchronize(s->st));
    unsigned char* w = (unsigned char*)host_buf;
    SavedHeader h{kMagic, 1u, p->N, p->O, p->LV, s->band, s->pos, s->flushed ? 1 : 0,
                  (int32_t)s->pending.size()};
    memcpy(w, &h, sizeof(h));
    w += sizeof(h);
    for (auto& kv : s->pending) {
        memcpy(w, &kv.first, sizeof(int64_t));
        w += sizeof(int64_t);
        memcpy(w, &kv.second, sizeof(int32_t));
        w += sizeof(int32_t);
    }
    VBW_CUDA(cudaMemcpy(w, s->d_tail[s->cur], sizeof(float2) * p->O, cudaMemcpyDeviceToHost));
    *bytes = need;
    return ok();
}

extern "C" vbw_status vbw_stream_restore(vbw_stream_t s, const void* host_buf, size_t bytes)
{
    if (!s || !host_buf) return fail(VBW_ERR_INVALID_ARG, "NULL argument");
    const vbw_plan_s* p = s->plan;
    if (bytes < sizeof(SavedHeader)) return fail(VBW_ERR_INVALID_ARG, "buffer too small");
    SavedHeader h;
    memcpy(&h, host_buf, sizeof(h));
    if (h.magic != kMagic || h.version != 1u) return fail(VBW_ERR_INVALID_ARG, "not a saved stream");
    if (h.N != p->N || h.O != p->O || h.LV != p->LV)
        return fail(VBW_ERR_INVALID_ARG, "saved geometry (N=%d, O=%d, L_V=%d) differs from the plan",
                    h.N, h.O, h.LV);
    if (h.npending < 0) return fail(VBW_ERR_INVALID_ARG, "corrupt pending count");
    const size_t need = sizeof(SavedHeader) + (size_t)h.npending * (sizeof(int64_t) + sizeof(int32_t)) +
                        sizeof(float2) * (size_t)p->O;
    if (bytes < need) return fail(VBW_ERR_INVALID_ARG, "buffer too small (%zu < %zu)", bytes, need);
    if (check_band(p, h.band) != VBW_OK) return VBW_ERR_BAND_RANGE;
    const unsigned char* r = (const unsigned char*)host_buf + sizeof(h);
    std::map<int64_t, int> pend;
    for (int i = 0; i < h.npending; ++i) {
        int64_t b;
        int32_t k;
        memcpy(&b, r, sizeof(b));
        r += sizeof(b);
        memcpy(&k, r, sizeof(k));
        r += sizeof(k);
        if (check_band(p, k) != VBW_OK) return VBW_ERR_BAND_RANGE;
        pend[b] = k;
    }
    VBW_CUDA(cudaStreamSynchronize(s->st));
    VBW_CUDA(cudaMemcpy(s->d_tail[s->cur], r, sizeof(float2) * p->O, cudaMemcpyHostToDevice));
    s->band = h.band;
    s->pos = h.pos;
    s->flushed = h.flushed != 0;
    s->pending.swap(pend);
    return ok();
}

// ------------------------------------------------------------------------------------------------
// batches

static void batch_free(vbw_batch_s* bt)
{
    if (bt->s_h2d) {
        cudaStreamSynchronize(bt->s_d2h);
        cudaStreamDestroy(bt->s_h2d);
        cudaStreamDestroy(bt->s_comp);
        cudaStreamDestroy(bt->s_d2h);
        cudaEventDestroy(bt->ev_start);
        cudaEventDestroy(bt->ev_h);
        cudaEventDestroy(bt->ev_c);
        cudaEventDestroy(bt->ev_done);
    }
    if (bt->s_side) {
        cudaStreamSynchronize(bt->s_side);
        cudaStreamDestroy(bt->s_side);
        cudaEventDestroy(bt->ev_fork);
        cudaEventDestroy(bt->ev_join);
    }
    for (auto& G : bt->groups) {
        cudaFree(G.d_jobs);
        cudaFree(G.d_tiles);
    }
    for (auto* z : bt->d_zjobs) cudaFree(z);
    cudaFree(bt->d_zmjobs);
    cudaFree(bt->d_mjobs);
    cudaFree(bt->d_mtiles);
    cudaFree(bt->d_bands);
    delete bt;
}

template <class T>
static cudaError_t upload(T** dst, const std::vector<T>& v)
{
    *dst = nullptr;
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc(dst, sizeof(T) * v.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

// Plans a mixed launch can take: overlap N/4 and N <= 1024 (N = 2048 keeps its own kernel, whose
// register and shared-memory footprint would otherwise apply to every N).
static bool mixable(const vbw_plan_s* p)
{
    return p->prec == VBW_PREC_FP32 && p->O == p->N / 4 && p->N <= 1024;
}

// Jobs of one real signal. Its blocks go through the kernel in pairs (2q, 2q+1) that share one
// complex block and therefore one band, so the signal is cut into jobs wherever a band change
// falls on an odd block: the next job starts at that block and reads its O samples of history
// from the signal itself (tail_in points O samples before its first input sample).
struct RealPiece {
    int64_t first_block, nblocks;   // real blocks [first_block, first_block + nblocks)
};
static std::vector<RealPiece> real_pieces(const int32_t* bands, int64_t nb)
{
    std::vector<RealPiece> out;
    int64_t start = 0;
    while (start < nb) {
        int64_t end = start;
        while (end < nb) {
            if (end + 1 < nb && bands[end] != bands[end + 1]) {
                end += 1;   // the pair would mix two bands: this piece ends after its first block
                break;
            }
            end += 2;
        }
        if (end > nb) end = nb;
        out.push_back(RealPiece{start, end - start});
        start = end;
    }
    return out;
}

static vbw_status batch_create_real(const vbw_signal* sig, int n, vbw_batch_t* out);

extern "C" vbw_status vbw_batch_create_real(const vbw_signal* sig, int n, vbw_batch_t* out)
{
    if (!out) return fail(VBW_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || (n > 0 && !sig)) return fail(VBW_ERR_INVALID_ARG, "bad signal array");
    return batch_create_real(sig, n, out);
}

extern "C" vbw_status vbw_batch_create(const vbw_signal* sig, int n, vbw_batch_t* out)
{
    if (!out) return fail(VBW_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || (n > 0 && !sig)) return fail(VBW_ERR_INVALID_ARG, "bad signal array");
    // validate and count
    int64_t total_blocks = 0;
    for (int i = 0; i < n; ++i) {
        const vbw_signal& g = sig[i];
        if (!g.plan) return fail(VBW_ERR_INVALID_ARG, "signal %d: plan is NULL", i);
        if (g.nsamples < 0) return fail(VBW_ERR_INVALID_ARG, "signal %d: nsamples < 0", i);
        if (g.nsamples > 0 && (!g.in || !g.out))
            return fail(VBW_ERR_INVALID_ARG, "signal %d: in/out is NULL", i);
        if (g.nsamples > 0 && (misaligned(g.in) || misaligned(g.out)))
            return fail(VBW_ERR_INVALID_ARG, "signal %d: in/out not 8-byte aligned", i);
        if (g.nsamples > 0 && ranges_overlap(g.in, g.out, sizeof(float2) * (size_t)g.nsamples))
            return fail(VBW_ERR_INVALID_ARG, "signal %d: in and out overlap", i);
        const int64_t nb = (g.nsamples + g.plan->M - 1) / g.plan->M;
        if (nb > INT32_MAX) return fail(VBW_ERR_INVALID_ARG, "signal %d: too many blocks", i);
        if (g.band_per_block) {
            for (int64_t b = 0; b < nb; ++b)
                if (check_band(g.plan, g.band_per_block[b]) != VBW_OK)
                    return fail(VBW_ERR_BAND_RANGE, "signal %d block %lld: band %d out of range", i,
                                (long long)b, g.band_per_block[b]);
        } else if (nb > 0 && check_band(g.plan, g.band) != VBW_OK) {
            return fail(VBW_ERR_BAND_RANGE, "signal %d: band %d out of range", i, g.band);
        }
        total_blocks += nb;
    }
    vbw_batch_s* bt = new (std::nothrow) vbw_batch_s();
    if (!bt) return fail(VBW_ERR_NOMEM, "host allocation failed");
    memset(&bt->margs, 0, sizeof(bt->margs));
    bt->sigs.assign(sig, sig + n);

    // per-block bands of every signal, one device array
    std::vector<int32_t> bands;
    bands.reserve((size_t)total_blocks);
    std::vector<int64_t> band_off(n, 0);
    std::map<vbw_plan_s*, std::vector<int>> by_plan;
    for (int i = 0; i < n; ++i) {
        const vbw_signal& g = sig[i];
        const int64_t nb = (g.nsamples + g.plan->M - 1) / g.plan->M;
        band_off[i] = (int64_t)bands.size();
        for (int64_t b = 0; b < nb; ++b) bands.push_back(g.band_per_block ? g.band_per_block[b] : g.band);
        if (nb > 0) by_plan[g.plan].push_back(i);
    }
    cudaError_t e = upload(&bt->d_bands, bands);
    if (e != cudaSuccess) {
        batch_free(bt);
        return fail(VBW_ERR_NOMEM, "batch band upload failed: %s", cudaGetErrorString(e));
    }

    // one group per plan (single-plan launches), and the mixed work list over mixable plans
    std::vector<OlsJob> mjobs;
    std::vector<int2> mtiles;
    int nmixed = 0;
    size_t mixed_warp_bytes = 0;
    int32_t tw_off = 0;
    for (auto& kv : by_plan) {
        vbw_plan_s* p = kv.first;
        const int B = tile_blocks(p);
        const bool mix = mixable(p) && nmixed < kMaxMixedPlans;
        const int plan_idx = mix ? nmixed : 0;
        std::vector<OlsJob> jobs;
        std::vector<int2> tiles;
        BatchGroup gr;
        gr.plan = p;
        for (int i : kv.second) {
            const vbw_signal& g = sig[i];
            OlsJob j;
            memset(&j, 0, sizeof(j));
            j.in = (const float2*)g.in;
            j.out = (float2*)g.out;
            j.band = bt->d_bands + band_off[i];
            j.nsamp = g.nsamples;
            j.band0 = bands[(size_t)band_off[i]];
            j.plan = 0;
            const int64_t nb = (g.nsamples + p->M - 1) / p->M;
            gr.sig.push_back(i);
            gr.tile_off.push_back((int64_t)tiles.size());
            for (int64_t b = 0; b < nb; b += B) tiles.push_back(make_int2((int)jobs.size(), (int)b));
            jobs.push_back(j);
            gr.cost += (double)nb * p->N * std::log2((double)p->N);
            if (mix) {
                j.plan = plan_idx;
                for (int64_t b = 0; b < nb; b += B) mtiles.push_back(make_int2((int)mjobs.size(), (int)b));
                mjobs.push_back(j);
            }
        }
        gr.tile_off.push_back((int64_t)tiles.size());
        gr.ntiles = (int64_t)tiles.size();
        cudaError_t e1 = upload(&gr.d_jobs, jobs);
        cudaError_t e2 = e1 == cudaSuccess ? upload(&gr.d_tiles, tiles) : e1;
        bt->groups.push_back(gr);
        if (e2 != cudaSuccess) {
            batch_free(bt);
            return fail(VBW_ERR_NOMEM, "batch work-list upload failed: %s", cudaGetErrorString(e2));
        }
        if (mix) {
            MixedPlan& mp = bt->margs.plans[nmixed];
            mp.tw = p->d_tw;
            mp.V = p->d_V;
            mp.N = p->N;
            mp.LV = p->LV;
            mp.tw_off = tw_off;
            mp.tw_len = twiddle_entries(p->N);
            tw_off += (mp.tw_len + 1) / 2 * 2;   // keep every table 16-byte aligned
            mixed_warp_bytes = std::max(mixed_warp_bytes, ols_warp_bytes(p->N));
            bt->mixed_groups.push_back((int)bt->groups.size() - 1);
            bt->mixed_cost += gr.cost;
            ++nmixed;
        }
    }
    if (nmixed > 0) {
        cudaError_t e1 = upload(&bt->d_mjobs, mjobs);
        cudaError_t e2 = e1 == cudaSuccess ? upload(&bt->d_mtiles, mtiles) : e1;
        if (e2 != cudaSuccess) {
            batch_free(bt);
            return fail(VBW_ERR_NOMEM, "mixed work-list upload failed: %s", cudaGetErrorString(e2));
        }
        bt->margs.jobs = bt->d_mjobs;
        bt->margs.tiles = bt->d_mtiles;
        bt->margs.ntiles = (int64_t)mtiles.size();
        bt->margs.nplans = nmixed;
        bt->margs.tw_bytes = (int32_t)(sizeof(float2) * (size_t)tw_off);
        bt->margs.warp_bytes = (int32_t)mixed_warp_bytes;
    }
    if (cudaStreamCreateWithFlags(&bt->s_side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&bt->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&bt->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        batch_free(bt);
        return fail(VBW_ERR_CUDA, "batch stream creation failed");
    }
    *out = bt;
    return ok();
}

static vbw_status batch_create_real(const vbw_signal* sig, int n, vbw_batch_t* out)
{
    for (int i = 0; i < n; ++i) {
        const vbw_signal& g = sig[i];
        if (!g.plan) return fail(VBW_ERR_INVALID_ARG, "signal %d: plan is NULL", i);
        if (g.plan->prec != VBW_PREC_FP32)
            return fail(VBW_ERR_UNSUPPORTED, "signal %d: real signals take FP32 plans", i);
        if (g.plan->O > g.plan->M)
            return fail(VBW_ERR_UNSUPPORTED, "signal %d: real signals need overlap <= N/2", i);
        if (g.nsamples < 0) return fail(VBW_ERR_INVALID_ARG, "signal %d: nsamples < 0", i);
        if (g.nsamples > 0 && (!g.in || !g.out))
            return fail(VBW_ERR_INVALID_ARG, "signal %d: in/out is NULL", i);
        if (g.nsamples > 0 && ((((uintptr_t)g.in) & 3) || (((uintptr_t)g.out) & 3)))
            return fail(VBW_ERR_INVALID_ARG, "signal %d: in/out not 4-byte aligned", i);
        if (g.nsamples > 0 && ranges_overlap(g.in, g.out, sizeof(float) * (size_t)g.nsamples))
            return fail(VBW_ERR_INVALID_ARG, "signal %d: in and out overlap", i);
        const int64_t nb = (g.nsamples + g.plan->M - 1) / g.plan->M;
        if (nb > INT32_MAX) return fail(VBW_ERR_INVALID_ARG, "signal %d: too many blocks", i);
        for (int64_t b = 0; b < nb; ++b) {
            const int k = g.band_per_block ? g.band_per_block[b] : g.band;
            if (check_band(g.plan, k) != VBW_OK)
                return fail(VBW_ERR_BAND_RANGE, "signal %d block %lld: band %d out of range", i, (long long)b, k);
        }
    }
    vbw_batch_s* bt = new (std::nothrow) vbw_batch_s();
    if (!bt) return fail(VBW_ERR_NOMEM, "host allocation failed");
    memset(&bt->margs, 0, sizeof(bt->margs));
    bt->real = true;
    bt->mode = VBW_BATCH_PER_PLAN;
    bt->sigs.assign(sig, sig + n);

    // pieces of every signal, and one band per block pair of every piece
    struct Piece {
        int sig;
        RealPiece r;
        int64_t band_off;
    };
    std::vector<Piece> pieces;
    std::vector<int32_t> pair_bands;
    std::map<vbw_plan_s*, std::vector<int>> by_plan;   // plan -> piece indices
    for (int i = 0; i < n; ++i) {
        const vbw_signal& g = sig[i];
        const int64_t nb = (g.nsamples + g.plan->M - 1) / g.plan->M;
        std::vector<int32_t> b(nb);
        for (int64_t k = 0; k < nb; ++k) b[k] = g.band_per_block ? g.band_per_block[k] : g.band;
        for (const RealPiece& r : real_pieces(b.data(), nb)) {
            Piece pc{i, r, (int64_t)pair_bands.size()};
            for (int64_t k = 0; k < r.nblocks; k += 2) pair_bands.push_back(b[r.first_block + k]);
            by_plan[g.plan].push_back((int)pieces.size());
            pieces.push_back(pc);
        }
    }
    cudaError_t e = upload(&bt->d_bands, pair_bands);
    if (e != cudaSuccess) {
        batch_free(bt);
        return fail(VBW_ERR_NOMEM, "batch band upload failed: %s", cudaGetErrorString(e));
    }
    for (auto& kv : by_plan) {
        vbw_plan_s* p = kv.first;
        const int B = tile_blocks(p);
        std::vector<OlsJob> jobs;
        std::vector<int2> tiles;
        BatchGroup gr;
        gr.plan = p;
        for (int pi : kv.second) {
            const Piece& pc = pieces[pi];
            const vbw_signal& g = sig[pc.sig];
            const float* in = static_cast<const float*>(g.in) + pc.r.first_block * p->M;
            float* o = static_cast<float*>(g.out) + pc.r.first_block * p->M;
            OlsJob j;
            memset(&j, 0, sizeof(j));
            j.in = reinterpret_cast<const float2*>(in);
            j.out = reinterpret_cast<float2*>(o);
            // history: zeros at the signal start, else the O samples before the piece
            j.tail_in = pc.r.first_block > 0 ? reinterpret_cast<const float2*>(in - p->O) : nullptr;
            j.band = bt->d_bands + pc.band_off;
            j.nsamp = std::min<int64_t>(g.nsamples - pc.r.first_block * p->M, pc.r.nblocks * p->M);
            j.band0 = pair_bands[(size_t)pc.band_off];
            j.plan = 0;
            const int64_t npairs = (pc.r.nblocks + 1) / 2;
            gr.sig.push_back(pc.sig);
            gr.tile_off.push_back((int64_t)tiles.size());
            for (int64_t q = 0; q < npairs; q += B) tiles.push_back(make_int2((int)jobs.size(), (int)q));
            jobs.push_back(j);
            gr.cost += (double)npairs * p->N * std::log2((double)p->N);
        }
        gr.tile_off.push_back((int64_t)tiles.size());
        gr.ntiles = (int64_t)tiles.size();
        cudaError_t e1 = upload(&gr.d_jobs, jobs);
        cudaError_t e2 = e1 == cudaSuccess ? upload(&gr.d_tiles, tiles) : e1;
        bt->groups.push_back(gr);
        if (e2 != cudaSuccess) {
            batch_free(bt);
            return fail(VBW_ERR_NOMEM, "batch work-list upload failed: %s", cudaGetErrorString(e2));
        }
    }
    if (cudaStreamCreateWithFlags(&bt->s_side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&bt->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&bt->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        batch_free(bt);
        return fail(VBW_ERR_CUDA, "batch stream creation failed");
    }
    *out = bt;
    return ok();
}

extern "C" vbw_status vbw_batch_set_mode(vbw_batch_t bt, int mode, double mixed_share)
{
    if (!bt) return fail(VBW_ERR_INVALID_ARG, "batch is NULL");
    if (mode < VBW_BATCH_AUTO || mode > VBW_BATCH_MIXED)
        return fail(VBW_ERR_INVALID_ARG, "unknown batch mode %d", mode);
    if (!(mixed_share >= 0.0 && mixed_share < 1.0))
        return fail(VBW_ERR_INVALID_ARG, "mixed_share must be in [0, 1)");
    bt->mode = mode;
    bt->split = mixed_share;
    return ok();
}

static cudaError_t launch_group_range(const BatchGroup& G, int64_t t0, int64_t t1, cudaStream_t st,
                                      int max_ctas = 0, const OlsJob* jobs = nullptr, int flags = 0)
{
    vbw_plan_s* p = G.plan;
    OlsArgs a;
    memset(&a, 0, sizeof(a));
    a.jobs = jobs ? jobs : G.d_jobs;
    a.tiles = G.d_tiles + t0;
    a.ntiles = t1 - t0;
    fill_plan_args(a, p);
    a.flags = flags;
    return launch_plan(p, a, st, max_ctas);
}

// Device-side run of a prepared batch. PER_PLAN: one full-GPU persistent launch per plan, in
// order. MIXED: one persistent launch over every mixable plan, with the remaining plans (N = 2048
// or other overlaps) launched beside it on a forked stream; the SMs are shared in proportion to
// the transform work unless a share was set. AUTO: MIXED when at least two plans mix.
static vbw_status batch_launch(vbw_batch_s* bt, cudaStream_t st, bool zero_copy = false)
{
    int launches = 0;
    const int flags = (zero_copy ? kOlsNoBulk : 0) | (bt->real ? kOlsReal : 0);
    const bool use_mixed = !bt->real && bt->mode == VBW_BATCH_MIXED
                               ? !bt->mixed_groups.empty()
                               : (!bt->real && bt->mode == VBW_BATCH_AUTO && bt->mixed_groups.size() >= 2);
    if (!use_mixed) {
        for (size_t gi = 0; gi < bt->groups.size(); ++gi) {
            const BatchGroup& G = bt->groups[gi];
            cudaError_t e = launch_group_range(G, 0, G.ntiles, st, 0,
                                               zero_copy ? bt->d_zjobs[gi] : nullptr, flags);
            if (e != cudaSuccess) return fail(VBW_ERR_CUDA, "batch launch failed: %s", cudaGetErrorString(e));
            ++launches;
        }
        bt->last_launches = launches;
        return VBW_OK;
    }
    double rest_cost = 0;
    for (size_t gi = 0; gi < bt->groups.size(); ++gi)
        if (std::find(bt->mixed_groups.begin(), bt->mixed_groups.end(), (int)gi) == bt->mixed_groups.end())
            rest_cost += bt->groups[gi].cost;
    const int sms = bt->groups[0].plan->sms;
    double share = bt->split > 0 ? bt->split : bt->mixed_cost / (bt->mixed_cost + rest_cost);
    if (rest_cost == 0) share = 1.0;
    int mixed_sms = std::max(1, std::min(sms, (int)std::lround(share * sms)));
    if (rest_cost > 0 && mixed_sms == sms) mixed_sms = sms - 1;
    const int mwarps = warps_for(1024);   // the largest mixed transform decides the CTA shape
    int mixed_per_sm = 0;
    {
        // CTAs of the mixed kernel that fit on one SM decide how many CTAs its SM share is
        const size_t smem = (size_t)bt->margs.tw_bytes + (size_t)mwarps * bt->margs.warp_bytes;
        mixed_per_sm = (int)std::max<size_t>(1, (228 * 1024) / std::max<size_t>(smem, 1));
    }
    if (rest_cost > 0) {
        VBW_CUDA(cudaEventRecord(bt->ev_fork, st));
        VBW_CUDA(cudaStreamWaitEvent(bt->s_side, bt->ev_fork, 0));
    }
    MixedArgs ma = bt->margs;
    ma.flags = flags;
    if (zero_copy) ma.jobs = bt->d_zmjobs;
    int grid = 0;
    cudaError_t e = launch_ols_mixed(ma, 1024, mwarps, sms, mixed_per_sm * mixed_sms, st, &grid);
    if (e != cudaSuccess) return fail(VBW_ERR_CUDA, "mixed launch failed: %s", cudaGetErrorString(e));
    ++launches;
    if (rest_cost > 0) {
        const int side_sms = sms - mixed_sms;
        for (size_t gi = 0; gi < bt->groups.size(); ++gi) {
            if (std::find(bt->mixed_groups.begin(), bt->mixed_groups.end(), (int)gi) != bt->mixed_groups.end())
                continue;
            const BatchGroup& G = bt->groups[gi];
            const int per_sm = G.plan->N >= 2048 ? 2 : 4;
            e = launch_group_range(G, 0, G.ntiles, bt->s_side, per_sm * side_sms,
                                   zero_copy ? bt->d_zjobs[gi] : nullptr, flags);
            if (e != cudaSuccess) return fail(VBW_ERR_CUDA, "batch launch failed: %s", cudaGetErrorString(e));
            ++launches;
        }
        VBW_CUDA(cudaEventRecord(bt->ev_join, bt->s_side));
        VBW_CUDA(cudaStreamWaitEvent(st, bt->ev_join, 0));
    }
    bt->last_launches = launches;
    return VBW_OK;
}

// Device address of pinned host memory, or nullptr when p is not pinned (pageable memory).
static const void* mapped_host(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return at.devicePointer;
}

// Zero-copy run from pinned host memory: on a coherent CPU-GPU link (Grace-Blackwell NVLink-C2C)
// the fused kernel reads its input from and writes its output to host memory directly, so nothing
// is staged and the run is bound by the link instead of the copy engines. The kernels then use
// plain loads and stores only (no TMA staging, no bulk prefetch). Returns VBW_ERR_UNSUPPORTED when
// any buffer is not pinned (the caller then takes the staged path).
static vbw_status batch_zero_copy(vbw_batch_s* bt, const void* const* host_in, void* const* host_out,
                                  cudaStream_t st)
{
    const size_t n = bt->sigs.size();
    std::vector<const void*> din(n), dout(n);
    for (size_t i = 0; i < n; ++i) {
        if (bt->sigs[i].nsamples == 0) continue;
        din[i] = mapped_host(host_in[i]);
        dout[i] = mapped_host(host_out[i]);
        if (!din[i] || !dout[i] || misaligned(din[i]) || misaligned(dout[i])) return VBW_ERR_UNSUPPORTED;
    }
    const bool same = bt->z_in.size() == n &&
                      std::equal(din.begin(), din.end(), bt->z_in.begin()) &&
                      std::equal(dout.begin(), dout.end(), bt->z_out.begin());
    if (!same) {
        // job arrays with the host addresses, same order as the device arrays
        VBW_CUDA(cudaStreamSynchronize(st));
        if (bt->d_zjobs.size() != bt->groups.size()) bt->d_zjobs.assign(bt->groups.size(), nullptr);
        std::vector<std::vector<OlsJob>> zj(bt->groups.size());
        for (size_t gi = 0; gi < bt->groups.size(); ++gi) {
            const BatchGroup& G = bt->groups[gi];
            std::vector<OlsJob>& jobs = zj[gi];
            jobs.resize(G.sig.size());
            VBW_CUDA(cudaMemcpy(jobs.data(), G.d_jobs, sizeof(OlsJob) * jobs.size(), cudaMemcpyDeviceToHost));
            for (size_t j = 0; j < jobs.size(); ++j) {
                jobs[j].in = (const float2*)din[G.sig[j]];
                jobs[j].out = (float2*)dout[G.sig[j]];
            }
            if (!bt->d_zjobs[gi]) VBW_CUDA(cudaMalloc(&bt->d_zjobs[gi], sizeof(OlsJob) * jobs.size()));
            VBW_CUDA(cudaMemcpy(bt->d_zjobs[gi], jobs.data(), sizeof(OlsJob) * jobs.size(), cudaMemcpyHostToDevice));
        }
        if (bt->d_mjobs) {
            // same order as the mixed array: mixed groups in order, their jobs in order; the
            // mixed array numbers plans by mixed-group position
            std::vector<OlsJob> mj;
            for (size_t m = 0; m < bt->mixed_groups.size(); ++m)
                for (OlsJob jj : zj[bt->mixed_groups[m]]) {
                    jj.plan = (int32_t)m;
                    mj.push_back(jj);
                }
            if (!bt->d_zmjobs) VBW_CUDA(cudaMalloc(&bt->d_zmjobs, sizeof(OlsJob) * mj.size()));
            VBW_CUDA(cudaMemcpy(bt->d_zmjobs, mj.data(), sizeof(OlsJob) * mj.size(), cudaMemcpyHostToDevice));
        }
        bt->z_in = din;
        bt->z_out = dout;
    }
    vbw_status s = batch_launch(bt, st, true);
    if (s != VBW_OK) return s;
    VBW_CUDA(cudaStreamSynchronize(st));
    return VBW_OK;
}

extern "C" vbw_status vbw_batch_run_host(vbw_batch_t bt, const void* const* host_in,
                                         void* const* host_out, void* cuda_stream)
{
    if (!bt || (!bt->sigs.empty() && (!host_in || !host_out)))
        return fail(VBW_ERR_INVALID_ARG, "NULL argument");
    if (bt->real) return fail(VBW_ERR_UNSUPPORTED, "host buffers are not supported for real batches");
    for (size_t i = 0; i < bt->sigs.size(); ++i)
        if (bt->sigs[i].nsamples > 0 && (!host_in[i] || !host_out[i]))
            return fail(VBW_ERR_INVALID_ARG, "signal %zu: host buffer is NULL", i);
    if (!bt->s_h2d) {
        VBW_CUDA(cudaStreamCreateWithFlags(&bt->s_h2d, cudaStreamNonBlocking));
        VBW_CUDA(cudaStreamCreateWithFlags(&bt->s_comp, cudaStreamNonBlocking));
        VBW_CUDA(cudaStreamCreateWithFlags(&bt->s_d2h, cudaStreamNonBlocking));
        VBW_CUDA(cudaEventCreateWithFlags(&bt->ev_start, cudaEventDisableTiming));
        VBW_CUDA(cudaEventCreateWithFlags(&bt->ev_h, cudaEventDisableTiming));
        VBW_CUDA(cudaEventCreateWithFlags(&bt->ev_c, cudaEventDisableTiming));
        VBW_CUDA(cudaEventCreateWithFlags(&bt->ev_done, cudaEventDisableTiming));
    }
    cudaStream_t user = (cudaStream_t)cuda_stream;
    if (env_int("VBW_ZERO_COPY", 1) != 0 && !bt->sigs.empty()) {
        vbw_status zs = batch_zero_copy(bt, host_in, host_out, user);
        if (zs != VBW_ERR_UNSUPPORTED) return zs == VBW_OK ? ok() : zs;
    }
    VBW_CUDA(cudaEventRecord(bt->ev_start, user));
    VBW_CUDA(cudaStreamWaitEvent(bt->s_h2d, bt->ev_start, 0));
    VBW_CUDA(cudaStreamWaitEvent(bt->s_comp, bt->ev_start, 0));
    VBW_CUDA(cudaStreamWaitEvent(bt->s_d2h, bt->ev_start, 0));
    const size_t unit_bytes = size_t(64) << 20;  // pipeline unit: about 64 MiB of input
    int launches = 0;
    for (auto& G : bt->groups) {
        const int njobs = (int)G.sig.size();
        int j0 = 0;
        while (j0 < njobs) {
            size_t bytes = 0;
            int j1 = j0;
            while (j1 < njobs && (j1 == j0 || bytes < unit_bytes)) {
                bytes += sizeof(float2) * (size_t)bt->sigs[G.sig[j1]].nsamples;
                ++j1;
            }
            // one copy per run of signals that are contiguous on both sides
            for (int j = j0; j < j1;) {
                const vbw_signal& g = bt->sigs[G.sig[j]];
                const char* hsrc = (const char*)host_in[G.sig[j]];
                char* ddst = (char*)g.in;
                size_t len = sizeof(float2) * (size_t)g.nsamples;
                int k = j + 1;
                while (k < j1 && (const char*)host_in[G.sig[k]] == hsrc + len &&
                       (const char*)bt->sigs[G.sig[k]].in == ddst + len) {
                    len += sizeof(float2) * (size_t)bt->sigs[G.sig[k]].nsamples;
                    ++k;
                }
                if (len) VBW_CUDA(cudaMemcpyAsync(ddst, hsrc, len, cudaMemcpyHostToDevice, bt->s_h2d));
                j = k;
            }
            VBW_CUDA(cudaEventRecord(bt->ev_h, bt->s_h2d));
            VBW_CUDA(cudaStreamWaitEvent(bt->s_comp, bt->ev_h, 0));
            cudaError_t e = launch_group_range(G, G.tile_off[j0], G.tile_off[j1], bt->s_comp);
            if (e != cudaSuccess) return fail(VBW_ERR_CUDA, "batch launch failed: %s", cudaGetErrorString(e));
            ++launches;
            VBW_CUDA(cudaEventRecord(bt->ev_c, bt->s_comp));
            VBW_CUDA(cudaStreamWaitEvent(bt->s_d2h, bt->ev_c, 0));
            for (int j = j0; j < j1;) {
                const vbw_signal& g = bt->sigs[G.sig[j]];
                char* hdst = (char*)host_out[G.sig[j]];
                const char* dsrc = (const char*)g.out;
                size_t len = sizeof(float2) * (size_t)g.nsamples;
                int k = j + 1;
                while (k < j1 && (char*)host_out[G.sig[k]] == hdst + len &&
                       (const char*)bt->sigs[G.sig[k]].out == dsrc + len) {
                    len += sizeof(float2) * (size_t)bt->sigs[G.sig[k]].nsamples;
                    ++k;
                }
                if (len) VBW_CUDA(cudaMemcpyAsync(hdst, dsrc, len, cudaMemcpyDeviceToHost, bt->s_d2h));
                j = k;
            }
            j0 = j1;
        }
    }
    VBW_CUDA(cudaEventRecord(bt->ev_done, bt->s_d2h));
    VBW_CUDA(cudaStreamWaitEvent(user, bt->ev_done, 0));
    VBW_CUDA(cudaStreamSynchronize(bt->s_d2h));
    bt->last_launches = launches;
    return ok();
}

extern "C" vbw_status vbw_batch_run(vbw_batch_t bt, void* cuda_stream)
{
    if (!bt) return fail(VBW_ERR_INVALID_ARG, "batch is NULL");
    vbw_status st = batch_launch(bt, (cudaStream_t)cuda_stream);
    return st == VBW_OK ? ok() : st;
}

extern "C" vbw_status vbw_batch_launches(vbw_batch_t bt, int* launches)
{
    if (!bt || !launches) return fail(VBW_ERR_INVALID_ARG, "NULL argument");
    *launches = bt->last_launches;
    return ok();
}

extern "C" vbw_status vbw_batch_destroy(vbw_batch_t bt)
{
    if (!bt) return fail(VBW_ERR_INVALID_ARG, "batch is NULL");
    batch_free(bt);
    return ok();
}

// ------------------------------------------------------------------------------------------------
// test hook

extern "C" vbw_status vbw_debug_export_HR(vbw_plan_t p, int band, float* host_out)
{
    if (!p || !host_out) return fail(VBW_ERR_INVALID_ARG, "NULL argument");
    vbw_status st = check_band(p, band);
    if (st != VBW_OK) return st;
    float* d = nullptr;
    if (cudaMalloc(&d, sizeof(float) * p->N) != cudaSuccess) {
        cudaGetLastError();
        return fail(VBW_ERR_NOMEM, "device allocation failed");
    }
    cudaError_t e;
    switch (p->N) {
    case 128: e = launch_export_hr<128>(p->d_V, p->LV, band, d, 0); break;
    case 256: e = launch_export_hr<256>(p->d_V, p->LV, band, d, 0); break;
    case 512: e = launch_export_hr<512>(p->d_V, p->LV, band, d, 0); break;
    case 1024: e = launch_export_hr<1024>(p->d_V, p->LV, band, d, 0); break;
    default:
        // the kernel this plan's filtering runs: the split kernel's tables and bin mapping for
        // overlap N/4, else the four-step kernel's
        e = (p->O == p->N / 4 && split2048_choice(-1, p->sms)) ? launch_split2048_export_hr(p->d_V, p->LV, band, d, 0)
                                                      : launch_export_hr<2048>(p->d_V, p->LV, band, d, 0);
        break;
    }
    if (e == cudaSuccess) e = cudaMemcpy(host_out, d, sizeof(float) * p->N, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(VBW_ERR_CUDA, "export failed: %s", cudaGetErrorString(e));
    return ok();
}

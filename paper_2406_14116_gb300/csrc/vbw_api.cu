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

namespace vbw {
template <int N>
cudaError_t launch_ols_fp32(const OlsArgs& a, int warps, int sms, cudaStream_t st, int* grid_out);
template <int N>
cudaError_t launch_export_hr(const float* V, int LV, int k1, float* out, cudaStream_t st);
}  // namespace vbw

using namespace vbw;

// ------------------------------------------------------------------------------------------------
// errors

static thread_local std::string g_last_error;

static vbw_status fail(vbw_status st, const char* fmt, ...)
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

static vbw_status ok()
{
    g_last_error.clear();
    return VBW_OK;
}

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

__global__ void vbw_round_table_kernel(const double* Vd, float* Vf, int LV)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < LV) Vf[i] = (float)Vd[i];
}

// ------------------------------------------------------------------------------------------------
// objects

struct vbw_plan_s {
    int N = 0, O = 0, M = 0, LV = 0, prec = 0;
    int device = 0, sms = 0;
    int warps = 8;
    std::vector<double> V;
    float2* d_tw = nullptr;
    float* d_V = nullptr;
};

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
    std::vector<int> sig;           // signal index of each job
    std::vector<int64_t> tile_off;  // first tile of each job (size jobs + 1)
};

struct vbw_batch_s {
    std::vector<BatchGroup> groups;
    std::vector<vbw_signal> sigs;
    int32_t* d_bands = nullptr;
    int last_launches = 0;
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_start = nullptr, ev_h = nullptr, ev_c = nullptr, ev_done = nullptr;
};

// ------------------------------------------------------------------------------------------------
// validation helpers (pure host logic: no CUDA call before the arguments are known to be valid)

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static vbw_status check_band(const vbw_plan_s* p, int band)
{
    const int kmax = p->N / 2 - p->LV - 1;
    if (band < 1 || band > kmax)
        return fail(VBW_ERR_BAND_RANGE, "band k1=%d outside [1, %d] for N=%d, L_V=%d", band, kmax,
                    p->N, p->LV);
    return VBW_OK;
}

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

// Warps per CTA for each N: the largest CTA whose register footprint still gives 16 resident
// warps per SM (N <= 1024) or 8 (N = 2048). VBW_WARPS overrides it (4 or 8).
static int default_warps(int N)
{
    const int w = env_int("VBW_WARPS", 0);
    if (w == 4 || w == 8) return w;
    return (N <= 1024) ? 8 : 4;
}

static cudaError_t launch_fp32(int N, const OlsArgs& a, int warps, int sms, cudaStream_t st)
{
    int grid = 0;
    switch (N) {
    case 128: return launch_ols_fp32<128>(a, warps, sms, st, &grid);
    case 256: return launch_ols_fp32<256>(a, warps, sms, st, &grid);
    case 512: return launch_ols_fp32<512>(a, warps, sms, st, &grid);
    case 1024: return launch_ols_fp32<1024>(a, warps, sms, st, &grid);
    case 2048: return launch_ols_fp32<2048>(a, warps, sms, st, &grid);
    default: return cudaErrorInvalidValue;
    }
}

static int blocks_per_warp(int N) { return 32 / layout_T(N); }

// entries of the per-plan twiddle table: T rows of E + 2 (see OlsGeom::TW)
static int twiddle_entries(int N) { return layout_T(N) * (N / layout_T(N) + 2); }

// ------------------------------------------------------------------------------------------------
// plans

extern "C" vbw_status vbw_plan(int N, int overlap, const double* V, int LV, int precision,
                               vbw_plan_t* out)
{
    if (!out) return fail(VBW_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!is_pow2(N) || N < 128 || N > 2048)
        return fail(VBW_ERR_INVALID_ARG, "N=%d: must be a power of two in [128, 2048]", N);
    if (overlap <= 0 || overlap >= N || (overlap & 1))
        return fail(VBW_ERR_INVALID_ARG, "overlap=%d: must be even and in (0, N)", overlap);
    if (LV < 1 || LV > N / 2 - 2)
        return fail(VBW_ERR_INVALID_ARG, "L_V=%d: must be in [1, N/2-2]", LV);
    if (!V) return fail(VBW_ERR_INVALID_ARG, "transition_samples is NULL");
    for (int i = 0; i < LV; ++i)
        if (!std::isfinite(V[i])) return fail(VBW_ERR_INVALID_ARG, "V[%d] is not finite", i);
    if (precision != VBW_PREC_FP32)
        return fail(VBW_ERR_INVALID_ARG, "precision %d is not a known precision", precision);

    vbw_plan_s* p = new (std::nothrow) vbw_plan_s();
    if (!p) return fail(VBW_ERR_NOMEM, "host allocation failed");
    p->N = N;
    p->O = overlap;
    p->M = N - overlap;
    p->LV = LV;
    p->prec = precision;
    p->V.assign(V, V + LV);
    p->warps = default_warps(N);
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
        if (cudaMalloc(&p->d_tw, sizeof(float2) * twiddle_entries(N)) != cudaSuccess ||
            cudaMalloc(&p->d_V, sizeof(float) * LV) != cudaSuccess ||
            cudaMalloc(&d_Vd, sizeof(double) * LV) != cudaSuccess) {
            cudaGetLastError();
            st = fail(VBW_ERR_NOMEM, "device allocation for the plan failed");
            break;
        }
        if ((e = cudaMemcpy(d_Vd, V, sizeof(double) * LV, cudaMemcpyHostToDevice)) != cudaSuccess) {
            st = fail(VBW_ERR_CUDA, "V upload failed: %s", cudaGetErrorString(e));
            break;
        }
        vbw_twiddle_kernel<<<(twiddle_entries(N) + 255) / 256, 256>>>(p->d_tw, N, layout_T(N),
                                                                       N / layout_T(N));
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
    delete p;
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
    const int B = blocks_per_warp(p->N);
    a.ntiles = (nb + B - 1) / B;
    a.tw = p->d_tw;
    a.V = p->d_V;
    a.overlap = p->O;
    a.LV = p->LV;
    cudaError_t e = launch_fp32(p->N, a, p->warps, p->sms, s->st);
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
        if (g.nsamples > 0 && ranges_overlap(g.in, g.out, sizeof(float2) * (size_t)g.nsamples))
            return fail(VBW_ERR_INVALID_ARG, "signal %d: in and out overlap", i);
        const int64_t nb = (g.nsamples + g.plan->M - 1) / g.plan->M;
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
    std::vector<int32_t> bands;
    bands.reserve((size_t)total_blocks);
    std::map<vbw_plan_s*, std::vector<int>> by_plan;
    std::vector<int64_t> band_off(n, 0);
    for (int i = 0; i < n; ++i) {
        const vbw_signal& g = sig[i];
        const int64_t nb = (g.nsamples + g.plan->M - 1) / g.plan->M;
        band_off[i] = (int64_t)bands.size();
        for (int64_t b = 0; b < nb; ++b) bands.push_back(g.band_per_block ? g.band_per_block[b] : g.band);
        if (nb > 0) by_plan[g.plan].push_back(i);
    }
    auto cleanup = [&]() {
        for (auto& gr : bt->groups) {
            cudaFree(gr.d_jobs);
            cudaFree(gr.d_tiles);
        }
        cudaFree(bt->d_bands);
        delete bt;
    };
    if (!bands.empty()) {
        if (cudaMalloc(&bt->d_bands, sizeof(int32_t) * bands.size()) != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            return fail(VBW_ERR_NOMEM, "batch band array allocation failed");
        }
        cudaError_t e = cudaMemcpy(bt->d_bands, bands.data(), sizeof(int32_t) * bands.size(),
                                   cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cleanup();
            return fail(VBW_ERR_CUDA, "batch band upload failed: %s", cudaGetErrorString(e));
        }
    }
    for (auto& kv : by_plan) {
        vbw_plan_s* p = kv.first;
        const int B = blocks_per_warp(p->N);
        std::vector<OlsJob> jobs;
        std::vector<int2> tiles;
        std::vector<int> gr_sig;
        std::vector<int64_t> gr_off;
        for (int i : kv.second) {
            const vbw_signal& g = sig[i];
            OlsJob j;
            memset(&j, 0, sizeof(j));
            j.in = (const float2*)g.in;
            j.out = (float2*)g.out;
            j.tail_in = nullptr;
            j.tail_out = nullptr;
            j.band = bt->d_bands + band_off[i];
            j.nsamp = g.nsamples;
            j.band0 = bands[(size_t)band_off[i]];
            const int64_t nb = (g.nsamples + p->M - 1) / p->M;
            if (nb > INT32_MAX) {
                cleanup();
                return fail(VBW_ERR_INVALID_ARG, "signal %d: too many blocks", i);
            }
            const int ji = (int)jobs.size();
            jobs.push_back(j);
            gr_sig.push_back(i);
            gr_off.push_back((int64_t)tiles.size());
            for (int64_t b = 0; b < nb; b += B) tiles.push_back(make_int2(ji, (int)b));
        }
        gr_off.push_back((int64_t)tiles.size());
        BatchGroup gr;
        gr.plan = p;
        gr.ntiles = (int64_t)tiles.size();
        gr.sig.swap(gr_sig);
        gr.tile_off.swap(gr_off);
        bt->groups.push_back(gr);
        BatchGroup& G = bt->groups.back();
        if (cudaMalloc(&G.d_jobs, sizeof(OlsJob) * jobs.size()) != cudaSuccess ||
            cudaMalloc(&G.d_tiles, sizeof(int2) * tiles.size()) != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            return fail(VBW_ERR_NOMEM, "batch work-list allocation failed");
        }
        cudaError_t e1 = cudaMemcpy(G.d_jobs, jobs.data(), sizeof(OlsJob) * jobs.size(), cudaMemcpyHostToDevice);
        cudaError_t e2 = cudaMemcpy(G.d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            cleanup();
            return fail(VBW_ERR_CUDA, "batch work-list upload failed");
        }
    }
    bt->sigs.assign(sig, sig + n);
    *out = bt;
    return ok();
}

static cudaError_t launch_group_range(const BatchGroup& G, int64_t t0, int64_t t1, cudaStream_t st)
{
    vbw_plan_s* p = G.plan;
    OlsArgs a;
    memset(&a, 0, sizeof(a));
    a.jobs = G.d_jobs;
    a.tiles = G.d_tiles + t0;
    a.ntiles = t1 - t0;
    a.tw = p->d_tw;
    a.V = p->d_V;
    a.overlap = p->O;
    a.LV = p->LV;
    return launch_fp32(p->N, a, p->warps, p->sms, st);
}

extern "C" vbw_status vbw_batch_run_host(vbw_batch_t bt, const void* const* host_in,
                                         void* const* host_out, void* cuda_stream)
{
    if (!bt || (!bt->sigs.empty() && (!host_in || !host_out)))
        return fail(VBW_ERR_INVALID_ARG, "NULL argument");
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
            for (int j = j0; j < j1; ++j) {
                const vbw_signal& g = bt->sigs[G.sig[j]];
                VBW_CUDA(cudaMemcpyAsync((void*)g.in, host_in[G.sig[j]], sizeof(float2) * g.nsamples,
                                         cudaMemcpyHostToDevice, bt->s_h2d));
            }
            VBW_CUDA(cudaEventRecord(bt->ev_h, bt->s_h2d));
            VBW_CUDA(cudaStreamWaitEvent(bt->s_comp, bt->ev_h, 0));
            cudaError_t e = launch_group_range(G, G.tile_off[j0], G.tile_off[j1], bt->s_comp);
            if (e != cudaSuccess) return fail(VBW_ERR_CUDA, "batch launch failed: %s", cudaGetErrorString(e));
            ++launches;
            VBW_CUDA(cudaEventRecord(bt->ev_c, bt->s_comp));
            VBW_CUDA(cudaStreamWaitEvent(bt->s_d2h, bt->ev_c, 0));
            for (int j = j0; j < j1; ++j) {
                const vbw_signal& g = bt->sigs[G.sig[j]];
                VBW_CUDA(cudaMemcpyAsync(host_out[G.sig[j]], g.out, sizeof(float2) * g.nsamples,
                                         cudaMemcpyDeviceToHost, bt->s_d2h));
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
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int launches = 0;
    for (auto& G : bt->groups) {
        cudaError_t e = launch_group_range(G, 0, G.ntiles, st);
        if (e != cudaSuccess) return fail(VBW_ERR_CUDA, "batch launch failed: %s", cudaGetErrorString(e));
        ++launches;
    }
    bt->last_launches = launches;
    return ok();
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
    for (auto& G : bt->groups) {
        cudaFree(G.d_jobs);
        cudaFree(G.d_tiles);
    }
    cudaFree(bt->d_bands);
    delete bt;
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
    default: e = launch_export_hr<2048>(p->d_V, p->LV, band, d, 0); break;
    }
    if (e == cudaSuccess) e = cudaMemcpy(host_out, d, sizeof(float) * p->N, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(VBW_ERR_CUDA, "export failed: %s", cudaGetErrorString(e));
    return ok();
}

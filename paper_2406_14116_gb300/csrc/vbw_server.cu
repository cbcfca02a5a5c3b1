// Continuous-batching serving engine of libvbw (vbw_server_* in include/vbw.h).
//
// Many streams send chunks of any length at any time. Each stream's filter state lives on the
// device: the O-sample overlap tail (two buffers, read one / write the other) and the input
// samples that do not fill a block yet (the residual). The host mirrors only counts, the band
// and the list of pending band changes.
//
// vbw_server_poll drives the engine:
//   1. retire finished batches (their chunks become completions, in submission order);
//   2. while a batch slot is free and chunks are queued, admit chunks first in first out until
//      the slot's share of the device pool is used (admission by memory), merge each stream's
//      admitted chunks into one job (residual ++ chunks), and launch the batch.
// The phases of a batch run on three CUDA streams, so batch k+1's copies overlap batch k's
// kernels:
//   h2d   one work-list upload, then the chunks into their jobs         (copy-in stream)
//   comp  residual in, one fused launch per plan, residual out          (compute stream)
//   d2h   each chunk's completed output blocks to its host buffer       (copy-out stream)
// Each of the four copy steps is one launch of vbw_copy_kernel over a descriptor list, whatever
// the number of chunks and streams: the kernel reads and writes pinned host memory directly
// (NVLink-C2C) and moves residuals inside HBM. Chunks in pageable host memory, which the GPU
// cannot address, take a cudaMemcpyAsync each instead.
// Batches depend on each other only through the per-stream device state, which the compute
// stream orders. Every block runs through the same kernel code whatever else shares its launch,
// so a stream's output is bit-identical alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <utility>
#include <vector>

#include "vbw_internal.h"

using namespace vbw;

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

struct SrvStream {
    int plan = 0;
    int band = 1;              // band of the last block launched (the next one's unless a change is due)
    bool open = false, closing = false;
    int64_t blocks = 0;        // blocks launched
    int64_t submitted = 0;     // input samples submitted (the stream position of the next chunk)
    int64_t resid = 0;         // samples in the device residual after the launched batches (< M)
    std::deque<std::pair<int64_t, int>> pending;   // (first block, k1), in block order
    float2* d_tail[2] = {nullptr, nullptr};
    int cur = 0;
    float2* d_resid = nullptr;
};

struct Req {
    int stream = 0;
    const float2* in = nullptr;
    int64_t n = 0;
    float2* out = nullptr;
    const float2* in_dev = nullptr;   // device address of `in` (pinned memory), or nullptr
    float2* out_dev = nullptr;        // device address of `out` (pinned memory), or nullptr
    uint64_t tag = 0;
    bool final_flush = false;  // end of stream: the residual becomes a zero-padded last block
    int64_t produced = 0;      // output samples this chunk completes (set when it is launched)
    double t_submit = 0;
};

struct Slot {
    bool busy = false;
    unsigned char* d_region = nullptr;   // chunk inputs and block outputs of one batch
    size_t bytes = 0;
    unsigned char* h_work = nullptr;     // pinned staging of the work list (packed per batch)
    unsigned char* d_work = nullptr;
    size_t work_bytes = 0;
    int64_t max_blocks = 0;
    cudaEvent_t ev_h2d = nullptr, ev_comp = nullptr, ev_done = nullptr;
    std::vector<Req> reqs;
    int launches = 0;
};

// One job being assembled: a stream's residual plus its admitted chunks, in order.
struct JobBuild {
    int stream = 0;
    int64_t r0 = 0;            // residual samples at the front of the job's input
    int64_t total = 0;         // r0 + chunk samples
    bool final_flush = false;
    size_t in_off = 0, out_off = 0;
    std::vector<size_t> reqs;  // indices into the slot's request list
};

int64_t blocks_of(const JobBuild& jb, int M)
{
    return jb.final_flush ? (jb.total + M - 1) / M : jb.total / M;
}

// device bytes a job occupies in a slot: its input, then its output blocks
size_t job_bytes(const JobBuild& jb, int M)
{
    return round256(sizeof(float2) * (size_t)jb.total) + round256(sizeof(float2) * (size_t)(blocks_of(jb, M) * M));
}

// One contiguous copy of n samples; piece0 = index of its first piece in the launch.
struct CopyDesc {
    const float2* src;
    float2* dst;
    int64_t n;
    int64_t piece0;
};
constexpr int64_t kCopyPiece = 4096;   // samples per CTA iteration
constexpr int kMaxReqsPerBatch = 16384;

// Copies every descriptor's samples; a CTA takes one piece of kCopyPiece samples at a time. Each
// thread keeps eight loads in flight before it stores them: the sources may be host memory across
// the CPU-GPU link, where a load takes microseconds.
constexpr int kCopyThreads = 256, kCopyUnroll = 8;
__global__ void __launch_bounds__(kCopyThreads) vbw_copy_kernel(const CopyDesc* __restrict__ d, int nd,
                                                                int64_t npieces)
{
    for (int64_t p = blockIdx.x; p < npieces; p += gridDim.x) {
        int lo = 0, hi = nd - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (d[mid].piece0 <= p) lo = mid;
            else hi = mid - 1;
        }
        const float2* __restrict__ src = d[lo].src;
        float2* __restrict__ dst = d[lo].dst;
        const int64_t s0 = (p - d[lo].piece0) * kCopyPiece;
        const int64_t s1 = s0 + kCopyPiece < d[lo].n ? s0 + kCopyPiece : d[lo].n;
        int64_t i = s0 + threadIdx.x;
        for (; i + (kCopyUnroll - 1) * kCopyThreads < s1; i += kCopyUnroll * kCopyThreads) {
            float2 v[kCopyUnroll];
#pragma unroll
            for (int u = 0; u < kCopyUnroll; ++u) v[u] = __ldcs(src + i + u * kCopyThreads);
#pragma unroll
            for (int u = 0; u < kCopyUnroll; ++u) __stcs(dst + i + u * kCopyThreads, v[u]);
        }
        for (; i < s1; i += kCopyThreads) dst[i] = src[i];
    }
}

// Device address of pinned host memory, or nullptr for pageable memory.
const void* mapped_host(const void* p)
{
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (at.type == cudaMemoryTypeHost && at.devicePointer) ? at.devicePointer : nullptr;
}

// A descriptor list being filled in the work staging: appends and numbers the pieces.
struct CopyList {
    CopyDesc* h = nullptr;
    int n = 0;
    int64_t pieces = 0;
    void add(const float2* src, float2* dst, int64_t cnt)
    {
        if (cnt <= 0) return;
        h[n++] = CopyDesc{src, dst, cnt, pieces};
        pieces += (cnt + kCopyPiece - 1) / kCopyPiece;
    }
};

}  // namespace

struct vbw_server_s {
    std::vector<vbw_plan_s*> plans;
    std::vector<SrvStream> streams;
    std::vector<Slot> slots;
    std::deque<Req> queue;
    std::deque<int> inflight;            // slot indices, in launch order
    std::deque<vbw_completion> done;     // retired, not yet handed out
    unsigned char* d_pool = nullptr;
    float2* d_state = nullptr;           // per-stream tails and residuals
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    int sms = 0;
    int64_t batches = 0, launches = 0, admitted = 0;
};

// One launch of the copy kernel over a descriptor list already on the device.
static cudaError_t launch_copies(const vbw_server_s* sv, const CopyDesc* d_desc, const CopyList& l, cudaStream_t st)
{
    if (l.n == 0) return cudaSuccess;
    const int64_t cap = (int64_t)sv->sms * 8;
    const int grid = (int)(l.pieces < cap ? l.pieces : cap);
    vbw_copy_kernel<<<grid, kCopyThreads, 0, st>>>(d_desc, l.n, l.pieces);
    return cudaGetLastError();
}

static void server_free(vbw_server_s* sv)
{
    if (sv->s_h2d) cudaStreamSynchronize(sv->s_h2d);
    if (sv->s_comp) cudaStreamSynchronize(sv->s_comp);
    if (sv->s_d2h) cudaStreamSynchronize(sv->s_d2h);
    for (auto& sl : sv->slots) {
        cudaFreeHost(sl.h_work);
        cudaFree(sl.d_work);
        if (sl.ev_h2d) cudaEventDestroy(sl.ev_h2d);
        if (sl.ev_comp) cudaEventDestroy(sl.ev_comp);
        if (sl.ev_done) cudaEventDestroy(sl.ev_done);
    }
    cudaFree(sv->d_pool);
    cudaFree(sv->d_state);
    if (sv->s_h2d) cudaStreamDestroy(sv->s_h2d);
    if (sv->s_comp) cudaStreamDestroy(sv->s_comp);
    if (sv->s_d2h) cudaStreamDestroy(sv->s_d2h);
    delete sv;
}

extern "C" vbw_status vbw_server_create(const vbw_plan_t* plans, int nplans, int max_streams, size_t pool_bytes,
                                        int slots, vbw_server_t* out)
{
    if (!out) return fail(VBW_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!plans || nplans < 1 || nplans > 64 || max_streams < 1 || slots < 1 || slots > 64)
        return fail(VBW_ERR_INVALID_ARG, "need 1..64 plans, max_streams >= 1 and 1..64 slots");
    int minM = 1 << 30, maxM = 0, maxO = 0;
    for (int i = 0; i < nplans; ++i) {
        if (!plans[i]) return fail(VBW_ERR_INVALID_ARG, "plan %d is NULL", i);
        minM = std::min(minM, plans[i]->M);
        maxM = std::max(maxM, plans[i]->M);
        maxO = std::max(maxO, plans[i]->O);
    }
    const size_t slot_bytes = pool_bytes / (size_t)slots / 256 * 256;
    if (slot_bytes < (size_t)8 * sizeof(float2) * (size_t)maxM)
        return fail(VBW_ERR_INVALID_ARG, "pool too small for %d slots", slots);
    vbw_server_s* sv = new (std::nothrow) vbw_server_s();
    if (!sv) return fail(VBW_ERR_NOMEM, "host allocation failed");
    sv->plans.assign(plans, plans + nplans);
    sv->streams.resize(max_streams);
    sv->slots.resize(slots);
    const size_t stride = round256(sizeof(float2) * (2 * (size_t)maxO + maxM)) / sizeof(float2);
    int dev = 0;
    bool good = cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&sv->sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                cudaMalloc(&sv->d_pool, slot_bytes * slots) == cudaSuccess &&
                cudaMalloc(&sv->d_state, sizeof(float2) * stride * max_streams) == cudaSuccess &&
                cudaStreamCreateWithFlags(&sv->s_h2d, cudaStreamNonBlocking) == cudaSuccess &&
                cudaStreamCreateWithFlags(&sv->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
                cudaStreamCreateWithFlags(&sv->s_d2h, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; good && i < max_streams; ++i) {
        SrvStream& st = sv->streams[i];
        st.d_tail[0] = sv->d_state + stride * i;
        st.d_tail[1] = st.d_tail[0] + maxO;
        st.d_resid = st.d_tail[1] + maxO;
    }
    // a complete block occupies 16 M bytes of a slot (input and output), so a slot holds at most
    // slot_bytes / (16 minM) complete blocks, plus one final partial block per stream
    const int64_t max_blocks = (int64_t)(slot_bytes / (16 * (size_t)minM)) + max_streams + 8;
    for (int i = 0; good && i < slots; ++i) {
        Slot& sl = sv->slots[i];
        sl.d_region = sv->d_pool + slot_bytes * i;
        sl.bytes = slot_bytes;
        sl.max_blocks = max_blocks;
        // packed work list: jobs, tiles, four copy lists (chunks in, residuals in and out, chunks
        // out), bands; each part 256-byte aligned
        sl.work_bytes = round256(sizeof(OlsJob) * (size_t)max_streams) + round256(sizeof(int2) * (size_t)max_blocks) +
                        2 * round256(sizeof(CopyDesc) * (size_t)kMaxReqsPerBatch) +
                        2 * round256(sizeof(CopyDesc) * (size_t)max_streams) +
                        round256(sizeof(int32_t) * (size_t)max_blocks);
        good = cudaMallocHost(&sl.h_work, sl.work_bytes) == cudaSuccess &&
               cudaMalloc(&sl.d_work, sl.work_bytes) == cudaSuccess &&
               cudaEventCreateWithFlags(&sl.ev_h2d, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&sl.ev_comp, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&sl.ev_done, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!good) {
        cudaGetLastError();
        server_free(sv);
        return fail(VBW_ERR_NOMEM, "server allocation failed");
    }
    *out = sv;
    return ok();
}

extern "C" vbw_status vbw_server_destroy(vbw_server_t sv)
{
    if (!sv) return fail(VBW_ERR_INVALID_ARG, "server is NULL");
    server_free(sv);
    return ok();
}

extern "C" vbw_status vbw_server_open_stream(vbw_server_t sv, int stream, int plan, int band)
{
    if (!sv || stream < 0 || stream >= (int)sv->streams.size() || plan < 0 || plan >= (int)sv->plans.size())
        return fail(VBW_ERR_INVALID_ARG, "bad server, stream or plan index");
    SrvStream& st = sv->streams[stream];
    if (st.open) return fail(VBW_ERR_STATE, "stream %d is open", stream);
    const vbw_plan_s* p = sv->plans[plan];
    const vbw_status s = check_band(p, band);
    if (s != VBW_OK) return s;
    // zero tail, ordered on the compute stream behind every batch already launched
    if (cudaMemsetAsync(st.d_tail[0], 0, sizeof(float2) * p->O, sv->s_comp) != cudaSuccess)
        return fail(VBW_ERR_CUDA, "tail reset failed");
    st.plan = plan;
    st.band = band;
    st.open = true;
    st.closing = false;
    st.blocks = 0;
    st.submitted = 0;
    st.resid = 0;
    st.cur = 0;
    st.pending.clear();
    return ok();
}

extern "C" vbw_status vbw_server_submit(vbw_server_t sv, int stream, const void* host_in, int64_t n,
                                        int new_band, void* host_out, int64_t out_capacity, uint64_t tag)
{
    if (!sv || stream < 0 || stream >= (int)sv->streams.size())
        return fail(VBW_ERR_INVALID_ARG, "bad server or stream index");
    SrvStream& st = sv->streams[stream];
    if (!st.open || st.closing) return fail(VBW_ERR_STATE, "stream %d is not open", stream);
    if (n < 0 || (n > 0 && (!host_in || misaligned(host_in)))) return fail(VBW_ERR_INVALID_ARG, "bad input");
    const vbw_plan_s* p = sv->plans[st.plan];
    if (new_band >= 0) {
        const vbw_status s = check_band(p, new_band);
        if (s != VBW_OK) return s;
    }
    const int64_t produce = ((st.submitted + n) / p->M - st.submitted / p->M) * p->M;
    if (produce > 0 && (!host_out || misaligned(host_out) || out_capacity < produce))
        return fail(VBW_ERR_INVALID_ARG, "output buffer needs %lld samples", (long long)produce);
    // the largest job this chunk can make (residual ++ chunk) must fit one slot
    if (2 * round256(sizeof(float2) * (size_t)(n + p->M)) > sv->slots[0].bytes)
        return fail(VBW_ERR_INVALID_ARG, "chunk larger than a batch slot");
    if (new_band >= 0) {
        // the change takes effect at the first block boundary at or after the chunk's first sample
        const int64_t blk = (st.submitted + p->M - 1) / p->M;
        while (!st.pending.empty() && st.pending.back().first == blk) st.pending.pop_back();
        st.pending.push_back({blk, new_band});
    }
    Req r;
    r.stream = stream;
    r.in = static_cast<const float2*>(host_in);
    r.n = n;
    r.out = static_cast<float2*>(host_out);
    r.in_dev = n > 0 ? static_cast<const float2*>(mapped_host(host_in)) : nullptr;
    r.out_dev = produce > 0 ? static_cast<float2*>(const_cast<void*>(mapped_host(host_out))) : nullptr;
    r.tag = tag;
    r.t_submit = now_s();
    st.submitted += n;
    sv->queue.push_back(r);
    return ok();
}

extern "C" vbw_status vbw_server_submit_many(vbw_server_t sv, const vbw_request* reqs, int count, int* submitted)
{
    if (!sv || !submitted || count < 0 || (count > 0 && !reqs)) return fail(VBW_ERR_INVALID_ARG, "bad argument");
    *submitted = 0;
    for (int i = 0; i < count; ++i) {
        const vbw_request& q = reqs[i];
        const vbw_status st = vbw_server_submit(sv, q.stream, q.host_in, q.n, q.new_band, q.host_out,
                                                q.out_capacity, q.tag);
        if (st != VBW_OK) return st;
        ++*submitted;
    }
    return ok();
}

extern "C" vbw_status vbw_server_close_stream(vbw_server_t sv, int stream, void* host_out, int64_t out_capacity,
                                              uint64_t tag)
{
    if (!sv || stream < 0 || stream >= (int)sv->streams.size())
        return fail(VBW_ERR_INVALID_ARG, "bad server or stream index");
    SrvStream& st = sv->streams[stream];
    if (!st.open || st.closing) return fail(VBW_ERR_STATE, "stream %d is not open", stream);
    const vbw_plan_s* p = sv->plans[st.plan];
    const int64_t produce = st.submitted % p->M;   // the final partial block
    if (produce > 0 && (!host_out || misaligned(host_out) || out_capacity < produce))
        return fail(VBW_ERR_INVALID_ARG, "output buffer needs %lld samples", (long long)produce);
    Req r;
    r.stream = stream;
    r.out = static_cast<float2*>(host_out);
    r.out_dev = produce > 0 ? static_cast<float2*>(const_cast<void*>(mapped_host(host_out))) : nullptr;
    r.tag = tag;
    r.final_flush = true;
    r.t_submit = now_s();
    st.closing = true;
    sv->queue.push_back(r);
    return ok();
}

// Admits chunks from the head of the queue into slot `si` and launches the batch. Returns the
// number of chunks admitted (0: nothing queued or the head does not fit), or -1 on error.
static int launch_batch(vbw_server_s* sv, int si, vbw_status* err)
{
    Slot& sl = sv->slots[si];
    sl.reqs.clear();
    std::vector<JobBuild> jobs;
    std::vector<int> job_of(sv->streams.size(), -1);
    size_t used = 0;
    int64_t nblocks = 0;

    // ---- admission: first in first out, merged per stream, until the slot is full
    while (!sv->queue.empty()) {
        const Req q = sv->queue.front();
        const SrvStream& st = sv->streams[q.stream];
        const int M = sv->plans[st.plan]->M;
        const int j = job_of[q.stream];
        JobBuild probe;
        if (j >= 0) {
            probe = jobs[j];
        } else {
            probe.stream = q.stream;
            probe.r0 = probe.total = st.resid;
        }
        const int64_t nb_before = j >= 0 ? blocks_of(probe, M) : 0;
        const size_t bytes_before = j >= 0 ? job_bytes(probe, M) : 0;
        probe.total += q.n;
        probe.final_flush = q.final_flush;
        const int64_t nb_after = blocks_of(probe, M);
        const size_t bytes_after = job_bytes(probe, M);
        if (used - bytes_before + bytes_after > sl.bytes) break;
        if (nblocks - nb_before + nb_after > sl.max_blocks) break;
        if ((int)sl.reqs.size() >= kMaxReqsPerBatch) break;
        used = used - bytes_before + bytes_after;
        nblocks += nb_after - nb_before;
        probe.reqs.push_back(sl.reqs.size());
        if (j >= 0) {
            jobs[j] = std::move(probe);
        } else {
            job_of[q.stream] = (int)jobs.size();
            jobs.push_back(std::move(probe));
        }
        sl.reqs.push_back(q);
        sv->queue.pop_front();
    }
    if (sl.reqs.empty()) return 0;

    // ---- region layout: per job [input: total samples][output: blocks x M]
    size_t off = 0;
    for (auto& jb : jobs) {
        const int M = sv->plans[sv->streams[jb.stream].plan]->M;
        jb.in_off = off;
        off += round256(sizeof(float2) * (size_t)jb.total);
        jb.out_off = off;
        off += round256(sizeof(float2) * (size_t)(blocks_of(jb, M) * M));
    }

    // ---- work list, packed: jobs | tiles | chunk-in copies | residual-in | residual-out |
    //      chunk-out copies | bands (each part 256-byte aligned; sizes counted first)
    int64_t cnt_jobs = 0, cnt_tiles = 0, cnt_bands = 0;
    int cnt_cin = 0, cnt_cout = 0, cnt_res = 0;
    for (auto& jb : jobs) {
        const vbw_plan_s* p = sv->plans[sv->streams[jb.stream].plan];
        const int64_t nb = blocks_of(jb, p->M);
        const int B = tile_blocks(p);
        cnt_bands += nb;
        cnt_tiles += (nb + B - 1) / B;
        cnt_jobs += nb > 0;
        cnt_res += 2;
        for (size_t ri : jb.reqs) {
            cnt_cin += sl.reqs[ri].n > 0;
            cnt_cout += 1;
        }
    }
    size_t woff = 0;
    auto take = [&](size_t bytes) {
        const size_t o = woff;
        woff += round256(bytes);
        return o;
    };
    const size_t o_jobs = take(sizeof(OlsJob) * (size_t)cnt_jobs);
    const size_t o_tiles = take(sizeof(int2) * (size_t)cnt_tiles);
    const size_t o_cin = take(sizeof(CopyDesc) * (size_t)cnt_cin);
    const size_t o_rin = take(sizeof(CopyDesc) * (size_t)cnt_res / 2);
    const size_t o_rout = take(sizeof(CopyDesc) * (size_t)cnt_res / 2);
    const size_t o_cout = take(sizeof(CopyDesc) * (size_t)cnt_cout);
    const size_t o_bands = take(sizeof(int32_t) * (size_t)cnt_bands);
    if (woff > sl.work_bytes) {
        *err = fail(VBW_ERR_NOMEM, "work list exceeds its staging");
        return -1;
    }
    OlsJob* h_jobs = reinterpret_cast<OlsJob*>(sl.h_work + o_jobs);
    int2* h_tiles = reinterpret_cast<int2*>(sl.h_work + o_tiles);
    int32_t* h_bands = reinterpret_cast<int32_t*>(sl.h_work + o_bands);
    const OlsJob* d_jobs = reinterpret_cast<const OlsJob*>(sl.d_work + o_jobs);
    const int2* d_tiles = reinterpret_cast<const int2*>(sl.d_work + o_tiles);
    const int32_t* d_bands = reinterpret_cast<const int32_t*>(sl.d_work + o_bands);
    CopyList c_in{reinterpret_cast<CopyDesc*>(sl.h_work + o_cin)}, rin{reinterpret_cast<CopyDesc*>(sl.h_work + o_rin)},
        rout{reinterpret_cast<CopyDesc*>(sl.h_work + o_rout)}, c_out{reinterpret_cast<CopyDesc*>(sl.h_work + o_cout)};
    std::vector<const Req*> pageable_in;   // chunks the GPU cannot address: one memcpy each
    std::vector<std::pair<const Req*, size_t>> pageable_out;

    // chunks behind their job's residual; the residual itself comes in on the compute stream
    for (auto& jb : jobs) {
        SrvStream& st = sv->streams[jb.stream];
        float2* jin = reinterpret_cast<float2*>(sl.d_region + jb.in_off);
        rin.add(st.d_resid, jin, jb.r0);
        int64_t pos = jb.r0;
        for (size_t ri : jb.reqs) {
            const Req& q = sl.reqs[ri];
            if (q.n > 0) {
                if (q.in_dev) c_in.add(q.in_dev, jin + pos, q.n);
                else pageable_in.push_back(&q);
            }
            pos += q.n;
        }
    }

    // jobs grouped by plan, one warp-tile per B blocks, a band per block
    std::vector<std::pair<int64_t, int64_t>> tile_range(sv->plans.size(), {0, 0});
    int njobs = 0;
    int64_t ntiles = 0, nbands = 0;
    for (size_t pl = 0; pl < sv->plans.size(); ++pl) {
        const vbw_plan_s* p = sv->plans[pl];
        const int B = tile_blocks(p);
        tile_range[pl].first = ntiles;
        for (auto& jb : jobs) {
            SrvStream& st = sv->streams[jb.stream];
            if (st.plan != (int)pl) continue;
            const int64_t nb = blocks_of(jb, p->M);
            const int64_t band_off = nbands;
            for (int64_t b = 0; b < nb; ++b) {
                while (!st.pending.empty() && st.pending.front().first <= st.blocks + b) {
                    st.band = st.pending.front().second;
                    st.pending.pop_front();
                }
                h_bands[nbands++] = st.band;
            }
            if (nb == 0) continue;
            OlsJob& J = h_jobs[njobs];
            memset(&J, 0, sizeof(J));
            J.in = reinterpret_cast<const float2*>(sl.d_region + jb.in_off);
            J.out = reinterpret_cast<float2*>(sl.d_region + jb.out_off);
            J.tail_in = st.d_tail[st.cur];
            J.tail_out = jb.final_flush ? nullptr : st.d_tail[st.cur ^ 1];
            J.band = d_bands + band_off;
            J.nsamp = jb.final_flush ? jb.total : nb * p->M;
            J.band0 = h_bands[band_off];
            J.plan = 0;
            for (int64_t b = 0; b < nb; b += B) h_tiles[ntiles++] = make_int2(njobs, (int)b);
            ++njobs;
        }
        tile_range[pl].second = ntiles;
    }

    // stream state after this batch: residuals out, block counts, tails flipped
    for (auto& jb : jobs) {
        SrvStream& st = sv->streams[jb.stream];
        const int M = sv->plans[st.plan]->M;
        const int64_t nb = blocks_of(jb, M);
        st.blocks += nb;
        if (jb.final_flush) {
            st.resid = 0;
            st.open = false;
            continue;
        }
        const int64_t keep = jb.total - nb * M;
        rout.add(reinterpret_cast<const float2*>(sl.d_region + jb.in_off) + nb * M, st.d_resid, keep);
        st.resid = keep;
        if (nb > 0) st.cur ^= 1;
    }

    // each chunk's completed blocks
    for (auto& jb : jobs) {
        const int M = sv->plans[sv->streams[jb.stream].plan]->M;
        const float2* jout = reinterpret_cast<const float2*>(sl.d_region + jb.out_off);
        int64_t cum = jb.r0, emitted = 0;   // job samples through this chunk; output samples handed out
        for (size_t ri : jb.reqs) {
            Req& q = sl.reqs[ri];
            cum += q.n;
            const int64_t upto = q.final_flush ? jb.total : cum / M * M;
            q.produced = upto - emitted;
            if (q.produced > 0) {
                if (q.out_dev) c_out.add(jout + emitted, q.out_dev, q.produced);
                else pageable_out.push_back({&q, (size_t)emitted});
            }
            emitted = upto;
        }
    }

    // ---- h2d: work list (one copy), chunks in
    cudaError_t e = cudaMemcpyAsync(sl.d_work, sl.h_work, woff, cudaMemcpyHostToDevice, sv->s_h2d);
    if (e == cudaSuccess) e = launch_copies(sv, reinterpret_cast<const CopyDesc*>(sl.d_work + o_cin), c_in, sv->s_h2d);
    for (size_t i = 0; e == cudaSuccess && i < pageable_in.size(); ++i) {
        const Req& q = *pageable_in[i];
        const JobBuild& jb = jobs[job_of[q.stream]];
        int64_t pos = jb.r0;
        for (size_t ri : jb.reqs) {
            if (&sl.reqs[ri] == &q) break;
            pos += sl.reqs[ri].n;
        }
        e = cudaMemcpyAsync(sl.d_region + jb.in_off + sizeof(float2) * (size_t)pos, q.in, sizeof(float2) * (size_t)q.n,
                            cudaMemcpyHostToDevice, sv->s_h2d);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev_h2d, sv->s_h2d);

    // ---- compute: residuals in, kernels, residuals out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sv->s_comp, sl.ev_h2d, 0);
    if (e == cudaSuccess) e = launch_copies(sv, reinterpret_cast<const CopyDesc*>(sl.d_work + o_rin), rin, sv->s_comp);
    sl.launches = 0;
    for (size_t pl = 0; e == cudaSuccess && pl < sv->plans.size(); ++pl) {
        if (tile_range[pl].second <= tile_range[pl].first) continue;
        OlsArgs a;
        memset(&a, 0, sizeof(a));
        a.jobs = d_jobs;
        a.tiles = d_tiles + tile_range[pl].first;
        a.ntiles = tile_range[pl].second - tile_range[pl].first;
        fill_plan_args(a, sv->plans[pl]);
        e = launch_plan(sv->plans[pl], a, sv->s_comp);
        ++sl.launches;
    }
    if (e == cudaSuccess) e = launch_copies(sv, reinterpret_cast<const CopyDesc*>(sl.d_work + o_rout), rout, sv->s_comp);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev_comp, sv->s_comp);

    // ---- d2h: chunks out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sv->s_d2h, sl.ev_comp, 0);
    if (e == cudaSuccess) e = launch_copies(sv, reinterpret_cast<const CopyDesc*>(sl.d_work + o_cout), c_out, sv->s_d2h);
    for (size_t i = 0; e == cudaSuccess && i < pageable_out.size(); ++i) {
        const Req& q = *pageable_out[i].first;
        const JobBuild& jb = jobs[job_of[q.stream]];
        e = cudaMemcpyAsync(q.out, sl.d_region + jb.out_off + sizeof(float2) * pageable_out[i].second,
                            sizeof(float2) * (size_t)q.produced, cudaMemcpyDeviceToHost, sv->s_d2h);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev_done, sv->s_d2h);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = fail(VBW_ERR_CUDA, "batch enqueue failed: %s", cudaGetErrorString(e));
        return -1;
    }
    sv->launches += sl.launches + (c_in.n > 0) + (rin.n > 0) + (rout.n > 0) + (c_out.n > 0);
    sl.busy = true;
    sv->inflight.push_back(si);
    sv->batches++;
    sv->admitted += (int64_t)sl.reqs.size();
    return (int)sl.reqs.size();
}

// Moves finished batches' chunks to the completion list, oldest batch first. With `block`, waits
// for the oldest batch in flight.
static vbw_status retire(vbw_server_s* sv, bool block)
{
    while (!sv->inflight.empty()) {
        Slot& sl = sv->slots[sv->inflight.front()];
        const cudaError_t q = block ? cudaEventSynchronize(sl.ev_done) : cudaEventQuery(sl.ev_done);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) return fail(VBW_ERR_CUDA, "batch failed: %s", cudaGetErrorString(q));
        const double t = now_s();
        for (const Req& r : sl.reqs) {
            vbw_completion c;
            c.tag = r.tag;
            c.stream = r.stream;
            c.final_flush = r.final_flush ? 1 : 0;
            c.produced = r.produced;
            c.t_submit = r.t_submit;
            c.t_done = t;
            sv->done.push_back(c);
        }
        sl.busy = false;
        sl.reqs.clear();
        sv->inflight.pop_front();
        block = false;
    }
    return VBW_OK;
}

static vbw_status admit(vbw_server_s* sv)
{
    while (!sv->queue.empty()) {
        int si = -1;
        for (size_t i = 0; i < sv->slots.size(); ++i)
            if (!sv->slots[i].busy) {
                si = (int)i;
                break;
            }
        if (si < 0) break;
        vbw_status err = VBW_OK;
        const int n = launch_batch(sv, si, &err);
        if (n < 0) return err;
        if (n == 0) break;
    }
    return VBW_OK;
}

static void hand_out(vbw_server_s* sv, vbw_completion* out, int max_out, int* nout)
{
    *nout = 0;
    while (*nout < max_out && !sv->done.empty()) {
        out[(*nout)++] = sv->done.front();
        sv->done.pop_front();
    }
}

extern "C" vbw_status vbw_server_poll(vbw_server_t sv, vbw_completion* out, int max_out, int* nout)
{
    if (!sv || !nout || max_out < 0 || (max_out > 0 && !out)) return fail(VBW_ERR_INVALID_ARG, "bad argument");
    *nout = 0;
    vbw_status s = retire(sv, false);
    if (s == VBW_OK) s = admit(sv);
    hand_out(sv, out, max_out, nout);
    return s == VBW_OK ? ok() : s;
}

extern "C" vbw_status vbw_server_wait(vbw_server_t sv, vbw_completion* out, int max_out, int* nout)
{
    if (!sv || !nout || max_out < 0 || (max_out > 0 && !out)) return fail(VBW_ERR_INVALID_ARG, "bad argument");
    *nout = 0;
    vbw_status s = admit(sv);
    if (s == VBW_OK && sv->done.empty()) s = retire(sv, true);
    if (s == VBW_OK) s = admit(sv);
    hand_out(sv, out, max_out, nout);
    return s == VBW_OK ? ok() : s;
}

extern "C" vbw_status vbw_server_info(vbw_server_t sv, vbw_server_stats* out)
{
    if (!sv || !out) return fail(VBW_ERR_INVALID_ARG, "NULL argument");
    out->queued = (int64_t)sv->queue.size();
    out->inflight_batches = (int64_t)sv->inflight.size();
    out->completions_ready = (int64_t)sv->done.size();
    out->batches = sv->batches;
    out->launches = sv->launches;
    out->admitted = sv->admitted;
    out->slot_bytes = sv->slots.empty() ? 0 : (int64_t)sv->slots[0].bytes;
    out->slots = (int64_t)sv->slots.size();
    return ok();
}

extern "C" double vbw_server_clock(void) { return now_s(); }

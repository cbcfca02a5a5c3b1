// Overlap-add (OLA) VBW filtering: the other fast-convolution method of Sec. I, with the same
// coefficients (eq. (FS_Hk_exp), eq. (FS_Hk_real)) and the same steps 1-3 of Sec. II as the OLS
// path. Block m takes the M = N - O input samples x(mM .. mM + M - 1), zero padded to N; its N
// outputs z_m(0..N-1) overlap the next block's by O samples and are added:
//     y(mM + n) = z_m(n) + z_{m-1}(n + M)   (n < O),     y(mM + n) = z_m(n)   (O <= n < M),
// which needs M >= O (only the previous block overlaps). The linear phase of eq. (FS_Hk_exp) is
// the circular shift z_m(n) = z'((n - D) mod N), D = O/2, of the zero-phase result z', as in the
// OLS kernel; even overlaps only.
//
// Work split as in the OLS kernel (ols_fp32.cuh): a warp takes a contiguous range of warp-tiles of
// B = 32/T consecutive blocks, one lane group per block, with the same gather -> four-step DFT ->
// gains -> inverse DFT body. The tail z_m(M..N-1) of each block waits in a per-warp shared-memory
// slot for the next block:
//   * B = 1 (N >= 1024): one slot. A block first adds the previous block's tail in place, then,
//     after a warp barrier, leaves its own.
//   * B > 1: B + 1 slots indexed by m mod (B + 1). Every lane group leaves its tail first; after a
//     warp barrier each adds its predecessor's (the previous lane group's, or for the first lane
//     group the previous tile's last one, whose slot this tile does not reuse).
// A warp whose range starts inside a signal first runs the preceding tile for its tails only.
// Each tile also asks L2 for the next tile's input span (one bulk prefetch), as the OLS kernel does.
// For overlap N/4 (every workload's geometry) D = N/8 is a whole number of register rows, so the
// position of every register and the carry / tail / store tests are compile-time; other even
// overlaps compute them at run time.
// Nothing is stored per band: the gains come from (k1, V) through the per-lane-group table.
#include "ols_fp32.cuh"
#include "vbw_internal.h"

namespace vbw {
namespace {

struct OlaArgs {
    const float2* in;        // nsignals x nsamples
    float2* out;             // nsignals x nsamples
    const int32_t* band;     // nsignals x nblocks k1 per block, or null (band0 everywhere)
    int64_t nsamples, nblocks, tiles_per_signal, ntiles;
    const float2* tw;        // plan twiddle rows
    const float* V;
    int32_t band0, O, LV;
    int32_t slot_bytes;      // shared bytes of one tail slot (O float2, 16-byte multiple)
};

template <int N>
struct OlaGeom {
    static constexpr int B = OlsGeom<N>::B;
    static constexpr int SLOTS = (B == 1) ? 1 : B + 1;
};

// One warp-tile: blocks tl B .. tl B + B - 1 of signal sig. prime: only leave the tails (the
// warp's range starts inside the signal and the next tile needs its predecessor's tail).
// QOVL: the overlap is N/4, so D = N/8 is a whole number E/8 of register rows and every position
// test below is a compile-time row test; otherwise positions are computed at run time.
template <int N, bool QOVL>
__device__ __forceinline__ void ola_tile(const OlaArgs& a, int64_t sig, int64_t tl, bool prime, bool has_next,
                                         const float2* tw_s, unsigned char* wbase, int lane, int& table_key)
{
    using G = OlsGeom<N>;
    constexpr int E = G::E, T = G::T, B = G::B, SLOTS = OlaGeom<N>::SLOTS;
    const int bsub = lane / T, t = lane % T;
    float2* buf = reinterpret_cast<float2*>(wbase + G::BUF_OFF) + bsub * G::BLK;
    float* gtab = reinterpret_cast<float*>(wbase + G::GAIN_OFF) + bsub * G::GT;
    unsigned char* slots = wbase + G::WARP_BYTES;
    const float4* twrow = reinterpret_cast<const float4*>(tw_s + t * G::TWROW);
    const int O = QOVL ? N / 4 : a.O, M = N - O, D = O >> 1;

    const int64_t blk = tl * B + bsub;
    const bool active = blk < a.nblocks;
    const float2* in = a.in + sig * a.nsamples;
    const int64_t s0 = blk * (int64_t)M;

    // ---- gather u_m(i) = x(mM + i), i = T n1 + t < M; zero padding above M and past the end
    float2 x[E];
    if (__all_sync(0xffffffffu, active && s0 + M <= a.nsamples)) {
        const float2* sp = in + s0 + t;
        static_for<0, E>([&](auto n1) {
            constexpr int N1 = decltype(n1)::value;
            constexpr int K = N1 * T;
            if constexpr (QOVL) x[n1] = (N1 < 3 * E / 4) ? ld_stream(sp + K) : make_float2(0.f, 0.f);
            else x[n1] = (K + t < M) ? ld_stream(sp + K) : make_float2(0.f, 0.f);
        });
    } else {
        static_for<0, E>([&](auto n1) {
            const int i = decltype(n1)::value * T + t;
            x[n1] = (active && i < M && s0 + i < a.nsamples) ? ld_stream(in + s0 + i) : make_float2(0.f, 0.f);
        });
    }

    // ---- ask L2 for the next tile's input span (B M samples after this tile's), one bulk
    //      prefetch from a 16-byte aligned start
    if (lane == 0 && has_next) {
        int64_t e = (tl + 1) * (int64_t)B * M;
        int64_t e2 = e + (int64_t)B * M;
        if (e2 > a.nsamples) e2 = a.nsamples;
        if ((reinterpret_cast<uintptr_t>(in + e) & 15) != 0) ++e;
        const int64_t cnt = (e2 - e) & ~int64_t(1);
        if (cnt > 0) prefetch_l2_bulk(in + e, (uint32_t)(cnt * sizeof(float2)));
    }

    // ---- gain table for this block's band (re-indexing only: eq. (FS_Hk_real))
    const int k1 = active ? (a.band ? a.band[sig * a.nblocks + blk] : a.band0) : 0;
    const int key = active ? k1 : table_key;
    if (__any_sync(0xffffffffu, key != table_key)) {
        __syncwarp();
        if (active) build_gains<N>(gtab, t, k1, a.LV, a.V);
        table_key = key;
        __syncwarp();
    }

#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        four_step_dft<N>(x, buf, twrow, t);
        if (pass == 0) {
            const uint32_t lo = smem_u32(gtab + t);
            const uint32_t hi = smem_u32(gtab + (N - t));
            static_for<0, E>([&](auto n1) {
                constexpr int N1 = decltype(n1)::value;
                constexpr int K = N1 * T;
                const float gk = (N1 < E / 2) ? lds_f32(lo + 4 * K) : lds_f32(hi - 4 * K);
                x[n1] = make_float2(gk * x[n1].y, gk * x[n1].x);
            });
        }
    }
    // z_m(n) = swap(x[n1]) at n = (T n1 + t + D) mod N. The position base t + D and the block's
    // coordinates are formed here, after the passes, through an opaque value, so that nothing of
    // them is held in registers across the transforms.
    int base = t + D;
    asm volatile("" : "+r"(base));
    const int64_t bk = tl * B + bsub;
    const int slot = (SLOTS == 1) ? 0 : (int)(bk % SLOTS);
    float2* own = reinterpret_cast<float2*>(slots + (size_t)slot * a.slot_bytes);
    // position of register row n1: n = (T n1 + t + D) mod N; for QOVL the row (n1 + E/8) mod E
    auto pos = [&](int n1) {
        int n = n1 * T + base;
        return n >= N ? n - N : n;
    };
    // is_carry: n < O (the previous block's tail adds here); is_tail: n >= M (left for the next
    // block at n - M); is_kept: n < M (stored)
    auto body = [&](auto n1, auto&& on_carry, auto&& on_tail, auto&& on_kept) {
        constexpr int N1 = decltype(n1)::value;
        if constexpr (QOVL) {
            constexpr int r = (N1 + E / 8) % E;
            if constexpr (r < E / 4) on_carry(r * T + t);
            if constexpr (r >= 3 * E / 4) on_tail((r - 3 * E / 4) * T + t);
            if constexpr (r < 3 * E / 4) on_kept(r * T + t);
        } else {
            const int n = pos(N1);
            if (n < O) on_carry(n);
            if (n >= M) on_tail(n - M);
            if (n < M) on_kept(n);
        }
    };
    auto none = [](int) {};
    auto leave_tail = [&](auto n1) {
        body(n1, none, [&](int i) { own[i] = make_float2(x[n1].y, x[n1].x); }, none);
    };
    auto add_from = [&](const float2* src, auto n1) {
        body(n1, [&](int i) {
            const float2 c = src[i];
            x[n1].y += c.x;
            x[n1].x += c.y;
        }, none, none);
    };
    if constexpr (SLOTS == 1) {
        // add the previous block's tail z_{m-1}(n + M), n < O, in place; then leave this one's
        if (!prime && bk > 0) static_for<0, E>([&](auto n1) { add_from(own, n1); });
        __syncwarp();
        static_for<0, E>([&](auto n1) { leave_tail(n1); });
        __syncwarp();
    } else {
        // leave this block's tail, then add the predecessor's (slot (m - 1) mod (B + 1))
        static_for<0, E>([&](auto n1) { leave_tail(n1); });
        __syncwarp();
        if (!prime && bk > 0) {
            const int ps = (int)((bk + SLOTS - 1) % SLOTS);
            const float2* prev = reinterpret_cast<const float2*>(slots + (size_t)ps * a.slot_bytes);
            static_for<0, E>([&](auto n1) { add_from(prev, n1); });
        }
        __syncwarp();
    }
    if (prime || bk >= a.nblocks) return;

    // ---- store y(mM + n), n < M (Sec. II step 5 with the overlap added)
    const int64_t so = bk * (int64_t)M;
    float2* out = a.out + sig * a.nsamples + so;
    const int64_t lim = a.nsamples - so;
    if (lim >= M) {
        static_for<0, E>([&](auto n1) {
            body(n1, none, none, [&](int n) { st_stream(out + n, make_float2(x[n1].y, x[n1].x)); });
        });
    } else {
        static_for<0, E>([&](auto n1) {
            body(n1, none, none, [&](int n) {
                if (n < lim) st_stream(out + n, make_float2(x[n1].y, x[n1].x));
            });
        });
    }
}

template <int N, int WARPS, bool QOVL>
__global__ void __launch_bounds__(WARPS * 32) ola_fp32_kernel(const OlaArgs a)
{
    using G = OlsGeom<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tw_s = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t warp_bytes = G::WARP_BYTES + (size_t)OlaGeom<N>::SLOTS * a.slot_bytes;
    unsigned char* wbase = smem_raw + sizeof(float2) * G::TW + (size_t)warp * warp_bytes;
    for (int i = threadIdx.x; i < G::TW / 2; i += blockDim.x)
        reinterpret_cast<float4*>(tw_s)[i] = reinterpret_cast<const float4*>(a.tw)[i];
    __syncthreads();

    int table_key = -1;
    int64_t tb, te;
    warp_range(a.ntiles, (int64_t)gridDim.x * WARPS, (int64_t)blockIdx.x * WARPS + warp, tb, te);
    if (tb >= te) return;
    // (signal, tile within it) of the range's first tile, stepped without divisions below; a
    // range that starts inside a signal first runs the preceding tile for its tails only
    int64_t sig = tb / a.tiles_per_signal;
    int64_t tl = tb - sig * a.tiles_per_signal;
    int64_t tile = tb;
    bool prime = tl != 0;
    if (prime) { --tl; --tile; }
#pragma unroll 1
    for (; tile < te; ++tile) {
        ola_tile<N, QOVL>(a, sig, tl, prime, tile + 1 < te, tw_s, wbase, lane, table_key);
        prime = false;
        if (++tl == a.tiles_per_signal) { tl = 0; ++sig; }
    }
}

template <int N>
cudaError_t launch_ola(const OlaArgs& a, int sms, cudaStream_t st)
{
    // 8-warp CTAs; N = 512 takes 4-warp CTAs, three of which fit the shared memory of an SM (two
    // lane groups' transpose buffers and three tail slots per warp)
    constexpr int WARPS = (N == 512) ? 4 : 8;
    using G = OlsGeom<N>;
    const size_t smem = sizeof(float2) * G::TW + (size_t)WARPS * (G::WARP_BYTES +
                        (size_t)OlaGeom<N>::SLOTS * a.slot_bytes);
    auto kern = (a.O == N / 4) ? ola_fp32_kernel<N, WARPS, true> : ola_fp32_kernel<N, WARPS, false>;
    int per_sm = 0;
    cudaError_t e = prepared_occupancy((const void*)kern, WARPS * 32, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t need = (a.ntiles + WARPS - 1) / WARPS;
    const int64_t cap = (int64_t)per_sm * sms;
    const int grid = (int)(need < cap ? need : cap);
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, WARPS * 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace
}  // namespace vbw

using namespace vbw;

extern "C" vbw_status vbw_filter_ola(vbw_plan_t plan, const void* in, void* out, int64_t nsamples,
                                     int nsignals, int band, const int* band_per_block, void* cuda_stream)
{
    if (!plan) return fail(VBW_ERR_INVALID_ARG, "vbw_filter_ola: null plan");
    if (plan->prec != VBW_PREC_FP32)
        return fail(VBW_ERR_UNSUPPORTED, "vbw_filter_ola: FP32 plans only");
    if ((plan->O & 1) || plan->O > plan->N / 2)
        return fail(VBW_ERR_UNSUPPORTED, "vbw_filter_ola: overlap %d must be even and at most N/2", plan->O);
    if (nsamples < 0 || nsignals < 0) return fail(VBW_ERR_INVALID_ARG, "vbw_filter_ola: negative size");
    if (nsamples == 0 || nsignals == 0) return ok();
    if (!band_per_block) {
        const vbw_status st = check_band(plan, band);
        if (st != VBW_OK) return st;
    }
    if (!in || !out) return fail(VBW_ERR_INVALID_ARG, "vbw_filter_ola: null signal pointer");
    if (misaligned(in) || misaligned(out) || (reinterpret_cast<uintptr_t>(band_per_block) & 3))
        return fail(VBW_ERR_INVALID_ARG, "vbw_filter_ola: misaligned pointer");
    const int64_t total = nsamples * (int64_t)nsignals;
    const uintptr_t ib = reinterpret_cast<uintptr_t>(in), ob = reinterpret_cast<uintptr_t>(out);
    const uintptr_t bytes = (uintptr_t)total * 8;
    if (ib < ob + bytes && ob < ib + bytes)
        return fail(VBW_ERR_INVALID_ARG, "vbw_filter_ola: input and output overlap");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device)
        return fail(VBW_ERR_INVALID_ARG, "vbw_filter_ola: the plan's device is not the current device");
    const int M = plan->N - plan->O;
    const int B = 32 / layout_T(plan->N);
    OlaArgs a{};
    a.in = static_cast<const float2*>(in);
    a.out = static_cast<float2*>(out);
    a.band = band_per_block;
    a.nsamples = nsamples;
    a.nblocks = (nsamples + M - 1) / M;
    a.tiles_per_signal = (a.nblocks + B - 1) / B;
    a.ntiles = a.tiles_per_signal * nsignals;
    a.tw = plan->d_tw;
    a.V = plan->d_V;
    a.band0 = band;
    a.O = plan->O;
    a.LV = plan->LV;
    a.slot_bytes = (int)(((size_t)plan->O * sizeof(float2) + 15) / 16 * 16);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e;
    switch (plan->N) {
    case 128: e = launch_ola<128>(a, plan->sms, st); break;
    case 256: e = launch_ola<256>(a, plan->sms, st); break;
    case 512: e = launch_ola<512>(a, plan->sms, st); break;
    case 1024: e = launch_ola<1024>(a, plan->sms, st); break;
    case 2048: e = launch_ola<2048>(a, plan->sms, st); break;
    default: return fail(VBW_ERR_INVALID_ARG, "vbw_filter_ola: N=%d", plan->N);
    }
    if (e != cudaSuccess) return fail(VBW_ERR_CUDA, "vbw_filter_ola: launch failed: %s", cudaGetErrorString(e));
    return ok();
}

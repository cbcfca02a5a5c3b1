// Fused FP32 overlap-save VBW kernels: gather -> N-point DFT -> H_R on the fly -> inverse DFT ->
// discard and store, one kernel, one pass over HBM (Sec. II steps 1-5 with eq. (FS_Hk_exp) and
// eq. (FS_Hk_real)).
//
// Four-step DFT, N = E * T, T threads per block, thread t holding x(T n1 + t) in register n1:
//   F1  E-point register DFT over n1                      -> A(ka, t)
//   F2  A(ka, t) *= W_N^{t ka}                            (shared-memory row of thread t)
//   F3  shared-memory transpose: thread t now owns ka = s T + t (s < E/T), every n2
//   F4  T-point register DFTs over n2                     -> X(ka + E k'), k' = 0..T-1
// With n1 = s + (E/T) k' the output index ka + E k' equals T n1 + t: the output layout is the
// input layout. So the inverse DFT reuses the same four steps through
// IDFT(y) = swap(DFT(swap(y))), swap(a + jb) = b + ja, whose swaps are register renaming.
// Between the two passes each register is scaled by its real gain g = H_R(k)/N (k = T n1 + t),
// read from a per-warp table rebuilt only when the band changes; 1/N (eq. (OLS_dn)) is a power of
// two, so the scaling is exact. The linear phase exp(-j 2 pi k D / N), D = O/2, of eq. (FS_Hk_exp)
// is an exact circular shift of the inverse output by D samples: the kept outputs w(O..N-1) of
// Sec. II step 4 are z(D..D+M-1), written to y(mM .. mM+M-1).
#pragma once

#include "fft_reg.cuh"

namespace vbw {

template <int N>
struct OlsGeom {
    static constexpr int E = Layout<N>::E;
    static constexpr int T = Layout<N>::T;
    static constexpr int B = 32 / T;    // blocks per warp
    static constexpr int S = E / T;     // pass-2 DFTs per thread
    // padded transpose row (float2 elements): T + 2 keeps every row 16-byte aligned, so the
    // row side of each transpose moves two samples per 128-bit access, and offsets consecutive
    // rows by 16 bytes mod 128, so those accesses are conflict-free
    static constexpr int ROW = T + 2;
    // N = 2048 (two pass-2 DFTs per thread): the transpose runs in two halves of E/2 rows, which
    // halves the buffer and raises residency from 8 to 12 warps per SM
    static constexpr bool HALF = (N == 2048);
    // per-block transpose buffer; for T = 8 two blocks share a half-warp on the column side, so
    // their buffers are offset by 64 bytes mod 128
    static constexpr int BLK = (HALF ? E / 2 : E) * ROW + ((T == 8) ? 8 : 0);
    // twiddle table row of thread t: W_N^{t ka}, ka = 0..E-1, padded to E + 2
    static constexpr int TWROW = E + 2;
    static constexpr int TW = T * TWROW;
    // per-block gain table g(kk), kk = 0..N/2; when several blocks share a warp their tables are
    // offset by T banks so the lane groups never collide
    static constexpr int GT_MIN = N / 2 + 1;
    static constexpr int GT = (B == 1) ? ((GT_MIN + 3) & ~3)
                                       : GT_MIN + ((T - GT_MIN % 32) % 32 + 32) % 32;
    // per warp: B transpose buffers, then B gain tables
    static constexpr size_t BUF_OFF = 0;
    static constexpr size_t GAIN_OFF = BUF_OFF + sizeof(float2) * B * BLK;
    static constexpr size_t WARP_BYTES = (GAIN_OFF + sizeof(float) * B * GT + 15) / 16 * 16;
    static_assert(E * T == N && E % T == 0, "layout must satisfy N = E*T with T | E");
    static_assert(!HALF || S == 2, "the half transpose assumes two pass-2 DFTs per thread");
    static_assert(BLK % 2 == 0 && T % 2 == 0, "transpose rows must stay 16-byte aligned");
};

// Shared memory of one CTA: twiddles (T rows of E + 2 float2), then per warp the transpose
// buffers and gains.
template <int N>
__host__ __device__ inline size_t ols_smem_bytes(int warps)
{
    return sizeof(float2) * (size_t)OlsGeom<N>::TW + (size_t)warps * OlsGeom<N>::WARP_BYTES;
}

// g(kk) = H_R / N with H_R of eq. (FS_Hk_real) on the non-negative half, kk = 0..N/2:
// kk <= k1 - 1 passband (1), k1 <= kk <= k1 + L_V - 1 transition (V(kk - k1)), else stopband (0).
// 1/N is a power of two, so g * N recovers H_R exactly. Written by the T lanes of one lane group.
// H_R at the non-negative bin kk (0 <= kk <= N/2) for band k1: 1, V(kk - k1) or 0.
__device__ __forceinline__ float hr_gain(int kk, int k1, int LV, const float* V)
{
    const int r = kk - k1;
    return r < 0 ? 1.f : (r < LV ? V[r] : 0.f);
}

template <int N>
__device__ __forceinline__ void build_gains(float* gtab, int t, int k1, int LV, const float* V)
{
    constexpr int T = OlsGeom<N>::T;
    constexpr float inv_n = 1.0f / N;
    for (int kk = t; kk <= N / 2; kk += T) gtab[kk] = hr_gain(kk, k1, LV, V) * inv_n;
}

// L2 prefetch of a contiguous byte range with one bulk-copy instruction (16-byte aligned start,
// size a multiple of 16).
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ---- shared-memory addresses and mbarriers (the tensor-core kernel waits on its MMAs with these)
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// generic-proxy accesses to shared memory made before this point are ordered before later
// async-proxy accesses (the tensor cores' operand reads)
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the mbarrier phase `parity`: gives up after about `limit` SM clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

constexpr long long kWaitLimitCycles = 4000000000LL;   // ~2 s at 2 GHz
constexpr int kStatusWaitTimeout = 1;   // status word bit: a bounded device wait gave up

// Gains for the pass-2 layout: g[s][k'] = H_R(k), k = s T + t + E k'. For k' < T/2, k < N/2;
// otherwise the mirror N - k is used, which makes H_R(N - k) = H_R(k).
template <int N>
__device__ __forceinline__ void load_gains(float (&g)[OlsGeom<N>::S][OlsGeom<N>::T], const float* gtab,
                                           int t)
{
    constexpr int E = OlsGeom<N>::E, T = OlsGeom<N>::T, S = OlsGeom<N>::S;
    const float* lo = gtab + t;
    const float* hi = gtab + (N - t);
    static_for<0, S>([&](auto s) {
        static_for<0, T>([&](auto kp) {
            constexpr int KP = decltype(kp)::value;
            constexpr int base = decltype(s)::value * T + E * KP;
            if constexpr (KP < T / 2) g[s][kp] = lo[base];
            else g[s][kp] = hi[-base];
        });
    });
}

__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldg(p); }
__device__ __forceinline__ void st_stream(float2* p, float2 v) { __stcs(p, v); }

// Returns p unchanged but opaque to the optimizer, so loads through it stay where they are
// written instead of being hoisted out of the loops.
template <class P>
__device__ __forceinline__ P* opaque(P* p)
{
    asm volatile("" : "+l"(p));
    return p;
}

// Shared-memory loads by 32-bit shared address, for tables read inside the tile loop (twiddle
// rows, gains, half-sample phases). The state space is explicit: a load through a pointer the
// compiler cannot trace to shared memory would be a generic load on the L1TEX path. The asm is
// volatile, so each load stays where it is written (its value is not held in registers across
// the DFT passes).
__device__ __forceinline__ float lds_f32(uint32_t a)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ float2 lds_f2(uint32_t a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ float4 lds_f4(uint32_t a)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory");
    return v;
}

// F2 and F3 of the four-step DFT below: the twiddle W_N^{t ka} (row t of the table), then the
// transpose through buf, after which register SS + S k' holds row ka = SS T + t, column n2 = k'.
// TW0: the table's ka = 0 entries are not 1 (a table that carries an extra per-thread factor), so
// F2 multiplies them too; otherwise that multiply is skipped.
template <int N, bool TW0 = false>
__device__ __forceinline__ void four_step_f2f3(float2 (&x)[OlsGeom<N>::E], float2* buf,
                                               const float4* twrow, int t)
{
    using G = OlsGeom<N>;
    constexpr int E = G::E, T = G::T, S = G::S, ROW = G::ROW;
    const uint32_t tr = smem_u32(twrow);
    static_for<0, E / 2>([&](auto kh) {                                      // F2
        constexpr int ka = 2 * decltype(kh)::value;
        const float4 w = lds_f4(tr + 16 * decltype(kh)::value);
        if constexpr (ka != 0 || TW0) x[ka] = cmul(x[ka], make_float2(w.x, w.y));
        x[ka + 1] = cmul(x[ka + 1], make_float2(w.z, w.w));
    });
    if constexpr (!G::HALF) {
        static_for<0, E>([&](auto ka) { buf[decltype(ka)::value * ROW + t] = x[ka]; });   // F3
        __syncwarp();
        static_for<0, S>([&](auto s) {
            constexpr int SS = decltype(s)::value;
            const float4* row = reinterpret_cast<const float4*>(buf + (SS * T + t) * ROW);
            static_for<0, T / 2>([&](auto h) {
                constexpr int H = decltype(h)::value;
                const float4 q = row[h];
                x[SS + S * (2 * H)] = make_float2(q.x, q.y);
                x[SS + S * (2 * H + 1)] = make_float2(q.z, q.w);
            });
        });
        __syncwarp();
    } else {
        // F3 in two halves: rows ka = SS T + r (r < T) pass through the buffer as rows r; thread
        // t then reads row t, i.e. ka = SS T + t, the input of its pass-2 DFT number SS
        float2 half[S][T];
        static_for<0, S>([&](auto s) {
            constexpr int SS = decltype(s)::value;
            static_for<0, T>([&](auto r) { buf[decltype(r)::value * ROW + t] = x[SS * T + decltype(r)::value]; });
            __syncwarp();
            const float4* row = reinterpret_cast<const float4*>(buf + t * ROW);
            static_for<0, T / 2>([&](auto h) {
                constexpr int H = decltype(h)::value;
                const float4 q = row[h];
                half[SS][2 * H] = make_float2(q.x, q.y);
                half[SS][2 * H + 1] = make_float2(q.z, q.w);
            });
            __syncwarp();
        });
        static_for<0, S>([&](auto s) {
            static_for<0, T>([&](auto kp) {
                x[decltype(s)::value + S * decltype(kp)::value] = half[decltype(s)::value][decltype(kp)::value];
            });
        });
    }
}

// One forward N-point four-step DFT on the register array x (see the top of this file):
// in:  x[n1] = u(T n1 + t)
// out: x[n1] = U(T n1 + t)      (with n1 = s + S k', this is X(ka + E k') for ka = s T + t)
// F1 E-point DFT, F2 twiddle, F3 transpose through buf, F4 S T-point DFTs.
template <int N, bool TW0 = false>
__device__ __forceinline__ void four_step_dft(float2 (&x)[OlsGeom<N>::E], float2* buf,
                                              const float4* twrow, int t)
{
    using G = OlsGeom<N>;
    constexpr int E = G::E, T = G::T, S = G::S;
    fft_reg<E, false>(x);                                                    // F1
    four_step_f2f3<N, TW0>(x, buf, twrow, t);                                // F2, F3
    static_for<0, S>([&](auto s) {
        constexpr int SS = decltype(s)::value;
        float2 c[T];
        static_for<0, T>([&](auto kp) { c[kp] = x[SS + S * decltype(kp)::value]; });
        fft_reg<T, false>(c);                                                // F4
        static_for<0, T>([&](auto kp) { x[SS + S * decltype(kp)::value] = c[kp]; });
    });
}

// The fused kernel. Each block is two passes of the same four-step DFT (which keeps the loop body
// small enough for the instruction cache):
//   pass 0: X = DFT(x_m)                                   (Sec. II step 1)
//   pass 1: z = IDFT(H_R X / N) = swap(DFT(swap(H_R X / N)))  (steps 2-3), swap(a + jb) = b + ja,
// where both swaps are free (they only choose which register holds which component). Between the
// passes each register is scaled by its real gain g(kk) = H_R(k)/N, k = T n1 + t, kk = min(k, N-k).
// QOVL: the overlap is N/4 (D = N/8, M = 3N/4) as a compile-time constant; otherwise a.overlap.
#ifndef VBW_MIN_WARPS_PER_SM
#define VBW_MIN_WARPS_PER_SM 0   // 0: no occupancy hint, the compiler chooses the register count
#endif

#if VBW_MIN_WARPS_PER_SM > 0
#define VBW_OLS_BOUNDS(W) __launch_bounds__((W) * 32, (VBW_MIN_WARPS_PER_SM / (W)) > 0 ? VBW_MIN_WARPS_PER_SM / (W) : 1)
#else
#define VBW_OLS_BOUNDS(W) __launch_bounds__((W) * 32)
#endif

// Job sources. A tile reads its descriptor at its start; the store keeps only the output
// pointer, the length and the block index in registers across the DFT passes (complex signals)
// and re-reads the rest through opaque pointers where it is needed.
struct SingleJobSource {        // one stream segment held in the kernel parameters
    const OlsArgs& a;
    template <int B>
    __device__ __forceinline__ void get(int64_t tile, int bsub, OlsJob& job, int64_t& blk) const
    {
        job = a.job;
        blk = tile * B + bsub;
    }
    __device__ __forceinline__ int band(const OlsJob& job, int64_t blk, bool) const
    {
        int k1 = job.band0;
        for (int i = 0; i < a.nchg; ++i)
            if (a.chg_block[i] <= blk) k1 = a.chg_band[i];
        return k1;
    }
};

struct JobListSource {          // device job array + warp-tile list (batches)
    const OlsJob* jobs;
    const int2* tiles;
    template <int B>
    __device__ __forceinline__ void get(int64_t tile, int bsub, OlsJob& job, int64_t& blk) const
    {
        const int2 td = opaque(tiles)[tile];
        job = opaque(jobs)[td.x];
        blk = (int64_t)td.y + bsub;
    }
    __device__ __forceinline__ int band(const OlsJob& job, int64_t blk, bool active) const
    {
        return (job.band && active) ? job.band[blk] : job.band0;
    }
};

// State a warp carries from one tile to the next.
struct WarpState {
    int table_key;        // (plan << 16) | k1 of this lane group's gain table; -1 = none
    int2 ntd;             // job lists: the next tile's (job, first block), read one tile early
    bool ntd_ok;
};

// CARRY (signals in host memory, read over the host link): the last O input samples of a block
// are the first O of the next, and the same thread holds them (rows 3E/4..E-1 become rows
// 0..E/4-1 when the overlap is N/4 and one block fills a warp-tile). They are kept in registers,
// so consecutive blocks of a warp read each input sample from the link once instead of 4/3 times.
template <int NC>
struct CarryState {
    float2 v[NC > 0 ? NC : 1];   // this thread's rows of the last O samples of the previous block
    const float2* in;            // the signal they belong to; nullptr = none
    int64_t blk;                 // the block that starts with them
};

// Per-launch switches of a warp-tile.
struct TileCtl {
    bool bulk;            // bulk L2 prefetch allowed (signals in device memory)
    const float2* half;   // odd overlap: exp(-j pi kk / N), kk = 0..N/2, in shared memory; else null
};

// REAL: the job's signal is real (float32). Each lane group then takes the pair of real blocks
// (2 blk, 2 blk + 1) as one complex block x_{2 blk} + j x_{2 blk + 1}: the filter is real and
// symmetric (eq. (FS_Hk_exp) is conjugate symmetric), so the real part of the result is the
// first block's output and the imaginary part the second's. blk counts pairs, and the band is
// one per pair.
// One warp-tile: 32/T blocks of plan `plan`, transform size N.
template <int N, bool QOVL, class Src, bool REAL = false, bool CARRY = false>
__device__ __forceinline__ void ols_tile(const Src& src, int64_t tile, bool has_next, int plan,
                                         const float2* tw_plan, const float* V, int LV, int O_rt,
                                         unsigned char* wbase, int lane, WarpState& ws,
                                         const TileCtl& ctl,
                                         CarryState<CARRY ? OlsGeom<N>::E / 4 : 0>* cs = nullptr)
{
    using G = OlsGeom<N>;
    constexpr int E = G::E, T = G::T, B = G::B;
    static_assert(!CARRY || (QOVL && !REAL && B == 1), "the carry needs overlap N/4 and one block per warp-tile");
    const int bsub = lane / T, t = lane % T;
    float2* buf = reinterpret_cast<float2*>(wbase + G::BUF_OFF) + bsub * G::BLK;
    float* gtab = reinterpret_cast<float*>(wbase + G::GAIN_OFF) + bsub * G::GT;
    const float4* twrow = reinterpret_cast<const float4*>(tw_plan + t * G::TWROW);
    const int O = QOVL ? N / 4 : O_rt;
    // D: the store shift, ceil(O/2). For odd O the delay O/2 is a half sample: the whole part
    // (O - 1)/2 is a shift and the half sample a phase exp(-j pi k_s / N) on every bin, so the kept
    // outputs start one sample later (z(O + i) of Sec. II steps 4-5 is z'(ceil(O/2) + i))
    const int M = N - O, D = (O + 1) >> 1;
    const int64_t P = REAL ? 2 * (int64_t)M : (int64_t)M;   // input samples per lane-group step
    const int SPAN = REAL ? N + M : N;                      // input samples one step reads

    float2 x[E];
    float2* kout;              // kept for the store (complex signals)
    int64_t knsamp, kblk;
    {
        // ---- which job and block this lane group works on, and its band
        OlsJob job;
        int64_t blk;
        if constexpr (std::is_same<Src, JobListSource>::value) {
            // the tile list entry was read one tile early: the descriptor read starts at once
            const int2 td = ws.ntd_ok ? ws.ntd : opaque(src.tiles)[tile];
            job = opaque(src.jobs)[td.x];
            blk = (int64_t)td.y + bsub;
            ws.ntd_ok = has_next;
            if (has_next) ws.ntd = opaque(src.tiles)[tile + 1];
        } else {
            src.template get<B>(tile, bsub, job, blk);
        }
        const int64_t nsamp = job.nsamp;
        kout = job.out;
        knsamp = nsamp;
        kblk = blk;
        const bool active = blk * P < nsamp;
        const int k1 = src.band(job, blk, active);
        const int key = active ? ((plan << 16) | k1) : ws.table_key;

        // ---- gather x_m(n) = x(mM - O + n), n = T n1 + t (Sec. II segmentation), coalesced
        //      loads from L2 (the span was prefetched by the warp's previous tile). They are issued
        //      first; the prefetch and the gain table below overlap their latency.
        const int64_t s0 = blk * P - O;
        const bool interior = active && s0 >= 0 && s0 + SPAN <= nsamp;
        if constexpr (REAL) {
            // x(n) = u(s0 + n) + j u(s0 + M + n): the pair's two blocks
            const float* in_r = reinterpret_cast<const float*>(job.in);
            const float* tl_r = reinterpret_cast<const float*>(job.tail_in);
            if (__all_sync(0xffffffffu, interior)) {
                const float* sp = in_r + s0 + t;
                static_for<0, E>([&](auto n1) {
                    constexpr int K = decltype(n1)::value * T;
                    x[n1] = make_float2(__ldg(sp + K), __ldg(sp + M + K));
                });
            } else {
                auto fr = [&](int64_t si) {
                    float v = 0.f;
                    if (active) {
                        if (si >= 0) {
                            if (si < nsamp) v = __ldg(in_r + si);
                        } else if (tl_r) {
                            v = tl_r[O + si];
                        }
                    }
                    return v;
                };
                static_for<0, E>([&](auto n1) {
                    const int64_t si = s0 + decltype(n1)::value * T + t;
                    x[n1] = make_float2(fr(si), fr(si + M));
                });
            }
        } else if (__all_sync(0xffffffffu, interior)) {
            const float2* sp = job.in + s0 + t;
            if constexpr (CARRY) {
                // the block's first O samples are the previous block's last O (same warp, same rows)
                if (cs->in == job.in && cs->blk == blk) {
                    static_for<0, E / 4>([&](auto n1) { x[n1] = cs->v[n1]; });
                    static_for<E / 4, E>([&](auto n1) { x[n1] = ld_stream(sp + decltype(n1)::value * T); });
                } else {
                    static_for<0, E>([&](auto n1) { x[n1] = ld_stream(sp + decltype(n1)::value * T); });
                }
            } else {
                static_for<0, E>([&](auto n1) { x[n1] = ld_stream(sp + decltype(n1)::value * T); });
            }
        } else {
            static_for<0, E>([&](auto n1) {
                const int64_t si = s0 + decltype(n1)::value * T + t;
                float2 v = make_float2(0.f, 0.f);
                if (active) {
                    if (si >= 0) {
                        if (si < nsamp) v = ld_stream(job.in + si);
                    } else if (job.tail_in) {
                        v = job.tail_in[O + si];
                    }
                }
                x[n1] = v;
            });
        }

        if constexpr (CARRY) {
            // samples M .. N-1 of this span (rows 3E/4 .. E-1) open the next block's span
            static_for<0, E / 4>([&](auto i) { cs->v[i] = x[3 * E / 4 + decltype(i)::value]; });
            cs->in = active ? job.in : nullptr;
            cs->blk = blk + 1;
        }

        // ---- ask L2 for the samples the warp's next tile adds (the rest is this span). The bulk
        //      prefetch needs a 16-byte aligned start and a multiple of 16 bytes: a stream whose
        //      base is only 8-byte aligned starts one sample later.
        if (lane == 0 && has_next && ctl.bulk) {
            if constexpr (REAL) {
                const float* in_r = reinterpret_cast<const float*>(job.in);
                int64_t e = (blk + B - 1) * P - O + SPAN;
                int64_t e2 = e + (int64_t)B * P;
                if (e2 > nsamp) e2 = nsamp;
                while (e >= 0 && e < e2 && (reinterpret_cast<uintptr_t>(in_r + e) & 15) != 0) ++e;
                const int64_t cnt = (e2 - e) & ~int64_t(3);
                if (e >= 0 && cnt > 0 && (reinterpret_cast<uintptr_t>(in_r + e) & 15) == 0)
                    prefetch_l2_bulk(in_r + e, (uint32_t)(cnt * sizeof(float)));
            } else {
                int64_t e = (blk + B - 1) * (int64_t)M - O + N;
                int64_t e2 = e + (int64_t)B * M;
                if (e2 > nsamp) e2 = nsamp;
                if (e >= 0 && (reinterpret_cast<uintptr_t>(job.in + e) & 15) != 0) ++e;
                const int64_t cnt = (e2 - e) & ~int64_t(1);
                if (e >= 0 && cnt > 0 && (reinterpret_cast<uintptr_t>(job.in + e) & 15) == 0)
                    prefetch_l2_bulk(job.in + e, (uint32_t)(cnt * sizeof(float2)));
            }
        }

        // ---- gain table for this block's band (re-indexing only: eq. (FS_Hk_real))
        if (__any_sync(0xffffffffu, key != ws.table_key)) {
            __syncwarp();
            if (active) build_gains<N>(gtab, t, k1, LV, V);
            ws.table_key = key;
            __syncwarp();
        }
    }

#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        four_step_dft<N>(x, buf, twrow, t);
        if (pass == 0) {
            // swap(g X): H_R(k)/N of eq. (FS_Hk_real) for k = T n1 + t (Sec. II step 2)
            const uint32_t lo = smem_u32(gtab + t);
            const uint32_t hi = smem_u32(gtab + (N - t));
            bool odd = false;
            if constexpr (!QOVL) odd = ctl.half != nullptr;
            if (!odd) {
                static_for<0, E>([&](auto n1) {
                    constexpr int N1 = decltype(n1)::value;
                    constexpr int K = N1 * T;
                    const float gk = (N1 < E / 2) ? lds_f32(lo + 4 * K) : lds_f32(hi - 4 * K);
                    x[n1] = make_float2(gk * x[n1].y, gk * x[n1].x);
                });
            } else {
                // the half-sample phase of eq. (FS_Hk_exp) with the signed bin k_s: the table's
                // exp(-j pi k / N) below N/2, its conjugate at the mirror bin N - k above
                const uint32_t plo = smem_u32(ctl.half + t);
                const uint32_t phi = smem_u32(ctl.half + (N - t));
                static_for<0, E>([&](auto n1) {
                    constexpr int N1 = decltype(n1)::value;
                    constexpr int K = N1 * T;
                    float gk;
                    float2 c;
                    if constexpr (N1 < E / 2) {
                        gk = lds_f32(lo + 4 * K);
                        c = lds_f2(plo + 8 * K);
                    } else {
                        gk = lds_f32(hi - 4 * K);
                        const float2 m = lds_f2(phi - 8 * K);
                        c = make_float2(m.x, -m.y);
                    }
                    const float2 v = cmul(x[n1], c);
                    x[n1] = make_float2(gk * v.y, gk * v.x);
                });
            }
        }
    }

    // ---- discard and store (steps 4-5): z(n) = swap(x[n1]), n = T n1 + t, kept for
    //      D <= n < D + M (the exp(-j 2 pi k D / N) phase of eq. (FS_Hk_exp) as a shift)
    if constexpr (REAL) {
        OlsJob job;
        int64_t blk;
        src.template get<B>(tile, bsub, job, blk);
        const int64_t nsamp = job.nsamp;
        // z(n) = swap(x[n1]): Re z -> block 2 blk, Im z -> block 2 blk + 1, kept D <= n < D + M
        if (blk * P < nsamp) {
            float* out_r = reinterpret_cast<float*>(job.out);
            const int64_t ob = blk * P - D;
            const bool full = blk * P + P <= nsamp;
            static_for<0, E>([&](auto n1) {
                constexpr int N1 = decltype(n1)::value;
                const int n = N1 * T + t;
                const bool kept = QOVL ? (N1 >= E / 8 && N1 < 7 * E / 8) : (n >= D && n < D + M);
                if (kept) {
                    const int64_t oa = ob + n, obb = ob + M + n;
                    if (full || oa < nsamp) __stcs(out_r + oa, x[n1].y);
                    if (full || obb < nsamp) __stcs(out_r + obb, x[n1].x);
                }
            });
            if ((blk + 1) * P >= nsamp && job.tail_out) {
                const float* in_r = reinterpret_cast<const float*>(job.in);
                const float* tl_r = reinterpret_cast<const float*>(job.tail_in);
                float* to_r = reinterpret_cast<float*>(job.tail_out);
                for (int i = t; i < O; i += T) {
                    const int64_t si = nsamp - O + i;
                    float v = 0.f;
                    if (si >= 0) v = in_r[si];
                    else if (tl_r) v = tl_r[O + si];
                    to_r[i] = v;
                }
            }
        }
        return;
    }
    const int64_t blk = kblk;
    const int64_t nsamp = knsamp;
    if (blk * M < nsamp) {
        const int64_t obase = blk * M - D;
        if constexpr (QOVL) {
            // kept rows n1 in [E/8, 7E/8): every lane stores, no per-sample test when the block
            // is complete
            float2* dst = kout + obase + t;
            if (obase + D + M <= nsamp) {
                static_for<E / 8, 7 * E / 8>([&](auto n1) {
                    st_stream(dst + decltype(n1)::value * T, make_float2(x[n1].y, x[n1].x));
                });
            } else {
                static_for<E / 8, 7 * E / 8>([&](auto n1) {
                    const int64_t oi = obase + decltype(n1)::value * T + t;
                    if (oi < nsamp) st_stream(kout + oi, make_float2(x[n1].y, x[n1].x));
                });
            }
        } else {
            static_for<0, E>([&](auto n1) {
                const int n = decltype(n1)::value * T + t;
                if (n >= D && n < D + M) {
                    const int64_t oi = obase + n;
                    if (oi < nsamp) st_stream(kout + oi, make_float2(x[n1].y, x[n1].x));
                }
            });
        }
        // the lane group of the job's last block hands the stream's last O input samples on
        if ((blk + 1) * M >= nsamp) {
            OlsJob job;
            int64_t bj;
            src.template get<B>(tile, bsub, job, bj);
            if (job.tail_out) {
                for (int i = t; i < O; i += T) {
                    const int64_t si = nsamp - O + i;
                    float2 v = make_float2(0.f, 0.f);
                    if (si >= 0) v = job.in[si];
                    else if (job.tail_in) v = job.tail_in[O + si];
                    job.tail_out[i] = v;
                }
            }
        }
    }
}

// Contiguous range of warp-tiles of warp gw out of nwarps.
__device__ __forceinline__ void warp_range(int64_t ntiles, int64_t nwarps, int64_t gw, int64_t& b, int64_t& e)
{
    const int64_t per = ntiles / nwarps, extra = ntiles % nwarps;
    b = gw * per + (gw < extra ? gw : extra);
    e = b + per + (gw < extra ? 1 : 0);
}

// Single-plan kernel: every tile has the same N (one stream, or a batch grouped by plan).
// Each warp takes one contiguous range of tiles, so consecutive blocks of a stream stay in one
// warp: the overlap samples are L2 hits and the gain table survives until the band changes.
// QOVL: the overlap is N/4 (D = N/8, M = 3N/4) as a compile-time constant; otherwise a.overlap.
template <int N, int WARPS, bool QOVL, bool BATCH, bool REAL = false, bool CARRY = false>
__device__ __forceinline__ void ols_fp32_body(const OlsArgs& a)
{
    using G = OlsGeom<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tw_s = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // odd overlap: the plan's half-sample phase table follows its twiddle rows
    const int ph_len = (!QOVL && (a.overlap & 1)) ? half_phase_entries(N) : 0;
    unsigned char* wbase = smem_raw + sizeof(float2) * (G::TW + ph_len) + (size_t)warp * G::WARP_BYTES;

    // job lists: the warp's first tile-list entry is read before the twiddle rows are copied, so
    // the two reads overlap (the tile loop takes it as its one-tile-ahead entry)
    int64_t tb, te;
    warp_range(a.ntiles, (int64_t)gridDim.x * WARPS, (int64_t)blockIdx.x * WARPS + warp, tb, te);
    WarpState ws{-1, make_int2(0, 0), false};
    if constexpr (BATCH) {
        if (tb < te) {
            ws.ntd = opaque(a.tiles)[tb];
            ws.ntd_ok = true;
        }
    }
    for (int i = threadIdx.x; i < (G::TW + ph_len) / 2; i += blockDim.x)
        reinterpret_cast<float4*>(tw_s)[i] = reinterpret_cast<const float4*>(a.tw)[i];
    __syncthreads();

    const TileCtl ctl{(a.flags & kOlsNoBulk) == 0, ph_len ? tw_s + G::TW : nullptr};
    CarryState<CARRY ? G::E / 4 : 0> cs;
    cs.in = nullptr;
    cs.blk = -1;
    for (int64_t tile = tb; tile < te; ++tile) {
        if constexpr (BATCH)
            ols_tile<N, QOVL, JobListSource, REAL, CARRY>(JobListSource{a.jobs, a.tiles}, tile, tile + 1 < te, 0,
                                                          tw_s, a.V, a.LV, a.overlap, wbase, lane, ws, ctl, &cs);
        else
            ols_tile<N, QOVL>(SingleJobSource{a}, tile, tile + 1 < te, 0, tw_s, a.V, a.LV, a.overlap,
                              wbase, lane, ws, ctl);
    }
}

template <int N, int WARPS, bool QOVL, bool BATCH, bool REAL = false, bool CARRY = false>
__global__ void VBW_OLS_BOUNDS(WARPS) ols_fp32_kernel(const OlsArgs a)
{
    ols_fp32_body<N, WARPS, QOVL, BATCH, REAL, CARRY>(a);
}

// N = 2048: registers capped so that three 4-warp CTAs (12 warps) are resident per SM
template <int WARPS, bool QOVL, bool BATCH, bool REAL = false>
__global__ void __launch_bounds__(WARPS * 32, (12 / WARPS) > 0 ? 12 / WARPS : 1) ols_fp32_kernel_2048(const OlsArgs a)
{
    ols_fp32_body<2048, WARPS, QOVL, BATCH, REAL>(a);
}

// Mixed-plan persistent kernel: one launch over a tile list whose jobs use different plans with
// N <= MAXN and overlap N/4. Every plan's twiddle rows sit in shared memory; a warp switches the
// transform size per tile (jobs are grouped by plan, so a warp's contiguous range crosses few
// plan boundaries).
template <int MAXN, int WARPS>
__global__ void VBW_OLS_BOUNDS(WARPS) ols_mixed_kernel(const MixedArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int p = 0; p < a.nplans; ++p) {
        float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float2*>(smem_raw) + a.plans[p].tw_off);
        const float4* srcp = reinterpret_cast<const float4*>(a.plans[p].tw);
        for (int i = threadIdx.x; i < a.plans[p].tw_len / 2; i += blockDim.x) dst[i] = srcp[i];
    }
    unsigned char* wbase = smem_raw + a.tw_bytes + (size_t)warp * a.warp_bytes;
    __syncthreads();

    const JobListSource src{a.jobs, a.tiles};
    const TileCtl ctl{(a.flags & kOlsNoBulk) == 0, nullptr};
    WarpState ws{-1, make_int2(0, 0), false};
    int64_t tb, te;
    warp_range(a.ntiles, (int64_t)gridDim.x * WARPS, (int64_t)blockIdx.x * WARPS + warp, tb, te);
    for (int64_t tile = tb; tile < te; ++tile) {
        const int2 td = opaque(a.tiles)[tile];
        const int plan = opaque(a.jobs)[td.x].plan;
        const MixedPlan& P = a.plans[plan];
        const float2* tw = reinterpret_cast<const float2*>(smem_raw) + P.tw_off;
        const bool nx = tile + 1 < te;
        switch (P.N) {
        case 128: ols_tile<128, true>(src, tile, nx, plan, tw, P.V, P.LV, 32, wbase, lane, ws, ctl); break;
        case 256: ols_tile<256, true>(src, tile, nx, plan, tw, P.V, P.LV, 64, wbase, lane, ws, ctl); break;
        case 512: ols_tile<512, true>(src, tile, nx, plan, tw, P.V, P.LV, 128, wbase, lane, ws, ctl); break;
        default:
            if constexpr (MAXN >= 1024) {
                if (P.N == 1024) { ols_tile<1024, true>(src, tile, nx, plan, tw, P.V, P.LV, 256, wbase, lane, ws, ctl); break; }
            }
            if constexpr (MAXN >= 2048) {
                if (P.N == 2048) { ols_tile<2048, true>(src, tile, nx, plan, tw, P.V, P.LV, 512, wbase, lane, ws, ctl); break; }
            }
            break;
        }
    }
}

// Writes the H_R(k) that the kernel applies for band k1 (test hook): the same table build and
// the same load_gains indexing, one lane group of T threads; the table's 1/N is undone exactly.
template <int N>
__global__ void export_hr_kernel(const float* V, int LV, int k1, float* out)
{
    using G = OlsGeom<N>;
    constexpr int E = G::E, T = G::T, S = G::S;
    __shared__ float gtab[G::GT];
    const int t = threadIdx.x;
    if (t < T) build_gains<N>(gtab, t, k1, LV, V);
    __syncthreads();
    if (t >= T) return;
    float g[S][T];
    load_gains<N>(g, gtab, t);
    static_for<0, S>([&](auto s) {
        static_for<0, T>([&](auto kp) {
            out[decltype(s)::value * T + t + E * decltype(kp)::value] = g[s][kp] * (float)N;
        });
    });
}

// Launch helpers (instantiated per N in ols_fp32_n<N>.cu).
template <class Kern>
cudaError_t launch_persistent(Kern kern, int warps, size_t smem, int64_t ntiles, int sms, int max_ctas,
                              cudaStream_t st, int* grid_out, const void* arg_ptr)
{
    int per_sm = 0;
    cudaError_t e = prepared_occupancy((const void*)kern, warps * 32, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t ctas_needed = (ntiles + warps - 1) / warps;
    int64_t cap = (int64_t)per_sm * sms;
    if (max_ctas > 0 && cap > max_ctas) cap = max_ctas;
    const int grid = (int)(ctas_needed < cap ? ctas_needed : cap);
    if (grid_out) *grid_out = grid;
    if (grid <= 0) return cudaSuccess;
    void* args[] = {const_cast<void*>(arg_ptr)};
    return cudaLaunchKernel((const void*)kern, dim3(grid), dim3(warps * 32), args, smem, st);
}

template <int N, int WARPS, bool QOVL, bool BATCH, bool REAL = false, bool CARRY = false>
cudaError_t launch_ols_fp32_w(const OlsArgs& a, int sms, int max_ctas, cudaStream_t st, int* grid_out)
{
    const size_t smem = ols_smem_bytes<N>(WARPS) +
                        ((!QOVL && (a.overlap & 1)) ? sizeof(float2) * half_phase_entries(N) : 0);
    if constexpr (N == 2048)
        return launch_persistent(ols_fp32_kernel_2048<WARPS, QOVL, BATCH, REAL>, WARPS, smem, a.ntiles, sms,
                                 max_ctas, st, grid_out, &a);
    else
        return launch_persistent(ols_fp32_kernel<N, WARPS, QOVL, BATCH, REAL, CARRY>, WARPS, smem, a.ntiles,
                                 sms, max_ctas, st, grid_out, &a);
}

template <int N>
cudaError_t launch_ols_fp32(const OlsArgs& a, int warps, int sms, int max_ctas, cudaStream_t st, int* grid_out)
{
    const bool q = (a.overlap == N / 4);
    const bool b = (a.jobs != nullptr);
    if (a.flags & kOlsReal) {   // real signals: job lists only
        if (!b) return cudaErrorInvalidValue;
        if (!q) return launch_ols_fp32_w<N, 4, false, true, true>(a, sms, max_ctas, st, grid_out);
        switch (warps) {
        case 4: return launch_ols_fp32_w<N, 4, true, true, true>(a, sms, max_ctas, st, grid_out);
        case 8: return launch_ols_fp32_w<N, 8, true, true, true>(a, sms, max_ctas, st, grid_out);
        default: return cudaErrorInvalidValue;
        }
    }
    if (!q) {   // any other even overlap: runtime geometry, 4 warps per CTA
        return b ? launch_ols_fp32_w<N, 4, false, true>(a, sms, max_ctas, st, grid_out)
                 : launch_ols_fp32_w<N, 4, false, false>(a, sms, max_ctas, st, grid_out);
    }
    if constexpr (N == 1024) {
        // signals in host memory: consecutive blocks of a warp pass their overlap samples in
        // registers instead of reading them over the host link again
        if (b && (a.flags & kOlsNoBulk)) {
            switch (warps) {
            case 4: return launch_ols_fp32_w<N, 4, true, true, false, true>(a, sms, max_ctas, st, grid_out);
            case 8: return launch_ols_fp32_w<N, 8, true, true, false, true>(a, sms, max_ctas, st, grid_out);
            default: return cudaErrorInvalidValue;
            }
        }
    }
    switch (warps) {
    case 4: return b ? launch_ols_fp32_w<N, 4, true, true>(a, sms, max_ctas, st, grid_out)
                     : launch_ols_fp32_w<N, 4, true, false>(a, sms, max_ctas, st, grid_out);
    case 8: return b ? launch_ols_fp32_w<N, 8, true, true>(a, sms, max_ctas, st, grid_out)
                     : launch_ols_fp32_w<N, 8, true, false>(a, sms, max_ctas, st, grid_out);
    default: return cudaErrorInvalidValue;
    }
}

template <int N>
cudaError_t launch_export_hr(const float* V, int LV, int k1, float* out, cudaStream_t st)
{
    export_hr_kernel<N><<<1, 32, 0, st>>>(V, LV, k1, out);
    return cudaGetLastError();
}

#define VBW_INSTANTIATE_OLS(N)                                                                   \
    template cudaError_t launch_ols_fp32<N>(const OlsArgs&, int, int, int, cudaStream_t, int*);  \
    template cudaError_t launch_export_hr<N>(const float*, int, int, float*, cudaStream_t);

}  // namespace vbw

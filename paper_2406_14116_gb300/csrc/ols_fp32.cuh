// Fused FP32 overlap-save VBW kernel: gather -> N-point FFT -> H_R on the fly -> IFFT -> discard
// and store, one kernel, one pass over HBM (Sec. II steps 1-5 with eq. (FS_Hk_exp)/(FS_Hk_real)).
//
// Decomposition (four-step FFT, N = E * T):
//   thread t of a block holds x(T n1 + t), n1 = 0..E-1 (coalesced loads),
//   F1  E-point register DFT over n1                      -> A(ka, t)
//   F2  A(ka, t) *= W_N^{t ka}                            (shared-memory table; ka = 0 is 1)
//   F3  shared-memory transpose: thread t now owns ka = s T + t (s < E/T), every n2
//   F4  T-point register DFTs over n2                     -> X(ka + E k'), k' = 0..T-1
//   H   X(k) *= H_R(k) / N: the real gains come from a per-warp table g(kk), kk = min(k, N-k),
//       rebuilt from (k1, L_V, V) only when the block's band differs from the table's; they are
//       folded into the first stage of I1, so passband and stopband bins cost no extra work, and
//       they carry the 1/N of eq. (OLS_dn) (a power of two, so the scaling is exact)
//   I1  T-point inverse register DFTs over k'             -> B(ka, n2)
//   I3  transpose back: thread t owns n2 = t, every ka
//   I2  B(ka, t) *= conj(W_N^{t ka})
//   I4  E-point inverse register DFT over ka              -> z(T n1 + t)
// The linear phase exp(-j 2 pi k D / N), D = O/2, of eq. (FS_Hk_exp) is an exact circular shift of
// the IDFT output by D samples, so nothing multiplies it: the kept outputs w(O..N-1) of Sec. II
// step 4 are z(D..D+M-1), written to y(mM .. mM+M-1).
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
    // per-block transpose buffer; for T = 8 two blocks share a half-warp on the column side, so
    // their buffers are offset by 64 bytes mod 128
    static constexpr int BLK = E * ROW + ((T == 8) ? 8 : 0);
    // twiddle table row of thread t: W_N^{t ka}, ka = 0..E-1, padded to E + 2
    static constexpr int TWROW = E + 2;
    static constexpr int TW = T * TWROW;
    // per-block gain table g(kk), kk = 0..N/2; when several blocks share a warp their tables are
    // offset by T banks so the lane groups never collide
    static constexpr int GT_MIN = N / 2 + 1;
    static constexpr int GT = (B == 1) ? ((GT_MIN + 3) & ~3)
                                       : GT_MIN + ((T - GT_MIN % 32) % 32 + 32) % 32;
    // per warp: B transpose buffers, B gain tables, B mbarriers (8 bytes each)
    static constexpr size_t BAR_OFF = (sizeof(float2) * B * BLK + sizeof(float) * B * GT + 7) / 8 * 8;
    static constexpr size_t WARP_BYTES = (BAR_OFF + 8 * B + 15) / 16 * 16;
    static_assert(E * T == N && E % T == 0, "layout must satisfy N = E*T with T | E");
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
template <int N>
__device__ __forceinline__ void build_gains(float* gtab, int t, int k1, int LV, const float* V)
{
    constexpr int T = OlsGeom<N>::T;
    constexpr float inv_n = 1.0f / N;
    for (int kk = t; kk <= N / 2; kk += T) {
        const int r = kk - k1;
        gtab[kk] = (r < 0 ? 1.f : (r < LV ? V[r] : 0.f)) * inv_n;
    }
}

// L2 prefetch of a contiguous byte range with one bulk-copy instruction (16-byte aligned start,
// size a multiple of 16).
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ---- TMA bulk copy of a block's input span into shared memory, completing on an mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// generic-proxy accesses to shared memory made before this point are ordered before later
// async-proxy (TMA) writes
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_span(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%3], %2;\n\t"
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n\t}"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
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
constexpr int kStatusTmaTimeout = 1;

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

// One forward N-point four-step DFT on the register array x (see the top of this file):
// in:  x[n1] = u(T n1 + t)
// out: x[n1] = U(T n1 + t)      (with n1 = s + S k', this is X(ka + E k') for ka = s T + t)
// F1 E-point DFT, F2 twiddle, F3 transpose through buf, F4 S T-point DFTs.
template <int N, class Hook>
__device__ __forceinline__ void four_step_dft(float2 (&x)[OlsGeom<N>::E], float2* buf,
                                              const float4* twrow, int t, Hook&& after_transpose)
{
    using G = OlsGeom<N>;
    constexpr int E = G::E, T = G::T, S = G::S, ROW = G::ROW;
    fft_reg<E, false>(x);                                                    // F1
    const float4* tr = opaque(twrow);
    static_for<0, E / 2>([&](auto kh) {                                      // F2
        constexpr int ka = 2 * decltype(kh)::value;
        const float4 w = tr[kh];
        if constexpr (ka != 0) x[ka] = cmul(x[ka], make_float2(w.x, w.y));
        x[ka + 1] = cmul(x[ka + 1], make_float2(w.z, w.w));
    });
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
    after_transpose();                  // buf is free from here until the next F3
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
#ifndef VBW_TMA_STAGE
#define VBW_TMA_STAGE 1          // 1: a warp TMA-stages its next block's span into shared memory
#endif

#if VBW_MIN_WARPS_PER_SM > 0
#define VBW_OLS_BOUNDS(W) __launch_bounds__((W) * 32, (VBW_MIN_WARPS_PER_SM / (W)) > 0 ? VBW_MIN_WARPS_PER_SM / (W) : 1)
#else
#define VBW_OLS_BOUNDS(W) __launch_bounds__((W) * 32)
#endif

// The job and block of lane group bsub in warp-tile `tile`. The descriptors are re-read through
// opaque pointers (L1 hits) wherever they are needed, so none of their fields stays live in
// registers across the DFT passes.
template <int B>
__device__ __forceinline__ void job_of(const OlsArgs& a, int64_t tile, int bsub, OlsJob& job, int64_t& blk)
{
    if (a.jobs) {
        const int2 td = opaque(a.tiles)[tile];
        job = opaque(a.jobs)[td.x];
        blk = (int64_t)td.y + bsub;
    } else {
        job = a.job;
        blk = tile * B + bsub;
    }
}

// The fused kernel. Each block is two passes of the same four-step DFT (which keeps the loop body
// small enough for the instruction cache):
//   pass 0: X = DFT(x_m)                                   (Sec. II step 1)
//   pass 1: z = IDFT(H_R X / N) = swap(DFT(swap(H_R X / N)))  (steps 2-3), swap(a + jb) = b + ja,
// where both swaps are free (they only choose which register holds which component). Between the
// passes each register is scaled by its real gain g(kk) = H_R(k)/N, k = T n1 + t, kk = min(k, N-k).
// QOVL: the overlap is N/4 (D = N/8, M = 3N/4) as a compile-time constant; otherwise a.overlap.
template <int N, int WARPS, bool QOVL>
__global__ void VBW_OLS_BOUNDS(WARPS) ols_fp32_kernel(const OlsArgs a)
{
    using G = OlsGeom<N>;
    constexpr int E = G::E, T = G::T, B = G::B;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tw_s = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bsub = lane / T, t = lane % T;
    unsigned char* wbase = smem_raw + sizeof(float2) * G::TW + (size_t)warp * G::WARP_BYTES;
    float2* buf = reinterpret_cast<float2*>(wbase) + bsub * G::BLK;
    float* gtab = reinterpret_cast<float*>(wbase + sizeof(float2) * B * G::BLK) + bsub * G::GT;
    uint64_t* bar = reinterpret_cast<uint64_t*>(wbase + G::BAR_OFF) + bsub;
    const float4* twrow = reinterpret_cast<const float4*>(tw_s + t * G::TWROW);

    for (int i = threadIdx.x; i < G::TW / 2; i += blockDim.x)
        reinterpret_cast<float4*>(tw_s)[i] = reinterpret_cast<const float4*>(a.tw)[i];
    if (t == 0) mbar_init(bar, 1);
    __syncthreads();

    const int O = QOVL ? N / 4 : a.overlap;
    const int M = N - O, D = O >> 1;
    int table_k1 = -1;      // band the gain table currently holds
    bool staged = false;    // this lane group's current block was requested into buf by TMA
    uint32_t phase = 0;     // mbarrier phase that staged copy completes

    // each warp takes one contiguous range of tiles, so consecutive blocks of a stream stay in
    // one warp: the overlap samples are L2 hits and the gain table survives until the band changes
    const int64_t nwarps = (int64_t)gridDim.x * WARPS;
    const int64_t gw = (int64_t)blockIdx.x * WARPS + warp;
    const int64_t per = a.ntiles / nwarps, extra = a.ntiles % nwarps;
    const int64_t tile_begin = gw * per + (gw < extra ? gw : extra);
    const int64_t tile_end = tile_begin + per + (gw < extra ? 1 : 0);
    for (int64_t tile = tile_begin; tile < tile_end; ++tile) {
        float2 x[E];
        {
            // ---- which job and block this lane group works on, and its band
            OlsJob job;
            int64_t blk;
            job_of<B>(a, tile, bsub, job, blk);
            const int64_t nsamp = job.nsamp;
            const bool active = blk * M < nsamp;
            int k1 = job.band0;
            if (job.band) {
                if (active) k1 = job.band[blk];
            } else {
                for (int i = 0; i < a.nchg; ++i)
                    if (a.chg_block[i] <= blk) k1 = a.chg_band[i];
            }
            if (!active) k1 = table_k1;

            // ---- ask L2 for the samples the warp's next tile adds (the rest is this span)
            if (lane == 0 && tile + 1 < tile_end) {
                const int64_t e = (blk + B - 1) * (int64_t)M - O + N;
                int64_t e2 = e + (int64_t)B * M;
                if (e2 > nsamp) e2 = nsamp;
                const int64_t cnt = (e2 - e) & ~int64_t(1);
                if (e >= 0 && cnt > 0) prefetch_l2_bulk(job.in + e, (uint32_t)(cnt * sizeof(float2)));
            }

            // ---- gain table for this block's band (re-indexing only: eq. (FS_Hk_real))
            if (__any_sync(0xffffffffu, k1 != table_k1)) {
                __syncwarp();
                if (k1 >= 1) build_gains<N>(gtab, t, k1, a.LV, a.V);
                table_k1 = k1;
                __syncwarp();
            }

            // ---- gather x_m(n) = x(mM - O + n), n = T n1 + t (Sec. II segmentation): from
            //      the TMA staging copy when the previous block requested it, else from global
            const int64_t s0 = blk * M - O;
            const bool interior = active && s0 >= 0 && s0 + N <= nsamp;
            bool have = false, lost = false;
            if (staged) {
                have = mbar_wait_bounded(bar, phase, kWaitLimitCycles);
                if (!have) {
                    // flag it, then wait once more for the copy that may still be in flight
                    if (t == 0 && a.status) atomicOr(a.status, kStatusTmaTimeout);
                    have = mbar_wait_bounded(bar, phase, kWaitLimitCycles);
                    lost = !have;
                }
                if (have) phase ^= 1u;
                staged = false;
            }
            if (__any_sync(0xffffffffu, lost)) return;   // the warp stops; the host sees the flag
            if (__all_sync(0xffffffffu, have)) {
                static_for<0, E>([&](auto n1) { x[n1] = buf[decltype(n1)::value * T + t]; });
            } else if (__all_sync(0xffffffffu, interior)) {
                const float2* src = job.in + s0 + t;
                static_for<0, E>([&](auto n1) { x[n1] = ld_stream(src + decltype(n1)::value * T); });
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
        }

#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            four_step_dft<N>(x, buf, twrow, t, [&]() {
#if VBW_TMA_STAGE
                if (pass != 1 || tile + 1 >= tile_end) return;
                // the lane group's next block: TMA-staged into buf when its span is interior
                OlsJob nj;
                int64_t nb;
                job_of<B>(a, tile + 1, bsub, nj, nb);
                const int64_t ns0 = nb * M - O;
                if (ns0 >= 0 && ns0 + N <= nj.nsamp &&
                    (reinterpret_cast<uintptr_t>(nj.in + ns0) & 15) == 0) {
                    if (t == 0) {
                        fence_proxy_async_smem();
                        tma_load_span(buf, nj.in + ns0, (uint32_t)(N * sizeof(float2)), bar);
                    }
                    staged = true;
                }
#endif
            });
            if (pass == 0) {
                // swap(g X): H_R(k)/N of eq. (FS_Hk_real) for k = T n1 + t (Sec. II step 2)
                const float* lo = opaque(gtab + t);
                const float* hi = opaque(gtab + (N - t));
                static_for<0, E>([&](auto n1) {
                    constexpr int N1 = decltype(n1)::value;
                    constexpr int K = N1 * T;
                    const float gk = (N1 < E / 2) ? lo[K] : hi[-K];
                    x[n1] = make_float2(gk * x[n1].y, gk * x[n1].x);
                });
            }
        }

        // ---- discard and store (steps 4-5): z(n) = swap(x[n1]), n = T n1 + t, kept for
        //      D <= n < D + M (the exp(-j 2 pi k D / N) phase of eq. (FS_Hk_exp) as a shift)
        OlsJob job;
        int64_t blk;
        job_of<B>(a, tile, bsub, job, blk);
        const int64_t nsamp = job.nsamp;
        if (blk * M < nsamp) {
            const int64_t obase = blk * M - D;
            if constexpr (QOVL) {
                // kept rows n1 in [E/8, 7E/8): every lane stores, no per-sample test when the
                // block is complete
                float2* dst = job.out + obase + t;
                if (obase + D + M <= nsamp) {
                    static_for<E / 8, 7 * E / 8>([&](auto n1) {
                        st_stream(dst + decltype(n1)::value * T, make_float2(x[n1].y, x[n1].x));
                    });
                } else {
                    static_for<E / 8, 7 * E / 8>([&](auto n1) {
                        const int64_t oi = obase + decltype(n1)::value * T + t;
                        if (oi < nsamp) st_stream(job.out + oi, make_float2(x[n1].y, x[n1].x));
                    });
                }
            } else {
                static_for<0, E>([&](auto n1) {
                    const int n = decltype(n1)::value * T + t;
                    if (n >= D && n < D + M) {
                        const int64_t oi = obase + n;
                        if (oi < nsamp) st_stream(job.out + oi, make_float2(x[n1].y, x[n1].x));
                    }
                });
            }
            // the lane group of the job's last block hands the stream's last O input samples on
            if ((blk + 1) * M >= nsamp && job.tail_out) {
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
template <int N, int WARPS, bool QOVL>
cudaError_t launch_ols_fp32_w(const OlsArgs& a, int sms, cudaStream_t st, int* grid_out)
{
    const size_t smem = ols_smem_bytes<N>(WARPS);
    auto kern = ols_fp32_kernel<N, WARPS, QOVL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t ctas_needed = (a.ntiles + WARPS - 1) / WARPS;
    const int64_t cap = (int64_t)per_sm * sms;
    const int grid = (int)(ctas_needed < cap ? ctas_needed : cap);
    if (grid_out) *grid_out = grid;
    if (grid <= 0) return cudaSuccess;
    kern<<<grid, WARPS * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_ols_fp32(const OlsArgs& a, int warps, int sms, cudaStream_t st, int* grid_out)
{
    const bool q = (a.overlap == N / 4);
    switch (warps) {
    case 4: return q ? launch_ols_fp32_w<N, 4, true>(a, sms, st, grid_out)
                     : launch_ols_fp32_w<N, 4, false>(a, sms, st, grid_out);
    case 8: return q ? launch_ols_fp32_w<N, 8, true>(a, sms, st, grid_out)
                     : launch_ols_fp32_w<N, 8, false>(a, sms, st, grid_out);
    default: return cudaErrorInvalidValue;
    }
}

template <int N>
cudaError_t launch_export_hr(const float* V, int LV, int k1, float* out, cudaStream_t st)
{
    export_hr_kernel<N><<<1, 32, 0, st>>>(V, LV, k1, out);
    return cudaGetLastError();
}

#define VBW_INSTANTIATE_OLS(N)                                                                 \
    template cudaError_t launch_ols_fp32<N>(const OlsArgs&, int, int, cudaStream_t, int*);     \
    template cudaError_t launch_export_hr<N>(const float*, int, int, float*, cudaStream_t);

}  // namespace vbw

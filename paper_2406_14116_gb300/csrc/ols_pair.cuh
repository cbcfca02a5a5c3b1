// N = 2048 on a warp pair: one radix-2 split of the 2048-point DFT into two 1024-point halves,
// each a four-step DFT held by one warp (32 samples per thread, like N = 1024), instead of one
// warp holding 64 samples per thread.
//
// Forward, decimation in frequency (H = N/2, W = exp(-j 2 pi / N), u = the block's N inputs):
//   warp 0: a(n) = u(n) + u(n + H)                 -> X(2r)     = DFT_H(a)(r)
//   warp 1: b(n) = (u(n) - u(n + H)) W^n           -> X(2r + 1) = DFT_H(b)(r)
// Gains H_R(k)/N of eq. (FS_Hk_real) for k = 2r + h, then the inverse, decimation in time:
//   warp h: Q_h = sum_r Y(2r + h) W_H^{-nr}        (the swap identity of the four-step pass)
//   z(n)     = Q_0(n) + W^{-n} Q_1(n),   z(n + H) = Q_0(n) - W^{-n} Q_1(n),   n < H
// which is the IDFT of eq. (OLS_dn) (the 1/N sits in the gains). With overlap N/4 the kept
// outputs z(D .. D + M - 1), D = 256, M = 1536, are n in [256, 1024) (warp 0) and n + H with
// n in [0, 768) (warp 1): 24 of each thread's 32 registers on both warps. The halves meet once,
// through shared memory, after the inverse; the block's register n1 of thread t is index
// n = 32 n1 + t on both warps, so the exchange is position for position.
#pragma once

#include "ols_fp32.cuh"

namespace vbw {

struct PairGeom {
    static constexpr int N = 2048, H = 1024;
    using G = OlsGeom<1024>;                   // E = T = 32, ROW = 34
    static constexpr int E = G::E, T = G::T;
    static constexpr int O = N / 4, M = N - O, D = O / 2;
    // CTA tables (float2 entries): the four-step rows of the 1024-point halves, W_1024^{t ka},
    // then the split twiddles W_2048^{32 n1 + t} as row t; both T x (E + 2)
    static constexpr int TW = G::TW;
    static constexpr size_t TABLE_BYTES = 2 * sizeof(float2) * TW;
    // per pair: the two warps' transpose buffers (also the exchange area), then the gains
    // de-interleaved by parity: ge[j] = g(2j), j = 0..512, and go[j] = g(2j + 1), j = 0..511
    static constexpr int GE = 516, GO = 512;
    static constexpr size_t GAIN_OFF = 2 * sizeof(float2) * G::BLK;
    static constexpr size_t PAIR_BYTES = GAIN_OFF + sizeof(float) * (GE + GO);
    static_assert(E == 32 && T == 32, "the pair layout assumes the 32 x 32 four-step");
    static_assert(PAIR_BYTES % 16 == 0, "pair areas stay 16-byte aligned");
};

// Offset (float2 entries) of the pair tables inside an N = 2048 plan's twiddle array: after the
// single-warp table (T = 32 rows of E + 2 = 66 entries).
constexpr int kPairTwOffset = 32 * 66;

__host__ __device__ inline size_t ols_pair_smem_bytes(int warps)
{
    return PairGeom::TABLE_BYTES + (size_t)(warps / 2) * PairGeom::PAIR_BYTES;
}

// Named barrier of the pair (ids 1.. ; id 0 is __syncthreads).
__device__ __forceinline__ void pair_sync(int pair)
{
    asm volatile("bar.sync %0, 64;" ::"r"(pair + 1) : "memory");
}

template <int WARPS, bool BATCH>
__global__ void __launch_bounds__(WARPS * 32, 16 / WARPS) ols_pair_kernel(const OlsArgs a)
{
    using P = PairGeom;
    constexpr int E = P::E, H = P::H, M = P::M, O = P::O, D = P::D;
    static_assert(WARPS % 2 == 0 && WARPS / 2 <= 15, "warp pairs need named barriers 1..15");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
    const int pair = warp >> 1, h = warp & 1;
    float2* tw_s = reinterpret_cast<float2*>(smem_raw);
    const float2* w2_s = tw_s + P::TW;
    unsigned char* pbase = smem_raw + P::TABLE_BYTES + (size_t)pair * P::PAIR_BYTES;
    float2* buf_own = reinterpret_cast<float2*>(pbase) + h * P::G::BLK;
    const float2* buf_peer = reinterpret_cast<const float2*>(pbase) + (h ^ 1) * P::G::BLK;
    float* ge = reinterpret_cast<float*>(pbase + P::GAIN_OFF);
    float* go = ge + P::GE;

    {
        const float4* src = reinterpret_cast<const float4*>(a.tw + kPairTwOffset);
        float4* dst = reinterpret_cast<float4*>(tw_s);
        for (int i = threadIdx.x; i < P::TW; i += blockDim.x) dst[i] = src[i];   // both tables
    }
    __syncthreads();

    const float4* twrow = reinterpret_cast<const float4*>(tw_s + t * P::G::TWROW);
    const float4* w2row = reinterpret_cast<const float4*>(w2_s + t * P::G::TWROW);
    const bool bulk = (a.flags & kOlsNoBulk) == 0;
    int table_key = -1;
    int64_t tb, te;
    warp_range(a.ntiles, (int64_t)gridDim.x * (WARPS / 2), (int64_t)blockIdx.x * (WARPS / 2) + pair, tb, te);
    for (int64_t tile = tb; tile < te; ++tile) {
        float2 x[E];
        {
            OlsJob job;
            int64_t blk;
            int k1;
            if constexpr (BATCH) {
                const JobListSource src{a.jobs, a.tiles};
                src.template get<1>(tile, 0, job, blk);
                k1 = src.band(job, blk, blk * M < job.nsamp);
            } else {
                const SingleJobSource src{a};
                src.template get<1>(tile, 0, job, blk);
                k1 = src.band(job, blk, blk * M < job.nsamp);
            }
            const int64_t nsamp = job.nsamp;
            const bool active = blk * M < nsamp;

            // L2 prefetch of the samples the next block adds: [blk M + M, blk M + 2M)
            if (h == 0 && t == 0 && tile + 1 < te && bulk && active) {
                int64_t e = blk * M + M;
                int64_t e2 = e + M;
                if (e2 > nsamp) e2 = nsamp;
                if ((reinterpret_cast<uintptr_t>(job.in + e) & 15) != 0) ++e;
                const int64_t cnt = (e2 - e) & ~int64_t(1);
                if (cnt > 0 && (reinterpret_cast<uintptr_t>(job.in + e) & 15) == 0)
                    prefetch_l2_bulk(job.in + e, (uint32_t)(cnt * sizeof(float2)));
            }

            // gains of this block's band (eq. (FS_Hk_real)), de-interleaved by parity; the
            // decision is the same on both warps of the pair
            if (active && k1 != table_key) {
                constexpr float inv_n = 1.0f / (2 * H);
                for (int kk = h * 32 + t; kk <= H; kk += 64) {
                    const float g = hr_gain(kk, k1, a.LV, a.V) * inv_n;
                    if (kk & 1) go[kk >> 1] = g;
                    else ge[kk >> 1] = g;
                }
                table_key = k1;
            }

            // gather u(n), u(n + H), n = 32 n1 + t (Sec. II segmentation, O samples of history),
            // and form a(n) (warp 0) or b(n) (warp 1), eight rows at a time
            const int64_t s0 = blk * M - O;
            const bool interior = active && s0 >= 0 && s0 + 2 * H <= nsamp;
            const float4* wr = opaque(w2row);
            auto fetch = [&](int64_t si) {
                float2 v = make_float2(0.f, 0.f);
                if (active) {
                    if (si >= 0) {
                        if (si < nsamp) v = ld_stream(job.in + si);
                    } else if (job.tail_in) {
                        v = job.tail_in[O + si];
                    }
                }
                return v;
            };
            static_for<0, E / 8>([&](auto c) {
                constexpr int C = decltype(c)::value;
                float2 u1[8];
                if (interior) {
                    const float2* sp = job.in + s0 + t + 32 * 8 * C;
                    static_for<0, 8>([&](auto i) {
                        constexpr int I = decltype(i)::value;
                        x[8 * C + I] = ld_stream(sp + 32 * I);
                        u1[I] = ld_stream(sp + 32 * I + H);
                    });
                } else {
                    static_for<0, 8>([&](auto i) {
                        constexpr int I = decltype(i)::value;
                        x[8 * C + I] = fetch(s0 + 32 * (8 * C + I) + t);
                        u1[I] = fetch(s0 + 32 * (8 * C + I) + t + H);
                    });
                }
                if (h == 0) {
                    static_for<0, 8>([&](auto i) { x[8 * C + decltype(i)::value] = cadd(x[8 * C + decltype(i)::value], u1[decltype(i)::value]); });
                } else {
                    static_for<0, 4>([&](auto q) {
                        constexpr int Q = 4 * C + decltype(q)::value;
                        const float4 w = wr[Q];
                        const float2 b0 = csub(x[2 * Q], u1[2 * decltype(q)::value]);
                        const float2 b1 = csub(x[2 * Q + 1], u1[2 * decltype(q)::value + 1]);
                        x[2 * Q] = cmul(b0, make_float2(w.x, w.y));   // W^t on row 0 too
                        x[2 * Q + 1] = cmul(b1, make_float2(w.z, w.w));
                    });
                }
                asm volatile("" ::: "memory");   // keep the eight-row groups apart (registers)
            });
        }
        // past this point the partner has read this warp's buffer (previous exchange) and the
        // gains of this block are complete
        pair_sync(pair);

        // forward half-DFT, gains, inverse half-DFT (swap identity)
        four_step_dft<1024>(x, buf_own, twrow, t, [] {});
        {
            const float* gh = h == 0 ? ge : go;
            const float* lo = opaque(gh + t);
            const float* hi = opaque(gh + (h == 0 ? H : H - 1) - t);
            static_for<0, E>([&](auto n1) {
                constexpr int NN = decltype(n1)::value;
                // bin k = 2 r + h, r = 32 n1 + t: below N/2 for r < 512, else its mirror N - k
                const float g = NN < E / 2 ? lo[32 * NN] : hi[-32 * NN];
                x[NN] = make_float2(g * x[NN].y, g * x[NN].x);
            });
        }
        four_step_dft<1024>(x, buf_own, twrow, t, [] {});
        // x[n1] = swap(Q_h(32 n1 + t))

        // exchange what the partner keeps: warp 0 sends Q_0 of rows 0..23, warp 1 Q_1 of rows
        // 8..31 (stored as rows 0..23)
        if (h == 0) {
            static_for<0, 24>([&](auto j) { buf_own[decltype(j)::value * 32 + t] = x[decltype(j)::value]; });
        } else {
            static_for<0, 24>([&](auto j) { buf_own[decltype(j)::value * 32 + t] = x[8 + decltype(j)::value]; });
        }
        pair_sync(pair);

        OlsJob job;
        int64_t blk;
        if constexpr (BATCH) JobListSource{a.jobs, a.tiles}.template get<1>(tile, 0, job, blk);
        else SingleJobSource{a}.template get<1>(tile, 0, job, blk);
        const int64_t nsamp = job.nsamp;
        if (blk * M < nsamp) {
            const float4* wr = opaque(w2row);
            const bool full = blk * M + M <= nsamp;
            // warp 0, rows n1 = 8 + j: z(n) = Q_0(n) + W^{-n} Q_1(n) -> y(blk M + n - D)
            // warp 1, rows n1 = j:     z(n + H) = Q_0(n) - W^{-n} Q_1(n) -> y(blk M + n + H - D)
            // (n = 32 n1 + t; either way the output index is blk M + 32 j + t (+ 768 on warp 1))
            float2* dst = job.out + blk * M + (h == 0 ? 0 : H - D) + t;
            const int64_t lim = nsamp - blk * M - (h == 0 ? 0 : H - D) - t;   // valid: 32 j < lim
            if (h == 0) {
                static_for<0, 12>([&](auto q) {
                    constexpr int Q = decltype(q)::value;
                    const float4 w = wr[4 + Q];
                    static_for<0, 2>([&](auto i) {
                        constexpr int J = 2 * Q + decltype(i)::value;
                        const float2 wv = decltype(i)::value == 0 ? make_float2(w.x, w.y) : make_float2(w.z, w.w);
                        const float2 own = x[8 + J], peer = buf_peer[J * 32 + t];
                        const float2 c = cmul_conj(make_float2(peer.y, peer.x), wv);
                        const float2 z = cadd(make_float2(own.y, own.x), c);
                        if (full || 32 * J < lim) st_stream(dst + 32 * J, z);
                    });
                });
            } else {
                static_for<0, 12>([&](auto q) {
                    constexpr int Q = decltype(q)::value;
                    const float4 w = wr[Q];
                    static_for<0, 2>([&](auto i) {
                        constexpr int J = 2 * Q + decltype(i)::value;
                        const float2 wv = decltype(i)::value == 0 ? make_float2(w.x, w.y) : make_float2(w.z, w.w);
                        const float2 own = x[J], peer = buf_peer[J * 32 + t];
                        const float2 c = cmul_conj(make_float2(own.y, own.x), wv);
                        const float2 z = csub(make_float2(peer.y, peer.x), c);
                        if (full || 32 * J < lim) st_stream(dst + 32 * J, z);
                    });
                });
            }
            // the last block of a job hands the stream's last O input samples on
            if (h == 0 && (blk + 1) * M >= nsamp && job.tail_out) {
                for (int i = t; i < O; i += 32) {
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

// Writes the H_R(k) the pair kernel applies for band k1 (test hook): the same de-interleaved
// table build and the same lo/hi indexing, on one pair; the table's 1/N is undone exactly.
__global__ void export_hr_pair_kernel(const float* V, int LV, int k1, float* out)
{
    using P = PairGeom;
    constexpr int H = P::H;
    __shared__ float ge[P::GE], go[P::GO];
    const int h = threadIdx.x >> 5, t = threadIdx.x & 31;
    for (int kk = h * 32 + t; kk <= H; kk += 64) {
        const float g = hr_gain(kk, k1, LV, V) * (1.0f / (2 * H));
        if (kk & 1) go[kk >> 1] = g;
        else ge[kk >> 1] = g;
    }
    __syncthreads();
    const float* gh = h == 0 ? ge : go;
    const float* lo = gh + t;
    const float* hi = gh + (h == 0 ? H : H - 1) - t;
    static_for<0, P::E>([&](auto n1) {
        constexpr int NN = decltype(n1)::value;
        const float g = NN < P::E / 2 ? lo[32 * NN] : hi[-32 * NN];
        out[2 * (32 * NN + t) + h] = g * (float)(2 * H);
    });
}

template <int WARPS, bool BATCH>
cudaError_t launch_ols_pair_w(const OlsArgs& a, int sms, int max_ctas, cudaStream_t st, int* grid_out)
{
    // tiles are single blocks; a CTA takes WARPS/2 of them at a time
    return launch_persistent(ols_pair_kernel<WARPS, BATCH>, WARPS, ols_pair_smem_bytes(WARPS), a.ntiles * 2, sms,
                             max_ctas, st, grid_out, &a);
}

}  // namespace vbw

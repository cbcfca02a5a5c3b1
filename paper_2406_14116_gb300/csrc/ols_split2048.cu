// Fused FP32 overlap-save kernel for N = 2048 with overlap N/4: one radix-2 split into two
// 1024-point transforms that reuse the N = 1024 four-step of ols_fp32.cuh, with the half that is
// not being transformed parked in tensor memory.
//
// Decimation in frequency by 2 of the block DFT (Sec. II step 1), n = 32 n1 + t < 1024:
//   a(n) = x(n) + x(n + 1024)                X(2k)     = DFT_1024(a)(k)
//   b(n) = (x(n) - x(n + 1024)) W_2048^n      X(2k + 1) = DFT_1024(b)(k)
// Thread t holds x(32 n1 + t) and x(1024 + 32 n1 + t), n1 < 32: for both halves that is the
// N = 1024 layout (E = T = 32, thread t holding u(32 n1 + t) in register n1).
// W_2048^n = W_64^{n1} W_2048^t. The first factor is a compile-time constant. The second is the
// same for all of a thread's values, so it passes through the register DFT over n1 and joins that
// thread's four-step twiddle: W_1024^{t ka} W_2048^t = W_2048^{t (2 ka + 1)}.
// Each half then takes its gains H_R(K)/N (eq. (FS_Hk_real)) at K = 2k or 2k + 1 and the inverse
// IDFT(Y) = swap(DFT(swap(Y))). With e and o the two halves' inverse transforms (no 1/N: the gains
// carry it),
//   y(n) = e(n) + W_2048^{-n} o(n),   y(n + 1024) = e(n) - W_2048^{-n} o(n),
// and swap(W_2048^{-n} o) = W_2048^{n} swap(o). Of W_2048^n = W_64^{n1} W_2048^{ka} (the thread
// that owns output n after the transpose holds ka = n mod 32), the second factor joins the odd
// inverse pass's four-step twiddle, W_1024^{t ka} W_2048^{ka} = W_2048^{ka (2 t + 1)}, and the
// first is applied to the output registers. The kept outputs z(D .. D + M - 1), D = O/2, are
// rows n1 >= 8 of y(n) and rows n1 < 24 of y(n + 1024).
//
// Tensor memory: b waits there while the even half runs, then the even half's output waits there
// while the odd half runs. Each warp owns 2 x 64 columns of its 32 lanes (lanes 32 (w mod 4) ..,
// columns 128 (w div 4) ..): the default 12-warp CTA holds 384 of the SM's 512 columns, a 16-warp
// CTA all of them. The register budget per thread then holds 32 complex values instead of 64.
#include "ols_fp32.cuh"
#include "tc_common.cuh"

namespace vbw {
namespace {

struct Split {
    static constexpr int N = 2048, O = 512, M = 1536, D = 256;
    static constexpr int TWROW = OlsGeom<1024>::TWROW;           // 34: row of one F2 table
    static constexpr int TWTAB = 32 * TWROW;                      // one F2 table (float2)
    static constexpr int TW_ENTRIES = 3 * TWTAB;                  // W_1024^{t ka}, odd forward, odd inverse
    static constexpr int GO = 516;                                // odd-bin gains start (floats)
    static constexpr int GT = GO + 512;                           // gains per warp (floats)
    static constexpr size_t BUF_BYTES = sizeof(float2) * OlsGeom<1024>::BLK;
    static constexpr size_t CARRY_OFF = BUF_BYTES + sizeof(float) * GT;   // per-warp SplitCarry
    static constexpr size_t WARP_BYTES = CARRY_OFF + 16;
    static constexpr size_t TW_BYTES = sizeof(float2) * TW_ENTRIES;
    static_assert(GO >= 513 && GO % 4 == 0 && WARP_BYTES % 16 == 0, "gain tables must stay 16-byte aligned");
};

// Signals in host memory (CARRY): the last O = 512 samples of a block's span, rows 16..31 of its
// second half, are the first 512 of the next block's span, rows 0..15 of its first half, in the
// same lanes. They wait in 32 more tensor-memory columns per warp, so consecutive blocks of a warp
// read each input sample from the host link once. The block they open, in shared memory per warp:
struct SplitCarry {
    const float2* in;     // the signal they belong to; nullptr = none
    int64_t blk;          // the block whose span starts with them
};

// Tensor-memory columns per warp: b and the parked even half (2 x 64), plus the carry.
constexpr int split_warp_cols(bool carry) { return carry ? 160 : 128; }

// Tensor-memory columns of one CTA: the per-warp columns times the warps of each lane quarter, as
// a power of two.
constexpr uint32_t split_cols(int warps, bool carry = false)
{
    const int need = split_warp_cols(carry) * ((warps + 3) / 4);
    uint32_t c = 32;
    while ((int)c < need) c <<= 1;
    return c;
}

// v * exp(-j 2 pi J / L) with compile-time J, L.
template <int J, int L>
__device__ __forceinline__ float2 rot_const(float2 v)
{
    constexpr int j = ((J % L) + L) % L;
    if constexpr (j == 0) {
        return v;
    } else if constexpr (4 * j == L) {            // -j
        return make_float2(v.y, -v.x);
    } else if constexpr (2 * j == L) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (4 * j == 3 * L) {        // +j
        return make_float2(-v.y, v.x);
    } else {
        constexpr CosSin cs = cos_sin_2pi(j, L);
        constexpr float c = static_cast<float>(cs.c);
        constexpr float s = static_cast<float>(-cs.s);
        return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
    }
}

// ---- tensor-memory stores and loads of this thread's lane (32x32b shape, warp-wide)
__device__ __forceinline__ void tm_st16(uint32_t ta, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
        ::"r"(ta), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
          "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

// 16 words whose load is still in flight: tm_wait16 must come before they are used
__device__ __forceinline__ void tm_ld16(uint32_t ta, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta)
        : "memory");
}

// Waits for this thread's tensor-memory loads; r is tied to the wait, so its uses follow it.
__device__ __forceinline__ void tm_wait16(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// x[B .. B + 8) -> 16 columns at ta
template <int B>
__device__ __forceinline__ void park8(uint32_t ta, const float2 (&x)[32])
{
    uint32_t r[16];
    static_for<0, 8>([&](auto i) {
        r[2 * i] = __float_as_uint(x[B + i].x);
        r[2 * i + 1] = __float_as_uint(x[B + i].y);
    });
    tm_st16(ta, r);
}

// 64 columns at ta -> 32 complex values, four loads in flight before one wait
__device__ __forceinline__ void unpark32(uint32_t ta, uint32_t (&r)[4][16])
{
    static_for<0, 4>([&](auto c) { tm_ld16(ta + 16 * decltype(c)::value, r[c]); });
    static_for<0, 4>([&](auto c) { tm_wait16(r[c]); });
}

// Gains of the split layout, g(K) = H_R(K)/N for the DFT bin K, folded to kk = min(K, N - K):
// gtab[j] = g(2j) for j = 0..512, gtab[GO + j] = g(2j + 1) for j = 0..511.
__device__ __forceinline__ void build_split_gains(float* gtab, int t, int k1, int LV, const float* V)
{
    constexpr float inv_n = 1.0f / Split::N;
    for (int j = t; j <= 512; j += 32) gtab[j] = hr_gain(2 * j, k1, LV, V) * inv_n;
    for (int j = t; j < 512; j += 32) gtab[Split::GO + j] = hr_gain(2 * j + 1, k1, LV, V) * inv_n;
}

// Gains of register n1 of thread t in half h, i.e. of bin K = 2 (32 n1 + t) + h: kk = K below
// N/2 (n1 < 16), else N - K. Shared-memory addresses of row n1 = 0 on each side.
struct SplitGainRow {
    uint32_t lo, hi;
};

__device__ __forceinline__ SplitGainRow split_gain_row(const float* gtab, int h, int t)
{
    const uint32_t gb = smem_u32(gtab + h * Split::GO);
    return SplitGainRow{gb + 4 * t, gb + 4 * ((1024 - h) - t)};
}

template <int N1>
__device__ __forceinline__ float split_gain(const SplitGainRow& g)
{
    return (N1 < 16) ? lds_f32(g.lo + 4 * 32 * N1) : lds_f32(g.hi - 4 * 32 * N1);
}

// One block of N = 2048 per warp. LEAN: a register budget of 128 (16 warps per SM), so the merge
// reads the parked half back 8 rows at a time instead of all at once.
template <bool LEAN, bool CARRY, class Src>
__device__ __forceinline__ void split_tile(const Src& src, int64_t tile, bool has_next, const float2* tw_s,
                                           const float* V, int LV, unsigned char* wbase, int t,
                                           WarpState& ws, bool bulk, uint32_t tP, uint32_t tQ, uint32_t tC)
{
    constexpr int N = Split::N, O = Split::O, M = Split::M, D = Split::D;
    float2* buf = reinterpret_cast<float2*>(wbase);
    float* gtab = reinterpret_cast<float*>(wbase + Split::BUF_BYTES);

    float2 x[32];
    float2* kout;
    int64_t knsamp, kblk;
    {
        OlsJob job;
        int64_t blk;
        if constexpr (std::is_same<Src, JobListSource>::value) {
            const int2 td = ws.ntd_ok ? ws.ntd : opaque(src.tiles)[tile];
            job = opaque(src.jobs)[td.x];
            blk = (int64_t)td.y;
            ws.ntd_ok = has_next;
            if (has_next) ws.ntd = opaque(src.tiles)[tile + 1];
        } else {
            src.template get<1>(tile, 0, job, blk);
        }
        const int64_t nsamp = job.nsamp;
        kout = job.out;
        knsamp = nsamp;
        kblk = blk;
        const bool active = blk * M < nsamp;
        const int k1 = src.band(job, blk, active);
        const int key = active ? k1 : ws.table_key;

        // ---- gather x_m(n) = x(mM - O + n) (Sec. II segmentation), then the split: a(n) stays
        //      in registers, b(n) W_2048^{-t} goes to tensor memory, 8 rows at a time
        const int64_t s0 = blk * M - O;
        const bool fast = __all_sync(0xffffffffu, active && s0 >= 0 && s0 + N <= nsamp);
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
        SplitCarry* cm = reinterpret_cast<SplitCarry*>(wbase + Split::CARRY_OFF);
        bool carried = false;
        if constexpr (CARRY) carried = fast && cm->in == job.in && cm->blk == blk;   // same for all lanes
        if (carried) {
            // rows 0..15: the previous block's rows 16..31 of its second half, from tensor memory
            uint32_t r[2][16];
            tm_ld16(tC, r[0]);
            tm_ld16(tC + 16, r[1]);
            tm_wait16(r[0]);
            tm_wait16(r[1]);
            static_for<0, 16>([&](auto i) {
                constexpr int I = decltype(i)::value;
                x[I] = make_float2(__uint_as_float(r[I / 8][2 * (I % 8)]), __uint_as_float(r[I / 8][2 * (I % 8) + 1]));
            });
            const float2* sp = job.in + s0 + t;
            static_for<16, 32>([&](auto n1) { x[n1] = ld_stream(sp + 32 * decltype(n1)::value); });
        } else if (fast) {
            const float2* sp = job.in + s0 + t;
            static_for<0, 32>([&](auto n1) { x[n1] = ld_stream(sp + 32 * decltype(n1)::value); });
        } else {
            static_for<0, 32>([&](auto n1) { x[n1] = fetch(s0 + 32 * decltype(n1)::value + t); });
        }
        static_for<0, 4>([&](auto c) {
            constexpr int C = decltype(c)::value;
            float2 h[8];
            if (fast) {
                const float2* sp = job.in + s0 + 1024 + t;
                static_for<0, 8>([&](auto i) { h[i] = ld_stream(sp + 32 * (8 * C + decltype(i)::value)); });
            } else {
                static_for<0, 8>([&](auto i) { h[i] = fetch(s0 + 1024 + 32 * (8 * C + decltype(i)::value) + t); });
            }
            if constexpr (CARRY && C >= 2) {
                // rows 16..31 of the second half open the next block's span
                uint32_t q[16];
                static_for<0, 8>([&](auto i) {
                    q[2 * i] = __float_as_uint(h[i].x);
                    q[2 * i + 1] = __float_as_uint(h[i].y);
                });
                tm_st16(tC + 16 * (C - 2), q);
            }
            uint32_t r[16];
            static_for<0, 8>([&](auto i) {
                constexpr int n1 = 8 * C + decltype(i)::value;
                const float2 u = x[n1], v = h[i];
                x[n1] = make_float2(u.x + v.x, u.y + v.y);
                const float2 d = rot_const<n1, 64>(make_float2(u.x - v.x, u.y - v.y));
                r[2 * i] = __float_as_uint(d.x);
                r[2 * i + 1] = __float_as_uint(d.y);
            });
            tm_st16(tP + 16 * C, r);
        });

        if constexpr (CARRY) {
            __syncwarp();
            if (t == 0) {
                cm->in = active ? job.in : nullptr;
                cm->blk = blk + 1;
            }
            __syncwarp();
        }

        // ---- L2 prefetch of the samples the warp's next tile adds (16-byte aligned bulk copy)
        if (t == 0 && has_next && bulk) {
            int64_t e = blk * (int64_t)M - O + N;
            int64_t e2 = e + M;
            if (e2 > nsamp) e2 = nsamp;
            if (e >= 0 && (reinterpret_cast<uintptr_t>(job.in + e) & 15) != 0) ++e;
            const int64_t cnt = (e2 - e) & ~int64_t(1);
            if (e >= 0 && cnt > 0 && (reinterpret_cast<uintptr_t>(job.in + e) & 15) == 0)
                prefetch_l2_bulk(job.in + e, (uint32_t)(cnt * sizeof(float2)));
        }

        // ---- gain tables for this block's band (re-indexing only: eq. (FS_Hk_real))
        if (__any_sync(0xffffffffu, key != ws.table_key)) {
            __syncwarp();
            if (active) build_split_gains(gtab, t, k1, LV, V);
            ws.table_key = key;
            __syncwarp();
        }
    }

    // ---- eight 32-point register DFTs (one code body, for the instruction cache). Steps 0-1
    //      and 2-3 are the even half's forward and swapped inverse four-steps, steps 4-5 and 6-7
    //      the odd half's. After an even step: F2 and F3 with the step's table (W_1024^{t ka}; the
    //      odd half's forward and inverse tables); after steps 1 and 5: gains and swap; after
    //      step 3: the even output goes to tensor memory and b comes back.
#pragma unroll 1
    for (int step = 0; step < 8; ++step) {
        fft_reg<32, false>(x);
        if ((step & 1) == 0) {
            const int tab = step < 4 ? 0 : (step >> 1) - 1;
            // the odd forward table's ka = 0 entries are W_2048^t, not 1 (the others' are exactly 1)
            four_step_f2f3<1024, true>(x, buf, reinterpret_cast<const float4*>(tw_s + tab * Split::TWTAB + t * Split::TWROW), t);
        } else if (step != 7) {
            if (step == 3) {
                tm_wait_st();   // b's stores (long done) before it is read back
                park8<0>(tQ, x);
                park8<8>(tQ + 16, x);
                park8<16>(tQ + 32, x);
                park8<24>(tQ + 48, x);
                if constexpr (LEAN) {
                    static_for<0, 4>([&](auto c) {
                        constexpr int C = decltype(c)::value;
                        uint32_t r[16];
                        tm_ld16(tP + 16 * C, r);
                        tm_wait16(r);
                        static_for<0, 8>([&](auto i) {
                            x[8 * C + i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
                        });
                    });
                } else {
                    uint32_t r[4][16];
                    unpark32(tP, r);
                    static_for<0, 32>([&](auto i) {
                        constexpr int I = decltype(i)::value;
                        x[I] = make_float2(__uint_as_float(r[I / 8][2 * (I % 8)]), __uint_as_float(r[I / 8][2 * (I % 8) + 1]));
                    });
                }
            } else {
                const SplitGainRow g = split_gain_row(gtab, step >> 2, t);
                static_for<0, 32>([&](auto n1) {
                    const float gk = split_gain<decltype(n1)::value>(g);
                    x[n1] = make_float2(gk * x[n1].y, gk * x[n1].x);
                });
            }
        }
    }

    // ---- merge, discard and store (Sec. II steps 4-5): x holds W_2048^{t} swap(o) per register,
    //      the even half's swap(e) is in tensor memory
    const int64_t blk = kblk;
    const int64_t nsamp = knsamp;
    const bool act = blk * M < nsamp;
    const int64_t obase = blk * M - D;
    const bool full = blk * M + M <= nsamp;
    tm_wait_st();       // the even half's stores (long done) before it is read back
    float2* dst = kout + obase + t;
    auto merge_row = [&](auto i, const uint32_t* rr) {
        constexpr int n1 = decltype(i)::value;
        const float2 e = make_float2(__uint_as_float(rr[2 * (n1 % 8)]), __uint_as_float(rr[2 * (n1 % 8) + 1]));
        const float2 o = rot_const<n1, 64>(x[n1]);
        if constexpr (n1 >= D / 32) {
            if (full || obase + 32 * n1 + t < nsamp) st_stream(dst + 32 * n1, make_float2(e.y + o.y, e.x + o.x));
        }
        if constexpr (n1 < (D + M - 1024) / 32) {
            if (full || obase + 1024 + 32 * n1 + t < nsamp)
                st_stream(dst + 1024 + 32 * n1, make_float2(e.y - o.y, e.x - o.x));
        }
    };
    if constexpr (LEAN) {
        static_for<0, 4>([&](auto c) {
            constexpr int C = decltype(c)::value;
            uint32_t r[16];
            tm_ld16(tQ + 16 * C, r);
            tm_wait16(r);
            if (act) static_for<8 * C, 8 * C + 8>([&](auto i) { merge_row(i, r); });
        });
    } else {
        uint32_t r[4][16];
        unpark32(tQ, r);
        if (act) static_for<0, 32>([&](auto i) { merge_row(i, r[decltype(i)::value / 8]); });
    }
    // the warp of the job's last block hands the stream's last O input samples on
    if (act && (blk + 1) * M >= nsamp) {
        OlsJob job;
        int64_t bj;
        src.template get<1>(tile, 0, job, bj);
        if (job.tail_out) {
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

// One CTA per SM (its shared memory and tensor memory take the SM); warps walk contiguous tile
// ranges as in the other fused kernels.
template <int WARPS, bool BATCH, bool CARRY = false>
__global__ void __launch_bounds__(WARPS * 32, 1) ols_split2048_kernel(const OlsArgs a, const float2* tws)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t tmem_slot;
    constexpr uint32_t kCols = split_cols(WARPS, CARRY);
    static_assert(split_warp_cols(CARRY) * ((WARPS + 3) / 4) <= 512, "the warps' columns exceed the SM's tensor memory");
    float2* tw_s = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* wbase = smem_raw + Split::TW_BYTES + (size_t)warp * Split::WARP_BYTES;
    // job lists: the warp's first tile-list entry is read before the tables are copied (the tile
    // loop takes it as its one-tile-ahead entry)
    int64_t tb, te;
    warp_range(a.ntiles, (int64_t)gridDim.x * WARPS, (int64_t)blockIdx.x * WARPS + warp, tb, te);
    WarpState ws{-1, make_int2(0, 0), false};
    if constexpr (BATCH) {
        if (tb < te) {
            ws.ntd = opaque(a.tiles)[tb];
            ws.ntd_ok = true;
        }
    }
    for (int i = threadIdx.x; i < Split::TW_ENTRIES / 2; i += blockDim.x)
        reinterpret_cast<float4*>(tw_s)[i] = reinterpret_cast<const float4*>(tws)[i];
    if (warp == 0) {
        tmem_alloc(&tmem_slot, kCols);
        tmem_relinquish();
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tP = tmem_slot + ((uint32_t)(32 * (warp & 3)) << 16) +
                        (uint32_t)(split_warp_cols(CARRY) * (warp >> 2));
    const uint32_t tQ = tP + 64, tC = tP + 128;
    if constexpr (CARRY) {
        if (lane == 0) reinterpret_cast<SplitCarry*>(wbase + Split::CARRY_OFF)->in = nullptr;
        __syncwarp();
    }

    const bool bulk = (a.flags & kOlsNoBulk) == 0;
    for (int64_t tile = tb; tile < te; ++tile) {
        if constexpr (BATCH)
            split_tile<(WARPS > 12), CARRY>(JobListSource{a.jobs, a.tiles}, tile, tile + 1 < te, tw_s, a.V, a.LV,
                                            wbase, lane, ws, bulk, tP, tQ, tC);
        else
            split_tile<(WARPS > 12), false>(SingleJobSource{a}, tile, tile + 1 < te, tw_s, a.V, a.LV, wbase, lane,
                                            ws, bulk, tP, tQ, tC);
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(tmem_slot, kCols);
    }
}

// F2 tables of the split kernel, FP64 on the GPU rounded once: table 0 row t = W_2048^{2 t ka},
// table 1 = W_2048^{t (2 ka + 1)}, table 2 = W_2048^{ka (2 t + 1)}, ka < 32 (pad entries 0).
__global__ void split2048_twiddle_kernel(float2* tw)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Split::TW_ENTRIES) return;
    const int tab = idx / Split::TWTAB, r = idx % Split::TWTAB;
    const int t = r / Split::TWROW, ka = r % Split::TWROW;
    if (ka >= 32) {
        tw[idx] = make_float2(0.f, 0.f);
        return;
    }
    const int e = tab == 0 ? 2 * t * ka : (tab == 1 ? t * (2 * ka + 1) : ka * (2 * t + 1));
    double s, c;
    sincospi(-2.0 * (double)(e % 2048) / 2048.0, &s, &c);
    tw[idx] = make_float2((float)c, (float)s);
}

// Writes the H_R(K) that the split kernel applies for band k1 (test hook): its table build and its
// register-to-bin mapping, one warp; the tables' 1/N is undone exactly.
__global__ void split2048_export_hr_kernel(const float* V, int LV, int k1, float* out)
{
    __shared__ __align__(16) float gtab[Split::GT];
    const int t = threadIdx.x;
    build_split_gains(gtab, t, k1, LV, V);
    __syncwarp();
    for (int h = 0; h < 2; ++h) {
        const SplitGainRow g = split_gain_row(gtab, h, t);
        static_for<0, 32>([&](auto n1) {
            out[2 * (32 * decltype(n1)::value + t) + h] = split_gain<decltype(n1)::value>(g) * (float)Split::N;
        });
    }
}

template <int WARPS, bool BATCH, bool CARRY = false>
cudaError_t launch_split_w(const OlsArgs& a, const float2* tws, int sms, int max_ctas, cudaStream_t st,
                           int* grid_out)
{
    auto kern = ols_split2048_kernel<WARPS, BATCH, CARRY>;
    const size_t smem = Split::TW_BYTES + (size_t)WARPS * Split::WARP_BYTES;
    int per_sm = 0;
    cudaError_t e = prepared_occupancy((const void*)kern, WARPS * 32, smem, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t ctas_needed = (a.ntiles + WARPS - 1) / WARPS;
    int64_t cap = (int64_t)per_sm * sms;
    if (max_ctas > 0 && cap > max_ctas) cap = max_ctas;
    const int grid = (int)(ctas_needed < cap ? ctas_needed : cap);
    if (grid_out) *grid_out = grid;
    if (grid <= 0) return cudaSuccess;
    void* args[] = {const_cast<OlsArgs*>(&a), const_cast<const float2**>(&tws)};
    return cudaLaunchKernel((const void*)kern, dim3(grid), dim3(WARPS * 32), args, smem, st);
}

}  // namespace

// Entries (float2) of the split kernel's F2 tables; they follow the N = 2048 plan's four-step rows.
int split2048_table_entries() { return Split::TW_ENTRIES; }

cudaError_t build_split2048_table(float2* tw, cudaStream_t st)
{
    split2048_twiddle_kernel<<<(Split::TW_ENTRIES + 255) / 256, 256, 0, st>>>(tw);
    return cudaGetLastError();
}

cudaError_t launch_split2048_export_hr(const float* V, int LV, int k1, float* out, cudaStream_t st)
{
    split2048_export_hr_kernel<<<1, 32, 0, st>>>(V, LV, k1, out);
    return cudaGetLastError();
}

// a.tw: the plan's table, whose split tables start after its OlsGeom<2048>::TW four-step entries.
// Overlap N/4 and complex signals only.
cudaError_t launch_ols_split2048(const OlsArgs& a, int warps, int sms, int max_ctas, cudaStream_t st,
                                 int* grid_out)
{
    if (a.overlap != Split::O || (a.flags & kOlsReal)) return cudaErrorInvalidValue;
    const float2* tws = a.tw + OlsGeom<2048>::TW;
    const bool b = a.jobs != nullptr;
    // batches in host memory: the overlap samples are carried in tensor memory (8 or 12 warps)
    if (b && (a.flags & kOlsNoBulk) && warps <= 12)
        return warps == 8 ? launch_split_w<8, true, true>(a, tws, sms, max_ctas, st, grid_out)
                          : launch_split_w<12, true, true>(a, tws, sms, max_ctas, st, grid_out);
    switch (warps) {
    case 8: return b ? launch_split_w<8, true>(a, tws, sms, max_ctas, st, grid_out)
                     : launch_split_w<8, false>(a, tws, sms, max_ctas, st, grid_out);
    case 12: return b ? launch_split_w<12, true>(a, tws, sms, max_ctas, st, grid_out)
                      : launch_split_w<12, false>(a, tws, sms, max_ctas, st, grid_out);
    case 16: return b ? launch_split_w<16, true>(a, tws, sms, max_ctas, st, grid_out)
                      : launch_split_w<16, false>(a, tws, sms, max_ctas, st, grid_out);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace vbw

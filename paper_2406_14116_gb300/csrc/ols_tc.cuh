// OLS VBW filtering with the DFT and IDFT stages as complex DFT-matrix GEMMs on the tensor cores
// (tcgen05, FP32 accumulation in TMEM): the precision variant of the fused FP32 kernel.
//
// Four-step DFT with N = R1 * R2, on a tile of 8 consecutive blocks of one stream:
//   round 1  rows (b, n2), n2 < R2: DFT-R1 of x_b(R2 n1 + n2) over n1   -> A1(k1), k1 < R1
//            twiddle W_N^{n2 k1}, transpose through shared memory (FP32)
//   round 2  rows (b, k1), k1 < R1: DFT-R2 over n2                      -> X_b(k1 + R1 k2)
//            gains H_R(k)/N of eq. (FS_Hk_real), then swap(a + jb) = b + ja
//   round 3  rows (b, k1): DFT-R2 over k2                                -> A'(k1'), k1' < R2
//            twiddle W_N^{k1 k1'}, transpose
//   round 4  rows (b, k1'): DFT-R1 over k1                               -> Z(k1' + R2 k2')
// Rounds 3-4 are the forward four-step of size R2 x R1 applied to swap(H_R X / N); since
// IDFT(y) = swap(DFT(swap(y))), z = swap(Z) is the IDFT of eq. (OLS_dn). The linear phase of
// eq. (FS_Hk_exp) is the store shift by D = O/2, as in the FP32 kernel.
//
// Each round is D[row, :] = A[row, :] B with the DFT-R matrix in real form (K = N_out = 2R):
// out = [yr; yi] = [[Fr, -Fi], [Fi, Fr]] [xr; xi]; B is stored K-major, i.e. as those rows.
// Operands are 16-bit pieces in shared memory:
//   BF16x3  v ~ hi + lo (bfloat16), products hi*hi + hi*lo + lo*hi          (3 MMAs per K step)
//   BF16x6  v ~ hi + mid + lo, products hh hm mh hl lh mm                   (6 MMAs per K step)
//   FP16S   each data row scaled into (-1, 1) by a power of two, hi + lo in fp16, products
//           hi*hi + hi*lo + lo*hi; the accumulator row is scaled back exactly.
// The DFT matrices are generated in FP64 at plan time and split into the pieces there.
#pragma once

#include "ols_fp32.cuh"
#include "tc_common.cuh"

namespace vbw {

enum TcPrec { kTcBf16x3 = 1, kTcFp16s = 2, kTcBf16x6 = 3 };

template <int PREC>
struct TcSplit {
    static constexpr bool BF16 = PREC != kTcFp16s;
    static constexpr int PIECES = PREC == kTcBf16x6 ? 3 : 2;
    static constexpr int PRODUCTS = PREC == kTcBf16x6 ? 6 : 3;
    static constexpr bool SCALED = PREC == kTcFp16s;
    // (A piece, B piece) of product i
    __host__ __device__ static constexpr int pa(int i)
    {
        return PREC == kTcBf16x6 ? (i == 2 ? 1 : i == 4 ? 2 : i == 5 ? 1 : 0) : (i == 2 ? 1 : 0);
    }
    __host__ __device__ static constexpr int pb(int i)
    {
        return PREC == kTcBf16x6 ? (i == 1 ? 1 : i == 3 ? 2 : i == 5 ? 1 : 0) : (i == 1 ? 1 : 0);
    }
};

template <int N>
struct TcGeom;
template <> struct TcGeom<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct TcGeom<512> { static constexpr int R1 = 32, R2 = 16; };

constexpr int kTcBlocks = 8;     // blocks per tile
constexpr int kTcThreads = 128;  // one warpgroup
constexpr int kTcTmemCols = 64;

// Shared-memory plan of one CTA (bytes).
template <int N, int PREC>
struct TcSmem {
    static constexpr int R1 = TcGeom<N>::R1, R2 = TcGeom<N>::R2;
    static constexpr int P = TcSplit<PREC>::PIECES;
    static constexpr int A_PIECE = kTcBlocks * N * 2 * 2;          // rows x K = 16 N in every round
    static constexpr int B1_PIECE = (2 * R1) * (2 * R1) * 2;       // DFT-R1 matrix, one piece
    static constexpr int B2_PIECE = (2 * R2) * (2 * R2) * 2;       // DFT-R2 matrix, one piece
    static constexpr int TROW1 = 2 * R2 + 1;                       // transpose after round 1
    static constexpr int TROW3 = 2 * R1 + 1;                       // transpose after round 3
    static constexpr int T_FLOATS = (kTcBlocks * R1 * TROW1 > kTcBlocks * R2 * TROW3)
                                        ? kTcBlocks * R1 * TROW1 : kTcBlocks * R2 * TROW3;
    // ALIAS (one round-2 row per thread, N = 256): the transpose buffer shares the operand
    // buffer. A transpose is written only after the previous round's MMAs completed (their
    // operands are consumed), and every thread reads its transposed row into registers before
    // any thread writes the next operands (a barrier in between).
    static constexpr bool ALIAS = kTcBlocks * R1 == kTcThreads;
    static constexpr size_t A_BYTES = (size_t)P * A_PIECE;
    static constexpr size_t T_BYTES = sizeof(float) * T_FLOATS;
    static constexpr size_t OFF_A = 0;
    static constexpr size_t OFF_B1 =
        ALIAS ? ((A_BYTES > T_BYTES ? A_BYTES : T_BYTES) + 127) / 128 * 128 : OFF_A + A_BYTES;
    static constexpr size_t OFF_B2 = OFF_B1 + (size_t)P * B1_PIECE;
    static constexpr size_t OFF_T = ALIAS ? OFF_A : OFF_B2 + (size_t)P * B2_PIECE;
    static constexpr size_t OFF_END = ALIAS ? OFF_B2 + (size_t)P * B2_PIECE : OFF_T + T_BYTES;
    // the twiddles W[a][b], W[b][a] stay in the plan's device table and are read through L1
    static constexpr size_t OFF_V = (OFF_END + 127) / 128 * 128;
    static constexpr size_t OFF_BAR = (OFF_V + sizeof(float) * (N / 2) + 127) / 128 * 128;
    static constexpr size_t BYTES = OFF_BAR + 64;
    // per-plan device table: B1 pieces then B2 pieces (shared-memory image), then the twiddles
    static constexpr size_t MAT_BYTES = (size_t)P * (B1_PIECE + B2_PIECE);
    static constexpr size_t TABLE_BYTES = MAT_BYTES + 2 * sizeof(float2) * N;
    static_assert(OFF_B1 % 128 == 0 && OFF_B2 % 128 == 0 && OFF_T % 16 == 0, "alignment");
    static_assert(MAT_BYTES % 16 == 0, "16-byte copies");
    static_assert(MAT_BYTES == OFF_B2 + (size_t)P * B2_PIECE - OFF_B1, "matrix image is contiguous");
};

// Power-of-two scale of a data row for the FP16 variant: v * inv lies in (-1, 1), v = (v * inv) * s.
__device__ __forceinline__ void row_scale(float maxabs, float& s, float& inv)
{
    const uint32_t E = (__float_as_uint(maxabs) >> 23) & 0xFFu;
    if (E == 0 || E >= 250) {
        s = 1.f;
        inv = 1.f;
        return;
    }
    const int e = (int)E - 126;                        // maxabs < 2^e
    s = __uint_as_float((uint32_t)(127 + e) << 23);
    inv = __uint_as_float((uint32_t)(127 - e) << 23);
}

// Writes row `row` (K real values v, times inv) of the 16-bit operand pieces in core-matrix layout.
template <int PREC, int K>
__device__ __forceinline__ void put_row(unsigned char* A, size_t piece_bytes, int row, const float* v, float inv)
{
    using S = TcSplit<PREC>;
    using H = Half16<S::BF16>;
    using T16 = typename H::T;
    constexpr int P = S::PIECES;
#pragma unroll
    for (int c = 0; c < K / 8; ++c) {
        T16 pc[P][8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float r = v[c * 8 + e] * inv;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const T16 q = H::from(r);
                pc[p][e] = q;
                r -= H::to(q);
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            uint4 w;
            memcpy(&w, pc[p], 16);
            *reinterpret_cast<uint4*>(A + (size_t)p * piece_bytes + core_offset(row, c * 8, K)) = w;
        }
    }
}

// One GEMM round, issued by one thread: D[half h] (TMEM columns h*K ..) = A[rows of half h] B.
template <int PREC, int K>
__device__ __forceinline__ void issue_round(unsigned char* A, size_t a_piece, unsigned char* Bm, size_t b_piece,
                                            int halves, uint32_t tmem, uint64_t* bar)
{
    using S = TcSplit<PREC>;
    constexpr uint32_t idesc = umma_idesc(S::BF16, 128, K);
    constexpr uint32_t sbo = (K / 8) * 128;
    for (int h = 0; h < halves; ++h) {
#pragma unroll
        for (int s = 0; s < K / 16; ++s) {
#pragma unroll
            for (int i = 0; i < S::PRODUCTS; ++i) {
                const uint64_t ad = umma_desc(A + S::pa(i) * a_piece + (size_t)h * 128 * K * 2 + s * 256, 128, sbo);
                const uint64_t bd = umma_desc(Bm + S::pb(i) * b_piece + s * 256, 128, sbo);
                umma_f16(tmem + (uint32_t)(h * K), ad, bd, idesc, (s > 0 || i > 0) ? 1u : 0u);
            }
        }
    }
    umma_commit(bar);
}

template <int N, int PREC, bool BATCH>
__global__ void __launch_bounds__(kTcThreads) ols_tc_kernel(const OlsArgs a)
{
    using G = TcSmem<N, PREC>;
    using S = TcSplit<PREC>;
    constexpr int R1 = G::R1, R2 = G::R2, K1 = 2 * R1, K2 = 2 * R2;
    constexpr int O = N / 4, M = N - O, D = O / 2;
    constexpr int H2 = kTcBlocks * R1 / kTcThreads;   // row halves of rounds 2-3 (1 or 2)
    static_assert(kTcBlocks * R2 == kTcThreads, "rounds 1 and 4 have one row per thread");

    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* Abuf = sm + G::OFF_A;
    unsigned char* B1 = sm + G::OFF_B1;
    unsigned char* B2 = sm + G::OFF_B2;
    float* Tb = reinterpret_cast<float*>(sm + G::OFF_T);
    const float2* twA = reinterpret_cast<const float2*>(a.tc_tables + G::MAT_BYTES);   // [k1][n2]
    const float2* twB = twA + N;                                                       // [k1'][k1]
    float* Vs = reinterpret_cast<float*>(sm + G::OFF_V);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + G::OFF_BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + G::OFF_BAR + 8);
    const int tid = threadIdx.x, warp = tid >> 5;

    {
        const uint4* src = reinterpret_cast<const uint4*>(a.tc_tables);
        uint4* dst = reinterpret_cast<uint4*>(sm + G::OFF_B1);
        for (int i = tid; i < (int)(G::MAT_BYTES / 16); i += kTcThreads) dst[i] = src[i];
        for (int i = tid; i < a.LV; i += kTcThreads) Vs[i] = a.V[i];
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(tslot, kTcTmemCols);
        tmem_relinquish();
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t lane_tmem = tmem + ((uint32_t)(warp * 32) << 16);
    const long long limit = a.wait_limit > 0 ? a.wait_limit : kWaitLimitCycles;
    uint32_t phase = 0;
    bool alive = true;

    // MMA round: operands written -> issue -> bounded wait for the accumulator
    auto round = [&](auto kc, unsigned char* Bm, size_t b_piece, int halves) -> bool {
        constexpr int K = decltype(kc)::value;
        fence_proxy_async_smem();
        tc_fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after_sync();
            // test hook (debug bit 0): no MMAs, so nothing arrives and the bounded wait runs out
            if (!(a.debug & 1)) issue_round<PREC, K>(Abuf, G::A_PIECE, Bm, b_piece, halves, tmem, bar);
        }
        bool ok = mbar_wait_bounded(bar, phase, limit);
        if (!__syncthreads_and(ok)) {
            if (tid == 0 && a.status) atomicOr(a.status, kStatusWaitTimeout);
            mbar_wait_bounded(bar, phase, limit);   // the MMAs may still be running: wait once more
            __syncthreads();
            return false;
        }
        phase ^= 1u;
        tc_fence_after_sync();
        return true;
    };

    const int64_t ntiles = a.ntiles;
    const int64_t per = ntiles / gridDim.x, extra = ntiles % gridDim.x;
    const int64_t tb = (int64_t)blockIdx.x * per + ((int64_t)blockIdx.x < extra ? blockIdx.x : extra);
    const int64_t te = tb + per + ((int64_t)blockIdx.x < extra ? 1 : 0);
    for (int64_t tile = tb; tile < te && alive; ++tile) {
        OlsJob job;
        int64_t blk0;
        if constexpr (BATCH) {
            const int2 td = a.tiles[tile];
            job = a.jobs[td.x];
            blk0 = td.y;
        } else {
            job = a.job;
            blk0 = tile * kTcBlocks;
        }
        const int64_t nsamp = job.nsamp;
        const int64_t nblocks = (nsamp + M - 1) / M;
        float rs[H2];   // FP16 row scales of the current round's rows

        // ask L2 for the next tile's input span while this tile runs its four rounds
        if (tid == 0 && tile + 1 < te && (a.flags & kOlsNoBulk) == 0) {
            OlsJob nj;
            int64_t nb0;
            if constexpr (BATCH) {
                const int2 nd = a.tiles[tile + 1];
                nj = a.jobs[nd.x];
                nb0 = nd.y;
            } else {
                nj = a.job;
                nb0 = (tile + 1) * kTcBlocks;
            }
            int64_t e = nb0 * M - O;
            int64_t e2 = (nb0 + kTcBlocks) * M;
            if (e < 0) e = 0;
            if (e2 > nj.nsamp) e2 = nj.nsamp;
            if ((reinterpret_cast<uintptr_t>(nj.in + e) & 15) != 0) ++e;
            const int64_t cnt = (e2 - e) & ~int64_t(1);
            if (cnt > 0 && (reinterpret_cast<uintptr_t>(nj.in + e) & 15) == 0)
                prefetch_l2_bulk(nj.in + e, (uint32_t)(cnt * sizeof(float2)));
        }

        // ---- round 1 input: row tid = (b, n2), x_b(R2 n1 + n2), n1 < R1
        {
            const int b = tid / R2, n2 = tid % R2;
            const int64_t blk = blk0 + b;
            const int64_t s0 = blk * M - O;
            float v[K1];
            float mx = 0.f;
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) {
                const int64_t si = s0 + (int64_t)R2 * n1 + n2;
                float2 x = make_float2(0.f, 0.f);
                if (blk < nblocks) {
                    if (si >= 0) {
                        if (si < nsamp) x = ld_stream(job.in + si);
                    } else if (job.tail_in) {
                        x = job.tail_in[O + si];
                    }
                }
                v[n1] = x.x;
                v[R1 + n1] = x.y;
                mx = fmaxf(mx, fmaxf(fabsf(x.x), fabsf(x.y)));
            }
            float inv = 1.f;
            rs[0] = 1.f;
            if constexpr (S::SCALED) row_scale(mx, rs[0], inv);
            put_row<PREC, K1>(Abuf, G::A_PIECE, tid, v, inv);
        }
        if (!(alive = round(std::integral_constant<int, K1>{}, B1, G::B1_PIECE, 1))) break;

        // ---- round 1 output: twiddle W_N^{n2 k1}, transpose to rows (b, k1)
        {
            const int b = tid / R2, n2 = tid % R2;
#pragma unroll
            for (int c = 0; c < K1; c += 32) {
                float d[32];
                tmem_ld32(lane_tmem + c, d);
                // columns c..c+31 hold re (k1 < R1) then im; pair them after both halves are in
                if constexpr (K1 == 32) {
#pragma unroll
                    for (int k1 = 0; k1 < R1; ++k1) {
                        const float2 w = __ldg(twA + k1 * R2 + n2);
                        const float re = d[k1] * rs[0], im = d[R1 + k1] * rs[0];
                        float* row = Tb + (b * R1 + k1) * G::TROW1;
                        row[n2] = re * w.x - im * w.y;
                        row[R2 + n2] = re * w.y + im * w.x;
                    }
                } else {
                    // K1 = 64: first ld holds re of k1 0..31, the second im of k1 0..31
                    float* dst = Tb;
#pragma unroll
                    for (int k1 = 0; k1 < 32; ++k1) {
                        // stash re in the transpose row, combine with im on the second pass
                        float* row = dst + (b * R1 + k1) * G::TROW1;
                        if (c == 0) {
                            row[n2] = d[k1] * rs[0];
                        } else {
                            const float2 w = __ldg(twA + k1 * R2 + n2);
                            const float re = row[n2], im = d[k1] * rs[0];
                            row[n2] = re * w.x - im * w.y;
                            row[R2 + n2] = re * w.y + im * w.x;
                        }
                    }
                }
            }
        }
        tc_fence_before_sync();
        __syncthreads();

        // ---- round 2 input: rows (b, k1) from the transpose buffer
#pragma unroll
        for (int h = 0; h < H2; ++h) {
            const int r = tid + h * kTcThreads;
            const float* row = Tb + r * G::TROW1;
            float v[K2];
            float mx = 0.f;
#pragma unroll
            for (int i = 0; i < K2; ++i) {
                v[i] = row[i];
                mx = fmaxf(mx, fabsf(v[i]));
            }
            float inv = 1.f;
            rs[h] = 1.f;
            if constexpr (S::SCALED) row_scale(mx, rs[h], inv);
            if constexpr (G::ALIAS) __syncthreads();   // every transposed row read before overwriting
            put_row<PREC, K2>(Abuf, G::A_PIECE, r, v, inv);
        }
        if (!(alive = round(std::integral_constant<int, K2>{}, B2, G::B2_PIECE, H2))) break;

        // ---- round 2 output: X_b(k1 + R1 k2); gains H_R(k)/N; swap; round 3 input (same rows)
#pragma unroll
        for (int h = 0; h < H2; ++h) {
            const int r = tid + h * kTcThreads;
            const int b = r / R1, k1 = r % R1;
            const int64_t blk = blk0 + b;
            int band = job.band0;
            if (job.band) {
                if (blk < nblocks) band = job.band[blk];
            } else {
                for (int i = 0; i < a.nchg; ++i)
                    if (a.chg_block[i] <= blk) band = a.chg_band[i];
            }
            float d[32];
            tmem_ld32(lane_tmem + (uint32_t)(h * K2), d);
            float v[K2];
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) {
                const int k = k1 + R1 * k2;
                const int kk = k <= N / 2 ? k : N - k;
                const float g = hr_gain(kk, band, a.LV, Vs) * (1.0f / N) * rs[h];
                v[k2] = g * d[R2 + k2];        // swap: new re = im
                v[R2 + k2] = g * d[k2];        //       new im = re
            }
            float mx = 0.f;
#pragma unroll
            for (int i = 0; i < K2; ++i) mx = fmaxf(mx, fabsf(v[i]));
            float inv = 1.f;
            rs[h] = 1.f;
            if constexpr (S::SCALED) row_scale(mx, rs[h], inv);
            put_row<PREC, K2>(Abuf, G::A_PIECE, r, v, inv);
        }
        if (!(alive = round(std::integral_constant<int, K2>{}, B2, G::B2_PIECE, H2))) break;

        // ---- round 3 output: twiddle W_N^{k1 k1'}, transpose to rows (b, k1')
#pragma unroll
        for (int h = 0; h < H2; ++h) {
            const int r = tid + h * kTcThreads;
            const int b = r / R1, k1 = r % R1;
            float d[32];
            tmem_ld32(lane_tmem + (uint32_t)(h * K2), d);
#pragma unroll
            for (int kp = 0; kp < R2; ++kp) {
                const float2 w = __ldg(twB + kp * R1 + k1);
                const float re = d[kp] * rs[h], im = d[R2 + kp] * rs[h];
                float* row = Tb + (b * R2 + kp) * G::TROW3;
                row[k1] = re * w.x - im * w.y;
                row[R1 + k1] = re * w.y + im * w.x;
            }
        }
        tc_fence_before_sync();
        __syncthreads();

        // ---- round 4 input: rows (b, k1') = tid
        {
            const float* row = Tb + tid * G::TROW3;
            float v[K1];
            float mx = 0.f;
#pragma unroll
            for (int i = 0; i < K1; ++i) {
                v[i] = row[i];
                mx = fmaxf(mx, fabsf(v[i]));
            }
            float inv = 1.f;
            rs[0] = 1.f;
            if constexpr (S::SCALED) row_scale(mx, rs[0], inv);
            if constexpr (G::ALIAS) __syncthreads();   // every transposed row read before overwriting
            put_row<PREC, K1>(Abuf, G::A_PIECE, tid, v, inv);
        }
        if (!(alive = round(std::integral_constant<int, K1>{}, B1, G::B1_PIECE, 1))) break;

        // ---- round 4 output: z(n) = swap(Z(n)), n = k1' + R2 k2'; keep D <= n < D + M
        {
            const int b = tid / R2, kp = tid % R2;
            const int64_t blk = blk0 + b;
            float zr[R1], zi[R1];
#pragma unroll
            for (int c = 0; c < K1; c += 32) {
                float d[32];
                tmem_ld32(lane_tmem + c, d);
                if constexpr (K1 == 32) {
#pragma unroll
                    for (int i = 0; i < R1; ++i) {
                        zr[i] = d[R1 + i] * rs[0];   // swap
                        zi[i] = d[i] * rs[0];
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (c == 0) zi[i] = d[i] * rs[0];
                        else zr[i] = d[i] * rs[0];
                    }
                }
            }
            if (blk < nblocks) {
                const int64_t obase = blk * M - D;
#pragma unroll
                for (int k2 = 0; k2 < R1; ++k2) {
                    const int n = kp + R2 * k2;
                    if (n >= D && n < D + M) {
                        const int64_t oi = obase + n;
                        if (oi < nsamp) st_stream(job.out + oi, make_float2(zr[k2], zi[k2]));
                    }
                }
                // the rows of the job's last block hand the stream's last O input samples on
                if ((blk + 1) * M >= nsamp && job.tail_out) {
                    for (int i = kp; i < O; i += R2) {
                        const int64_t si = nsamp - O + i;
                        float2 x = make_float2(0.f, 0.f);
                        if (si >= 0) x = job.in[si];
                        else if (job.tail_in) x = job.tail_in[O + si];
                        job.tail_out[i] = x;
                    }
                }
            }
        }
        tc_fence_before_sync();
        __syncthreads();
    }

    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTcTmemCols);
}

// Per-plan table (device): the B pieces of the DFT-R1 and DFT-R2 matrices in the shared-memory
// image, then the twiddles W_N^{ab} as [k1 < R1][n2 < R2] and [k1' < R2][k1 < R1]. Built in FP64.
template <int N, int PREC>
__global__ void tc_table_kernel(unsigned char* out)
{
    using G = TcSmem<N, PREC>;
    using S = TcSplit<PREC>;
    constexpr int R1 = G::R1, R2 = G::R2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int n1 = (2 * R1) * (2 * R1), n2 = (2 * R2) * (2 * R2);
    if (i < n1 + n2) {
        const bool first = i < n1;
        const int R = first ? R1 : R2;
        const int j = first ? i : i - n1;
        const int K = 2 * R;
        const int row = j / K, col = j % K;   // out index, in index
        // [[Fr, -Fi], [Fi, Fr]], F(k, n) = exp(-j 2 pi k n / R)
        const int kq = row % R, nq = col % R;
        const long long e = ((long long)kq * nq) % R;
        double sn, cs;
        sincospi(-2.0 * (double)e / (double)R, &sn, &cs);
        double w;
        if (row < R) w = col < R ? cs : -sn;   // yr = Fr xr - Fi xi
        else w = col < R ? sn : cs;            // yi = Fi xr + Fr xi
        unsigned char* base = out + (first ? 0 : (size_t)S::PIECES * G::B1_PIECE);
        const size_t piece = first ? G::B1_PIECE : G::B2_PIECE;
        double rem = w;
        for (int p = 0; p < S::PIECES; ++p) {
            if constexpr (S::BF16) {
                const __nv_bfloat16 q = __double2bfloat16(rem);
                *reinterpret_cast<__nv_bfloat16*>(base + p * piece + core_offset(row, col, K)) = q;
                rem -= (double)__bfloat162float(q);
            } else {
                const __half q = __double2half(rem);
                *reinterpret_cast<__half*>(base + p * piece + core_offset(row, col, K)) = q;
                rem -= (double)__half2float(q);
            }
        }
    }
    if (i < N) {
        // twA[k1][n2] = W_N^{k1 n2}, twB[k1'][k1] = W_N^{k1' k1}
        float2* tw = reinterpret_cast<float2*>(out + G::MAT_BYTES);
        {
            const int k1 = i / R2, q = i % R2;
            const long long e = ((long long)k1 * q) % N;
            double sn, cs;
            sincospi(-2.0 * (double)e / (double)N, &sn, &cs);
            tw[i] = make_float2((float)cs, (float)sn);
        }
        {
            const int kp = i / R1, k1 = i % R1;
            const long long e = ((long long)kp * k1) % N;
            double sn, cs;
            sincospi(-2.0 * (double)e / (double)N, &sn, &cs);
            tw[N + i] = make_float2((float)cs, (float)sn);
        }
    }
}

}  // namespace vbw

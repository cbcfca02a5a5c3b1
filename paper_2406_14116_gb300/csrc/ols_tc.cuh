// OLS VBW filtering with the DFT and IDFT stages as complex DFT-matrix GEMMs on the tensor cores
// (tcgen05, FP32 accumulation in TMEM): the precision variant of the fused FP32 kernel.
//
// Four-step DFT with N = R1 * R2 (R2 = 16), on a tile of 8 consecutive blocks of one stream:
//   round 1  rows (b, n2), n2 < R2: DFT-R1 of x_b(R2 n1 + n2) over n1   -> A1(k1), k1 < R1
//            twiddle W_N^{n2 k1} (FP32)
//   round 2  rows (b, k1), k1 < R1: DFT-R2 over n2                      -> X_b(k1 + R1 k2)
//            gains H_R(k)/N of eq. (FS_Hk_real), then swap(a + jb) = b + ja
//   round 3  rows (b, k1): DFT-R2 over k2                                -> A'(k1'), k1' < R2
//            twiddle W_N^{k1 k1'}
//   round 4  rows (b, k1'): DFT-R1 over k1                               -> Z(k1' + R2 k2')
// Rounds 3-4 are the forward four-step of size R2 x R1 applied to swap(H_R X / N); since
// IDFT(y) = swap(DFT(swap(y))), z = swap(Z) is the IDFT of eq. (OLS_dn). The linear phase of
// eq. (FS_Hk_exp) is the store shift by D = O/2, as in the FP32 kernel.
//
// Each round is D[row, :] = A[row, :] B with the DFT-R matrix in real form: for out = [yr; yi],
// in = [xr; xi], B = [[Fr, -Fi], [Fi, Fr]], stored K-major (one row per output). Operands are
// 16-bit pieces in shared memory:
//   BF16x3  v ~ hi + lo (bfloat16), products hi*hi + hi*lo + lo*hi          (3 MMAs per K step)
//   BF16x6  v ~ hi + mid + lo, products hh hm mh hl lh mm                   (6 MMAs per K step)
//   FP16S   each block's operand values scaled into (-1, 1) by one power of two per block and
//           round, hi + lo in fp16, products hi*hi + hi*lo + lo*hi; the accumulator rows are scaled
//           back exactly.
// The DFT matrices are generated in FP64 at plan time and split into the pieces there.
//
// No transposes: a round's epilogue thread holds one row of the accumulator, i.e. one column of
// the next round's operand for 16 or 32 consecutive operand rows. Rounds 2 and 4 therefore take
// their A operand in MN-major layout (8 consecutive rows of one column per 16-byte line), which the
// epilogue writes with 128-bit stores straight from registers; rounds 1 and 3 take K-major rows.
//
// Stopband pruning (Sec. III-D: the bins where H_R = 0 cost nothing). The outputs of round 2 and the
// inputs of round 3 are ordered so that the first 16 real slots hold the 8 bins k2 nearest 0 (mod
// R2) and the last 16 slots the 8 inner bins k2 in [4, R2 - 5]. Those inner bins cover
// k in [N/4, 3N/4 - 1], inside the stopband [k2b + 1, N - k2b - 1] whenever k2b = k1 + L_V - 1 <=
// N/4 - 1. When every block of a tile has such a band, round 2 computes only the outer 16 output
// columns and round 3 reads only the outer 16 inputs: half of both rounds' tensor work and of the
// gain / split / store work between them is skipped.
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

// Real slot s (0..31) of the round-2 outputs and round-3 inputs: bin k2 and part (0 re, 1 im).
// Slots 0-7 re and 8-15 im of the outer bins {0, 1, 2, 3, 12, 13, 14, 15}; slots 16-23 re and
// 24-31 im of the inner bins {4 .. 11}.
__host__ __device__ constexpr int tc_slot_bin(int s)
{
    return (s >> 4) == 0 ? ((s & 7) < 4 ? (s & 7) : (s & 7) + 8) : (s & 7) + 4;
}
__host__ __device__ constexpr int tc_slot_part(int s) { return (s >> 3) & 1; }

// Byte offset of 16-bit element (row, k) of an R x K operand in K-major core matrices (a core
// matrix is 8 rows x 16 bytes along K), and of the 16-byte line holding rows row0 .. row0 + 7 of
// column k in MN-major core matrices (8 K-lines x 16 bytes along the rows). Both use the same grid:
// 128 bytes between core matrices along K, K/8 * 128 bytes between them along the rows.
__host__ __device__ constexpr uint32_t mn_line_offset(int row0, int k, int K)
{
    return (uint32_t)(((row0 >> 3) * (K >> 3) + (k >> 3)) * 128 + (k & 7) * 16);
}

// Shared-memory plan of one CTA (bytes).
template <int N, int PREC>
struct TcSmem {
    static constexpr int R1 = TcGeom<N>::R1, R2 = TcGeom<N>::R2;
    static_assert(R2 == 16, "the slot order of rounds 2-3 assumes R2 = 16");
    static constexpr int P = TcSplit<PREC>::PIECES;
    static constexpr int A_PIECE = kTcBlocks * N * 2 * 2;          // rows x K = 16 N in every round
    static constexpr int B1_PIECE = (2 * R1) * (2 * R1) * 2;       // DFT-R1 matrix, one piece
    static constexpr int B2_PIECE = (2 * R2) * (2 * R2) * 2;       // DFT-R2 matrices, one piece each
    // per-block gain table g(kk) = H_R / N, kk = 0..N/2; the stride is 16 banks mod 32 so that two
    // blocks read by one warp use disjoint banks
    static constexpr int GT = ((N / 2 + 1 + 31) / 32) * 32 + 16;
    static constexpr size_t OFF_A = 0;
    static constexpr size_t OFF_B1 = OFF_A + (size_t)P * A_PIECE;
    static constexpr size_t OFF_B2 = OFF_B1 + (size_t)P * B1_PIECE;    // round 2: slot-ordered outputs
    static constexpr size_t OFF_B3 = OFF_B2 + (size_t)P * B2_PIECE;    // round 3: slot-ordered inputs
    static constexpr size_t OFF_G = OFF_B3 + (size_t)P * B2_PIECE;
    static constexpr size_t OFF_V = OFF_G + sizeof(float) * kTcBlocks * GT;
    static constexpr size_t OFF_SC = OFF_V + sizeof(float) * (N / 2);  // FP16: block scales of A2, A4
    static constexpr size_t OFF_BAR = OFF_SC + sizeof(float) * 2 * kTcBlocks;
    static constexpr size_t BYTES = OFF_BAR + 16;
    // per-plan device table: the B1, B2, B3 pieces (shared-memory image), then the FP32 twiddles
    // W_N^{k1 n2} as [k1 < R1][n2 < R2] and W_N^{k1' k1} as [k1' < R2][k1 < R1]
    static constexpr size_t MAT_BYTES = (size_t)P * (B1_PIECE + 2 * B2_PIECE);
    static constexpr size_t TABLE_BYTES = MAT_BYTES + 2 * sizeof(float2) * N;
    static_assert(OFF_B1 % 128 == 0 && OFF_B2 % 128 == 0 && OFF_B3 % 128 == 0 && OFF_G % 16 == 0, "alignment");
    static_assert(MAT_BYTES % 16 == 0 && OFF_BAR % 8 == 0, "16-byte copies, mbarrier alignment");
};

// Power-of-two scale for the FP16 variant: v * inv lies in (-1, 1), v = (v * inv) * s.
__device__ __forceinline__ void pow2_scale(float maxabs, float& s, float& inv)
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

// Maximum over the LANES consecutive lanes (a power of two <= 32) that hold one block.
template <int LANES>
__device__ __forceinline__ float lane_group_max(float m)
{
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    return m;
}

// (v0, v1) -> one 32-bit word per piece, element v0 in the low half (the lower address).
template <int PREC>
__device__ __forceinline__ void split_pair(float v0, float v1, uint32_t (&w)[TcSplit<PREC>::PIECES])
{
    using S = TcSplit<PREC>;
    if constexpr (S::BF16) {
        uint32_t h;
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(v1), "f"(v0));
        w[0] = h;
        float r0 = v0 - __uint_as_float(h << 16), r1 = v1 - __uint_as_float(h & 0xFFFF0000u);
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(r1), "f"(r0));
        w[1] = h;
        if constexpr (S::PIECES == 3) {
            r0 -= __uint_as_float(h << 16);
            r1 -= __uint_as_float(h & 0xFFFF0000u);
            asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(r1), "f"(r0));
            w[2] = h;
        }
    } else {
        uint32_t h;
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(v1), "f"(v0));
        w[0] = h;
        float f0, f1;
        asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\tcvt.f32.f16 %0, lo;\n\tcvt.f32.f16 %1, hi;\n\t}"
            : "=f"(f0), "=f"(f1) : "r"(h));
        const float r0 = v0 - f0, r1 = v1 - f1;
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(r1), "f"(r0));
        w[1] = h;
    }
}

// Splits 8 values (times inv for the scaled variant) and stores their 16-byte line in every piece.
template <int PREC, int A_PIECE>
__device__ __forceinline__ void store_line(uint32_t a_smem, uint32_t off, const float* v, float inv)
{
    using S = TcSplit<PREC>;
    constexpr int P = S::PIECES;
    uint32_t w[P][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t t[P];
        if constexpr (S::SCALED) split_pair<PREC>(v[2 * j] * inv, v[2 * j + 1] * inv, t);
        else split_pair<PREC>(v[2 * j], v[2 * j + 1], t);
#pragma unroll
        for (int p = 0; p < P; ++p) w[p][j] = t[p];
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a_smem + p * A_PIECE + off), "r"(w[p][0]),
                     "r"(w[p][1]), "r"(w[p][2]), "r"(w[p][3])
                     : "memory");
}

// 16 consecutive TMEM columns of this thread's lane (warp-wide, 32x32b shape); not waited.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// One GEMM round, issued by one thread: D[half h] (TMEM columns h * tcol ..) = A[rows of half h] B
// over the first `kuse` of the operand's KA columns, into `nout` output columns (B stored K-major,
// KB columns per row). A_MN: A in MN-major core matrices.
template <int PREC, bool A_MN, int KA, int KB>
__device__ __forceinline__ void issue_round(uint32_t a_smem, uint32_t a_piece, uint32_t b_smem, uint32_t b_piece,
                                            int halves, int kuse, int nout, uint32_t tmem, uint32_t tcol,
                                            uint64_t* bar)
{
    using S = TcSplit<PREC>;
    const uint32_t idesc = umma_idesc(S::BF16, 128, nout) | (A_MN ? (1u << 15) : 0u);
    constexpr uint32_t sbo_a = (KA / 8) * 128, sbo_b = (KB / 8) * 128;
    for (int h = 0; h < halves; ++h) {
        for (int s = 0; s < kuse / 16; ++s) {
#pragma unroll
            for (int i = 0; i < S::PRODUCTS; ++i) {
                const uint64_t ad = umma_desc_u32(a_smem + S::pa(i) * a_piece + (uint32_t)h * 128 * KA * 2 + s * 256,
                                                  128, sbo_a);
                const uint64_t bd = umma_desc_u32(b_smem + S::pb(i) * b_piece + s * 256, 128, sbo_b);
                umma_f16(tmem + (uint32_t)h * tcol, ad, bd, idesc, (s > 0 || i > 0) ? 1u : 0u);
            }
        }
    }
    umma_commit(bar);
}

// k1 of block blk of a job: its per-block band array, else band0 with the launch's inline changes
__device__ __forceinline__ int tc_block_band(const OlsArgs& a, const OlsJob& job, int64_t blk)
{
    if (job.band) return job.band[blk];
    int band = job.band0;
    for (int i = 0; i < a.nchg; ++i)
        if (a.chg_block[i] <= blk) band = a.chg_band[i];
    return band;
}

// Resident CTAs per SM the N = 256 kernel is compiled for (its register budget: 4 CTAs leave 128
// registers, enough for the tables each epilogue loads while the GEMMs run); N = 512 is held to
// three CTAs by shared memory.
#ifndef VBW_TC_MIN_CTAS_256
#define VBW_TC_MIN_CTAS_256 4
#endif

template <int N, int PREC, bool BATCH>
__global__ void __launch_bounds__(kTcThreads, N == 256 ? VBW_TC_MIN_CTAS_256 : 3) ols_tc_kernel(const OlsArgs a)
{
    using G = TcSmem<N, PREC>;
    using S = TcSplit<PREC>;
    constexpr int R1 = G::R1, R2 = G::R2, K1 = 2 * R1, K2 = 2 * R2, GT = G::GT;
    constexpr int O = N / 4, M = N - O, D = O / 2;
    constexpr int H2 = kTcBlocks * R1 / kTcThreads;   // row halves of rounds 2-3 (1 or 2)
    constexpr int L23 = R1 < 32 ? R1 : 32;            // lanes that hold one block in rounds 2-3
    constexpr uint32_t AP = G::A_PIECE;
    // kept outputs n = k1' + R2 k2' in [D, N - D): k2' in [D / R2, (N - D) / R2)
    constexpr int KLO = D / R2, KHI = (N - D) / R2;
    static_assert(kTcBlocks * R2 == kTcThreads, "rounds 1 and 4 have one row per thread");
    static_assert(D % R2 == 0, "the kept outputs are whole columns of round 4");

    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t sA = smem_u32(sm + G::OFF_A);
    const uint32_t sB1 = smem_u32(sm + G::OFF_B1), sB2 = smem_u32(sm + G::OFF_B2), sB3 = smem_u32(sm + G::OFF_B3);
    float* gtab = reinterpret_cast<float*>(sm + G::OFF_G);
    float* Vs = reinterpret_cast<float*>(sm + G::OFF_V);
    float* sc = reinterpret_cast<float*>(sm + G::OFF_SC);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + G::OFF_BAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + G::OFF_BAR + 8);
    // twiddles, read through L1 with the reading thread's index fastest (coalesced)
    const float2* twA = reinterpret_cast<const float2*>(a.tc_tables + G::MAT_BYTES);   // [k1][n2]
    const float2* twB = twA + N;                                                       // [k1'][k1]
    const int tid = threadIdx.x, warp = tid >> 5;

    {
        const uint4* src = reinterpret_cast<const uint4*>(a.tc_tables);
        uint4* dst = reinterpret_cast<uint4*>(sm + G::OFF_B1);
        for (int i = tid; i < (int)(G::MAT_BYTES / 16); i += kTcThreads) dst[i] = src[i];
        for (int i = tid; i < a.LV; i += kTcThreads) Vs[i] = a.V[i];
        for (int i = tid; i < kTcBlocks * GT; i += kTcThreads) gtab[i] = 0.f;
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
    int gband = -1;   // band of this thread's gain-table slot (tid & 7) when it was last built

    // MMA round: operands written -> issue -> `pre` (loads the next epilogue's tables while the
    // GEMMs run) -> bounded wait for the accumulator. The barrier also returns the AND of every
    // thread's `vote`.
    auto round = [&](auto amn, auto ka, auto kb, uint32_t sB, uint32_t b_piece, int halves, int kuse,
                     int nout, uint32_t tcol, int vote, int* vote_all, auto&& pre) -> bool {
        fence_proxy_async_smem();
        tc_fence_before_sync();
        const int all = __syncthreads_and(vote);
        if (vote_all) *vote_all = all;
        if (tid == 0) {
            tc_fence_after_sync();
            // test hook (debug bit 0): no MMAs, so nothing arrives and the bounded wait runs out
            if (!(a.debug & 1))
                issue_round<PREC, decltype(amn)::value, decltype(ka)::value, decltype(kb)::value>(
                    sA, AP, sB, b_piece, halves, kuse, nout, tmem, tcol, bar);
        }
        pre();
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

        // ---- gain table of block tid & 7 (rebuilt only when its band changes: eq. (FS_Hk_real) is
        //      a re-indexing of V), and this block's vote for stopband pruning
        int vote;
        {
            const int b = tid & 7;
            const int64_t blk = blk0 + b;
            const bool act = blk < nblocks;
            const int band = act ? tc_block_band(a, job, blk) : gband;
            if (act && band != gband) {
                float* g = gtab + b * GT;
                for (int kk = tid >> 3; kk <= N / 2; kk += kTcThreads / kTcBlocks)
                    g[kk] = hr_gain(kk, band, a.LV, Vs) * (1.0f / N);
                gband = band;
            }
            vote = !act || (band + a.LV - 1 <= N / 4 - 1);
        }

        // ---- round 1 input: row tid = (b, n2), x_b(R2 n1 + n2), n1 < R1 (K-major)
        float s1 = 1.f;   // FP16: scale of this block's round-1 rows
        {
            const int b = tid / R2, n2 = tid % R2;
            const int64_t blk = blk0 + b;
            const int64_t s0 = blk * M - O;
            float v[K1];
            const bool interior = blk < nblocks && s0 >= 0 && s0 + N <= nsamp;
            if (__all_sync(0xffffffffu, interior)) {
                const float2* sp = job.in + s0 + n2;
#pragma unroll
                for (int n1 = 0; n1 < R1; ++n1) {
                    const float2 x = ld_stream(sp + R2 * n1);
                    v[n1] = x.x;
                    v[R1 + n1] = x.y;
                }
            } else {
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
                }
            }
            float inv = 1.f;
            if constexpr (S::SCALED) {
                float mx = 0.f;
#pragma unroll
                for (int i = 0; i < K1; ++i) mx = fmaxf(mx, fabsf(v[i]));
                pow2_scale(lane_group_max<R2>(mx), s1, inv);
            }
#pragma unroll
            for (int c = 0; c < K1 / 8; ++c) store_line<PREC, AP>(sA, core_offset(tid, 8 * c, K1), v + 8 * c, inv);
        }
        int prune = 0;
        float2 tw1[R1];   // W_N^{n2 k1}, k1 < R1, for this thread's round-1 row
        if (!(alive = round(std::false_type{}, std::integral_constant<int, K1>{}, std::integral_constant<int, K1>{},
                            sB1, G::B1_PIECE, 1, K1, K1, 0, vote, &prune, [&] {
                                const float2* tw = twA + tid % R2;
#pragma unroll
                                for (int k = 0; k < R1; ++k) tw1[k] = __ldg(tw + k * R2);
                            })))
            break;

        // ---- round 1 output: twiddle W_N^{n2 k1}; rows (b, k1) of round 2 as MN-major lines
        {
            const int b = tid / R2, n2 = tid % R2;
            float re[R1], im[R1];
#pragma unroll
            for (int c = 0; c < R1; c += 16) {
                tmem_ld16(lane_tmem + c, re + c);
                tmem_ld16(lane_tmem + R1 + c, im + c);
            }
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < R1 / 2; ++j) {
                const float4 w = make_float4(tw1[2 * j].x, tw1[2 * j].y, tw1[2 * j + 1].x, tw1[2 * j + 1].y);
                float r0 = re[2 * j], i0 = im[2 * j], r1 = re[2 * j + 1], i1 = im[2 * j + 1];
                if constexpr (S::SCALED) {
                    r0 *= s1; i0 *= s1; r1 *= s1; i1 *= s1;
                }
                re[2 * j] = r0 * w.x - i0 * w.y;
                im[2 * j] = r0 * w.y + i0 * w.x;
                re[2 * j + 1] = r1 * w.z - i1 * w.w;
                im[2 * j + 1] = r1 * w.w + i1 * w.z;
            }
            float inv = 1.f;
            if constexpr (S::SCALED) {
                float mx = 0.f;
#pragma unroll
                for (int i = 0; i < R1; ++i) mx = fmaxf(mx, fmaxf(fabsf(re[i]), fabsf(im[i])));
                float s2;
                pow2_scale(lane_group_max<R2>(mx), s2, inv);
                if (n2 == 0) sc[b] = s2;
            }
#pragma unroll
            for (int h = 0; h < R1 / 8; ++h) {
                store_line<PREC, AP>(sA, mn_line_offset(b * R1 + 8 * h, n2, K2), re + 8 * h, inv);
                store_line<PREC, AP>(sA, mn_line_offset(b * R1 + 8 * h, R2 + n2, K2), im + 8 * h, inv);
            }
        }
        // gains of this thread's round-2 rows: gp[h][i] for slot i (outer bins) and slot i + 8
        // (inner bins, i >= 8), read from the block's table while the GEMMs run
        float gp[H2][16];
        if (!(alive = round(std::true_type{}, std::integral_constant<int, K2>{}, std::integral_constant<int, K2>{},
                            sB2, G::B2_PIECE, H2, K2, prune ? K2 / 2 : K2, K2, 1, nullptr, [&] {
#pragma unroll
                                for (int h = 0; h < H2; ++h) {
                                    const int r = tid + h * kTcThreads;
                                    const int b = r / R1, k1 = r % R1;
                                    const uint32_t glo = smem_u32(gtab + b * GT + k1);
                                    const uint32_t ghi = smem_u32(gtab + b * GT + N - k1);
                                    auto load = [&](auto ii) {
                                        constexpr int i = decltype(ii)::value;
                                        constexpr int k2 = tc_slot_bin(i < 8 ? i : i + 8);
                                        gp[h][i] = k2 < R2 / 2 ? lds_f32(glo + 4 * R1 * k2) : lds_f32(ghi - 4 * R1 * k2);
                                    };
                                    static_for<0, 8>(load);
                                    if (!prune) static_for<8, 16>(load);
                                }
                            })))
            break;

        // ---- round 2 output: X_b(k1 + R1 k2) in slot order; gains H_R(k)/N; swap; round-3 rows
        float s3[H2];   // FP16: scale of this thread's round-3 rows
#pragma unroll
        for (int h = 0; h < H2; ++h) {
            const int r = tid + h * kTcThreads;
            const int b = r / R1;
            float d[K2];
            tmem_ld16(lane_tmem + (uint32_t)(h * K2), d);
            if (!prune) tmem_ld16(lane_tmem + (uint32_t)(h * K2 + 16), d + 16);
            tmem_ld_wait();
            float sc2 = 1.f;
            if constexpr (S::SCALED) sc2 = sc[b];
            float v[K2];
            auto gain_swap = [&](auto sre) {
                constexpr int s = decltype(sre)::value;
                float gk = gp[h][s < 8 ? s : s - 8];
                if constexpr (S::SCALED) gk *= sc2;
                v[s] = gk * d[s + 8];       // swap: new re = im
                v[s + 8] = gk * d[s];       //       new im = re
            };
            static_for<0, 8>(gain_swap);
            if (!prune) static_for<16, 24>(gain_swap);
            float inv = 1.f;
            s3[h] = 1.f;
            if constexpr (S::SCALED) {
                float mx = 0.f;
#pragma unroll
                for (int i = 0; i < 16; ++i) mx = fmaxf(mx, fabsf(v[i]));
                if (!prune) {
#pragma unroll
                    for (int i = 16; i < K2; ++i) mx = fmaxf(mx, fabsf(v[i]));
                }
                pow2_scale(lane_group_max<L23>(mx), s3[h], inv);
            }
            store_line<PREC, AP>(sA, core_offset(r, 0, K2), v, inv);
            store_line<PREC, AP>(sA, core_offset(r, 8, K2), v + 8, inv);
            if (!prune) {
                store_line<PREC, AP>(sA, core_offset(r, 16, K2), v + 16, inv);
                store_line<PREC, AP>(sA, core_offset(r, 24, K2), v + 24, inv);
            }
        }
        float2 tw3[H2][R2];   // W_N^{k1 k1'}, k1' < R2, for this thread's round-3 rows
        if (!(alive = round(std::false_type{}, std::integral_constant<int, K2>{}, std::integral_constant<int, K2>{},
                            sB3, G::B2_PIECE, H2, prune ? K2 / 2 : K2, K2, K2, 1, nullptr, [&] {
#pragma unroll
                                for (int h = 0; h < H2; ++h) {
                                    const float2* tw = twB + (tid + h * kTcThreads) % R1;
#pragma unroll
                                    for (int k = 0; k < R2; ++k) tw3[h][k] = __ldg(tw + k * R1);
                                }
                            })))
            break;

        // ---- round 3 output: twiddle W_N^{k1 k1'}; rows (b, k1') of round 4 as MN-major lines
#pragma unroll
        for (int h = 0; h < H2; ++h) {
            const int r = tid + h * kTcThreads;
            const int b = r / R1, k1 = r % R1;
            float re[R2], im[R2];
            tmem_ld16(lane_tmem + (uint32_t)(h * K2), re);
            tmem_ld16(lane_tmem + (uint32_t)(h * K2 + R2), im);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < R2 / 2; ++j) {
                const float4 w = make_float4(tw3[h][2 * j].x, tw3[h][2 * j].y, tw3[h][2 * j + 1].x, tw3[h][2 * j + 1].y);
                float r0 = re[2 * j], i0 = im[2 * j], r1 = re[2 * j + 1], i1 = im[2 * j + 1];
                if constexpr (S::SCALED) {
                    r0 *= s3[h]; i0 *= s3[h]; r1 *= s3[h]; i1 *= s3[h];
                }
                re[2 * j] = r0 * w.x - i0 * w.y;
                im[2 * j] = r0 * w.y + i0 * w.x;
                re[2 * j + 1] = r1 * w.z - i1 * w.w;
                im[2 * j + 1] = r1 * w.w + i1 * w.z;
            }
            float inv = 1.f;
            if constexpr (S::SCALED) {
                float mx = 0.f;
#pragma unroll
                for (int i = 0; i < R2; ++i) mx = fmaxf(mx, fmaxf(fabsf(re[i]), fabsf(im[i])));
                float s4;
                pow2_scale(lane_group_max<L23>(mx), s4, inv);
                if (k1 == 0) sc[kTcBlocks + b] = s4;
            }
#pragma unroll
            for (int hh = 0; hh < R2 / 8; ++hh) {
                store_line<PREC, AP>(sA, mn_line_offset(b * R2 + 8 * hh, k1, K1), re + 8 * hh, inv);
                store_line<PREC, AP>(sA, mn_line_offset(b * R2 + 8 * hh, R1 + k1, K1), im + 8 * hh, inv);
            }
        }
        if (!(alive = round(std::true_type{}, std::integral_constant<int, K1>{}, std::integral_constant<int, K1>{},
                            sB1, G::B1_PIECE, 1, K1, K1, 0, 1, nullptr, [] {})))
            break;

        // ---- round 4 output: z(n) = swap(Z(n)), n = k1' + R2 k2'; keep D <= n < D + M
        {
            const int b = tid / R2, kp = tid % R2;
            const int64_t blk = blk0 + b;
            float zr[R1], zi[R1];
#pragma unroll
            for (int c = 0; c < R1; c += 16) {
                tmem_ld16(lane_tmem + c, zr + c);
                tmem_ld16(lane_tmem + R1 + c, zi + c);
            }
            tmem_ld_wait();
            float s4 = 1.f;
            if constexpr (S::SCALED) s4 = sc[kTcBlocks + b];
            if (blk < nblocks) {
                float2* dst = job.out + (blk * M - D) + kp;
                if ((blk + 1) * M <= nsamp) {
#pragma unroll
                    for (int k2 = KLO; k2 < KHI; ++k2)
                        st_stream(dst + R2 * k2, make_float2(zi[k2] * s4, zr[k2] * s4));
                } else {
                    const int64_t obase = blk * M - D + kp;
#pragma unroll
                    for (int k2 = KLO; k2 < KHI; ++k2)
                        if (obase + R2 * k2 < nsamp) st_stream(dst + R2 * k2, make_float2(zi[k2] * s4, zr[k2] * s4));
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
    }

    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTcTmemCols);
}

// Real-form DFT-R matrix entry for output (bin kq, part po) and input (bin nq, part pi):
// [[Fr, -Fi], [Fi, Fr]] with F(k, n) = exp(-j 2 pi k n / R), from FP64 sincospi with the exponent
// k n reduced exactly mod R.
__device__ __forceinline__ double dft_real_entry(int R, int kq, int po, int nq, int pi)
{
    const long long e = ((long long)kq * nq) % R;
    double sn, cs;
    sincospi(-2.0 * (double)e / (double)R, &sn, &cs);
    if (po == 0) return pi == 0 ? cs : -sn;   // yr = Fr xr - Fi xi
    return pi == 0 ? sn : cs;                 // yi = Fi xr + Fr xi
}

// Per-plan table (device): the B pieces of the DFT-R1 matrix (rounds 1 and 4, natural order), the
// DFT-R2 matrix of round 2 (natural inputs, slot-ordered outputs) and of round 3 (slot-ordered
// inputs, natural outputs), all in the shared-memory image; then the twiddles W_N^{k1 n2} as
// [k1 < R1][n2 < R2] and W_N^{k1' k1} as [k1' < R2][k1 < R1]. Built in FP64.
template <int N, int PREC>
__global__ void tc_table_kernel(unsigned char* out)
{
    using G = TcSmem<N, PREC>;
    using S = TcSplit<PREC>;
    constexpr int R1 = G::R1, R2 = G::R2, K1 = 2 * R1, K2 = 2 * R2;
    constexpr int n1 = K1 * K1, n2 = K2 * K2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1 + 2 * n2) {
        int K, row, col, which;
        if (i < n1) {
            which = 0; K = K1; row = i / K1; col = i % K1;
        } else {
            which = (i - n1) < n2 ? 1 : 2;
            const int j = (i - n1) % n2;
            K = K2; row = j / K2; col = j % K2;
        }
        double w;
        if (which == 0) {
            w = dft_real_entry(R1, row % R1, row / R1, col % R1, col / R1);
        } else if (which == 1) {
            w = dft_real_entry(R2, tc_slot_bin(row), tc_slot_part(row), col % R2, col / R2);
        } else {
            w = dft_real_entry(R2, row % R2, row / R2, tc_slot_bin(col), tc_slot_part(col));
        }
        unsigned char* base = out + (which == 0 ? 0
                                                : (size_t)S::PIECES * G::B1_PIECE +
                                                      (size_t)(which - 1) * S::PIECES * G::B2_PIECE);
        const size_t piece = which == 0 ? G::B1_PIECE : G::B2_PIECE;
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

// Fused FP32 overlap-save VBW kernel: gather -> N-point FFT -> H_R on the fly -> IFFT -> discard
// and store, one kernel, one pass over HBM (Sec. II steps 1-5 with eq. (FS_Hk_exp)/(FS_Hk_real)).
//
// Decomposition (four-step FFT, N = E * T):
//   thread t of a block holds x(T n1 + t), n1 = 0..E-1 (coalesced loads),
//   F1  E-point register DFT over n1                      -> A(ka, t)
//   F2  A(ka, t) *= W_N^{t ka} / sqrt(N)                  (shared-memory table)
//   F3  shared-memory transpose: thread t now owns ka = s T + t (s < E/T), every n2
//   F4  T-point register DFTs over n2                     -> X(ka + E k'), k' = 0..T-1
//   H   X(k) *= H_R(k) from (k1, L_V, V): passband untouched, transition scaled, stopband zeroed
//   I1  T-point inverse register DFTs over k'             -> B(ka, n2)
//   I3  transpose back: thread t owns n2 = t, every ka
//   I2  B(ka, t) *= conj(W_N^{t ka}) / sqrt(N)            (the two 1/sqrt(N) give eq. (OLS_dn)'s 1/N)
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
    static constexpr int ROW = T + 1;   // padded transpose row (float2 elements)
    // per-block transpose buffer; for T = 8 two blocks share a half-warp, so their buffers are
    // offset by 8 elements mod 16 to keep 64-bit accesses conflict-free
    static constexpr int BLK = E * ROW + ((T == 8) ? 8 : 0);
    static constexpr int WARP_BUF = B * BLK;
    static_assert(E * T == N && E % T == 0, "layout must satisfy N = E*T with T | E");
};

// Shared memory of one CTA: twiddles (N float2), V (L_V floats, padded to 4), transpose buffers.
template <int N>
__host__ __device__ inline size_t ols_smem_bytes(int warps, int LV)
{
    const int lvpad = (LV + 3) & ~3;
    return sizeof(float2) * (size_t)N + sizeof(float) * (size_t)lvpad +
           sizeof(float2) * (size_t)warps * OlsGeom<N>::WARP_BUF;
}

// H_R(k) of eq. (FS_Hk_real) applied to the spectrum held in the pass-2 layout:
// c[s][k'] = X(k) with k = s T + t + E k'. For k' < T/2, k < N/2; otherwise the mirror
// index N - k is used, so H_R(N - k) = H_R(k). With r = min(k, N-k) - k1: r < 0 passband (x1),
// 0 <= r < L_V transition (x V(r)), r >= L_V stopband (x0; k = N/2 is always stopband).
template <int N>
__device__ __forceinline__ void apply_band(float2 (&c)[OlsGeom<N>::S][OlsGeom<N>::T], int t, int k1,
                                           int LV, const float* V)
{
    constexpr int E = OlsGeom<N>::E, T = OlsGeom<N>::T, S = OlsGeom<N>::S;
    static_for<0, S>([&](auto s) {
        static_for<0, T>([&](auto kp) {
            constexpr int KP = decltype(kp)::value;
            constexpr int base = decltype(s)::value * T + E * KP;
            int kk;
            if constexpr (KP < T / 2) kk = base + t;
            else kk = N - base - t;
            const int r = kk - k1;
            float2 v = c[s][kp];
            if (r >= LV) {
                v = make_float2(0.f, 0.f);
            } else if (r >= 0) {
                const float g = V[r];
                v.x *= g;
                v.y *= g;
            }
            c[s][kp] = v;
        });
    });
}

__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldg(p); }
__device__ __forceinline__ void st_stream(float2* p, float2 v) { __stcs(p, v); }

template <int N, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) ols_fp32_kernel(const OlsArgs a)
{
    using G = OlsGeom<N>;
    constexpr int E = G::E, T = G::T, B = G::B, S = G::S, ROW = G::ROW;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tw_s = reinterpret_cast<float2*>(smem_raw);
    float* V_s = reinterpret_cast<float*>(tw_s + N);
    const int LV = a.LV;
    float2* bufs = reinterpret_cast<float2*>(V_s + ((LV + 3) & ~3));

    for (int i = threadIdx.x; i < N; i += blockDim.x) tw_s[i] = a.tw[i];
    for (int i = threadIdx.x; i < LV; i += blockDim.x) V_s[i] = a.V[i];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bsub = lane / T, t = lane % T;
    float2* buf = bufs + warp * G::WARP_BUF + bsub * G::BLK;
    const int O = a.overlap, M = N - O, D = O >> 1;

    const int64_t warp_stride = (int64_t)gridDim.x * WARPS;
    for (int64_t tile = (int64_t)blockIdx.x * WARPS + warp; tile < a.ntiles; tile += warp_stride) {
        // ---- which job and block this lane group works on
        OlsJob job;
        int64_t blk;
        if (a.jobs) {
            const int2 td = a.tiles[tile];
            job = a.jobs[td.x];
            blk = (int64_t)td.y + bsub;
        } else {
            job = a.job;
            blk = tile * B + bsub;
        }
        const float2* in = job.in;
        float2* out = job.out;
        const float2* tail_in = job.tail_in;
        const int64_t nsamp = job.nsamp;
        const int64_t nblocks = (nsamp + M - 1) / M;
        const bool active = blk < nblocks;

        int k1 = job.band0;
        if (job.band) {
            if (active) k1 = job.band[blk];
        } else {
            for (int i = 0; i < a.nchg; ++i)
                if (a.chg_block[i] <= blk) k1 = a.chg_band[i];
        }

        // ---- gather x_m(n) = x(mM - O + n), n = T n1 + t (Sec. II segmentation)
        const int64_t s0 = blk * M - O;
        float2 v[E];
        const bool interior = active && s0 >= 0 && s0 + N <= nsamp;
        if (__all_sync(0xffffffffu, interior)) {
            const float2* src = in + s0 + t;
            static_for<0, E>([&](auto n1) { v[n1] = ld_stream(src + decltype(n1)::value * T); });
        } else {
            static_for<0, E>([&](auto n1) {
                const int64_t si = s0 + decltype(n1)::value * T + t;
                float2 x = make_float2(0.f, 0.f);
                if (active) {
                    if (si >= 0) {
                        if (si < nsamp) x = ld_stream(in + si);
                    } else if (tail_in) {
                        x = tail_in[O + si];
                    }
                }
                v[n1] = x;
            });
        }

        // ---- forward DFT (Sec. II step 1)
        fft_reg<E, false>(v);
        static_for<0, E>([&](auto ka) { v[ka] = cmul(v[ka], tw_s[decltype(ka)::value * T + t]); });
        static_for<0, E>([&](auto ka) { buf[decltype(ka)::value * ROW + t] = v[ka]; });
        __syncwarp();
        float2 c[S][T];
        static_for<0, S>([&](auto s) {
            static_for<0, T>([&](auto n2) {
                c[s][n2] = buf[(decltype(s)::value * T + t) * ROW + decltype(n2)::value];
            });
        });
        __syncwarp();
        static_for<0, S>([&](auto s) { fft_reg<T, false>(c[s]); });

        // ---- multiply by H_R(k, b) (step 2; the phase term is the output shift below)
        apply_band<N>(c, t, k1, LV, V_s);

        // ---- inverse DFT (step 3)
        static_for<0, S>([&](auto s) { fft_reg<T, true>(c[s]); });
        static_for<0, S>([&](auto s) {
            static_for<0, T>([&](auto n2) {
                buf[(decltype(s)::value * T + t) * ROW + decltype(n2)::value] = c[s][n2];
            });
        });
        __syncwarp();
        static_for<0, E>([&](auto ka) { v[ka] = buf[decltype(ka)::value * ROW + t]; });
        __syncwarp();
        static_for<0, E>([&](auto ka) { v[ka] = cmul_conj(v[ka], tw_s[decltype(ka)::value * T + t]); });
        fft_reg<E, true>(v);

        // ---- discard and store (steps 4-5): z(n), n = T n1 + t, kept for D <= n < D + M
        if (active) {
            const int64_t obase = blk * M - D;
            static_for<0, E>([&](auto n1) {
                const int n = decltype(n1)::value * T + t;
                if (n >= D && n < D + M) {
                    const int64_t oi = obase + n;
                    if (oi < nsamp) st_stream(out + oi, v[n1]);
                }
            });
            // the lane group of the job's last block hands the stream's last O input samples on
            if (blk == nblocks - 1 && job.tail_out) {
                float2* tail_out = job.tail_out;
                for (int i = t; i < O; i += T) {
                    const int64_t si = nsamp - O + i;
                    float2 x = make_float2(0.f, 0.f);
                    if (si >= 0) x = in[si];
                    else if (tail_in) x = tail_in[O + si];
                    tail_out[i] = x;
                }
            }
        }
    }
}

// Writes the H_R(k) that apply_band<N> applies for band k1 (test hook), using the same code and
// register layout: one lane group of T threads, spectrum of ones.
template <int N>
__global__ void export_hr_kernel(const float* V, int LV, int k1, float* out)
{
    using G = OlsGeom<N>;
    constexpr int E = G::E, T = G::T, S = G::S;
    const int t = threadIdx.x;
    if (t >= T) return;
    float2 c[S][T];
    static_for<0, S>([&](auto s) {
        static_for<0, T>([&](auto kp) { c[s][kp] = make_float2(1.f, 0.f); });
    });
    apply_band<N>(c, t, k1, LV, V);
    static_for<0, S>([&](auto s) {
        static_for<0, T>([&](auto kp) {
            out[decltype(s)::value * T + t + E * decltype(kp)::value] = c[s][kp].x;
        });
    });
}

// Launch helpers (instantiated per N in ols_fp32_n<N>.cu).
template <int N, int WARPS>
cudaError_t launch_ols_fp32_w(const OlsArgs& a, int sms, cudaStream_t st, int* grid_out)
{
    const size_t smem = ols_smem_bytes<N>(WARPS, a.LV);
    auto kern = ols_fp32_kernel<N, WARPS>;
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
    switch (warps) {
    case 4: return launch_ols_fp32_w<N, 4>(a, sms, st, grid_out);
    case 8: return launch_ols_fp32_w<N, 8>(a, sms, st, grid_out);
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

// PTVIR error analysis of the VBW filter on the GPU (Sec. II, eq. (OLS_Hn); Sec. III-C,
// eq. (err_min)): for every band b and frequency w of a grid, the largest error over the M output
// phases of the OLS block, max_n |H_n(w, b) e^{j w O/2} - d(w)|, and the phase that reaches it.
// This is the search over (n, w, b) that the minimax design of the transition samples V
// (eq. (minimax)) repeats on every iteration.
//
// Output phase n of a block sees tap q of h = IDFT(H) (eq. (OLS_dn)) q samples back when
// q <= n + O and, through the circular wrap, N - q samples ahead otherwise. With
// a_q = h(q) e^{-j w (q - O/2)}, P0 = sum_{q <= O} a_q, R = sum_{q > O} a_q and the partial sums
// A(p) = sum_{O < q <= p} a_q, phase n = p - O has
//     E_n = P0 + A(p) + e^{j w N} (R - A(p)) - d = alpha + u A(p),
//     alpha = P0 + e^{j w N} R - d,   u = 1 - e^{j w N},
// so one pass for R and one prefix pass give every phase in O(N) work per (w, b) instead of
// O(N M). Phase M - 1 (A = R) is the plain DTFT of h, the response d_{M-1} of eq. (OLS_dn).
//
// h is built per band in shared memory from the cosine form of d_{M-1}(q, b) (Sec. III-B), with
// the passband part summed in closed form (a Dirichlet kernel):
//     N h(q) = sin((2 k1 - 1) theta / 2) / sin(theta / 2) + sum_r 2 V(r) cos((k1 + r) theta),
//     theta = pi (2q - O) / N,
// every angle reduced exactly in integers before sinpif / cospif. Stored coefficients: none per
// band, only V (eq. (FS_Hk_real)).
//
// Phasors e^{-j w x} (x a multiple of 1/2) come from the turn count (w / 4 pi) (2x) mod 1, split
// into a 24-bit fixed-point part reduced exactly in integer arithmetic and a small float
// remainder, then one sincospif per pair of 16-tap groups (the second group's seed is the first's
// times e^{-j w 16}, one extra rounding). Inside a group the taps are summed against
// a per-thread table e^{-j w l}, l < 16 (seeded the same way), and the group's seed multiplies the
// group sum once: a tap costs two FMAs in the sums and, in the phase scan, one complex
// multiply-add and a squared modulus. The running sums across groups are compensated (two-sum),
// so the arithmetic error stays near a few float32 roundings of the terms.
//
// h is symmetric about (L-1)/2 (H_R is real and even, eq. (FS_Hk_real)): h(q) = h((O - q) mod N),
// so the CTA evaluates the closed form once per pair of taps.
#include <math.h>
#include <stdint.h>

#include "vbw_internal.h"

namespace {

constexpr int kPtThreads = 256;   // grid points per CTA (one per thread)
constexpr int kGroup = 16;        // taps per phasor seed

struct PtArgs {
    int N, O, LV;
    const float* V;         // L_V transition samples (float32, as the filter applies them)
    const int* bands;       // k1 per band row
    const double* omega;    // nbands x K radians per sample
    const float* desired;   // nbands x K desired values d
    int K;
    float* err;             // nbands x K: max_n |E_n|
    int* phase;             // nbands x K: the n reaching it (first on ties), or null
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// e^{-j w a / 2} for an integer a with |a| < 2^13: the turn count g a mod 1 (g = w / 4 pi mod 1,
// split as n1 2^-24 + g2) is r = (n1 a mod 2^24) 2^-24 + g2 a, the first term exact in 32-bit
// integer arithmetic (only the low 24 bits of the product matter, so the wrap-around of the
// unsigned product is harmless), centred into [-1/2, 1/2).
__device__ __forceinline__ float2 phasor(uint32_t n1, float g2, int a)
{
    const uint32_t u = (n1 * static_cast<uint32_t>(a)) & 0xFFFFFFu;
    const int c = static_cast<int>(u) - ((u & 0x800000u) ? 0x1000000 : 0);
    const float r = fmaf(g2, static_cast<float>(a), static_cast<float>(c) * 5.9604644775390625e-8f);
    float s, co;
    sincospif(2.0f * r, &s, &co);
    return make_float2(co, -s);
}

// (s, c) += x with the two-sum error term kept in c (compensated summation)
__device__ __forceinline__ void two_sum_add(float& s, float& c, float x)
{
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

// N h(q) of band k1 (see the top of this file), a = 2q - O.
__device__ float h_scaled(int N, int O, int k1, int LV, const float* V, int q)
{
    const int a = 2 * q - O;                  // |a| < 2N, and a = 0 only for q = O/2
    const int n4 = 4 * N, n2 = 2 * N;
    float pass;
    if (a == 0) {
        pass = static_cast<float>(2 * k1 - 1);
    } else {
        const int num = (((2 * k1 - 1) * a) % n4 + n4) % n4;
        const int den = (a % n4 + n4) % n4;
        const float inv2n = 1.0f / static_cast<float>(n2);   // a power of two: exact
        pass = sinpif(static_cast<float>(num) * inv2n) / sinpif(static_cast<float>(den) * inv2n);
    }
    float tr = 0.f;
    const float invn = 1.0f / static_cast<float>(N);
    for (int r = 0; r < LV; ++r) {
        const int idx = (((k1 + r) * a) % n2 + n2) % n2;
        tr = fmaf(2.0f * __ldg(V + r), cospif(static_cast<float>(idx) * invn), tr);
    }
    return pass + tr;
}

__global__ void __launch_bounds__(kPtThreads) ptvir_error_kernel(const PtArgs p)
{
    extern __shared__ __align__(16) float hsh[];
    const int N = p.N, O = p.O, M = N - O;
    const int row = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * kPtThreads + threadIdx.x;
    const int64_t at = (int64_t)row * p.K + i;
    const int k1 = __ldg(p.bands + row);
    if (k1 < 1 || k1 + p.LV - 1 > N / 2 - 2) {   // outside the range of eq. (k_var)
        if (i < p.K) {
            p.err[at] = __int_as_float(0x7fc00000);
            if (p.phase) p.phase[at] = -1;
        }
        return;
    }
    // hA: taps q = O + 1 .. N - 1, hB: taps q = 0 .. O, each zero padded to whole groups
    const int nA = M - 1, nB = O + 1;
    const int pA = (nA + kGroup - 1) / kGroup * kGroup, pB = (nB + kGroup - 1) / kGroup * kGroup;
    float* hA = hsh;
    float* hB = hsh + pA;
    const float invn = 1.0f / static_cast<float>(N);
    for (int idx = threadIdx.x; idx < pA + pB; idx += blockDim.x)   // the padding
        if ((idx < pA && idx >= nA) || (idx >= pA && idx - pA >= nB)) hsh[idx] = 0.f;
    // taps q with 2q - O in [0, N] (q = (O + a)/2), each written with its mirror q' = (O - q) mod N
    for (int q = (O + 1) / 2 + threadIdx.x; 2 * q - O <= N && q < N; q += blockDim.x) {
        const float v = h_scaled(N, O, k1, p.LV, p.V, q) * invn;
        const int qm = ((O - q) % N + N) % N;
        hsh[q > O ? q - (O + 1) : pA + q] = v;
        hsh[qm > O ? qm - (O + 1) : pA + qm] = v;
    }
    __syncthreads();
    if (i >= p.K) return;

    const double w = p.omega[at];
    const float d = p.desired[at];
    double g = w * (1.0 / (4.0 * 3.141592653589793238462643383279502884));
    g -= rint(g);
    const double gs = g * 16777216.0;
    const double n1d = rint(gs);
    const uint32_t n1 = static_cast<uint32_t>(static_cast<int>(n1d));
    const float g2 = static_cast<float>((gs - n1d) * (1.0 / 16777216.0));

    float2 rot[kGroup];
#pragma unroll
    for (int l = 0; l < kGroup; ++l) rot[l] = phasor(n1, g2, 2 * l);   // e^{-j w l}
    const float2 rotg = phasor(n1, g2, 2 * kGroup);                      // e^{-j w 16}
    // seed of the group starting at tap offset c0 (a = a0 + 2 c0): exact for even groups, the
    // previous seed times e^{-j w 16} for odd ones
    float2 seed = make_float2(1.f, 0.f);
    auto group_seed = [&](int a0, int c0) {
        seed = ((c0 / kGroup) & 1) ? cmulf(seed, rotg) : phasor(n1, g2, a0 + 2 * c0);
        return seed;
    };

    // R = sum_{q > O} a_q: a_q = h(q) e^{-j w (q - O/2)}, 2 (q - O/2) = O + 2 + 2 idx
    float Rx = 0.f, Ry = 0.f, Rcx = 0.f, Rcy = 0.f;
    for (int c0 = 0; c0 < pA; c0 += kGroup) {
        const float2 base = group_seed(O + 2, c0);
        float qx = 0.f, qy = 0.f;
#pragma unroll
        for (int l = 0; l < kGroup; ++l) {
            const float hv = hA[c0 + l];
            qx = fmaf(hv, rot[l].x, qx);
            qy = fmaf(hv, rot[l].y, qy);
        }
        const float2 loc = cmulf(base, make_float2(qx, qy));
        two_sum_add(Rx, Rcx, loc.x);
        two_sum_add(Ry, Rcy, loc.y);
    }
    // P0 = sum_{q <= O} a_q, 2 (q - O/2) = 2 q - O
    float Px = 0.f, Py = 0.f, Pcx = 0.f, Pcy = 0.f;
    for (int c0 = 0; c0 < pB; c0 += kGroup) {
        const float2 base = group_seed(-O, c0);
        float qx = 0.f, qy = 0.f;
#pragma unroll
        for (int l = 0; l < kGroup; ++l) {
            const float hv = hB[c0 + l];
            qx = fmaf(hv, rot[l].x, qx);
            qy = fmaf(hv, rot[l].y, qy);
        }
        const float2 loc = cmulf(base, make_float2(qx, qy));
        two_sum_add(Px, Pcx, loc.x);
        two_sum_add(Py, Pcy, loc.y);
    }
    const float2 ewn = phasor(n1, g2, -2 * N);                    // e^{+j w N}
    const float2 R = make_float2(Rx + Rcx, Ry + Rcy);
    const float2 eR = cmulf(ewn, R);
    const float2 alpha = make_float2((Px + Pcx) + eR.x - d, (Py + Pcy) + eR.y);
    const float2 u = make_float2(1.0f - ewn.x, -ewn.y);

    // phase n = 0 (p = O): A = 0
    float best = alpha.x * alpha.x + alpha.y * alpha.y;
    int arg = 0;
    // phases n = 1 .. M - 1 (p = O + n): A(p) = sum of a_q, O < q <= p, i.e. the sum before the
    // group plus base * Q_l with Q_l = sum_{i <= l} h e^{-j w i}; padded taps add zero and repeat
    // the previous phase's value, which never replaces it (the first maximum is kept)
    float Ax = 0.f, Ay = 0.f, Acx = 0.f, Acy = 0.f;
    for (int c0 = 0; c0 < pA; c0 += kGroup) {
        const float2 base = group_seed(O + 2, c0);
        const float2 A = make_float2(Ax + Acx, Ay + Acy);
        const float2 ac = make_float2(alpha.x + (u.x * A.x - u.y * A.y), alpha.y + (u.x * A.y + u.y * A.x));
        const float2 ub = cmulf(u, base);
        float qx = 0.f, qy = 0.f;
        float m2[kGroup];
#pragma unroll
        for (int l = 0; l < kGroup; ++l) {
            const float hv = hA[c0 + l];
            qx = fmaf(hv, rot[l].x, qx);
            qy = fmaf(hv, rot[l].y, qy);
            const float ex = fmaf(ub.x, qx, fmaf(-ub.y, qy, ac.x));
            const float ey = fmaf(ub.x, qy, fmaf(ub.y, qx, ac.y));
            m2[l] = fmaf(ex, ex, ey * ey);
        }
        float gmax = m2[0];
#pragma unroll
        for (int l = 1; l < kGroup; ++l) gmax = fmaxf(gmax, m2[l]);
        if (gmax > best) {
            int first = kGroup - 1;
#pragma unroll
            for (int l = kGroup - 1; l >= 0; --l)
                if (m2[l] == gmax) first = l;
            best = gmax;
            arg = c0 + first + 1;
        }
        const float2 loc = cmulf(base, make_float2(qx, qy));
        two_sum_add(Ax, Acx, loc.x);
        two_sum_add(Ay, Acy, loc.y);
    }
    p.err[at] = sqrtf(best);
    if (p.phase) p.phase[at] = arg;
}

}  // namespace

extern "C" vbw_status vbw_ptvir_error(vbw_plan_t plan, const int* bands, int nbands, const double* omega,
                                      const float* desired, int K, float* err, int* phase,
                                      void* cuda_stream)
{
    if (!plan) return fail(VBW_ERR_INVALID_ARG, "vbw_ptvir_error: null plan");
    if (nbands < 0 || nbands > 65535 || K < 0)
        return fail(VBW_ERR_INVALID_ARG, "vbw_ptvir_error: nbands %d (0..65535) or K %d (>= 0) out of range",
                    nbands, K);
    if (nbands == 0 || K == 0) return ok();
    if (!bands || !omega || !desired || !err)
        return fail(VBW_ERR_INVALID_ARG, "vbw_ptvir_error: null array");
    if ((reinterpret_cast<uintptr_t>(omega) & 7) || (reinterpret_cast<uintptr_t>(bands) & 3) ||
        (reinterpret_cast<uintptr_t>(desired) & 3) || (reinterpret_cast<uintptr_t>(err) & 3) ||
        (reinterpret_cast<uintptr_t>(phase) & 3))
        return fail(VBW_ERR_INVALID_ARG, "vbw_ptvir_error: misaligned array");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device)
        return fail(VBW_ERR_INVALID_ARG, "vbw_ptvir_error: the plan's device is not the current device");
    PtArgs a{};
    a.N = plan->N;
    a.O = plan->O;
    a.LV = plan->LV;
    a.V = plan->d_V;
    a.bands = bands;
    a.omega = omega;
    a.desired = desired;
    a.K = K;
    a.err = err;
    a.phase = phase;
    const int M = a.N - a.O;
    const int pA = (M - 1 + kGroup - 1) / kGroup * kGroup, pB = (a.O + 1 + kGroup - 1) / kGroup * kGroup;
    const size_t smem = sizeof(float) * (size_t)(pA + pB);
    const dim3 grid((unsigned)((K + kPtThreads - 1) / kPtThreads), (unsigned)nbands);
    ptvir_error_kernel<<<grid, kPtThreads, smem, static_cast<cudaStream_t>(cuda_stream)>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(VBW_ERR_CUDA, "vbw_ptvir_error: launch failed: %s", cudaGetErrorString(e));
    return ok();
}

// Register-resident DFT codelets (FP32) with compile-time twiddles.
//
// fft_reg<R, INV>(a) overwrites a[0..R) with its R-point DFT:
//   forward (INV = false): A(k) = sum_n a(n) exp(-j 2 pi n k / R)
//   inverse (INV = true):  A(k) = sum_n a(n) exp(+j 2 pi n k / R)      (no 1/R)
// as radix-2 decimation-in-time stages over a bit-reversed copy. All indices are compile-time
// constants, so the bit reversal is register renaming and the twiddles are FFMA immediates.
//
// Butterfly cost (FP32 instructions per (u, v) pair):
//   w = 1, -1, +-j                  4 adds (signs folded)
//   w = (+-1 +-j)/sqrt(2)           2 adds + 4 FFMA
//   any other w = c + j s           "tangent" form w v = c ((v.x - t v.y) + j (v.y + t v.x)) with
//                                   t = s/c (or the cotangent form when |s| > |c|, so |t| <= 1):
//                                   2 FFMA for the rotation + 4 FFMA for u +- c(.)  = 6
#pragma once

#include "vbw_common.cuh"

namespace vbw {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// a * w
__device__ __forceinline__ float2 cmul(float2 a, float2 w)
{
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}

// a * conj(w)
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 w)
{
    return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

template <int R>
constexpr int bit_reverse(int i)
{
    int r = 0;
    for (int b = 1; b < R; b <<= 1) {
        r = (r << 1) | (i & 1);
        i >>= 1;
    }
    return r;
}

constexpr double cabs_d(double x) { return x < 0 ? -x : x; }

// (u, v) <- (u + w v, u - w v) with w = exp(-+ j 2 pi J / LEN) ('-' forward, '+' inverse).
template <int LEN, int J, bool INV>
__device__ __forceinline__ void bfly(float2& u, float2& v)
{
    constexpr int j = ((J % LEN) + LEN) % LEN;
    if constexpr (j == 0) {
        const float2 a = u, b = v;
        u = make_float2(a.x + b.x, a.y + b.y);
        v = make_float2(a.x - b.x, a.y - b.y);
    } else if constexpr (2 * j == LEN) {
        const float2 a = u, b = v;
        u = make_float2(a.x - b.x, a.y - b.y);
        v = make_float2(a.x + b.x, a.y + b.y);
    } else if constexpr (4 * j == LEN || 4 * j == 3 * LEN) {
        // w = -j (forward, j = LEN/4) or +j; the inverse flips the sign.
        constexpr bool minus_j = (4 * j == LEN) != INV;
        const float2 a = u, b = v;
        if constexpr (minus_j) {   // w v = (v.y, -v.x)
            u = make_float2(a.x + b.y, a.y - b.x);
            v = make_float2(a.x - b.y, a.y + b.x);
        } else {                   // w v = (-v.y, v.x)
            u = make_float2(a.x - b.y, a.y + b.x);
            v = make_float2(a.x + b.y, a.y - b.x);
        }
    } else {
        constexpr CosSin cs = cos_sin_2pi(j, LEN);
        constexpr double c = cs.c;
        constexpr double s = INV ? cs.s : -cs.s;
        const float2 a = u, b = v;
        if constexpr (8 * j == LEN || 8 * j == 3 * LEN || 8 * j == 5 * LEN || 8 * j == 7 * LEN) {
            // w = h (sc + j ss), sc, ss in {+1, -1}, h = sqrt(1/2)
            constexpr float h = static_cast<float>(cabs_d(c));
            constexpr float sc = c > 0 ? 1.f : -1.f;
            constexpr float ss = s > 0 ? 1.f : -1.f;
            const float p = sc * b.x - ss * b.y;      // sign products fold into FADD
            const float q = sc * b.y + ss * b.x;
            u = make_float2(fmaf(h, p, a.x), fmaf(h, q, a.y));
            v = make_float2(fmaf(-h, p, a.x), fmaf(-h, q, a.y));
        } else if constexpr (cabs_d(c) >= cabs_d(s)) {
            constexpr float cf = static_cast<float>(c);
            constexpr float t = static_cast<float>(s / c);
            const float p = fmaf(-t, b.y, b.x);
            const float q = fmaf(t, b.x, b.y);
            u = make_float2(fmaf(cf, p, a.x), fmaf(cf, q, a.y));
            v = make_float2(fmaf(-cf, p, a.x), fmaf(-cf, q, a.y));
        } else {
            constexpr float sf = static_cast<float>(s);
            constexpr float t = static_cast<float>(c / s);
            const float p = fmaf(t, b.x, -b.y);
            const float q = fmaf(t, b.y, b.x);
            u = make_float2(fmaf(sf, p, a.x), fmaf(sf, q, a.y));
            v = make_float2(fmaf(-sf, p, a.x), fmaf(-sf, q, a.y));
        }
    }
}

// Radix-2 DIT stages of length FIRST_LEN..R over the bit-reversed array b.
template <int R, int FIRST_LOG, bool INV>
__device__ __forceinline__ void dit_stages(float2 (&b)[R])
{
    static_for<FIRST_LOG, ilog2(R) + 1>([&](auto sl) {
        constexpr int len = 1 << decltype(sl)::value;
        constexpr int half = len / 2;
        static_for<0, R, len>([&](auto g) {
            static_for<0, half>([&](auto jj) {
                constexpr int lo = decltype(g)::value + decltype(jj)::value;
                bfly<len, decltype(jj)::value, INV>(b[lo], b[lo + half]);
            });
        });
    });
}

template <int R, bool INV>
__device__ __forceinline__ void fft_reg(float2 (&a)[R])
{
    static_assert((R & (R - 1)) == 0 && R >= 1, "radix-2 codelet needs a power of two");
    if constexpr (R > 1) {
        float2 b[R];
        static_for<0, R>([&](auto i) { b[bit_reverse<R>(decltype(i)::value)] = a[i]; });
        dit_stages<R, 1, INV>(b);
        static_for<0, R>([&](auto i) { a[i] = b[i]; });
    }
}

}  // namespace vbw

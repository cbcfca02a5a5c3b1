// Register-resident DFT codelets (FP32) with compile-time twiddles.
//
// fft_reg<R, INV>(a) overwrites a[0..R) with its R-point DFT:
//   forward (INV = false): A(k) = sum_n a(n) exp(-j 2 pi n k / R)
//   inverse (INV = true):  A(k) = sum_n a(n) exp(+j 2 pi n k / R)      (no 1/R)
// as radix-2 decimation-in-time stages over a bit-reversed copy. All indices are compile-time
// constants, so the bit reversal is register renaming and the twiddles are FFMA immediates;
// multiplications by +-1 and +-j are turned into sign flips and swaps.
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

// v * exp(-+ j 2 pi J / LEN): '-' for the forward transform, '+' for the inverse.
template <int LEN, int J, bool INV>
__device__ __forceinline__ float2 twiddle_const(float2 v)
{
    constexpr int j = ((J % LEN) + LEN) % LEN;
    if constexpr (j == 0) {
        return v;
    } else if constexpr (2 * j == LEN) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (4 * j == LEN) {          // fwd: -j, inv: +j
        if constexpr (INV) return make_float2(-v.y, v.x);
        else return make_float2(v.y, -v.x);
    } else if constexpr (4 * j == 3 * LEN) {      // fwd: +j, inv: -j
        if constexpr (INV) return make_float2(v.y, -v.x);
        else return make_float2(-v.y, v.x);
    } else {
        constexpr CosSin cs = cos_sin_2pi(j, LEN);
        constexpr float wr = static_cast<float>(cs.c);
        constexpr float wi = INV ? static_cast<float>(cs.s) : -static_cast<float>(cs.s);
        return make_float2(fmaf(v.x, wr, -v.y * wi), fmaf(v.x, wi, v.y * wr));
    }
}

template <int R, bool INV>
__device__ __forceinline__ void fft_reg(float2 (&a)[R])
{
    static_assert((R & (R - 1)) == 0 && R >= 1, "radix-2 codelet needs a power of two");
    if constexpr (R == 1) {
        return;
    } else {
        float2 b[R];
        static_for<0, R>([&](auto i) { b[bit_reverse<R>(decltype(i)::value)] = a[i]; });
        static_for<1, ilog2(R) + 1>([&](auto s) {
            constexpr int len = 1 << decltype(s)::value;
            constexpr int half = len / 2;
            static_for<0, R, len>([&](auto g) {
                static_for<0, half>([&](auto jj) {
                    constexpr int lo = decltype(g)::value + decltype(jj)::value;
                    const float2 u = b[lo];
                    const float2 w = twiddle_const<len, decltype(jj)::value, INV>(b[lo + half]);
                    b[lo] = cadd(u, w);
                    b[lo + half] = csub(u, w);
                });
            });
        });
        static_for<0, R>([&](auto i) { a[i] = b[i]; });
    }
}

}  // namespace vbw

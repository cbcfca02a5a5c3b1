/*
 * FP64 CPU oracle for overlap-save (OLS) variable-bandwidth (VBW) filtering whose DFT
 * coefficients come from the hybrid frequency-sampling / optimization (HFSO) rule of
 * Moryakova & Johansson, "Efficient Design and Implementation of Fast-Convolution-Based
 * Variable-Bandwidth Filters".
 *
 * THIS IS TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it. It shares no code, header, table or constant with the CUDA path, and the
 * CUDA path never calls it.
 *
 * It is deliberately plain and slow: a direct O(N^2) DFT per block in double precision, the
 * coefficient H(k) built with the literal complex exponential of eq. (FS_Hk_exp), and the five
 * OLS steps of Sec. II taken in order.
 *
 * Conventions (readings of the paper, stated once here):
 *   overlap O = N - M = L - 1 (Sec. II, L = N - M + 1); the delay (L-1)/2 = O/2 is a whole
 *   sample count for even O and a half sample for odd O. The phase of eq. (FS_Hk_exp) takes the
 *   signed bin index k_s (k for k <= N/2, k - N above), which keeps H conjugate symmetric and the
 *   impulse response real for odd O too; for even O it equals the unsigned form exactly.
 *   band = k1(b): bins 0..k1-1 are passband; k2 = k1 + L_V - 1 (eq. (k_var), L_V = Delta_N - 1).
 *   Upper-side transition bins use V(N - k - k1) (the real-impulse-response reading of
 *   eq. (FS_Hk_real); it is the one the cosine form of d_{M-1}(q,b) in Sec. III-B implies).
 *   Stream alignment: O zero samples (or the caller's tail) precede x(0), so block m covers
 *   x(mM - O .. mM + M - 1) and writes y(mM .. mM + M - 1); the final partial block is zero
 *   padded and only its valid outputs are written.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define VBWO_PI 3.14159265358979323846264338327950288

/* H_R(k,b) of eq. (FS_Hk_real) for k = 0..N-1, with the regions k_p, k_t, k_s of Sec. III-B
 * written out as the paper lists them. V holds the L_V transition samples V(0..L_V-1).
 * Returns 0, or -1 if the arguments are outside the ranges the paper states
 * (Delta_N/2 <= b_N <= N/2 - Delta_N/2 - 1, i.e. 1 <= k1 and k2 <= N/2 - 2). */
int vbwo_HR(int N, int LV, const float* V, int k1, double* HR)
{
    if (N < 4 || (N & 1) || LV < 1 || k1 < 1) return -1;
    const int k2 = k1 + LV - 1;
    if (k2 > N / 2 - 2) return -1;
    for (int k = 0; k < N; ++k) {
        double v;
        if (k <= k1 - 1 || k >= N - k1 + 1) {            /* k_p(b) */
            v = 1.0;
        } else if (k >= k1 && k <= k2) {                 /* lower part of k_t(b) */
            v = (double)V[k - k1];
        } else if (k >= N - k2 && k <= N - k1) {         /* upper (mirror) part of k_t(b) */
            v = (double)V[N - k - k1];
        } else {                                         /* k_s(b) = [k2+1, N-k2-1] */
            v = 0.0;
        }
        HR[k] = v;
    }
    return 0;
}

/* H(k,b) = H_R(k,b) * exp(-j 2 pi k ((L-1)/2) / N), eq. (FS_Hk_exp), with (L-1)/2 = O/2.
 * The product k*(O/2) is reduced mod N in integers before the angle is formed, so the angle
 * is exact up to one rounding of 2*pi*j/N. H is written as interleaved (re, im) pairs. */
int vbwo_H(int N, int O, int LV, const float* V, int k1, double* H)
{
    if (O <= 0 || O >= N) return -1;
    double* HR = (double*)malloc(sizeof(double) * (size_t)N);
    if (!HR) return -1;
    if (vbwo_HR(N, LV, V, k1, HR) != 0) { free(HR); return -1; }
    /* exp(-j 2 pi k_s (O/2) / N) = exp(-j pi (k_s O mod 2N) / N), reduced exactly in integers */
    for (int k = 0; k < N; ++k) {
        const int64_t ks = k <= N / 2 ? k : (int64_t)k - N;
        const int64_t j = (((ks * O) % (2 * (int64_t)N)) + 2 * (int64_t)N) % (2 * (int64_t)N);
        const double ang = -VBWO_PI * (double)j / (double)N;
        H[2 * k] = HR[k] * cos(ang);
        H[2 * k + 1] = HR[k] * sin(ang);
    }
    free(HR);
    return 0;
}

/* Table c[j] = exp(sign * j 2 pi j / N), j = 0..N-1, used with exact index reduction. */
static void unit_roots(int N, int sign, double complex* c)
{
    for (int j = 0; j < N; ++j) {
        const double ang = 2.0 * VBWO_PI * (double)j / (double)N;
        c[j] = cos(ang) + (double)sign * I * sin(ang);
    }
}

/* Direct DFT: out(k) = sum_n in(n) exp(sign * j 2 pi n k / N), no scaling (Sec. II step 1 with
 * sign = -1; step 3 / eq. (OLS_dn) uses sign = +1 followed by 1/N). */
static void direct_dft(int N, const double complex* roots, const double complex* in, double complex* out)
{
    for (int k = 0; k < N; ++k) {
        double complex acc = 0.0;
        for (int n = 0; n < N; ++n) {
            const int64_t idx = ((int64_t)n * (int64_t)k) % N;
            acc += in[n] * roots[idx];
        }
        out[k] = acc;
    }
}

/* Exported direct DFT on interleaved (re, im) doubles. sign = -1 forward, +1 inverse (no 1/N). */
int vbwo_dft(int N, const double* x, double* X, int sign)
{
    if (N < 1 || (sign != 1 && sign != -1)) return -1;
    double complex* roots = (double complex*)malloc(sizeof(double complex) * (size_t)N);
    double complex* in = (double complex*)malloc(sizeof(double complex) * (size_t)N);
    double complex* out = (double complex*)malloc(sizeof(double complex) * (size_t)N);
    if (!roots || !in || !out) { free(roots); free(in); free(out); return -1; }
    unit_roots(N, sign, roots);
    for (int n = 0; n < N; ++n) in[n] = x[2 * n] + I * x[2 * n + 1];
    direct_dft(N, roots, in, out);
    for (int k = 0; k < N; ++k) { X[2 * k] = creal(out[k]); X[2 * k + 1] = cimag(out[k]); }
    free(roots); free(in); free(out);
    return 0;
}

/* One OLS block m (Sec. II steps 1-4) with coefficients H (N complex). x: T complex64 samples as
 * interleaved floats; tail: O complex64 samples that precede x(0) (NULL means zeros). Writes
 * y(mM + i) for i in [0, M) with mM + i < T, as interleaved doubles. */
static void ols_block(int N, int O, const double complex* H, const double complex* fwd,
                      const double complex* inv, const float* x, int64_t T, const float* tail,
                      int64_t m, double* y, double complex* work)
{
    const int M = N - O;
    double complex* xb = work;
    double complex* X = work + N;
    double complex* z = work + 2 * N;
    /* segment x_m(i) = x(mM - O + i), i = 0..N-1 (Sec. II, with the O-sample prefix) */
    for (int i = 0; i < N; ++i) {
        const int64_t s = m * (int64_t)M - O + i;
        double re = 0.0, im = 0.0;
        if (s < 0) {
            if (tail) { re = tail[2 * (O + s)]; im = tail[2 * (O + s) + 1]; }
        } else if (s < T) {
            re = x[2 * s]; im = x[2 * s + 1];
        }
        xb[i] = re + I * im;
    }
    direct_dft(N, fwd, xb, X);                         /* step 1: N-point DFT */
    for (int k = 0; k < N; ++k) X[k] *= H[k];          /* step 2: multiply by H(k) */
    direct_dft(N, inv, X, z);                          /* step 3: N-point IDFT ... */
    for (int n = 0; n < N; ++n) z[n] /= (double)N;     /* ... with the 1/N of eq. (OLS_dn) */
    for (int i = 0; i < M; ++i) {                      /* steps 4-5: discard O, keep M */
        const int64_t t = m * (int64_t)M + i;
        if (t >= T) break;
        y[2 * t] = creal(z[O + i]);
        y[2 * t + 1] = cimag(z[O + i]);
    }
}

static int check_geometry(int N, int O)
{
    return (N >= 2 && O >= 0 && O < N) ? 0 : -1;
}

/* OLS filtering of blocks [b0, b0 + nb) of a stream of T samples with one fixed complex H for
 * every block (H: 2N interleaved doubles). Used for the identity and hand-made-H checks. */
int vbwo_filter_H(int N, int O, const double* Hri, const float* x, int64_t T, const float* tail,
                  int64_t b0, int64_t nb, double* y, int nthreads)
{
    if (check_geometry(N, O) != 0 || T < 0 || b0 < 0 || nb < 0) return -1;
    const int M = N - O;
    const int64_t nblocks = (T + M - 1) / M;
    if (b0 + nb > nblocks) nb = nblocks > b0 ? nblocks - b0 : 0;
    double complex* H = (double complex*)malloc(sizeof(double complex) * (size_t)N);
    double complex* fwd = (double complex*)malloc(sizeof(double complex) * (size_t)N);
    double complex* inv = (double complex*)malloc(sizeof(double complex) * (size_t)N);
    if (!H || !fwd || !inv) { free(H); free(fwd); free(inv); return -1; }
    for (int k = 0; k < N; ++k) H[k] = Hri[2 * k] + I * Hri[2 * k + 1];
    unit_roots(N, -1, fwd);
    unit_roots(N, +1, inv);
    int err = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        double complex* work = (double complex*)malloc(sizeof(double complex) * 3 * (size_t)N);
        if (!work) {
#pragma omp atomic write
            err = -1;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int64_t m = b0; m < b0 + nb; ++m)
                ols_block(N, O, H, fwd, inv, x, T, tail, m, y, work);
            free(work);
        }
    }
    free(H); free(fwd); free(inv);
    return err;
}

/* OLS VBW filtering of blocks [b0, b0 + nb) of a stream of T samples. band[m] is k1 for block m
 * (m indexes the whole stream, so band has ceil(T/M) entries); H(k, band[m]) is rebuilt from
 * eq. (FS_Hk_exp)/(FS_Hk_real) for every block, exactly as the definition reads. */
int vbwo_filter(int N, int O, int LV, const float* V, const int32_t* band, const float* x,
                int64_t T, const float* tail, int64_t b0, int64_t nb, double* y, int nthreads)
{
    if (check_geometry(N, O) != 0 || O == 0 || T < 0 || b0 < 0 || nb < 0) return -1;
    const int M = N - O;
    const int64_t nblocks = (T + M - 1) / M;
    if (b0 + nb > nblocks) nb = nblocks > b0 ? nblocks - b0 : 0;
    for (int64_t m = b0; m < b0 + nb; ++m) {
        const int k1 = band[m];
        if (k1 < 1 || k1 + LV - 1 > N / 2 - 2) return -2;
    }
    double complex* fwd = (double complex*)malloc(sizeof(double complex) * (size_t)N);
    double complex* inv = (double complex*)malloc(sizeof(double complex) * (size_t)N);
    if (!fwd || !inv) { free(fwd); free(inv); return -1; }
    unit_roots(N, -1, fwd);
    unit_roots(N, +1, inv);
    int err = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        double complex* work = (double complex*)malloc(sizeof(double complex) * 3 * (size_t)N);
        double complex* H = (double complex*)malloc(sizeof(double complex) * (size_t)N);
        double* Hri = (double*)malloc(sizeof(double) * 2 * (size_t)N);
        if (!work || !H || !Hri) {
#pragma omp atomic write
            err = -1;
        } else {
#pragma omp for schedule(dynamic, 4)
            for (int64_t m = b0; m < b0 + nb; ++m) {
                vbwo_H(N, O, LV, V, band[m], Hri);
                for (int k = 0; k < N; ++k) H[k] = Hri[2 * k] + I * Hri[2 * k + 1];
                ols_block(N, O, H, fwd, inv, x, T, tail, m, y, work);
            }
        }
        free(work); free(H); free(Hri);
    }
    free(fwd); free(inv);
    return err;
}

/* Number of OpenMP threads a parallel region would use by default (for reporting). */
int vbwo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* PTVIR view of OLS (Sec. II, eq. (OLS_Hn)): output phase n = 0..M-1 of every block is a
 * time-invariant filter. Written out from the OLS definition (Sec. II steps 1-5 with
 * h = IDFT(H) of eq. (OLS_dn)): output sample mM + n is sample O + n of the circular convolution
 * of the block with h, so tap q reaches the input q samples back when q <= n + O and, through the
 * circular wrap, N - q samples ahead otherwise. Its response is
 *     H_n(w) = sum_q h(q) exp(-j w s_n(q)),   s_n(q) = q (q <= n + O),  q - N (q > n + O).
 * The error of eq. (err_min) against the desired response of eq. (VBW_des) with its delay
 * (L-1)/2 = O/2 removed is E_n(w) = H_n(w) exp(j w O/2) - d.
 * h: N complex values, interleaved (re, im). omega, d: K grid points and desired values.
 * Writes |E_n(w_i)| to E[n * K + i] for n = 0..M-1, i = 0..K-1. Every exponential is evaluated
 * directly from its angle, one (n, i) pair at a time. */
int vbwo_ptvir(int N, int O, const double* h, const double* omega, const double* d, int K,
               double* E, int nthreads)
{
    if (check_geometry(N, O) != 0 || K < 0) return -1;
    const int M = N - O;
    const double D = 0.5 * (double)O;
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int n = 0; n < M; ++n) {
        for (int i = 0; i < K; ++i) {
            const double w = omega[i];
            double complex Hn = 0.0;
            for (int q = 0; q < N; ++q) {
                const double s = (q <= n + O) ? (double)q : (double)q - (double)N;
                const double ang = -w * s;
                Hn += (h[2 * q] + I * h[2 * q + 1]) * (cos(ang) + I * sin(ang));
            }
            const double complex e = Hn * (cos(w * D) + I * sin(w * D)) - d[i];
            E[(size_t)n * (size_t)K + (size_t)i] = cabs(e);
        }
    }
    return 0;
}

/* Overlap-add (OLA) fast convolution, the FC method the paper names beside OLS (Sec. I): the
 * input is cut into non-overlapping blocks u_m(i) = x(mM + i), i = 0..M-1, each zero padded to N
 * samples; each block goes through the same steps 1-3 of Sec. II (N-point DFT, multiply by H(k),
 * N-point IDFT with 1/N); the N-sample results overlap by N - M = O samples and are added:
 *     y(t) = sum_m z_m(t - mM),  0 <= t - mM < N.
 * Samples past the end of x are zero; y is written for t = 0..T-1. band[m] is k1 of block m and
 * H(k, band[m]) is built as in vbwo_filter (eq. (FS_Hk_exp)/(FS_Hk_real)). Sequential over
 * blocks (the additions of overlapping blocks are done in block order). */
/* One OLA block m with coefficients H (N complex): adds z_m(n) to y(mM + n) for mM + n < T. */
static void ola_block(int N, int O, const double complex* H, const double complex* fwd,
                      const double complex* inv, const float* x, int64_t T, int64_t m, double* y,
                      double complex* work)
{
    const int M = N - O;
    double complex* u = work;
    double complex* X = work + N;
    double complex* z = work + 2 * N;
    for (int i = 0; i < N; ++i) {                      /* u_m: M samples, zero padded */
        const int64_t s = m * (int64_t)M + i;
        u[i] = (i < M && s < T) ? (x[2 * s] + I * x[2 * s + 1]) : 0.0;
    }
    direct_dft(N, fwd, u, X);                          /* step 1 */
    for (int k = 0; k < N; ++k) X[k] *= H[k];          /* step 2 */
    direct_dft(N, inv, X, z);                          /* step 3 with 1/N */
    for (int n = 0; n < N; ++n) {                      /* overlap and add */
        const int64_t t = m * (int64_t)M + n;
        if (t >= T) break;
        y[2 * t] += creal(z[n]) / (double)N;
        y[2 * t + 1] += cimag(z[n]) / (double)N;
    }
}

static int ola_run(int N, int O, const double* Hfixed, int LV, const float* V, const int32_t* band,
                   const float* x, int64_t T, double* y)
{
    if (check_geometry(N, O) != 0 || O == 0 || T < 0) return -1;
    const int M = N - O;
    const int64_t nblocks = (T + M - 1) / M;
    if (!Hfixed) {
        for (int64_t m = 0; m < nblocks; ++m) {
            const int k1 = band[m];
            if (k1 < 1 || k1 + LV - 1 > N / 2 - 2) return -2;
        }
    }
    double complex* fwd = (double complex*)malloc(sizeof(double complex) * (size_t)N);
    double complex* inv = (double complex*)malloc(sizeof(double complex) * (size_t)N);
    double complex* work = (double complex*)malloc(sizeof(double complex) * 3 * (size_t)N);
    double complex* H = (double complex*)malloc(sizeof(double complex) * (size_t)N);
    double* Hri = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    if (!fwd || !inv || !work || !H || !Hri) {
        free(fwd); free(inv); free(work); free(H); free(Hri);
        return -1;
    }
    unit_roots(N, -1, fwd);
    unit_roots(N, +1, inv);
    for (int64_t t = 0; t < 2 * T; ++t) y[t] = 0.0;
    for (int64_t m = 0; m < nblocks; ++m) {
        if (Hfixed) {
            for (int k = 0; k < N; ++k) H[k] = Hfixed[2 * k] + I * Hfixed[2 * k + 1];
        } else {
            vbwo_H(N, O, LV, V, band[m], Hri);
            for (int k = 0; k < N; ++k) H[k] = Hri[2 * k] + I * Hri[2 * k + 1];
        }
        ola_block(N, O, H, fwd, inv, x, T, m, y, work);
    }
    free(fwd); free(inv); free(work); free(H); free(Hri);
    return 0;
}

/* OLA with the VBW coefficients H(k, band[m]) of eq. (FS_Hk_exp)/(FS_Hk_real) for block m. */
int vbwo_filter_ola(int N, int O, int LV, const float* V, const int32_t* band, const float* x,
                    int64_t T, double* y)
{
    return ola_run(N, O, NULL, LV, V, band, x, T, y);
}

/* OLA with one fixed complex H (2N interleaved doubles) for every block. */
int vbwo_filter_ola_H(int N, int O, const double* Hri, const float* x, int64_t T, double* y)
{
    return ola_run(N, O, Hri, 0, NULL, NULL, x, T, y);
}

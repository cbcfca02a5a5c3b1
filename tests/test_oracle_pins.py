"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each check is independent of the oracle's own formulation (frequency-domain regions, direct DFT,
literal exponential): the cosine closed form of d_{M-1}(q,b) (Sec. III-B), time-domain circular
and linear convolution, exactly representable tones, numpy's FFT, and hand-built spectra.
A dropped term, a wrong sign or index, a missing 1/N or a transposed region fails one of them.
"""
import numpy as np
import pytest

import oracle
from paper_2406_14116_gb300 import workloads as wl


def closed_form_h(N, overlap, V, k1):
    """d_{M-1}(q,b) of Sec. III-B: (1/N)[1 + 2 sum_{k=1}^{k1-1} cos(2 pi k (q - (L-1)/2)/N)
    + 2 sum_{k=k1}^{k2} V(k-k1) cos(2 pi k (q - (L-1)/2)/N)], with L - 1 = overlap."""
    V32 = np.asarray(V, dtype=np.float32).astype(np.float64)
    q = np.arange(N, dtype=np.float64)
    D = overlap / 2.0
    acc = np.ones(N)
    for k in range(1, k1):
        acc += 2.0 * np.cos(2.0 * np.pi * k * (q - D) / N)
    for r, v in enumerate(V32):
        k = k1 + r
        acc += 2.0 * v * np.cos(2.0 * np.pi * k * (q - D) / N)
    return acc / N


def segments(x, N, overlap, tail=None):
    """x_m(i) = x(mM - O + i) with the O-sample prefix (tail or zeros) and zero padding."""
    M = N - overlap
    T = len(x)
    nb = (T + M - 1) // M
    pre = np.zeros(overlap, np.complex128) if tail is None else np.asarray(tail, np.complex128)
    ext = np.concatenate([pre, np.asarray(x, np.complex128), np.zeros(N, np.complex128)])
    return np.stack([ext[m * M: m * M + N] for m in range(nb)])


def rand_c64(g, n):
    return (g.standard_normal(n) + 1j * g.standard_normal(n)).astype(np.complex64)


CASES = [
    # N, overlap, LV, k1
    (8, 2, 1, 1), (8, 4, 1, 2), (16, 4, 2, 3), (16, 6, 3, 1), (32, 8, 4, 5),
    (32, 10, 6, 9), (32, 16, 2, 13), (32, 30, 3, 4),
    # odd overlap: half-sample delay O/2 with the signed-bin phase of eq. (FS_Hk_exp)
    (16, 5, 2, 3), (32, 9, 4, 5), (32, 15, 3, 7),
]


@pytest.mark.parametrize("N,overlap,LV,k1", CASES)
def test_brute_force_circular_convolution(N, overlap, LV, k1):
    """OLS block output = circular convolution of the segment with h = d_{M-1} (eq. OLS_dn),
    h taken from the paper's cosine closed form, then discard O and concatenate (Sec. II)."""
    g = np.random.default_rng(N * 1000 + overlap * 10 + k1)
    M = N - overlap
    V = np.sort(g.uniform(0.05, 1.0, LV))[::-1]
    T = 5 * M + M // 2 + 1
    x = rand_c64(g, T)
    tail = rand_c64(g, overlap)
    nb = (T + M - 1) // M
    bands = g.integers(1, N // 2 - LV, size=nb).astype(np.int32)
    y = oracle.filter(N, overlap, V, bands, x, tail=tail, nthreads=2)
    seg = segments(x, N, overlap, tail)
    ref = np.zeros(T, np.complex128)
    for m in range(nb):
        h = closed_form_h(N, overlap, V, int(bands[m]))
        for n in range(M):
            t = m * M + n
            if t >= T:
                break
            ref[t] = sum(h[q] * seg[m][(overlap + n - q) % N] for q in range(N))
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("N,overlap,LV,k1", [(64, 16, 5, 7), (128, 32, 15, 41), (128, 32, 15, 48),
                                             (256, 64, 6, 60), (256, 64, 12, 115),
                                             (64, 15, 5, 7), (128, 33, 15, 41), (256, 63, 12, 100)])
def test_H_inverse_dft_is_closed_form(N, overlap, LV, k1):
    """IDFT of the oracle's H(k,b) (numpy's inverse FFT) equals the real cosine sum of
    Sec. III-B: pins the regions, the mirror reading of the upper transition band and the sign of
    the linear phase."""
    g = np.random.default_rng(N + k1)
    V = np.sort(g.uniform(0, 1, LV))[::-1]
    h = np.fft.ifft(oracle.H(N, overlap, V, k1))
    ref = closed_form_h(N, overlap, V, k1)
    np.testing.assert_allclose(h.real, ref, rtol=0, atol=1e-15 * N)
    np.testing.assert_allclose(h.imag, 0.0, rtol=0, atol=1e-15 * N)


@pytest.mark.parametrize("N,overlap,LV", [(32, 8, 3), (64, 16, 6), (128, 32, 15), (256, 64, 12),
                                          (32, 7, 3), (128, 33, 15)])
def test_last_kept_sample_is_linear_fir(N, overlap, LV):
    """d_{M-1} = IDFT(H) (eq. OLS_dn): the last kept sample of each block equals the linear
    convolution sum_q h(q) x(t - q), t = mM + M - 1, with h the closed form."""
    g = np.random.default_rng(7 * N)
    M = N - overlap
    V = np.sort(g.uniform(0, 1, LV))[::-1]
    k1 = int(g.integers(1, N // 2 - LV))
    T = 9 * M
    x = rand_c64(g, T)
    y = oracle.filter(N, overlap, V, k1, x, nthreads=2)
    h = closed_form_h(N, overlap, V, k1)
    lin = np.convolve(x.astype(np.complex128), h)[:T]
    idx = np.arange(M - 1, T, M)
    np.testing.assert_allclose(y[idx], lin[idx], rtol=0, atol=1e-12)
    # every other position differs in general (the LPTV aliasing of Sec. II)
    other = np.setdiff1d(np.arange(N, T), idx)
    assert np.abs(y[other] - lin[other]).max() > 1e-6


@pytest.mark.parametrize("N,overlap", [(8, 2), (16, 4), (128, 32), (1024, 256)])
def test_identity_filter_returns_input(N, overlap):
    """H(k) = 1 for every k: the discarded-prefix output is the input itself."""
    g = np.random.default_rng(N)
    M = N - overlap
    T = 3 * M + 5
    x = rand_c64(g, T)
    y = oracle.filter_H(N, overlap, np.ones(N), x, nthreads=2)
    np.testing.assert_allclose(y, x.astype(np.complex128), rtol=0, atol=1e-12)


@pytest.mark.parametrize("N,overlap", [(16, 4), (64, 16), (256, 64), (512, 128)])
def test_full_band_is_pure_delay(N, overlap):
    """H_R = 1 everywhere with the linear phase of eq. (FS_Hk_exp): y(t) = x(t - (L-1)/2)."""
    g = np.random.default_rng(N + 1)
    M = N - overlap
    D = overlap // 2
    T = 4 * M + 3
    x = rand_c64(g, T)
    k = np.arange(N)
    Hfull = np.exp(-2j * np.pi * k * D / N)
    y = oracle.filter_H(N, overlap, Hfull, x, nthreads=2)
    ref = np.concatenate([np.zeros(D), x.astype(np.complex128)])[:T]
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N", [8, 16, 128, 1024])
def test_dft_against_numpy_and_parseval(N):
    g = np.random.default_rng(N)
    x = g.standard_normal(N) + 1j * g.standard_normal(N)
    X = oracle.dft(x, -1)
    np.testing.assert_allclose(X, np.fft.fft(x), rtol=0, atol=1e-11 * N)
    np.testing.assert_allclose(np.sum(np.abs(x) ** 2), np.sum(np.abs(X) ** 2) / N, rtol=1e-13)
    np.testing.assert_allclose(oracle.dft(X, +1) / N, x, rtol=0, atol=1e-13 * N)


def test_linearity_exact_inputs():
    """filter(a x1 + b x2) = a filter(x1) + b filter(x2) with inputs exactly representable in
    complex64 (small integers), so no input rounding enters."""
    N, overlap, LV = 64, 16, 5
    g = np.random.default_rng(3)
    M = N - overlap
    T = 6 * M + 7
    V = np.sort(g.uniform(0, 1, LV))[::-1]
    x1 = (g.integers(-8, 9, T) + 1j * g.integers(-8, 9, T)).astype(np.complex64)
    x2 = (g.integers(-8, 9, T) + 1j * g.integers(-8, 9, T)).astype(np.complex64)
    a, b = 3.0, -2.0j
    mix = (a * x1.astype(np.complex128) + b * x2.astype(np.complex128)).astype(np.complex64)
    bands = g.integers(1, N // 2 - LV, size=(T + M - 1) // M).astype(np.int32)
    y = oracle.filter(N, overlap, V, bands, mix, nthreads=2)
    ref = a * oracle.filter(N, overlap, V, bands, x1, nthreads=2) + \
        b * oracle.filter(N, overlap, V, bands, x2, nthreads=2)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-11)


def exact_tone(N, k0, T):
    """exp(j 2 pi k0 t / N) for k0 a multiple of N/4: values in {1, j, -1, -j}, exact."""
    assert (4 * k0) % N == 0
    q = (np.arange(T) * (4 * k0 // N)) % 4
    return np.array([1, 1j, -1, -1j], dtype=np.complex64)[q]


@pytest.mark.parametrize("N,overlap,LV", [(32, 8, 3), (64, 16, 6), (128, 32, 15)])
def test_tones_pass_scale_and_stop(N, overlap, LV):
    """A tone at bin k0 that is whole in every segment comes out as H(k0) times the tone:
    k0 = 0 and N/4 in the passband -> delayed copy; N/4 (and its mirror 3N/4) in the transition
    band -> V(r) times the delayed tone with r = N/4 - k1; N/4 and N/2 in the stopband -> 0."""
    M = N - overlap
    D = overlap // 2
    g = np.random.default_rng(N)
    V = np.sort(g.uniform(0.05, 1, LV))[::-1]
    V32 = V.astype(np.float32).astype(np.float64)
    T = 8 * M
    steady = np.arange(N, T)          # every block after the first sees a whole tone
    for k0 in (0, N // 4, 3 * N // 4, N // 2):
        x = exact_tone(N, k0, T)
        delayed = np.concatenate([np.zeros(D, np.complex64), x])[:T]
        kk = min(k0, N - k0)
        for k1 in (1, kk - LV + 1, kk - 2, kk, kk + 1, N // 2 - LV - 1):
            if k1 < 1 or k1 > N // 2 - LV - 1:
                continue
            y = oracle.filter(N, overlap, V, k1, x, nthreads=2)
            if kk <= k1 - 1:
                want = 1.0
            elif kk <= k1 + LV - 1:
                want = V32[kk - k1]
            else:
                want = 0.0
            np.testing.assert_allclose(y[steady], want * delayed[steady].astype(np.complex128),
                                       rtol=0, atol=1e-12)


def test_tail_prefix_and_stream_split():
    """Filtering a stream in two calls, the second with the first call's last O input samples as
    its prefix, equals filtering it in one call (OLS continuity, Sec. II)."""
    N, overlap, LV = 64, 16, 4
    M = N - overlap
    g = np.random.default_rng(11)
    V = np.sort(g.uniform(0, 1, LV))[::-1]
    T = 10 * M
    x = rand_c64(g, T)
    bands = g.integers(1, N // 2 - LV, size=T // M).astype(np.int32)
    y = oracle.filter(N, overlap, V, bands, x, nthreads=2)
    cut = 4 * M
    y1 = oracle.filter(N, overlap, V, bands[:4], x[:cut], nthreads=2)
    y2 = oracle.filter(N, overlap, V, bands[4:], x[cut:], tail=x[cut - overlap:cut], nthreads=2)
    np.testing.assert_array_equal(np.concatenate([y1, y2]), y)


def test_block_subset_matches_full_run():
    N, overlap = 128, 32
    M = N - overlap
    g = np.random.default_rng(5)
    V = np.sort(g.uniform(0, 1, 12))[::-1]
    x = rand_c64(g, 20 * M + 17)
    full = oracle.filter(N, overlap, V, 30, x, nthreads=2)
    part = oracle.filter(N, overlap, V, 30, x, blocks=(7, 3), nthreads=2)
    sl = slice(7 * M, 10 * M)
    np.testing.assert_array_equal(part[sl], full[sl])
    assert np.isnan(part[: 7 * M]).all() and np.isnan(part[10 * M:]).all()


def test_band_range_matches_paper_bounds():
    """eq. (k_var): Delta_N/2 <= b_N <= N/2 - Delta_N/2 - 1 with k1 = b_N - Delta_N/2 + 1 and
    L_V = Delta_N - 1, i.e. 1 <= k1 <= N/2 - L_V - 1."""
    V = np.linspace(0.9, 0.1, 15)
    for N in (64, 128, 1024):
        kmax = wl.max_band(N, 15)
        oracle.HR(N, V, 1)
        oracle.HR(N, V, kmax)
        for bad in (0, kmax + 1):
            with pytest.raises(ValueError):
                oracle.HR(N, V, bad)


def test_HR_region_sizes():
    """|k_p| = 2 k1 - 1, |k_t| = 2 L_V, |k_s| = N - 2 k2 - 1 (eq. FS_Hk_real regions)."""
    N, LV = 256, 12
    V = np.linspace(0.95, 0.05, LV)
    for k1 in (1, 17, 60, wl.max_band(N, LV)):
        hr = oracle.HR(N, V, k1)
        k2 = k1 + LV - 1
        assert np.count_nonzero(hr == 1.0) == 2 * k1 - 1
        assert np.count_nonzero(hr == 0.0) == N - 2 * k2 - 1
        assert np.count_nonzero((hr > 0) & (hr < 1)) == 2 * LV
        np.testing.assert_array_equal(hr[1:], hr[1:][::-1])    # H_R(N - k) = H_R(k)

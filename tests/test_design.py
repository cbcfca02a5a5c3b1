"""The HFSO minimax designer (paper_2406_14116_gb300/design.py), CPU only.

Pins: the per-phase responses H_n it optimizes equal what the OLS definition (the FP64 oracle)
does to a complex exponential at each output phase; the order and N estimates give the paper's
printed values (Sec. IV); the paper's example (N=128, L=33, M=96, Delta_N=16, b_N in [48, 55],
K=1000) meets the paper's -60 dB (delta <= 0.001)."""
import math

import numpy as np
import pytest

import oracle
from paper_2406_14116_gb300 import design


def test_order_and_size_estimates_match_the_example():
    # Sec. IV: Delta = 0.25 pi, delta_p = delta_s = 0.001 give N_D = 28 (the estimate, 26.7,
    # rounded up to an even order) and N = 127 -> 128
    nd = design.order_estimate(1e-3, 1e-3, 0.25 * math.pi)
    assert nd == pytest.approx(80.0 / 3.0)
    assert design.choose_N(28 + 1) == 128
    assert 0.9 * 29 * math.log2(29) == pytest.approx(126.8, abs=0.05)
    # bins of the example: Delta_N = 16, b in [0.75 pi, 0.8594 pi] -> b_N in [48, 55]
    assert round(0.25 * math.pi * 128 / (2 * math.pi)) == 16
    assert (round(0.75 * 128 / 2), round(0.8594 * 128 / 2)) == (48, 55)
    assert design.band_bins(48, 16) == (41, 55) and design.band_bins(55, 16) == (48, 62)


@pytest.mark.parametrize("N,O,k1,LV", [(32, 8, 4, 5), (64, 16, 10, 7)])
def test_phase_responses_are_what_ols_does_to_a_tone(N, O, k1, LV):
    """y(mM + n) = H_n(w) e^{jw(mM+n)} for x(t) = e^{jwt}: the oracle's OLS output at each phase
    n of a middle block, divided by the input, equals the designer's response of phase n."""
    M = N - O
    L = O + 1
    g = np.random.default_rng(N)
    V = np.sort(g.uniform(0, 1, LV))[::-1].astype(np.float32).astype(np.float64)
    C = design.h_basis(N, L, k1, LV)
    w = np.array([0.3, 1.1, 2.9, np.pi * 2 * (k1 + 1) / N])
    F = design.phase_responses(C, N, L, w)                   # (M, K, LV + 1), delay D removed
    Hn = (F[:, :, 0] + F[:, :, 1:] @ V) * np.exp(-1j * w * O / 2)[None, :]
    T = 12 * M
    t = np.arange(T)
    m = 6
    for i, wi in enumerate(w):
        x = np.exp(1j * wi * t).astype(np.complex64)         # complex64 exact enough: compare to it
        y = oracle.filter(N, O, V, k1, x)
        xin = x.astype(np.complex128)
        for n in range(M):
            tt = m * M + n
            np.testing.assert_allclose(y[tt] / xin[tt], Hn[n, i], rtol=0, atol=1e-5)


def test_h_basis_is_the_idft_of_the_hfso_coefficients():
    """Column algebra of the cosine form: C [1, V] = IDFT(H) with H from eq. (FS_Hk_exp)."""
    N, O, k1, LV = 64, 16, 9, 6
    V = np.linspace(0.9, 0.1, LV).astype(np.float32).astype(np.float64)
    h = design.h_basis(N, O + 1, k1, LV) @ np.concatenate([[1.0], V])
    H = oracle.H(N, O, V, k1)
    np.testing.assert_allclose(h, np.fft.ifft(H).real, atol=1e-14)
    np.testing.assert_allclose(np.fft.ifft(H).imag, 0, atol=1e-14)


def test_paper_example_meets_minus_60_db():
    d = design.design_transition(128, 33, 16, 48, 55, K=1000)
    assert d.M == 96 and len(d.V) == 15
    assert d.delta <= 1e-3                       # the paper: every response below -60 dB
    assert np.all(np.diff(d.V) < 0) and 0 < d.V[-1] and d.V[0] < 1


def test_design_procedure_meets_the_specification():
    d = design.design_procedure(0.25 * math.pi, 1e-3, 0.75 * math.pi, 0.8594 * math.pi)
    assert d.N == 128 and d.delta <= 1e-3 and d.bN == (48, 55)
    assert d.L <= 33
    # one order lower than the returned one fails the specification
    lower = design.design_transition(d.N, d.L - 2, d.Delta_N, *d.bN)
    assert lower.delta > 1e-3


def test_candidate_rows_equal_the_full_responses():
    """The GPU-search designer builds LP rows only at the points the GPU reports; those rows must
    be the full error system's rows at the same (band, phase, frequency)."""
    N, L, LV = 64, 17, 6
    M = N - L + 1
    g = np.random.default_rng(3)
    for k1 in (3, 12):
        w = g.uniform(0, np.pi, 7)
        d = (g.uniform(0, 1, 7) < 0.5).astype(float)
        F = design.phase_responses(design.h_basis(N, L, k1, LV), N, L, w)   # (M, K, LV + 1)
        n = g.integers(0, M, 20)
        i = g.integers(0, 7, 20)
        A, c = design.candidate_rows(N, L, LV, np.full(20, k1), n, w[i], d[i])
        np.testing.assert_allclose(A, F[n, i, 1:], atol=1e-14)
        np.testing.assert_allclose(c, F[n, i, 0] - d[i], atol=1e-14)


def test_candidate_rows_match_the_oracle_ptvir_errors():
    """|A V + c| at (band, phase, frequency) points equals the oracle's PTVIR error there
    (eq. (OLS_Hn), eq. (err_min), from the OLS definition), for float32-exact V."""
    N, L, LV = 64, 17, 5
    O = L - 1
    g = np.random.default_rng(9)
    V = np.sort(g.uniform(0, 1, LV))[::-1].astype(np.float32).astype(np.float64)
    for k1 in (2, 9, 64 // 2 - LV - 1):
        w = g.uniform(0, np.pi, 9)
        d = (g.uniform(0, 1, 9) < 0.5).astype(float)
        E = oracle.ptvir_errors(N, O, V, k1, w, d)                      # (M, K)
        n = g.integers(0, N - O, 25)
        i = g.integers(0, 9, 25)
        A, c = design.candidate_rows(N, L, LV, np.full(25, k1), n, w[i], d[i])
        np.testing.assert_allclose(np.abs(A @ V + c), E[n, i], atol=1e-12)

"""Pins of the oracle's PTVIR errors (eq. (OLS_Hn), eq. (err_min)) against what the OLS
definition and the mathematics fix (CPU only).

* Tones through the OLS oracle: output phase n of an interior block is H_n(w) times the input
  (exact at the quarter-turn frequencies, whose complex64 samples are exact).
* An impulse response of length L = O + 1 makes OLS time-invariant (Sec. II): every phase has
  the same response, numpy's DTFT of h.
* The last phase has no wrapped tap: its response is the DTFT of h = d_{M-1} (eq. (OLS_dn)).
* A single tap q0 > O shows where the wrap starts: phases n < q0 - O see it N samples ahead.
* At the DFT bins every phase sees H(k) itself (frequency sampling, Sec. III-B).
A dropped wrap term, a wrong boundary (q <= n + O), sign or delay fails one of them.
"""
import numpy as np
import pytest

import oracle


def dtft(h, omega, delay):
    """sum_q h(q) e^{-j w (q - delay)} by numpy (no oracle code)."""
    q = np.arange(len(h))
    return np.exp(-1j * np.outer(omega, q - delay)) @ np.asarray(h, np.complex128)


@pytest.mark.parametrize("N,overlap,k1,LV", [(32, 8, 5, 3), (64, 16, 9, 6), (64, 21, 7, 4)])
def test_tones_through_ols_give_the_phase_responses(N, overlap, k1, LV):
    """x(t) = e^{j w t} through oracle.filter: y(mM + n) / x(mM + n) = H_n(w) for interior
    blocks, so |ratio e^{j w O/2} - d| is the oracle's |E_n|."""
    M = N - overlap
    g = np.random.default_rng(N + overlap)
    V = np.sort(g.uniform(0.05, 1.0, LV))[::-1]
    T = 6 * M
    t = np.arange(T)
    # quarter turns are exact in complex64; the others carry the input's float32 rounding
    omegas = np.concatenate([[0.0, np.pi / 2, np.pi, -np.pi / 2], g.uniform(-np.pi, np.pi, 5)])
    d = g.uniform(0.0, 1.0, len(omegas))
    E = oracle.ptvir_errors(N, overlap, V, k1, omegas, d)
    for i, w in enumerate(omegas):
        x = np.exp(1j * w * t).astype(np.complex64)
        y = oracle.filter(N, overlap, V, k1, x)
        m = 3
        n = np.arange(M)
        ratio = y[m * M + n] / x[m * M + n].astype(np.complex128)
        got = np.abs(ratio * np.exp(1j * w * overlap / 2) - d[i])
        tol = 1e-12 if i < 4 else 2e-6
        assert np.abs(got - E[:, i]).max() <= tol, (w, np.abs(got - E[:, i]).max())


@pytest.mark.parametrize("N,overlap", [(32, 8), (64, 15), (128, 32)])
def test_fir_of_length_L_is_time_invariant(N, overlap):
    """h(q) = 0 for q > O: no tap wraps for any phase; every |E_n| equals |DTFT(h) - d|."""
    g = np.random.default_rng(overlap)
    h = np.zeros(N, np.complex128)
    h[: overlap + 1] = g.standard_normal(overlap + 1) + 1j * g.standard_normal(overlap + 1)
    omega = g.uniform(-np.pi, np.pi, 40)
    d = g.uniform(0, 1, 40)
    E = oracle.ptvir_errors_h(N, overlap, h, omega, d)
    ref = np.abs(dtft(h, omega, overlap / 2) - d)
    assert np.abs(E - ref[None, :]).max() <= 1e-12


@pytest.mark.parametrize("N,overlap", [(32, 8), (64, 16), (64, 9)])
def test_last_phase_is_the_dtft_of_h(N, overlap):
    """d_{M-1} = IDFT(H) (eq. (OLS_dn)): phase M - 1 has no wrapped tap, for any h of length N;
    the other phases differ from it (the LPTV aliasing)."""
    g = np.random.default_rng(N * overlap)
    h = g.standard_normal(N) + 1j * g.standard_normal(N)
    omega = g.uniform(-np.pi, np.pi, 30)
    E = oracle.ptvir_errors_h(N, overlap, h, omega, 0.0)
    ref = np.abs(dtft(h, omega, overlap / 2))
    assert np.abs(E[-1] - ref).max() <= 1e-11
    assert np.abs(E[0] - ref).max() > 1e-3


@pytest.mark.parametrize("N,overlap,q0", [(32, 8, 20), (32, 8, 31), (64, 17, 40)])
def test_single_wrapped_tap(N, overlap, q0):
    """h = delta(q - q0), q0 > O: phases n < q0 - O read the tap through the circular wrap
    (delay q0 - N), phases n >= q0 - O directly (delay q0)."""
    M = N - overlap
    h = np.zeros(N, np.complex128)
    h[q0] = 1.0
    omega = np.linspace(-3.0, 3.0, 25)
    d = 0.5
    E = oracle.ptvir_errors_h(N, overlap, h, omega, d)
    D = overlap / 2
    for n in range(M):
        delay = q0 - N if n < q0 - overlap else q0
        ref = np.abs(np.exp(-1j * omega * (delay - D)) - d)
        assert np.abs(E[n] - ref).max() <= 1e-12, n


@pytest.mark.parametrize("N,overlap,k1,LV", [(32, 8, 5, 3), (64, 16, 11, 5), (64, 13, 3, 2)])
def test_bins_see_the_sampled_response(N, overlap, k1, LV):
    """At w = 2 pi k / N every phase sees H(k): |E_n| = |H_R(k) - d| (eq. (FS_Hk_real); the
    linear phase of eq. (FS_Hk_exp) cancels the delay)."""
    g = np.random.default_rng(k1)
    V = g.uniform(0.05, 1.0, LV)
    k = np.arange(-N // 2 + 1, N // 2)
    omega = 2 * np.pi * k / N
    d = g.uniform(0, 1, len(k))
    E = oracle.ptvir_errors(N, overlap, V, k1, omega, d)
    HR = oracle.HR(N, V, k1)[k % N]
    assert np.abs(E - np.abs(HR - d)[None, :]).max() <= 1e-12

"""Pins of the oracle's overlap-add filtering (Sec. I / Sec. II: the other fast-convolution
method, with the same H(k) and steps 1-3 on zero-padded, non-overlapping blocks), CPU only.

* An impulse response of length L = O + 1 (the classical FC condition, Sec. II) makes OLA an
  exact linear convolution: numpy's convolve.
* H = 1 returns the input; H = exp(-j 2 pi k_s D / N) delays it by D = O/2 (eq. (FS_Hk_exp) with
  H_R = 1).
* The VBW filter: brute-force time-domain circular convolution of each zero-padded block with h
  from the paper's cosine closed form of d_{M-1}(q, b) (Sec. III-B), overlapped and added, with a
  band change between blocks.
A wrong overlap, a dropped block tail, a wrong block length or a wrong H fails one of them.
"""
import numpy as np
import pytest

import oracle
from test_oracle_pins import closed_form_h


def rand_c64(g, n):
    return (g.standard_normal(n) + 1j * g.standard_normal(n)).astype(np.complex64)


@pytest.mark.parametrize("N,overlap", [(16, 4), (32, 8), (32, 16), (64, 21), (128, 32)])
def test_fir_of_length_L_is_a_linear_convolution(N, overlap):
    g = np.random.default_rng(N + overlap)
    M = N - overlap
    h = g.standard_normal(overlap + 1) + 1j * g.standard_normal(overlap + 1)
    Hk = np.fft.fft(np.concatenate([h, np.zeros(N - overlap - 1)]))
    T = 7 * M + M // 3
    x = rand_c64(g, T)
    y = oracle.filter_ola_H(N, overlap, Hk, x)
    ref = np.convolve(x.astype(np.complex128), h)[:T]
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("N,overlap", [(16, 4), (64, 16), (64, 30)])
def test_identity_and_pure_delay(N, overlap):
    g = np.random.default_rng(N)
    x = rand_c64(g, 9 * (N - overlap) + 5)
    y = oracle.filter_ola_H(N, overlap, np.ones(N), x)
    assert np.abs(y - x).max() <= 1e-12
    D = overlap // 2
    k = np.arange(N)
    ks = np.where(k <= N // 2, k, k - N)
    y = oracle.filter_ola_H(N, overlap, np.exp(-2j * np.pi * ks * D / N), x)
    ref = np.concatenate([np.zeros(D), x[: len(x) - D]])
    assert np.abs(y - ref).max() <= 1e-12


@pytest.mark.parametrize("N,overlap,LV", [(16, 4, 2), (32, 8, 3), (32, 10, 5), (64, 16, 6)])
def test_vbw_ola_is_blockwise_circular_convolution_overlapped_and_added(N, overlap, LV):
    g = np.random.default_rng(10 * N + LV)
    M = N - overlap
    V = np.sort(g.uniform(0.05, 1.0, LV))[::-1]
    T = 6 * M + M // 2 + 1
    nb = (T + M - 1) // M
    kmax = N // 2 - LV - 1
    bands = g.integers(1, kmax + 1, nb).astype(np.int32)
    x = rand_c64(g, T)
    y = oracle.filter_ola(N, overlap, V, bands, x)
    ref = np.zeros(T + N, np.complex128)
    xe = np.concatenate([x.astype(np.complex128), np.zeros(N)])
    for m in range(nb):
        h = closed_form_h(N, overlap, V, int(bands[m]))
        u = np.zeros(N, np.complex128)
        u[:M] = xe[m * M: m * M + M]
        z = np.array([sum(h[q] * u[(n - q) % N] for q in range(N)) for n in range(N)])
        ref[m * M: m * M + N] += z
    assert np.abs(y - ref[:T]).max() <= 1e-12 * max(1.0, np.abs(ref).max())

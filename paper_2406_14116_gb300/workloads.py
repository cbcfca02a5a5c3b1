"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no filtering arithmetic: it only draws signals, transition tables, band
schedules and stream mixes. Both the CUDA path and the FP64 oracle consume what it returns.

Every draw comes from ``numpy.random.Generator(PCG64(SeedSequence([seed, stream, purpose])))``,
so any one stream of a large workload can be regenerated on its own (the parity tests use that to
check sampled streams of the full-size workloads without materialising the rest).

Workloads (sizes as the paper's problem statement is exercised here; the paper itself prints no
signals and no transition values, so all of them are synthetic):
  * ``single``:   one stream of 2^16 samples, N=256, overlap 64, k1=60, L_V=6.
  * ``channels``: 64 channels x 2^22 samples, N=1024, overlap 256, L_V=12, k1 redrawn from
                  U{32..480} every 16 blocks per channel.
  * ``mixed``:    4096 streams, lengths floor(2^U(12,20)), N from {128..2048}, overlap N/4,
                  k1 ~ U{1..N/2-13}, L_V=12; noise plus 1-8 tones.
  * ``precision``: 16384 channels x 2^16 samples, N in {256, 512}, overlap N/4, L_V=12.
  * ``serving``:  2000 streams, N from {512, 1024, 2048}, Poisson chunk arrivals.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# purpose tags for SeedSequence entropy
_SIGNAL, _TABLE, _BANDS, _MIX, _TONES, _ARRIVALS = 1, 2, 3, 4, 5, 6


def rng_for(seed: int, stream: int, purpose: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, stream, purpose])))


def complex_gaussian(seed: int, stream: int, n: int) -> np.ndarray:
    """Unit-variance circular complex Gaussian, (N(0,1) + jN(0,1))/sqrt(2), complex64."""
    g = rng_for(seed, stream, _SIGNAL)
    v = g.standard_normal(2 * n, dtype=np.float32)
    v *= np.float32(1.0 / np.sqrt(2.0))
    return v.view(np.complex64)


def transition_table(seed: int, LV: int) -> np.ndarray:
    """L_V transition samples in (0, 1), sorted descending so they fall across the band edge.

    The paper prints no optimized V(r) (its figures are absent), so the values are drawn
    U(0, 1) and sorted; float64 (the library and the oracle both round them to float32)."""
    g = rng_for(seed, 0, _TABLE)
    v = g.uniform(0.0, 1.0, LV)
    v = np.where(v <= 0.0, 0.5, v)
    return np.sort(v)[::-1].copy()


def nblocks_for(nsamples: int, N: int, overlap: int) -> int:
    M = N - overlap
    return (nsamples + M - 1) // M


def band_schedule(seed: int, stream: int, nblocks: int, every: int, lo: int, hi: int) -> np.ndarray:
    """k1 per block: a fresh U{lo..hi} draw every ``every`` blocks (int32, length nblocks)."""
    g = rng_for(seed, stream, _BANDS)
    ngroups = max(1, -(-nblocks // every))
    draws = g.integers(lo, hi + 1, size=ngroups).astype(np.int32)
    return np.repeat(draws, every)[:nblocks].copy()


def max_band(N: int, LV: int) -> int:
    """Largest k1 allowed for N and L_V: k2 = k1 + L_V - 1 <= N/2 - 2 (eq. (k_var) bounds)."""
    return N // 2 - LV - 1


@dataclass
class Signal:
    """One stream of a workload: its plan geometry, per-block band and samples."""
    N: int
    overlap: int
    x: np.ndarray            # complex64
    band: np.ndarray         # int32, one k1 per block
    stream: int = 0


@dataclass
class Workload:
    name: str
    seed: int
    LV: int
    V: np.ndarray
    signals: list = field(default_factory=list)

    @property
    def total_samples(self) -> int:
        return int(sum(len(s.x) for s in self.signals))


def single(seed: int = 1, nsamples: int = 1 << 16, N: int = 256, overlap: int = 64,
           k1: int = 60, LV: int = 6) -> Workload:
    V = transition_table(seed, LV)
    x = complex_gaussian(seed, 0, nsamples)
    nb = nblocks_for(nsamples, N, overlap)
    band = np.full(nb, k1, dtype=np.int32)
    return Workload("single", seed, LV, V, [Signal(N, overlap, x, band, 0)])


def channels_band(seed: int, ch: int, nsamples: int, N: int, overlap: int,
                  every: int = 16, lo: int = 32, hi: int = 480) -> np.ndarray:
    return band_schedule(seed, ch, nblocks_for(nsamples, N, overlap), every, lo, hi)


def channels(seed: int = 2, nch: int = 64, nsamples: int = 1 << 22, N: int = 1024,
             overlap: int = 256, LV: int = 12, every: int = 16, lo: int = 32,
             hi: int = 480) -> Workload:
    V = transition_table(seed, LV)
    sigs = []
    for ch in range(nch):
        x = complex_gaussian(seed, ch, nsamples)
        band = channels_band(seed, ch, nsamples, N, overlap, every, lo, hi)
        sigs.append(Signal(N, overlap, x, band, ch))
    return Workload("channels", seed, LV, V, sigs)


def mixed_stream_params(seed: int, nstreams: int, log2_lo: float = 12.0, log2_hi: float = 20.0,
                        Ns=(128, 256, 512, 1024, 2048), LV: int = 12):
    """Per-stream (length, N, overlap, k1) of the mixed batch, drawn from one generator."""
    g = rng_for(seed, 0, _MIX)
    lengths = np.floor(2.0 ** g.uniform(log2_lo, log2_hi, nstreams)).astype(np.int64)
    Nsel = g.choice(np.asarray(Ns, dtype=np.int64), size=nstreams)
    k1 = np.array([g.integers(1, max_band(int(n), LV) + 1) for n in Nsel], dtype=np.int32)
    return lengths, Nsel.astype(np.int32), (Nsel // 4).astype(np.int32), k1


def tones_signal(seed: int, stream: int, n: int) -> np.ndarray:
    """Unit complex Gaussian noise plus K ~ U{1..8} tones: amplitude U(0.5, 2), frequency
    U(-0.5, 0.5) cycles/sample, phase U(0, 2 pi). complex64."""
    x = complex_gaussian(seed, stream, n).astype(np.complex128)
    g = rng_for(seed, stream, _TONES)
    K = int(g.integers(1, 9))
    t = np.arange(n, dtype=np.float64)
    for _ in range(K):
        a = g.uniform(0.5, 2.0)
        f = g.uniform(-0.5, 0.5)
        ph = g.uniform(0.0, 2.0 * np.pi)
        x += a * np.exp(1j * (2.0 * np.pi * f * t + ph))
    return x.astype(np.complex64)


def mixed(seed: int = 3, nstreams: int = 4096, LV: int = 12, log2_lo: float = 12.0,
          log2_hi: float = 20.0, Ns=(128, 256, 512, 1024, 2048), which=None) -> Workload:
    """Mixed batch; ``which`` (an iterable of stream ids) materialises only those streams."""
    V = transition_table(seed, LV)
    lengths, Nsel, ovl, k1 = mixed_stream_params(seed, nstreams, log2_lo, log2_hi, Ns, LV)
    ids = range(nstreams) if which is None else which
    sigs = []
    for i in ids:
        N, O, n = int(Nsel[i]), int(ovl[i]), int(lengths[i])
        band = np.full(nblocks_for(n, N, O), int(k1[i]), dtype=np.int32)
        sigs.append(Signal(N, O, tones_signal(seed, i, n), band, i))
    return Workload("mixed", seed, LV, V, sigs)


def precision_bands(seed: int, nch: int, N: int, LV: int = 12) -> np.ndarray:
    g = rng_for(seed, N, _BANDS)
    return g.integers(1, max_band(N, LV) + 1, size=nch).astype(np.int32)


def precision(seed: int = 4, nch: int = 16384, nsamples: int = 1 << 16, N: int = 256,
              LV: int = 12, which=None) -> Workload:
    V = transition_table(seed, LV)
    O = N // 4
    k1 = precision_bands(seed, nch, N, LV)
    ids = range(nch) if which is None else which
    sigs = []
    nb = nblocks_for(nsamples, N, O)
    for ch in ids:
        sigs.append(Signal(N, O, complex_gaussian(seed, ch, nsamples),
                           np.full(nb, int(k1[ch]), dtype=np.int32), ch))
    return Workload("precision", seed, LV, V, sigs)


@dataclass
class Chunk:
    t_arrival: float   # seconds from the start of the run
    stream: int
    nsamples: int
    new_band: int      # -1: no change; else k1 taking effect at the stream's next block


def serving_streams(seed: int = 5, nstreams: int = 2000, LV: int = 12, Ns=(512, 1024, 2048)):
    g = rng_for(seed, 0, _MIX)
    Nsel = g.choice(np.asarray(Ns, dtype=np.int64), size=nstreams).astype(np.int32)
    k1 = np.array([g.integers(1, max_band(int(n), LV) + 1) for n in Nsel], dtype=np.int32)
    return Nsel, (Nsel // 4).astype(np.int32), k1


def serving_arrivals(seed: int = 5, nstreams: int = 2000, rate: float = 50_000.0,
                     duration: float = 10.0, lo: int = 1024, hi: int = 65536,
                     change_frac: float = 0.01, Nsel=None, LV: int = 12):
    """Open-loop Poisson arrivals (aggregate ``rate`` chunks/s), stream chosen uniformly, chunk
    length U{lo..hi}; a fraction ``change_frac`` of chunks carry a new k1."""
    g = rng_for(seed, 0, _ARRIVALS)
    n = int(rate * duration * 1.2) + 16
    t = np.cumsum(g.exponential(1.0 / rate, n))
    t = t[t < duration]
    n = len(t)
    streams = g.integers(0, nstreams, n)
    lens = g.integers(lo, hi + 1, n)
    chg = g.uniform(0, 1, n) < change_frac
    nb = np.full(n, -1, dtype=np.int64)
    if Nsel is not None:
        for i in np.nonzero(chg)[0]:
            nb[i] = g.integers(1, max_band(int(Nsel[streams[i]]), LV) + 1)
    return t, streams.astype(np.int32), lens.astype(np.int64), nb.astype(np.int32)

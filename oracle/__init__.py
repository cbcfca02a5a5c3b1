"""FP64 CPU oracle for OLS variable-bandwidth filtering (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package. It shares no code with the CUDA path: the arithmetic lives in ``vbw_oracle.c``
(plain C99, double complex, direct O(N^2) DFT), built here with gcc and called through ctypes.

Paper passages followed (Moryakova & Johansson):
  * Sec. II, steps 1-5: segment, N-point DFT, multiply by H(k), IDFT, discard N-M, concatenate.
  * eq. (OLS_dn): the IDFT carries +j and 1/N.
  * eq. (FS_Hk_exp): H(k,b) = H_R(k,b) exp(-j 2 pi k (L-1)/2 / N).
  * eq. (FS_Hk_real) with the regions k_p, k_t, k_s and eq. (k_var) for k1, k2.
  * eq. (OLS_Hn): the time-invariant response H_n of each output phase n (the PTVIR view of OLS),
    and the error E_n of eq. (err_min) against eq. (VBW_des).
  * Sec. I / Sec. II: overlap-add, the other FC method, with the same H(k) and the same steps 1-3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vbw_oracle.c")
_LIB = os.path.join(_HERE, "libvbw_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``vbw_oracle.c`` into ``libvbw_oracle.so`` (gcc, -O2, OpenMP). Returns the path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i32, i64, p = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        lib.vbwo_HR.argtypes = [i32, i32, p, i32, p]
        lib.vbwo_H.argtypes = [i32, i32, i32, p, i32, p]
        lib.vbwo_dft.argtypes = [i32, p, p, i32]
        lib.vbwo_filter_H.argtypes = [i32, i32, p, p, i64, p, i64, i64, p, i32]
        lib.vbwo_filter.argtypes = [i32, i32, i32, p, p, p, i64, p, i64, i64, p, i32]
        lib.vbwo_max_threads.argtypes = []
        lib.vbwo_ptvir.argtypes = [i32, i32, p, p, p, i32, p, i32]
        lib.vbwo_filter_ola.argtypes = [i32, i32, i32, p, p, p, i64, p]
        lib.vbwo_filter_ola_H.argtypes = [i32, i32, p, p, i64, p]
        for f in (lib.vbwo_HR, lib.vbwo_H, lib.vbwo_dft, lib.vbwo_filter_H, lib.vbwo_filter,
                  lib.vbwo_max_threads, lib.vbwo_ptvir, lib.vbwo_filter_ola, lib.vbwo_filter_ola_H):
            f.restype = i32
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex64))


def _f32(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.float32))


def max_threads() -> int:
    return int(_load().vbwo_max_threads())


def HR(N: int, V, k1: int) -> np.ndarray:
    """H_R(k, b) for k = 0..N-1 (eq. FS_Hk_real); V is rounded to float32 first."""
    V = _f32(V)
    out = np.empty(N, dtype=np.float64)
    if _load().vbwo_HR(N, len(V), _ptr(V), k1, _ptr(out)) != 0:
        raise ValueError(f"band k1={k1} outside the valid range for N={N}, L_V={len(V)}")
    return out


def H(N: int, overlap: int, V, k1: int) -> np.ndarray:
    """H(k, b) = H_R(k, b) exp(-j 2 pi k (L-1)/2 / N) (eq. FS_Hk_exp), complex128."""
    V = _f32(V)
    out = np.empty(2 * N, dtype=np.float64)
    if _load().vbwo_H(N, overlap, len(V), _ptr(V), k1, _ptr(out)) != 0:
        raise ValueError("invalid H arguments")
    return out[0::2] + 1j * out[1::2]


def dft(x, sign: int = -1) -> np.ndarray:
    """Direct DFT sum_n x(n) exp(sign j 2 pi n k / N), unscaled, complex128."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    out = np.empty(2 * len(x), dtype=np.float64)
    if _load().vbwo_dft(len(x), _ptr(x.view(np.float64)), _ptr(out), sign) != 0:
        raise ValueError("invalid DFT arguments")
    return out[0::2] + 1j * out[1::2]


def _nthreads(nthreads):
    return max_threads() if nthreads is None else int(nthreads)


def filter_H(N: int, overlap: int, Hk, x, tail=None, blocks=None, nthreads=None) -> np.ndarray:
    """OLS filtering (Sec. II) of a whole complex64 stream with one fixed complex H(k).

    Returns complex128 output of the same length as ``x``. ``blocks=(b0, nb)`` restricts the
    computation to those blocks (other outputs are left as NaN)."""
    x = _c64(x)
    T = len(x)
    M = N - overlap
    Hk = np.ascontiguousarray(np.asarray(Hk, dtype=np.complex128))
    tail = None if tail is None else _c64(tail)
    y = np.full(2 * T, np.nan, dtype=np.float64)
    b0, nb = (0, (T + M - 1) // M) if blocks is None else blocks
    rc = _load().vbwo_filter_H(N, overlap, _ptr(Hk.view(np.float64)), _ptr(x.view(np.float32)),
                               T, _ptr(tail.view(np.float32) if tail is not None else None),
                               b0, nb, _ptr(y), _nthreads(nthreads))
    if rc != 0:
        raise ValueError("vbwo_filter_H failed")
    return y[0::2] + 1j * y[1::2]


def filter(N: int, overlap: int, V, band, x, tail=None, blocks=None, nthreads=None) -> np.ndarray:
    """OLS VBW filtering of a complex64 stream; ``band`` is k1 per block (an int applies to all).

    Returns complex128 output (length len(x)); with ``blocks=(b0, nb)`` only those blocks are
    computed and every other output is NaN."""
    x = _c64(x)
    T = len(x)
    M = N - overlap
    nblocks = (T + M - 1) // M
    band = np.asarray(band, dtype=np.int32)
    if band.ndim == 0:
        band = np.full(max(nblocks, 1), int(band), dtype=np.int32)
    band = np.ascontiguousarray(band)
    if len(band) < nblocks:
        raise ValueError("band must have one entry per block")
    V = _f32(V)
    tail = None if tail is None else _c64(tail)
    y = np.full(2 * T, np.nan, dtype=np.float64)
    b0, nb = (0, nblocks) if blocks is None else blocks
    rc = _load().vbwo_filter(N, overlap, len(V), _ptr(V), _ptr(band), _ptr(x.view(np.float32)),
                             T, _ptr(tail.view(np.float32) if tail is not None else None),
                             b0, nb, _ptr(y), _nthreads(nthreads))
    if rc != 0:
        raise ValueError(f"vbwo_filter failed ({rc})")
    return y[0::2] + 1j * y[1::2]


def impulse_response(N: int, overlap: int, V, k1: int) -> np.ndarray:
    """h(q) = (1/N) sum_k H(k, b) e^{+j 2 pi q k / N} (eq. OLS_dn), by the direct inverse DFT of
    the oracle's H (complex128; real up to rounding)."""
    return dft(H(N, overlap, V, k1), +1) / N


def ptvir_errors_h(N: int, overlap: int, h, omega, desired, nthreads=None) -> np.ndarray:
    """|E_n(w_i)| = |H_n(w_i) e^{j w_i O/2} - d_i| for every output phase n = 0..M-1 and grid
    point i (eq. OLS_Hn, eq. err_min), for any impulse response h of length N. Shape (M, K)."""
    h = np.ascontiguousarray(np.asarray(h, dtype=np.complex128))
    if len(h) != N:
        raise ValueError("h must have N entries")
    omega = np.ascontiguousarray(np.asarray(omega, dtype=np.float64))
    d = np.ascontiguousarray(np.broadcast_to(np.asarray(desired, dtype=np.float64), omega.shape))
    K = len(omega)
    M = N - overlap
    E = np.empty((M, K), dtype=np.float64)
    if _load().vbwo_ptvir(N, overlap, _ptr(h.view(np.float64)), _ptr(omega), _ptr(d), K, _ptr(E),
                          _nthreads(nthreads)) != 0:
        raise ValueError("vbwo_ptvir failed")
    return E


def ptvir_errors(N: int, overlap: int, V, k1: int, omega, desired, nthreads=None) -> np.ndarray:
    """PTVIR errors |E_n(w_i, b)| (shape (M, K)) of the VBW filter with band k1 (V rounded to
    float32, as the plan keeps it)."""
    return ptvir_errors_h(N, overlap, impulse_response(N, overlap, V, k1), omega, desired, nthreads)


def filter_ola(N: int, overlap: int, V, band, x) -> np.ndarray:
    """Overlap-add VBW filtering (Sec. I, Sec. II steps 1-3 on zero-padded blocks of M = N - O
    samples, results overlapped by O and added) of a complex64 signal; ``band`` is k1 per block
    (an int applies to all). Returns complex128 output of the input's length."""
    x = _c64(x)
    T = len(x)
    M = N - overlap
    nblocks = (T + M - 1) // M
    band = np.asarray(band, dtype=np.int32)
    if band.ndim == 0:
        band = np.full(max(nblocks, 1), int(band), dtype=np.int32)
    band = np.ascontiguousarray(band)
    if len(band) < nblocks:
        raise ValueError("band must have one entry per block")
    V = _f32(V)
    y = np.empty(2 * T, dtype=np.float64)
    rc = _load().vbwo_filter_ola(N, overlap, len(V), _ptr(V), _ptr(band), _ptr(x.view(np.float32)), T,
                                 _ptr(y))
    if rc != 0:
        raise ValueError(f"vbwo_filter_ola failed ({rc})")
    return y[0::2] + 1j * y[1::2]


def filter_ola_H(N: int, overlap: int, Hk, x) -> np.ndarray:
    """Overlap-add filtering with one fixed complex H(k) for every block (complex128 output)."""
    x = _c64(x)
    T = len(x)
    Hk = np.ascontiguousarray(np.asarray(Hk, dtype=np.complex128))
    y = np.empty(2 * T, dtype=np.float64)
    if _load().vbwo_filter_ola_H(N, overlap, _ptr(Hk.view(np.float64)), _ptr(x.view(np.float32)), T,
                                 _ptr(y)) != 0:
        raise ValueError("vbwo_filter_ola_H failed")
    return y[0::2] + 1j * y[1::2]

"""Thin Python binding of libvbw (include/vbw.h), argument marshalling only.

Functions named ``vbw_*`` mirror the C entry points one to one; the classes ``Plan``, ``Stream``
and ``Batch`` only hold handles and turn tensors into pointers. Every filtering step runs in the
CUDA kernels of the library; there is no fallback: if ``libvbw.so`` is missing or fails to load,
every call raises ``VbwError``.

Device arrays are passed as ``torch.Tensor`` (complex64, CUDA, contiguous) or as raw integer
device pointers; host arrays as ``numpy.ndarray``.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvbw.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "vbw.h")

VBW_OK = 0
STATUS_NAMES = {0: "VBW_OK", 1: "VBW_ERR_INVALID_ARG", 2: "VBW_ERR_BAND_RANGE", 3: "VBW_ERR_NOMEM",
                4: "VBW_ERR_CUDA", 5: "VBW_ERR_TIMEOUT", 6: "VBW_ERR_BUSY", 7: "VBW_ERR_STATE",
                8: "VBW_ERR_UNSUPPORTED"}
VBW_PREC_FP32, VBW_PREC_BF16_SPLIT, VBW_PREC_FP16_SCALED, VBW_PREC_BF16_SPLIT3 = 0, 1, 2, 3
VBW_BATCH_AUTO, VBW_BATCH_PER_PLAN, VBW_BATCH_MIXED = 0, 1, 2


class VbwError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


# vbw_completion / vbw_server_stats of include/vbw.h as numpy record types
COMPLETION_DTYPE = np.dtype([("tag", "<u8"), ("stream", "<i4"), ("final_flush", "<i4"),
                             ("produced", "<i8"), ("t_submit", "<f8"), ("t_done", "<f8")])
REQUEST_DTYPE = np.dtype([("stream", "<i4"), ("new_band", "<i4"), ("host_in", "<u8"), ("n", "<i8"),
                          ("host_out", "<u8"), ("out_capacity", "<i8"), ("tag", "<u8")])
SERVER_STATS_FIELDS = ("queued", "inflight_batches", "completions_ready", "batches", "launches",
                       "admitted", "slot_bytes", "slots")


class vbw_signal(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("nsamples", ctypes.c_int64), ("band", ctypes.c_int32),
                ("band_per_block", ctypes.c_void_p)]


_lib = None


def declared_functions() -> list[str]:
    """Names of the functions include/vbw.h declares."""
    text = open(HEADER_PATH).read()
    return sorted(set(re.findall(r"\b(vbw_[a-z_A-Z0-9]+)\s*\(", text)))


def lib():
    """Loads libvbw.so (built by paper_2406_14116_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise VbwError(-1, f"{LIB_PATH} is missing: run paper_2406_14116_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    i32, i64, p, sz = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "vbw_plan": [i32, i32, p, i32, i32, pp],
        "vbw_plan_destroy": [p],
        "vbw_plan_info": [p, p, p, p, p],
        "vbw_stream_create": [p, i32, p, pp],
        "vbw_stream_destroy": [p],
        "vbw_stream_reset": [p, i32],
        "vbw_set_bandwidth": [p, i32],
        "vbw_set_bandwidth_at": [p, i64, i32],
        "vbw_filter": [p, p, p, i64],
        "vbw_flush": [p, p, p, i32],
        "vbw_filter_host": [p, p, p, i64],
        "vbw_stream_position": [p, p],
        "vbw_stream_save": [p, p, ctypes.POINTER(sz)],
        "vbw_stream_restore": [p, p, sz],
        "vbw_batch_create": [p, i32, pp],
        "vbw_batch_create_real": [p, i32, pp],
        "vbw_batch_run": [p, p],
        "vbw_batch_run_host": [p, p, p, p],
        "vbw_batch_destroy": [p],
        "vbw_batch_launches": [p, p],
        "vbw_debug_export_HR": [p, i32, p],
        "vbw_batch_set_mode": [p, i32, ctypes.c_double],
        "vbw_tune_set": [i32, i32, i32],
        "vbw_plan_status": [p, p, i32],
        "vbw_debug_set": [i32],
        "vbw_filter_static": [i32, i32, p, i32, i32, p, p, i64, p],
        "vbw_debug_tc_gemm": [i32, i32, i32, p, p, p],
        "vbw_ptvir_error": [p, p, i32, p, p, i32, p, p, p],
        "vbw_filter_ola": [p, p, p, i64, i32, i32, p, p],
        "vbw_server_create": [p, i32, i32, sz, i32, pp],
        "vbw_server_destroy": [p],
        "vbw_server_open_stream": [p, i32, i32, i32],
        "vbw_server_submit": [p, i32, p, i64, i32, p, i64, ctypes.c_uint64],
        "vbw_server_close_stream": [p, i32, p, i64, ctypes.c_uint64],
        "vbw_server_submit_many": [p, p, i32, p],
        "vbw_server_poll": [p, p, i32, p],
        "vbw_server_wait": [p, p, i32, p],
        "vbw_server_info": [p, p],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.vbw_last_error.argtypes = []
    L.vbw_last_error.restype = ctypes.c_char_p
    L.vbw_version.argtypes = []
    L.vbw_version.restype = ctypes.c_char_p
    L.vbw_server_clock.argtypes = []
    L.vbw_server_clock.restype = ctypes.c_double
    _lib = L
    return L


def vbw_last_error() -> str:
    return lib().vbw_last_error().decode()


def vbw_version() -> str:
    return lib().vbw_version().decode()


def _check(code: int):
    if code != VBW_OK:
        raise VbwError(code, vbw_last_error())


def _dev_ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        import torch
        if x.dtype != torch.complex64:
            raise ValueError("expected complex64 samples")
        return int(x.data_ptr())
    raise TypeError(f"cannot take a device pointer of {type(x)}")


def _host_ptr(a: np.ndarray):
    if not a.flags.c_contiguous:
        raise ValueError("expected a C-contiguous host array")
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(cuda_stream) -> int:
    if cuda_stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(cuda_stream, int):
        return cuda_stream
    return int(cuda_stream.cuda_stream)


# ---- C entry points ---------------------------------------------------------------------------

def vbw_plan(N: int, overlap: int, transition_samples, precision: int = VBW_PREC_FP32) -> int:
    V = np.ascontiguousarray(np.asarray(transition_samples, dtype=np.float64))
    h = ctypes.c_void_p()
    _check(lib().vbw_plan(N, overlap, _host_ptr(V), len(V), precision, ctypes.byref(h)))
    return h.value


def vbw_plan_destroy(plan: int):
    _check(lib().vbw_plan_destroy(plan))


def vbw_plan_info(plan: int):
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().vbw_plan_info(plan, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)   # N, overlap, L_V, M


def vbw_stream_create(plan: int, band: int, cuda_stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().vbw_stream_create(plan, band, _stream_handle(cuda_stream), ctypes.byref(h)))
    return h.value


def vbw_stream_destroy(s: int):
    _check(lib().vbw_stream_destroy(s))


def vbw_stream_reset(s: int, band: int):
    _check(lib().vbw_stream_reset(s, band))


def vbw_set_bandwidth(s: int, band: int):
    _check(lib().vbw_set_bandwidth(s, band))


def vbw_set_bandwidth_at(s: int, block: int, band: int):
    _check(lib().vbw_set_bandwidth_at(s, block, band))


def vbw_filter(s: int, inp, out, nblocks: int):
    _check(lib().vbw_filter(s, _dev_ptr(inp), _dev_ptr(out), nblocks))


def vbw_flush(s: int, inp, out, nvalid: int):
    _check(lib().vbw_flush(s, _dev_ptr(inp), _dev_ptr(out), nvalid))


def vbw_filter_host(s: int, inp: np.ndarray, out: np.ndarray, nblocks: int):
    _check(lib().vbw_filter_host(s, _host_ptr(inp), _host_ptr(out), nblocks))


def vbw_stream_position(s: int) -> int:
    v = ctypes.c_int64()
    _check(lib().vbw_stream_position(s, ctypes.byref(v)))
    return v.value


def vbw_stream_save(s: int) -> bytes:
    n = ctypes.c_size_t(0)
    _check(lib().vbw_stream_save(s, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().vbw_stream_save(s, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def vbw_stream_restore(s: int, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(lib().vbw_stream_restore(s, buf, len(state)))


def _dev_ptr_real(x) -> int:
    if isinstance(x, int):
        return x
    import torch
    if not (hasattr(x, "data_ptr") and x.is_cuda and x.is_contiguous() and x.dtype == torch.float32):
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return int(x.data_ptr())


def vbw_batch_create(signals, real: bool = False) -> int:
    """signals: sequence of (plan, in, out, nsamples, band, band_per_block or None); real=True
    takes float32 signals (vbw_batch_create_real)."""
    arr = (vbw_signal * max(1, len(signals)))()
    keep = []
    ptr_of = _dev_ptr_real if real else _dev_ptr
    for i, (plan, inp, out, nsamp, band, bpb) in enumerate(signals):
        ptr = None
        if bpb is not None:
            bpb = np.ascontiguousarray(np.asarray(bpb, dtype=np.int32))
            keep.append(bpb)
            ptr = bpb.ctypes.data
        arr[i] = vbw_signal(plan, ptr_of(inp), ptr_of(out), int(nsamp), int(band), ptr)
    h = ctypes.c_void_p()
    create = lib().vbw_batch_create_real if real else lib().vbw_batch_create
    _check(create(arr, len(signals), ctypes.byref(h)))
    return h.value


def vbw_batch_run(b: int, cuda_stream=None):
    _check(lib().vbw_batch_run(b, _stream_handle(cuda_stream)))


def host_pointers(arrays) -> np.ndarray:
    """The addresses of C-contiguous numpy arrays, as the pointer array vbw_batch_run_host takes.
    Building it costs about 1 us per array, so callers that run the same buffers repeatedly
    make it once and pass it instead of the arrays."""
    for a in arrays:
        if not a.flags.c_contiguous:
            raise ValueError("expected C-contiguous host arrays")
    return np.array([a.__array_interface__["data"][0] for a in arrays], dtype=np.uintp)


def _pointer_array(bufs):
    if isinstance(bufs, np.ndarray) and bufs.dtype == np.uintp and bufs.ndim == 1:
        return np.ascontiguousarray(bufs)
    return host_pointers(bufs)


def vbw_batch_run_host(b: int, host_in, host_out, cuda_stream=None):
    """host_in / host_out: sequences of C-contiguous numpy arrays (one per signal), or their
    address arrays from host_pointers()."""
    ins, outs = _pointer_array(host_in), _pointer_array(host_out)
    _check(lib().vbw_batch_run_host(b, ins.ctypes.data_as(ctypes.c_void_p),
                                    outs.ctypes.data_as(ctypes.c_void_p), _stream_handle(cuda_stream)))


def vbw_batch_destroy(b: int):
    _check(lib().vbw_batch_destroy(b))


def vbw_batch_launches(b: int) -> int:
    v = ctypes.c_int()
    _check(lib().vbw_batch_launches(b, ctypes.byref(v)))
    return v.value


def vbw_batch_set_mode(b: int, mode: int, mixed_share: float = 0.0):
    _check(lib().vbw_batch_set_mode(b, mode, mixed_share))


def vbw_tune_set(N: int, warps: int, ctas_per_sm: int = 0):
    _check(lib().vbw_tune_set(N, warps, ctas_per_sm))


def vbw_plan_status(plan: int, clear: bool = False) -> int:
    """Returns the plan's device status word; raises VbwError(VBW_ERR_TIMEOUT) if bit 0 is set."""
    v = ctypes.c_int(0)
    _check(lib().vbw_plan_status(plan, ctypes.byref(v), 1 if clear else 0))
    return v.value


def vbw_plan_status_raw(plan: int, clear: bool = False) -> tuple[int, int]:
    """(status code, flags) without raising."""
    v = ctypes.c_int(0)
    rc = lib().vbw_plan_status(plan, ctypes.byref(v), 1 if clear else 0)
    return rc, v.value


def vbw_debug_set(flags: int):
    _check(lib().vbw_debug_set(flags))


def vbw_filter_static(N: int, overlap: int, transition_samples, band: int, inp, out,
                      nsamples: int, cuda_stream=None):
    """Whole-signal filtering that allocates nothing (tables in the library's static scratch)."""
    V = np.ascontiguousarray(np.asarray(transition_samples, dtype=np.float64))
    _check(lib().vbw_filter_static(N, overlap, _host_ptr(V), len(V), band, _dev_ptr(inp),
                                   _dev_ptr(out), nsamples, _stream_handle(cuda_stream)))


def vbw_debug_tc_gemm(A: np.ndarray, B: np.ndarray, bf16: bool = True, a_mn_major: bool = False) -> np.ndarray:
    """D = A B on the tensor cores (A 128 x K, B K x NN, float32 host arrays); A stored K-major or
    MN-major."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    D = np.empty((A.shape[0], B.shape[1]), dtype=np.float32)
    flags = (1 if bf16 else 0) | (2 if a_mn_major else 0)
    _check(lib().vbw_debug_tc_gemm(flags, A.shape[1], B.shape[1], _host_ptr(A),
                                   _host_ptr(B), _host_ptr(D)))
    return D


def vbw_debug_export_HR(plan: int, band: int) -> np.ndarray:
    N = vbw_plan_info(plan)[0]
    out = np.empty(N, dtype=np.float32)
    _check(lib().vbw_debug_export_HR(plan, band, _host_ptr(out)))
    return out


def vbw_filter_ola(plan: int, inp, out, nsamples: int, nsignals: int = 1, band: int = 0,
                   band_per_block=None, cuda_stream=None):
    """Overlap-add filtering of nsignals back-to-back complex64 rows (device tensors); band_per_block
    is an int32 CUDA tensor of nsignals x ceil(nsamples / M) k1 values, or None."""
    bpb = None if band_per_block is None else _dev_ptr_typed(band_per_block, "int32")
    _check(lib().vbw_filter_ola(plan, _dev_ptr(inp), _dev_ptr(out), nsamples, nsignals, band, bpb,
                                _stream_handle(cuda_stream)))


def _dev_ptr_typed(x, dtype_name: str) -> int:
    """Device pointer of a contiguous CUDA tensor of the given torch dtype name."""
    import torch
    if not (hasattr(x, "data_ptr") and x.is_cuda and x.is_contiguous()
            and x.dtype == getattr(torch, dtype_name)):
        raise ValueError(f"expected a contiguous {dtype_name} CUDA tensor")
    return int(x.data_ptr())


def vbw_ptvir_error(plan: int, bands, omega, desired, err, phase=None, cuda_stream=None):
    """PTVIR errors on the GPU: bands (int32, nbands), omega (float64, nbands x K), desired
    (float32, nbands x K); writes err (float32, nbands x K) and phase (int32, or None)."""
    nb = int(bands.numel())
    K = int(omega.shape[-1]) if omega.dim() == 2 else (int(omega.numel()) if nb == 1 else -1)
    if K < 0 or omega.numel() != nb * K or desired.numel() != nb * K or err.numel() != nb * K:
        raise ValueError("omega, desired and err must hold nbands x K values")
    if phase is not None and phase.numel() != nb * K:
        raise ValueError("phase must hold nbands x K values")
    _check(lib().vbw_ptvir_error(plan, _dev_ptr_typed(bands, "int32"), nb, _dev_ptr_typed(omega, "float64"),
                                 _dev_ptr_typed(desired, "float32"), K, _dev_ptr_typed(err, "float32"),
                                 None if phase is None else _dev_ptr_typed(phase, "int32"),
                                 _stream_handle(cuda_stream)))


def _hptr(a) -> int:
    """Address of a host buffer: a C-contiguous numpy array or a raw integer address."""
    if a is None:
        return 0
    if isinstance(a, int):
        return a
    if not a.flags.c_contiguous:
        raise ValueError("expected a C-contiguous host array")
    return int(a.ctypes.data)


def vbw_server_create(plans, max_streams: int, pool_bytes: int, slots: int) -> int:
    arr = (ctypes.c_void_p * len(plans))(*plans)
    h = ctypes.c_void_p()
    _check(lib().vbw_server_create(arr, len(plans), max_streams, pool_bytes, slots, ctypes.byref(h)))
    return h.value


def vbw_server_destroy(sv: int):
    _check(lib().vbw_server_destroy(sv))


def vbw_server_open_stream(sv: int, stream: int, plan: int, band: int):
    _check(lib().vbw_server_open_stream(sv, stream, plan, band))


def vbw_server_submit(sv: int, stream: int, host_in, n: int, new_band: int, host_out,
                      out_capacity: int, tag: int):
    _check(lib().vbw_server_submit(sv, stream, _hptr(host_in), n, new_band, _hptr(host_out),
                                   out_capacity, tag))


def vbw_server_submit_many(sv: int, requests: np.ndarray) -> int:
    """requests: REQUEST_DTYPE records (vbw_request). Returns how many were queued; raises on the
    first failing chunk."""
    req = np.ascontiguousarray(requests, dtype=REQUEST_DTYPE)
    n = ctypes.c_int(0)
    code = lib().vbw_server_submit_many(sv, req.ctypes.data, len(req), ctypes.byref(n))
    if code != VBW_OK:
        raise VbwError(code, f"{vbw_last_error()} (after {n.value} queued)")
    return n.value


def vbw_server_close_stream(sv: int, stream: int, host_out, out_capacity: int, tag: int):
    _check(lib().vbw_server_close_stream(sv, stream, _hptr(host_out), out_capacity, tag))


def vbw_server_poll(sv: int, out: np.ndarray) -> int:
    """Fills out (COMPLETION_DTYPE records) from the front; returns how many."""
    n = ctypes.c_int(0)
    _check(lib().vbw_server_poll(sv, out.ctypes.data, len(out), ctypes.byref(n)))
    return n.value


def vbw_server_wait(sv: int, out: np.ndarray) -> int:
    n = ctypes.c_int(0)
    _check(lib().vbw_server_wait(sv, out.ctypes.data, len(out), ctypes.byref(n)))
    return n.value


def vbw_server_info(sv: int) -> dict:
    v = (ctypes.c_int64 * len(SERVER_STATS_FIELDS))()
    _check(lib().vbw_server_info(sv, v))
    return dict(zip(SERVER_STATS_FIELDS, list(v)))


def vbw_server_clock() -> float:
    return float(lib().vbw_server_clock())


# ---- handle holders ---------------------------------------------------------------------------

class Plan:
    def __init__(self, N: int, overlap: int, V, precision: int = VBW_PREC_FP32):
        self.handle = vbw_plan(N, overlap, V, precision)
        self.N, self.overlap, self.LV, self.M = vbw_plan_info(self.handle)

    def close(self):
        if self.handle:
            vbw_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stream:
    def __init__(self, plan: Plan, band: int, cuda_stream=None):
        self.plan = plan
        self.handle = vbw_stream_create(plan.handle, band, cuda_stream)

    def filter(self, inp, out, nblocks: int | None = None):
        if nblocks is None:
            nblocks = inp.numel() // self.plan.M
        vbw_filter(self.handle, inp, out, nblocks)

    def flush(self, inp, out, nvalid: int):
        vbw_flush(self.handle, inp, out, nvalid)

    def filter_host(self, inp: np.ndarray, out: np.ndarray, nblocks: int | None = None):
        if nblocks is None:
            nblocks = len(inp) // self.plan.M
        vbw_filter_host(self.handle, inp, out, nblocks)

    def set_bandwidth(self, band: int):
        vbw_set_bandwidth(self.handle, band)

    def set_bandwidth_at(self, block: int, band: int):
        vbw_set_bandwidth_at(self.handle, block, band)

    def reset(self, band: int):
        vbw_stream_reset(self.handle, band)

    @property
    def position(self) -> int:
        return vbw_stream_position(self.handle)

    def save(self) -> bytes:
        return vbw_stream_save(self.handle)

    def restore(self, state: bytes):
        vbw_stream_restore(self.handle, state)

    def close(self):
        if self.handle:
            vbw_stream_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A prepared batch: signals = [(Plan, in_tensor, out_tensor, band or per-block array)];
    real=True for float32 signals (pairs of real blocks per complex transform)."""

    def __init__(self, signals, real: bool = False):
        rows = []
        for plan, inp, out, band in signals:
            n = int(inp.numel())
            if np.ndim(band) == 0:
                rows.append((plan.handle, inp, out, n, int(band), None))
            else:
                b = np.asarray(band, dtype=np.int32)
                rows.append((plan.handle, inp, out, n, int(b[0]) if len(b) else 1, b))
        self.handle = vbw_batch_create(rows, real)
        self.signals = signals

    def run(self, cuda_stream=None):
        vbw_batch_run(self.handle, cuda_stream)

    def run_host(self, host_in, host_out, cuda_stream=None):
        vbw_batch_run_host(self.handle, host_in, host_out, cuda_stream)

    def set_mode(self, mode: int, mixed_share: float = 0.0):
        vbw_batch_set_mode(self.handle, mode, mixed_share)

    @property
    def launches(self) -> int:
        return vbw_batch_launches(self.handle)

    def close(self):
        if self.handle:
            vbw_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server over ``plans`` (a list of Plan)."""

    def __init__(self, plans, max_streams: int, pool_bytes: int, slots: int = 4,
                 max_completions: int = 65536):
        self.plans = list(plans)
        self.handle = vbw_server_create([p.handle for p in self.plans], max_streams, pool_bytes, slots)
        self._buf = np.zeros(max_completions, dtype=COMPLETION_DTYPE)

    def open_stream(self, stream: int, plan: int, band: int):
        vbw_server_open_stream(self.handle, stream, plan, band)

    def submit(self, stream: int, host_in, n: int | None = None, new_band: int = -1, host_out=None,
               out_capacity: int | None = None, tag: int = 0):
        if n is None:
            n = len(host_in)
        if out_capacity is None:
            out_capacity = 0 if host_out is None or isinstance(host_out, int) else len(host_out)
        vbw_server_submit(self.handle, stream, host_in, n, new_band, host_out, out_capacity, tag)

    def submit_many(self, requests: np.ndarray) -> int:
        return vbw_server_submit_many(self.handle, requests)

    def close_stream(self, stream: int, host_out=None, out_capacity: int | None = None, tag: int = 0):
        if out_capacity is None:
            out_capacity = 0 if host_out is None or isinstance(host_out, int) else len(host_out)
        vbw_server_close_stream(self.handle, stream, host_out, out_capacity, tag)

    def poll(self) -> np.ndarray:
        return self._buf[:vbw_server_poll(self.handle, self._buf)].copy()

    def wait(self) -> np.ndarray:
        return self._buf[:vbw_server_wait(self.handle, self._buf)].copy()

    def drain(self) -> np.ndarray:
        """Runs until nothing is queued or in flight; returns every completion."""
        got = []
        while True:
            c = self.wait()
            if len(c) == 0:
                break
            got.append(c)
        return np.concatenate(got) if got else np.zeros(0, dtype=COMPLETION_DTYPE)

    def info(self) -> dict:
        return vbw_server_info(self.handle)

    def close(self):
        if self.handle:
            vbw_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

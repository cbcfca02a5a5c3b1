"""vbw_filter_static: filtering for callers that cannot allocate device memory.

Those callers are frameworks that own every device allocation through their own pool, real-time
loops that cannot afford cudaMalloc's device synchronization, and code that must not touch the
CUDA allocator. The entry point keeps its tables in a fixed array that belongs to the library.
This file is collected last, so a run that stops at the first failure has already run every
other test."""
import ctypes

import numpy as np
import pytest

from conftest import assert_parity
from paper_2406_14116_gb300 import build as vbw_build
from paper_2406_14116_gb300 import vbw
from paper_2406_14116_gb300 import workloads as wl


def _call(L, N, O, V, band, inp, out, n, stream):
    V = np.ascontiguousarray(np.asarray(V, dtype=np.float64))
    return L.vbw_filter_static(N, O, V.ctypes.data_as(ctypes.c_void_p), len(V), band,
                               ctypes.c_void_p(inp), ctypes.c_void_p(out), n, ctypes.c_void_p(stream))


def test_no_alloc_rejects_bad_requests_before_touching_the_gpu():
    vbw_build.build()
    L = vbw.lib()
    V = np.linspace(0.9, 0.1, 12)
    assert _call(L, 100, 24, V, 5, 0, 0, 10, 0) == 1          # N not a power of two
    assert _call(L, 256, 256, V, 5, 0, 0, 10, 0) == 1         # overlap = N
    assert _call(L, 256, 64, V, 0, 0, 0, 10, 0) == 2          # band below range
    assert _call(L, 256, 64, V, 128 - 12, 0, 0, 10, 0) == 2   # band above range
    assert _call(L, 256, 64, V, 5, 0, 0, -1, 0) == 1          # negative length
    assert _call(L, 256, 64, V, 5, 0, 0, 0, 0) == 0           # empty signal: nothing to do


@pytest.mark.gpu
def test_no_alloc_matches_existing_entry_point_on_two_calls(cuda):
    """Two calls in a row (different N, overlap, table and band) through the C ABI: each output
    equals the existing path's (a plan and a one-signal batch) within the FP32 parity tolerance."""
    torch = cuda
    L = vbw.lib()
    stream = torch.cuda.current_stream()
    cases = [(1024, 256, 12, 200, 300_000, 41), (256, 64, 6, 60, (1 << 16) + 77, 42)]
    for N, O, LV, band, n, seed in cases:
        V = wl.transition_table(seed, LV)
        x = torch.from_numpy(wl.complex_gaussian(seed, 0, n)).cuda()
        y_static = torch.full_like(x, float("nan"))
        rc = _call(L, N, O, V, band, x.data_ptr(), y_static.data_ptr(), n, stream.cuda_stream)
        assert rc == 0, vbw.vbw_last_error()
        plan = vbw.Plan(N, O, V)
        y_ref = torch.full_like(x, float("nan"))
        vbw.Batch([(plan, x, y_ref, band)]).run(stream)
        torch.cuda.synchronize()
        assert_parity(y_static.cpu().numpy(), y_ref.cpu().numpy(), what=f"N={N}")


@pytest.mark.gpu
def test_no_alloc_split_kernel_equals_batch_path(cuda, monkeypatch):
    """N = 2048 with overlap N/4 through the split kernel (forced for this size): the no-alloc call
    and a one-signal batch run the same kernel on the same data, so their outputs are identical."""
    monkeypatch.setenv("VBW_SPLIT2048", "2")
    torch = cuda
    L = vbw.lib()
    stream = torch.cuda.current_stream()
    N, O, band, n = 2048, 512, 700, 400_000 + 123
    V = wl.transition_table(46, 12)
    x = torch.from_numpy(wl.complex_gaussian(46, 0, n)).cuda()
    y_static = torch.full_like(x, float("nan"))
    assert _call(L, N, O, V, band, x.data_ptr(), y_static.data_ptr(), n, stream.cuda_stream) == 0
    plan = vbw.Plan(N, O, V)
    y_ref = torch.full_like(x, float("nan"))
    vbw.Batch([(plan, x, y_ref, band)]).run(stream)
    torch.cuda.synchronize()
    assert torch.equal(y_static.view(torch.float32), y_ref.view(torch.float32))


@pytest.mark.gpu
def test_no_alloc_call_leaves_device_memory_unchanged(cuda):
    """After a warm-up call, a call with another geometry (so its tables are rebuilt) and a call
    that repeats it (tables reused) leave the device's free memory exactly where it was."""
    torch = cuda
    L = vbw.lib()
    stream = torch.cuda.current_stream()
    n = 200_000
    x = torch.from_numpy(wl.complex_gaussian(43, 0, n)).cuda()
    y = torch.empty_like(x)
    y2 = torch.empty_like(x)
    V1, V2 = wl.transition_table(44, 12), wl.transition_table(45, 10)
    assert _call(L, 512, 128, V1, 50, x.data_ptr(), y.data_ptr(), n, stream.cuda_stream) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _call(L, 2048, 512, V2, 300, x.data_ptr(), y.data_ptr(), n, stream.cuda_stream) == 0
    assert _call(L, 2048, 512, V2, 300, x.data_ptr(), y2.data_ptr(), n, stream.cuda_stream) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(y.view(torch.float32), y2.view(torch.float32))

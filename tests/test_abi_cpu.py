"""The C ABI on a machine without a GPU: the library builds, loads and exports every entry point
include/vbw.h declares, and argument validation answers before any CUDA call is made."""
import ctypes

import numpy as np
import pytest

from paper_2406_14116_gb300 import build as vbw_build
from paper_2406_14116_gb300 import vbw


@pytest.fixture(scope="module")
def L():
    vbw_build.build()
    return vbw.lib()


def test_every_declared_symbol_is_exported(L):
    names = vbw.declared_functions()
    assert "vbw_plan" in names and "vbw_filter" in names and "vbw_set_bandwidth" in names
    for name in names:
        assert hasattr(L, name), name


def test_version_and_empty_error(L):
    assert "sm_103a" in vbw.vbw_version()
    assert isinstance(vbw.vbw_last_error(), str)


@pytest.mark.parametrize("N,overlap,LV", [
    (100, 24, 6),      # N not a power of two
    (64, 16, 6),       # N below 128
    (4096, 1024, 12),  # N above 2048
    (256, -2, 6),      # negative overlap
    (256, 0, 6),       # no overlap
    (256, 256, 6),     # overlap = N
    (256, 64, 0),      # empty transition table
    (256, 64, 127),    # L_V above N/2 - 2
])
def test_plan_rejects_bad_geometry(L, N, overlap, LV):
    with pytest.raises(vbw.VbwError) as e:
        vbw.vbw_plan(N, overlap, np.linspace(0.9, 0.1, max(LV, 1))[:LV] if LV else np.zeros(0))
    assert e.value.code == 1


def test_plan_rejects_nonfinite_V(L):
    V = np.array([0.9, np.nan, 0.1])
    with pytest.raises(vbw.VbwError) as e:
        vbw.vbw_plan(256, 64, V)
    assert e.value.code == 1 and "finite" in str(e.value)


def test_plan_rejects_unknown_precision(L):
    with pytest.raises(vbw.VbwError) as e:
        vbw.vbw_plan(256, 64, np.linspace(0.9, 0.1, 6), precision=7)
    assert e.value.code == 1


def test_null_handles_are_rejected(L):
    for f, args in ((L.vbw_filter, (None, None, None, 1)), (L.vbw_set_bandwidth, (None, 3)),
                    (L.vbw_stream_reset, (None, 3)), (L.vbw_batch_run, (None, None)),
                    (L.vbw_plan_destroy, (None,)), (L.vbw_stream_destroy, (None,)),
                    (L.vbw_filter_ola, (None, None, None, 100, 1, 5, None, None)),
                    (L.vbw_ptvir_error, (None, None, 1, None, None, 10, None, None, None))):
        assert f(*args) == 1
        assert vbw.vbw_last_error()


def test_valid_plan_without_gpu_reports_cuda_error(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    V = np.linspace(0.9, 0.1, 6)
    rc = L.vbw_plan(256, 64, V.ctypes.data_as(ctypes.c_void_p), 6, 0, ctypes.byref(h))
    assert rc == 4 and h.value is None


def test_host_pointer_arrays_for_run_host():
    """vbw_batch_run_host takes the signals' host arrays or, for repeated runs, their address
    array from host_pointers(): the addresses, in order; non-contiguous arrays are refused."""
    import numpy as np
    from paper_2406_14116_gb300 import vbw as V
    buf = np.zeros(1000, np.complex64)
    views = [buf[0:10], buf[10:250], buf[250:1000]]
    p = V.host_pointers(views)
    assert p.dtype == np.uintp and list(p) == [v.ctypes.data for v in views]
    assert V._pointer_array(p) is p or np.array_equal(V._pointer_array(p), p)
    assert np.array_equal(V._pointer_array(views), p)
    with pytest.raises(ValueError):
        V.host_pointers([buf[::2]])

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libvbw.so")


import numpy as np  # noqa: E402
import pytest  # noqa: E402

FP32_RMS_TOL = 2e-6        # RMS relative error bound of the FP32 path vs the FP64 oracle
FP32_ELEM_TOL = 2e-5       # per-sample bound, relative to the RMS of the reference output


def rms_rel(y, ref):
    y = np.asarray(y, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    den = np.sum(np.abs(ref) ** 2)
    return float(np.sqrt(np.sum(np.abs(y - ref) ** 2) / den)) if den > 0 else float(np.abs(y).max(initial=0))


def assert_parity(y, ref, rms_tol=FP32_RMS_TOL, elem_tol=FP32_ELEM_TOL, what=""):
    """RMS relative error within rms_tol and every sample within elem_tol * rms(ref)."""
    y = np.asarray(y, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    assert y.shape == ref.shape, (y.shape, ref.shape)
    if ref.size == 0:
        return
    assert np.isfinite(y).all(), f"{what}: non-finite output"
    err = rms_rel(y, ref)
    assert err <= rms_tol, f"{what}: RMS relative error {err:.3e} > {rms_tol:.1e}"
    scale = np.sqrt(np.mean(np.abs(ref) ** 2))
    worst = np.abs(y - ref).max()
    assert worst <= elem_tol * scale, f"{what}: worst sample error {worst:.3e} > {elem_tol * scale:.3e}"


@pytest.fixture(scope="session")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_14116_gb300 import build
    build.build()
    torch.cuda.init()
    return torch

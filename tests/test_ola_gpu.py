"""GPU parity of vbw_filter_ola (overlap-add with the HFSO coefficients) against the FP64 OLA
oracle, through the C ABI, at the FP32 tolerances of the OLS path (RMS relative error <= 2e-6,
every sample within 2e-5 x RMS)."""
import numpy as np
import pytest

import oracle
from conftest import assert_parity
from paper_2406_14116_gb300 import vbw
from paper_2406_14116_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def run_ola(torch, plan, x2d, band=0, bands=None):
    xd = torch.from_numpy(np.ascontiguousarray(x2d)).cuda()
    yd = torch.full_like(xd, float("nan"))
    bd = None if bands is None else torch.from_numpy(np.ascontiguousarray(bands, dtype=np.int32)).cuda()
    vbw.vbw_filter_ola(plan.handle, xd, yd, x2d.shape[1], x2d.shape[0], band, bd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("N,overlap", [(128, 32), (256, 64), (512, 128), (1024, 256), (2048, 512),
                                       (256, 2), (512, 256), (1024, 100)])
def test_ola_matches_oracle(cuda, N, overlap):
    """Three signals of a ragged length (many tiles, warps whose ranges start inside a signal),
    a band per block drawn over the whole valid range."""
    torch = cuda
    g = np.random.default_rng(N + overlap)
    LV = 12 if N >= 256 else 6
    V = np.sort(g.uniform(0.0, 1.0, LV))[::-1]
    M = N - overlap
    nblk = 40 if N <= 512 else 14
    T = nblk * M + M // 3 + 1
    nb = (T + M - 1) // M
    kmax = N // 2 - LV - 1
    x = np.stack([wl.complex_gaussian(7, c, T) for c in range(3)])
    bands = g.integers(1, kmax + 1, (3, nb)).astype(np.int32)
    plan = vbw.Plan(N, overlap, V)
    y = run_ola(torch, plan, x, bands=bands)
    for c in range(3):
        ref = oracle.filter_ola(N, overlap, V, bands[c], x[c])
        assert_parity(y[c], ref, what=f"N={N} O={overlap} signal {c}")
    # one band for every block
    y1 = run_ola(torch, plan, x[:1], band=kmax)
    assert_parity(y1[0], oracle.filter_ola(N, overlap, V, kmax, x[0]), what="fixed band")


@pytest.mark.parametrize("N", [128, 1024])
def test_ola_long_signals_sampled(cuda, N):
    """Signals long enough that every warp walks many tiles (tails handed on in shared memory),
    checked on runs of blocks at seeded positions; the oracle runs over the run and the block
    before it (only the previous block's tail reaches a block)."""
    torch = cuda
    overlap, LV = N // 4, 12
    M = N - overlap
    V = wl.transition_table(2, LV)
    nsig, T = 4, 3000 * M + 17
    nb = (T + M - 1) // M
    g = np.random.default_rng(N)
    x = np.stack([wl.complex_gaussian(8, c, T) for c in range(nsig)])
    bands = np.stack([wl.band_schedule(2, c, nb, 16, 32, N // 2 - LV - 1) for c in range(nsig)])
    plan = vbw.Plan(N, overlap, V)
    y = run_ola(torch, plan, x, bands=bands)
    assert np.isfinite(y).all()
    for c in range(nsig):
        for b0 in [0, int(g.integers(1, nb - 20)), nb - 6]:
            lo = max(0, b0 - 1)
            hi = min(T, (b0 + 6) * M)
            ref = oracle.filter_ola(N, overlap, V, bands[c][lo:], x[c][lo * M: hi])
            assert_parity(y[c][b0 * M: hi], ref[(b0 - lo) * M:], what=f"signal {c} block {b0}")


def test_ola_argument_errors(cuda):
    torch = cuda
    L = vbw.lib()
    V = np.linspace(0.9, 0.1, 6)
    x = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    for N, O in [(256, 63), (256, 192)]:   # odd overlap; overlap above N/2
        plan = vbw.Plan(N, O, V)
        assert L.vbw_filter_ola(plan.handle, x.data_ptr(), y.data_ptr(), 1000, 1, 5, None, None) == 8
    plan = vbw.Plan(256, 64, V)
    assert L.vbw_filter_ola(plan.handle, x.data_ptr(), y.data_ptr(), 1000, 1, 0, None, None) == 2
    assert L.vbw_filter_ola(plan.handle, x.data_ptr(), y.data_ptr(), 1000, 1, 128 - 6, None, None) == 2
    assert L.vbw_filter_ola(plan.handle, x.data_ptr(), x.data_ptr() + 800, 1000, 1, 5, None, None) == 1
    assert L.vbw_filter_ola(plan.handle, x.data_ptr() + 4, y.data_ptr(), 1000, 1, 5, None, None) == 1
    assert L.vbw_filter_ola(plan.handle, x.data_ptr(), y.data_ptr(), 0, 1, 5, None, None) == 0
    assert L.vbw_filter_ola(plan.handle, x.data_ptr(), y.data_ptr(), -1, 1, 5, None, None) == 1
    tc = vbw.Plan(256, 64, V, vbw.VBW_PREC_BF16_SPLIT)
    assert L.vbw_filter_ola(tc.handle, x.data_ptr(), y.data_ptr(), 1000, 1, 5, None, None) == 8

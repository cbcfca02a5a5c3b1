"""Sizes past 32-bit sample indices: one stream of 2^31 + 777 complex64 samples (16 GiB in, 16 GiB
out) through the stream API and a batch, checked against the FP64 oracle on sampled blocks at
the start, the middle (around sample 2^31) and the ragged end."""
import numpy as np
import pytest

import oracle
from conftest import assert_parity
from paper_2406_14116_gb300 import vbw
from paper_2406_14116_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_stream_beyond_two_to_the_31_samples(cuda):
    torch = cuda
    free, _ = torch.cuda.mem_get_info()
    T = (1 << 31) + 777
    if free < 3 * 8 * T + (4 << 30):
        pytest.skip("needs about 56 GB of free device memory")
    N, O = 1024, 256
    M = N - O
    V = wl.transition_table(11, 12)
    plan = vbw.Plan(N, O, V)
    g = torch.Generator(device="cuda").manual_seed(11)
    x = torch.randn(T, dtype=torch.complex64, device="cuda", generator=g)
    y = torch.zeros_like(x)
    nb_full = T // M
    s = vbw.Stream(plan, 200)
    s.set_bandwidth_at(nb_full // 2 + 1, 350)
    s.filter(x[:nb_full * M], y[:nb_full * M], nb_full)
    s.flush(x[nb_full * M:], y[nb_full * M:], T - nb_full * M)
    torch.cuda.synchronize()
    mid = (1 << 31) // M
    for b0, cnt in ((0, 8), (mid - 4, 8), (nb_full // 2 - 2, 6), (nb_full - 5, 6)):
        lo, hi = b0 * M, min(T, (b0 + cnt) * M)
        xs = x[max(0, lo - O):hi].cpu().numpy()
        tail = None
        if lo >= O:
            tail, xs = xs[:O], xs[O:]
        bands = [200 if b0 + k <= nb_full // 2 else 350 for k in range(cnt)]
        ref = oracle.filter(N, O, V, np.array(bands, dtype=np.int32), xs, tail=tail)
        assert_parity(y[lo:hi].cpu().numpy(), ref, what=f"blocks {b0}..{b0 + cnt}")
    # the same signal as a one-signal batch (job descriptor with 64-bit sample counts)
    y2 = torch.zeros_like(x)
    b = vbw.Batch([(plan, x, y2, 200)])
    b.run()
    torch.cuda.synchronize()
    for lo in (0, (mid - 2) * M, (nb_full - 3) * M):
        hi = min(T, lo + 4 * M)
        xs = x[max(0, lo - O):hi].cpu().numpy()
        tail = None
        if lo >= O:
            tail, xs = xs[:O], xs[O:]
        ref = oracle.filter(N, O, V, 200, xs, tail=tail)
        assert_parity(y2[lo:hi].cpu().numpy(), ref, what=f"batch from {lo}")


def test_overlap_add_beyond_two_to_the_31_samples(cuda):
    """vbw_filter_ola on two signals of 2^30 + 333 samples each (2^31 + 666 in all, so the second
    signal's samples sit past 32-bit indices of the back-to-back rows), against the OLA oracle on
    sampled runs: each run starts one block early, since only the previous block's tail reaches
    a block."""
    torch = cuda
    free, _ = torch.cuda.mem_get_info()
    T = (1 << 30) + 333
    if free < 2 * 8 * 2 * T + (4 << 30):
        pytest.skip("needs about 38 GB of free device memory")
    N, O = 1024, 256
    M = N - O
    V = wl.transition_table(12, 12)
    plan = vbw.Plan(N, O, V)
    g = torch.Generator(device="cuda").manual_seed(12)
    x = torch.randn((2, T), dtype=torch.complex64, device="cuda", generator=g)
    y = torch.zeros_like(x)
    vbw.vbw_filter_ola(plan.handle, x, y, T, 2, 300)
    torch.cuda.synchronize()
    nb = (T + M - 1) // M
    for c in range(2):
        for b0 in (0, nb // 2, nb - 4):
            lo = max(0, b0 - 1)
            hi = min(T, (b0 + 4) * M)
            ref = oracle.filter_ola(N, O, V, 300, x[c, lo * M:hi].cpu().numpy())
            assert_parity(y[c, b0 * M:hi].cpu().numpy(), ref[(b0 - lo) * M:], what=f"signal {c} block {b0}")

"""The designed HFSO filter through the CUDA path: the minimax V of the paper's example
(N=128, L=33, M=96, Delta_N=16, b_N in [48, 55]) keeps every output within delta of the desired
response on the GPU. Passband tones leave with unit magnitude, stopband tones below -60 dB."""
import math

import numpy as np
import pytest

from paper_2406_14116_gb300 import design
from paper_2406_14116_gb300 import vbw

pytestmark = pytest.mark.gpu


def test_designed_filter_meets_minus_60_db_on_the_gpu(cuda):
    torch = cuda
    d = design.design_transition(128, 33, 16, 48, 55, K=1000)
    N, O, M = 128, 32, 96
    plan = vbw.Plan(N, O, d.V)
    t = np.arange(60 * M)
    eps = 2e-5                                   # FP32 arithmetic and complex64 input
    for bN in (48, 51, 55):
        k1, _ = design.band_bins(bN, 16)
        wc, ws = (bN - 8) * 2 * math.pi / N, (bN + 8) * 2 * math.pi / N
        tones = [(0.1, True), (0.5 * wc, True), (0.99 * wc, True),
                 (1.01 * ws, False), (0.5 * (ws + math.pi), False), (math.pi, False)]
        for w, passband in tones:
            x = np.exp(1j * w * t).astype(np.complex64)
            xd = torch.from_numpy(x).cuda()
            yd = torch.zeros_like(xd)
            s = vbw.Stream(plan, k1)
            s.filter(xd, yd, len(x) // M)
            torch.cuda.synchronize()
            mag = np.abs(yd.cpu().numpy()[2 * M:])   # past the zero history of the first blocks
            if passband:
                assert np.abs(mag - 1).max() <= d.delta + eps, (bN, w)
            else:
                assert mag.max() <= d.delta + eps, (bN, w)
            assert d.delta <= 1e-3
            s.close()


def test_gpu_search_reproduces_the_cpu_design(cuda):
    """design_transition_gpu (the search over bands, phases and frequencies by vbw_ptvir_error)
    solves the same eq. (minimax) as the CPU designer: on the paper's example both deltas lie
    within the stopping tolerance (1e-3 relative) of the minimax value, so within 2e-3 of each
    other, and below the paper's -60 dB."""
    cpu = design.design_transition(128, 33, 16, 48, 55, K=1000)
    gpu = design.design_transition_gpu(128, 33, 16, 48, 55, K=1000)
    assert gpu.delta <= 1e-3
    assert abs(gpu.delta - cpu.delta) <= 2.5e-3 * cpu.delta, (gpu.delta, cpu.delta)


def test_gpu_search_designs_the_channel_geometry(cuda):
    """The channel workload's filter (N=1024, L=257 i.e. overlap 256, L_V=12, k1 in 32..480: 449
    bands x 768 output phases x 1000 frequencies) is designed through the GPU search. The FP64
    oracle's PTVIR errors at sampled bands and frequencies, over every phase, stay within the
    returned delta."""
    import time
    import oracle
    t0 = time.perf_counter()
    d = design.design_transition_gpu(1024, 257, 13, 37, 485, K=1000)
    secs = time.perf_counter() - t0
    print(f"channel geometry: delta={d.delta:.3e} ({20 * np.log10(d.delta):.1f} dB) in {d.iterations} "
          f"rounds, {secs:.1f} s")
    assert d.delta < 3e-3             # measured 2.34e-3 (-52.6 dB) in 19 rounds
    g = np.random.default_rng(5)
    for bN in g.choice(np.arange(37, 486), 2, replace=False):
        k1, _ = design.band_bins(int(bN), 13)
        w, dd = design.grid(int(bN), 13, 1024, 1000)
        cols = g.choice(len(w), 12, replace=False)
        E = oracle.ptvir_errors(1024, 256, d.V, k1, w[cols], dd[cols])
        # the oracle rounds V to float32 as the filter does: allow that perturbation
        assert E.max() <= d.delta * (1 + 1e-3) + 1e-6, (bN, E.max(), d.delta)

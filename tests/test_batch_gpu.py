"""Batched filtering of many streams with mixed lengths, transform sizes and bands (one prepared
batch, single-plan or mixed-plan persistent launches, CUDA-graph replay), the bounded-wait failure
path, all through the C ABI and checked against the FP64 oracle."""
import os

import numpy as np
import pytest

import oracle
from conftest import assert_parity
from paper_2406_14116_gb300 import vbw
from paper_2406_14116_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def mixed_batch(torch, nstreams=40, seed=33, log2_lo=10.0, log2_hi=15.0):
    w = wl.mixed(seed=seed, nstreams=nstreams, log2_lo=log2_lo, log2_hi=log2_hi)
    plans = {N: vbw.Plan(N, N // 4, w.V) for N in (128, 256, 512, 1024, 2048)}
    xs = [torch.from_numpy(s.x).cuda() for s in w.signals]
    ys = [torch.full_like(x, float("nan")) for x in xs]
    rows = [(plans[s.N], x, y, s.band) for s, x, y in zip(w.signals, xs, ys)]
    return w, plans, xs, ys, vbw.Batch(rows)


def test_mixed_batch_all_modes_match_oracle_and_each_other(cuda):
    torch = cuda
    w, plans, xs, ys, b = mixed_batch(torch)
    outs = {}
    for mode in (vbw.VBW_BATCH_PER_PLAN, vbw.VBW_BATCH_MIXED, vbw.VBW_BATCH_AUTO):
        for y in ys:
            y.fill_(float("nan"))
        b.set_mode(mode)
        b.run()
        torch.cuda.synchronize()
        outs[mode] = [y.cpu().numpy() for y in ys]
        if mode == vbw.VBW_BATCH_MIXED:
            assert b.launches == 2      # one mixed launch + the N = 2048 plan beside it
        if mode == vbw.VBW_BATCH_PER_PLAN:
            assert b.launches == 5
    for s, y in zip(w.signals, outs[vbw.VBW_BATCH_PER_PLAN]):
        ref = oracle.filter(s.N, s.overlap, w.V, s.band, s.x)
        assert_parity(y, ref, what=f"stream {s.stream} N={s.N} len={len(s.x)}")
    for mode in (vbw.VBW_BATCH_MIXED, vbw.VBW_BATCH_AUTO):
        for a, c in zip(outs[vbw.VBW_BATCH_PER_PLAN], outs[mode]):
            np.testing.assert_array_equal(a, c)


def test_mixed_share_and_single_stream_batch(cuda):
    torch = cuda
    w, plans, xs, ys, b = mixed_batch(torch, nstreams=12, seed=7)
    b.set_mode(vbw.VBW_BATCH_MIXED, 0.5)
    b.run()
    torch.cuda.synchronize()
    for s, y in zip(w.signals, ys):
        assert_parity(y.cpu().numpy(), oracle.filter(s.N, s.overlap, w.V, s.band, s.x))
    with pytest.raises(vbw.VbwError):
        b.set_mode(7)
    with pytest.raises(vbw.VbwError):
        b.set_mode(vbw.VBW_BATCH_MIXED, 1.5)


def test_batch_replays_in_cuda_graph(cuda):
    torch = cuda
    w, plans, xs, ys, b = mixed_batch(torch, nstreams=24, seed=5)
    b.set_mode(vbw.VBW_BATCH_MIXED)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(s)                     # warm-up (lazy attribute setting happens outside capture)
    torch.cuda.synchronize()
    ref = [y.clone() for y in ys]
    for y in ys:
        y.fill_(float("nan"))
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(s)
    for _ in range(3):
        for y in ys:
            y.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for a, c in zip(ref, ys):
            assert torch.equal(a, c)


def test_empty_and_tiny_signals_in_batch(cuda):
    torch = cuda
    V = wl.transition_table(3, 12)
    p1 = vbw.Plan(256, 64, V)
    p2 = vbw.Plan(1024, 256, V)
    sig = [np.zeros(0, np.complex64), wl.complex_gaussian(3, 1, 5), wl.complex_gaussian(3, 2, 192),
           wl.complex_gaussian(3, 3, 193), wl.complex_gaussian(3, 4, 3000)]
    plans = [p1, p1, p1, p2, p2]
    xs = [torch.from_numpy(x).cuda() if len(x) else torch.zeros(0, dtype=torch.complex64, device="cuda")
          for x in sig]
    ys = [torch.zeros_like(x) for x in xs]
    b = vbw.Batch([(p, x, y, 9) for p, x, y in zip(plans, xs, ys)])
    b.run()
    torch.cuda.synchronize()
    for p, x, y in zip(plans, sig, ys):
        if len(x):
            assert_parity(y.cpu().numpy(), oracle.filter(p.N, p.overlap, V, 9, x))


@pytest.mark.parametrize("N", [256, 512])
def test_bounded_wait_runs_out_and_reports(cuda, N):
    """A wait that nothing ends (test hook: the tensor-core kernel issues no MMAs, so no
    accumulator completes) runs out after its bound: the kernel sets the status word and the CTA
    frees its tensor memory and returns; the context stays usable and the next launch is correct.
    (The FP32 kernels have no device-side waits.)"""
    torch = cuda
    O = N // 4
    M = N - O
    nb = 8000                     # several tiles per CTA
    V = wl.transition_table(4, 12)
    plan = vbw.Plan(N, O, V, precision=vbw.VBW_PREC_BF16_SPLIT)
    x = wl.complex_gaussian(4, 0, nb * M)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    assert vbw.vbw_plan_status(plan.handle, clear=True) == 0
    vbw.vbw_debug_set(1)
    try:
        s = vbw.Stream(plan, 100)
        s.filter(xd, yd, nb)
        torch.cuda.synchronize()
    finally:
        vbw.vbw_debug_set(0)
    rc, flags = vbw.vbw_plan_status_raw(plan.handle, clear=True)
    assert rc == 5 and flags & 1
    assert vbw.vbw_plan_status(plan.handle) == 0
    s = vbw.Stream(plan, 100)
    s.filter(xd, yd, nb)
    torch.cuda.synchronize()
    assert vbw.vbw_plan_status(plan.handle) == 0
    y = yd.cpu().numpy()
    for b0, cnt in ((0, 64), (nb // 2, 32), (nb - 64, 64)):
        ref = oracle.filter(N, O, V, 100, x, blocks=(b0, cnt))
        sl = slice(b0 * M, (b0 + cnt) * M)
        assert_parity(y[sl], ref[sl], rms_tol=1e-5, elem_tol=2e-4, what=f"blocks {b0}..{b0 + cnt}")


def test_fp32_kernels_have_no_device_waits(cuda):
    """The FP32 kernels wait on nothing: under the same test hook (debug bit 0, short wait limit)
    an FP32 plan filters correctly and its status word stays clear."""
    torch = cuda
    N, O = 1024, 256
    M = N - O
    nb = 4000
    V = wl.transition_table(5, 12)
    plan = vbw.Plan(N, O, V)
    x = wl.complex_gaussian(5, 0, nb * M)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    assert vbw.vbw_plan_status(plan.handle, clear=True) == 0
    vbw.vbw_debug_set(1)
    try:
        s = vbw.Stream(plan, 200)
        s.filter(xd, yd, nb)
        torch.cuda.synchronize()
    finally:
        vbw.vbw_debug_set(0)
    assert vbw.vbw_plan_status(plan.handle) == 0
    y = yd.cpu().numpy()
    for b0, cnt in ((0, 32), (nb - 32, 32)):
        ref = oracle.filter(N, O, V, 200, x, blocks=(b0, cnt))
        sl = slice(b0 * M, (b0 + cnt) * M)
        assert_parity(y[sl], ref[sl], what=f"blocks {b0}..{b0 + cnt}")


def test_tune_set_changes_shape_not_result(cuda):
    torch = cuda
    N, O = 512, 128
    M = N - O
    V = wl.transition_table(9, 12)
    plan = vbw.Plan(N, O, V)
    x = wl.complex_gaussian(9, 0, 300 * M)
    xd = torch.from_numpy(x).cuda()
    outs = []
    try:
        for w in (4, 8, 0):
            vbw.vbw_tune_set(N, w)
            yd = torch.zeros_like(xd)
            vbw.Stream(plan, 77).filter(xd, yd, 300)
            torch.cuda.synchronize()
            outs.append(yd.cpu().numpy())
    finally:
        vbw.vbw_tune_set(N, 0)
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])
    with pytest.raises(vbw.VbwError):
        vbw.vbw_tune_set(300, 4)
    with pytest.raises(vbw.VbwError):
        vbw.vbw_tune_set(512, 6)


def test_signals_at_odd_offsets_of_one_buffer(cuda):
    """Signals packed back to back in one device buffer start at arbitrary sample offsets, so
    some are only 8-byte aligned: the bulk L2 prefetch must realign (or skip) those, and the
    results must not change. Also covers vbw_batch_run_host on packed buffers."""
    torch = cuda
    w = wl.mixed(seed=21, nstreams=30, log2_lo=11.0, log2_hi=14.5)
    lens = [len(s.x) for s in w.signals]
    offs = np.concatenate([[1], 1 + np.cumsum(lens)])         # odd start: every base shifts
    assert any(o % 2 for o in offs[:-1])
    total = int(offs[-1]) + 1
    host = np.zeros(total, np.complex64)
    for s, o in zip(w.signals, offs):
        host[o:o + len(s.x)] = s.x
    d_in = torch.from_numpy(host).cuda()
    d_out = torch.full_like(d_in, float("nan"))
    plans = {N: vbw.Plan(N, N // 4, w.V) for N in (128, 256, 512, 1024, 2048)}
    rows = [(plans[s.N], d_in[o:o + len(s.x)], d_out[o:o + len(s.x)], s.band)
            for s, o in zip(w.signals, offs)]
    b = vbw.Batch(rows)
    for mode in (vbw.VBW_BATCH_PER_PLAN, vbw.VBW_BATCH_MIXED):
        d_out.fill_(float("nan"))
        b.set_mode(mode)
        b.run()
        torch.cuda.synchronize()
        y = d_out.cpu().numpy()
        for s, o in zip(w.signals, offs):
            assert_parity(y[o:o + len(s.x)], oracle.filter(s.N, s.overlap, w.V, s.band, s.x),
                          what=f"stream {s.stream} offset {o}")
    hout = np.zeros_like(host)
    b.run_host([host[o:o + len(s.x)] for s, o in zip(w.signals, offs)],
               [hout[o:o + len(s.x)] for s, o in zip(w.signals, offs)])
    for s, o in zip(w.signals, offs):
        np.testing.assert_array_equal(hout[o:o + len(s.x)], y[o:o + len(s.x)])


def test_misaligned_pointer_is_rejected(cuda):
    torch = cuda
    plan = vbw.Plan(256, 64, wl.transition_table(1, 6))
    buf = torch.zeros(4096, dtype=torch.complex64, device="cuda")
    s = vbw.Stream(plan, 10)
    with pytest.raises(vbw.VbwError) as e:
        vbw.vbw_filter(s.handle, buf.data_ptr() + 4, buf[2048:].data_ptr(), 1)
    assert e.value.code == 1


def test_run_host_zero_copy_split_kernel(cuda, monkeypatch):
    """N = 2048 batches through the split kernel (forced for this size) with pinned host buffers:
    the kernel reads and writes host memory directly (no L2 prefetch), and the output equals the
    device path's bit for bit and the oracle within the FP32 gate."""
    monkeypatch.setenv("VBW_SPLIT2048", "2")
    torch = cuda
    V = wl.transition_table(58, 12)
    plan = vbw.Plan(2048, 512, V)
    rng = np.random.default_rng(58)
    xs = [wl.complex_gaussian(58, i, int(n)) for i, n in enumerate(rng.integers(1000, 60000, 5))]
    bands = [int(b) for b in rng.integers(1, wl.max_band(2048, 12) + 1, 5)]
    dx = [torch.from_numpy(x).cuda() for x in xs]
    dy = [torch.full_like(x, float("nan")) for x in dx]
    b = vbw.Batch([(plan, x, y, k) for x, y, k in zip(dx, dy, bands)])
    b.run()
    torch.cuda.synchronize()
    hin = [torch.from_numpy(x).pin_memory() for x in xs]
    hout = [torch.zeros_like(h).pin_memory() for h in hin]
    b.run_host([h.numpy() for h in hin], [h.numpy() for h in hout])
    for x, y, h, k in zip(xs, dy, hout, bands):
        np.testing.assert_array_equal(y.cpu().numpy(), h.numpy())
        assert_parity(h.numpy(), oracle.filter(2048, 512, V, k, x), what="split zero copy")


def test_run_host_zero_copy_matches_device_path(cuda):
    """Pinned host buffers: the kernels work on host memory directly (zero copy); pageable
    buffers: staged copies. Both give the device path's output bit for bit."""
    torch = cuda
    w, plans, xs, ys, b = mixed_batch(torch, nstreams=20, seed=12)
    b.run()
    torch.cuda.synchronize()
    dev = [y.cpu().numpy() for y in ys]
    for mode in (vbw.VBW_BATCH_PER_PLAN, vbw.VBW_BATCH_MIXED):
        b.set_mode(mode)
        hin = [torch.from_numpy(s.x).pin_memory() for s in w.signals]
        hout = [torch.zeros_like(h).pin_memory() for h in hin]
        b.run_host([h.numpy() for h in hin], [h.numpy() for h in hout])
        for a, h in zip(dev, hout):
            np.testing.assert_array_equal(a, h.numpy())
        pin = [np.ascontiguousarray(s.x) for s in w.signals]
        pout = [np.zeros_like(p) for p in pin]
        b.run_host(pin, pout)
        for a, h in zip(dev, pout):
            np.testing.assert_array_equal(a, h)


def test_tune_shapes_n2048_probes_four_step_and_restores_switch(cuda, monkeypatch):
    """The autotuner's N = 2048 probe runs the 64 x 32 four-step kernel (the shape it sets is that
    kernel's; the split kernel has its own) and leaves the VBW_SPLIT2048 setting as it found it."""
    from paper_2406_14116_gb300 import tune
    torch = cuda
    monkeypatch.setenv("VBW_SPLIT2048", "2")
    out = tune.tune_shapes(torch, Ns=(2048,), nch=2, nsamples=1 << 16, reps=2)
    assert os.environ["VBW_SPLIT2048"] == "2"
    d = out["2048"]
    assert d["warps"] in tune.WARPS and d["ctas_per_sm"] in tune.CTAS
    assert len(d["table"]) == len(tune.WARPS) * len(tune.CTAS) and all(r["ms"] > 0 for r in d["table"])
    monkeypatch.delenv("VBW_SPLIT2048")
    tune.tune_shapes(torch, Ns=(2048,), nch=2, nsamples=1 << 16, reps=2)
    assert "VBW_SPLIT2048" not in os.environ

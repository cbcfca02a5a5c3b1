"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

FP32 path: RMS relative error <= 2e-6 per stream and every sample within 2e-5 of the reference
RMS; band indexing bit-exact; chunking, checkpoints and host-buffer calls bitwise identical to a
single device call.
"""
import numpy as np
import pytest

import oracle
from conftest import assert_parity
from paper_2406_14116_gb300 import vbw
from paper_2406_14116_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ALL_N = (128, 256, 512, 1024, 2048)


def to_dev(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run_stream(torch, plan, x, band, changes=(), chunks=None):
    """Filters x through a Stream: full blocks with vbw_filter (optionally in chunks), the rest
    with vbw_flush. changes: (block, k1) pairs scheduled with vbw_set_bandwidth_at."""
    M = plan.M
    s = vbw.Stream(plan, band)
    for b, k in changes:
        s.set_bandwidth_at(b, k)
    xd = to_dev(torch, x)
    yd = torch.zeros_like(xd)
    nfull = len(x) // M
    if chunks is None:
        chunks = [nfull]
    b0 = 0
    for nb in chunks:
        s.filter(xd[b0 * M:(b0 + nb) * M], yd[b0 * M:(b0 + nb) * M], nb)
        b0 += nb
    assert b0 == nfull
    rem = len(x) - nfull * M
    s.flush(xd[nfull * M:], yd[nfull * M:], rem)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    s.close()
    return y


def bands_from_changes(nblocks, band, changes):
    out = np.full(nblocks, band, dtype=np.int32)
    for b, k in sorted(changes):
        out[b:] = k
    return out


@pytest.mark.parametrize("N", ALL_N)
@pytest.mark.parametrize("LV", [1, 6, 12, "max"])
def test_band_indexing_bit_exact(cuda, N, LV):
    """H_R(k) applied by the kernel code for every valid band equals eq. (FS_Hk_real) with V
    rounded to float32, bit for bit."""
    LV = N // 2 - 2 - 1 if LV == "max" else LV
    V = wl.transition_table(100 + N, LV)
    plan = vbw.Plan(N, N // 4, V)
    bands = range(1, wl.max_band(N, LV) + 1)
    if len(bands) > 300:
        bands = sorted(set(list(range(1, 100)) + list(range(len(bands) - 100, len(bands) + 1)) +
                           list(np.random.default_rng(N).integers(1, len(bands) + 1, 100))))
    for k1 in bands:
        got = vbw.vbw_debug_export_HR(plan.handle, int(k1))
        want = oracle.HR(N, V, int(k1)).astype(np.float32)
        np.testing.assert_array_equal(got, want, err_msg=f"N={N} L_V={LV} k1={k1}")
    for bad in (0, wl.max_band(N, LV) + 1):
        with pytest.raises(vbw.VbwError) as e:
            vbw.vbw_debug_export_HR(plan.handle, bad)
        assert e.value.code == 2


@pytest.mark.parametrize("LV", [1, 12, "max"])
def test_band_indexing_bit_exact_four_step_2048(cuda, monkeypatch, LV):
    """N = 2048 with overlap N/4 exports the split kernel's gain tables and bin mapping (above);
    with VBW_SPLIT2048=0 it exports the 64 x 32 four-step kernel's, which also serves other
    overlaps and real signals. Both must equal eq. (FS_Hk_real) bit for bit."""
    monkeypatch.setenv("VBW_SPLIT2048", "0")
    N = 2048
    LV = N // 2 - 2 - 1 if LV == "max" else LV
    V = wl.transition_table(300 + LV, LV)
    plan = vbw.Plan(N, N // 4, V)
    top = wl.max_band(N, LV)
    cand = [1, 2, 3, top - 1, top] + list(np.random.default_rng(LV).integers(1, top + 1, 60))
    for k1 in sorted(set(int(k) for k in cand if 1 <= k <= top)):
        got = vbw.vbw_debug_export_HR(plan.handle, int(k1))
        want = oracle.HR(N, V, int(k1)).astype(np.float32)
        np.testing.assert_array_equal(got, want, err_msg=f"four-step N=2048 L_V={LV} k1={k1}")


GEOMS = [(128, 32), (128, 2), (128, 126), (256, 64), (256, 100), (512, 128), (512, 384),
         (1024, 256), (1024, 6), (2048, 512), (2048, 30), (2048, 1800)]


@pytest.mark.parametrize("N,overlap", GEOMS)
def test_stream_parity_ragged(cuda, N, overlap):
    """Several tiles and CTAs, a ragged final block, random band; all overlaps the ABI allows
    (small, N/4, large)."""
    torch = cuda
    M = N - overlap
    LV = 12 if N > 128 else 6
    g = np.random.default_rng(N + overlap)
    V = wl.transition_table(N * 7 + overlap, LV)
    k1 = int(g.integers(1, wl.max_band(N, LV) + 1))
    nblocks = max(40, 3000 // (N // 128))
    T = nblocks * M + int(g.integers(1, M))
    x = wl.complex_gaussian(N + overlap, 1, T)
    plan = vbw.Plan(N, overlap, V)
    y = run_stream(torch, plan, x, k1)
    ref = oracle.filter(N, overlap, V, k1, x)
    assert_parity(y, ref, what=f"N={N} O={overlap}")


@pytest.mark.parametrize("N", ALL_N)
def test_edge_bands(cuda, N):
    torch = cuda
    O = N // 4
    M = N - O
    LV = 12
    V = wl.transition_table(N, LV)
    plan = vbw.Plan(N, O, V)
    x = wl.complex_gaussian(9, N, 20 * M + 3)
    for k1 in (1, 2, wl.max_band(N, LV) - 1, wl.max_band(N, LV)):
        y = run_stream(torch, plan, x, k1)
        assert_parity(y, oracle.filter(N, O, V, k1, x), what=f"N={N} k1={k1}")


def test_band_changes_inline_and_split(cuda):
    """vbw_set_bandwidth between calls and vbw_set_bandwidth_at inside calls, including more
    than 16 changes inside one call (the library splits the launch)."""
    torch = cuda
    N, O, LV = 256, 64, 12
    M = N - O
    V = wl.transition_table(21, LV)
    plan = vbw.Plan(N, O, V)
    g = np.random.default_rng(21)
    nblocks = 120
    x = wl.complex_gaussian(21, 0, nblocks * M + 50)
    changes = [(int(b), int(g.integers(1, wl.max_band(N, LV) + 1)))
               for b in sorted(g.choice(np.arange(1, nblocks), 40, replace=False))]
    y = run_stream(torch, plan, x, 30, changes=changes, chunks=[7, 50, 1, 62])
    bands = bands_from_changes(nblocks + 1, 30, changes)
    ref = oracle.filter(N, O, V, bands, x)
    assert_parity(y, ref, what="band changes")
    # every block switches band
    changes = [(b, 1 + (b * 37) % wl.max_band(N, LV)) for b in range(1, nblocks + 1)]
    y = run_stream(torch, plan, x, 5, changes=changes)
    assert_parity(y, oracle.filter(N, O, V, bands_from_changes(nblocks + 1, 5, changes), x),
                  what="change every block")


def test_set_bandwidth_applies_at_next_block(cuda):
    torch = cuda
    N, O, LV = 512, 128, 12
    M = N - O
    V = wl.transition_table(3, LV)
    plan = vbw.Plan(N, O, V)
    x = wl.complex_gaussian(3, 3, 30 * M)
    xd = to_dev(torch, x)
    yd = torch.zeros_like(xd)
    s = vbw.Stream(plan, 40)
    s.filter(xd[:10 * M], yd[:10 * M], 10)
    s.set_bandwidth(200)
    s.filter(xd[10 * M:25 * M], yd[10 * M:25 * M], 15)
    s.set_bandwidth(7)
    s.set_bandwidth(90)          # the later call for the same block wins
    s.filter(xd[25 * M:], yd[25 * M:], 5)
    assert s.position == 30
    torch.cuda.synchronize()
    bands = np.array([40] * 10 + [200] * 15 + [90] * 5, dtype=np.int32)
    assert_parity(yd.cpu().numpy(), oracle.filter(N, O, V, bands, x), what="set_bandwidth")


@pytest.mark.parametrize("N,O", [(128, 32), (1024, 256), (2048, 512), (512, 127), (2048, 1023)])
def test_chunked_equals_one_shot_bitwise(cuda, N, O):
    torch = cuda
    M = N - O
    V = wl.transition_table(5, 12)
    plan = vbw.Plan(N, O, V)
    nblocks = 97
    x = wl.complex_gaussian(5, N, nblocks * M + M // 2)
    y1 = run_stream(torch, plan, x, 17)
    y2 = run_stream(torch, plan, x, 17, chunks=[1, 13, 2, 40, 41])
    y3 = run_stream(torch, plan, x, 17, chunks=[1] * nblocks)
    np.testing.assert_array_equal(y1, y2)
    np.testing.assert_array_equal(y1, y3)


@pytest.mark.parametrize("N,O", [(1024, 256), (1024, 255)])
def test_save_restore_bitwise(cuda, N, O):
    torch = cuda
    M = N - O
    V = wl.transition_table(8, 12)
    plan = vbw.Plan(N, O, V)
    x = wl.complex_gaussian(8, 0, 60 * M)
    xd = to_dev(torch, x)
    ref = torch.zeros_like(xd)
    s = vbw.Stream(plan, 100)
    s.set_bandwidth_at(45, 300)
    s.filter(xd, ref, 60)
    y = torch.zeros_like(xd)
    a = vbw.Stream(plan, 100)
    a.set_bandwidth_at(45, 300)
    a.filter(xd[:23 * M], y[:23 * M], 23)
    state = a.save()
    a.close()
    b = vbw.Stream(plan, 7)
    b.restore(state)
    assert b.position == 23
    b.filter(xd[23 * M:], y[23 * M:], 37)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y.cpu().numpy(), ref.cpu().numpy())
    plan2 = vbw.Plan(512, 128, V)
    c = vbw.Stream(plan2, 7)
    with pytest.raises(vbw.VbwError):
        c.restore(state)


@pytest.mark.parametrize("N,O", [(256, 64), (256, 63)])
def test_filter_host_matches_device(cuda, N, O):
    torch = cuda
    M = N - O
    V = wl.transition_table(6, 6)
    plan = vbw.Plan(N, O, V)
    nblocks = 200_000         # > one 32 MiB staging chunk, so the pipeline takes several steps
    x = wl.complex_gaussian(6, 0, nblocks * M)
    dev = run_stream(torch, plan, x, 60)
    s = vbw.Stream(plan, 60)
    out = np.empty_like(x)
    s.filter_host(x, out, nblocks)
    np.testing.assert_array_equal(out, dev)


def test_empty_and_invalid_calls(cuda):
    torch = cuda
    N, O = 256, 64
    M = N - O
    plan = vbw.Plan(N, O, wl.transition_table(1, 6))
    s = vbw.Stream(plan, 60)
    xd = torch.zeros(4 * M, dtype=torch.complex64, device="cuda")
    s.filter(xd, xd, 0)                                  # empty: no-op, no pointer checks
    assert s.position == 0
    with pytest.raises(vbw.VbwError) as e:
        s.filter(xd[:2 * M], xd[M:3 * M], 2)             # overlapping in/out
    assert e.value.code == 1
    with pytest.raises(vbw.VbwError) as e:
        s.set_bandwidth(0)
    assert e.value.code == 2
    with pytest.raises(vbw.VbwError) as e:
        vbw.Stream(plan, wl.max_band(N, 6) + 1)
    assert e.value.code == 2
    with pytest.raises(vbw.VbwError) as e:
        s.flush(xd[:M], xd[M:2 * M], M)                  # nvalid must be < M
    assert e.value.code == 1
    s.flush(None, None, 0)
    with pytest.raises(vbw.VbwError) as e:
        s.filter(xd[:M], xd[2 * M:3 * M], 1)
    assert e.value.code == 7
    s.reset(60)
    s.filter(xd[:M], xd[2 * M:3 * M], 1)
    torch.cuda.synchronize()


def test_single_stream_workload(cuda):
    """One stream of 2^16 samples, N=256, overlap 64, k1=60, L_V=6, checked in full."""
    torch = cuda
    w = wl.single()
    sig = w.signals[0]
    plan = vbw.Plan(sig.N, sig.overlap, w.V)
    y = run_stream(torch, plan, sig.x, int(sig.band[0]))
    assert_parity(y, oracle.filter(sig.N, sig.overlap, w.V, sig.band, sig.x), what="single")


def test_channels_workload_reduced(cuda):
    """The channel workload's geometry and band schedule (N=1024, overlap 256, k1 ~ U{32..480}
    every 16 blocks) on 6 channels x 2^17 samples, checked in full through a batch."""
    torch = cuda
    w = wl.channels(nch=6, nsamples=1 << 17)
    plan = vbw.Plan(1024, 256, w.V)
    xs = [to_dev(torch, s.x) for s in w.signals]
    ys = [torch.zeros_like(x) for x in xs]
    b = vbw.Batch([(plan, x, y, s.band) for x, y, s in zip(xs, ys, w.signals)])
    b.run()
    torch.cuda.synchronize()
    assert b.launches == 1
    for s, y in zip(w.signals, ys):
        ref = oracle.filter(1024, 256, w.V, s.band, s.x)
        assert_parity(y.cpu().numpy(), ref, what=f"channel {s.stream}")


@pytest.mark.parametrize("N,overlap,prec", [(N, N // 4, vbw.VBW_PREC_FP32) for N in ALL_N] +
                         [(1024, 6, vbw.VBW_PREC_FP32), (2048, 1800, vbw.VBW_PREC_FP32),
                          (256, 64, vbw.VBW_PREC_BF16_SPLIT), (512, 128, vbw.VBW_PREC_FP16_SCALED)])
def test_full_band_returns_the_input_delayed(cuda, N, overlap, prec):
    """With every bin in the passband (H_R = 1, test hook k1 = N/2 + 1) eq. (FS_Hk_exp) leaves
    only the linear phase, so y(t) = x(t - D), D = O/2, with zeros before the stream (no oracle:
    the expected output is the shifted input)."""
    torch = cuda
    D = overlap // 2
    V = wl.transition_table(7, 12)
    M = N - overlap
    x = wl.complex_gaussian(8, N + overlap, 37 * M + M // 3)
    vbw.vbw_debug_set(2)
    try:
        plan = vbw.Plan(N, overlap, V, precision=prec)
        y = run_stream(torch, plan, x, N // 2 + 1)
    finally:
        vbw.vbw_debug_set(0)
    want = np.concatenate([np.zeros(D, dtype=np.complex128), x[:len(x) - D]])
    tol = 2e-6 if prec == vbw.VBW_PREC_FP32 else 1e-5
    assert_parity(y, want, rms_tol=tol, elem_tol=10 * tol, what=f"N={N} O={overlap} prec={prec}")
    with pytest.raises(vbw.VbwError) as e:      # outside the test hook the band is rejected
        vbw.Stream(plan, N // 2 + 1)
    assert e.value.code == 2


ODD = [(128, 33), (128, 1), (256, 63), (512, 127), (512, 255), (1024, 255), (1024, 7), (2048, 511),
       (2048, 1023)]


@pytest.mark.parametrize("N,overlap", ODD)
def test_odd_overlap_half_sample_delay(cuda, N, overlap):
    """Odd overlap: the delay O/2 is a half sample; the phase of eq. (FS_Hk_exp) takes the signed
    bin index. Streams in two chunks with a ragged end and band changes, against the oracle."""
    torch = cuda
    M = N - overlap
    V = wl.transition_table(40 + N, 12)
    plan = vbw.Plan(N, overlap, V)
    nb = 23
    x = wl.complex_gaussian(41, N + overlap, nb * M + M // 3 + 1)
    k1 = int(np.random.default_rng(N + overlap).integers(1, wl.max_band(N, 12) + 1))
    changes = [(5, max(1, k1 // 2)), (14, wl.max_band(N, 12))]
    y = run_stream(torch, plan, x, k1, changes=changes, chunks=[9, nb - 9])
    bands = bands_from_changes((len(x) + M - 1) // M, k1, changes)
    ref = oracle.filter(N, overlap, V, bands, x)
    assert_parity(y, ref, what=f"N={N} O={overlap}")


@pytest.mark.parametrize("N,overlap", [(256, 63), (1024, 255), (2048, 511)])
def test_odd_overlap_batch_real_and_no_alloc(cuda, N, overlap):
    """The same half-sample filter through a batch, the real-signal batch and the no-alloc call."""
    torch = cuda
    M = N - overlap
    V = wl.transition_table(50 + N, 12)
    plan = vbw.Plan(N, overlap, V)
    n = 31 * M + 11
    x = wl.complex_gaussian(51, N, n)
    nbk = (n + M - 1) // M
    bands = wl.band_schedule(51, N, nbk, 4, 1, wl.max_band(N, 12))
    xd = to_dev(torch, x)
    yd = torch.zeros_like(xd)
    vbw.Batch([(plan, xd, yd, bands)]).run()
    xr = np.ascontiguousarray(x.real)
    xrd = torch.from_numpy(xr).cuda()
    yrd = torch.zeros_like(xrd)
    vbw.Batch([(plan, xrd, yrd, bands)], real=True).run()
    ys = torch.zeros_like(xd)
    vbw.vbw_filter_static(N, overlap, V, 9, xd, ys, n)
    torch.cuda.synchronize()
    assert_parity(yd.cpu().numpy(), oracle.filter(N, overlap, V, bands, x), what="batch")
    assert_parity(yrd.cpu().numpy(), oracle.filter(N, overlap, V, bands, xr.astype(np.complex64)).real,
                  what="real batch")
    assert_parity(ys.cpu().numpy(), oracle.filter(N, overlap, V, 9, x), what="no-alloc")



_N2048_CASE = {}


def _n2048_case():
    """Input, band schedule and oracle output shared by the N = 2048 kernel-shape tests."""
    if not _N2048_CASE:
        N, O, LV = 2048, 512, 12
        M = N - O
        V = wl.transition_table(2048 + 77, LV)
        nblocks = 3000
        x = wl.complex_gaussian(2048 + 5, 1, nblocks * M + 777)
        band0 = 300
        changes = [(150, 37), (2301, wl.max_band(N, LV)), (2950, 5)]
        ref = oracle.filter(N, O, V, bands_from_changes(nblocks + 1, band0, changes), x)
        _N2048_CASE.update(V=V, x=x, band0=band0, changes=changes, nblocks=nblocks, ref=ref)
    return _N2048_CASE


@pytest.mark.parametrize("shape", ["split8", "split12", "split16", "four_step"])
def test_n2048_kernel_shapes(cuda, monkeypatch, shape):
    """N = 2048, overlap N/4: the split kernel (one radix-2 step into two 1024-point halves, the
    idle half parked in tensor memory) at 8, 12 or 16 warps per CTA, forced for every launch size
    (VBW_SPLIT2048=2; by default only launches that fill the GPU take it), and the 64 x 32
    four-step kernel (VBW_SPLIT2048=0). Each against the oracle: a first call with more blocks
    than warps (some warps take two tiles), band changes inside the calls, the stream continued
    in a second call and a ragged end."""
    torch = cuda
    if shape == "four_step":
        monkeypatch.setenv("VBW_SPLIT2048", "0")
    else:
        monkeypatch.setenv("VBW_SPLIT2048", "2")
        monkeypatch.setenv("VBW_SPLIT2048_WARPS", shape[len("split"):])
    c = _n2048_case()
    plan = vbw.Plan(2048, 512, c["V"])
    y = run_stream(torch, plan, c["x"], c["band0"], changes=c["changes"], chunks=[2600, c["nblocks"] - 2600])
    assert_parity(y, c["ref"], what=f"N=2048 {shape}")

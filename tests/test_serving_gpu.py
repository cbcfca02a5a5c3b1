"""Serving engine (vbw_server_*): continuous batching of many live streams.

Each stream's output must equal the OLS VBW filter of its concatenated chunks (the FP64 oracle,
within the FP32 tolerance), with each band change taking effect at the first block boundary at or
after the chunk that carries it (ceil(S / M), S = samples submitted before the chunk), and must be
bit-identical whether the stream is served alone or mixed with others, whatever the batch slots
and pool size make of the batches.
"""
import numpy as np
import pytest

import oracle
from paper_2406_14116_gb300 import workloads as wl
from tests.conftest import assert_parity

pytestmark = pytest.mark.gpu

LV = 12


def _pinned(torch, n):
    return torch.empty(2 * max(n, 1), dtype=torch.float32, pin_memory=True).numpy().view(np.complex64)[:n]


def _expected_bands(M, band0, chunks):
    """Per-block k1 of a stream fed `chunks` = [(n, new_band)], closed at the end."""
    S = 0
    changes = []
    for n, nb in chunks:
        if nb >= 0:
            changes.append(((S + M - 1) // M, nb))
        S += n
    nblocks = (S + M - 1) // M
    bands = np.full(max(nblocks, 1), band0, dtype=np.int32)
    for blk, nb in changes:           # in submission order: a later change at a block wins
        bands[blk:] = nb
    return bands[:max(nblocks, 1)], S


def _make_streams(seed, specs, torch, pageable=()):
    """specs: [(plan_index, N, O, band0, [(n, new_band)])] -> input arrays and output buffers.
    Streams listed in `pageable` use pageable numpy memory (copied by the CUDA runtime), the
    others pinned memory (read and written by the engine's copy kernels)."""
    streams = []
    for i, (pi, N, O, band0, chunks) in enumerate(specs):
        S = sum(n for n, _ in chunks)
        x = wl.complex_gaussian(seed, i, S)
        alloc = (lambda n: np.empty(n, dtype=np.complex64)) if i in pageable else (lambda n: _pinned(torch, n))
        xin = alloc(S)
        xin[:] = x
        yout = alloc(S)
        yout[:] = np.nan
        streams.append(dict(plan=pi, N=N, O=O, band0=band0, chunks=chunks, x=xin, y=yout))
    return streams


def _serve(vbw, plans, streams, pool_bytes, slots, order, poll_every=1):
    """Submits every stream's chunks in the interleaving `order` (a list of stream indices, one
    entry per chunk, closes included), polling every `poll_every` submissions. Returns the
    completions and the server statistics."""
    sv = vbw.Server(plans, max_streams=len(streams), pool_bytes=pool_bytes, slots=slots)
    for i, s in enumerate(streams):
        sv.open_stream(i, s["plan"], s["band0"])
    nxt = [0] * len(streams)
    pos = [0] * len(streams)
    tag = 0
    got = []
    for k, i in enumerate(order):
        s = streams[i]
        M = s["N"] - s["O"]
        if nxt[i] < len(s["chunks"]):
            n, nb = s["chunks"][nxt[i]]
            S = pos[i]
            o0 = S // M * M
            outn = (S + n) // M * M - o0
            x = s["x"][S:S + n]
            y = s["y"][o0:o0 + outn]
            sv.submit(i, x if n else None, n, nb, y if outn else None, outn, tag)
            pos[i] += n
        else:
            o0 = pos[i] // M * M
            y = s["y"][o0:]
            sv.close_stream(i, y if len(y) else None, len(y), tag)
        nxt[i] += 1
        tag += 1
        if poll_every and k % poll_every == 0:
            got.append(sv.poll())
    got.append(sv.drain())
    info = sv.info()
    sv.close()
    return np.concatenate(got), info


def _order(streams, rng):
    order = []
    for i, s in enumerate(streams):
        order += [i] * (len(s["chunks"]) + 1)
    rng.shuffle(order)
    return order


def _random_chunks(rng, M, nchunks, band_max, change_p=0.3):
    out = []
    for _ in range(nchunks):
        kind = rng.integers(0, 4)
        if kind == 0:
            n = int(rng.integers(0, M))            # shorter than a block (may be 0)
        elif kind == 1:
            n = int(M * rng.integers(1, 4))        # whole blocks
        else:
            n = int(rng.integers(M, 6 * M))        # several blocks and a ragged end
        nb = int(rng.integers(1, band_max + 1)) if rng.uniform() < change_p else -1
        out.append((n, nb))
    return out


@pytest.fixture(scope="module")
def plans(cuda):
    from paper_2406_14116_gb300 import vbw
    V = wl.transition_table(5, LV)
    geo = [(256, 64), (512, 128), (1024, 256), (2048, 512), (512, 96)]
    ps = [vbw.Plan(N, O, V) for N, O in geo]
    yield vbw, V, geo, ps
    for p in ps:
        p.close()


def _specs(rng, geo, nstreams, nchunks=6):
    specs = []
    for i in range(nstreams):
        pi = int(rng.integers(0, len(geo)))
        N, O = geo[pi]
        bmax = wl.max_band(N, LV)
        specs.append((pi, N, O, int(rng.integers(1, bmax + 1)),
                      _random_chunks(rng, N - O, nchunks, bmax)))
    return specs


def test_serving_matches_oracle_per_stream(cuda, plans):
    vbw, V, geo, ps = plans
    rng = np.random.default_rng(51)
    streams = _make_streams(51, _specs(rng, geo, 10), cuda, pageable={2, 5})
    comp, info = _serve(vbw, ps, streams, pool_bytes=64 << 20, slots=3, order=_order(streams, rng))
    assert info["queued"] == 0 and info["inflight_batches"] == 0
    assert len(comp) == sum(len(s["chunks"]) + 1 for s in streams)
    # completions arrive in submission order
    np.testing.assert_array_equal(comp["tag"], np.arange(len(comp)))
    for i, s in enumerate(streams):
        M = s["N"] - s["O"]
        bands, S = _expected_bands(M, s["band0"], s["chunks"])
        assert comp["produced"][comp["stream"] == i].sum() == S
        ref = oracle.filter(s["N"], s["O"], V, bands, s["x"])
        assert_parity(s["y"], ref, what=f"stream {i} (N={s['N']}, O={s['O']})")


def test_serving_split_kernel_for_n2048(cuda, plans, monkeypatch):
    """The serving engine's N = 2048 launches through the split kernel (forced for these small
    batches; by default only launches that fill the GPU take it): per-stream oracle parity."""
    monkeypatch.setenv("VBW_SPLIT2048", "2")
    vbw, V, geo, ps = plans
    rng = np.random.default_rng(57)
    specs = [s for s in _specs(rng, geo, 16) if s[1] == 2048][:4]
    assert specs, "the seed must draw N = 2048 streams"
    streams = _make_streams(57, specs, cuda)
    _serve(vbw, ps, streams, pool_bytes=64 << 20, slots=2, order=_order(streams, rng))
    for i, s in enumerate(streams):
        M = s["N"] - s["O"]
        bands, _ = _expected_bands(M, s["band0"], s["chunks"])
        assert_parity(s["y"], oracle.filter(s["N"], s["O"], V, bands, s["x"]), what=f"split stream {i}")


def test_alone_vs_mix_bitwise(cuda, plans):
    vbw, V, geo, ps = plans
    rng = np.random.default_rng(52)
    specs = _specs(rng, geo, 12, nchunks=8)
    mixed = _make_streams(52, specs, cuda, pageable={0, 3, 7, 11})
    _serve(vbw, ps, mixed, pool_bytes=256 << 20, slots=4, order=_order(mixed, rng), poll_every=3)
    for i in (0, 5, 11):
        alone = _make_streams(52, specs, cuda)
        order = [i] * (len(specs[i][4]) + 1)
        _serve(vbw, ps, alone, pool_bytes=32 << 20, slots=1, order=order)
        np.testing.assert_array_equal(alone[i]["y"], mixed[i]["y"])


def test_admission_by_memory_in_a_small_pool(cuda, plans):
    """A pool that holds only a few chunks per slot forces many small batches; the result is
    bit-identical to a roomy pool, every completion carries its full output, in order."""
    vbw, V, geo, ps = plans
    rng = np.random.default_rng(53)
    specs = _specs(rng, geo, 8, nchunks=6)
    big = _make_streams(53, specs, cuda)
    order = _order(big, rng)
    _, info_big = _serve(vbw, ps, big, pool_bytes=256 << 20, slots=2, order=order, poll_every=0)
    small = _make_streams(53, specs, cuda)
    max_chunk = max(n for s in specs for n, _ in s[4])
    pool = 2 * 2 * 8 * (max_chunk + 2048) + 4096   # two slots of roughly one chunk each
    comp, info_small = _serve(vbw, ps, small, pool_bytes=pool, slots=2, order=order, poll_every=0)
    assert info_small["batches"] > info_big["batches"]
    np.testing.assert_array_equal(comp["tag"], np.arange(len(comp)))
    for a, b in zip(big, small):
        np.testing.assert_array_equal(a["y"], b["y"])


def test_band_change_lands_on_block_boundary(cuda, plans):
    """Chunks whose edges fall inside blocks: a change takes effect at ceil(S / M); two changes due
    at one block keep the later."""
    vbw, V, geo, ps = plans
    N, O = 512, 128
    M = N - O
    chunks = [(M + 100, -1), (50, 40), (300, -1), (M // 2, 90), (10, 120), (3 * M + 7, -1),
              (M - 7, 150), (2 * M, -1)]
    streams = _make_streams(54, [(1, N, O, 20, chunks)], cuda)
    _serve(vbw, ps, streams, pool_bytes=32 << 20, slots=2, order=[0] * (len(chunks) + 1))
    bands, S = _expected_bands(M, 20, chunks)
    # by hand (M = 384): the change at S = 484 lands on block 2; those at S = 834 and S = 1026
    # both land on block 3, where the later (120) wins; the one at S = 2195 lands on block 6
    assert list(bands) == [20, 20, 40, 120, 120, 120, 150, 150, 150] and S == 3340
    ref = oracle.filter(N, O, V, bands, streams[0]["x"])
    assert_parity(streams[0]["y"], ref, what="band change at block boundary")


def test_reopen_and_errors(cuda, plans):
    vbw, V, geo, ps = plans
    sv = vbw.Server(ps[:2], max_streams=2, pool_bytes=8 << 20, slots=2)
    x = _pinned(cuda, 4096)
    x[:] = wl.complex_gaussian(55, 0, 4096)
    y = _pinned(cuda, 4096)
    with pytest.raises(vbw.VbwError) as e:
        sv.submit(0, x, 100, -1, None, 0, 0)              # not open
    assert e.value.code == 7
    sv.open_stream(0, 0, 10)
    with pytest.raises(vbw.VbwError) as e:
        sv.open_stream(0, 0, 10)                          # already open
    assert e.value.code == 7
    with pytest.raises(vbw.VbwError) as e:
        sv.submit(0, x, 1000, -1, y, 10, 0)               # output too small (1000 -> 960)
    assert e.value.code == 1
    with pytest.raises(vbw.VbwError) as e:
        sv.submit(0, x, 100, 10_000, None, 0, 0)          # band out of range
    assert e.value.code == 2
    with pytest.raises(vbw.VbwError) as e:
        sv.submit(0, x, 1 << 22, -1, None, 0, 0)          # job larger than a slot
    assert e.value.code == 1
    with pytest.raises(vbw.VbwError):
        sv.open_stream(1, 5, 10)                          # no such plan
    # a closed stream opens again with zero history: same output as the first time
    outs = []
    for _ in range(2):
        yy = _pinned(cuda, 4096)
        sv.submit(0, x, 4096, -1, yy, 4096 // 192 * 192, 0)
        sv.close_stream(0, yy[4096 // 192 * 192:], 4096 % 192, 1)
        sv.drain()
        outs.append(yy.copy())
        sv.open_stream(0, 0, 10)
    np.testing.assert_array_equal(outs[0], outs[1])
    ref = oracle.filter(256, 64, V, 10, x)
    assert_parity(outs[0], ref, what="reopened stream")
    sv.close()


def test_serving_workload_sample(cuda):
    """A short slice of the serving workload (2000 streams, N in {512, 1024, 2048}, O = N/4,
    chunks U{1024..65536}, 1% band changes): sampled streams against the oracle."""
    from paper_2406_14116_gb300 import vbw
    V = wl.transition_table(5, LV)
    Ns = (512, 1024, 2048)
    Nsel, Osel, k1 = wl.serving_streams(5)
    t, sid, lens, nb = wl.serving_arrivals(5, duration=0.01, Nsel=Nsel)
    ps = [vbw.Plan(N, N // 4, V) for N in Ns]
    pidx = {N: i for i, N in enumerate(Ns)}
    nst = len(Nsel)
    total = np.zeros(nst, dtype=np.int64)
    for s, n in zip(sid, lens):
        total[s] += n
    sv = vbw.Server(ps, max_streams=nst, pool_bytes=512 << 20, slots=4)
    xs, ys, chunks = {}, {}, {i: [] for i in range(nst)}
    for i in range(nst):
        sv.open_stream(i, pidx[int(Nsel[i])], int(k1[i]))
    for i in np.unique(sid):
        xs[i] = _pinned(cuda, int(total[i]))
        xs[i][:] = wl.complex_gaussian(5, int(i), int(total[i]))
        ys[i] = _pinned(cuda, int(total[i]))
    pos = np.zeros(nst, dtype=np.int64)
    for k, (s, n, b) in enumerate(zip(sid, lens, nb)):
        M = int(Nsel[s]) * 3 // 4
        S = int(pos[s])
        o0 = S // M * M
        outn = (S + int(n)) // M * M - o0
        sv.submit(int(s), xs[s][S:S + n], int(n), int(b), ys[s][o0:o0 + outn] if outn else None, outn, k)
        chunks[s].append((int(n), int(b)))
        pos[s] += n
        if k % 8 == 0:
            sv.poll()
    for i in np.unique(sid):
        M = int(Nsel[i]) * 3 // 4
        o0 = int(pos[i]) // M * M
        sv.close_stream(int(i), ys[i][o0:], int(pos[i]) - o0, 1 << 40)
    sv.drain()
    sv.close()
    for i in list(np.unique(sid))[:6]:
        N = int(Nsel[i])
        bands, S = _expected_bands(N * 3 // 4, int(k1[i]), chunks[i])
        ref = oracle.filter(N, N // 4, V, bands, xs[i])
        assert_parity(ys[i], ref, what=f"serving stream {i} (N={N})")
    for p in ps:
        p.close()


def test_submit_many_equals_single_submits(cuda, plans):
    """vbw_server_submit_many queues the same chunks as one vbw_server_submit per chunk: the outputs
    are bit-identical; a failing chunk stops the call and reports how many were queued."""
    vbw, V, geo, ps = plans
    rng = np.random.default_rng(56)
    specs = _specs(rng, geo, 6, nchunks=5)
    one = _make_streams(56, specs, cuda)
    order = _order(one, rng)
    _serve(vbw, ps, one, pool_bytes=64 << 20, slots=2, order=order)
    many = _make_streams(56, specs, cuda)
    sv = vbw.Server(ps, max_streams=len(many), pool_bytes=64 << 20, slots=2)
    for i, s in enumerate(many):
        sv.open_stream(i, s["plan"], s["band0"])
    nxt, pos, reqs, closes = [0] * len(many), [0] * len(many), [], []
    for tag, i in enumerate(order):
        s = many[i]
        M = s["N"] - s["O"]
        if nxt[i] < len(s["chunks"]):
            n, nb = s["chunks"][nxt[i]]
            S = pos[i]
            o0 = S // M * M
            outn = (S + n) // M * M - o0
            reqs.append((i, nb, s["x"][S:].ctypes.data if n else 0, n,
                         s["y"][o0:].ctypes.data if outn else 0, outn, tag))
            pos[i] += n
        else:
            closes.append((i, tag))
        nxt[i] += 1
    req = np.array(reqs, dtype=vbw.REQUEST_DTYPE)
    assert sv.submit_many(req) == len(req)
    for i, tag in closes:
        s = many[i]
        M = s["N"] - s["O"]
        o0 = pos[i] // M * M
        y = s["y"][o0:]
        sv.close_stream(i, y if len(y) else None, len(y), tag)
    sv.drain()
    for a, b in zip(one, many):
        np.testing.assert_array_equal(a["y"], b["y"])
    # a chunk on a stream that is not open stops the call after the good ones
    bad = np.array([(0, -1, many[0]["x"].ctypes.data, 16, 0, 0, 1), (99, -1, 0, 0, 0, 0, 2)],
                   dtype=vbw.REQUEST_DTYPE)
    sv.open_stream(0, many[0]["plan"], many[0]["band0"])
    with pytest.raises(vbw.VbwError) as e:
        sv.submit_many(bad)
    assert "after 1 queued" in str(e.value)
    sv.close()


def test_serving_tensor_core_plans(cuda):
    """Streams on tensor-core plans (BF16 split, scaled FP16) go through the same engine: the
    outputs meet the split variants' 1e-5 gate against the oracle."""
    from paper_2406_14116_gb300 import vbw
    V = wl.transition_table(57, LV)
    ps = [vbw.Plan(256, 64, V, precision=vbw.VBW_PREC_BF16_SPLIT),
          vbw.Plan(512, 128, V, precision=vbw.VBW_PREC_FP16_SCALED)]
    geo = [(256, 64), (512, 128)]
    rng = np.random.default_rng(57)
    specs = []
    for i in range(6):
        pi = i % 2
        N, O = geo[pi]
        bmax = wl.max_band(N, LV)
        specs.append((pi, N, O, int(rng.integers(1, bmax + 1)), _random_chunks(rng, N - O, 6, bmax)))
    streams = _make_streams(57, specs, cuda)
    _serve(vbw, ps, streams, pool_bytes=64 << 20, slots=3, order=_order(streams, rng))
    for i, s in enumerate(streams):
        M = s["N"] - s["O"]
        bands, S = _expected_bands(M, s["band0"], s["chunks"])
        ref = oracle.filter(s["N"], s["O"], V, bands, s["x"])
        assert_parity(s["y"], ref, rms_tol=1e-5, elem_tol=2e-4, what=f"tensor-core stream {i}")
    for p in ps:
        p.close()

"""Parity at the full sizes of the mixed and the precision workloads, in the launch configuration
bench.py times (one prepared batch over every stream): the whole batch runs on the GPU, and a
seeded 5% of its streams (plus the first and the last) are checked sample by sample, in full,
against the FP64 oracle of Sec. II.

  * mixed: 4096 streams of floor(2^U(12,20)) samples (about 7.7e8 in all), N ~ U{128..2048},
    overlap N/4, one k1 per stream, unit noise plus 1-8 tones; per-plan launches and the mixed
    one-launch mode, which must agree bit for bit.
  * precision: 16384 channels x 2^16 samples at N = 256 and 512 (overlap N/4), one k1 per
    channel, for the FP32 path and every tensor-core split (BF16 x3, row-scaled FP16, BF16 x6).
Gates: RMS relative error <= 2e-6 (FP32) or 1e-5 (splits) per stream, and every sample within
2e-5 (FP32) or 2e-4 (splits) of the stream's reference RMS.
"""
import concurrent.futures as cf
import math
import os

import numpy as np
import pytest

import oracle
from conftest import assert_parity
from paper_2406_14116_gb300 import vbw
from paper_2406_14116_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FRACTION = 0.05
LV = 12


def checked_streams(n, seed):
    """A seeded 5% of n stream ids, plus the first and the last stream."""
    g = np.random.default_rng(seed)
    pick = set(g.choice(n, size=math.ceil(FRACTION * n), replace=False).tolist())
    return sorted(pick | {0, n - 1})


def fill(views, make):
    with cf.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 8)) as ex:
        list(ex.map(lambda i: views[i].__setitem__(slice(None), make(i)), range(len(views))))


def test_mixed_workload_full_batch(cuda):
    torch = cuda
    n = 4096
    lengths, Nsel, ovl, k1 = wl.mixed_stream_params(3, n)
    V = wl.transition_table(3, LV)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    x = np.empty(int(offs[-1]), np.complex64)
    views = [x[offs[i]:offs[i + 1]] for i in range(n)]
    fill(views, lambda i: wl.tones_signal(3, i, int(lengths[i])))
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    plans = {N: vbw.Plan(N, N // 4, V) for N in (128, 256, 512, 1024, 2048)}
    bands = [np.full(wl.nblocks_for(int(lengths[i]), int(Nsel[i]), int(ovl[i])), int(k1[i]), np.int32)
             for i in range(n)]
    b = vbw.Batch([(plans[int(Nsel[i])], xd[offs[i]:offs[i + 1]], yd[offs[i]:offs[i + 1]], bands[i])
                   for i in range(n)])
    b.set_mode(vbw.VBW_BATCH_PER_PLAN)
    b.run()
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    yd.fill_(float("nan"))
    b.set_mode(vbw.VBW_BATCH_MIXED)
    b.run()
    torch.cuda.synchronize()
    assert np.array_equal(y.view(np.uint64), yd.cpu().numpy().view(np.uint64)), \
        "per-plan and mixed launches differ"
    b.close()
    for p in plans.values():
        p.close()
    del xd, yd
    for i in checked_streams(n, 3003):
        ref = oracle.filter(int(Nsel[i]), int(ovl[i]), V, bands[i], views[i])
        assert_parity(y[offs[i]:offs[i + 1]], ref,
                      what=f"mixed stream {i} N={int(Nsel[i])} len={int(lengths[i])}")


PRECISION_NCH = 16384
PRECISION_T = 1 << 16
PRECS = {"fp32": (vbw.VBW_PREC_FP32, 2e-6, 2e-5), "bf16x3": (vbw.VBW_PREC_BF16_SPLIT, 1e-5, 2e-4),
         "fp16s": (vbw.VBW_PREC_FP16_SCALED, 1e-5, 2e-4), "bf16x6": (vbw.VBW_PREC_BF16_SPLIT3, 1e-5, 2e-4)}


@pytest.fixture(scope="module")
def precision_input(cuda):
    """The precision workload's 16384 x 2^16 complex64 input, on the host and on the device."""
    torch = cuda
    x = np.empty((PRECISION_NCH, PRECISION_T), np.complex64)
    fill(list(x), lambda i: wl.complex_gaussian(4, i, PRECISION_T))
    xd = torch.from_numpy(x).cuda()
    yield x, xd
    del xd
    torch.cuda.empty_cache()


_REFS = {}


def precision_refs(x, N):
    """Oracle outputs of the checked channels at transform size N (one set for every precision)."""
    if N not in _REFS:
        V = wl.transition_table(4, LV)
        k1 = wl.precision_bands(4, PRECISION_NCH, N, LV)
        nb = wl.nblocks_for(PRECISION_T, N, N // 4)
        _REFS[N] = {ch: oracle.filter(N, N // 4, V, np.full(nb, int(k1[ch]), np.int32), x[ch])
                    for ch in checked_streams(PRECISION_NCH, 4004 + N)}
    return _REFS[N]


@pytest.mark.parametrize("N", [256, 512])
@pytest.mark.parametrize("prec", list(PRECS))
def test_precision_workload_full_sweep(cuda, precision_input, N, prec):
    torch = cuda
    x, xd = precision_input
    code, rms_tol, elem_tol = PRECS[prec]
    V = wl.transition_table(4, LV)
    k1 = wl.precision_bands(4, PRECISION_NCH, N, LV)
    nb = wl.nblocks_for(PRECISION_T, N, N // 4)
    plan = vbw.Plan(N, N // 4, V, precision=code)
    yd = torch.full_like(xd, float("nan"))
    b = vbw.Batch([(plan, xd[c], yd[c], np.full(nb, int(k1[c]), np.int32))
                   for c in range(PRECISION_NCH)])
    b.run()
    torch.cuda.synchronize()
    refs = precision_refs(x, N)
    ids = sorted(refs)
    y = yd[torch.tensor(ids, device=yd.device)].cpu().numpy()
    assert torch.isfinite(torch.view_as_real(yd)).all().item(), "non-finite output"
    b.close()
    plan.close()
    del yd
    for j, ch in enumerate(ids):
        assert_parity(y[j], refs[ch], rms_tol=rms_tol, elem_tol=elem_tol,
                      what=f"precision N={N} {prec} channel {ch} k1={int(k1[ch])}")

"""Real-valued signals (vbw_batch_create_real): two real blocks per complex transform.

Parity: the FP64 oracle filtering x + 0j (its real part) for every N, small / N/4 / N/2 overlaps,
ragged ends, band changes on even and odd blocks (odd ones cut the signal into pieces), and
signals at odd float offsets (the bulk L2 prefetch realigns). The result must also match the complex path on
x + 0j within FP32 rounding."""
import numpy as np
import pytest

import oracle
from conftest import assert_parity
from paper_2406_14116_gb300 import vbw
from paper_2406_14116_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _real(seed, stream, n):
    return np.ascontiguousarray(wl.complex_gaussian(seed, stream, n).real * np.float32(np.sqrt(2.0)))


@pytest.mark.parametrize("N,overlap", [(128, 32), (256, 64), (256, 128), (512, 128), (512, 6),
                                       (1024, 256), (2048, 512), (2048, 1024)])
def test_real_batch_matches_oracle(cuda, N, overlap):
    torch = cuda
    M = N - overlap
    V = wl.transition_table(30 + N, 12)
    plan = vbw.Plan(N, overlap, V)
    g = np.random.default_rng(N + overlap)
    sigs, refs = [], []
    for i, n in enumerate([0, 1, M - 1, M, 2 * M + 3, 37 * M + 5, 64 * M]):
        x = _real(N, i, n)
        nb = (n + M - 1) // M
        # changes every 5 blocks hit odd and even block indices
        bands = wl.band_schedule(N + i, i, nb, 5, 1, wl.max_band(N, 12)) if nb else np.zeros(0, np.int32)
        xd = torch.from_numpy(x).cuda()
        yd = torch.full_like(xd, float("nan"))
        sigs.append((plan, xd, yd, bands if nb else 7))
        refs.append(oracle.filter(N, overlap, V, bands if nb else 7, x.astype(np.complex64)) if n else np.zeros(0))
    b = vbw.Batch(sigs, real=True)
    b.run()
    torch.cuda.synchronize()
    for (p, xd, yd, _), ref in zip(sigs, refs):
        y = yd.cpu().numpy().astype(np.float64)
        assert np.abs(ref.imag).max(initial=0) < 1e-12
        if len(y) >= M:
            assert_parity(y, ref.real, what=f"N={N} O={overlap} n={len(y)}")
        else:
            # shorter than a block: a few tiny outputs, so bound the error by the input scale
            np.testing.assert_allclose(y, ref.real, rtol=0, atol=2e-6)


def test_real_equals_complex_path_and_odd_offsets(cuda):
    torch = cuda
    N, O = 1024, 256
    M = N - O
    V = wl.transition_table(9, 12)
    plan = vbw.Plan(N, O, V)
    n = 50 * M + 17
    x = _real(9, 0, n)
    nb = (n + M - 1) // M
    bands = wl.band_schedule(9, 0, nb, 3, 32, 480)
    buf = torch.from_numpy(np.concatenate([[0.0], x]).astype(np.float32)).cuda()
    xd = buf[1:]                                   # 4-byte but not 16-byte aligned
    yr = torch.zeros(n + 1, dtype=torch.float32, device="cuda")[1:]
    xa = torch.from_numpy(x).cuda()
    ya = torch.zeros_like(xa)
    vbw.Batch([(plan, xd, yr, bands)], real=True).run()
    vbw.Batch([(plan, xa, ya, bands)], real=True).run()
    xc = torch.from_numpy(x.astype(np.complex64)).cuda()
    yc = torch.zeros_like(xc)
    vbw.Batch([(plan, xc, yc, bands)]).run()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(yr.cpu().numpy(), ya.cpu().numpy())
    yc = yc.cpu().numpy()
    np.testing.assert_allclose(ya.cpu().numpy(), yc.real, rtol=0, atol=2e-5 * np.abs(yc).max())
    ref = oracle.filter(N, O, V, bands, x.astype(np.complex64))
    assert_parity(ya.cpu().numpy(), ref.real, what="aligned real")


def test_real_batch_rejects_unsupported(cuda):
    torch = cuda
    V = wl.transition_table(1, 12)
    x = torch.zeros(4096, dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    for plan in (vbw.Plan(256, 64, V, precision=vbw.VBW_PREC_BF16_SPLIT), vbw.Plan(256, 200, V)):
        with pytest.raises(vbw.VbwError) as e:
            vbw.Batch([(plan, x, y, 10)], real=True)
        assert e.value.code == 8

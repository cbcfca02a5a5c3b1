"""The tensor-core (tcgen05) precision variant: the GEMM building block against a host GEMM with
the same 16-bit rounding, then OLS VBW filtering with BF16 / FP16 split DFT-matrix GEMMs against
the FP64 oracle (RMS relative error gate 1e-5 for the split variants), through the C ABI."""
import numpy as np
import pytest

import oracle
from conftest import assert_parity, rms_rel
from paper_2406_14116_gb300 import vbw
from paper_2406_14116_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def to_bf16(x):
    """Round float32 to bfloat16 (nearest even), returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = ((b >> 16) & 1) + np.uint32(0x7FFF)
    return ((b + r) & np.uint32(0xFFFF0000)).view(np.float32)


def to_fp16(x):
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


@pytest.mark.parametrize("a_mn", [False, True])
@pytest.mark.parametrize("bf16", [True, False])
@pytest.mark.parametrize("K,NN", [(32, 32), (64, 64), (32, 64), (64, 32)])
def test_tcgen05_gemm_layout(cuda, bf16, K, NN, a_mn):
    """One tcgen05 GEMM with A in K-major core matrices (rounds 1 and 3 of the OLS kernel) or in
    MN-major core matrices (rounds 2 and 4) against a host GEMM with the same 16-bit rounding."""
    g = np.random.default_rng(K * 100 + NN + bf16 + 7 * a_mn)
    A = g.uniform(-1, 1, (128, K)).astype(np.float32)
    B = g.uniform(-1, 1, (K, NN)).astype(np.float32)
    D = vbw.vbw_debug_tc_gemm(A, B, bf16, a_mn_major=a_mn)
    r = to_bf16 if bf16 else to_fp16
    ref = r(A).astype(np.float64) @ r(B).astype(np.float64)
    np.testing.assert_allclose(D, ref, rtol=0, atol=1e-5 * np.abs(ref).max())


PRECS = {vbw.VBW_PREC_BF16_SPLIT: 1e-5, vbw.VBW_PREC_FP16_SCALED: 1e-5,
         vbw.VBW_PREC_BF16_SPLIT3: 1e-5}


@pytest.mark.parametrize("N", [256, 512])
@pytest.mark.parametrize("prec", list(PRECS))
def test_tensor_ols_parity(cuda, N, prec):
    """Stream filtering (two calls with the tail carried between them, then a partial block) on
    the tensor-core kernel vs the oracle, against the 1e-5 RMS gate of the split variants."""
    torch = cuda
    O = N // 4
    M = N - O
    V = wl.transition_table(60 + N, 12)
    plan = vbw.Plan(N, O, V, precision=prec)
    g = np.random.default_rng(N + prec)
    k1 = int(g.integers(1, wl.max_band(N, 12) + 1))
    nb = 203
    x = wl.complex_gaussian(70 + N, prec, nb * M + M // 3)
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    s = vbw.Stream(plan, k1)
    s.set_bandwidth_at(150, max(1, k1 // 2))
    s.filter(xd[:77 * M], yd[:77 * M], 77)
    s.filter(xd[77 * M:nb * M], yd[77 * M:nb * M], nb - 77)
    s.flush(xd[nb * M:], yd[nb * M:], len(x) - nb * M)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    bands = np.array([k1] * 150 + [max(1, k1 // 2)] * (nb + 1 - 150), dtype=np.int32)
    ref = oracle.filter(N, O, V, bands, x)
    tol = PRECS[prec]
    assert_parity(y, ref, rms_tol=tol, elem_tol=20 * tol, what=f"N={N} prec={prec}")


def test_tensor_batch_and_fp32_batch_agree_with_oracle(cuda):
    """A batch mixing tensor-core plans (N = 256, 512) and an FP32 plan, with per-block bands."""
    torch = cuda
    V = wl.transition_table(77, 12)
    plans = [vbw.Plan(256, 64, V, precision=vbw.VBW_PREC_FP16_SCALED),
             vbw.Plan(512, 128, V, precision=vbw.VBW_PREC_BF16_SPLIT3),
             vbw.Plan(1024, 256, V)]
    rows, refs = [], []
    for i, p in enumerate(plans * 2):
        n = 20000 + 3000 * i
        x = wl.complex_gaussian(77, i, n)
        nbk = wl.nblocks_for(n, p.N, p.overlap)
        bands = wl.band_schedule(77, i, nbk, 5, 1, wl.max_band(p.N, 12))
        xd = torch.from_numpy(x).cuda()
        rows.append((p, xd, torch.zeros_like(xd), bands))
        refs.append(oracle.filter(p.N, p.overlap, V, bands, x))
    b = vbw.Batch(rows)
    b.run()
    torch.cuda.synchronize()
    for (p, xd, yd, bands), ref in zip(rows, refs):
        assert_parity(yd.cpu().numpy(), ref, rms_tol=1e-5, elem_tol=2e-4, what=f"N={p.N}")


def test_tensor_precision_rejects_other_geometries(cuda):
    V = wl.transition_table(1, 12)
    for N, O in ((1024, 256), (256, 32), (128, 32)):
        with pytest.raises(vbw.VbwError) as e:
            vbw.Plan(N, O, V, precision=vbw.VBW_PREC_BF16_SPLIT)
        assert e.value.code == 8

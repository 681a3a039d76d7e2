"""GPU parity of the FP8 E4M3 path: the quantiser bit for bit against the
oracle's E4M3 encoder, the GEMM against the FP64 oracle on the dequantised
inputs (and, as a report, on the unquantised ones)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import fp8
import workloads
from gpu_common import assert_within_bound, dev, sk, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return sk()


@pytest.mark.parametrize("n", [1, 2, 1023, 100_003])
def test_quantize_bit_exact(m, n):
    d = dev()
    x = workloads.normal((n,), seed=60 + n) * 3.0
    q, s = m.quantize_e4m3(x.to(d))
    q_ref, s_ref = fp8.quantize_e4m3(x.numpy())
    assert np.float32(s.item()) == s_ref
    assert np.array_equal(q.cpu().numpy(), q_ref)


def test_quantize_zero_and_extremes(m):
    d = dev()
    z = torch.zeros(64, device=d)
    q, s = m.quantize_e4m3(z)
    assert s.item() == 1.0 and int(q.max()) == 0
    x = torch.tensor([1e-30, -448.0, 448.0, 3.0, -1e-8] * 13, dtype=torch.float32)
    q, s = m.quantize_e4m3(x.to(d))
    q_ref, s_ref = fp8.quantize_e4m3(x.numpy())
    assert np.array_equal(q.cpu().numpy(), q_ref)


def _quant(m, x, d):
    q, s = m.quantize_e4m3(x.to(d).contiguous())
    return q, s


@pytest.mark.parametrize("tile_m", [128, 256])
@pytest.mark.parametrize("shape", [(256, 512, 1024), (300, 520, 1024), (1024, 1024, 4096)])
@pytest.mark.parametrize("mode", ["sk", "hybrid2", "dp"])
def test_fp8_gemm_vs_dequantised(m, shape, mode, tile_m):
    M, N, K = shape
    d = dev()
    xa = workloads.normal((M, K), seed=70)
    xb = workloads.normal((N, K), seed=71)          # B^T rows: column-major B
    qa, sa = _quant(m, xa, d)
    qb, sb = _quant(m, xb, d)
    A = qa.view(torch.float8_e4m3fn)
    Bm = qb.view(torch.float8_e4m3fn).t()
    c = m.gemm(A, Bm, out_dtype=torch.float32, scale_a=sa, scale_b=sb, config=m.Config(mode=mode, tile_m=tile_m))
    assert m.default_workspace(d).status() == 0
    deq_a = fp8.dequantize_e4m3(qa.cpu().numpy(), sa.item())
    deq_b = fp8.dequantize_e4m3(qb.cpu().numpy(), sb.item()).T
    assert_within_bound(c, deq_a, deq_b, out="f32", what=f"fp8 {shape} {mode}")
    # against the unquantised product: report-only sanity cap from the E4M3
    # unit roundoff on both operands
    ref, S = oracle.gemm(xa.numpy(), xb.numpy().T)
    rel = np.abs(to_np(c) - ref) / S
    assert np.max(rel) <= 2 * 2 ** -4 + 2 ** -8


@pytest.mark.parametrize("K", [32, 128, 1024])
def test_fp8_accumulator_width(m, K):
    """How wide is the kind::f8f6f4 accumulation?  One product 2^8 * 2^8 =
    2^16 plus K-1 products 2^-3 * 2^-3 = 2^-6: the exact sum 2^16 + (K-1)
    2^-6 needs 23 significand bits, so an FP32 accumulator keeps it exactly
    and a narrower one drops the small terms.  The result must meet the
    oracle bound in any case; the measured shortfall is printed."""
    d = dev()
    M, N = 128, 128
    x = torch.full((M, K), 2.0 ** -3)
    x[:, 0] = 256.0
    y = torch.full((N, K), 2.0 ** -3)          # B^T rows (column-major B)
    y[:, 0] = 256.0
    # codes with scale 1 (the values are exact E4M3 numbers)
    qa = torch.from_numpy(fp8.encode_e4m3(x.numpy())).to(d)
    qb = torch.from_numpy(fp8.encode_e4m3(y.numpy())).to(d)
    one = torch.ones((), dtype=torch.float32, device=d)
    c = m.gemm(qa.view(torch.float8_e4m3fn), qb.view(torch.float8_e4m3fn).t(), out_dtype=torch.float32,
               scale_a=one, scale_b=one, config=m.Config(mode="dp", tile_m=128, tile_n=128))
    exact = 2.0 ** 16 + (K - 1) * 2.0 ** -6
    got = to_np(c)
    err = float(np.max(np.abs(got - exact)))
    S = exact
    assert err <= 5e-5 * S, (K, err)
    lost = err / 2.0 ** -6      # small products lost
    print(f"K={K}: exact {exact!r}, max |err| {err} = {lost:.1f} of the {K - 1} small products")

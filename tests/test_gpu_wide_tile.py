"""GPU parity of the 256 x 512 CTA-pair tile (two N = 256 MMAs per k-step
into one 512-column TMEM accumulator).

A data-parallel tile sums each output element over the same k-blocks in
the same order as the 256 x 256 pair (the MMA splits only the columns), so
DP results are bit-identical to it; Stream-K plans split tiles differently
and are checked exactly on small integers and within the oracle's bound on
random inputs.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from oracle import fp8
from gpu_common import assert_sampled, assert_within_bound, dev, same_strides, sk as _sk, to_np

pytestmark = pytest.mark.gpu

W = dict(tile_m=256, tile_n=512)


@pytest.fixture(scope="module")
def m():
    return _sk()


def _dev(a, b):
    d = dev()
    return same_strides(a, d), same_strides(b, d)


@pytest.mark.parametrize("out_dtype", [torch.bfloat16, torch.float32])
@pytest.mark.parametrize("shape", [(256, 512, 64), (700, 1300, 1000), (1536, 1536, 8192), (520, 2100, 4104)])
def test_wide_dp_bit_identical_to_pair(m, shape, out_dtype):
    M, N, K = shape
    a, b = _dev(*workloads.gemm_inputs(M, N, K, dtype="bf16", seed=M + N))
    cw = m.gemm(a, b, out_dtype=out_dtype, config=m.Config(mode="dp", **W))
    assert m.default_workspace(dev()).status() == 0
    cp = m.gemm(a, b, out_dtype=out_dtype, config=m.Config(mode="dp", tile_m=256, tile_n=256))
    assert torch.equal(cw, cp)
    if M * N * K <= 2 ** 31:
        assert_within_bound(cw, a.cpu(), b.cpu(), out="bf16" if out_dtype == torch.bfloat16 else "f32",
                            what="256x512 dp")


@pytest.mark.parametrize("layouts", [("col", "row"), ("row", "row"), ("col", "col")])
def test_wide_transposed_layouts(m, layouts):
    """MN-major A and/or B (the pair kernel's chunked loads, B split over
    the two MMAs): DP equals the 256 x 256 pair bit for bit."""
    M, N, K = 600, 1104, 1000   # (row pitches of MN-major operands: multiples of 16 bytes)
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=7)
    d = dev()
    al, bl = layouts
    A = a.to(d) if al == "row" else a.t().contiguous().to(d).t()
    B = b.t().contiguous().to(d).t() if bl == "col" else b.contiguous().to(d)
    cw = m.gemm(A, B, out_dtype=torch.float32, config=m.Config(mode="dp", **W))
    assert m.default_workspace(d).status() == 0
    cp = m.gemm(A, B, out_dtype=torch.float32, config=m.Config(mode="dp", tile_m=256, tile_n=256))
    assert torch.equal(cw, cp), layouts
    assert_within_bound(cw, a, b, out="f32", what=f"256x512 layouts {layouts}")


@pytest.mark.parametrize("fixup", ["owner", "last_arriver", "split"])
@pytest.mark.parametrize("mode", ["sk", "hybrid1", "hybrid2"])
def test_wide_small_int_exact(m, mode, fixup):
    """Stream-K and hybrid plans with every fixup: integer inputs make every
    partial and the sum exact in FP32."""
    M, N, K = 1100, 1700, 3072
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=11, dist="int")
    ref, _ = oracle.gemm(a, b)
    A, B = _dev(a, b)
    cfg = m.Config(mode=mode, fixup=fixup, min_iters_per_unit=1, **W)
    if fixup == "split":
        cfg = m.Config(mode="sk", fixup="split", min_iters_per_unit=1, num_ctas=120, **W)   # 15 tiles x 4
    c = m.gemm(A, B, out_dtype=torch.float32, config=cfg)
    assert m.default_workspace(dev()).status() == 0
    assert np.array_equal(to_np(c), ref), (mode, fixup)


def test_wide_unit_count_sweep(m):
    """Stream-K over 1..76 pairs on two tiles: exact on integers."""
    M, N, K = 256, 1024, 2048
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=12, dist="int")
    ref, _ = oracle.gemm(a, b)
    A, B = _dev(a, b)
    for pairs in (1, 2, 3, 7, 31, 64, 76):
        c = m.gemm(A, B, out_dtype=torch.float32,
                   config=m.Config(mode="sk", num_ctas=2 * pairs, min_iters_per_unit=1, **W))
        assert m.default_workspace(dev()).status() == 0
        assert np.array_equal(to_np(c), ref), pairs


def test_wide_alpha_beta(m):
    M, N, K = 512, 1536, 1024
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=13)
    c0 = workloads.uniform((M, N), seed=14).to(torch.bfloat16)
    A, B = _dev(a, b)
    c = m.gemm(A, B, alpha=0.5, beta=-2.0, C_in=c0.to(A.device), config=m.Config(mode="hybrid2", **W))
    assert m.default_workspace(dev()).status() == 0
    assert_within_bound(c, a, b, alpha=0.5, beta=-2.0, C0=c0, out="bf16", what="256x512 alpha/beta")


def test_wide_full_size_sampled(m):
    """8192^3 on the 256 x 512 tile, DP and hybrid, on sampled rows and
    columns (first and last tiles included)."""
    d = dev()
    A = workloads.device_uniform((8192, 8192), seed=15, device=d)
    B = workloads.device_uniform((8192, 8192), seed=16, device=d).t()
    for mode in ("dp", "hybrid2"):
        c = m.gemm(A, B, config=m.Config(mode=mode, **W))
        assert m.default_workspace(d).status() == 0
        assert_sampled(c, A, B, out="bf16", tile_m=256, tile_n=512, what=f"256x512 8192^3 {mode}")


def test_wide_fp8_dp_bit_identical_to_pair(m):
    """E4M3 inputs: the 256 x 512 DP tile equals the 256 x 256 pair."""
    d = dev()
    x = workloads.normal((1024, 2048), seed=17).to(d)
    y = workloads.normal((1536, 2048), seed=18).to(d)
    qa, sa = m.quantize_e4m3(x)
    qb, sb = m.quantize_e4m3(y)
    A = qa.view(torch.float8_e4m3fn)
    Bm = qb.view(torch.float8_e4m3fn).t()   # column-major B
    cw = m.gemm(A, Bm, scale_a=sa, scale_b=sb, config=m.Config(mode="dp", **W))
    assert m.default_workspace(d).status() == 0
    cp = m.gemm(A, Bm, scale_a=sa, scale_b=sb, config=m.Config(mode="dp", tile_m=256, tile_n=256))
    assert torch.equal(cw, cp)
    cs = m.gemm(A, Bm, out_dtype=torch.float32, scale_a=sa, scale_b=sb, config=m.Config(mode="hybrid2", **W))
    assert m.default_workspace(d).status() == 0
    deq_a = fp8.dequantize_e4m3(qa.cpu().numpy(), sa.item())
    deq_b = fp8.dequantize_e4m3(qb.cpu().numpy(), sb.item()).T
    assert_within_bound(cs, deq_a, deq_b, out="f32", what="fp8 256x512 hybrid2")


def test_wide_rejections(m):
    """256 x 512 needs a CTA pair, BF16 or E4M3, and one problem."""
    d = dev()
    a = torch.zeros(256, 64, dtype=torch.bfloat16, device=d)
    b = torch.zeros(512, 64, dtype=torch.bfloat16, device=d).t()
    with pytest.raises(m.SkError):
        m.gemm(a, b, config=m.Config(tile_m=128, tile_n=512))
    with pytest.raises(m.SkError):
        m.grouped_gemm([a, a], [b, b], config=m.Config(tile_m=256, tile_n=512))
    f = torch.zeros(256, 64, dtype=torch.float32, device=d)
    g = torch.zeros(512, 64, dtype=torch.float32, device=d).t()
    with pytest.raises(m.SkError):
        m.gemm(f, g, config=m.Config(tile_m=256, tile_n=512))


def test_library_picks_wide_tile_at_8192_cube(m):
    """8192^3: the library's own choice is the 256 x 512 DP tile, and it
    equals the explicit configuration bit for bit."""
    d = dev()
    A = workloads.device_uniform((8192, 8192), seed=19, device=d)
    B = workloads.device_uniform((8192, 8192), seed=20, device=d).t()
    c = m.gemm(A, B)
    info = m.plan(m.make_problem(A, B, c))
    assert (info.tile_m, info.tile_n, info.mode) == (256, 512, m.binding.SK_MODE_DP)
    assert torch.equal(c, m.gemm(A, B, config=m.Config(mode="dp", **W)))
    assert m.default_workspace(d).status() == 0


@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_wide_f32_out_plain_stores(m, beta):
    """FP32 C whose row pitch TMA cannot store (ldc = N + 1 floats) or with
    beta != 0: the per-thread store path of the 256 x 512 tile, ragged N."""
    M, N, K = 520, 1030, 2048
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=21)
    A, B = _dev(a, b)
    d = dev()
    C = torch.empty_strided((M, N), (N + 1, 1), dtype=torch.float32, device=d)
    c0 = workloads.uniform((M, N), seed=22)
    C_in = (torch.empty_strided((M, N), (N + 1, 1), dtype=torch.float32, device=d).copy_(c0)
            if beta != 0.0 else None)   # C_in shares C's strides
    m.gemm(A, B, C, beta=beta, C_in=C_in, config=m.Config(mode="hybrid2", **W))
    assert m.default_workspace(d).status() == 0
    assert_within_bound(C, a, b, beta=beta, C0=c0 if beta != 0.0 else None, out="f32", what=f"256x512 f32 beta={beta}")

"""Parity at the full workload sizes (sampled outputs), in the library's
default launch configuration: FP8 E4M3 (8192^3 and 4096x14336x4096), the
64-problem grouped launch captured in a CUDA graph, and the autograd layer
(8192x11008x4096).  Rows/columns checked: the first and last (ragged) tile
plus random ones, against the FP64 oracle on exactly those rows/columns."""
import numpy as np
import pytest
import torch

import oracle
from oracle import fp8
import workloads
from gpu_common import assert_sampled, assert_within_bound, dev, sk, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return sk()


def _rows_cols(M, N, seed, tile_m=256, tile_n=256, n_rand=24):
    g = np.random.default_rng(seed)
    rows = set(range(min(tile_m, M))) | set(range(max(0, (M - 1) // tile_m * tile_m), M))
    cols = set(range(min(tile_n, N))) | set(range(max(0, (N - 1) // tile_n * tile_n), N))
    rows |= set(g.integers(0, M, size=n_rand).tolist())
    cols |= set(g.integers(0, N, size=n_rand).tolist())
    return sorted(rows), sorted(cols)


@pytest.mark.parametrize("shape", workloads.FP8_SHAPES)
def test_fp8_full_size_sampled(m, shape):
    M, N, K = shape
    d = dev()
    xa = workloads.device_normal((M, K), seed=500, device=d)
    xb = workloads.device_normal((N, K), seed=501, device=d)      # B^T rows (column-major B)
    qa, sa = m.quantize_e4m3(xa)
    qb, sb = m.quantize_e4m3(xb)
    c = m.gemm(qa.view(torch.float8_e4m3fn), qb.view(torch.float8_e4m3fn).t(), out_dtype=torch.bfloat16,
               scale_a=sa, scale_b=sb)
    assert m.default_workspace(d).status() == 0
    rows, cols = _rows_cols(M, N, seed=1)
    r = torch.tensor(rows, device=d)
    q = torch.tensor(cols, device=d)
    a_deq = fp8.dequantize_e4m3(qa.index_select(0, r).cpu().numpy(), sa.item())
    b_deq = fp8.dequantize_e4m3(qb.index_select(0, q).cpu().numpy(), sb.item()).T
    got = c.index_select(0, r).index_select(1, q)
    assert_within_bound(got, a_deq, b_deq, out="bf16", what=f"fp8 {shape}")
    # against the unquantised inputs: the E4M3 rounding of both operands
    # bounds the error by (2 * 2^-4 + 2^-8) * sum |a||b| (plus BF16 output)
    ref, S = oracle.gemm(xa.index_select(0, r).cpu(), xb.index_select(0, q).cpu().t())
    rel = np.abs(to_np(got) - ref) / (S + 1e-30)
    assert np.max(rel) <= 2 * 2 ** -4 + 2 ** -8 + 2 ** -8


def test_grouped_64_full_size_graph(m):
    d = dev()
    shapes = workloads.grouped_shapes(count=64, seed=0)
    As, Bs = [], []
    for i, (M, N, K) in enumerate(shapes):
        As.append(workloads.device_uniform((M, K), seed=600 + 2 * i, device=d))
        Bs.append(workloads.device_uniform((N, K), seed=601 + 2 * i, device=d).t())
    outs = [torch.empty(a.shape[0], b.shape[1], dtype=torch.bfloat16, device=d) for a, b in zip(As, Bs)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        m.grouped_gemm(As, Bs, outs)      # first call outside the capture (sets up s's workspace)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            m.grouped_gemm(As, Bs, outs)
    for o in outs:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        assert m.default_workspace(d).status() == 0
    for i, (a, b, o) in enumerate(zip(As, Bs, outs)):
        assert_sampled(o, a, b, out="bf16", n_rand=8, seed=i, what=f"grouped problem {i} {shapes[i]}")


def test_autograd_full_size_sampled(m):
    M, N, K = workloads.AUTOGRAD_SHAPE
    d = dev()
    A = workloads.device_uniform((M, K), seed=700, device=d).requires_grad_(True)
    Bm = workloads.device_uniform((N, K), seed=701, device=d).t().detach().requires_grad_(True)
    G = workloads.device_normal((M, N), seed=702, device=d, dtype=torch.bfloat16)
    C = m.sk_matmul(A, Bm)
    C.backward(G)
    torch.cuda.synchronize()
    assert m.default_workspace(d).status() == 0
    assert_sampled(C, A.detach(), Bm.detach(), out="bf16", n_rand=24, what="forward")
    # dA = G B^T (M x K), dB = A^T G (K x N): sampled rows/columns
    assert_sampled(A.grad, G, Bm.detach().t(), out="bf16", n_rand=24, what="dA")
    assert_sampled(Bm.grad, A.detach().t(), G, out="bf16", n_rand=24, what="dB")
    assert A.grad.stride() == A.stride() and Bm.grad.stride() == Bm.stride()


@pytest.mark.parametrize("f32k", ["tf32x3", "ffma"])
def test_fp32_4096_cube_sampled(m, f32k):
    """FP32 4096^3 in the library's default launch configuration for each
    FP32 kernel (3xTF32: 128x128 tiles, hybrid Stream-K over 1024 tiles),
    sampled rows/columns against the FP64 oracle within the FP32 bound."""
    d = dev()
    M = N = K = 4096
    A = workloads.device_uniform((M, K), seed=61, device=d, dtype=torch.float32)
    Bm = workloads.device_uniform((N, K), seed=62, device=d, dtype=torch.float32).t()
    C = m.gemm(A, Bm, config=m.Config(f32_kernel=f32k))
    assert m.default_workspace(d).status() == 0
    assert_sampled(C, A, Bm, out="f32", tile_m=128, tile_n=128, n_rand=32, what=f"fp32 4096^3 {f32k}")

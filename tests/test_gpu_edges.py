"""Edge cases of the tcgen05 path against the FP64 oracle: empty and
degenerate problems, the smallest TMA-legal shapes on every tile, and an
output larger than 2^31 elements (64-bit offsets in both store paths)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_common import assert_sampled, dev, same_strides, sk, to_np

pytestmark = pytest.mark.gpu

TILES = [(128, 128), (128, 256), (256, 128), (256, 256)]


@pytest.fixture(scope="module")
def m():
    return sk()


@pytest.mark.parametrize("shape", [(0, 64, 64), (64, 0, 64), (0, 0, 0)])
def test_empty_problem_is_a_no_op(m, shape):
    M, N, K = shape
    d = dev()
    a = torch.zeros(M, K, dtype=torch.bfloat16, device=d)
    b = torch.zeros(N, K, dtype=torch.bfloat16, device=d).t()
    c = torch.full((M, N), 7.0, dtype=torch.float32, device=d)
    m.gemm(a, b, c)
    assert m.default_workspace(d).status() == 0
    assert bool((c == 7.0).all())


def test_grouped_with_empty_members(m):
    d = dev()
    shapes = [(0, 256, 64), (200, 264, 136), (64, 0, 64), (130, 72, 8)]
    As, Bs, refs = [], [], []
    for i, (M, N, K) in enumerate(shapes):
        a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=120 + i, dist="int")
        As.append(a.to(d))
        Bs.append(same_strides(b, d))
        refs.append(oracle.gemm(a, b)[0])
    outs = m.grouped_gemm(As, Bs, out_dtype=torch.float32, config=m.Config(mode="sk"))
    assert m.default_workspace(d).status() == 0
    for o, r, s in zip(outs, refs, shapes):
        assert o.shape == (s[0], s[1])
        assert np.array_equal(to_np(o), r), s


@pytest.mark.parametrize("out_dtype", [torch.float32, torch.bfloat16])
def test_bf16_k_zero(m, out_dtype):
    """K = 0: C = beta * C_in (the sum over k is empty)."""
    d = dev()
    M, N = 130, 264
    a = torch.empty(M, 0, dtype=torch.bfloat16, device=d)
    b = torch.empty(N, 0, dtype=torch.bfloat16, device=d).t()
    c_in = workloads.small_int((M, N), seed=121).to(out_dtype).to(d)
    c = torch.full((M, N), 3.0, dtype=out_dtype, device=d)
    m.gemm(a, b, c, C_in=c_in, beta=0.5)
    assert torch.equal(c, (0.5 * c_in.float()).to(out_dtype))
    m.gemm(a, b, c)
    assert bool((c == 0).all())


TINY = [(1, 1, 8), (1, 8, 8), (7, 24, 40), (3, 300, 8), (257, 1, 64), (1, 4096, 8), (2, 2, 4096), (129, 130, 72)]


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("mode", ["dp", "sk"])
@pytest.mark.parametrize("shape", TINY)
def test_bf16_tiny_shapes_exact(m, shape, mode, tile):
    """The smallest shapes TMA allows (K a multiple of 8), on every tile:
    integer inputs make the FP32 result exact."""
    M, N, K = shape
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=122, dist="int")
    d = dev()
    c = m.gemm(same_strides(a, d), same_strides(b, d), out_dtype=torch.float32,
               config=m.Config(mode=mode, tile_m=tile[0], tile_n=tile[1]))
    assert m.default_workspace(d).status() == 0
    ref, _ = oracle.gemm(a, b)
    assert np.array_equal(to_np(c), ref), (shape, mode, tile)


@pytest.mark.parametrize("beta", [0.0, 1.0])
def test_bf16_output_beyond_int32_elements(m, beta):
    """C with 65536 x 32776 > 2^31 elements: the TMA store path (beta = 0)
    and the per-thread store path (beta != 0) both address past 2^31."""
    M, N, K = 65536, 32776, 64
    d = dev()
    A = workloads.device_uniform((M, K), seed=123, device=d)
    Bm = workloads.device_uniform((N, K), seed=124, device=d).t()
    C = torch.empty(M, N, dtype=torch.bfloat16, device=d)
    C_in = None
    if beta != 0.0:
        C_in = torch.zeros(M, N, dtype=torch.bfloat16, device=d)
        C_in[-3:, -40:] = 1.0      # a few nonzero entries in the far corner
    m.gemm(A, Bm, C, C_in=C_in, beta=beta)
    assert m.default_workspace(d).status() == 0
    if beta == 0.0:
        assert_sampled(C, A, Bm, out="bf16", tile_m=256, tile_n=256, what="int32-overflow C")
    else:
        # the corner holds A B + 1 for the marked entries
        r = torch.arange(M - 3, M, device=d)
        got = C.index_select(0, r)[:, -40:].float().cpu()
        want = (A.index_select(0, r).float() @ Bm[:, -40:].float()).cpu() + 1.0
        assert torch.allclose(got, want, rtol=2 ** -7, atol=2e-2)
    del C, C_in
    torch.cuda.empty_cache()


def test_default_workspace_per_stream(m):
    """Calls without a workspace on different streams use different
    workspaces, so concurrent GEMMs never share partial slots or flags;
    both give the oracle's exact result."""
    d = dev()
    a, b = workloads.gemm_inputs(600, 520, 4096, dtype="bf16", seed=130, dist="int")
    ref, _ = oracle.gemm(a, b)
    ad, bd = same_strides(a, d), same_strides(b, d)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    cfg = m.Config(mode="sk")
    wss = []
    for s in (s1, s2):
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            wss.append(m.default_workspace(d))
            outs.append(m.gemm(ad, bd, out_dtype=torch.float32, config=cfg))
    assert wss[0] is not wss[1]
    torch.cuda.synchronize()
    for s, ws, c in zip((s1, s2), wss, outs):
        assert ws.status() == 0
        assert np.array_equal(to_np(c), ref)


LONG_K = 1048616   # 16385 k-blocks of 64, the last one ragged (40)
_long_k_cache = {}


def _long_k_case(n):
    """Integer operands n x LONG_K and LONG_K x n and their FP64 oracle
    product, computed once per n."""
    if n not in _long_k_cache:
        a, b = workloads.gemm_inputs(n, n, LONG_K, dtype="bf16", seed=131, dist="int")
        _long_k_cache[n] = (a, b, oracle.gemm(a, b)[0])
    return _long_k_cache[n]


@pytest.mark.parametrize("tile,mode,fixup,ctas", [
    ((128, 128), "sk", "owner", 0),           # 152 units on one tile: the owner adds 151 partials
    ((128, 128), "sk", "last_arriver", 0),
    ((128, 128), "sk", "split", 145),         # 145 equal ranges of 113 k-blocks
    ((128, 128), "dp", "owner", 0),           # one unit walks all 16385 k-blocks
    ((256, 256), "sk", "owner", 0),           # 76 CTA pairs on one tile
    ((256, 256), "dp", "owner", 0),
])
def test_bf16_long_k_single_tile_exact(m, tile, mode, fixup, ctas):
    """K ~ 2^20 on a single output tile: every unit of the grid holds a range
    of the same tile (the longest fixup chain the unit count allows), or one
    unit runs the whole k-loop.  Integer inputs in [-2, 2] keep every partial
    and the sum below 2^24, so the FP32 result equals the FP64 oracle."""
    M, N = tile
    a, b, ref = _long_k_case(M)
    d = dev()
    cfg = m.Config(mode=mode, tile_m=tile[0], tile_n=tile[1], fixup=fixup, num_ctas=ctas, min_iters_per_unit=1)
    c = m.gemm(same_strides(a, d), same_strides(b, d), out_dtype=torch.float32, config=cfg)
    assert m.default_workspace(d).status() == 0
    info = m.plan(m.make_problem(a, b, torch.empty(M, N, dtype=torch.float32)), cfg, num_sms=152)
    assert info.tiles == 1
    assert np.array_equal(to_np(c), ref), (tile, mode, fixup)

"""GPU parity of the cluster split (SK_FIXUP_SPLIT_CLUSTER).

Each tile is cut into k = 2, 4 or 8 tile-aligned Stream-K ranges; the k
units run as one thread-block cluster and exchange, through distributed
shared memory, the blocks of their partial accumulators that the others
sum.  C must be bit-identical to the owner protocol on the same plan (the
partials added in ascending unit order), within the oracle's bound, and
the same from run to run.
"""
import numpy as np
import pytest
import torch

import workloads
from gpu_common import assert_sampled, assert_within_bound, dev, same_strides, sk as _sk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return _sk()


def _inputs(M, N, K, seed, dist="uniform"):
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=seed, dist=dist)   # A row-, B column-major
    d = dev()
    return same_strides(a, d), same_strides(b, d)


CASES = [
    # shape, tile (m, n), CTAs, units per tile
    ((1536, 1536, 8192), (256, 256), 144, 2),
    ((512, 512, 2048), (256, 256), 16, 2),
    ((700, 900, 1024), (256, 256), 48, 2),      # ragged M and N
    ((128, 8192, 16384), (128, 128), 128, 2),
    ((300, 520, 768), (128, 128), 30, 2),       # ragged
    ((600, 1000, 2048), (128, 256), 40, 2),
    ((512, 512, 8192), (256, 256), 32, 4),      # clusters of 8 CTAs (4 pairs)
    ((512, 512, 8192), (128, 128), 64, 4),
    ((512, 512, 8192), (128, 128), 128, 8),
    ((300, 520, 1024), (128, 128), 120, 8),     # ragged, 2 k-blocks per unit
    ((640, 384, 2048), (128, 256), 40, 4),
]


@pytest.mark.parametrize("out_dtype", [torch.bfloat16, torch.float32])
@pytest.mark.parametrize("shape,tile,ctas,k", CASES)
def test_cluster_split_equals_owner(m, shape, tile, ctas, k, out_dtype):
    M, N, K = shape
    a, b = _inputs(M, N, K, seed=M + N + K)
    base = dict(mode="sk", tile_m=tile[0], tile_n=tile[1], num_ctas=ctas, min_iters_per_unit=1)
    info = m.plan(m.make_problem(a, b, torch.empty(M, N, dtype=out_dtype, device=a.device)),
                  m.Config(**base, fixup="split_cluster"))
    assert info.fixup == m.binding.SK_FIXUP_SPLIT_CLUSTER
    assert info.num_ctas == k * info.tiles
    c_xs = m.gemm(a, b, config=m.Config(**base, fixup="split_cluster"), out_dtype=out_dtype)
    assert m.default_workspace(dev()).status() == 0
    c_own = m.gemm(a, b, config=m.Config(**base, fixup="owner"), out_dtype=out_dtype)
    assert torch.equal(c_xs, c_own)
    c_again = m.gemm(a, b, config=m.Config(**base, fixup="split_cluster"), out_dtype=out_dtype)
    assert torch.equal(c_xs, c_again)   # deterministic
    out = "bf16" if out_dtype == torch.bfloat16 else "f32"
    if M * N * K <= 2 ** 31:
        assert_within_bound(c_xs, a.cpu(), b.cpu(), out=out, what="cluster split")
    else:
        assert_sampled(c_xs, a, b, out=out, tile_m=tile[0], tile_n=tile[1], what="cluster split")


def test_cluster_split_small_integers_exact(m):
    """Small-integer inputs: every partial and the sum are exact in FP32."""
    M, N, K = 512, 768, 4096
    a, b = _inputs(M, N, K, seed=5, dist="int")
    for tile, ctas in (((256, 256), 24), ((128, 128), 48), ((128, 256), 24)):
        c = m.gemm(a, b, out_dtype=torch.float32,
                   config=m.Config(mode="sk", tile_m=tile[0], tile_n=tile[1], num_ctas=ctas,
                                   fixup="split_cluster", min_iters_per_unit=1))
        ref = a.double().cpu() @ b.double().cpu()
        assert np.array_equal(c.double().cpu().numpy(), ref.numpy()), tile


def test_cluster_split_alpha_beta(m):
    M, N, K = 384, 640, 2048
    a, b = _inputs(M, N, K, seed=9)
    c0 = workloads.uniform((M, N), seed=10).to(torch.bfloat16).to(a.device)
    cfg = dict(mode="sk", tile_m=128, tile_n=128, num_ctas=30, min_iters_per_unit=1)
    c_xs = m.gemm(a, b, alpha=0.75, beta=-1.25, C_in=c0, config=m.Config(**cfg, fixup="split_cluster"))
    c_own = m.gemm(a, b, alpha=0.75, beta=-1.25, C_in=c0, config=m.Config(**cfg, fixup="owner"))
    assert torch.equal(c_xs, c_own)
    assert_within_bound(c_xs, a.cpu(), b.cpu(), alpha=0.75, beta=-1.25, C0=c0.cpu(), out="bf16",
                        what="cluster split alpha/beta")


@pytest.mark.parametrize("shape", [(1536, 1536, 8192), (128, 8192, 16384)])
def test_library_picks_cluster_split(m, shape):
    """On the sweep's split shapes the library's own choice is the cluster
    split (one co-resident cluster per tile on this GPU), and its C equals
    the owner protocol's on the same plan."""
    M, N, K = shape
    a, b = _inputs(M, N, K, seed=3)
    c = m.gemm(a, b)
    info = m.plan(m.make_problem(a, b, c))
    assert info.fixup == m.binding.SK_FIXUP_SPLIT_CLUSTER, info.fixup
    cfg = dict(mode=["auto", "dp", "sk", "hybrid1", "hybrid2"][info.mode], tile_m=info.tile_m,
               tile_n=info.tile_n, num_ctas=info.num_ctas * (2 if info.tile_m == 256 else 1))
    assert torch.equal(c, m.gemm(a, b, config=m.Config(**cfg, fixup="owner")))


@pytest.mark.parametrize("shape,tile,ctas,k", [((384, 384, 2048), (128, 128), 18, 2),
                                               ((384, 384, 2048), (128, 128), 36, 4),
                                               ((384, 384, 2048), (128, 128), 72, 8),
                                               ((1024, 1024, 4096), (256, 256), 128, 4),
                                               ((520, 390, 1024), (128, 128), 80, 4)])
def test_cluster_split_3xtf32(m, shape, tile, ctas, k):
    """FP32 problems on the tensor cores (3xTF32): the cluster split equals
    the owner protocol bit for bit and meets the FP32 bound."""
    M, N, K = shape
    a, b = workloads.gemm_inputs(M, N, K, dtype="f32", seed=M + K)
    d = dev()
    a, b = same_strides(a, d), same_strides(b, d)
    base = dict(mode="sk", tile_m=tile[0], tile_n=tile[1], num_ctas=ctas, min_iters_per_unit=1,
                f32_kernel="tf32x3")
    info = m.plan(m.make_problem(a, b, torch.empty(M, N, dtype=torch.float32, device=d)),
                  m.Config(**base, fixup="split_cluster"))
    assert info.fixup == m.binding.SK_FIXUP_SPLIT_CLUSTER and info.num_ctas == k * info.tiles
    c_xs = m.gemm(a, b, config=m.Config(**base, fixup="split_cluster"))
    assert m.default_workspace(d).status() == 0
    c_own = m.gemm(a, b, config=m.Config(**base, fixup="owner"))
    assert torch.equal(c_xs, c_own)
    assert_within_bound(c_xs, a.cpu(), b.cpu(), out="f32", what="cluster split 3xTF32")

"""GPU parity of the BF16 tcgen05 Stream-K path against the FP64 oracle.

Inputs are rounded to BF16 once (by torch); the oracle sees exactly those
values.  Bounds: |C - ref| <= 5e-5 * sum_k |a_ik||b_kj| for FP32 output,
plus 2^-8 |ref| for BF16 output (its final rounding).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_common import assert_sampled, assert_within_bound, dev, same_strides, sk, to_np

pytestmark = pytest.mark.gpu

MODES = ["dp", "sk", "hybrid1", "hybrid2"]


@pytest.fixture(scope="module")
def m():
    return sk()


def _run(m, a, b, out_dtype=torch.bfloat16, **kw):
    d = dev()
    cfg = kw.pop("config", None)
    c = m.gemm(same_strides(a, d), same_strides(b, d), out_dtype=out_dtype, config=cfg, **kw)
    assert m.default_workspace(d).status() == 0
    return c


def test_bf16_first_small_dp(m):
    """Smallest case first: one whole 128x256 tile, DP, FP32 output."""
    a, b = workloads.gemm_inputs(128, 256, 64, dtype="bf16", seed=0, dist="int")
    c = _run(m, a, b, out_dtype=torch.float32, config=m.Config(mode="dp"))
    ref, _ = oracle.gemm(a, b)
    assert np.array_equal(to_np(c), ref)


def test_bf16_pair_first_small_dp(m):
    """Smallest CTA-pair case first: one whole 256x256 tile, DP, FP32 output."""
    a, b = workloads.gemm_inputs(256, 256, 64, dtype="bf16", seed=0, dist="int")
    c = _run(m, a, b, out_dtype=torch.float32, config=m.Config(mode="dp", tile_m=256))
    ref, _ = oracle.gemm(a, b)
    assert np.array_equal(to_np(c), ref)


TILES = [(128, 128), (128, 256), (256, 128), (256, 256), (256, 512)]


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("mode", MODES)
def test_bf16_small_int_exact(m, mode, tile):
    """Integer inputs in [-2, 2]: every product and partial sum is exact in
    FP32, so the FP32-output result must equal the oracle bit for bit."""
    a, b = workloads.gemm_inputs(384, 768, 2048, dtype="bf16", seed=1, dist="int")
    ref, _ = oracle.gemm(a, b)
    c = _run(m, a, b, out_dtype=torch.float32, config=m.Config(mode=mode, tile_m=tile[0], tile_n=tile[1]))
    assert np.array_equal(to_np(c), ref), (mode, tile)


@pytest.mark.parametrize("tile_m", [128, 256])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("shape", [(300, 520, 1000), (1920, 2000, 2000), (480, 512, 512), (129, 1000, 4160)])
def test_bf16_bound_modes(m, mode, shape, tile_m):
    M, N, K = shape
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=2)
    c = _run(m, a, b, config=m.Config(mode=mode, tile_m=tile_m))
    assert_within_bound(c, a, b, out="bf16", what=f"{shape} {mode} {tile_m}")
    c32 = _run(m, a, b, out_dtype=torch.float32, config=m.Config(mode=mode, tile_m=tile_m))
    assert_within_bound(c32, a, b, out="f32", what=f"{shape} {mode} {tile_m} f32-out")


def test_bf16_identity(m):
    """A = I: C = B exactly in every mode (B's values are BF16 already)."""
    K = 512
    a = torch.eye(K, dtype=torch.bfloat16)
    b = workloads.gemm_inputs(K, 700, K, dtype="bf16", seed=3)[1]
    for mode in MODES:
        c = _run(m, a, b, config=m.Config(mode=mode))
        assert torch.equal(c.cpu(), b.contiguous()), mode


def test_bf16_rank_one(m):
    """A_ik = u_i, B_kj = v_j (small integers): C = K u v^T exactly."""
    M, N, K = 200, 300, 1024
    u = workloads.small_int((M,), seed=4)
    v = workloads.small_int((N,), seed=5)
    a = u[:, None].expand(M, K).to(torch.bfloat16).contiguous()
    b = workloads.as_layout(v[None, :].expand(K, N).to(torch.bfloat16), "col")
    c = _run(m, a, b, out_dtype=torch.float32, config=m.Config(mode="sk"))
    assert np.array_equal(to_np(c), K * np.outer(u.numpy(), v.numpy()))


@pytest.mark.parametrize("tile_m", [128, 256])
def test_bf16_unit_count_sweep(m, tile_m):
    sms = torch.cuda.get_device_properties(dev()).multi_processor_count
    a, b = workloads.gemm_inputs(384, 768, 4096, dtype="bf16", seed=6, dist="int")
    ref, _ = oracle.gemm(a, b)
    for g in sorted({2, 3, 4, 7, 14, sms // 2, sms - 1, sms} | ({1} if tile_m == 128 else set())):
        for mode in ("sk", "hybrid2"):
            c = _run(m, a, b, out_dtype=torch.float32,
                     config=m.Config(mode=mode, num_ctas=g, min_iters_per_unit=1, tile_m=tile_m))
            assert np.array_equal(to_np(c), ref), (g, mode)


@pytest.mark.parametrize("stages", [2, 3, 4])
def test_bf16_stages(m, stages):
    a, b = workloads.gemm_inputs(640, 1280, 1536, dtype="bf16", seed=7, dist="int")
    ref, _ = oracle.gemm(a, b)
    c = _run(m, a, b, out_dtype=torch.float32, config=m.Config(mode="hybrid2", stages=stages))
    assert np.array_equal(to_np(c), ref)


def test_bf16_beta(m):
    M, N, K = 260, 530, 776   # K * 2 bytes must be a multiple of 16 (TMA)
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=8)
    d = dev()
    c0 = workloads.uniform((M, N), seed=9).to(torch.bfloat16)
    out = torch.empty(M, N, dtype=torch.bfloat16, device=d)
    m.gemm(a.to(d), b.to(d), out, alpha=1.25, beta=-0.5, C_in=c0.to(d), config=m.Config(mode="sk"))
    assert m.default_workspace(d).status() == 0
    ref, S = oracle.gemm(a, b, alpha=1.25, beta=-0.5, C0=c0)
    tol = oracle.bound(S, ref, "bf16", beta_c0=-0.5 * oracle.to_f64(c0))
    assert np.all(np.abs(to_np(out) - ref) <= tol)


@pytest.mark.parametrize("tile_m", [128, 256])
@pytest.mark.parametrize("al,bl,cl", [("col", "col", "row"), ("row", "row", "row"),
                                      ("col", "row", "row"), ("row", "col", "col"),
                                      ("col", "row", "col")])
def test_bf16_transposed_layouts(m, al, bl, cl, tile_m):
    """MN-major operands (A column-major / B row-major) and column-major C,
    on the single-CTA and the CTA-pair kernel."""
    M, N, K = 328, 272, 648   # multiples of 8: 16-byte leading dimensions for TMA
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", a_layout=al, b_layout=bl, seed=10, dist="int")
    d = dev()
    out = workloads.as_layout(torch.empty(M, N, dtype=torch.float32), cl)
    out = torch.empty_strided(out.shape, out.stride(), dtype=torch.float32, device=d)
    m.gemm(same_strides(a, d), same_strides(b, d), out, config=m.Config(mode="sk", tile_m=tile_m))
    assert m.default_workspace(d).status() == 0
    ref, _ = oracle.gemm(a, b)
    assert np.array_equal(to_np(out), ref), (al, bl, cl)


def test_bf16_rejects_unaligned_leading_dimension(m):
    """K = 777 BF16 elements is not a 16-byte row pitch: TMA cannot read it,
    so the call must fail before launching anything."""
    d = dev()
    a = torch.zeros(64, 777, dtype=torch.bfloat16, device=d)
    b = torch.zeros(777, 64, dtype=torch.bfloat16, device=d)
    with pytest.raises(m.SkError) as e:
        m.gemm(a, b)
    assert e.value.status == m.binding.SK_ERR_UNSUPPORTED


def test_bf16_deterministic(m):
    a, b = workloads.gemm_inputs(1536, 1536, 8192, dtype="bf16", seed=11)
    d = dev()
    ad, bd = a.to(d), b.to(d)
    for tile_m in (128, 256):
        for mode in ("sk", "hybrid2"):
            c1 = m.gemm(ad, bd, config=m.Config(mode=mode, tile_m=tile_m))
            c2 = m.gemm(ad, bd, config=m.Config(mode=mode, tile_m=tile_m))
            assert torch.equal(c1, c2), (mode, tile_m)


def test_bf16_timeout_status_and_recovery(m):
    d = dev()
    a, b = workloads.gemm_inputs(512, 512, 4096, dtype="bf16", seed=12)
    ad, bd = a.to(d), b.to(d)
    ws = m.Workspace(d)
    sms = torch.cuda.get_device_properties(d).multi_processor_count
    # owner protocol on every tile (count fixed), then the split reduce
    # (512 x 512 = 4 pair tiles on 64 pairs: k = 16)
    for cfg in (dict(tile_m=128, num_ctas=sms), dict(tile_m=256, num_ctas=sms),
                dict(tile_m=256, tile_n=256, num_ctas=128, fixup="split")):
        m.gemm(ad, bd, config=m.Config(mode="sk", timeout_ns=50_000_000, debug_flags=1, **cfg), workspace=ws)
        assert ws.status(clear=True) == m.binding.SK_ERR_TIMEOUT, cfg
        m.binding.check(m.binding.sk_workspace_init(ws.ptr, ws.nbytes, None))
        c = m.gemm(ad, bd, config=m.Config(mode="sk", **cfg), workspace=ws)
        assert ws.status() == 0
        assert_within_bound(c, a, b, out="bf16", what=f"after timeout {cfg}")


@pytest.mark.parametrize("shape", workloads.BF16_SWEEP)
def test_bf16_sweep_full_size_sampled(m, shape):
    """The sweep shapes at full size, in the launch configuration the
    benchmark times (library defaults), checked on sampled rows/columns
    including the first and the (ragged) last tile."""
    M, N, K = shape
    d = dev()
    a = workloads.device_uniform((M, K), seed=100, device=d)
    b = workloads.device_uniform((N, K), seed=101, device=d).t()   # column-major K x N
    c = m.gemm(a, b)
    assert m.default_workspace(d).status() == 0
    assert_sampled(c, a, b, out="bf16", what=str(shape))
    cdp = m.gemm(a, b, config=m.Config(mode="dp"))
    assert_sampled(cdp, a, b, out="bf16", what=str(shape) + " dp")
    c128 = m.gemm(a, b, config=m.Config(tile_m=128))
    assert_sampled(c128, a, b, out="bf16", what=str(shape) + " 128-row tiles")


def test_trace_timeline(m):
    """Per-CTA timeline tracing: every launched CTA records start/end, every
    item's MMA and epilogue events in order, and the result is unchanged."""
    a, b = workloads.gemm_inputs(768, 1024, 2048, dtype="bf16", seed=13, dist="int")
    d = dev()
    ref, _ = oracle.gemm(a, b)
    for tile_m in (128, 256):
        c, ev = m.trace_gemm(a.to(d), b.to(d), out_dtype=torch.float32,
                             config=m.Config(mode="sk", tile_m=tile_m))
        assert np.array_equal(to_np(c), ref)
        active = [e for e in ev if e]
        assert len(active) >= 2
        for evs in active:
            names = [n for n, _, _ in evs]
            assert names[:2] == ["entry", "start"]
            assert sorted(i for n, i, _ in evs if n == "end") == [0, 1, 2]   # every role reported
            t_end = max(t for n, _, t in evs if n == "end")
            assert all(t <= t_end for _, _, t in evs)
            for it in {i for n, i, _ in evs if n == "mma_begin"}:
                t = {n: tt for n, i, tt in evs if i == it and n != "start" and n != "end"}
                if "epi_end" in t and "mma_begin" in t:
                    assert t["mma_begin"] <= t["mma_end"] <= t["epi_end"]

"""The last-arriver fixup against the owner-waits fixup and the FP64 oracle.

Both protocols add the partials of a split tile in the same order (the
partial holding k-block 0, then the other units' partials by ascending unit
index), so their outputs must agree bit for bit whatever the arrival order
was; the oracle bound holds for both.  Counters must be back at zero after
every call, so calls with either protocol can share one workspace.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import fp8
import workloads
from gpu_common import assert_within_bound, dev, same_strides, sk, to_np

pytestmark = pytest.mark.gpu

TILES = [(128, 128), (128, 256), (256, 128), (256, 256)]


@pytest.fixture(scope="module")
def m():
    return sk()


def _both(m, call, **cfg):
    ws = m.default_workspace(dev())
    c0 = call(m.Config(fixup="owner", **cfg))
    c1 = call(m.Config(fixup="last_arriver", **cfg))
    assert ws.status() == 0
    return c0, c1


def _flags_zero(m, ctas=None):
    """Every flag / counter word a call with `ctas` CTAs used (default: one
    per SM) is zero.  The flag region holds exactly the call's CTA count
    (rounded up to 256 bytes); the partial slots follow it."""
    ws = m.default_workspace(dev())
    if ctas is None:
        ctas = torch.cuda.get_device_properties(ws.device).multi_processor_count
    words = ws.buf[256:256 + 4 * ctas].view(torch.int32)
    return int(words.abs().sum().item()) == 0


def _ctas(m, problems, cfg):
    """CTAs of the library's plan for these problems and config."""
    info = m.plan(problems, cfg)
    return info.num_ctas * (2 if info.tile_m == 256 else 1)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("mode", ["sk", "hybrid1", "hybrid2"])
@pytest.mark.parametrize("num_ctas", [0, 6, 34])
def test_bf16_last_arriver_bitwise(m, tile, mode, num_ctas):
    # ragged M and N, K not a multiple of the 64-wide k-block
    a, b = workloads.gemm_inputs(392, 776, 1544, dtype="bf16", seed=61)
    d = dev()
    A, Bm = same_strides(a, d), same_strides(b, d)
    c0, c1 = _both(m, lambda cfg: m.gemm(A, Bm, out_dtype=torch.float32, config=cfg),
                   tile_m=tile[0], tile_n=tile[1], mode=mode, num_ctas=num_ctas)
    assert torch.equal(c0, c1), (tile, mode, num_ctas)
    assert _flags_zero(m, _ctas(m, m.shape_problem(392, 776, 1544),
                               m.Config(tile_m=tile[0], tile_n=tile[1], mode=mode, num_ctas=num_ctas)))


@pytest.mark.parametrize("tile", TILES)
def test_bf16_last_arriver_oracle(m, tile):
    """BF16 output, many units per tile (K = 8192 over 36 or 72 tiles)."""
    a, b = workloads.gemm_inputs(1536, 1536, 8192, dtype="bf16", seed=62)
    d = dev()
    c = m.gemm(same_strides(a, d), same_strides(b, d),
               config=m.Config(fixup="last_arriver", mode="sk", tile_m=tile[0], tile_n=tile[1]))
    assert m.default_workspace(d).status() == 0
    r = torch.arange(0, 1536, 97)
    assert_within_bound(c[r.to(d)], a[r], b, out="bf16", what=f"last-arriver {tile}")
    assert _flags_zero(m, _ctas(m, m.shape_problem(1536, 1536, 8192),
                               m.Config(fixup="last_arriver", mode="sk", tile_m=tile[0], tile_n=tile[1])))


def test_bf16_last_arriver_int_exact_repeat(m):
    """Integer inputs (every partial sum exact): equal to the oracle, and
    identical over repeated calls sharing the workspace with owner calls."""
    a, b = workloads.gemm_inputs(520, 1032, 4104, dtype="bf16", seed=63, dist="int")
    d = dev()
    A, Bm = same_strides(a, d), same_strides(b, d)
    ref, _ = oracle.gemm(a, b)
    for i in range(3):
        for fix in ("last_arriver", "owner"):
            c = m.gemm(A, Bm, out_dtype=torch.float32, config=m.Config(fixup=fix, mode="sk", num_ctas=76))
            assert np.array_equal(to_np(c), ref), (i, fix)
    assert m.default_workspace(d).status() == 0
    assert _flags_zero(m, 76)


@pytest.mark.parametrize("num_ctas", [0, 5, 40])
def test_f32_last_arriver_bitwise(m, num_ctas):
    a, b = workloads.gemm_inputs(384, 384, 2048, dtype="f32", seed=64)
    d = dev()
    A, Bm = same_strides(a, d), same_strides(b, d)
    c0, c1 = _both(m, lambda cfg: m.gemm(A, Bm, config=cfg), mode="sk", num_ctas=num_ctas)
    assert torch.equal(c0, c1)
    assert_within_bound(c1, a, b, out="f32", what="f32 last-arriver")
    assert _flags_zero(m, _ctas(m, m.shape_problem(384, 384, 2048, dtype="f32"), m.Config(mode="sk", num_ctas=num_ctas)))


@pytest.mark.parametrize("tile_m", [128, 256])
def test_fp8_last_arriver_bitwise(m, tile_m):
    d = dev()
    xa = workloads.normal((300, 1024), seed=65)
    xb = workloads.normal((520, 1024), seed=66)
    qa, sa = m.quantize_e4m3(xa.to(d).contiguous())
    qb, sb = m.quantize_e4m3(xb.to(d).contiguous())
    A = qa.view(torch.float8_e4m3fn)
    Bm = qb.view(torch.float8_e4m3fn).t()
    c0, c1 = _both(m, lambda cfg: m.gemm(A, Bm, out_dtype=torch.float32, scale_a=sa, scale_b=sb, config=cfg),
                   mode="sk", tile_m=tile_m)
    assert torch.equal(c0, c1)
    deq_a = fp8.dequantize_e4m3(qa.cpu().numpy(), sa.item())
    deq_b = fp8.dequantize_e4m3(qb.cpu().numpy(), sb.item()).T
    assert_within_bound(c1, deq_a, deq_b, out="f32", what="fp8 last-arriver")


@pytest.mark.parametrize("tile_m", [128, 256])
def test_grouped_last_arriver_bitwise(m, tile_m):
    d = dev()
    shapes = [(256, 1024, 1024), (300, 512, 2048), (1024, 768, 128), (512, 2048, 64), (777, 256, 4096)]
    As, Bs = [], []
    for i, (M, N, K) in enumerate(shapes):
        a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=90 + i)
        As.append(a.to(d))
        Bs.append(b.to(d))
    o0, o1 = _both(m, lambda cfg: m.grouped_gemm(As, Bs, out_dtype=torch.float32, config=cfg),
                   mode="sk", tile_m=tile_m)
    for x, y, s in zip(o0, o1, shapes):
        assert torch.equal(x, y), s
    assert _flags_zero(m, _ctas(m, [m.shape_problem(*s) for s in shapes], m.Config(mode="sk", tile_m=tile_m)))


def test_backward_last_arriver_bitwise(m):
    a, b = workloads.gemm_inputs(264, 392, 520, dtype="bf16", seed=67)
    d = dev()
    dC = workloads.draw((264, 392), 69, "uniform").to(torch.bfloat16).to(d)
    A, Bm = same_strides(a, d), same_strides(b, d)
    r0, r1 = _both(m, lambda cfg: m.gemm_backward(A, Bm, dC, config=cfg), mode="sk")
    assert torch.equal(r0[0], r1[0]) and torch.equal(r0[1], r1[1])


# ---------------------------------------------------------------- split reduce
# Plans where every unit holds one range inside one tile: each tile's k
# contributors all spill, wait for each other, and each sums a share of the
# tile in the owner protocol's order -- so the bits must match it exactly.

@pytest.mark.parametrize("num_ctas", [144, 72, 36, 18])
def test_f32_split_bitwise(m, num_ctas):
    a, b = workloads.gemm_inputs(384, 384, 2048, dtype="f32", seed=150)   # 9 tiles, k = num_ctas / 9
    d = dev()
    A, Bm = same_strides(a, d), same_strides(b, d)
    c0 = m.gemm(A, Bm, config=m.Config(mode="sk", num_ctas=num_ctas, fixup="owner"))
    c1 = m.gemm(A, Bm, config=m.Config(mode="sk", num_ctas=num_ctas, fixup="split"))
    assert m.default_workspace(d).status() == 0
    assert torch.equal(c0, c1)
    assert_within_bound(c1, a, b, out="f32", what="f32 split")
    assert _flags_zero(m, num_ctas)


# (tile, num_ctas, shape): 600 x 600 = 9 pair tiles or 25 128-row tiles, K = 4096
SPLIT_BF16 = [((256, 256), 144, (600, 600, 4096)),    # 9 tiles on 72 pairs: k = 8
              ((256, 256), 36, (600, 600, 4096)),     # k = 2
              ((256, 128), 120, (600, 600, 4096)),    # 15 tiles on 60 pairs: k = 4
              ((128, 128), 100, (600, 520, 4096)),    # 25 tiles: k = 4
              ((128, 256), 80, (600, 900, 4096))]     # 20 tiles: k = 4


@pytest.mark.parametrize("tile,num_ctas,shape", SPLIT_BF16)
@pytest.mark.parametrize("out_dtype", [torch.float32, torch.bfloat16])
def test_bf16_split_bitwise(m, tile, num_ctas, shape, out_dtype):
    M, N, K = shape
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=151)
    cfg = dict(mode="sk", tile_m=tile[0], tile_n=tile[1], num_ctas=num_ctas)
    p = m.shape_problem(M, N, K)
    try:
        m.plan(p, m.Config(fixup="split", **cfg))
    except m.SkError:
        pytest.skip("not a tile-aligned plan")
    d = dev()
    A, Bm = same_strides(a, d), same_strides(b, d)
    c0 = m.gemm(A, Bm, out_dtype=out_dtype, config=m.Config(fixup="owner", **cfg))
    c1 = m.gemm(A, Bm, out_dtype=out_dtype, config=m.Config(fixup="split", **cfg))
    assert m.default_workspace(d).status() == 0
    assert torch.equal(c0, c1), (tile, num_ctas)
    assert_within_bound(c1, a, b, out="f32" if out_dtype == torch.float32 else "bf16", what="bf16 split")
    assert _flags_zero(m, num_ctas)


def test_grouped_split_bitwise(m):
    d = dev()
    shapes = [(300, 520, 2048), (600, 256, 2048)]   # 15 + 10 tiles of 128 x 128, 32 k-blocks each
    As, Bs = [], []
    for i, (M, N, K) in enumerate(shapes):
        a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=152 + i)
        As.append(a.to(d))
        Bs.append(b.to(d))
    cfg = dict(mode="sk", tile_m=128, tile_n=128, num_ctas=100)   # k = 4, ranges of 8
    o0 = m.grouped_gemm(As, Bs, out_dtype=torch.float32, config=m.Config(fixup="owner", **cfg))
    o1 = m.grouped_gemm(As, Bs, out_dtype=torch.float32, config=m.Config(fixup="split", **cfg))
    assert m.default_workspace(d).status() == 0
    for x, y in zip(o0, o1):
        assert torch.equal(x, y)
    assert _flags_zero(m, 100)


def test_fp8_split_bitwise(m):
    d = dev()
    xa = workloads.normal((512, 8192), seed=154)
    xb = workloads.normal((512, 8192), seed=155)
    qa, sa = m.quantize_e4m3(xa.to(d).contiguous())
    qb, sb = m.quantize_e4m3(xb.to(d).contiguous())
    A = qa.view(torch.float8_e4m3fn)
    Bm = qb.view(torch.float8_e4m3fn).t()
    cfg = dict(mode="sk", tile_m=256, num_ctas=128)   # 4 pair tiles, 64 pairs: k = 16, ranges of 4
    c0 = m.gemm(A, Bm, out_dtype=torch.float32, scale_a=sa, scale_b=sb, config=m.Config(fixup="owner", **cfg))
    c1 = m.gemm(A, Bm, out_dtype=torch.float32, scale_a=sa, scale_b=sb, config=m.Config(fixup="split", **cfg))
    assert m.default_workspace(d).status() == 0
    assert torch.equal(c0, c1)
    assert _flags_zero(m, 128)


def test_split_chosen_by_the_library_matches_oracle(m):
    """The library's own choice for a few-tile, long-K problem (the split
    reduce where the model prefers it), against the oracle."""
    a, b = workloads.gemm_inputs(768, 768, 32768, dtype="bf16", seed=156, dist="int")
    d = dev()
    c = m.gemm(same_strides(a, d), same_strides(b, d), out_dtype=torch.float32)
    assert m.default_workspace(d).status() == 0
    r = torch.arange(0, 768, 37)
    ref, _ = oracle.gemm(a[r], b)
    assert np.array_equal(to_np(c[r.to(d)]), ref)
    assert _flags_zero(m, _ctas(m, m.shape_problem(768, 768, 32768), m.Config()))


def test_workspace_shared_across_unit_counts(m):
    """Calls with different CTA counts share one workspace without
    re-initialisation: a call's partial slots must never land where a later
    call with more CTAs keeps its flags."""
    d = dev()
    a32, b32 = workloads.gemm_inputs(384, 384, 2048, dtype="f32", seed=160)
    abf, bbf = workloads.gemm_inputs(600, 600, 4096, dtype="bf16", seed=161, dist="int")
    A32, B32 = same_strides(a32, d), same_strides(b32, d)
    Abf, Bbf = same_strides(abf, d), same_strides(bbf, d)
    ref, _ = oracle.gemm(abf, bbf)
    for _ in range(2):
        for g in (18, 36, 72):   # few CTAs: their slots start early in the workspace
            m.gemm(A32, B32, config=m.Config(mode="sk", num_ctas=g, fixup="split"))
            m.gemm(A32, B32, config=m.Config(mode="sk", num_ctas=g))
        for fix in ("owner", "split", "last_arriver"):   # then every CTA
            cfg = dict(mode="sk", tile_m=256, num_ctas=144)
            c = m.gemm(Abf, Bbf, out_dtype=torch.float32, config=m.Config(fixup=fix, **cfg))
            assert np.array_equal(to_np(c), ref), fix
            assert _flags_zero(m, 152)
    assert m.default_workspace(d).status() == 0


def test_library_split_random_shapes(m):
    """Random shapes where the library picks the split reduce by itself:
    the result equals, bit for bit, the same plan with the owner protocol
    (integer inputs: both are also the oracle's exact result)."""
    import random
    d = dev()
    rng = random.Random(11)
    sms = torch.cuda.get_device_properties(d).multi_processor_count
    done = 0
    for _ in range(40):
        if done >= 8:
            break
        M = rng.choice([128, 200, 256, 384, 520, 768])
        N = rng.choice([128, 136, 256, 384, 512, 640])
        K = rng.choice([1024, 2048, 4096, 8192])
        dtype = rng.choice(["bf16", "f32"])
        info = m.plan(m.shape_problem(M, N, K, dtype=dtype), num_sms=sms)
        if info.fixup != m.binding.SK_FIXUP_SPLIT:
            continue
        a, b = workloads.gemm_inputs(M, N, K, dtype=dtype, seed=700 + done, dist="int")
        ad, bd = same_strides(a, d), same_strides(b, d)
        kw = {} if dtype == "f32" else {"out_dtype": torch.float32}
        c_auto = m.gemm(ad, bd, **kw)
        units = info.num_ctas
        c_owner = m.gemm(ad, bd, config=m.Config(mode="sk", tile_m=info.tile_m, tile_n=info.tile_n,
                                                 num_ctas=2 * units if info.tile_m == 256 else units), **kw)
        assert m.default_workspace(d).status() == 0
        assert torch.equal(c_auto, c_owner), (M, N, K, dtype)
        assert np.array_equal(to_np(c_auto), oracle.gemm(a, b)[0]), (M, N, K, dtype)
        done += 1
    assert done > 0

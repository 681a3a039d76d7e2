"""Device coverage counts against the oracle's schedule simulator.

The debug variant of the tensor-core kernel counts, on the GPU, which unit
issued every (tile, k-block) MAC-loop iteration and which unit stored every
32 x 32 block of C (``sk_config.coverage``).  The schedule the paper's
Background and Methodology describe requires every iteration to be computed
exactly once, by the unit the Stream-K / DP / hybrid decomposition assigns
it to, and every output element to be written exactly once.  Here the counts
the kernel took are compared with ``oracle/schedule.py``'s explicit walk over
every iteration, for each mode, unit counts g in {1, 7, 76, 151, 152} (CTA
pairs: the same CTA counts), every fixup protocol and a grouped set.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest
import torch

from oracle import schedule as sch
from gpu_common import dev, sk as _sk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return _sk()


def _operands(shapes, seed=0):
    d = dev()
    g = torch.Generator(device=d)
    g.manual_seed(seed)
    As, Bs = [], []
    for (M, N, K) in shapes:
        As.append(torch.randint(-2, 3, (M, K), generator=g, device=d).to(torch.bfloat16))
        Bs.append(torch.randint(-2, 3, (N, K), generator=g, device=d).to(torch.bfloat16).t())
    return As, Bs


_MODE = {1: "dp", 2: "sk", 3: "hybrid1", 4: "hybrid2"}


def _expected(shapes, info, cfg):
    """Oracle plan and, per global iteration, the unit that computes it
    (the resolved tile, mode and unit count come from the library's plan;
    0 iterations per unit means the library default, 4)."""
    BM, BN, BK = info.tile_m, info.tile_n, info.tile_k
    problems = []
    for (M, N, K) in shapes:
        tm, tn = sch.tile_grid(M, N, BM, BN)
        problems.append((tm * tn, -(-K // BK)))
    plan = sch.simulate(problems, info.num_ctas, _MODE[info.mode],
                        min_iters_per_unit=cfg.min_iters_per_unit or 4)
    first_iter = np.concatenate([[0], np.cumsum(plan.tiles)])
    unit_of = np.full(int(first_iter[-1]), -1, dtype=np.int64)
    contributors = [set() for _ in plan.tiles]
    owner = [None] * len(plan.tiles)
    for segs in plan.units:
        for s in segs:
            unit_of[first_iter[s.tile] + s.k0:first_iter[s.tile] + s.k1] = s.unit
            contributors[s.tile].add(s.unit)
            if s.k0 == 0:
                owner[s.tile] = s.unit
    assert (unit_of >= 0).all()
    return plan, unit_of, contributors, owner


def _check(m, shapes, cfg, grouped=False, out_dtype=torch.bfloat16):
    B = m.binding
    As, Bs = _operands(shapes)
    args = (As, Bs) if grouped else (As[0], Bs[0])
    outs, words, info = m.api.coverage_counts(*args, config=cfg, out_dtype=out_dtype)
    ws = m.default_workspace(dev())
    assert ws.status() == 0
    words = words.numpy()
    plan, unit_of, contributors, owner = _expected(shapes, info, cfg)
    n_it = unit_of.size
    blocks = (info.tile_m // 32) * (info.tile_n // 32)
    assert info.coverage_words == n_it + len(plan.tiles) * blocks
    it_words, st_words = words[:n_it], words[n_it:].reshape(len(plan.tiles), blocks)
    # every MAC-loop iteration exactly once, by the unit the oracle assigns
    bad = np.nonzero((it_words & 0xFF) != 1)[0]
    assert bad.size == 0, f"iterations visited != once: {bad[:8]} counts {it_words[bad[:8]] & 0xFF}"
    got_unit = (it_words >> 8) - 1
    bad = np.nonzero(got_unit != unit_of)[0]
    assert bad.size == 0, f"iteration {bad[0]}: unit {got_unit[bad[0]]}, oracle {unit_of[bad[0]]}"
    # every 32 x 32 block of every tile stored exactly once, by a unit that
    # computed part of the tile (the owner, under the owner protocol)
    assert ((st_words & 0xFF) == 1).all(), "output blocks stored != once"
    st_unit = (st_words >> 8) - 1
    for t in range(len(plan.tiles)):
        units = set(st_unit[t].tolist())
        assert units <= contributors[t], f"tile {t}: stored by {units}, computed by {contributors[t]}"
        if info.fixup == B.SK_FIXUP_OWNER:
            assert units == {owner[t]}, f"tile {t}: stored by {units}, owner {owner[t]}"
    # the debug variant computes what the normal kernel computes, bit for bit
    plain = dataclasses.replace(cfg, coverage=0)
    if grouped:
        ref = m.grouped_gemm(As, Bs, config=plain, out_dtype=out_dtype)
        for a, b in zip(outs, ref):
            assert torch.equal(a, b)
    else:
        assert torch.equal(outs, m.gemm(As[0], Bs[0], config=plain, out_dtype=out_dtype))
    return info


@pytest.mark.parametrize("mode", ["dp", "sk", "hybrid1", "hybrid2"])
@pytest.mark.parametrize("ctas", [1, 7, 76, 151, 152])
@pytest.mark.parametrize("tile", [(128, 128), (128, 256), (256, 256), (256, 512)])
def test_coverage_single(m, mode, ctas, tile):
    if tile[0] == 256 and ctas < 2:
        ctas = 2   # a pair is the smallest unit
    cfg = m.Config(mode=mode, tile_m=tile[0], tile_n=tile[1], num_ctas=ctas, min_iters_per_unit=1)
    _check(m, [(700, 900, 1000)], cfg)


@pytest.mark.parametrize("fixup", ["owner", "last_arriver"])
@pytest.mark.parametrize("ctas", [7, 76, 95])
def test_coverage_fixups(m, fixup, ctas):
    # the last-arriver protocol keeps two slots per CTA: 128 x 128 tiles
    cfg = m.Config(mode="sk", tile_m=128, tile_n=128, num_ctas=ctas, min_iters_per_unit=1, fixup=fixup)
    _check(m, [(520, 390, 3000)], cfg)


@pytest.mark.parametrize("shape,tile,ctas", [((384, 384, 2048), (128, 128), 144),
                                             ((512, 512, 8192), (256, 256), 128),
                                             ((1536, 1536, 8192), (256, 256), 144)])
def test_coverage_split_reduce(m, shape, tile, ctas):
    cfg = m.Config(mode="sk", tile_m=tile[0], tile_n=tile[1], num_ctas=ctas, fixup="split", min_iters_per_unit=1)
    info = _check(m, [shape], cfg)
    assert info.fixup == m.binding.SK_FIXUP_SPLIT


@pytest.mark.parametrize("shape,tile,ctas", [((384, 384, 2048), (128, 128), 18),
                                             ((700, 900, 1024), (128, 256), 48),
                                             ((1536, 1536, 8192), (256, 256), 144),
                                             ((512, 512, 8192), (256, 256), 32),
                                             ((384, 384, 2048), (128, 128), 72),
                                             ((640, 384, 2048), (128, 256), 40)])
def test_coverage_cluster_split(m, shape, tile, ctas):
    cfg = m.Config(mode="sk", tile_m=tile[0], tile_n=tile[1], num_ctas=ctas, fixup="split_cluster",
                   min_iters_per_unit=1)
    info = _check(m, [shape], cfg)
    assert info.fixup == m.binding.SK_FIXUP_SPLIT_CLUSTER


@pytest.mark.parametrize("shape", [(1536, 1536, 2048), (128, 4096, 4096), (1000, 1000, 1000), (384, 384, 2048)])
def test_coverage_library_default(m, shape):
    """The tile, mode, unit count and fixup the library picks by itself."""
    _check(m, [shape], m.Config())


@pytest.mark.parametrize("mode", ["dp", "sk", "hybrid2"])
@pytest.mark.parametrize("tile,ctas", [((128, 128), 152), ((128, 256), 7), ((256, 256), 152), ((256, 256), 14)])
def test_coverage_grouped(m, mode, tile, ctas):
    shapes = [(300, 520, 704), (1024, 256, 256), (64, 1000, 1504), (777, 333, 2048), (256, 256, 64)]
    cfg = m.Config(mode=mode, tile_m=tile[0], tile_n=tile[1], num_ctas=ctas, min_iters_per_unit=1)
    _check(m, shapes, cfg, grouped=True)

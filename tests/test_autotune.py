"""Autotuner: candidate ranking and cache on CPU; a measured tune on GPU."""
import os

import numpy as np
import pytest
import torch

import workloads


@pytest.fixture(scope="module")
def sk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_00044_gb300 as sk
    return sk


def test_candidates_ranked_and_valid(sk):
    p = sk.shape_problem(3840, 4096, 4096)
    c = sk.autotune.candidates(p, num_sms=152)
    assert len(c) >= 12
    preds = [u for _, u in c]
    assert preds == sorted(preds) and preds[0] > 0
    tiles = {(cfg.tile_m, cfg.tile_n) for cfg, _ in c}
    assert tiles == {(128, 128), (128, 256), (256, 256), (256, 512)}
    # transposed A: the CTA pair reads MN-major operands too
    p = sk.shape_problem(4096, 4096, 4096, a_layout="col")
    assert {cfg.tile_m for cfg, _ in sk.autotune.candidates(p, num_sms=152)} == {128, 256}
    # transposed E4M3 operands are refused by both kernels: no candidates
    p = sk.shape_problem(4096, 4096, 4096, dtype="e4m3", a_layout="col")
    assert sk.autotune.candidates(p, num_sms=152) == []
    # FP32: 128 x 128 tiles (3xTF32 and FFMA) and 256 x 256 pairs (3xTF32 only)
    p = sk.shape_problem(384, 384, 2048, dtype="f32")
    c = sk.autotune.candidates(p, num_sms=152)
    assert {(cfg.tile_m, cfg.tile_n) for cfg, _ in c} == {(128, 128), (256, 256)}
    assert all(cfg.f32_kernel == "tf32x3" for cfg, _ in c if cfg.tile_m == 256)
    # tiles split in two: the cluster split is among the candidates
    c = sk.autotune.candidates(sk.shape_problem(1536, 1536, 8192), num_sms=152)
    assert any(cfg.fixup == "split_cluster" for cfg, _ in c)


def test_cache_round_trip(sk, tmp_path):
    path = str(tmp_path / "tune.json")
    cache = sk.autotune.TuneCache(path)
    cfg = sk.Config(tile_m=256, tile_n=256, stages=6, mode="dp")
    cache.put("k1", cfg, 12.5)
    again = sk.autotune.TuneCache(path)
    assert again.get("k1") == cfg
    assert again.get("missing") is None


@pytest.mark.gpu
def test_tune_picks_a_fast_correct_config(sk, tmp_path):
    import oracle
    from gpu_common import assert_within_bound
    d = torch.device("cuda", torch.cuda.current_device())
    a, b = workloads.gemm_inputs(1536, 1536, 8192, dtype="bf16", seed=400)
    ad, bd = a.to(d), b.to(d)
    cache = sk.autotune.TuneCache(str(tmp_path / "t.json"))
    cfg = sk.autotune.tune(ad, bd, cache=cache, top_k=4, iters=5)
    c = sk.gemm(ad, bd, config=cfg)
    assert_within_bound(c, a, b, out="bf16", what="tuned")
    assert cache.get(next(iter(cache._load()))) == cfg

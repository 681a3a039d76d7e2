"""Measured autotuner for the Stream-K GEMM.

Candidates are every valid combination of tile (128x128, 128x256, 256x256
CTA pair), pipeline depth and decomposition (DP, SK, HYBRID1, HYBRID2),
plus, where every tile is split and there are fewer tiles than units, the
same with the unit count cut to a multiple of the tile count.  The
library's runtime model (sk_plan_query's predicted_us) ranks them; the best
`top_k` are timed on the GPU with CUDA events (L2 flushed before each run)
and the fastest is cached in a JSON file keyed by problem shape, layouts,
dtypes and SM count.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import api
from . import binding as B

_MODES = ["hybrid2", "dp", "sk", "hybrid1"]
# (256 x 128 pairs never measured faster; 256 x 512 pairs: BF16 / E4M3
# single problems, whose plan queries refuse the rest)
_TILES = [(128, 128), (128, 256), (256, 256), (256, 512)]
_STAGES = {(128, 128): (6, 4), (128, 256): (4, 3), (256, 128): (8, 6), (256, 256): (6, 4), (256, 512): (4, 3)}


def default_cache_path() -> str:
    return os.environ.get("SKGEMM_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "skgemm_tune.json"))


def problem_key(p: B.sk_problem, sms: int) -> str:
    return (f"{p.m},{p.n},{p.k}|a{p.a_type}{p.a_layout}|b{p.b_type}{p.b_layout}|"
            f"c{p.c_type}{p.c_layout}|beta{int(p.beta != 0)}|sm{sms}")


class TuneCache:
    def __init__(self, path: str | None = None):
        self.path = path or default_cache_path()
        self._lock = threading.Lock()
        self._data = None

    def _load(self):
        if self._data is None:
            try:
                with open(self.path) as f:
                    self._data = json.load(f)
            except (OSError, ValueError):
                self._data = {}
        return self._data

    def get(self, key):
        with self._lock:
            v = self._load().get(key)
        return None if v is None else api.Config(**v["config"])

    def put(self, key, cfg: api.Config, us: float):
        with self._lock:
            d = self._load()
            d[key] = {"config": cfg.__dict__, "us": us}
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            tmp = self.path + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(d, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def _try(problem, cfg, num_sms):
    try:
        return api.plan(problem, cfg, num_sms=num_sms)
    except B.SkError:
        return None


def _signature(info):
    """What the kernel runs: modes that resolve to the same split of the
    tiles give the same launch."""
    return (info.tile_m, info.tile_n, info.tile_k, info.stages, info.num_ctas, info.sk_units,
            info.sk_tiles, info.dp_tiles, info.iters_per_unit, info.extra_units, info.fixup)


def candidates(problem: B.sk_problem, num_sms: int = 0):
    """All valid configs with their predicted time, fastest first.  FP32
    problems try both FP32 kernels (3xTF32 on 128 x 128 tiles and on CTA
    pairs); where every tile is split and there are fewer tiles than units,
    the largest multiple of the tile count is tried as well, with the owner
    fixup and with the split reduce, and twice the tile count with the
    cluster split."""
    out = []
    seen = set()

    def add(cfg, info):
        sig = _signature(info)
        if sig not in seen:
            seen.add(sig)
            out.append((cfg, float(info.predicted_us)))

    f32_kernels = ["tf32x3", "ffma"] if problem.a_type == B.SK_F32 else ["auto"]
    for (tm, tn) in _TILES:
        for st in _STAGES[(tm, tn)]:
            for mode in _MODES:
                for fk in f32_kernels:
                    cfg = api.Config(tile_m=tm, tile_n=tn, stages=st, mode=mode, f32_kernel=fk)
                    if problem.a_type == B.SK_F32:
                        if st != _STAGES[(tm, tn)][0] or (tm, tn) not in ((128, 128), (256, 256)) or (
                                fk == "ffma" and tm != 128):
                            continue
                        cfg = api.Config(tile_m=tm, tile_n=tn, mode=mode, f32_kernel=fk)
                    info = _try(problem, cfg, num_sms)
                    if info is None:
                        continue
                    add(cfg, info)
                    # fewer tiles than units, all split: the largest multiple of
                    # the tile count (every tile cut into equal parts), with
                    # either fixup
                    T, g = info.tiles, info.num_ctas
                    if info.sk_tiles == T and 0 < T and 2 * T <= g:
                        per = 2 if cfg.tile_m == 256 else 1
                        for fx in ("owner", "split", "split_cluster"):
                            units = 2 * T if fx == "split_cluster" else g // T * T
                            if fx == "owner" and units == g:
                                continue   # the plan above
                            cfg2 = api.Config(tile_m=cfg.tile_m, tile_n=cfg.tile_n, stages=cfg.stages,
                                              mode=cfg.mode, num_ctas=per * units, fixup=fx,
                                              f32_kernel=fk)
                            info2 = _try(problem, cfg2, num_sms)
                            if info2 is not None:
                                add(cfg2, info2)
    out.sort(key=lambda x: x[1])
    return out


def _time_config(A, Bm, out, cfg, ws, warmup, iters, flush):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        api.gemm(A, Bm, out, config=cfg, workspace=ws)
    times = []
    for _ in range(iters):
        if flush is not None:
            flush[0].fill_(1.0)
            torch.sum(flush[0], dim=0, out=flush[1])
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        api.gemm(A, Bm, out, config=cfg, workspace=ws)
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b) for a, b in times)
    return ms[len(ms) // 2] * 1e3   # median, microseconds


def tune(A: torch.Tensor, Bm: torch.Tensor, out: torch.Tensor | None = None, *, out_dtype=None,
         top_k: int = 6, warmup: int = 3, iters: int = 10, flush_l2: bool = True,
         cache: TuneCache | None = None, force: bool = False):
    """Return the fastest measured Config for C = A @ B (cached)."""
    if out is None:
        dt = out_dtype or (torch.float32 if A.dtype == torch.float32 else torch.bfloat16)
        out = torch.empty((A.shape[0], Bm.shape[1]), dtype=dt, device=A.device)
    prob = api.make_problem(A, Bm, out)
    sms = torch.cuda.get_device_properties(A.device).multi_processor_count
    key = problem_key(prob, sms)
    cache = cache or TuneCache()
    if not force:
        hit = cache.get(key)
        if hit is not None:
            return hit
    ws = api.default_workspace(A.device)
    flush = None
    if flush_l2:
        flush = (torch.empty(64 << 20, dtype=torch.float32, device=A.device),
                 torch.empty((), dtype=torch.float32, device=A.device))
    ranked = candidates(prob)[:max(1, top_k)]
    best = None
    for cfg, _pred in ranked:
        us = _time_config(A, Bm, out, cfg, ws, warmup, iters, flush)
        if best is None or us < best[1]:
            best = (cfg, us)
    cache.put(key, best[0], best[1])
    return best[0]


def gemm_tuned(A: torch.Tensor, Bm: torch.Tensor, out: torch.Tensor | None = None, **kw):
    """api.gemm with the autotuned config for this shape."""
    cfg = tune(A, Bm, out, out_dtype=kw.get("out_dtype"))
    return api.gemm(A, Bm, out, config=cfg, **kw)

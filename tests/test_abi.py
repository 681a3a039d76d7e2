"""C-ABI checks that need no GPU: the library loads, exports every entry
point include/skgemm.h declares, rejects bad arguments before launching, and
its host-side scheduler (the same code the kernels run) reproduces the
oracle's schedule simulator exactly."""
import ctypes
import os
import random
import re

import pytest

from oracle import schedule as sch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_00044_gb300 as sk
    return sk


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "skgemm.h")).read()
    return sorted(set(re.findall(r"SK_API\s+[\w\s\*]+?\b(sk_\w+)\s*\(", txt)))


def test_header_declares_expected_api():
    syms = header_symbols()
    for name in ("sk_gemm", "sk_gemm_grouped", "sk_gemm_backward", "sk_workspace_size",
                 "sk_get_status", "sk_status_string"):
        assert name in syms


def test_library_exports_every_declared_symbol(sk):
    lib = ctypes.CDLL(sk.binding.LIB_PATH)
    for name in header_symbols():
        assert hasattr(lib, name), name
    assert set(header_symbols()) == set(sk.binding.declared_symbols())


def test_status_strings(sk):
    B = sk.binding
    assert B.sk_status_string(B.SK_OK) == "SK_OK"
    assert B.sk_status_string(B.SK_ERR_TIMEOUT) == "SK_ERR_TIMEOUT"
    assert B.sk_status_string(99) == "SK_ERR_UNKNOWN"


def _q(sk, p, cfg=None, sms=148):
    B = sk.binding
    arr = (B.sk_problem * 1)(p)
    info = B.sk_plan_info()
    c = sk.api._cfg(cfg)
    return B.sk_plan_query(arr, 1, ctypes.byref(c), sms, ctypes.byref(info)), info


def test_argument_errors(sk):
    B = sk.binding
    p = sk.shape_problem(64, 64, 64)
    assert _q(sk, p)[0] == B.SK_OK
    bad = sk.shape_problem(64, 64, 64)
    bad.m = -1
    assert _q(sk, bad)[0] == B.SK_ERR_INVALID_ARG
    bad = sk.shape_problem(64, 64, 64)
    bad.lda = 10        # < K for row-major A
    assert _q(sk, bad)[0] == B.SK_ERR_INVALID_ARG
    bad = sk.shape_problem(64, 64, 64)
    bad.b_type = B.SK_F32   # mixed input types
    assert _q(sk, bad)[0] == B.SK_ERR_UNSUPPORTED
    bad = sk.shape_problem(64, 64, 64)
    bad.A = None
    assert _q(sk, bad)[0] == B.SK_ERR_INVALID_ARG
    bad = sk.shape_problem(64, 64, 64)
    bad.beta = 1.0      # beta != 0 needs C_in
    assert _q(sk, bad)[0] == B.SK_ERR_INVALID_ARG
    assert _q(sk, p, {"tile_n": 96})[0] == B.SK_ERR_UNSUPPORTED
    assert _q(sk, p, {"num_ctas": 149}, sms=148)[0] == B.SK_ERR_INVALID_ARG
    assert _q(sk, p, {"stages": 9})[0] == B.SK_ERR_UNSUPPORTED
    assert _q(sk, p, {"mode": 7})[0] == B.SK_ERR_INVALID_ARG
    # m == 0: valid, nothing to do
    z = sk.shape_problem(0, 64, 64)
    assert _q(sk, z)[0] == B.SK_OK


def test_workspace_size(sk):
    B = sk.binding
    p = sk.shape_problem(384, 384, 2048, dtype="f32")
    n = ctypes.c_size_t(0)
    c = sk.api._cfg({"num_ctas": 148})
    assert B.sk_workspace_size(ctypes.byref(p), 1, ctypes.byref(c), ctypes.byref(n)) == B.SK_OK
    assert n.value == 256 + 4096 + 148 * 128 * 128 * 4
    p = sk.shape_problem(384, 384, 2048)
    c = sk.api._cfg({"num_ctas": 148, "tile_m": 128, "tile_n": 256})
    assert B.sk_workspace_size(ctypes.byref(p), 1, ctypes.byref(c), ctypes.byref(n)) == B.SK_OK
    assert n.value == 256 + 4096 + 148 * 128 * 256 * 4
    # pairs: one 128 x tile_n slot per CTA as well
    for tn in (256, 128):
        c = sk.api._cfg({"num_ctas": 148, "tile_m": 256, "tile_n": tn})
        assert B.sk_workspace_size(ctypes.byref(p), 1, ctypes.byref(c), ctypes.byref(n)) == B.SK_OK
        assert n.value == 256 + 4096 + 148 * 128 * tn * 4
    # 256 x 128 pairs are BF16 only
    q8 = sk.shape_problem(384, 384, 2048, dtype="e4m3")
    c = sk.api._cfg({"num_ctas": 148, "tile_m": 256, "tile_n": 128})
    assert B.sk_workspace_size(ctypes.byref(q8), 1, ctypes.byref(c), ctypes.byref(n)) == B.SK_ERR_UNSUPPORTED
    # whatever the library picks fits one 128 x 512 slot per CTA (the widest
    # tile, 256 x 512 pairs, which it picks for 8192^3)
    for shape in [(384, 384, 2048), (8192, 8192, 8192), (128, 8192, 16384)]:
        c = sk.api._cfg({"num_ctas": 148})
        q = sk.shape_problem(*shape)
        assert B.sk_workspace_size(ctypes.byref(q), 1, ctypes.byref(c), ctypes.byref(n)) == B.SK_OK
        assert n.value <= 256 + 4096 + 148 * 128 * 512 * 4
    # the last-arriver fixup keeps a second slot per CTA (owner segments)
    for tile in ((128, 128), (128, 256), (256, 256)):
        c = sk.api._cfg({"num_ctas": 148, "tile_m": tile[0], "tile_n": tile[1], "fixup": "last_arriver"})
        assert B.sk_workspace_size(ctypes.byref(p), 1, ctypes.byref(c), ctypes.byref(n)) == B.SK_OK
        assert n.value == 256 + 4096 + 2 * 148 * 128 * tile[1] * 4
    c = sk.api._cfg({"num_ctas": 148, "fixup": 4})
    assert B.sk_workspace_size(ctypes.byref(p), 1, ctypes.byref(c), ctypes.byref(n)) == B.SK_ERR_INVALID_ARG
    # the cluster split exchanges partials between shared memories: no slots
    q = sk.shape_problem(1536, 1536, 8192)
    c = sk.api._cfg({"num_ctas": 144, "tile_m": 256, "mode": "sk", "fixup": "split_cluster"})
    assert B.sk_workspace_size(ctypes.byref(q), 1, ctypes.byref(c), ctypes.byref(n)) == B.SK_OK
    assert n.value == 256 + 4096


def test_split_reduce_eligibility(sk):
    """The split reduce needs every unit to hold one range inside one tile;
    the library picks it by itself only together with the unit count."""
    B = sk.binding
    f32 = sk.shape_problem(384, 384, 2048, dtype="f32")   # 9 tiles of 16 k-blocks
    # 144 = 16 units per tile, ranges of 8 k-blocks: eligible
    info = sk.plan(f32, sk.Config(mode="sk", num_ctas=144, fixup="split"), num_sms=152)
    assert info.fixup == B.SK_FIXUP_SPLIT and info.extra_units == 0
    # 152 units: unequal ranges crossing tile boundaries: refused
    with pytest.raises(sk.SkError):
        sk.plan(f32, sk.Config(mode="sk", num_ctas=152, fixup="split"), num_sms=152)
    # DP tiles present: refused
    with pytest.raises(sk.SkError):
        sk.plan(sk.shape_problem(8192, 8192, 8192), sk.Config(mode="hybrid2", tile_m=256, fixup="split"), num_sms=152)
    # an explicit owner request is kept when the count is fixed
    info = sk.plan(f32, sk.Config(mode="sk", num_ctas=144), num_sms=152)
    assert info.fixup == B.SK_FIXUP_OWNER
    # left to the library: the tile-aligned count with the split reduce
    info = sk.plan(f32, num_sms=152)
    assert info.num_ctas % info.tiles == 0
    if info.fixup == B.SK_FIXUP_SPLIT:
        ctas = info.num_ctas * (2 if info.tile_m == 256 else 1)
        same = sk.Config(mode="sk", num_ctas=ctas, tile_m=info.tile_m, tile_n=info.tile_n, fixup="split")
        for u in range(info.num_ctas):
            its = sk.unit_items(f32, u, same, num_sms=152)
            assert len(its) == 1


def test_default_workspace_fits_both_fixups(sk):
    """The default workspace holds the largest plan of either fixup."""
    B = sk.binding
    n = ctypes.c_size_t(0)
    sms = 148
    default = 256 + 4096 + 2 * sms * 128 * 512 * 4
    assert sk.api.default_workspace_bytes(sms) == default
    for fix in ("owner", "last_arriver"):
        for shape in [(384, 384, 2048), (8192, 8192, 8192), (128, 8192, 16384), (1536, 1536, 8192)]:
            for tiles in ({}, {"tile_m": 256, "tile_n": 512}):   # library choice; the widest tile
                c = sk.api._cfg({"num_ctas": sms, "fixup": fix, **tiles})
                q = sk.shape_problem(*shape)
                assert B.sk_workspace_size(ctypes.byref(q), 1, ctypes.byref(c), ctypes.byref(n)) == B.SK_OK
                assert n.value <= default


def test_gemm_without_device_reports_no_device(sk):
    """No GPU here: the call must fail cleanly, never fall back."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    B = sk.binding
    p = sk.shape_problem(64, 64, 64)
    c = sk.api._cfg(None)
    assert B.sk_gemm(ctypes.byref(p), ctypes.byref(c), None, 0, None) == B.SK_ERR_NO_DEVICE


def _lib_schedule(sk, problems_shapes, cfg, sms, dtype="bf16"):
    probs = [sk.shape_problem(M, N, K, dtype=dtype) for (M, N, K) in problems_shapes]
    B = sk.binding
    arr = (B.sk_problem * len(probs))(*probs)
    info = B.sk_plan_info()
    c = sk.api._cfg(cfg)
    assert B.sk_plan_query(arr, len(probs), ctypes.byref(c), sms, ctypes.byref(info)) == B.SK_OK
    units = [sk.unit_items(probs, u, config=cfg, num_sms=sms) for u in range(info.num_ctas)]
    return info, units


_ROLE = {0: "whole", 1: "owner", 2: "peer", 3: "dp"}


def _compare(sk, shapes, mode, sms, dtype="bf16", tile_n=0, min_ipu=1, tile_m=0):
    cfg = {"mode": mode, "tile_n": tile_n, "min_iters_per_unit": min_ipu, "tile_m": tile_m, "num_ctas": sms}
    info, units = _lib_schedule(sk, shapes, cfg, sms, dtype)
    BM, BN, BK = info.tile_m, info.tile_n, info.tile_k
    problems = []
    for (M, N, K) in shapes:
        tm, tn = sch.tile_grid(M, N, BM, BN)
        problems.append((tm * tn, -(-K // BK)))
    g = info.num_ctas              # units: CTAs, or CTA pairs for 256-row tiles
    assert g == (sms // 2 if BM == 256 else sms)
    plan = sch.simulate(problems, g, mode, min_iters_per_unit=min_ipu)
    assert info.sk_tiles == plan.sk_tiles
    assert info.sk_iters == plan.sk_iters
    assert info.sk_units == plan.sk_units
    assert info.tiles == len(plan.tiles)
    for u in range(g):
        exp = [(s.tile, s.problem, s.local_tile, s.k0, s.k1, s.role,
                (s.peers[0], s.peers[-1]) if s.role == "owner" else None)
               for s in plan.units[u]]
        got = [(w.global_tile, w.problem, w.tile, w.k0, w.k1, _ROLE[w.role],
                (w.peer_first, w.peer_last) if w.role == 1 else None)
               for w in units[u]]
        assert got == exp, f"unit {u}"
    # rasterisation is a bijection on every problem's tile grid
    for p, (M, N, K) in enumerate(shapes):
        tm_n, tn_n = sch.tile_grid(M, N, BM, BN)
        coords = {}
        for us in units:
            for w in us:
                if w.problem == p:
                    assert 0 <= w.tile_row < tm_n and 0 <= w.tile_col < tn_n
                    coords.setdefault(w.tile, set()).add((w.tile_row, w.tile_col))
        flat = [c for s in coords.values() for c in s]
        assert all(len(s) == 1 for s in coords.values())
        assert len(set(flat)) == len(flat) == tm_n * tn_n


@pytest.mark.parametrize("mode", sch.MODES)
def test_host_scheduler_matches_simulator_sweep_shapes(sk, mode):
    for shape in [(3840, 4096, 4096), (1536, 1536, 8192), (2048, 7168, 1024),
                  (128, 8192, 16384), (1920, 2000, 2000), (480, 512, 512), (1, 1, 1)]:
        _compare(sk, [shape], mode, 148)


@pytest.mark.parametrize("mode", sch.MODES)
def test_host_scheduler_matches_simulator_random(sk, mode):
    rnd = random.Random(99)
    for _ in range(40):
        nprob = rnd.choice([1, 1, 2, 4, 9])
        shapes = [(rnd.randint(1, 1500), rnd.randint(1, 1500), rnd.randint(1, 3000)) for _ in range(nprob)]
        sms = rnd.randint(1, 152)
        _compare(sk, shapes, mode, sms, dtype=rnd.choice(["bf16", "f32", "e4m3"]),
                 min_ipu=rnd.choice([1, 1, 4]))


def test_tile_selection(sk):
    B = sk.binding
    # K-major operands and m >= 256: CTA pairs with 256 x 256 tiles
    info = _q(sk, sk.shape_problem(3840, 4096, 4096))[1]
    assert (info.tile_m, info.tile_n, info.num_ctas) == (256, 256, 74)
    # m <= 128 (memory-bound) or FP32: 128-row tiles; with fewer tiles than
    # CTAs the count is every SM or a multiple of the tile count
    for p in (sk.shape_problem(128, 8192, 16384), sk.shape_problem(384, 384, 2048, dtype="f32")):
        info = _q(sk, p)[1]
        assert info.tile_m == 128
        assert info.num_ctas == 148 or (info.tiles < 148 and info.num_ctas % info.tiles == 0)
    # a caller's explicit count is kept
    info = _q(sk, sk.shape_problem(384, 384, 2048, dtype="f32"), {"num_ctas": 148})[1]
    assert info.num_ctas == 148


@pytest.mark.parametrize("shape", [(512, 512, 8192), (256, 256, 65536), (1280, 1280, 8192), (640, 640, 16384)])
def test_library_split_choice_is_eligible(sk, shape):
    """When the library picks the split reduce by itself (possibly with
    fewer units than the largest tile-aligned count, so that the ranges
    divide every tile's k-blocks), each unit holds exactly one range."""
    B = sk.binding
    p = sk.shape_problem(*shape)
    info = sk.plan(p, num_sms=152)
    if info.fixup != B.SK_FIXUP_SPLIT:
        return
    units = info.num_ctas
    assert units % info.tiles == 0 and info.extra_units == 0
    k = units // info.tiles
    assert (-(-shape[2] // info.tile_k)) % k == 0
    cfg = sk.Config(mode="sk", tile_m=info.tile_m, tile_n=info.tile_n,
                    num_ctas=2 * units if info.tile_m == 256 else units)
    for u in range(units):
        assert len(sk.unit_items(p, u, cfg, num_sms=152)) == 1


def test_fault_injection_keeps_the_owner_protocol(sk):
    """With the test-only injection set (peers withhold their flags), the
    library never picks the split reduce (through the workspace or the
    cluster) by itself, and the decision cache keeps the two requests apart."""
    B = sk.binding
    p = sk.shape_problem(384, 384, 2048, dtype="f32")
    split = (B.SK_FIXUP_SPLIT, B.SK_FIXUP_SPLIT_CLUSTER)
    assert sk.plan(p, num_sms=152).fixup in split
    assert sk.plan(p, sk.Config(debug_flags=1), num_sms=152).fixup == B.SK_FIXUP_OWNER
    assert sk.plan(p, num_sms=152).fixup in split


def test_f32_kernel_choice(sk):
    """FP32 problems go to the 3xTF32 tensor-core kernel (32-deep k-blocks)
    when both operands are K-major and TMA-aligned, else to the FFMA
    kernel (16-deep); an explicit 3xTF32 request on other layouts is
    refused, an unknown kernel value is invalid."""
    B = sk.binding
    kmaj = sk.shape_problem(384, 384, 2048, dtype="f32")
    assert sk.plan(kmaj, num_sms=152).tile_k == 32
    assert sk.plan(kmaj, sk.Config(f32_kernel="ffma"), num_sms=152).tile_k == 16
    assert sk.plan(kmaj, sk.Config(f32_kernel="tf32x3"), num_sms=152).tile_k == 32
    for kw in ({"b_layout": "row"}, {"a_layout": "col"}):
        p = sk.shape_problem(384, 384, 2048, dtype="f32", **kw)
        assert sk.plan(p, num_sms=152).tile_k == 16
        with pytest.raises(sk.SkError):
            sk.plan(p, sk.Config(f32_kernel="tf32x3"), num_sms=152)
    assert _q(sk, kmaj, {"f32_kernel": 3})[0] == B.SK_ERR_INVALID_ARG
    # the 3xTF32 tile is 128 x 128 on single CTAs or 256 x 256 on CTA pairs
    pair = sk.plan(kmaj, sk.Config(f32_kernel="tf32x3", tile_m=256), num_sms=152)
    assert (pair.tile_m, pair.tile_n, pair.tile_k, pair.stages) == (256, 256, 32, 3)
    with pytest.raises(sk.SkError):
        sk.plan(kmaj, sk.Config(f32_kernel="tf32x3", tile_m=256, tile_n=128), num_sms=152)
    with pytest.raises(sk.SkError):
        sk.plan(kmaj, sk.Config(f32_kernel="ffma", tile_m=256), num_sms=152)


def test_tile_aligned_unit_count(sk):
    """With fewer tiles than units and the count left to the library, the
    runtime model may cut every tile into equal parts: k x T units, each
    tile then split among exactly k of them."""
    p = sk.shape_problem(1536, 1536, 8192)
    for cfg in ({"tile_m": 256, "tile_n": 256, "mode": "sk"}, {"tile_m": 128, "tile_n": 256, "mode": "sk"}):
        B = sk.binding
        info = B.sk_plan_info()
        c = sk.api._cfg(cfg)
        arr = (B.sk_problem * 1)(p)
        # tile and mode fixed by the caller: the count stays every unit
        assert B.sk_plan_query(arr, 1, ctypes.byref(c), 152, ctypes.byref(info)) == B.SK_OK
        assert info.num_ctas == (76 if cfg["tile_m"] == 256 else 152)
    info = sk.plan(p, num_sms=152)   # everything left to the library
    assert info.num_ctas in (info.tiles * (76 // info.tiles) if info.tile_m == 256 else info.tiles * (152 // info.tiles),
                             76 if info.tile_m == 256 else 152)
    for u in range(info.num_ctas):
        for it in sk.unit_items(p, u, num_sms=152):
            if it.role == 1:   # owner: with k = g / T units per tile, exactly k - 1 peers
                k = info.num_ctas // info.tiles
                if info.num_ctas % info.tiles == 0:
                    assert it.peer_last - it.peer_first + 1 == k - 1
    # transposed (MN-major) BF16 operands may use pairs
    assert _q(sk, sk.shape_problem(4096, 4096, 4096, b_layout="row"), {"tile_m": 256})[0] == B.SK_OK
    # E4M3 transposed operands are refused by either kernel
    assert _q(sk, sk.shape_problem(4096, 4096, 4096, dtype="e4m3", b_layout="row"), {"tile_m": 256})[0] == \
        B.SK_ERR_UNSUPPORTED


@pytest.mark.parametrize("tile_m", [128, 256])
def test_host_scheduler_explicit_tiles(sk, tile_m):
    for mode in sch.MODES:
        for shape in [(3840, 4096, 4096), (2048, 7168, 1024), (300, 700, 5000)]:
            _compare(sk, [shape], mode, 152, tile_m=tile_m)


def test_host_scheduler_unit_count_sweep(sk):
    """The paper's 'compute unit' bug appeared for sub-maximal CU counts:
    every g from 1 to 152 must give the simulator's exact schedule."""
    for g in range(1, 153):
        _compare(sk, [(384, 384, 2048)], "sk", g, dtype="f32")
        _compare(sk, [(480, 512, 512)], "hybrid2", g)


@pytest.mark.parametrize("group", [1, 3, 8, 16, 64])
def test_raster_group_is_a_bijection(sk, group):
    """Any rasterisation group keeps the schedule identical to the simulator
    (tile indices) and maps tile indices one-to-one onto the tile grid."""
    B = sk.binding
    for shape in [(3840, 4096, 4096), (8192, 8192, 8192), (300, 2000, 700)]:
        _compare(sk, [shape], "hybrid2", 152, tile_m=256)
        cfg = {"mode": "dp", "raster_group": group, "tile_m": 128}
        probs = [sk.shape_problem(*shape)]
        info = sk.plan(probs, sk.Config(**cfg), num_sms=152)
        seen = set()
        for u in range(info.num_ctas):
            for w in sk.unit_items(probs, u, config=sk.Config(**cfg), num_sms=152):
                seen.add((w.tile_row, w.tile_col))
        tm = -(-shape[0] // info.tile_m)
        tn = -(-shape[1] // info.tile_n)
        assert seen == {(i, j) for i in range(tm) for j in range(tn)}
    bad = sk.shape_problem(64, 64, 64)
    assert _q(sk, bad, {"raster_group": 65})[0] == B.SK_ERR_INVALID_ARG


def test_layout_of_vector_operands(sk):
    """A single row or column is contiguous in both layouts; the preferred
    (K-major) one is returned, with a 16-element-padded leading dimension."""
    import torch
    B = sk.binding
    col = torch.empty(8, 1)
    assert sk.api.layout_of(col, B.SK_COL_MAJOR) == (B.SK_COL_MAJOR, 16)
    assert sk.api.layout_of(col.t().contiguous().t(), B.SK_COL_MAJOR) == (B.SK_COL_MAJOR, 16)
    row = torch.empty(1, 40)
    assert sk.api.layout_of(row, B.SK_ROW_MAJOR) == (B.SK_ROW_MAJOR, 48)
    # not vectors: the strides decide
    assert sk.api.layout_of(torch.empty(8, 24), B.SK_COL_MAJOR) == (B.SK_ROW_MAJOR, 24)
    assert sk.api.layout_of(torch.empty(24, 8).t(), B.SK_ROW_MAJOR) == (B.SK_COL_MAJOR, 8)
    # a K x 1 B plans on the tensor-core path (it used to read as row-major, ld 1)
    a = torch.empty(257, 64, dtype=torch.bfloat16)
    b = torch.empty(64, 1, dtype=torch.bfloat16)
    c = torch.empty(257, 1, dtype=torch.float32)
    p = sk.make_problem(a, b, c)
    assert (p.b_layout, p.ldb) == (B.SK_COL_MAJOR, 64)
    assert sk.plan(p, sk.Config(tile_m=128, tile_n=128), num_sms=152).tiles == 3


def test_library_split_choice_on_random_problem_sets(sk):
    """Random single and grouped problem sets: whenever the library picks
    the split reduce by itself, the plan it returns has every unit holding
    exactly one range (the kernels' precondition), the unit count is a
    multiple of the tile count, and the ranges cover every tile once."""
    import random
    B = sk.binding
    rng = random.Random(7)
    picked = 0
    for _ in range(60):
        n = rng.choice([1, 1, 1, 2, 3])
        shapes = [(rng.choice([128, 256, 384, 512, 768, 1024]), rng.choice([128, 256, 384, 512, 768]),
                   rng.choice([1024, 2048, 4096, 8192, 16384])) for _ in range(n)]
        dtype = rng.choice(["bf16", "bf16", "f32"])
        probs = [sk.shape_problem(*s, dtype=dtype) for s in shapes]
        info = sk.plan(probs, num_sms=152)
        if info.fixup != B.SK_FIXUP_SPLIT:
            continue
        picked += 1
        units = info.num_ctas
        assert units % info.tiles == 0 and info.extra_units == 0
        cfg = sk.Config(mode="sk", tile_m=info.tile_m, tile_n=info.tile_n,
                        num_ctas=2 * units if info.tile_m == 256 else units, fixup="split")
        seen = {}
        for u in range(units):
            its = sk.unit_items(probs, u, cfg, num_sms=152)
            assert len(its) == 1, (shapes, u)
            it = its[0]
            seen.setdefault((it.problem, it.tile), []).append((it.k0, it.k1))
        assert len(seen) == info.tiles
        for (p, t), ranges in seen.items():
            ranges.sort()
            assert ranges[0][0] == 0
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            assert ranges[-1][1] == -(-shapes[p][2] // info.tile_k)
    assert picked > 0


def test_workspace_size_large_groups(sk):
    """Up to 64 problems travel in the kernel's parameter block; a larger
    group's problem table is sized into the workspace (growing with the
    count), and more than 65536 problems are refused."""
    B = sk.binding
    n = ctypes.c_size_t(0)
    c = sk.api._cfg({"num_ctas": 148, "tile_m": 128, "tile_n": 128})

    def size(count):
        arr = (B.sk_problem * count)(*[sk.shape_problem(64 + i, 128, 256) for i in range(count)])
        assert B.sk_workspace_size(arr, count, ctypes.byref(c), ctypes.byref(n)) == B.SK_OK
        return n.value

    base = 256 + 4096 + 148 * 128 * 128 * 4
    assert size(1) == base and size(64) == base
    s65, s256 = size(65), size(256)
    assert base < s65 < s256
    assert (s65 - base) % 256 == 0 and (s256 - base) % 256 == 0
    # the FFMA kernel's records are smaller than the tensor-core ones (no tensor maps)
    f = sk.api._cfg({"num_ctas": 148, "f32_kernel": "ffma"})
    arr = (B.sk_problem * 256)(*[sk.shape_problem(64 + i, 128, 256, dtype="f32") for i in range(256)])
    assert B.sk_workspace_size(arr, 256, ctypes.byref(f), ctypes.byref(n)) == B.SK_OK
    assert base < n.value < s256
    big = (B.sk_problem * 65537)()
    assert B.sk_workspace_size(big, 65537, ctypes.byref(c), ctypes.byref(n)) == B.SK_ERR_INVALID_ARG


def test_coverage_words(sk):
    """sk_plan_info.coverage_words: one word per MAC-loop iteration of every
    tile of every problem, then one per 32 x 32 block of every tile."""
    B = sk.binding
    shapes = [(300, 520, 700), (1024, 256, 256), (64, 1000, 1500)]
    for cfg in ({"tile_m": 128, "tile_n": 128}, {"tile_m": 128, "tile_n": 256}, {"tile_m": 256, "tile_n": 256}):
        probs = [sk.shape_problem(*s) for s in shapes]
        info = sk.plan(probs, cfg, num_sms=152)
        BM, BN, BK = info.tile_m, info.tile_n, info.tile_k
        tiles = [sch.tile_grid(M, N, BM, BN) for (M, N, K) in shapes]
        iters = sum(tm * tn * -(-K // BK) for (tm, tn), (M, N, K) in zip(tiles, shapes))
        ntiles = sum(tm * tn for tm, tn in tiles)
        assert info.coverage_words == iters + ntiles * (BM // 32) * (BN // 32)
    assert B.sk_config().coverage is None   # NULL by default: the normal kernels run


def test_cluster_split_eligibility(sk):
    """SK_FIXUP_SPLIT_CLUSTER runs only where every tile has 2, 4 or 8
    tile-aligned units (at most 8 CTAs per cluster), on one BF16 or 3xTF32
    problem, with 128-row tiles or 256 x 256 pairs, and where the operand
    ring holds the exchanged blocks; elsewhere the request is
    SK_ERR_UNSUPPORTED."""
    B = sk.binding

    def q(shape, cfg, dtype="bf16", count=1):
        probs = [sk.shape_problem(*shape, dtype=dtype)] * count
        arr = (B.sk_problem * count)(*probs)
        info = B.sk_plan_info()
        c = sk.api._cfg(cfg)
        return B.sk_plan_query(arr, count, ctypes.byref(c), 152, ctypes.byref(info)), info

    xs = {"mode": "sk", "fixup": "split_cluster"}
    for shape, cfg, dt, k in [
            ((1536, 1536, 8192), {"tile_m": 256, "num_ctas": 144}, "bf16", 2),   # 36 tiles, 72 pairs
            ((512, 512, 8192), {"tile_m": 256, "num_ctas": 32}, "bf16", 4),     # 4 tiles, 16 pairs
            ((128, 8192, 16384), {"tile_m": 128, "tile_n": 128, "num_ctas": 128}, "bf16", 2),
            ((512, 512, 8192), {"tile_m": 128, "tile_n": 128, "num_ctas": 64}, "bf16", 4),
            ((512, 512, 8192), {"tile_m": 128, "tile_n": 128, "num_ctas": 128}, "bf16", 8),
            ((384, 384, 2048), {"tile_m": 128, "num_ctas": 72}, "f32", 8),        # 3xTF32, 9 tiles
            ((1024, 1024, 4096), {"tile_m": 256, "num_ctas": 128}, "f32", 4)]:   # 3xTF32 pairs
        rc, info = q(shape, {**xs, **cfg}, dtype=dt)
        assert rc == B.SK_OK and info.fixup == B.SK_FIXUP_SPLIT_CLUSTER, (shape, cfg)
        assert info.num_ctas == k * info.tiles, (shape, cfg)
    # not k units per tile, three units per tile, 8 pairs per tile (16 CTAs),
    # BF16 output with 8 units of 128 x 256 (the ring misses the blocks), the
    # FFMA kernel, E4M3, 256 x 128 pairs, two problems
    for shape, cfg, dt, cnt in [((1536, 1536, 8192), {"tile_m": 256, "num_ctas": 152}, "bf16", 1),
                                ((1536, 1536, 8192), {"tile_m": 256, "num_ctas": 108}, "bf16", 1),
                                ((512, 512, 8192), {"tile_m": 256, "num_ctas": 64}, "bf16", 1),
                                ((384, 384, 2048), {"tile_m": 128, "num_ctas": 18, "f32_kernel": "ffma"}, "f32", 1),
                                ((1536, 1536, 8192), {"tile_m": 256, "num_ctas": 144}, "e4m3", 1),
                                ((1536, 1536, 8192), {"tile_m": 256, "tile_n": 128, "num_ctas": 144}, "bf16", 1),
                                ((1536, 1536, 8192), {"tile_m": 256, "num_ctas": 144}, "bf16", 2)]:
        rc, _ = q(shape, {**xs, **cfg}, dtype=dt, count=cnt)
        assert rc == B.SK_ERR_UNSUPPORTED, (shape, cfg, dt, cnt)


def test_wide_pair_tile_plans(sk):
    """256 x 512 pair tiles: the tile grid is ceil(M/256) x ceil(N/512), the
    workspace holds a 128 x 512 FP32 slot per CTA, and the tile is refused
    off a CTA pair, for FP32, and for groups."""
    B = sk.binding
    p = sk.shape_problem(8192, 8192, 8192)
    info = sk.plan(p, sk.Config(tile_m=256, tile_n=512, mode="dp"), num_sms=152)
    assert (info.tile_m, info.tile_n, info.num_ctas, info.tiles) == (256, 512, 76, 32 * 16)
    assert info.stages == 4   # 48 KB stages
    assert info.workspace_bytes >= 152 * 128 * 512 * 4
    r = sk.plan(sk.shape_problem(700, 1300, 1000), sk.Config(tile_m=256, tile_n=512), num_sms=152)
    assert r.tiles == 3 * 3
    fp8 = sk.plan(sk.shape_problem(4096, 4096, 4096, dtype="e4m3"), sk.Config(tile_m=256, tile_n=512), num_sms=152)
    assert fp8.tile_n == 512
    for bad in (dict(tile_m=128, tile_n=512), dict(tile_m=256, tile_n=384)):
        with pytest.raises(sk.SkError):
            sk.plan(p, sk.Config(**bad), num_sms=152)
    with pytest.raises(sk.SkError):
        sk.plan(sk.shape_problem(1024, 1024, 1024, dtype="f32"), sk.Config(tile_m=256, tile_n=512), num_sms=152)
    with pytest.raises(sk.SkError):
        sk.plan([p, p], sk.Config(tile_m=256, tile_n=512), num_sms=152)
    assert B.SK_OK == 0


def test_backward_workspace_size(sk):
    """The backward's workspace: the two GEMMs' bytes, then one K-major copy
    per operand they would read MN-major (for the usual row-major A and
    column-major B: B for dA, A and dC for dB)."""
    B = sk.binding
    M, N, K = 8192, 11008, 4096
    fwd = sk.shape_problem(M, N, K)
    cfg = sk.Config(num_ctas=152).to_c()   # an SM count: no device needed
    n = ctypes.c_size_t(0)
    assert B.sk_gemm_backward_workspace_size(ctypes.byref(fwd), 1, 1, ctypes.byref(cfg), ctypes.byref(n)) == B.SK_OK
    copies = (K * N + K * M + M * N) * 2
    assert copies <= n.value <= copies + 256 + 4096 + 2 * 152 * 128 * 512 * 4 + 4 * 256
    # dA only: B's copy
    assert B.sk_gemm_backward_workspace_size(ctypes.byref(fwd), 1, 0, ctypes.byref(cfg), ctypes.byref(n)) == B.SK_OK
    assert K * N * 2 <= n.value < (K * N + K * M) * 2
    # both operands already in the backward's K-major order: no copies
    t = sk.shape_problem(M, N, K, a_layout="col", b_layout="row")
    assert B.sk_gemm_backward_workspace_size(ctypes.byref(t), 1, 0, ctypes.byref(cfg), ctypes.byref(n)) == B.SK_OK
    assert n.value < 256 + 4096 + 2 * 152 * 128 * 512 * 4 + 256
    f32 = sk.shape_problem(64, 64, 64, dtype="f32")
    assert B.sk_gemm_backward_workspace_size(ctypes.byref(f32), 1, 1, ctypes.byref(cfg), ctypes.byref(n)) == B.SK_ERR_UNSUPPORTED


def test_model_picks_wide_tile_for_long_k_dp(sk):
    """The runtime model takes 256 x 512 pairs, data-parallel, where they
    measured faster (long K, few tiles per pair) and 256 x 256 pairs where
    they measured slower (K = 4096, many tiles per pair, short shapes)."""
    def pick(M, N, K):
        i = sk.plan(sk.shape_problem(M, N, K), None, num_sms=152)
        return (i.tile_m, i.tile_n, i.mode)
    DP = sk.binding.SK_MODE_DP
    for shape in [(8192, 8192, 8192), (8192, 8192, 16384), (6144, 6144, 12288), (8192, 8192, 12288),
                  (16384, 16384, 8192), (3072, 3072, 16384)]:
        assert pick(*shape) == (256, 512, DP), shape
    for shape in [(8192, 8192, 4096), (4096, 14336, 4096), (16384, 16384, 4096), (3840, 4096, 4096),
                  (2048, 7168, 1024), (1536, 1536, 8192), (8192, 16384, 8192), (16384, 8192, 8192),
                  (12288, 12288, 8192), (2048, 2048, 32768)]:
        assert pick(*shape)[1] != 512, shape
    # never for groups, FP32, or Stream-K / hybrid plans of the library's own
    g = sk.plan([sk.shape_problem(8192, 8192, 8192)] * 2, None, num_sms=152)
    assert g.tile_n != 512
    f = sk.plan(sk.shape_problem(8192, 8192, 8192, dtype="f32"), None, num_sms=152)
    assert f.tile_n != 512


def test_backward_workspace_covers_single_launch_plans(sk):
    """The operand copies sit after the largest GEMM workspace the backward
    may use: the grouped plan or either single-problem plan (here 8192^3,
    whose single plans take 256 x 512 tiles with 128 x 512 slots)."""
    B = sk.binding
    cfg = sk.Config(num_ctas=152).to_c()
    fwd = sk.shape_problem(8192, 8192, 8192)
    n = ctypes.c_size_t(0)
    assert B.sk_gemm_backward_workspace_size(ctypes.byref(fwd), 1, 1, ctypes.byref(cfg), ctypes.byref(n)) == B.SK_OK
    single = ctypes.c_size_t(0)
    dA = sk.shape_problem(8192, 8192, 8192, b_layout="row")   # dA = dC B^T with B read MN-major
    assert B.sk_workspace_size(ctypes.byref(dA), 1, ctypes.byref(cfg), ctypes.byref(single)) == B.SK_OK
    assert single.value >= 152 * 128 * 512 * 4 // 2           # a 256 x 512 pair plan
    copies = 3 * 8192 * 8192 * 2                               # B, A and dC
    assert n.value >= single.value + copies


def test_transpose16_argument_checks(sk):
    """sk_transpose16 refuses bad arguments before touching a device, and an
    empty matrix is nothing to do."""
    B = sk.binding
    L = B.load()
    buf = (ctypes.c_uint16 * 64)()
    p = ctypes.addressof(buf)
    assert L.sk_transpose16(None, 4, 4, 4, None, 4, None) == B.SK_ERR_INVALID_ARG
    assert L.sk_transpose16(p, 4, 8, 4, p, 4, None) == B.SK_ERR_INVALID_ARG       # ld_src < cols
    assert L.sk_transpose16(p, 8, 4, 4, p, 4, None) == B.SK_ERR_INVALID_ARG       # ld_dst < rows
    assert L.sk_transpose16(p + 1, 4, 4, 4, p, 4, None) == B.SK_ERR_INVALID_ARG   # odd address
    assert L.sk_transpose16(p, -1, 4, 4, p, 4, None) == B.SK_ERR_INVALID_ARG
    assert L.sk_transpose16(None, 0, 5, 5, None, 1, None) == B.SK_OK

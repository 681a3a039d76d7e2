"""Pins for the Stream-K schedule simulator (CPU only).

The simulator is checked against invariants that any correct Stream-K
decomposition must satisfy, against closed forms of the hybrid rule, by
brute-force enumeration of tiny shapes, and by executing a schedule in FP64
and comparing with the plain triple-loop oracle.
"""
import itertools
import random

import numpy as np
import pytest

import oracle
from oracle import schedule as sch
import workloads


def check_invariants(plan, problems):
    g = plan.g
    tiles = plan.tiles
    T = len(tiles)
    # 1. coverage: every (tile, k) exactly once
    seen = {}
    for u, segs in enumerate(plan.units):
        for s in segs:
            assert s.unit == u
            assert 0 <= s.k0 < s.k1 <= tiles[s.tile]
            for k in range(s.k0, s.k1):
                key = (s.tile, k)
                assert key not in seen, f"{key} covered twice"
                seen[key] = u
    assert len(seen) == sum(tiles)
    # 2. SK balance: per-unit SK iteration counts differ by <= 1
    sk_counts = [sum(s.k1 - s.k0 for s in segs if s.role != "dp") for segs in plan.units]
    active = sk_counts[:plan.sk_units]
    if active:
        assert max(active) - min(active) <= 1
        assert sum(active) == plan.sk_iters
    assert all(c == 0 for c in sk_counts[plan.sk_units:])
    # 3. DP tiles whole, after SK, in whole waves for the hybrid modes
    for segs in plan.units:
        roles = [s.role for s in segs]
        if "dp" in roles:
            first_dp = roles.index("dp")
            assert all(r == "dp" for r in roles[first_dp:])
    dp_tiles = T - plan.sk_tiles
    if plan.mode in ("hybrid1", "hybrid2") and T > g:
        assert dp_tiles % g == 0
    # 4. owners and peers
    by_tile = {}
    for segs in plan.units:
        for s in segs:
            by_tile.setdefault(s.tile, []).append(s)
    for t, segs in by_tile.items():
        if len(segs) == 1:
            assert segs[0].role in ("whole", "dp")
            continue
        owners = [s for s in segs if s.role == "owner"]
        assert len(owners) == 1
        o = owners[0]
        assert o.k0 == 0
        peers = sorted((s for s in segs if s.role == "peer"), key=lambda s: s.unit)
        assert o.peers == [p.unit for p in peers]
        assert all(p.unit > o.unit for p in peers)
        # contributing units are consecutive and their k ranges chain
        units = [o.unit] + o.peers
        assert units == list(range(o.unit, o.unit + len(units)))
        k = o.k1
        for p in peers:
            assert p.k0 == k
            k = p.k1
        assert k == tiles[t]
    # 5. a unit is a peer at most once, and only in its first segment, so it
    #    needs one workspace slot; the wait graph (owner -> higher peers)
    #    is therefore acyclic
    for u, segs in enumerate(plan.units):
        peer_idx = [i for i, s in enumerate(segs) if s.role == "peer"]
        assert len(peer_idx) <= 1
        if peer_idx:
            assert peer_idx[0] == 0
    # 6. owner segment, if any, is the unit's last SK segment
    for segs in plan.units:
        sk = [s for s in segs if s.role != "dp"]
        for i, s in enumerate(sk):
            if s.role == "owner":
                assert i == len(sk) - 1


@pytest.mark.parametrize("mode", sch.MODES)
def test_invariants_random(mode):
    rnd = random.Random(1234)
    for _ in range(150):
        nprob = rnd.choice([1, 1, 1, 2, 5])
        problems = [(rnd.randint(1, 40), rnd.randint(1, 12)) for _ in range(nprob)]
        g = rnd.randint(1, 48)
        plan = sch.simulate(problems, g, mode)
        check_invariants(plan, problems)


@pytest.mark.parametrize("g", list(range(1, 153)))
def test_invariants_every_unit_count(g):
    """Sweep g = 1 .. 152 (the 'compute unit' count the paper's Methodology
    and Results found broken for sub-maximal values)."""
    for mode in sch.MODES:
        for problems in ([(9, 64)], [(480, 64)], [(2048, 128)], [(64, 256)], [(7, 3), (300, 5)]):
            check_invariants(sch.simulate(problems, g, mode), problems)


def test_min_iters_guard():
    plan = sch.simulate([(9, 32)], 148, "sk", min_iters_per_unit=4)
    assert plan.sk_units == 288 // 4
    check_invariants(plan, [(9, 32)])
    plan = sch.simulate([(1, 1)], 148, "sk")
    assert plan.sk_units == 1


def test_hybrid_closed_forms():
    g = 148
    for T in (1, 9, 147, 148, 149, 295, 296, 297, 480, 2048):
        assert sch.count_sk_tiles(T, g, "hybrid1") == T % g
        exp2 = T if T <= g else (0 if T % g == 0 else g + T % g)
        assert sch.count_sk_tiles(T, g, "hybrid2") == exp2
        assert sch.count_sk_tiles(T, g, "dp") == 0
        assert sch.count_sk_tiles(T, g, "sk") == T
    # 2048 tiles of 8192^2 at 128x256 over 148 units: 1776 DP tiles (12 waves),
    # 272 SK tiles (1.84 tiles per unit)
    plan = sch.simulate([(2048, 128)], 148, "hybrid2")
    assert plan.sk_tiles == 148 + 2048 % 148 == 272
    dp = sum(1 for segs in plan.units for s in segs if s.role == "dp")
    assert dp == 1776 and dp % 148 == 0


def test_split_tile_count_bound():
    """At most sk_units - 1 tiles are split (each range boundary inside a tile
    creates at most one split)."""
    for g in (1, 7, 64, 148):
        for problems in ([(9, 64)], [(300, 17)], [(33, 5), (1, 200)]):
            plan = sch.simulate(problems, g, "sk")
            owners = sum(1 for segs in plan.units for s in segs if s.role == "owner")
            assert owners <= max(0, plan.sk_units - 1)


def test_brute_force_tiny():
    """Enumerate all tiny shapes with 16x16 tiles and k-block 8 and check
    invariants plus FP64 execution against the plain oracle."""
    BM = BN = 16
    BK = 8
    for M, N, K in itertools.product((1, 16, 17, 40), (5, 32, 48), (1, 8, 9, 64)):
        tm, tn = sch.tile_grid(M, N, BM, BN)
        I = -(-K // BK)
        A = workloads.small_int((M, K), seed=M * 1000 + K).numpy()
        B = workloads.small_int((K, N), seed=N * 1000 + K + 1).numpy()
        Cref, _ = oracle.gemm(A, B)
        for g in (1, 2, 3, 5, 8):
            for mode in sch.MODES:
                plan = sch.simulate([(tm * tn, I)], g, mode)
                check_invariants(plan, [(tm * tn, I)])
                C = sch.execute_fp64(A, B, plan, M, N, K, BM, BN, BK)
                assert np.array_equal(C, Cref), (M, N, K, g, mode)


def test_execute_random_alpha_beta():
    M, N, K, BM, BN, BK = 100, 70, 200, 32, 16, 16
    A = workloads.uniform((M, K), seed=31).numpy()
    B = workloads.uniform((K, N), seed=32).numpy()
    C0 = workloads.uniform((M, N), seed=33).numpy()
    Cref, S = oracle.gemm(A, B, alpha=0.75, beta=-1.25, C0=C0)
    tm, tn = sch.tile_grid(M, N, BM, BN)
    for g in (3, 11, 29):
        for mode in sch.MODES:
            plan = sch.simulate([(tm * tn, -(-K // BK))], g, mode)
            C = sch.execute_fp64(A, B, plan, M, N, K, BM, BN, BK, alpha=0.75,
                                 beta=-1.25, C0=C0)
            assert np.max(np.abs(C - Cref) / (S + 1)) < 1e-13

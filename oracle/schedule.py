"""Stream-K / data-parallel / hybrid schedule simulator -- TEST INFRASTRUCTURE ONLY.

An independent restatement of the work decomposition, written as an explicit
walk over every MAC-loop iteration rather than with closed-form index
arithmetic, so that it shares no logic with the GPU scheduler it checks.

The decomposition (the paper defers to Osama et al., PPoPP 2023, for the
method -- Introduction, Background, Methodology, Future Work):

* The output is cut into tiles; tile t needs I_t MAC-loop iterations
  (one per k-block).  Tiles of several problems are concatenated.
* Data-parallel (DP): each tile is computed whole by one unit; tile j of
  the DP set goes to unit j mod g (Background, Fig. 1: the last wave of
  this scheme is what leaves cores idle).
* Stream-K (SK): the iterations of the SK tiles, laid end to end, are split
  into g contiguous ranges whose lengths differ by at most one (the first
  ``r = total mod g`` ranges get one extra iteration).
* Hybrid: the first ``sk_tiles`` tiles are SK, the rest are DP in whole
  waves.  "two-tile SK + DP" (HYBRID2): sk_tiles = g + T mod g when T > g
  and T mod g != 0, all tiles when T <= g, none when T mod g == 0.
  "one-tile SK + DP" (HYBRID1): sk_tiles = T mod g.
* A range cut inside a tile makes it a split tile.  The unit that holds the
  tile's first iteration (k = 0) is its owner; the others ("peers") have
  higher unit indices.  A peer writes its FP32 partial to workspace slot
  <its unit index> and raises a flag; the owner adds the peers' partials to
  its own in ascending unit order, then applies the epilogue.
* A unit does its SK range first, then its DP tiles in increasing order.

Roles: 'whole' (an SK segment that happens to cover a full tile), 'owner',
'peer', 'dp'.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MODES = ("dp", "sk", "hybrid1", "hybrid2")


@dataclass
class Segment:
    unit: int
    tile: int          # global tile index over the concatenated problems
    problem: int
    local_tile: int    # tile index within its problem
    k0: int            # first iteration (inclusive)
    k1: int            # last iteration (exclusive)
    role: str          # 'whole' | 'owner' | 'peer' | 'dp'
    peers: list = field(default_factory=list)  # owner only: ascending units


@dataclass
class Plan:
    g: int
    mode: str
    tiles: list          # I_t per global tile
    tile_problem: list   # problem index per global tile
    tile_local: list     # local tile index per global tile
    sk_tiles: int
    sk_iters: int
    sk_units: int
    units: list          # list of lists of Segment, one per unit


def count_sk_tiles(T: int, g: int, mode: str) -> int:
    """Number of leading tiles processed Stream-K for each mode."""
    if mode == "dp":
        return 0
    if mode == "sk":
        return T
    if mode == "hybrid1":
        return T % g
    if mode == "hybrid2":
        if T <= g:
            return T
        if T % g == 0:
            return 0
        return g + T % g
    raise ValueError(mode)


def simulate(problems, g: int, mode: str, min_iters_per_unit: int = 1) -> Plan:
    """problems: list of (tiles_p, iters_p).  Returns the full schedule."""
    if g < 1:
        raise ValueError("g must be >= 1")
    tiles, tile_problem, tile_local = [], [], []
    for p, (tp, ip) in enumerate(problems):
        for lt in range(tp):
            tiles.append(ip)
            tile_problem.append(p)
            tile_local.append(lt)
    T = len(tiles)
    sk_tiles = count_sk_tiles(T, g, mode)

    # Every SK iteration as (tile, k), in order.
    work = [(t, k) for t in range(sk_tiles) for k in range(tiles[t])]
    sk_iters = len(work)
    if sk_iters == 0:
        sk_units = 0
    else:
        sk_units = min(g, max(1, sk_iters // max(1, min_iters_per_unit)))

    # Hand out iterations one unit at a time: the first (sk_iters mod
    # sk_units) units take one more than the others.
    owner_of_iter = []
    if sk_units:
        base, extra = divmod(sk_iters, sk_units)
        for u in range(sk_units):
            owner_of_iter += [u] * (base + (1 if u < extra else 0))
    assert len(owner_of_iter) == sk_iters

    units = [[] for _ in range(g)]
    # Group each unit's consecutive iterations of one tile into segments.
    for idx, (t, k) in enumerate(work):
        u = owner_of_iter[idx]
        segs = units[u]
        if segs and segs[-1].tile == t and segs[-1].k1 == k:
            segs[-1].k1 = k + 1
        else:
            segs.append(Segment(u, t, tile_problem[t], tile_local[t], k, k + 1, "?"))

    # Roles and peer lists.
    by_tile = {}
    for segs in units:
        for s in segs:
            by_tile.setdefault(s.tile, []).append(s)
    for t, segs in by_tile.items():
        segs.sort(key=lambda s: s.unit)
        if len(segs) == 1:
            segs[0].role = "whole"
            continue
        for s in segs:
            s.role = "owner" if s.k0 == 0 else "peer"
        owner = [s for s in segs if s.role == "owner"]
        assert len(owner) == 1
        owner[0].peers = [s.unit for s in segs if s.role == "peer"]

    # DP tiles, round-robin, after the SK range.
    for j, t in enumerate(range(sk_tiles, T)):
        u = j % g
        units[u].append(Segment(u, t, tile_problem[t], tile_local[t], 0, tiles[t], "dp"))

    return Plan(g=g, mode=mode, tiles=tiles, tile_problem=tile_problem,
                tile_local=tile_local, sk_tiles=sk_tiles, sk_iters=sk_iters,
                sk_units=sk_units, units=units)


def tile_grid(M: int, N: int, BM: int, BN: int):
    return -(-M // BM), -(-N // BN)


def execute_fp64(A, B, plan: Plan, M: int, N: int, K: int, BM: int, BN: int,
                 BK: int, alpha: float = 1.0, beta: float = 0.0, C0=None,
                 tile_coords=None):
    """Run a single-problem schedule in FP64: every segment forms its own
    partial product over its k-blocks, owners add their peers' partials in
    ascending unit order, then C = alpha * acc + beta * C0.

    ``tile_coords(t) -> (tm, tn)`` maps a tile index to tile coordinates
    (row-major over tile columns by default)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    tm_n, tn_n = tile_grid(M, N, BM, BN)
    if tile_coords is None:
        def tile_coords(t):
            return divmod(t, tn_n)
    C = np.full((M, N), np.nan)
    partial = {}

    def seg_product(s):
        tm, tn = tile_coords(s.local_tile)
        r0, c0 = tm * BM, tn * BN
        r1, c1 = min(M, r0 + BM), min(N, c0 + BN)
        ka, kb = s.k0 * BK, min(K, s.k1 * BK)
        return (r0, r1, c0, c1), A[r0:r1, ka:kb] @ B[ka:kb, c0:c1]

    # Peers first (their order does not matter: each writes its own slot).
    for segs in plan.units:
        for s in segs:
            if s.role == "peer":
                partial[s.unit] = seg_product(s)[1]
    for segs in plan.units:
        for s in segs:
            if s.role == "peer":
                continue
            (r0, r1, c0, c1), acc = seg_product(s)
            for p in s.peers:
                acc = acc + partial[p]
            out = alpha * acc
            if beta != 0.0:
                out = out + beta * np.asarray(C0, dtype=np.float64)[r0:r1, c0:c1]
            C[r0:r1, c0:c1] = out
    return C

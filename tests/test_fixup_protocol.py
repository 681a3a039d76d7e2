"""Host model of the two fixup protocols over the library's own schedules.

For every tile split across units, the contributors are consecutive units
o..pl; unit o holds k-block 0 (the owner, whose item lists peers o+1..pl)
and the k-ranges, in unit order, cover the tile's k-blocks once.  The
kernels add the partials in that unit order, whichever protocol runs.

The last-arriver protocol is then checked over every interleaving of the
contributors' steps: a peer spills and counts its arrival (one atomic add);
the owner first reads the counter -- if every peer has arrived it sums at
once -- else spills and counts its own arrival.  Exactly one contributor
must sum the tile, only after every other contributor's partial is
written, and the counter must end at zero.
"""
import itertools

import pytest

ROLE_OWNER, ROLE_PEER = 1, 2


@pytest.fixture(scope="module")
def sk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_00044_gb300 as m
    return m


def split_tiles(sk, probs, cfg, sms):
    info = sk.plan(probs, cfg, num_sms=sms)
    tiles = {}
    for u in range(info.num_ctas):
        for it in sk.unit_items(probs, u, cfg, num_sms=sms):
            tiles.setdefault(it.global_tile, []).append((u, it))
    return info, {t: v for t, v in tiles.items() if len(v) > 1}


CASES = [
    ([(384, 384, 2048)], {"mode": "sk", "tile_m": 128, "tile_n": 128}, 148),
    ([(1536, 1536, 8192)], {"mode": "sk", "tile_m": 128, "tile_n": 256}, 152),
    ([(1536, 1536, 8192)], {"mode": "sk", "tile_m": 256}, 152),
    ([(3840, 4096, 4096)], {"mode": "hybrid2", "tile_m": 256}, 152),
    ([(3840, 4096, 4096)], {"mode": "hybrid1", "tile_m": 128, "tile_n": 256}, 148),
    ([(392, 776, 1544)], {"mode": "sk", "num_ctas": 6, "tile_m": 128, "tile_n": 128}, 148),
    ([(256, 1024, 1024), (300, 512, 2048), (777, 256, 4096)], {"mode": "sk", "tile_m": 128, "tile_n": 128}, 40),
]


@pytest.mark.parametrize("shapes,cfg,sms", CASES)
def test_split_tiles_have_consecutive_contributors(sk, shapes, cfg, sms):
    probs = [sk.shape_problem(*s) for s in shapes]
    info, tiles = split_tiles(sk, probs, cfg, sms)
    assert tiles, "the case must split some tile"
    for t, contrib in tiles.items():
        units = [u for u, _ in contrib]
        assert units == list(range(units[0], units[0] + len(units))), t
        o, first = contrib[0]
        assert first.role == ROLE_OWNER and first.k0 == 0
        assert (first.peer_first, first.peer_last) == (o + 1, units[-1])
        k = 0
        for u, it in contrib:
            assert it.k0 == k and it.k1 > it.k0
            assert it.role == (ROLE_OWNER if u == o else ROLE_PEER)
            k = it.k1
        # together they cover all ceil(K / tile_k) k-blocks of the tile
        assert k == -(-shapes[first.problem][2] // info.tile_k), t


def _interleavings(npeers):
    """All orders of the owner's steps (check, then possibly add) and each
    peer's add, with the owner's check before its add."""
    events = [("peer", p) for p in range(1, npeers + 1)] + [("check", 0), ("add", 0)]
    for perm in itertools.permutations(events):
        if perm.index(("check", 0)) < perm.index(("add", 0)):
            yield perm


def _run_last_arriver(npeers, order):
    counter = 0
    written = set()          # partials visible in the workspace
    reducers = []
    owner_done = False
    for kind, u in order:
        if kind == "check":
            if counter == npeers:          # every peer already arrived: sum from TMEM now
                assert written == set(range(1, npeers + 1))
                reducers.append(0)
                counter = 0
                owner_done = True
        elif kind == "add":
            if owner_done:
                continue
            written.add(0)                 # spill, fence, then count
            old, counter = counter, counter + 1
            if old == npeers:
                assert written == set(range(0, npeers + 1))
                reducers.append(0)
                counter = 0
        else:
            written.add(u)
            old, counter = counter, counter + 1
            if old == npeers:
                assert written == set(range(0, npeers + 1)), "owner partial missing"
                reducers.append(u)
                counter = 0
    return reducers, counter


@pytest.mark.parametrize("npeers", [1, 2, 3, 4])
def test_last_arriver_exactly_one_reducer(npeers):
    n = 0
    for order in _interleavings(npeers):
        reducers, counter = _run_last_arriver(npeers, order)
        assert len(reducers) == 1, order
        assert counter == 0, order
        n += 1
    assert n > 0

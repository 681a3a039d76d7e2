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


# ---- split reduce --------------------------------------------------------
# Every contributor of a split tile spills its partial, counts its arrival in
# the low 16 bits of the tile's counter and waits until all kc contributors
# have arrived.  Then each of its W epilogue warps stages the partials of its
# share of the tile's columns (reads the other contributors' slots), counts
# its own departure in the high bits -- before it sums, so the atomic's round
# trip overlaps the sum -- and sums from the staged copies.  The last of the
# kc * W departures resets the counter.  A warp with an empty share departs
# right after the wait; a contributor with an empty share arrives and departs
# (all W warps) in one atomic add.  Checked here over every interleaving of
# the steps of the contributors and of their warps.

DEPART = 1 << 16


def _split_share(j, kc, nu):
    return j * nu // kc, (j + 1) * nu // kc


@pytest.mark.parametrize("nu", [2, 4, 8, 16])
@pytest.mark.parametrize("kc", [2, 3, 4, 5, 7, 16, 33])
def test_split_shares_partition_the_tile(nu, kc):
    cols = []
    for j in range(kc):
        u0, u1 = _split_share(j, kc, nu)
        assert u0 <= u1
        cols.extend(range(u0, u1))
    assert cols == list(range(nu))


def _split_explore(kc, empty, warps=2, idle=()):
    """Search over all interleavings.  Processes: each contributor's head
    (spill, arrive, wait; or one arrive-and-depart if its share is empty)
    and, once the head has waited, each of its warps (stage, depart; or only
    depart for the (contributor, warp) pairs in `idle`).  Returns the number
    of distinct terminal states."""
    procs = []
    for j in range(kc):
        if j in empty:
            procs.append((j, None, ["spill", "arrive_depart"]))
        else:
            procs.append((j, None, ["spill", "arrive", "wait"]))
            for w in range(warps):
                procs.append((j, w, ["depart"] if (j, w) in idle else ["stage", "depart"]))
    head = {j: i for i, (j, w, _) in enumerate(procs) if w is None}
    last = kc * warps - 1
    terminals = set()
    seen = set()

    def go(pc, counter, written, staged):
        key = (pc, counter, written, staged)
        if key in seen:
            return
        seen.add(key)
        moved = False
        for i, (j, w, steps) in enumerate(procs):
            if pc[i] == len(steps):
                continue
            if w is not None and pc[head[j]] < 3:
                continue                     # the warps start after their CTA's wait
            s = steps[pc[i]]
            c2, w2, s2 = counter, written, staged
            if s == "spill":
                w2 = written | {j}
            elif s == "arrive":
                c2 = counter + 1
            elif s == "arrive_depart":
                c2 = counter + 1 + warps * DEPART
                if (counter >> 16) == last - (warps - 1):
                    c2 = 0
            elif s == "wait":
                if (counter & 0xFFFF) < kc:
                    continue                 # blocked: no move
            elif s == "stage":
                # every partial the warp reads must be written
                assert written == set(range(kc))
                s2 = staged | {(j, w)}
            elif s == "depart":
                c2 = counter + DEPART
                if (counter >> 16) == last:
                    # nobody reads a slot of the tile any more
                    need = {(jj, ww) for jj in range(kc) if jj not in empty
                            for ww in range(warps) if (jj, ww) not in idle}
                    assert staged == need
                    c2 = 0
            moved = True
            go(pc[:i] + (pc[i] + 1,) + pc[i + 1:], c2, w2, s2)
        if not moved:
            # no process can move: all must be finished (no deadlock)
            assert all(pc[i] == len(steps) for i, (_, _, steps) in enumerate(procs)), (pc, counter)
            assert counter == 0
            terminals.add(key)

    go(tuple([0] * len(procs)), 0, frozenset(), frozenset())
    return len(terminals)


@pytest.mark.parametrize("kc,empty,idle", [(2, (), ()), (3, (), ()), (3, (1,), ()), (4, (0, 2), ()),
                                           (3, (0, 1), ()), (2, (), ((1, 0),)), (3, (2,), ((0, 1),))])
def test_split_reduce_every_interleaving(kc, empty, idle):
    assert _split_explore(kc, empty, idle=idle) > 0


@pytest.mark.parametrize("bn,f32_out", [(128, True), (128, False), (256, True), (256, False)])
@pytest.mark.parametrize("kc", [2, 3, 4, 5, 8, 9, 16, 17, 32, 64])
def test_split_units_cover_the_tile_once(bn, f32_out, kc):
    """The tensor-core split reduce deals (column group x warp) units to the
    contributors: unit s is chunk group s // 4 of warp s % 4, contributor j
    takes [j*NS/kc, (j+1)*NS/kc).  Every (chunk, warp) block of the tile is
    summed by exactly one warp of one contributor, and a warp's units are
    what that warp keeps in TMEM (not spilled)."""
    uw = 1 if f32_out else 2                 # chunks per unit: 32 or 64 columns
    nch = bn // 32
    ns = 4 * nch // uw
    owner = {}
    for j in range(kc):
        s0, s1 = j * ns // kc, (j + 1) * ns // kc
        for q4 in range(4):
            s_first = s0 + ((q4 - s0 % 4) + 4) % 4
            n_w = (s1 - 1 - s_first) // 4 + 1 if s_first < s1 else 0
            # the warp's chunks, in the order the kernel walks them
            chunks = [((s_first + 4 * (k // uw)) // 4) * uw + k % uw for k in range(n_w * uw)]
            kept = [ch for ch in range(nch) if s0 <= (ch // uw) * 4 + q4 < s1]
            assert sorted(chunks) == kept
            for ch in chunks:
                assert (ch, q4) not in owner
                owner[(ch, q4)] = j
    assert set(owner) == {(ch, q4) for ch in range(nch) for q4 in range(4)}
    # BF16 output: a warp always holds both chunks of a 64-column TMA box
    if not f32_out:
        for (ch, q4), j in owner.items():
            assert owner[(ch ^ 1, q4)] == j


# ---- cluster split ----------------------------------------------------------
# The kc contributors of a tile form one cluster.  Each, once its MMAs are
# done (its operand ring is free), arms one data barrier per unit it sums
# (expecting kc - 1 blocks) and arrives on every partner's ring-free
# barrier; after all kc - 1 partners have arrived it sends each unit that
# another contributor sums as one block into that contributor's ring
# (counted on the receiver's barrier of that unit); it sums a unit of its
# own once that unit's barrier has seen kc - 1 blocks.  Checked over every
# interleaving: a block lands only in a ring that is free, every sum reads
# kc - 1 landed blocks, and every contributor finishes (no deadlock).

def _xs_layout(ns, kc):
    """Units each contributor sums (the split reduce's dealing)."""
    return [list(range(j * ns // kc, (j + 1) * ns // kc)) for j in range(kc)]


def _xs_explore(kc, ns):
    owned = _xs_layout(ns, kc)
    owner_of = {s: j for j in range(kc) for s in owned[j]}
    # per contributor: armed, ring-free arrivals received, blocks received
    # per own unit, sends done, sums done
    seen, terminals = set(), set()

    def steps(j):
        out = [("free", None)]
        out += [("send", s) for s in range(ns) if owner_of[s] != j]
        out += [("sum", s) for s in owned[j]]
        return out

    progs = [steps(j) for j in range(kc)]

    def go(pc, free, arrivals, landed):
        key = (pc, free, arrivals, landed)
        if key in seen:
            return
        seen.add(key)
        moved = False
        for j in range(kc):
            if pc[j] == len(progs[j]):
                continue
            op, s = progs[j][pc[j]]
            fr, ar, la = set(free), list(arrivals), dict(landed)
            if op == "free":
                fr.add(j)                    # MMAs done: ring free, barriers armed
                for i in range(kc):
                    if i != j:
                        ar[i] += 1           # remote arrival on i's ring-free barrier
            elif op == "send":
                if ar[j] < kc - 1:
                    continue                 # blocked until every partner's ring is free
                dst = owner_of[s]
                assert dst in fr, "a block written into a busy ring"
                la[s] = la.get(s, 0) + 1
            elif op == "sum":
                if la.get(s, 0) < kc - 1:
                    continue                 # blocked on the unit's barrier
                assert la[s] == kc - 1
            moved = True
            go(pc[:j] + (pc[j] + 1,) + pc[j + 1:], frozenset(fr), tuple(ar), tuple(sorted(la.items())))
        if not moved:
            assert all(pc[j] == len(progs[j]) for j in range(kc)), "deadlock"
            terminals.add(key)

    go(tuple([0] * kc), frozenset(), tuple([0] * kc), ())
    return len(terminals)


@pytest.mark.parametrize("kc,ns", [(2, 4), (2, 8), (4, 4), (4, 8), (3, 5)])
def test_cluster_split_every_interleaving(kc, ns):
    assert _xs_explore(kc, ns) > 0


@pytest.mark.parametrize("bn,f32_out", [(128, True), (128, False), (256, True), (256, False)])
@pytest.mark.parametrize("kc", [2, 4, 8])
def test_cluster_split_blocks_fit(bn, f32_out, kc):
    """Ring layout of the cluster split: each contributor's incoming slots
    (source, own unit) and the senders' destination offsets are a bijection
    onto [0, (kc - 1) x own units) blocks, and every contributor's outgoing
    staging indexes the other contributors' units once."""
    uw = 1 if f32_out else 2
    ns = 4 * (bn // 32) // uw
    if ns < kc:
        return
    lo = [j * ns // kc for j in range(kc + 1)]
    for j in range(kc):                      # receiver
        own_n = lo[j + 1] - lo[j]
        slots = set()
        for i in range(kc):                  # sender
            if i == j:
                continue
            src_slot = i if i < j else i - 1
            for s in range(lo[j], lo[j + 1]):
                slots.add(src_slot * own_n + (s - lo[j]))
        assert slots == set(range((kc - 1) * own_n))
        stg = [s - (own_n if s >= lo[j + 1] else 0) for s in range(ns) if not lo[j] <= s < lo[j + 1]]
        assert sorted(stg) == list(range(ns - own_n))

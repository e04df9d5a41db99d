"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test names the passage or the mathematical fact it checks.  None of these
needs a GPU.
"""
import os
import random

import numpy as np
import pytest

from oracle import bruteforce as B
from oracle import oracle as O
from triton_philox import triton_philox as _triton_philox

N_, E_, S_, W_ = 0, 1, 2, 3


# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11) against an independent implementation
# ---------------------------------------------------------------------------
def test_philox_matches_independent_implementation():
    rng = random.Random(11)
    for key in ([0, 0], [3, 0], [0xFFFFFFFF, 0xFFFFFFFF], [rng.getrandbits(32), rng.getrandbits(32)]):
        ctrs = [[0, 0, 0, 0], [0xFFFFFFFF] * 4] + [[rng.getrandbits(32) for _ in range(4)] for _ in range(14)]
        want = _triton_philox(ctrs, key)
        got = [O.philox(c, key) for c in ctrs]
        assert got == want


def test_sampled_genotypes_rederived_from_triton_philox():
    """The sampled workload of S_{3,8} (and of other spaces): genotype i is
    words 0 and 1 of Philox4x32-10(ctr = (0, 1 << 24, i_lo, i_hi), key = seed)
    as (w1 << 32 | w0), masked to the 4 n log2(c) genome bits -- re-derived
    here from Triton's Philox, on indices below and above 2^32."""
    rng = random.Random(5)
    idx = [0, 1, 2, (1 << 28) - 1, 1 << 32, (1 << 40) + 3] + [rng.getrandbits(36) for _ in range(20)]
    for (n, c, seed) in ((3, 8, 3), (2, 8, 2), (4, 8, 0xDEADBEEF12345678), (2, 4, 1)):
        bits = 4 * n * (c.bit_length() - 1)
        words = _triton_philox([[0, 1 << 24, i & 0xFFFFFFFF, i >> 32] for i in idx],
                               [seed & 0xFFFFFFFF, seed >> 32])
        for i, w in zip(idx, words):
            want = ((w[1] << 32) | w[0]) & ((1 << bits) - 1)
            assert O.sample_genotype(i, n, c, seed) == want, (n, c, seed, i)
        assert O.sample_genotypes(idx[0], 3, n, c, seed).tolist() == [O.sample_genotype(i, n, c, seed)
                                                                     for i in range(3)]


# ---------------------------------------------------------------------------
# Jenkins one-at-a-time hash (appendix "One-at-a-time Hash"; Jenkins 1997)
# ---------------------------------------------------------------------------
def test_oaat_published_values():
    # reference values published with Jenkins' one-at-a-time function
    assert O.oaat(b"a") == 0xCA2E9442
    assert O.oaat(b"The quick brown fox jumps over the lazy dog") == 0x519E91F5
    # no bytes: every step of the final avalanche maps 0 to 0
    assert O.oaat(b"") == 0


def test_collision_bound_of_32bit_hash():
    """Section 2.5: for 1000 phenotypes the probability of any collision of a
    32-bit hash is about 0.01 %."""
    p_none = 1.0
    for i in range(1001):
        p_none *= 1.0 - i * 2.0 ** -32
    assert abs((1.0 - p_none) - 1.0e-4) < 0.2e-4


# ---------------------------------------------------------------------------
# interaction matrix, encoding, rotation (Section 1.1; appendices)
# ---------------------------------------------------------------------------
def test_bind_is_adjacent_pairs():
    """Labels bind in pairs 1-2, 3-4, ...; 0 is inert; other pairs are neutral."""
    pairs = {(1, 2), (2, 1), (3, 4), (4, 3), (5, 6), (6, 5)}
    for a in range(8):
        for b in range(8):
            assert O.bind(a, b) == ((a, b) in pairs), (a, b)
    # with eight labels the literal matrix leaves 7 without a partner in 0..7
    assert not any(O.bind(7, b) for b in range(8))
    assert not any(O.bind(0, b) for b in range(8))


def test_decode_is_seed_first_nesw_msb_first():
    """Appendix "Encoding genome information": tiles in order from the seed,
    colours N, E, S, W, log2(c) bits each."""
    # S_{2,8}: 24 bits; the top 3 bits are the seed's north edge
    assert list(O.decode(0b111 << 21, 2, 8)[:8]) == [7, 0, 0, 0, 0, 0, 0, 0]
    assert list(O.decode(0b101, 2, 8)[:8]) == [0, 0, 0, 0, 0, 0, 0, 5]
    assert list(O.decode(0b001 << 12, 2, 8)[:8]) == [0, 0, 0, 1, 0, 0, 0, 0]
    # S_{2,4}: 16 bits, 2 per colour
    assert list(O.decode(0x1B1B, 2, 4)[:8]) == [0, 1, 2, 3, 0, 1, 2, 3]
    # S_{3,8} is 4096 times larger than S_{2,8} (Section 3.3): 36 vs 24 bits
    assert O.decode((1 << 36) - 1, 3, 8).tolist()[:12] == [7] * 12
    with pytest.raises(ValueError):
        O.decode(0, 2, 6)


def _grid_cells(r):
    g = r["grid"]
    return {(x, y): int(g[y, x]) for y in range(g.shape[0]) for x in range(g.shape[1]) if g[y, x] >= 0}


def test_rotation_is_clockwise_without_flips():
    """Tile (2,0,0,0) attaches east of a seed whose east edge is 1 only after
    three clockwise quarter turns (its north edge ends up facing west)."""
    L = 9
    col = [0, 1, 0, 0, 2, 0, 0, 0]
    r = O.classify(2, 4, L, 4, 1, col, 0, want_grid=True)
    assert (r["cls"], r["size"]) == (O.DET_BOUNDED, 2)
    cells = _grid_cells(r)
    assert cells == {(4, 4): 0, (5, 4): 4 * 1 + 3}
    # north of the seed: two quarter turns put the 2 on the south side
    r = O.classify(2, 4, L, 4, 1, [1, 0, 0, 0, 2, 0, 0, 0], 0, want_grid=True)
    assert _grid_cells(r) == {(4, 4): 0, (4, 3): 4 * 1 + 2}


def test_hand_built_tile_sets():
    L, k = 9, 8
    # every edge inert: the seed alone
    r = O.classify(2, 8, L, k, 5, [0, 7, 0, 7, 7, 0, 0, 0], 0)
    assert (r["cls"], r["size"], r["decided_rep"]) == (O.DET_BOUNDED, 1, k)
    # the seed binds itself north-south: an infinite column, unbounded in any grid
    for L2 in (3, 8, 16, 32):
        r = O.classify(1, 4, L2, k, 5, [1, 0, 2, 0], 0)
        assert (r["cls"], r["decided_rep"]) == (O.UNBOUNDED, 0)
    # two different tiles fit north of the seed: trivial non-determinism at once
    r = O.classify(3, 4, L, k, 5, [1, 0, 0, 0, 2, 0, 0, 0, 2, 3, 0, 0], 0)
    assert (r["cls"], r["decided_rep"], r["placements"]) == (O.ND_LOCAL, 0, 0)
    # a repeated tile type is not non-determinism (Section 2.4)
    r = O.classify(3, 4, L, k, 5, [1, 0, 0, 0, 2, 0, 0, 0, 2, 0, 0, 0], 0)
    assert (r["cls"], r["size"]) == (O.DET_BOUNDED, 2)
    # a tile with two equal rotations is not non-determinism either; the
    # inexhaustible seed type caps the column: seed, (2,0,2,0), seed turned twice
    r = O.classify(2, 4, L, k, 5, [1, 0, 0, 0, 2, 0, 2, 0], 0, want_grid=True)
    assert (r["cls"], r["size"]) == (O.DET_BOUNDED, 3)
    assert _grid_cells(r) == {(4, 4): 0, (4, 3): 4, (4, 2): 2}


def _monomer_closed_form(col, n, c):
    """The seed stays alone iff no edge of any tile (any rotation) can bond to
    any edge of the seed in its fixed orientation."""
    present = set(int(v) for v in col[: 4 * n])
    for a in col[:4]:
        a = int(a)
        partner = a + 1 if a % 2 == 1 else a - 1
        if a != 0 and 0 <= partner < c and partner in present:
            return False
    return True


def test_monomer_count_closed_form_full_s24():
    """All 4^8 genotypes of S_{2,4}: the number classified as the bounded
    deterministic monomer equals the closed-form count."""
    n, c, L, k = 2, 4, 16, 10
    res, _ = O.enumerate_space(n, c, L, k, 1, 0, 4 ** 8)
    mono = (res["cls"] == O.DET_BOUNDED) & (res["size"] == 1)
    want = np.array([_monomer_closed_form(O.decode(g, n, c), n, c) for g in range(4 ** 8)])
    assert np.array_equal(mono, want)
    assert int(want.sum()) > 0


# ---------------------------------------------------------------------------
# canonical form: free polyominoes (textbook counts)
# ---------------------------------------------------------------------------
def _fixed_polyominoes(max_size):
    shapes = {1: {frozenset({(0, 0)})}}
    for m in range(2, max_size + 1):
        nxt = set()
        for s in shapes[m - 1]:
            for (x, y) in s:
                for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    q = (x + dx, y + dy)
                    if q in s:
                        continue
                    t = s | {q}
                    mx = min(p[0] for p in t)
                    my = min(p[1] for p in t)
                    nxt.add(frozenset((p[0] - mx, p[1] - my) for p in t))
        shapes[m] = nxt
    return shapes


def test_canonical_form_counts_free_polyominoes():
    """Fixed polyominoes of size 1..7 number 1, 2, 6, 19, 63, 216, 760 and free
    ones (up to the 8 symmetries of the square) 1, 1, 2, 5, 12, 35, 108."""
    fixed = _fixed_polyominoes(7)
    assert [len(fixed[m]) for m in range(1, 8)] == [1, 2, 6, 19, 63, 216, 760]
    all_hashes = {}
    for m in range(1, 8):
        canon = set()
        for s in fixed[m]:
            bm = O.canonical(sorted(s))
            canon.add((bm.shape, bm.tobytes()))
        assert len(canon) == [1, 1, 2, 5, 12, 35, 108][m - 1]
        for shp, raw in canon:
            h = O.shape_hash(np.frombuffer(raw, np.uint8).reshape(shp))
            assert h not in all_hashes, "hash collision among small free polyominoes"
            all_hashes[h] = (shp, raw)


def test_canonical_form_invariant_and_minimal():
    rng = random.Random(3)
    fixed = sorted(_fixed_polyominoes(6)[6], key=sorted)
    maps = [lambda x, y: (x, y), lambda x, y: (-y, x), lambda x, y: (-x, -y), lambda x, y: (y, -x),
            lambda x, y: (-x, y), lambda x, y: (x, -y), lambda x, y: (y, x), lambda x, y: (-y, -x)]
    for s in rng.sample(fixed, 40):
        base = O.canonical(sorted(s))
        images = []
        for f in maps:
            img = O.canonical([f(x, y) for (x, y) in s])
            assert img.shape == base.shape and np.array_equal(img, base)
            pts = [f(x, y) for (x, y) in s]
            mx = min(p[0] for p in pts)
            my = min(p[1] for p in pts)
            h = max(p[1] for p in pts) - my + 1
            w = max(p[0] for p in pts) - mx + 1
            a = np.zeros((h, w), np.uint8)
            for (x, y) in pts:
                a[y - my, x - mx] = 1
            images.append((h, w, a.tobytes()))
        assert (base.shape[0], base.shape[1], base.tobytes()) == min(images)


def test_shape_hash_bytes_are_dims_then_x_y_row_major():
    # monomer: bytes h=1, w=1, then cell (0, 0)
    assert O.shape_hash(O.canonical([(5, 5)])) == O.oaat(bytes([1, 1, 0, 0]))
    # domino: canonical is the 1 x 2 image; cells (0,0), (1,0)
    bm = O.canonical([(0, 0), (0, 1)])
    assert bm.shape == (1, 2)
    assert O.shape_hash(bm) == O.oaat(bytes([1, 2, 0, 0, 1, 0]))
    # L-tromino: the smallest 2 x 2 image in row-major order is 01 / 11
    bm = O.canonical([(0, 0), (1, 0), (0, 1)])
    assert bm.tolist() == [[0, 1], [1, 1]]
    assert O.shape_hash(bm) == O.oaat(bytes([2, 2, 1, 0, 0, 1, 1, 1]))
    # a zero byte does not move the one-at-a-time state away from 0, which is
    # why the dimensions come first: without them the square and the
    # L-tromino would share a hash
    assert O.oaat(bytes([0, 0, 1, 0, 0, 1, 1, 1])) == O.oaat(bytes([1, 0, 0, 1, 1, 1]))
    sq = O.canonical([(0, 0), (1, 0), (0, 1), (1, 1)])
    assert O.shape_hash(sq) != O.shape_hash(bm)


# ---------------------------------------------------------------------------
# brute force over all assembly paths on tiny grids
# ---------------------------------------------------------------------------
def _oracle_config(r, col):
    cfg = set()
    g = r["grid"]
    for y in range(g.shape[0]):
        for x in range(g.shape[1]):
            u = int(g[y, x])
            if u >= 0:
                t, rot = divmod(u, 4)
                cfg.add(((x, y), B.rotated(tuple(int(v) for v in col[4 * t: 4 * t + 4]), rot)))
    return frozenset(cfg)


@pytest.mark.parametrize("n,c,L", [(2, 4, 5), (1, 8, 5), (2, 8, 4)])
def test_oracle_consistent_with_all_paths(n, c, L):
    """Local non-determinism, unboundedness and steric non-determinism found by
    the sampled paths must exist among all paths; a tile set whose every path
    ends in one bounded configuration must be classified deterministic with it
    for every seed (definitions in the appendix "Modifications to Winfree's
    aTAM")."""
    rng = random.Random(100 * n + c)
    k = 6
    bits = 4 * n * (c.bit_length() - 1)
    checked = det = 0
    seen_cls = set()
    while checked < 120:
        g = rng.getrandbits(bits)
        col = O.decode(g, n, c)
        truth = B.explore(col, n, L, max_states=400)
        if not truth.complete:
            continue
        checked += 1
        for seed in (1, 7):
            r = O.classify(n, c, L, k, seed, col, g, want_grid=True)
            cfg = _oracle_config(r, col)
            seen_cls.add(r["cls"])
            if r["cls"] == O.ND_LOCAL:
                assert truth.trivial_nd
            if r["cls"] == O.UNBOUNDED:
                assert truth.escape
            if r["cls"] == O.ND_STERIC:
                assert len(truth.terminals) >= 2
            if r["cls"] in (O.DET_BOUNDED, O.ND_STERIC):
                assert cfg in truth.terminals
                assert r["size"] == len(cfg)
            if truth.deterministic_bounded:
                det += 1
                assert r["cls"] == O.DET_BOUNDED and cfg in truth.terminals
            if not truth.trivial_nd and not truth.escape:
                assert r["cls"] in (O.DET_BOUNDED, O.ND_STERIC)
    assert det > 0 and len(seen_cls) >= 2


def test_steric_nondeterminism_found_against_all_paths():
    """Tile sets of S_{3,8} whose assembly paths end in several different
    bounded configurations: whenever the oracle reports steric
    non-determinism, replicate 0's configuration is one of the terminal
    configurations of the exhaustive search, and it does so for some seed."""
    n, c, L, k = 3, 8, 5, 20
    # genotypes with several terminal configurations on a 5 x 5 grid
    for g in (39322585744, 43408325656, 43573769726, 6387920665, 20890713338):
        col = O.decode(g, n, c)
        truth = B.explore(col, n, L, max_states=2000)
        assert truth.complete and not truth.escape and len(truth.terminals) >= 2
        classes = set()
        for seed in range(1, 13):
            r = O.classify(n, c, L, k, seed, col, g, want_grid=True)
            classes.add(r["cls"])
            assert r["cls"] in (O.DET_BOUNDED, O.ND_LOCAL, O.ND_STERIC)
            if r["cls"] in (O.DET_BOUNDED, O.ND_STERIC):
                assert _oracle_config(r, col) in truth.terminals
        assert O.ND_STERIC in classes


# ---------------------------------------------------------------------------
# exact invariances and monotonicity of the replicate rule
# ---------------------------------------------------------------------------
def _key(r):
    return (r["cls"], r["decided_rep"], r["size"], r["shape_hash"], r["placements"])


def test_invariance_under_label_automorphisms_and_tile_moves():
    """The process depends on colours only through M and tuple equality:
    relabelling by a permutation that preserves M, turning a non-seed tile's
    edges, or reordering the non-seed tiles changes nothing (same stream id)."""
    rng = random.Random(9)
    n, c, L, k = 3, 8, 12, 6
    autos = [
        {0: 0, 1: 2, 2: 1, 3: 3, 4: 4, 5: 5, 6: 6, 7: 7},   # swap inside one pair
        {0: 7, 7: 0, 1: 3, 2: 4, 3: 5, 4: 6, 5: 1, 6: 2},   # permute pairs, swap inert labels
        {0: 0, 7: 7, 1: 6, 2: 5, 3: 4, 4: 3, 5: 2, 6: 1},   # reverse the pairs
    ]
    done = 0
    while done < 150:
        g = rng.getrandbits(36)
        col = [int(v) for v in O.decode(g, n, c)[:12]]
        base = _key(O.classify(n, c, L, k, 4, col, 77))
        for a in autos:
            assert _key(O.classify(n, c, L, k, 4, [a[v] for v in col], 77)) == base
        t1 = col[4:8]
        turned = col[:4] + [t1[3], t1[0], t1[1], t1[2]] + col[8:]
        assert _key(O.classify(n, c, L, k, 4, turned, 77)) == base
        swapped = col[:4] + col[8:12] + col[4:8]
        assert _key(O.classify(n, c, L, k, 4, swapped, 77)) == base
        done += 1


def test_replicate_rule_is_monotone_in_k():
    """Replicate streams are keyed by the replicate index, so a class decided
    at replicate j < k is the same for every larger k, and the deterministic
    genotypes at k + 1 are a subset of those at k."""
    n, c, L = 2, 8, 10
    res = {k: O.enumerate_space(n, c, L, k, 2, 1 << 20, 3000)[0] for k in (1, 2, 5, 6, 12)}
    for k1, k2 in ((1, 2), (5, 6), (6, 12), (1, 12)):
        a, b = res[k1], res[k2]
        decided = a["decided_rep"] < k1
        assert np.array_equal(a[decided], b[decided])
        assert np.all(~(b["cls"] == O.DET_BOUNDED) | (a["cls"] == O.DET_BOUNDED))


# ---------------------------------------------------------------------------
# the draw order, re-derived step by step
# ---------------------------------------------------------------------------
def _frontier(occ, tuples, L):
    """Row-major list of in-grid empty sites with exactly one attachable
    rotated tuple, and that tuple."""
    out = []
    for y in range(L):
        for x in range(L):
            if (x, y) in occ:
                continue
            fits = set()
            for tup in tuples:
                for d, (dx, dy) in enumerate(((0, -1), (1, 0), (0, 1), (-1, 0))):
                    nb = occ.get((x + dx, y + dy))
                    if nb is not None and B.pair_bind(tup[d], nb[(d + 2) % 4]):
                        fits.add(tup)
                        break
            if len(fits) == 1:
                out.append(((x, y), fits.pop()))
    return out


def test_draw_order_rederived():
    """Every step: u is word (s mod 4) of Philox(ctr=(s>>2, rep, id_lo, id_hi),
    key=seed), the rank is floor(u |F| / 2^32) and F is in row-major order."""
    rng = random.Random(21)
    n, c, L, k, seed = 2, 8, 12, 4, 0x1234_0000_0042
    checked = 0
    while checked < 6:
        g = rng.getrandbits(24)
        col = O.decode(g, n, c)
        rep = rng.randrange(k)
        r = O.classify(n, c, L, k, seed, col, g, trace_rep=rep)
        tr = r["trace"]
        if len(tr) < 5 or r["decided_rep"] < rep:
            continue
        tiles = [tuple(int(v) for v in col[4 * t: 4 * t + 4]) for t in range(n)]
        tuples = sorted({B.rotated(t, q) for t in tiles for q in range(4)})
        occ = {(L // 2, L // 2): tiles[0]}
        ctrs = sorted({s >> 2 for s in range(len(tr))})
        words = dict(zip(ctrs, _triton_philox([[cc, rep, g & 0xFFFFFFFF, g >> 32] for cc in ctrs],
                                              [seed & 0xFFFFFFFF, seed >> 32])))
        for s, (nf, u, idx, x, y, tup) in enumerate(tr):
            assert u == words[s >> 2][s & 3]
            F = _frontier(occ, tuples, L)
            assert nf == len(F)
            assert idx == (u * nf) >> 32
            (fx, fy), ftup = F[idx]
            assert (fx, fy) == (x, y)
            t, q = divmod(tup, 4)
            assert B.rotated(tiles[t], q) == ftup
            occ[(x, y)] = ftup
        checked += 1


def test_edge_sizes():
    # L = 1: every neighbour of the seed lies outside the grid
    r = O.classify(1, 4, 1, 3, 1, [1, 0, 2, 0], 0)
    assert r["cls"] == O.UNBOUNDED and r["decided_rep"] == 0
    r = O.classify(1, 4, 1, 3, 1, [1, 0, 0, 0], 0)
    assert (r["cls"], r["size"]) == (O.DET_BOUNDED, 1)
    r = O.classify(1, 4, 1, 3, 1, [0, 0, 3, 0], 0)
    assert (r["cls"], r["size"]) == (O.DET_BOUNDED, 1)
    # n = 4 uses all sixteen tuple ids
    col = [1, 3, 5, 0, 2, 4, 6, 0, 2, 2, 2, 2, 0, 0, 0, 0]
    r = O.classify(4, 8, 32, 2, 1, col, 0)
    assert r["cls"] in (O.DET_BOUNDED, O.ND_LOCAL, O.ND_STERIC, O.UNBOUNDED)
    with pytest.raises(ValueError):
        O.classify(5, 8, 16, 1, 1, [0] * 16, 0)
    with pytest.raises(ValueError):
        O.classify(2, 8, 33, 1, 1, [0] * 8, 0)
    with pytest.raises(ValueError):
        O.classify(2, 4, 16, 1, 1, [0, 0, 0, 4, 0, 0, 0, 0], 0)


def test_c4_hash_counts_one_sided_polyominoes():
    """The rotation-only variant of Section 2.5 identifies the four rotations of
    a shape but not its mirror image: over the fixed polyominoes of size 1..7
    it takes 1, 1, 2, 7, 18, 60, 196 values (one-sided polyominoes)."""
    fixed = _fixed_polyominoes(7)
    for m in range(1, 8):
        hashes = {O.c4_hash(sorted(s)) for s in fixed[m]}
        assert len(hashes) == [1, 1, 2, 7, 18, 60, 196][m - 1]
    s_tet = [(1, 0), (2, 0), (0, 1), (1, 1)]
    z_tet = [(0, 0), (1, 0), (1, 1), (2, 1)]
    assert O.c4_hash(s_tet) != O.c4_hash(z_tet)
    assert O.c4_hash(s_tet) == O.c4_hash([(-y, x) for (x, y) in s_tet])


def test_c4_hash_mode_changes_only_the_hash():
    n, c, L, k, seed = 2, 8, 12, 6, 2
    first, count = 5 << 20, 3000
    d4, _ = O.enumerate_space(n, c, L, k, seed, first, count)
    with O.hash_mode(True):
        c4, _ = O.enumerate_space(n, c, L, k, seed, first, count)
    for f in ("cls", "decided_rep", "size"):
        assert np.array_equal(d4[f], c4[f])
    shaped = (d4["cls"] == O.DET_BOUNDED) | (d4["cls"] == O.ND_STERIC)
    assert shaped.any() and not np.array_equal(d4["shape_hash"][shaped], c4["shape_hash"][shaped])
    assert not c4["shape_hash"][~shaped].any()


# ---------------------------------------------------------------------------
# exact side table of the shape hash (Section 2.5)
# ---------------------------------------------------------------------------
def test_shape_table_counts_a_planted_collision():
    """The side table's collision rule on planted forms: the same hash for the
    2 x 2 square and the L-tromino is one collision; the same form again is
    none; a different hash is none."""
    square = np.ones((2, 2), np.uint8)
    ltro = np.array([[1, 1], [1, 0]], np.uint8)
    with O.shape_table() as T:
        T.add(5, square)
        T.add(5, square)
        T.add(6, ltro)
        T.add(5, ltro)
    assert T.collisions == 1 and T.overflow == 0
    assert set(T.forms) == {5, 6}
    assert np.array_equal(T.forms[5], square) and np.array_equal(T.forms[6], ltro)


def test_shape_table_of_s24_holds_canonical_forms_of_every_shaped_key():
    """All of S_{2,4}: the table holds exactly the hashes of the histogram's
    shaped keys, each stored form is its own canonical form (invariant under
    the 8 symmetries: canonical(cells) gives it back) and re-hashes to its key,
    and no two forms collide; each key's form is the canonical form of its
    smallest genotype's replicate-0 shape."""
    n, c, L, k, seed = 2, 4, 16, 10, 1
    with O.shape_table() as T:
        res, _ = O.enumerate_space(n, c, L, k, seed, 0, 1 << 16)
    assert T.collisions == 0 and T.overflow == 0
    h = O.histogram(res)
    shaped = h[(h["cls"] == 0) | (h["cls"] == 2)]
    assert sorted(T.forms) == sorted(set(int(v) for v in shaped["shape_hash"]))
    for key, bm in T.forms.items():
        cells = [(x, y) for y in range(bm.shape[0]) for x in range(bm.shape[1]) if bm[y, x]]
        assert np.array_equal(O.canonical(cells), bm)
        assert O.shape_hash(bm) == key
    for row in shaped:
        g = int(row["min_id"])
        r = O.classify(n, c, L, k, seed, O.decode(g, n, c), g, want_grid=True)
        cells = [(x, y) for y in range(L) for x in range(L) if r["grid"][y, x] >= 0]
        assert np.array_equal(O.canonical(cells), T.forms[int(row["shape_hash"])])


def test_ambiguity_kind_diagnostic_hand_cases():
    """The diagnostic split of local ambiguity (Section 2.4 detects trivial and
    first-order steric non-determinism with one check):
      * seed (1, 0, 0, 0) and tile (0, 0, 2, 2): the seed's north side alone
        offers two distinct rotated tuples (0,0,2,2) and (0,2,2,0) -- trivial,
        kind 1, at the seed step;
      * seed (0, 1, 3, 0) and tile (4, 5, 6, 2): the seed's east and south
        sides each take exactly one tuple of the tile, and the two arms offer
        the diagonal cell different tuples, (5,6,2,4) from the north and
        (2,4,5,6) from the west, while no single neighbour ever offers two --
        first-order steric, kind 2.
    The mode changes no class, replicate, hash or non-ND size."""
    with O.nd_detail():
        r = O.classify(2, 8, 9, 20, 1, [1, 0, 0, 0, 0, 0, 2, 2], 0)
        assert (r["cls"], r["decided_rep"], r["size"]) == (O.ND_LOCAL, 0, 1)
        for seed in range(6):
            r = O.classify(2, 8, 15, 20, seed, [0, 1, 3, 0, 4, 5, 6, 2], seed)
            assert (r["cls"], r["size"]) == (O.ND_LOCAL, 2), seed
    a, _ = O.enumerate_space(2, 8, 19, 8, 2, 1 << 22, 1 << 16)
    with O.nd_detail():
        b, _ = O.enumerate_space(2, 8, 19, 8, 2, 1 << 22, 1 << 16)
    same = ["cls", "decided_rep", "shape_hash"]
    assert all(np.array_equal(a[f], b[f]) for f in same)
    nd = b["cls"] == O.ND_LOCAL
    assert np.array_equal(a["size"][~nd], b["size"][~nd])
    assert set(np.unique(b["size"][nd]).tolist()) <= {1, 2}


def test_paper_facts_file_is_consistent():
    """The stored S_{2,8} counts at the paper's settings add up: the classes
    cover 8^8 genotypes and the two kinds of local ambiguity cover ND_LOCAL."""
    import json
    facts = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "s28_paper_facts.json")))
    cc = facts["class_counts"]
    assert sum(cc.values()) == 8 ** 8
    kinds = facts["nd_local_kinds"]
    assert kinds["trivial"] + kinds["first_order_steric"] == cc["nd_local"]
    r = facts["steric_to_unbounded"]
    assert abs(r["with_first_order"] - (cc["nd_steric"] + kinds["first_order_steric"]) / cc["unbounded"]) < 1e-4

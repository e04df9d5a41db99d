"""Pins of the oracle's movelist process (Section 2.4: a last-in-first-out
stack of frontier sites, new sites pushed in a drawn order, the top one
placed).  No GPU needed."""
import math
import random

import numpy as np
import pytest

from oracle import bruteforce as B
from oracle import oracle as O

from test_oracle_pins import _oracle_config, _triton_philox


def test_lifo_permutation_is_a_bijection():
    for m in range(5):
        orders = {tuple(O.lifo_permutation(i, m)) for i in range(math.factorial(m))}
        assert len(orders) == math.factorial(m)
        assert all(sorted(o) == list(range(m)) for o in orders)


@pytest.mark.parametrize("n,c,L", [(2, 4, 5), (1, 8, 5), (2, 8, 4)])
def test_lifo_consistent_with_all_paths(n, c, L):
    """Every movelist path is an assembly path: what it finds (local ambiguity,
    growth past the grid, final configurations) exists among all paths, and a
    tile set whose every path ends in one configuration is deterministic."""
    rng = random.Random(300 * n + c)
    k = 6
    bits = 4 * n * (c.bit_length() - 1)
    checked = det = 0
    with O.process_mode(True):
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
                if r["cls"] == O.ND_LOCAL:
                    assert truth.trivial_nd
                if r["cls"] == O.UNBOUNDED:
                    assert truth.escape
                if r["cls"] == O.ND_STERIC:
                    assert len(truth.terminals) >= 2
                if r["cls"] in (O.DET_BOUNDED, O.ND_STERIC):
                    assert cfg in truth.terminals and r["size"] == len(cfg)
                if truth.deterministic_bounded:
                    det += 1
                    assert r["cls"] == O.DET_BOUNDED and cfg in truth.terminals
    assert det > 0


def test_lifo_invariance_and_monotone_in_k():
    """The movelist process sees only geometry and the binding rule: relabelling
    by a permutation that preserves M or turning a non-seed tile changes
    nothing; a class decided at replicate j < k stays for larger k."""
    rng = random.Random(5)
    n, c, L, k = 2, 8, 12, 6
    swap_pair = {0: 0, 1: 2, 2: 1, 3: 3, 4: 4, 5: 5, 6: 6, 7: 7}
    with O.process_mode(True):
        for _ in range(150):
            g = rng.getrandbits(24)
            col = [int(v) for v in O.decode(g, n, c)[:8]]
            base = O.classify(n, c, L, k, 4, col, 77)
            assert O.classify(n, c, L, k, 4, [swap_pair[v] for v in col], 77) == base
            t1 = col[4:8]
            assert O.classify(n, c, L, k, 4, col[:4] + [t1[3], t1[0], t1[1], t1[2]], 77) == base
        res = {kk: O.enumerate_space(n, c, 10, kk, 2, 1 << 20, 3000)[0] for kk in (2, 5, 12)}
    for k1, k2 in ((2, 5), (5, 12)):
        a, b = res[k1], res[k2]
        decided = a["decided_rep"] < k1
        assert np.array_equal(a[decided], b[decided])
        assert np.all(~(b["cls"] == O.DET_BOUNDED) | (a["cls"] == O.DET_BOUNDED))


def _offers(occ, tuples, site):
    """Rotated tuples that fit an empty site next to the occupied ones."""
    x, y = site
    fits = set()
    for tup in tuples:
        for d, (dx, dy) in enumerate(((0, -1), (1, 0), (0, 1), (-1, 0))):
            nb = occ.get((x + dx, y + dy))
            if nb is not None and B.pair_bind(tup[d], nb[(d + 2) % 4]):
                fits.add(tup)
                break
    return fits


def test_lifo_steps_rederived():
    """Every step of traced replicates re-derived from the definition: word s of
    Philox(ctr = (s >> 2, rep, id_lo, id_hi)) orders the m sites that have just
    become frontier sites (N, E, S, W of the tile placed last), permutation
    number floor(u m! / 2^32) in the factorial number system, pushed first
    pick first; the next tile goes on the top site."""
    rng = random.Random(41)
    n, c, L, k, seed = 2, 8, 12, 4, 0x77
    checked = 0
    with O.process_mode(True):
        while checked < 8:
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
            frontier = set()
            stack = []
            last = (L // 2, L // 2)
            nctr = 1
            while nctr < (len(tr) >> 2) + 1:
                nctr *= 2  # the Philox helper takes a power-of-two batch
            ctrs = list(range(nctr))
            words = dict(zip(ctrs, _triton_philox([[cc, rep, g & 0xFFFFFFFF, g >> 32] for cc in ctrs],
                                                  [seed & 0xFFFFFFFF, seed >> 32])))
            for s, (m, u, idx, x, y, tup) in enumerate(tr):
                new = []
                for dx, dy in ((0, -1), (1, 0), (0, 1), (-1, 0)):
                    q = (last[0] + dx, last[1] + dy)
                    if 0 <= q[0] < L and 0 <= q[1] < L and q not in occ and q not in frontier:
                        if len(_offers(occ, tuples, q)) == 1:
                            new.append(q)
                assert m == len(new)
                assert u == words[s >> 2][s & 3]
                assert idx == (u * math.factorial(m)) >> 32
                # factorial number system: digit i picks among the sites left
                pool, code = list(new), idx
                for i in range(m):
                    f = math.factorial(m - 1 - i)
                    stack.append(pool.pop(code // f))
                    code %= f
                frontier.update(new)
                site = stack.pop()
                assert site == (x, y)
                fits = _offers(occ, tuples, site)
                assert len(fits) == 1
                t, q = divmod(tup, 4)
                assert B.rotated(tiles[t], q) == next(iter(fits))
                occ[site] = next(iter(fits))
                frontier.discard(site)
                last = site
            checked += 1

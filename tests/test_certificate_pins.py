"""Pins of the two certificates that end a DET genotype after replicate 0
(closed final shape; dominated offending offers): whenever either holds for
the oracle's replicate-0 configuration, the exhaustive explorer of every
assembly path finds no local ambiguity, no growth past the lattice and a single
final configuration, that configuration.  No GPU needed."""
import random
from collections import Counter

import pytest

from oracle import bruteforce as B
from oracle import oracle as O

from certificates import closed, dominated
from test_oracle_pins import _oracle_config


@pytest.mark.parametrize("n,c,L,count,seed", [(2, 8, 7, 1500, 11), (2, 8, 9, 1500, 12), (2, 4, 7, 800, 13),
                                              (3, 4, 6, 800, 14), (3, 8, 7, 800, 15)])
def test_certificates_agree_with_all_paths(n, c, L, count, seed):
    rng = random.Random(seed)
    bits = 4 * n * (c.bit_length() - 1)
    seen = Counter()
    for _ in range(count):
        g = rng.getrandbits(bits)
        col = O.decode(g, n, c)
        r = O.classify(n, c, L, 6, 3, col, g, want_grid=True)
        if r["decided_rep"] == 0 and r["cls"] in (O.ND_LOCAL, O.UNBOUNDED):
            continue  # replicate 0 did not end in a configuration
        is_closed = closed(list(col), n, c, r["grid"])
        is_dom = is_closed or dominated(list(col), n, c, r["grid"])
        truth = B.explore(col, n, L, max_states=20000)
        if not truth.complete:
            continue
        kind = "closed" if is_closed else "dominated" if is_dom else "neither"
        det = truth.deterministic_bounded and truth.terminals == {_oracle_config(r, col)}
        seen[kind, det] += 1
        if is_dom:
            assert det and r["cls"] == O.DET_BOUNDED, (n, c, L, g, kind)
    # the dominance test is not vacuous: it certifies genotypes the closure
    # test does not, and it refuses some that are not deterministic
    assert seen["dominated", True] > 0
    if (n, c, L) == (2, 8, 7):
        assert seen["neither", False] > 0


def test_dominance_worked_example():
    """n = 2, c = 4 (1-2 bind; 0 and 3 bind nothing), tiles (N, E, S, W):
    t0 = (0, 1, 0, 1), the seed, and t1 = (0, 0, 1, 2) with turns 4 = (0, 0, 1, 2),
    5 = (2, 0, 0, 1), 6 = (1, 2, 0, 0), 7 = (0, 1, 2, 0).  The seed's E side
    takes 4 and its W side 6 (two frontier sites: the draws choose the order);
    below 4 comes 5, west of 5 another 6; above the west 6 comes 7, east of 7
    another 4:
        7 4 .
        6 0 4
        . 6 5
    Each later tile of an arm offers a second tuple back to the cell it grew
    from -- 5 offers {4, 1} north, the lower 6 offers {5, 0} east, 7 offers
    {6, 1} south, the upper 4 offers {7, 0} west -- so the shape is not closed;
    but each offerer is reachable from the seed only through that cell, which is
    therefore always placed first: every path ends in this shape."""
    n, c, L = 2, 4, 9
    col = O.decode(4358, n, c)
    assert [int(v) for v in col[:8]] == [0, 1, 0, 1, 0, 0, 1, 2]
    r = O.classify(n, c, L, 20, 3, col, 4358, want_grid=True, trace_rep=0)
    g = r["grid"]
    crop = [[int(g[y, x]) for x in range(L // 2 - 1, L // 2 + 2)] for y in range(L // 2 - 1, L // 2 + 2)]
    assert crop == [[7, 4, -1], [6, 0, 4], [-1, 6, 5]]
    assert any(t[0] > 1 for t in r["trace"])  # not a forced path
    assert not closed(list(col), n, c, g) and dominated(list(col), n, c, g)
    truth = B.explore(col, n, L)
    assert truth.complete and truth.deterministic_bounded and truth.terminals == {_oracle_config(r, col)}
    assert r["cls"] == O.DET_BOUNDED and r["decided_rep"] == 20 and r["size"] == 7

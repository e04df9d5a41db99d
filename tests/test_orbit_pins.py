"""Pins of the oracle's orbit representatives (the orbit mode of the
enumeration).  The group is generated by hand-written moves taken from the
binding rule, not from the oracle's own enumeration of it: swapping the two
colours of a binding pair, exchanging two binding pairs, exchanging the two
colours that bind nothing, and turning a non-seed tile.  No GPU needed."""
import math

import numpy as np
import pytest

from oracle import oracle as O

scipy_sparse = pytest.importorskip("scipy.sparse")
from scipy.sparse.csgraph import connected_components  # noqa: E402


def _structure(c):
    """Binding pairs (1, 2), (3, 4), ... among 0 .. c-1, and the colours that bind nothing."""
    pairs = [(a, a + 1) for a in range(1, c, 2) if a + 1 < c]
    paired = {x for p in pairs for x in p}
    inert = [x for x in range(c) if x not in paired]
    return pairs, inert


def test_colour_automorphism_counts():
    # any permutation of the pairs, either order within each pair, any permutation of the inert colours
    for c in (1, 2, 4, 8):
        pairs, inert = _structure(c)
        want = math.factorial(len(pairs)) * 2 ** len(pairs) * math.factorial(len(inert))
        assert O.colour_automorphism_count(c) == want


def _decode_all(g, n, b):
    cols = np.zeros((g.shape[0], 4 * n), np.int64)
    for m in range(4 * n):
        cols[:, m] = (g >> np.uint64(b * (4 * n - 1 - m))) & np.uint64((1 << b) - 1)
    return cols


def _encode_all(cols, n, b):
    g = np.zeros(cols.shape[0], np.uint64)
    for m in range(4 * n):
        g |= cols[:, m].astype(np.uint64) << np.uint64(b * (4 * n - 1 - m))
    return g


def _generators(n, c):
    """Moves on colour arrays [N, 4n] that generate the symmetry group."""
    pairs, inert = _structure(c)
    moves = []

    def relabel(mapping):
        lut = np.arange(c)
        for a, b in mapping.items():
            lut[a] = b
        return lambda cols: lut[cols]

    for a, b in pairs:
        moves.append(relabel({a: b, b: a}))
    for (a1, b1), (a2, b2) in zip(pairs, pairs[1:]):
        moves.append(relabel({a1: a2, a2: a1, b1: b2, b2: b1}))
    if len(inert) == 2:
        moves.append(relabel({inert[0]: inert[1], inert[1]: inert[0]}))
    for t in range(1, n):
        def turn(cols, t=t):
            out = cols.copy()
            out[:, 4 * t: 4 * t + 4] = cols[:, [4 * t + (e - 1) % 4 for e in range(4)]]
            return out
        moves.append(turn)
    for t in range(1, n - 1):
        def swap(cols, t=t):
            out = cols.copy()
            out[:, 4 * t: 4 * t + 4], out[:, 4 * t + 4: 4 * t + 8] = cols[:, 4 * t + 4: 4 * t + 8], cols[:, 4 * t: 4 * t + 4]
            return out
        moves.append(swap)
    return moves


@pytest.mark.parametrize("n,c", [(2, 2), (2, 4), (3, 2)])
def test_orbits_equal_the_components_of_the_generated_group(n, c):
    b = int(math.log2(c))
    size = 1 << (4 * n * b)
    g = np.arange(size, dtype=np.uint64)
    cols = _decode_all(g, n, b)
    rows, cols_idx = [], []
    for move in _generators(n, c):
        h = _encode_all(move(cols), n, b)
        rows.append(g)
        cols_idx.append(h)
    graph = scipy_sparse.coo_matrix((np.ones(sum(r.shape[0] for r in rows)),
                                     (np.concatenate(rows).astype(np.int64),
                                      np.concatenate(cols_idx).astype(np.int64))), shape=(size, size))
    ncomp, comp = connected_components(graph, directed=False)
    reps = O.orbit_reps(n, c, 0, size)
    # one representative per component, and it is the component's smallest genotype
    comp_min = np.full(ncomp, np.iinfo(np.int64).max)
    np.minimum.at(comp_min, comp, g.astype(np.int64))
    assert np.array_equal(reps.astype(np.int64), comp_min[comp])
    assert np.unique(reps).shape[0] == ncomp


def test_orbit_mode_equals_the_process_with_representative_stream_ids():
    """Every genotype of S_{2,4} assembles, with its representative's stream id,
    exactly as the representative does: the orbit mode loses nothing."""
    n, c, L, k, seed = 2, 4, 16, 10, 1
    res, reps = O.enumerate_orbits(n, c, L, k, seed, 1 << 16)
    rng = np.random.default_rng(0)
    pick = rng.choice(1 << 16, size=400, replace=False)
    cols = np.zeros((pick.shape[0], 16), np.uint8)
    for i, gi in enumerate(pick.tolist()):
        cols[i, :8] = O.decode(gi, n, c)[:8]
    direct, _ = O.classify_batch(cols, n=n, c=c, L=L, k=k, seed=seed, ids=reps[pick])
    assert np.array_equal(direct, res[pick])
    # the orbit mode is not the plain enumeration: ids differ, so some results do
    plain, _ = O.enumerate_space(n, c, L, k, seed, 0, 1 << 16)
    assert np.unique(reps).shape[0] < (1 << 16) // 4
    assert np.array_equal(res[reps == np.arange(1 << 16, dtype=np.uint64)],
                          plain[reps == np.arange(1 << 16, dtype=np.uint64)])

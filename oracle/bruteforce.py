"""Exact all-paths explorer for tiny JaTAM tile sets -- TEST INFRASTRUCTURE.

Where the oracle follows ONE stochastic assembly path per replicate, this
module follows EVERY path: it enumerates the whole set Prod of configurations
reachable from the seed (appendix "Winfree's abstract tile assembly model":
Prod, Term, halting; appendix "Modifications to Winfree's aTAM": temperature
1, pair-binding matrix M, rotation without flips, seed first and centred,
trivial and steric non-determinism, boundedness by a square of dimension d).
It is written independently of ``jatam_oracle.c`` and works on rotated colour
tuples by value, so it pins the oracle's semantics without sharing its code:

* ``trivial_nd``  -- some reachable configuration has an empty site where two
  different rotated tuples could attach;
* ``escape``      -- some reachable configuration (inside the L x L grid) has an
  attachable site outside the grid, i.e. the set is unbounded by L;
* ``terminals``   -- the reachable configurations to which nothing more can
  attach, inside or outside the grid (Term restricted to the grid).

Only meant for tiny grids (L <= 7): the state space is exponential.
"""
from __future__ import annotations

from dataclasses import dataclass, field

# direction d: 0 = N, 1 = E, 2 = S, 3 = W; y grows to the south
_OFF = ((0, -1), (1, 0), (0, 1), (-1, 0))


def pair_bind(a: int, b: int) -> bool:
    """Colours bind in adjacent pairs 1-2, 3-4, 5-6, ...; 0 is inert."""
    if a == 0 or b == 0:
        return False
    lo, hi = min(a, b), max(a, b)
    return lo % 2 == 1 and hi == lo + 1


def rotated(tile, r):
    """Tile (N, E, S, W) turned clockwise by r quarter turns."""
    return tuple(tile[(d - r) % 4] for d in range(4))


@dataclass
class Truth:
    trivial_nd: bool = False
    escape: bool = False
    terminals: set = field(default_factory=set)
    n_states: int = 0
    complete: bool = True

    @property
    def deterministic_bounded(self) -> bool:
        return self.complete and not self.trivial_nd and not self.escape and len(self.terminals) == 1


def explore(col, n: int, L: int, max_states: int = 20000) -> Truth:
    """Explore all assembly paths of the tile set col[4t + e] on an L x L grid."""
    tiles = [tuple(int(v) for v in col[4 * t: 4 * t + 4]) for t in range(n)]
    options = sorted({rotated(tl, r) for tl in tiles for r in range(4)})
    centre = (L // 2, L // 2)
    start = frozenset({(centre, tiles[0])})
    seen = {start}
    stack = [start]
    truth = Truth()

    def inside(p):
        return 0 <= p[0] < L and 0 <= p[1] < L

    while stack:
        state = stack.pop()
        occ = dict(state)
        sites = set()
        for (x, y) in occ:
            for dx, dy in _OFF:
                q = (x + dx, y + dy)
                if q not in occ:
                    sites.add(q)
        grows = False
        for q in sites:
            fits = []
            for tup in options:
                for d, (dx, dy) in enumerate(_OFF):
                    nb = occ.get((q[0] + dx, q[1] + dy))
                    if nb is not None and pair_bind(tup[d], nb[(d + 2) % 4]):
                        fits.append(tup)
                        break
            if len(fits) >= 2:
                truth.trivial_nd = True
            if not fits:
                continue
            grows = True
            if not inside(q):
                truth.escape = True
                continue
            for tup in fits:
                nxt = state | {(q, tup)}
                if nxt not in seen:
                    if len(seen) >= max_states:
                        truth.complete = False
                        truth.n_states = len(seen)
                        return truth
                    seen.add(nxt)
                    stack.append(nxt)
        if not grows:
            truth.terminals.add(state)
    truth.n_states = len(seen)
    return truth


def shape_of(config) -> frozenset:
    return frozenset(p for p, _ in config)

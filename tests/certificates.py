"""Certificates that a final replicate-0 configuration fixes the outcome of
every replicate, written out from the binding rule (pairs 1-2, 3-4, 5-6 bind;
0 and an odd top colour bind nothing) on the oracle's replicate-0 grid of
tuple ids.  Test helpers: shared by the explorer pins and the GPU work-counter
test."""

_DX, _DY = (0, 1, 0, -1), (-1, 0, 1, 0)


def closed(col, n, c, grid):
    """The closure test of a final replicate-0 configuration, written out from
    the binding rule: for every two adjacent tiles, the tuples the one offers
    the other's cell are that cell's tuple or none (the seed's cell, occupied
    first in every replicate, may be offered anything)."""
    def bind(a, b):
        return a != 0 and b != 0 and min(a, b) % 2 == 1 and max(a, b) == min(a, b) + 1 and max(a, b) < c
    side = {4 * t + r: [col[4 * t + (d - r) % 4] for d in range(4)] for t in range(n) for r in range(4)}
    rep = {a: min(b for b in range(a + 1) if side[b] == side[a]) for a in side}
    L = grid.shape[0]
    for y in range(L):
        for x in range(L):
            u = grid[y, x]
            if u < 0:
                continue
            for d in range(4):
                qx, qy = x + _DX[d], y + _DY[d]
                if not (0 <= qx < L and 0 <= qy < L) or grid[qy, qx] < 0 or (qx, qy) == (L // 2, L // 2):
                    continue
                offered = {rep[a] for a in side if bind(side[a][(d + 2) % 4], side[u][d])}
                if offered and offered != {grid[qy, qx]}:
                    return False
    return True


def dominated(col, n, c, grid):
    """The dominance test of a final replicate-0 configuration A0 that is not
    closed, written out from the binding rule: u -> v when u offers v's own tuple
    to v; every offer u -> q (q not the seed's cell) of another tuple must come
    from a cell u that no path u -> ... from the seed reaches without passing q."""
    def bind(a, b):
        return a != 0 and b != 0 and min(a, b) % 2 == 1 and max(a, b) == min(a, b) + 1 and max(a, b) < c
    side = {4 * t + r: [col[4 * t + (d - r) % 4] for d in range(4)] for t in range(n) for r in range(4)}
    rep = {a: min(b for b in range(a + 1) if side[b] == side[a]) for a in side}
    L = grid.shape[0]
    seed = (L // 2, L // 2)
    cells = {(x, y) for y in range(L) for x in range(L) if grid[y, x] >= 0}
    good, bad = {p: [] for p in cells}, []
    for (x, y) in cells:
        u = grid[y, x]
        for d in range(4):
            q = (x + _DX[d], y + _DY[d])
            if q not in cells:
                continue
            offered = {rep[a] for a in side if bind(side[a][(d + 2) % 4], side[u][d])}
            if grid[q[1], q[0]] in offered:
                good[(x, y)].append(q)
            if q != seed and offered and offered != {grid[q[1], q[0]]}:
                bad.append(((x, y), q))
    for p, q in bad:
        seen, todo = {seed}, [seed]
        while todo:
            for v in good[todo.pop()]:
                if v != q and v not in seen:
                    seen.add(v)
                    todo.append(v)
        if p in seen:
            return False
    return True

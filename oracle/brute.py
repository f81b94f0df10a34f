"""Exhaustive chromatic number for tiny graphs (n <= 12).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  Backtracking over vertex
colorings with colors 1..k for k = 1, 2, ...; the first k that admits a
proper coloring is chi(G).  Any valid coloring uses at least chi(G) colors,
which bounds every heuristic from below.
"""
from __future__ import annotations


def chromatic_number(g) -> int:
    ro = [int(x) for x in g.row_offsets]
    ci = [int(x) for x in g.col_idx]
    n = len(ro) - 1
    if n == 0:
        return 0
    if n > 12:
        raise ValueError("brute force is limited to 12 vertices")
    adj = [ci[ro[v]:ro[v + 1]] for v in range(n)]

    def colorable(k: int) -> bool:
        col = [0] * n

        def place(v: int) -> bool:
            if v == n:
                return True
            used = {col[w] for w in adj[v] if w < v}
            # symmetry breaking: vertex v may open at most one new color
            top = max(col[:v], default=0)
            for c in range(1, min(k, top + 1) + 1):
                if c not in used:
                    col[v] = c
                    if place(v + 1):
                        return True
            col[v] = 0
            return False

        return place(0)

    k = 1
    while not colorable(k):
        k += 1
    return k

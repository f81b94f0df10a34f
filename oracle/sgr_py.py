"""Second, independently written det-SGR simulator in pure Python.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  Written from the round
loop of Algorithm 7 (Sect. 3.1) with sets instead of the colorMask stamp of
Algorithm 4, so that a slip in the C oracle's stamping or worklist handling
shows up as a disagreement.  Meant for graphs of at most a few thousand
vertices.
"""
from __future__ import annotations


def _adj(g):
    ro = [int(x) for x in g.row_offsets]
    ci = [int(x) for x in g.col_idx]
    return [ci[ro[v]:ro[v + 1]] for v in range(len(ro) - 1)]


def _priority_key(rule, adj):
    """Vertices with the larger key keep their color in a conflict."""
    if rule in (0, "low_keeps"):
        return lambda v: -v
    if rule in (1, "low_loses"):
        return lambda v: v
    if rule in (2, "degree"):
        return lambda v: (len(adj[v]), -v)
    raise ValueError(rule)


def det_sgr_py(g, rule=0):
    """Returns (colors list, k, rounds, [|W_r|], [sum of degrees of W_r])."""
    adj = _adj(g)
    n = len(adj)
    key = _priority_key(rule, adj)
    colors = [0] * n
    work = set(range(n))
    rounds, tw, td = 0, [], []
    while work:
        rounds += 1
        frozen = list(colors)
        tent = {}
        for v in work:
            used = {frozen[w] for w in adj[v]}
            c = 1
            while c in used:
                c += 1
            tent[v] = c
        tw.append(len(work))
        td.append(sum(len(adj[v]) for v in work))
        for v, c in tent.items():
            colors[v] = c
        losers = set()
        for v in work:
            for w in adj[v]:
                if colors[w] == colors[v] and key(w) > key(v):
                    losers.add(v)
                    break
        for v in losers:
            colors[v] = 0
        work = losers
    k = max(colors) if colors else 0
    return colors, k, rounds, tw, td


def serial_greedy_py(g):
    """Algorithm 1 with a Python set per vertex."""
    adj = _adj(g)
    colors = [0] * len(adj)
    for v in range(len(adj)):
        used = {colors[w] for w in adj[v]}
        c = 1
        while c in used:
            c += 1
        colors[v] = c
    return colors, (max(colors) if colors else 0)


def topo_sgr_py(g, rule=0):
    """The same deterministic rounds on the topology-driven schedule of
    Algorithm 6 (Sect. 3.1): every iteration visits every vertex, FirstFit for
    the ones not colored yet (reading the colors final at the start of the
    iteration), then ConflictResolve for them (judged on the iteration's
    tentative colors), which marks the non-conflicting ones colored; the loop
    stops when an iteration finds nothing to color.  Returns (colors list, k,
    rounds, [vertices colored tentatively per iteration], [their degree sums]).
    """
    adj = _adj(g)
    n = len(adj)
    key = _priority_key(rule, adj)
    color = [0] * n
    colored = [False] * n
    rounds, tw, td = 0, [], []
    while True:
        changed = False
        final = [color[w] if colored[w] else 0 for w in range(n)]
        open_now = [not colored[v] for v in range(n)]
        tent = [0] * n
        for v in range(n):
            if open_now[v]:
                used = {final[w] for w in adj[v]}
                c = 1
                while c in used:
                    c += 1
                tent[v] = c
                changed = True
        if not changed:
            break
        rounds += 1
        tw.append(sum(open_now))
        td.append(sum(len(adj[v]) for v in range(n) if open_now[v]))
        for v in range(n):
            if open_now[v] and not any(open_now[w] and tent[w] == tent[v] and key(w) > key(v) for w in adj[v]):
                color[v] = tent[v]
                colored[v] = True
    k = max(color) if color else 0
    return color, k, rounds, tw, td

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

"""Pins for the CPU oracle (no GPU).

Each check is tied to something fixed outside the oracle: closed forms for
graph families, brute-force chromatic numbers, invariants of Algorithms 1, 4,
5 and 7, and an independently written Python restatement.  A plausible slip in
the oracle fails at least one of them:

* live instead of frozen reads in FirstFit -> K_n would finish in 1 round;
* the loser rule flipped -> the star and path round counts change;
* judging conflicts after clearing instead of before -> the path round count
  and colors change (P_3: vertex 2 would keep color 1 in round 1);
* a dropped clearing step -> the C_9 and K_n colors change;
* an off-by-one in first-fit (colors from 0 or skipping 1) -> edgeless/star pins.
"""
import itertools
import random

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import brute, sgr_py


# ------------------------------------------------------------ small graphs

def complete(n):
    return gg.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def path(n):
    return gg.from_edges(n, [(i, i + 1) for i in range(n - 1)])


def cycle(n):
    return gg.from_edges(n, [(i, (i + 1) % n) for i in range(n)])


def star(n, center=0):
    return gg.from_edges(n, [(center, i) for i in range(n) if i != center])


def crown(p):
    # vertices u_i = 2i, v_i = 2i+1; u_i ~ v_j for i != j
    return gg.from_edges(2 * p, [(2 * i, 2 * j + 1) for i in range(p) for j in range(p) if i != j])


def petersen():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return gg.from_edges(10, outer + spokes + inner)


def random_graph(n, p, seed):
    rnd = random.Random(seed)
    return gg.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n) if rnd.random() < p])


def edgeless(n):
    return gg.from_edges(n, [])


def valid(g, colors):
    res = oracle.check(g, colors)
    return res["valid"]


# ------------------------------------------------------------ brute force

@pytest.mark.parametrize("g,chi", [
    (complete(1), 1), (complete(5), 5), (edgeless(4), 1), (path(7), 2), (cycle(8), 2),
    (cycle(9), 3), (petersen(), 3), (crown(4), 2), (star(6), 2),
    (gg.from_edges(4, [(0, 1), (1, 2), (2, 0), (2, 3)]), 3),
])
def test_bruteforce_chi_known_values(g, chi):
    assert brute.chromatic_number(g) == chi


# ------------------------------------------------------------ serial greedy

@pytest.mark.parametrize("n", [1, 2, 5, 17])
def test_serial_complete_graph(n):
    c, k = oracle.serial_greedy(complete(n))
    assert k == n and list(c) == list(range(1, n + 1))


@pytest.mark.parametrize("g", [path(2), path(9), cycle(10), star(7), star(7, center=3),
                               gg.stencil(6, 5, 1, 5), crown(2)])
def test_serial_bipartite_natural_order_two_colors(g):
    c, k = oracle.serial_greedy(g)
    assert k == 2 and valid(g, c)


def test_serial_edgeless_and_empty():
    c, k = oracle.serial_greedy(edgeless(5))
    assert k == 1 and list(c) == [1] * 5
    c, k = oracle.serial_greedy(edgeless(0))
    assert k == 0 and c.shape == (0,)


@pytest.mark.parametrize("p", [2, 3, 5, 8])
def test_serial_crown_graph_worst_case(p):
    # ordered u1, v1, u2, v2, ... first-fit gives u_i and v_i color i
    c, k = oracle.serial_greedy(crown(p))
    assert k == p
    assert list(c) == [i // 2 + 1 for i in range(2 * p)]


def test_serial_odd_cycle():
    c, k = oracle.serial_greedy(cycle(9))
    assert k == 3 and list(c[:8]) == [1, 2] * 4 and c[8] == 3


@pytest.mark.parametrize("dims,points,k", [((7, 6, 1), 9, 4), ((5, 5, 4), 27, 8), ((3, 4, 5), 7, 2)])
def test_serial_stencils_natural_order(dims, points, k):
    g = gg.stencil(*dims, points=points)
    c, kk = oracle.serial_greedy(g)
    assert kk == k and valid(g, c)


def test_serial_bounds_and_python_restatement():
    for seed in range(30):
        n = 1 + seed % 12
        g = random_graph(n, 0.45, seed)
        c, k = oracle.serial_greedy(g)
        assert valid(g, c)
        assert k <= int(g.degrees().max(initial=0)) + 1
        assert k >= brute.chromatic_number(g)
        cp, kp = sgr_py.serial_greedy_py(g)
        assert list(c) == cp and k == kp
        # every color 1..k is used (first-fit colors are contiguous)
        assert set(c.tolist()) == set(range(1, k + 1))


# ------------------------------------------------------------ det-SGR closed forms

@pytest.mark.parametrize("n", [1, 2, 6, 13])
def test_det_complete_graph_n_rounds(n):
    r = oracle.det_sgr(complete(n))
    assert r.rounds == n and r.num_colors == n
    assert list(r.colors) == list(range(1, n + 1))


@pytest.mark.parametrize("n", [2, 3, 4, 7, 10, 31])
def test_det_path(n):
    r = oracle.det_sgr(path(n))
    assert r.rounds == n // 2 + 1
    assert list(r.colors) == [1 + (i % 2) for i in range(n)]


def test_det_star_center_zero():
    r = oracle.det_sgr(star(9))
    assert r.rounds == 2 and r.colors[0] == 1 and set(r.colors[1:].tolist()) == {2}


def test_det_star_center_last():
    # center 8 loses to leaf 0 in round 1 only; leaves 1..7 have no lower neighbour
    r = oracle.det_sgr(star(9, center=8))
    assert r.rounds == 2 and r.colors[8] == 2 and set(r.colors[:8].tolist()) == {1}


def test_det_edgeless_one_round():
    r = oracle.det_sgr(edgeless(6))
    assert r.rounds == 1 and list(r.colors) == [1] * 6
    r = oracle.det_sgr(edgeless(0))
    assert r.rounds == 0 and r.num_colors == 0


def test_det_cycle9_differs_from_serial_but_three_colors():
    g = cycle(9)
    r = oracle.det_sgr(g)
    c, k = oracle.serial_greedy(g)
    assert r.num_colors == 3 and k == 3 and valid(g, r.colors)
    assert not np.array_equal(r.colors, c)


def test_det_first_round_keeps_exactly_vertices_without_lower_neighbour():
    for seed in range(10):
        g = random_graph(40, 0.1, seed)
        r = oracle.det_sgr(g, max_rounds=1)
        lower = np.array([np.any(g.col_idx[g.row_offsets[v]:g.row_offsets[v + 1]] < v)
                          for v in range(g.n)])
        assert np.array_equal(r.colors == 1, ~lower)
        assert np.all(r.colors[lower] == 0)
        assert r.trace_w[0] == g.n and r.trace_d[0] == g.m


@pytest.mark.parametrize("dims,points", [((9, 7, 1), 9), ((6, 5, 4), 27), ((11, 3, 1), 5)])
def test_det_equals_serial_on_natural_order_stencils(dims, points):
    g = gg.stencil(*dims, points=points)
    r = oracle.det_sgr(g)
    c, _ = oracle.serial_greedy(g)
    assert np.array_equal(r.colors, c)


@pytest.mark.parametrize("rule", ["low_keeps", "low_loses", "degree"])
def test_det_matches_python_restatement(rule):
    graphs = [random_graph(1 + s % 60, 0.08 + 0.05 * (s % 4), s) for s in range(40)]
    graphs += [gg.uniform(1500, 6.0, seed=5), gg.rmat(10, 8, seed=2), crown(6), petersen()]
    for g in graphs:
        r = oracle.det_sgr(g, rule)
        cp, kp, rp, twp, tdp = sgr_py.det_sgr_py(g, rule)
        assert list(r.colors) == cp and r.num_colors == kp and r.rounds == rp
        assert list(r.trace_w) == twp and list(r.trace_d) == tdp


@pytest.mark.parametrize("rule", ["low_keeps", "low_loses", "degree"])
def test_topology_driven_schedule_gives_the_same_rounds(rule):
    # Algorithm 6 visits every vertex each iteration and marks the
    # non-conflicting ones colored; under the deterministic readings it colors
    # exactly W_r per iteration, so colors, k, rounds and the per-round sums
    # equal the worklist loop's (reading 5: detect over V or over W is the same)
    graphs = [random_graph(1 + s % 50, 0.1 + 0.05 * (s % 3), 300 + s) for s in range(30)]
    graphs += [gg.uniform(800, 5.0, seed=8), gg.rmat(9, 8, seed=4), crown(5), petersen(), star(7, center=3)]
    for g in graphs:
        r = oracle.det_sgr(g, rule)
        ct, kt, rt, twt, tdt = sgr_py.topo_sgr_py(g, rule)
        assert list(r.colors) == ct and r.num_colors == kt and r.rounds == rt
        assert list(r.trace_w) == twt and list(r.trace_d) == tdt


@pytest.mark.parametrize("rule", ["low_keeps", "low_loses", "degree"])
def test_det_invariants(rule):
    for seed in range(25):
        n = 1 + seed % 12
        g = random_graph(n, 0.5, 100 + seed)
        r = oracle.det_sgr(g, rule)
        assert r.status == 0 and valid(g, r.colors)
        assert 1 <= r.rounds <= n
        assert r.num_colors <= r.max_degree + 1
        assert r.num_colors >= brute.chromatic_number(g)
        assert r.sum_w == int(r.trace_w.sum()) and r.sum_d == int(r.trace_d.sum())
        assert r.trace_w[0] == n
        assert np.all(np.diff(r.trace_w) < 0)  # at least one keeper per round


def test_det_rule_changes_outcome_on_star():
    # printed rule (lower id recolored): center 0 loses in round 1 to every leaf
    r = oracle.det_sgr(star(6), "low_loses")
    assert r.rounds == 2 and r.colors[0] == 2 and set(r.colors[1:].tolist()) == {1}
    # degree rule: the center has the larger degree and keeps wherever it sits
    r = oracle.det_sgr(star(6, center=5), "degree")
    assert r.rounds == 2 and r.colors[5] == 1 and set(r.colors[:5].tolist()) == {2}


def test_det_round_cap_reports_no_convergence():
    r = oracle.det_sgr(complete(6), max_rounds=3)
    assert r.status == -5 and r.rounds == 3


def test_check_counts_monochrome_entries():
    g = path(4)
    res = oracle.check(g, np.array([1, 1, 2, 1], dtype=np.int32))
    assert res["monochrome"] == 2 and not res["valid"]
    res = oracle.check(g, np.array([1, 0, 1, 2], dtype=np.int32))
    assert res["bad_range"] == 1 and not res["valid"]


@pytest.mark.slow
def test_er20k_config_numbers():
    g = gg.er20k()
    c, k = oracle.serial_greedy(g)
    r = oracle.det_sgr(g)
    assert valid(g, c) and valid(g, r.colors)
    assert r.num_colors <= int(g.degrees().max()) + 1
    assert r.num_colors <= 1.1 * k + 1

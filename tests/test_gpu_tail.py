"""GPU parity of the one-CTA tail of deterministic mode.

Once at most `tail_vertices` vertices are left on the worklist, the grid
builds the subgraph they induce and one CTA runs the remaining rounds with the
per-vertex state in shared memory.  The colors, k, the round count and the
per-round sums must equal the oracle's bit for bit whichever kernel hands the
rounds over (the whole-worklist rounds or the activation-list rounds), at any
hand-over size, under every loser rule, for batches, and when a vertex needs a
color above 256 (its bitmap is full and it scans its row).  With the tail
switched off the grid kernels must give the same answers.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture
def tuning(gpu_lib):
    saved = gpu_lib.sgr_get_tuning()
    yield gpu_lib
    gpu_lib.sgr_set_tuning(**saved)


def complete(n):
    return gg.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def run(lib, g, mode):
    import torch
    ro = torch.from_numpy(np.ascontiguousarray(g.row_offsets)).cuda()
    ci = torch.from_numpy(np.ascontiguousarray(g.col_idx)).cuda() if g.m else torch.zeros(
        4, dtype=torch.int32, device="cuda")
    out = torch.full((max(g.n, 1),), -7, dtype=torch.int32, device="cuda")
    k = lib.sgr_color(g.n, ro, ci, out, mode)
    torch.cuda.synchronize()
    return out[:g.n].cpu().numpy(), k, lib.sgr_last_stats()


def check(lib, g, rule, ref=None):
    ref = ref or oracle.det_sgr(g, rule)
    got, k, st = run(lib, g, "det+" + rule)
    assert np.array_equal(got, ref.colors), f"{g.name}: first diff at {np.argmax(got != ref.colors)}"
    assert k == ref.num_colors and st["rounds"] == ref.rounds
    assert st["sum_w"] == ref.sum_w and st["sum_d"] == ref.sum_d and st["sum_next"] == ref.sum_next
    return st


GRAPHS = [
    lambda: gg.rmat(14, 16, seed=7),
    lambda: gg.rmat(16, 16, seed=3),
    lambda: gg.uniform(20011, 7.0, seed=5),
    lambda: gg.stencil(24, 22, 20, 27),
    lambda: gg.stencil(60, 50, 1, 9),
]


@pytest.mark.parametrize("make", GRAPHS)
@pytest.mark.parametrize("rule", ["low_keeps", "low_loses", "degree"])
@pytest.mark.parametrize("policy", [0, 1, 2])
def test_tail_handover_sizes(tuning, make, rule, policy):
    g = make()
    ref = oracle.det_sgr(g, rule)
    tails = []
    for tv in (-1, 1, 40, 700, 0):
        tuning.sgr_set_tuning(active_lists=policy, tail_vertices=tv)
        st = check(tuning, g, rule, ref)
        tails.append(st["tail_rounds"])
    assert tails[0] == 0  # switched off
    assert tails[-1] > 0  # the default hands over on every one of these graphs


@pytest.mark.parametrize("rule", ["low_keeps", "low_loses", "degree"])
def test_tail_from_round_one_and_colors_above_256(tuning, rule):
    # n <= tail_vertices: the tail CTA runs every round; K_300 needs 300
    # colors, so the last 44 vertices fill their bitmaps and scan their rows
    tuning.sgr_set_tuning(tail_vertices=2880)
    for g in [complete(300), gg.from_edges(1, []), gg.from_edges(9, []), gg.uniform(2800, 30.0, seed=2),
              gg.rmat(11, 16, seed=4)]:
        st = check(tuning, g, rule)
        assert st["tail_rounds"] == st["rounds"]


def clique_and_falling_path():
    # K_45 on ids 0..44 beside a path 299-298-...-100 whose ids fall along
    # it: from round 33 to 45 the path's vertices still try color 1 while the
    # clique's try colors 33..45
    edges = [(i, j) for i in range(45) for j in range(i + 1, 45)]
    edges += [(v, v - 1) for v in range(299, 100, -1)]
    return gg.from_edges(300, edges)


@pytest.mark.parametrize("rule", ["low_keeps", "low_loses", "degree"])
def test_bit_matrix_rounds_with_colors_far_apart(tuning, rule):
    # at most 512 vertices: every round runs on the bit matrix, whose class
    # sets cover 32 tentative colors from the round's least one; colors above
    # that window are decided by a loop over the winners' tentative colors
    tuning.sgr_set_tuning(tail_vertices=0)
    st = check(tuning, clique_and_falling_path(), rule)
    assert st["tail_rounds"] == st["rounds"]


def test_tail_with_hubs_split_and_small_bins(tuning):
    for tune in [dict(light_max=4, chunk=64), dict(light_max=1, chunk=2048, blocks_per_sm=1)]:
        for tv in (100, 0):
            tuning.sgr_set_tuning(tail_vertices=tv, **tune)
            for g in [gg.rmat(15, 16, seed=9), complete(90)]:
                for rule in ["low_keeps", "degree"]:
                    check(tuning, g, rule)


@pytest.mark.parametrize("tv", [-1, 50, 0])
def test_tail_in_batches(tuning, tv):
    import torch
    tuning.sgr_set_tuning(tail_vertices=tv)
    graphs = [gg.mix_graph(s) for s in gg.mix_specs(20, 100, 30000, 5)]
    b = gg.pack(graphs)
    ro = torch.from_numpy(b.row_offsets).cuda()
    ci = torch.from_numpy(b.col_idx).cuda()
    n = int(b.vtx_off[-1])
    out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    k = np.zeros(b.G, dtype=np.int32)
    for rule in ["low_keeps", "degree"]:
        tuning.sgr_color_batch(b.G, b.vtx_off, b.edge_off, ro, ci, out, k, "det+" + rule)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for i, g in enumerate(graphs):
            ref = oracle.det_sgr(g, rule)
            assert np.array_equal(got[b.vtx_off[i]:b.vtx_off[i + 1]], ref.colors), f"graph {i}"
            assert k[i] == ref.num_colors


def test_activation_lists_past_the_push_buffer(tuning):
    # forced onto the activation lists, a uniform graph this size activates
    # about 8,000 vertices per CTA in round 2, more than a CTA's push buffer
    # holds: the rest go to the lists through warp-aggregated global appends
    g = gg.uniform(4_000_000, 10.0, seed=3)
    ref = oracle.det_sgr(g)
    tuning.sgr_set_tuning(active_lists=2)
    check(tuning, g, "low_keeps", ref)
    tuning.sgr_set_tuning(active_lists=2, tail_vertices=-1)
    check(tuning, g, "low_keeps", ref)

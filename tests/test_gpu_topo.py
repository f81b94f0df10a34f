"""GPU parity of the topology-driven schedule (Algorithm 6, SGR_MODE_TOPO).

Every iteration visits all vertices: FirstFit for those not final, then
ConflictResolve for those holding a tentative color.  Under the deterministic
readings an iteration colors exactly W_r, so the colors, k, the iteration
count and the per-round sums must equal the oracle's worklist loop bit for
bit, under every loser rule, through the device and the host-buffer entry
points, on rows of any length (lane and warp paths) and on unsorted rows.
The batched entry point refuses the mode.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def complete(n):
    return gg.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def star(n, center=0):
    return gg.from_edges(n, [(center, i) for i in range(n) if i != center])


def shuffled_rows(g, seed):
    rng = np.random.default_rng(seed)
    ci = g.col_idx.copy()
    for v in range(g.n):
        a, b = g.row_offsets[v], g.row_offsets[v + 1]
        rng.shuffle(ci[a:b])
    return gg.CSR(g.row_offsets.copy(), ci, g.name + "_shuf")


GRAPHS = [
    lambda: gg.from_edges(1, []),
    lambda: gg.from_edges(7, []),
    lambda: complete(2),
    lambda: complete(70),  # rows of 69 entries: the warp path
    lambda: star(300),
    lambda: star(300, center=299),
    lambda: gg.stencil(17, 13, 1, 9),
    lambda: gg.stencil(9, 8, 7, 27),
    lambda: gg.uniform(3000, 10.0, seed=4),
    lambda: gg.uniform(20011, 7.0, seed=5),
    lambda: gg.rmat(12, 16, seed=6),
    lambda: gg.rmat(14, 16, seed=7),
    lambda: shuffled_rows(gg.rmat(12, 16, seed=2), 1),
]


def run_device(lib, g, mode):
    import torch
    ro = torch.from_numpy(np.ascontiguousarray(g.row_offsets)).cuda()
    ci = torch.from_numpy(np.ascontiguousarray(g.col_idx)).cuda() if g.m else torch.zeros(
        4, dtype=torch.int32, device="cuda")
    out = torch.full((max(g.n, 1),), -7, dtype=torch.int32, device="cuda")
    k = lib.sgr_color(g.n, ro, ci, out, mode)
    torch.cuda.synchronize()
    return out[:g.n].cpu().numpy(), k, lib.sgr_last_stats()


@pytest.mark.parametrize("make", GRAPHS)
@pytest.mark.parametrize("rule", ["low_keeps", "low_loses", "degree"])
def test_topo_parity(gpu_lib, make, rule):
    g = make()
    ref = oracle.det_sgr(g, rule)
    got, k, st = run_device(gpu_lib, g, "topo+" + rule)
    assert np.array_equal(got, ref.colors), f"{g.name}: first diff at {np.argmax(got != ref.colors)}"
    assert k == ref.num_colors and st["rounds"] == ref.rounds
    assert st["sum_w"] == ref.sum_w and st["sum_d"] == ref.sum_d and st["sum_next"] == ref.sum_next


def test_topo_host_entry_and_same_as_worklist_mode(gpu_lib):
    g = gg.rmat(13, 16, seed=11)
    ref = oracle.det_sgr(g)
    colors = np.zeros(g.n, dtype=np.int32)
    k = gpu_lib.sgr_color_host(g.n, g.row_offsets, g.col_idx, colors, "topo")
    assert np.array_equal(colors, ref.colors) and k == ref.num_colors
    got, k2, _ = run_device(gpu_lib, g, "det")
    assert np.array_equal(got, colors) and k2 == k


def test_topo_refused_by_the_batched_entry_point(gpu_lib):
    import torch
    graphs = [gg.uniform(200, 4.0, seed=s) for s in range(3)]
    b = gg.pack(graphs)
    ro = torch.from_numpy(b.row_offsets).cuda()
    ci = torch.from_numpy(b.col_idx).cuda()
    out = torch.zeros(int(b.vtx_off[-1]), dtype=torch.int32, device="cuda")
    k = np.zeros(b.G, dtype=np.int32)
    with pytest.raises(gpu_lib.SgrError) as e:
        gpu_lib.sgr_color_batch(b.G, b.vtx_off, b.edge_off, ro, ci, out, k, "topo")
    assert e.value.status == gpu_lib.SGR_ERR_INVALID_ARG

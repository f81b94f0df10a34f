"""GPU parity of sgr_color_batch: many uneven graphs in one launch.

Coloring the disjoint union with per-graph id offsets must give every graph
exactly its own coloring (the loser rules only compare ids within a graph), so
in deterministic mode each graph of the batch must equal the oracle and
sgr_color on that graph alone, bit for bit; fast mode must give a valid
coloring per graph.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def run_batch(lib, batch, mode="det"):
    import torch
    ro = torch.from_numpy(batch.row_offsets).cuda()
    ci = torch.from_numpy(batch.col_idx).cuda() if batch.col_idx.size else torch.zeros(
        4, dtype=torch.int32, device="cuda")
    n = int(batch.vtx_off[-1])
    out = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    k = np.zeros(batch.G, dtype=np.int32)
    lib.sgr_color_batch(batch.G, batch.vtx_off, batch.edge_off, ro, ci, out, k, mode)
    torch.cuda.synchronize()
    colors = out[:n].cpu().numpy()
    return [colors[batch.vtx_off[i]:batch.vtx_off[i + 1]] for i in range(batch.G)], k


def small_mix(seed, count=24, n_lo=50, n_hi=6000):
    return [gg.mix_graph(s) for s in gg.mix_specs(count, n_lo, n_hi, seed)]


@pytest.fixture
def tuning(gpu_lib):
    saved = gpu_lib.sgr_get_tuning()
    yield gpu_lib
    gpu_lib.sgr_set_tuning(**saved)


@pytest.mark.parametrize("rule", ["low_keeps", "low_loses", "degree"])
def test_batch_det_equals_oracle_per_graph(gpu_lib, rule):
    graphs = small_mix(1)
    batch = gg.pack(graphs)
    got, k = run_batch(gpu_lib, batch, "det+" + rule)
    for i, g in enumerate(graphs):
        ref = oracle.det_sgr(g, rule)
        assert np.array_equal(got[i], ref.colors), f"graph {i} ({g.name})"
        assert k[i] == ref.num_colors


def test_batch_det_equals_single_graph_calls(gpu_lib):
    import torch
    graphs = small_mix(2, count=12, n_lo=500, n_hi=20000)
    got, k = run_batch(gpu_lib, gg.pack(graphs))
    for i, g in enumerate(graphs):
        ro = torch.from_numpy(g.row_offsets).cuda()
        ci = torch.from_numpy(g.col_idx).cuda()
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        kk = gpu_lib.sgr_color(g.n, ro, ci, out, "det")
        assert kk == k[i] and np.array_equal(out.cpu().numpy(), got[i])


def test_batch_with_empty_and_edgeless_graphs(gpu_lib):
    graphs = [gg.from_edges(0, []), gg.uniform(300, 5.0, seed=1), gg.from_edges(5, []),
              gg.from_edges(0, []), gg.stencil(7, 6, 1, 9), gg.from_edges(1, [])]
    got, k = run_batch(gpu_lib, gg.pack(graphs))
    for i, g in enumerate(graphs):
        ref = oracle.det_sgr(g)
        assert np.array_equal(got[i], ref.colors) and k[i] == ref.num_colors


@pytest.mark.parametrize("tune", [dict(light_max=4, chunk=64), dict(light_max=32, chunk=128),
                                  dict(light_max=1, chunk=2048, blocks_per_sm=1)])
def test_batch_det_across_bins(tuning, tune):
    tuning.sgr_set_tuning(**tune)
    graphs = small_mix(3, count=16, n_lo=100, n_hi=8000) + [gg.rmat(12, 16, seed=9)]
    got, k = run_batch(tuning, gg.pack(graphs))
    for i, g in enumerate(graphs):
        ref = oracle.det_sgr(g)
        assert np.array_equal(got[i], ref.colors) and k[i] == ref.num_colors


@pytest.mark.parametrize("policy", [1, 2])
def test_batch_det_active_list_policies(tuning, policy):
    tuning.sgr_set_tuning(active_lists=policy, light_max=8, chunk=128)
    graphs = small_mix(6, count=20, n_lo=100, n_hi=9000) + [gg.rmat(12, 16, seed=2)]
    got, k = run_batch(tuning, gg.pack(graphs))
    for i, g in enumerate(graphs):
        ref = oracle.det_sgr(g)
        assert np.array_equal(got[i], ref.colors) and k[i] == ref.num_colors


def test_batch_fast_valid(gpu_lib):
    graphs = small_mix(4)
    got, k = run_batch(gpu_lib, gg.pack(graphs), "fast")
    for i, g in enumerate(graphs):
        chk = oracle.check(g, got[i])
        assert chk["valid"] and chk["num_colors"] == k[i]


def test_batch_single_graph_and_zero_graphs(gpu_lib):
    g = gg.rmat(13, 16, seed=4)
    got, k = run_batch(gpu_lib, gg.pack([g]))
    ref = oracle.det_sgr(g)
    assert np.array_equal(got[0], ref.colors) and k[0] == ref.num_colors
    # G = 0 is a no-op
    assert gpu_lib._lib.sgr_color_batch(0, None, None, None, None, None, None, 0, None) == 0


def test_batch_rejects_bad_offsets(gpu_lib):
    import torch
    graphs = small_mix(5, count=3)
    b = gg.pack(graphs)
    ro = torch.from_numpy(b.row_offsets).cuda()
    ci = torch.from_numpy(b.col_idx).cuda()
    out = torch.empty(int(b.vtx_off[-1]), dtype=torch.int32, device="cuda")
    bad = b.vtx_off.copy()
    bad[1], bad[2] = bad[2], bad[1]  # not non-decreasing
    k = np.zeros(b.G, dtype=np.int32)
    with pytest.raises(gpu_lib.SgrError) as e:
        gpu_lib.sgr_color_batch(b.G, bad, b.edge_off, ro, ci, out, k, "det")
    assert e.value.status == gpu_lib.SGR_ERR_INVALID_GRAPH

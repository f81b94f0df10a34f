"""Full-size parity of the batched and served workloads against the oracle.

tests/golden/mix_digests.json holds, for every graph of the 512-graph batch
mix and for eight requests of the served mix (1.6k to 4M vertices), the
SHA-256 of the colors the CPU oracle's deterministic SGR (Algorithm 7 with
Algorithms 4 and 5, lower id keeps) gives that graph alone; it is written by
tests/golden/make_mix_golden.py, which calls only the oracle and the seeded
generators.  Here the GPU colors the same graphs

  * all 512 at once through sgr_color_batch (one persistent kernel over their
    disjoint union), and
  * the served set through the continuous-batching server, all submitted at
    once under a 64 GB budget (once with the large requests colored alone
    between the batched launches, once with every request in the batched
    rounds), and one at a time through sgr_color,

and every graph's colors must hash to the oracle's digest (bit-exact).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as gg

MIX = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mix_digests.json")))


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def graph_digest(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_offsets, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.col_idx, dtype="<i4").tobytes())
    return h.hexdigest()


def test_golden_file_covers_both_sets():
    assert len(MIX["batch512"]["graphs"]) == 512
    sizes = [r["n"] for r in MIX["serve_sizes"]["graphs"]]
    assert min(sizes) < 2000 and max(sizes) > 3_900_000
    assert {r["spec"][0] for r in MIX["serve_sizes"]["graphs"]} == {0, 1, 2, 3}


@pytest.mark.gpu
def test_batch512_full_size_equals_the_oracle_per_graph(gpu_lib):
    import torch
    b = gg.batch_mix(512, 1000, 200000, 0)
    recs = MIX["batch512"]["graphs"]
    assert b.G == len(recs)
    for g, rec in zip(b.graphs, recs):
        assert (g.n, g.m) == (rec["n"], rec["m"])
        assert graph_digest(g) == rec["graph_sha256"]
    ro = torch.from_numpy(b.row_offsets).cuda()
    ci = torch.from_numpy(b.col_idx).cuda()
    colors = torch.full((int(b.vtx_off[-1]),), -7, dtype=torch.int32, device="cuda")
    kk = np.zeros(b.G, dtype=np.int32)
    for _ in range(2):  # the second call runs on the arena the first one left
        gpu_lib.sgr_color_batch(b.G, b.vtx_off, b.edge_off, ro, ci, colors, kk, "det")
        got = colors.cpu().numpy()
        bad = [i for i, rec in enumerate(recs)
               if digest(got[b.vtx_off[i]:b.vtx_off[i + 1]]) != rec["det_colors_sha256"]
               or kk[i] != rec["det_num_colors"]]
        assert not bad, f"{len(bad)} graphs differ from the oracle, first {bad[:5]}"


def _serve_graphs():
    recs = MIX["serve_sizes"]["graphs"]
    graphs = [gg.mix_graph(tuple(r["spec"])) for r in recs]
    for g, rec in zip(graphs, recs):
        assert (g.n, g.m) == (rec["n"], rec["m"])
        assert graph_digest(g) == rec["graph_sha256"]
    return graphs, recs


@pytest.mark.gpu
@pytest.mark.parametrize("direct", [0, -1], ids=["large-alone", "all-batched"])
def test_server_sized_requests_equal_the_oracle_in_the_mix(gpu_lib, direct):
    graphs, recs = _serve_graphs()
    with gpu_lib.Server(hbm_budget_bytes=64 << 30, mode="det", direct_min_vertices=direct) as srv:
        ids = [srv.submit(g.row_offsets, g.col_idx) for g in graphs]  # all in flight together
        for rid, g, rec in zip(ids, graphs, recs):
            colors, k = srv.poll(rid, g.n, timeout_ms=600000)
            assert k == rec["det_num_colors"], rec["spec"]
            assert digest(colors) == rec["det_colors_sha256"], rec["spec"]
        st = srv.stats()
        assert st["completed"] == len(graphs) and st["failed"] == 0


@pytest.mark.gpu
def test_server_sized_requests_equal_the_oracle_alone(gpu_lib):
    import torch
    graphs, recs = _serve_graphs()
    for g, rec in zip(graphs, recs):
        ro = torch.from_numpy(g.row_offsets).cuda()
        ci = torch.from_numpy(g.col_idx).cuda()
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        k = gpu_lib.sgr_color(g.n, ro, ci, out, "det")
        assert k == rec["det_num_colors"], rec["spec"]
        assert gpu_lib.sgr_last_stats()["rounds"] == rec["det_rounds"], rec["spec"]
        assert digest(out.cpu().numpy()) == rec["det_colors_sha256"], rec["spec"]

"""The autotuner picks a candidate by measurement, installs it, caches it per
graph class, and the tuned coloring still equals the oracle."""
import json

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def test_autotune_installs_a_candidate_and_keeps_parity(gpu_lib, tmp_path):
    import torch
    from paper_1606_06025_gb300 import autotune
    saved = gpu_lib.sgr_get_tuning()
    try:
        g = gg.rmat(15, 16, seed=8)
        ro = torch.from_numpy(g.row_offsets).cuda()
        ci = torch.from_numpy(g.col_idx).cuda()
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        path = str(tmp_path / "tune.json")
        r1 = autotune.tune(ro, ci, out, int(g.degrees().max()), "det", path=path, budget_ms=500)
        t = r1["tuning"]
        assert r1["source"] == "measured" and r1["ms"] > 0
        assert t["light_max"] in (16, 32) and t["chunk"] in (256, 512, 1024, 2048)
        assert t["blocks_per_sm"] in (0, 2) and t["tail_vertices"] in (0, 1024, 2880)
        assert gpu_lib.sgr_get_tuning() == t
        assert oracle.check(g, out.cpu().numpy())["valid"]
        k = gpu_lib.sgr_color(g.n, ro, ci, out, "det")
        ref = oracle.det_sgr(g)
        assert np.array_equal(out.cpu().numpy(), ref.colors) and k == ref.num_colors
        r2 = autotune.tune(ro, ci, out, int(g.degrees().max()), "det", path=path)
        assert r2["source"] == "cache" and r2["tuning"] == t
        assert r1["key"] in json.load(open(path))
    finally:
        gpu_lib.sgr_set_tuning(**saved)


def test_batch_autotune_keeps_parity_per_graph(gpu_lib, tmp_path):
    """Every candidate of the batch tuner colors the batch; the installed one
    still gives every graph exactly the oracle's coloring."""
    import torch
    from paper_1606_06025_gb300 import autotune
    saved = gpu_lib.sgr_get_tuning()
    try:
        b = gg.batch_mix(24, 500, 30000, 5)
        ro = torch.from_numpy(b.row_offsets).cuda()
        ci = torch.from_numpy(b.col_idx).cuda()
        colors = torch.empty(int(b.vtx_off[-1]), dtype=torch.int32, device="cuda")
        kk = np.zeros(b.G, dtype=np.int32)
        path = str(tmp_path / "tune.json")
        r1 = autotune.tune_batch(b.G, b.vtx_off, b.edge_off, ro, ci, colors, kk, "det", path=path,
                                 budget_ms=300)
        assert r1["source"] == "measured" and r1["key"].startswith("batch:")
        assert gpu_lib.sgr_get_tuning() == r1["tuning"]
        gpu_lib.sgr_color_batch(b.G, b.vtx_off, b.edge_off, ro, ci, colors, kk, "det")
        got = colors.cpu().numpy()
        for i, g in enumerate(b.graphs):
            ref = oracle.det_sgr(g)
            assert np.array_equal(got[b.vtx_off[i]:b.vtx_off[i + 1]], ref.colors) and kk[i] == ref.num_colors
        r2 = autotune.tune_batch(b.G, b.vtx_off, b.edge_off, ro, ci, colors, kk, "det", path=path)
        assert r2["source"] == "cache" and r2["tuning"] == r1["tuning"]
    finally:
        gpu_lib.sgr_set_tuning(**saved)

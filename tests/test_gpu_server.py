"""GPU tests of the continuous-batching server (sgr_server_*).

Every result must equal sgr_color on the same graph (deterministic mode, bit
for bit) whether the graph ran alone or joined other graphs in flight, and
whatever the arrival order; a small HBM budget forces requests to wait for
admission until resident graphs retire.
"""
import random
import threading

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def mix(seed, count, n_lo=50, n_hi=20000):
    return [gg.mix_graph(s) for s in gg.mix_specs(count, n_lo, n_hi, seed)]


def test_server_results_equal_oracle(gpu_lib):
    graphs = mix(11, 20)
    with gpu_lib.Server(hbm_budget_bytes=256 << 20) as srv:
        ids = [srv.submit(g.row_offsets, g.col_idx) for g in graphs]
        for rid, g in zip(ids, graphs):
            colors, k = srv.poll(rid, g.n, timeout_ms=60000)
            ref = oracle.det_sgr(g)
            assert np.array_equal(colors, ref.colors) and k == ref.num_colors
        st = srv.stats()
        assert st["completed"] == len(graphs) and st["failed"] == 0
        assert st["p99_ms"] >= st["p50_ms"] > 0


def test_server_staggered_arrivals_and_small_budget(gpu_lib):
    """Requests arrive while others run; the budget holds only a few graphs at a
    time, so admission waits for retirements."""
    graphs = mix(12, 30, n_lo=2000, n_hi=40000)
    expect = [oracle.det_sgr(g).colors for g in graphs]
    rnd = random.Random(3)
    with gpu_lib.Server(hbm_budget_bytes=48 << 20, rounds_per_launch=2) as srv:
        cap = srv.stats()["vertex_capacity"]
        assert cap < sum(g.n for g in graphs)  # not everything fits at once
        done = {}
        order = list(range(len(graphs)))
        rnd.shuffle(order)
        live = []
        for i in order:
            live.append((i, srv.submit(graphs[i].row_offsets, graphs[i].col_idx)))
            if rnd.random() < 0.5 and live:  # collect one now and then
                j, rid = live.pop(0)
                done[j] = srv.poll(rid, graphs[j].n, timeout_ms=60000)
        for j, rid in live:
            done[j] = srv.poll(rid, graphs[j].n, timeout_ms=60000)
        for j, g in enumerate(graphs):
            colors, k = done[j]
            assert np.array_equal(colors, expect[j]), j
        st = srv.stats()
        assert st["completed"] == len(graphs) and st["launches"] > 1


def test_server_equals_sgr_color_and_rules(gpu_lib):
    import torch
    graphs = mix(13, 8, n_lo=500, n_hi=30000) + [gg.rmat(14, 16, seed=5)]
    for rule in ["low_keeps", "degree", "low_loses"]:
        with gpu_lib.Server(hbm_budget_bytes=512 << 20, mode="det+" + rule) as srv:
            ids = [srv.submit(g.row_offsets, g.col_idx) for g in graphs]
            for rid, g in zip(ids, graphs):
                colors, k = srv.poll(rid, g.n, timeout_ms=60000)
                ro = torch.from_numpy(g.row_offsets).cuda()
                ci = torch.from_numpy(g.col_idx).cuda()
                out = torch.empty(g.n, dtype=torch.int32, device="cuda")
                kk = gpu_lib.sgr_color(g.n, ro, ci, out, "det+" + rule)
                assert kk == k and np.array_equal(out.cpu().numpy(), colors)


def test_server_concurrent_submitters_and_unsorted_rows(gpu_lib):
    graphs = mix(14, 24, n_lo=100, n_hi=8000)
    rng = np.random.default_rng(0)
    shuffled = []
    for g in graphs[:6]:  # rows in random order: same coloring
        ci = g.col_idx.copy()
        for v in range(g.n):
            rng.shuffle(ci[g.row_offsets[v]:g.row_offsets[v + 1]])
        shuffled.append(gg.CSR(g.row_offsets, ci, g.name))
    graphs = shuffled + graphs[6:]
    results = {}
    with gpu_lib.Server(hbm_budget_bytes=128 << 20) as srv:
        def worker(idx):
            for i in idx:
                rid = srv.submit(graphs[i].row_offsets, graphs[i].col_idx)
                results[i] = srv.poll(rid, graphs[i].n, timeout_ms=60000)
        th = [threading.Thread(target=worker, args=(list(range(t, len(graphs), 4)),))
              for t in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
    for i, g in enumerate(graphs):
        ref = oracle.det_sgr(g)
        assert np.array_equal(results[i][0], ref.colors) and results[i][1] == ref.num_colors


def test_server_edge_cases(gpu_lib):
    with gpu_lib.Server(hbm_budget_bytes=32 << 20) as srv:
        rid = srv.submit(np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32))  # n = 0
        colors, k = srv.poll(rid, 0, timeout_ms=1000)
        assert colors.size == 0 and k == 0
        # unknown id
        import ctypes
        k = ctypes.c_int32(0)
        assert gpu_lib._lib.sgr_server_poll(srv._h, 987654321, None, ctypes.byref(k), 0) == \
            gpu_lib.SGR_ERR_NOT_FOUND
        # a self-loop entry is ignored: vertex 0 still gets color 1
        rid = srv.submit(np.array([0, 1, 1], dtype=np.int32), np.array([0], dtype=np.int32))
        colors, k = srv.poll(rid, 2, timeout_ms=10000)
        assert list(colors) == [1, 1] and k == 1
        # invalid graphs
        with pytest.raises(gpu_lib.SgrError) as e:
            srv.submit(np.array([0, 2, 1], dtype=np.int32), np.array([1, 0], dtype=np.int32))  # offsets
        assert e.value.status == gpu_lib.SGR_ERR_INVALID_GRAPH
        with pytest.raises(gpu_lib.SgrError) as e:
            srv.submit(np.array([0, 1, 2], dtype=np.int32), np.array([1, 5], dtype=np.int32))  # id 5 >= n
        assert e.value.status == gpu_lib.SGR_ERR_INVALID_GRAPH
        # larger than the whole server
        big = gg.uniform(400000, 4.0, seed=1)
        with pytest.raises(gpu_lib.SgrError) as e:
            srv.submit(big.row_offsets, big.col_idx)
        assert e.value.status == gpu_lib.SGR_ERR_OUT_OF_MEMORY
        # a normal request still works afterwards
        g = gg.uniform(1000, 6.0, seed=2)
        rid = srv.submit(g.row_offsets, g.col_idx)
        colors, k = srv.poll(rid, g.n, timeout_ms=60000)
        assert np.array_equal(colors, oracle.det_sgr(g).colors)
    with pytest.raises(gpu_lib.SgrError):
        gpu_lib.Server(hbm_budget_bytes=1 << 20)  # below the minimum
    with pytest.raises(gpu_lib.SgrError):
        gpu_lib.Server(mode="fast")  # deterministic mode only



def test_server_colors_large_requests_alone_between_batched_launches(gpu_lib):
    """Requests at or above direct_min_vertices run alone on the single-graph
    kernels (activation lists, one-CTA tail) between the batched launches of
    the small ones; every result still equals the oracle, whatever the mix."""
    graphs = mix(21, 18, n_lo=2000, n_hi=150000)
    expect = [oracle.det_sgr(g) for g in graphs]
    big = sum(g.n >= 40000 for g in graphs)
    assert 0 < big < len(graphs)
    with gpu_lib.Server(hbm_budget_bytes=512 << 20, rounds_per_launch=4, direct_min_vertices=40000) as srv:
        ids = [srv.submit(g.row_offsets, g.col_idx) for g in graphs]
        for rid, g, ref in zip(ids, graphs, expect):
            colors, k = srv.poll(rid, g.n, timeout_ms=60000)
            assert np.array_equal(colors, ref.colors) and k == ref.num_colors
        st = srv.stats()
        assert st["direct"] == big and st["completed"] == len(graphs)


def test_server_never_alone_when_disabled(gpu_lib):
    graphs = mix(22, 6, n_lo=100000, n_hi=200000)
    with gpu_lib.Server(hbm_budget_bytes=1 << 30, direct_min_vertices=-1) as srv:
        ids = [srv.submit(g.row_offsets, g.col_idx) for g in graphs]
        for rid, g in zip(ids, graphs):
            colors, k = srv.poll(rid, g.n, timeout_ms=60000)
            assert np.array_equal(colors, oracle.det_sgr(g).colors)
        assert srv.stats()["direct"] == 0

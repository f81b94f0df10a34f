"""GPU parity: libsgrcolor against the CPU oracle, through the C ABI.

Deterministic mode must equal the oracle's Algorithm 7 reading bit for bit:
the colors array, k, the round count and the per-round sums (|W_r|, degree
sums, pushed losers).  Fast mode (racy, in place) must give a valid coloring
with k <= max degree + 1.  Every code path of the kernel is forced at small
sizes by shrinking the degree bins (group-per-vertex, warp-per-vertex, and
hubs split into several warp work items).
"""
import hashlib
import json
import os
import random

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "configs.json")))


@pytest.fixture(scope="module")
def lib(gpu_lib):
    return gpu_lib


@pytest.fixture
def tuning(lib):
    saved = lib.sgr_get_tuning()
    yield lib
    lib.sgr_set_tuning(**saved)


def to_dev(g):
    import torch
    ro = torch.from_numpy(np.ascontiguousarray(g.row_offsets)).cuda()
    ci = torch.from_numpy(np.ascontiguousarray(g.col_idx)).cuda() if g.m else torch.zeros(
        4, dtype=torch.int32, device="cuda")
    return ro, ci


def run(lib, g, mode="det"):
    import torch
    ro, ci = to_dev(g)
    out = torch.full((max(g.n, 1),), -7, dtype=torch.int32, device="cuda")
    k = lib.sgr_color(g.n, ro, ci, out, mode)
    torch.cuda.synchronize()
    return out[:g.n].cpu().numpy(), k, lib.sgr_last_stats()


def assert_det_parity(lib, g, rule="low_keeps"):
    mode = "det+" + rule
    got, k, st = run(lib, g, mode)
    ref = oracle.det_sgr(g, rule)
    assert ref.status == 0
    assert np.array_equal(got, ref.colors), f"{g.name}: first diff at {np.argmax(got != ref.colors)}"
    assert k == ref.num_colors
    assert st["rounds"] == ref.rounds
    assert st["sum_w"] == ref.sum_w and st["sum_d"] == ref.sum_d
    assert st["sum_next"] == ref.sum_next
    return st


def complete(n):
    return gg.from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def star(n, center=0):
    return gg.from_edges(n, [(center, i) for i in range(n) if i != center])


def shuffled_rows(g, seed):
    """Same graph with every row in a random order (unsorted CSR)."""
    rng = np.random.default_rng(seed)
    ci = g.col_idx.copy()
    for v in range(g.n):
        a, b = g.row_offsets[v], g.row_offsets[v + 1]
        rng.shuffle(ci[a:b])
    return gg.CSR(g.row_offsets.copy(), ci, g.name + "_shuf")


SMALL = [
    lambda: gg.from_edges(1, []),
    lambda: gg.from_edges(7, []),
    lambda: complete(2),
    lambda: complete(40),
    lambda: star(300),
    lambda: star(300, center=299),
    lambda: gg.from_edges(5, [(0, 1), (1, 2), (2, 3), (3, 4)]),
    lambda: gg.stencil(17, 13, 1, 9),
    lambda: gg.stencil(9, 8, 7, 27),
    lambda: gg.uniform(3000, 10.0, seed=4),
    lambda: gg.uniform(20011, 7.0, seed=5),
    lambda: gg.rmat(12, 16, seed=6),
    lambda: gg.rmat(14, 16, seed=7),
]


@pytest.mark.parametrize("make", SMALL)
@pytest.mark.parametrize("rule", ["low_keeps", "low_loses", "degree"])
def test_det_parity_small(lib, make, rule):
    assert_det_parity(lib, make(), rule)


# Tunings that move vertices between the three bins and split hubs into many
# work items even on small graphs.
TUNINGS = [
    dict(light_max=32, chunk=4096),
    dict(light_max=8, chunk=64),
    dict(light_max=4, chunk=100),
    dict(light_max=1, chunk=64),
    dict(light_max=32, chunk=2048),
    dict(light_max=32, chunk=2048, blocks_per_sm=1),
]


@pytest.mark.parametrize("tune", TUNINGS)
def test_det_parity_across_bins(tuning, tune):
    tuning.sgr_set_tuning(**tune)
    for g in [gg.rmat(13, 16, seed=11), star(1000), complete(70), gg.stencil(10, 9, 8, 27),
              gg.uniform(5000, 20.0, seed=3)]:
        for rule in ["low_keeps", "degree"]:
            assert_det_parity(tuning, g, rule)


@pytest.mark.parametrize("rule", ["low_keeps", "low_loses", "degree"])
def test_det_parity_unsorted_rows(tuning, rule):
    tuning.sgr_set_tuning(light_max=16, chunk=128)
    for seed, g in enumerate([gg.rmat(12, 16, seed=2), gg.uniform(4000, 12.0, seed=9),
                              gg.stencil(8, 7, 6, 27)]):
        h = shuffled_rows(g, seed)
        st = assert_det_parity(tuning, h, rule)
        assert st["rows_sorted"] == 0
    st = assert_det_parity(tuning, gg.uniform(100, 4.0, seed=1), rule)
    assert st["rows_sorted"] == 1


# Deterministic rounds either run over the whole worklist or (active_lists)
# only over the vertices a commit made stale plus those whose witness they
# are; the automatic choice uses both on most inputs.  Forcing each one must
# give the oracle's result everywhere, including hubs split into work items,
# the fallback for full bitmaps, unsorted rows and every loser rule.
@pytest.mark.parametrize("policy", [1, 2])
@pytest.mark.parametrize("tune", [dict(), dict(light_max=4, chunk=64), dict(light_max=1, chunk=2048)])
def test_det_parity_active_lists(tuning, policy, tune):
    tuning.sgr_set_tuning(active_lists=policy, **tune)
    graphs = [gg.rmat(13, 16, seed=21), star(700), complete(300), gg.stencil(12, 11, 10, 27),
              gg.stencil(40, 37, 1, 9), gg.uniform(6000, 14.0, seed=8),
              shuffled_rows(gg.rmat(12, 16, seed=3), 1), gg.from_edges(9, [])]
    for g in graphs:
        for rule in ["low_keeps", "low_loses", "degree"]:
            assert_det_parity(tuning, g, rule)


def test_det_ragged_sizes_around_tiles(lib):
    # sizes straddling the 1024-vertex light tile and the 4-entry vector loads
    for n in [1, 2, 3, 31, 32, 33, 1023, 1024, 1025, 4097]:
        g = gg.uniform(n, 3.0, seed=n)
        assert_det_parity(lib, g)


def test_det_round_count_complete_graph(lib):
    g = complete(200)
    got, k, st = run(lib, g)
    assert k == 200 and st["rounds"] == 200
    assert list(got) == list(range(1, 201))


@pytest.mark.parametrize("make", SMALL)
def test_fast_mode_valid(lib, make):
    g = make()
    got, k, st = run(lib, g, "fast")
    chk = oracle.check(g, got)
    assert chk["valid"], chk
    assert k == chk["num_colors"]
    assert k <= int(g.degrees().max(initial=0)) + 1
    assert st["rounds"] <= g.n


@pytest.mark.parametrize("tune", TUNINGS)
def test_fast_mode_valid_across_bins(tuning, tune):
    tuning.sgr_set_tuning(**tune)
    for g in [gg.rmat(13, 16, seed=11), star(1000), complete(70), gg.stencil(10, 9, 8, 27)]:
        for rule in ["fast+low_keeps", "fast+low_loses", "fast+degree"]:
            got, k, _ = run(tuning, g, rule)
            assert oracle.check(g, got)["valid"]


def test_host_entry_matches_device_entry(lib):
    g = gg.rmat(13, 16, seed=5)
    dev, kd, _ = run(lib, g)
    out = np.zeros(g.n, dtype=np.int32)
    kh = lib.sgr_color_host(g.n, g.row_offsets, g.col_idx, out, "det")
    assert kh == kd and np.array_equal(out, dev)


def test_empty_graph(lib):
    import torch
    ro = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.sgr_color(0, ro, ro, ro, "det") == 0


def test_invalid_arguments(lib):
    import torch
    g = gg.uniform(100, 4.0, seed=0)
    ro, ci = to_dev(g)
    out = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(lib.SgrError) as e:
        lib.sgr_color(g.n, g.row_offsets, ci, out, "det")  # host pointer for row_offsets
    assert e.value.status == lib.SGR_ERR_INVALID_ARG
    big = torch.zeros(g.m + 4, dtype=torch.int32, device="cuda")
    big[1:g.m + 1] = ci
    with pytest.raises(lib.SgrError) as e:
        lib.sgr_color(g.n, ro, big.data_ptr() + 4, out, "det")  # col_idx not 16-byte aligned
    assert e.value.status == lib.SGR_ERR_INVALID_ARG
    bad = ro.clone()
    bad[0] = 1
    with pytest.raises(lib.SgrError) as e:
        lib.sgr_color(g.n, bad, ci, out, "det")
    assert e.value.status == lib.SGR_ERR_INVALID_GRAPH
    with pytest.raises(lib.SgrError):
        lib.sgr_color(g.n, ro, ci, out, 0x40)


def test_validate_csr(lib):
    import torch
    g = gg.rmat(12, 8, seed=1)
    ro, ci = to_dev(g)
    assert lib.sgr_validate_csr(g.n, ro, ci) == (0, 1)
    h = shuffled_rows(g, 3)
    ro2, ci2 = to_dev(h)
    assert lib.sgr_validate_csr(h.n, ro2, ci2) == (0, 0)
    # asymmetric: drop one direction of an edge by overwriting an entry
    bad = g.col_idx.copy()
    v = int(np.argmax(g.degrees() > 2))
    a = g.row_offsets[v]
    w_old = bad[a]
    cand = [u for u in range(g.n) if u != v and u not in set(bad[a:g.row_offsets[v + 1]])]
    bad[a] = cand[0]
    bad[a:g.row_offsets[v + 1]].sort()
    rc, _ = lib.sgr_validate_csr(g.n, ro, torch.from_numpy(bad).cuda())
    assert rc == lib.SGR_ERR_INVALID_GRAPH, w_old
    # self-loop
    loop = g.col_idx.copy()
    loop[a] = v
    rc, _ = lib.sgr_validate_csr(g.n, ro, torch.from_numpy(loop).cuda())
    assert rc == lib.SGR_ERR_INVALID_GRAPH
    # out of range id
    oor = g.col_idx.copy()
    oor[-1] = g.n
    rc, _ = lib.sgr_validate_csr(g.n, ro, torch.from_numpy(oor).cuda())
    assert rc == lib.SGR_ERR_INVALID_GRAPH


# ------------------------------------------------------------ full-size workloads

def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


FULL = {"er20k": lambda: gg.er20k(0), "rmat20": lambda: gg.rmat20(0),
        "stencil27_192": lambda: gg.stencil27(192)}


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_det_matches_oracle_digest(lib, name):
    """Bit-exact at the benchmark sizes, in the launch configuration bench.py
    times: the colors digest, k, rounds and sums equal those the oracle wrote
    into tests/golden/configs.json."""
    gold = GOLDEN[name]
    g = FULL[name]()
    assert g.n == gold["n"] and g.m == gold["m"]
    got, k, st = run(lib, g, "det")
    assert k == gold["det_num_colors"]
    assert st["rounds"] == gold["det_rounds"]
    assert st["sum_w"] == gold["det_sum_w"] and st["sum_d"] == gold["det_sum_d"]
    assert st["sum_next"] == gold["det_sum_next"]
    assert digest(got) == gold["det_colors_sha256"]


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_fast_valid(lib, name):
    g = FULL[name]()
    got, k, st = run(lib, g, "fast")
    chk = oracle.check(g, got)
    assert chk["valid"] and chk["num_colors"] == k
    assert k <= GOLDEN[name]["max_degree"] + 1


@pytest.mark.parametrize("policy", [1, 2])
@pytest.mark.parametrize("name", list(FULL))
def test_full_size_det_active_list_policies(tuning, policy, name):
    """The full-size digests again with the round mode forced each way."""
    tuning.sgr_set_tuning(active_lists=policy)
    gold = GOLDEN[name]
    g = FULL[name]()
    got, k, st = run(tuning, g, "det")
    assert k == gold["det_num_colors"] and st["rounds"] == gold["det_rounds"]
    assert st["sum_w"] == gold["det_sum_w"] and st["sum_d"] == gold["det_sum_d"]
    assert st["sum_next"] == gold["det_sum_next"]
    assert digest(got) == gold["det_colors_sha256"]


def test_host_entry_large_upload_matches_device_entry(lib):
    # col_idx of 38 MB through the host entry, twice in a row (the second
    # upload reuses the library's device buffers of the first call)
    g = gg.uniform(600_000, 16.0, seed=12)
    assert g.m * 4 > (16 << 20)
    dev, kd, _ = run(lib, g)
    out = np.zeros(g.n, dtype=np.int32)
    for _ in range(2):
        kh = lib.sgr_color_host(g.n, g.row_offsets, g.col_idx, out, "det")
        assert kh == kd and np.array_equal(out, dev)

"""GPU tests of the failure paths: bounded device waits, allocation failures,
the round cap on input that breaks the contract, and the server's own cap.

Every failure is made on the host (no GPU fault, trap or endless loop):
  * a grid barrier is made to run out by launching the round kernel with a
    barrier count one CTA larger than its grid (sgr_debug_inject) under a
    short wait limit (sgr_set_wait_limit): every CTA leaves at its next
    barrier and the call returns SGR_ERR_TIMEOUT;
  * a device allocation is made to fail on the host before cudaMalloc is
    called (sgr_debug_inject): the call returns SGR_ERR_OUT_OF_MEMORY;
  * a non-symmetric CSR (vertex 1 lists 0, vertex 0 lists nothing) never lets
    vertex 1 keep a color: Algorithm 7's loop would not end, and the round cap
    of n + 1 (the bound that holds for every symmetric graph, since the
    highest-priority worklist vertex always keeps its color) ends it.
After each failure the next normal call must equal the oracle, and host
out-parameters must be left untouched.
"""
import ctypes
import time

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _dev(g):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(g.row_offsets)).cuda(),
            torch.from_numpy(np.ascontiguousarray(g.col_idx)).cuda())


def _raw_color(lib, fn, n, ro, ci, mode="det"):
    """Call an entry point through the C ABI; returns (status, colors, k)."""
    import torch
    out = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    k = ctypes.c_int32(-7)
    rc = getattr(lib._lib, fn)(n, ro.data_ptr(), ci.data_ptr(), out.data_ptr(), ctypes.byref(k),
                               lib._mode(mode), lib._stream(None))
    torch.cuda.synchronize()
    return rc, out[:n].cpu().numpy(), k.value


@pytest.fixture
def clean(gpu_lib):
    yield gpu_lib
    gpu_lib.sgr_debug_inject(gpu_lib.SGR_INJECT_NONE)
    gpu_lib.sgr_set_wait_limit(0)


def test_grid_barrier_timeout_is_reported_and_the_device_stays_usable(clean):
    lib = clean
    g = gg.rmat(14, 16, seed=5)
    ro, ci = _dev(g)
    ref = oracle.det_sgr(g)
    lib.sgr_set_wait_limit(5_000_000)  # 5 ms
    lib.sgr_debug_inject(lib.SGR_INJECT_BARRIER, 1)
    t0 = time.time()
    rc, _, k = _raw_color(lib, "sgr_color", g.n, ro, ci)
    assert rc == lib.SGR_ERR_TIMEOUT
    assert k == -7  # host out-parameter untouched on error
    assert time.time() - t0 < 10.0
    lib.sgr_set_wait_limit(0)
    for _ in range(2):  # the injection was one-shot; the next calls are normal
        rc, got, k = _raw_color(lib, "sgr_color", g.n, ro, ci)
        assert rc == 0 and k == ref.num_colors and np.array_equal(got, ref.colors)


def test_barrier_timeout_through_the_batch_and_no_alloc_entries(clean):
    lib = clean
    graphs = [gg.uniform(3000, 8.0, seed=s) for s in range(3)]
    b = gg.pack(graphs)
    import torch
    ro = torch.from_numpy(b.row_offsets).cuda()
    ci = torch.from_numpy(b.col_idx).cuda()
    colors = torch.empty(int(b.vtx_off[-1]), dtype=torch.int32, device="cuda")
    kk = np.full(b.G, -7, dtype=np.int32)
    lib.sgr_set_wait_limit(5_000_000)
    lib.sgr_debug_inject(lib.SGR_INJECT_BARRIER, 1)
    rc = lib._lib.sgr_color_batch(b.G, b.vtx_off.ctypes.data, b.edge_off.ctypes.data, ro.data_ptr(),
                                  ci.data_ptr(), colors.data_ptr(), kk.ctypes.data, 0, None)
    assert rc == lib.SGR_ERR_TIMEOUT and (kk == -7).all()
    lib.sgr_debug_inject(lib.SGR_INJECT_BARRIER, 1)
    g = graphs[0]
    gro, gci = _dev(g)
    rc, _, k = _raw_color(lib, "sgr_color_noalloc", g.n, gro, gci)
    assert rc == lib.SGR_ERR_TIMEOUT and k == -7
    lib.sgr_set_wait_limit(0)
    lib.sgr_color_batch(b.G, b.vtx_off, b.edge_off, ro, ci, colors, kk)
    got = colors.cpu().numpy()
    for i, h in enumerate(graphs):
        ref = oracle.det_sgr(h)
        assert np.array_equal(got[b.vtx_off[i]:b.vtx_off[i + 1]], ref.colors)
        assert kk[i] == ref.num_colors


def test_allocation_failure_is_reported_and_the_next_call_succeeds(clean):
    lib = clean
    g = gg.uniform(20000, 10.0, seed=4)
    ro, ci = _dev(g)
    ref = oracle.det_sgr(g)
    lib.sgr_release_scratch()  # the next call must allocate its scratch arena
    lib.sgr_debug_inject(lib.SGR_INJECT_FAIL_ALLOC, 1)
    rc, _, k = _raw_color(lib, "sgr_color", g.n, ro, ci)
    assert rc == lib.SGR_ERR_OUT_OF_MEMORY and k == -7
    rc, got, k = _raw_color(lib, "sgr_color", g.n, ro, ci)
    assert rc == 0 and k == ref.num_colors and np.array_equal(got, ref.colors)
    # the host-buffer entry: its device copies are the first allocation
    lib.sgr_release_scratch()
    lib.sgr_debug_inject(lib.SGR_INJECT_FAIL_ALLOC, 1)
    out = np.full(g.n, -7, dtype=np.int32)
    kh = ctypes.c_int32(-7)
    rc = lib._lib.sgr_color_host(g.n, g.row_offsets.ctypes.data, g.col_idx.ctypes.data, out.ctypes.data,
                                 ctypes.byref(kh), 0, None)
    assert rc == lib.SGR_ERR_OUT_OF_MEMORY and kh.value == -7 and (out == -7).all()
    # the second allocation (the scratch arena behind the copies) fails too
    lib.sgr_release_scratch()
    lib.sgr_debug_inject(lib.SGR_INJECT_FAIL_ALLOC, 2)
    rc = lib._lib.sgr_color_host(g.n, g.row_offsets.ctypes.data, g.col_idx.ctypes.data, out.ctypes.data,
                                 ctypes.byref(kh), 0, None)
    assert rc == lib.SGR_ERR_OUT_OF_MEMORY and kh.value == -7
    assert lib.sgr_color_host(g.n, g.row_offsets, g.col_idx, out) == ref.num_colors
    assert np.array_equal(out, ref.colors)


def test_server_creation_reports_allocation_failure(clean):
    lib = clean
    lib.sgr_debug_inject(lib.SGR_INJECT_FAIL_ALLOC, 1)
    with pytest.raises(lib.SgrError) as ei:
        lib.Server(hbm_budget_bytes=64 << 20)
    assert ei.value.status == lib.SGR_ERR_OUT_OF_MEMORY
    g = gg.uniform(2000, 6.0, seed=8)
    with lib.Server(hbm_budget_bytes=64 << 20) as srv:
        colors, k = srv.poll(srv.submit(g.row_offsets, g.col_idx), g.n, timeout_ms=60000)
    assert np.array_equal(colors, oracle.det_sgr(g).colors)


def _one_sided():
    """Vertex 1 lists vertex 0; vertex 0 lists nothing (not symmetric)."""
    return gg.CSR(np.array([0, 0, 1], dtype=np.int32), np.array([0], dtype=np.int32), "one-sided")


def test_round_cap_ends_a_non_symmetric_graph(clean):
    lib = clean
    import torch
    g = _one_sided()
    ro = torch.from_numpy(g.row_offsets).cuda()
    ci = torch.from_numpy(np.array([0, 0, 0, 0], dtype=np.int32)).cuda()  # 16-byte padded
    t = lib.sgr_get_tuning()
    try:
        lib.sgr_set_tuning(**{**t, "tail_vertices": -1})
        rc, _, k = _raw_color(lib, "sgr_color", 2, ro, ci)
        assert rc == lib.SGR_ERR_NO_CONVERGENCE and k == -7
        assert lib.sgr_last_stats()["rounds"] == 3  # the cap: n + 1 rounds ran
    finally:
        lib.sgr_set_tuning(**t)
    # with the default tail the call ends too; the coloring is unspecified
    rc, _, _ = _raw_color(lib, "sgr_color", 2, ro, ci)
    assert rc in (0, lib.SGR_ERR_NO_CONVERGENCE)
    # a normal graph afterwards equals the oracle
    h = gg.uniform(5000, 10.0, seed=2)
    hro, hci = _dev(h)
    rc, got, k = _raw_color(lib, "sgr_color", h.n, hro, hci)
    assert rc == 0 and np.array_equal(got, oracle.det_sgr(h).colors)


def test_server_retires_a_non_symmetric_graph_at_its_round_cap(clean):
    lib = clean
    g = _one_sided()
    h = gg.rmat(12, 16, seed=6)
    ref = oracle.det_sgr(h)
    with lib.Server(hbm_budget_bytes=64 << 20, rounds_per_launch=4) as srv:
        bad = srv.submit(g.row_offsets, g.col_idx)
        good = srv.submit(h.row_offsets, h.col_idx)  # in flight at the same time
        with pytest.raises(lib.SgrError) as ei:
            srv.poll(bad, 2, timeout_ms=20000)
        assert ei.value.status == lib.SGR_ERR_NO_CONVERGENCE
        colors, k = srv.poll(good, h.n, timeout_ms=60000)
        assert np.array_equal(colors, ref.colors) and k == ref.num_colors
        later = srv.submit(h.row_offsets, h.col_idx)  # reuses the freed slot
        colors, k = srv.poll(later, h.n, timeout_ms=60000)
        assert np.array_equal(colors, ref.colors) and k == ref.num_colors
        st = srv.stats()
        assert st["failed"] == 1 and st["completed"] == 2 and st["resident"] == 0

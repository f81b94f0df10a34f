"""The allocation-free entry point, sgr_color_noalloc, through the C ABI.

Some callers must not let this library allocate device memory (an
application that owns every allocation through its own pool, or a loop that
cannot afford the device synchronisation a cudaMalloc / cudaFree brings).
sgr_color_noalloc serves them from a fixed scratch array in the library's
device image.  Its results must equal sgr_color's: bit for bit in
deterministic mode, on two calls in a row (the array keeps the previous
call's contents, so the second call checks that everything that must start at
zero is cleared).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _dev(g):
    import torch
    ro = torch.from_numpy(np.ascontiguousarray(g.row_offsets)).cuda()
    ci = torch.from_numpy(np.ascontiguousarray(g.col_idx)).cuda()
    return ro, ci


def _call(lib, fn, g, ro, ci, mode):
    import torch
    out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
    k = ctypes.c_int32(-1)
    rc = getattr(lib._lib, fn)(g.n, ro.data_ptr(), ci.data_ptr(), out.data_ptr(), ctypes.byref(k),
                               lib._mode(mode), lib._stream(None))
    torch.cuda.synchronize()
    return rc, out.cpu().numpy(), k.value


GRAPHS = [lambda: gg.rmat(14, 16, seed=3), lambda: gg.er20k(0),
          lambda: gg.stencil(24, 24, 24, 27), lambda: gg.uniform(3000, 40.0, seed=9)]


@pytest.mark.parametrize("make", GRAPHS)
def test_noalloc_equals_sgr_color_twice_in_a_row(gpu_lib, make):
    g = make()
    ro, ci = _dev(g)
    rc, ref, kref = _call(gpu_lib, "sgr_color", g, ro, ci, "det")
    assert rc == 0
    for _ in range(2):
        rc, got, k = _call(gpu_lib, "sgr_color_noalloc", g, ro, ci, "det")
        assert rc == 0
        assert k == kref and np.array_equal(got, ref)
    # fast mode may differ run to run; it must stay a valid coloring
    for _ in range(2):
        rc, got, k = _call(gpu_lib, "sgr_color_noalloc", g, ro, ci, "fast")
        assert rc == 0
        chk = oracle.check(g, got)
        assert chk["valid"] and chk["num_colors"] == k


def test_noalloc_refuses_graphs_beyond_its_scratch(gpu_lib):
    g = gg.rmat(20, 4, seed=1)  # about a million vertices: more scratch than the array holds
    ro, ci = _dev(g)
    rc, _, _ = _call(gpu_lib, "sgr_color_noalloc", g, ro, ci, "det")
    assert rc == gpu_lib.SGR_ERR_INVALID_ARG
    h = gg.uniform(500, 6.0, seed=2)  # a call that fits still works afterwards
    ro, ci = _dev(h)
    rc, got, k = _call(gpu_lib, "sgr_color_noalloc", h, ro, ci, "det")
    assert rc == 0 and np.array_equal(got, oracle.det_sgr(h).colors)


def test_noalloc_allocates_no_device_memory(gpu_lib):
    """The entry point's defining property: with the library's own scratch
    released, repeated calls leave the device's free memory unchanged (the
    fixed array is part of the loaded image, counted before the first call's
    measurement)."""
    import torch
    g = gg.rmat(14, 16, seed=4)
    ro, ci = _dev(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    ref = oracle.det_sgr(g)
    gpu_lib.sgr_release_scratch()
    k = gpu_lib.sgr_color_noalloc(g.n, ro, ci, out, "det")  # first call: looks up the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        k = gpu_lib.sgr_color_noalloc(g.n, ro, ci, out, "det")
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert gpu_lib.sgr_last_stats()["device_ms"] == 0.0
    assert k == ref.num_colors and np.array_equal(out.cpu().numpy(), ref.colors)
    # the timeline of the last call is that of this call
    tl = gpu_lib.sgr_last_trace()
    assert len(tl["w"]) == gpu_lib.sgr_last_stats()["rounds"] > 0


def test_noalloc_refuses_the_topology_driven_mode(gpu_lib):
    g = gg.uniform(500, 6.0, seed=2)
    ro, ci = _dev(g)
    rc, _, _ = _call(gpu_lib, "sgr_color_noalloc", g, ro, ci, "topo")
    assert rc == gpu_lib.SGR_ERR_INVALID_ARG


def test_noalloc_and_sgr_color_concurrently_on_one_device(gpu_lib):
    """Two host threads color at the same time, one through sgr_color and one
    through sgr_color_noalloc, each on its own stream.  The library serialises
    their cooperative launches on the device; both results equal the oracle."""
    import threading

    import torch
    ga, gb = gg.rmat(15, 16, seed=8), gg.uniform(30000, 12.0, seed=9)
    ra, rb = oracle.det_sgr(ga), oracle.det_sgr(gb)
    da, db = _dev(ga), _dev(gb)
    errors = []

    def worker(fn, g, d, ref):
        try:
            s = torch.cuda.Stream()
            out = torch.empty(g.n, dtype=torch.int32, device="cuda")
            for _ in range(6):
                k = fn(g.n, d[0], d[1], out, "det", s)
                s.synchronize()
                if k != ref.num_colors or not np.array_equal(out.cpu().numpy(), ref.colors):
                    errors.append(fn.__name__)
        except Exception as e:  # reported below
            errors.append(repr(e))

    ta = threading.Thread(target=worker, args=(gpu_lib.sgr_color, ga, da, ra))
    tb = threading.Thread(target=worker, args=(gpu_lib.sgr_color_noalloc, gb, db, rb))
    ta.start()
    tb.start()
    ta.join()
    tb.join()
    assert not errors, errors

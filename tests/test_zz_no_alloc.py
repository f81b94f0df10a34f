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

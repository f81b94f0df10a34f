"""Generator tests: the inputs are what they claim to be (CPU only)."""
import numpy as np
import pytest

import graphgen as gg


def _edges(g):
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    return src, g.col_idx.astype(np.int64)


def assert_simple_symmetric(g):
    ro, ci = g.row_offsets, g.col_idx
    assert ro[0] == 0 and ro[-1] == g.m
    assert np.all(np.diff(ro.astype(np.int64)) >= 0)
    if g.m == 0:
        return
    assert ci.min() >= 0 and ci.max() < g.n
    src, dst = _edges(g)
    assert not np.any(src == dst), "self-loop"
    # rows strictly increasing => sorted and duplicate-free
    same_row = src[1:] == src[:-1]
    assert np.all(ci[1:][same_row] > ci[:-1][same_row])
    fwd = np.sort(src * g.n + dst)
    bwd = np.sort(dst * g.n + src)
    assert np.array_equal(fwd, bwd), "not symmetric"


def test_splitmix64_published_outputs():
    # splitmix64 with state 0: first three outputs as published with the algorithm
    M = (1 << 64) - 1
    x = 0
    outs = []
    for _ in range(3):
        x = (x + 0x9E3779B97F4A7C15) & M
        outs.append(x)
    # the C code seeds xoshiro256** with four splitmix64 outputs; re-derive them
    # from the published constants and compare with the published values
    assert [hex(_sm(o)) for o in outs] == ["0xe220a8397b1dcdaf", "0x6e789e6aa1b965f4",
                                            "0x6c45d188009454f"]


def _sm(z):
    M = (1 << 64) - 1
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_xoshiro_stream_matches_definition():
    M = (1 << 64) - 1
    x, s = 12345, []
    for _ in range(4):
        x = (x + 0x9E3779B97F4A7C15) & M
        s.append(_sm(x))
    rotl = lambda v, k: ((v << k) | (v >> (64 - k))) & M
    ref = []
    for _ in range(8):
        ref.append((rotl((s[1] * 5) & M, 7) * 9) & M)
        t = (s[1] << 17) & M
        s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3]; s[2] ^= t
        s[3] = rotl(s[3], 45)
    assert [int(v) for v in gg.rng_stream(12345, 8)] == ref


@pytest.mark.parametrize("dims,points", [((5, 4, 1), 5), ((5, 4, 1), 9), ((4, 3, 5), 7),
                                         ((4, 3, 5), 27), ((1, 1, 1), 27), ((7, 1, 1), 9)])
def test_stencil_counts_and_shape(dims, points):
    g = gg.stencil(*dims, points=points)
    assert_simple_symmetric(g)
    nx, ny, nz = dims
    # brute-force count of lattice neighbours
    offs = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nnz = (dx != 0) + (dy != 0) + (dz != 0)
                if nnz == 0:
                    continue
                ok = {27: True, 9: dz == 0, 7: nnz == 1, 5: dz == 0 and nnz == 1}[points]
                if ok:
                    offs.append((dx, dy, dz))
    m = 0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for dx, dy, dz in offs:
                    if 0 <= x + dx < nx and 0 <= y + dy < ny and 0 <= z + dz < nz:
                        m += 1
    assert g.m == m and g.n == nx * ny * nz


def test_stencil_192_closed_form_edge_count():
    # 27-point stencil on s^3: pairs along 1, 2 and 3 axes, counted both ways
    s = 192
    m = 2 * (3 * (s - 1) * s * s + 6 * (s - 1) ** 2 * s + 4 * (s - 1) ** 3)
    assert m == 182041336
    nx = ny = nz = 6
    g = gg.stencil(nx, ny, nz, 27)
    t = 6
    assert g.m == 2 * (3 * (t - 1) * t * t + 6 * (t - 1) ** 2 * t + 4 * (t - 1) ** 3)


def test_uniform_graph_properties_and_seeds():
    a = gg.uniform(3000, 10.0, seed=7)
    b = gg.uniform(3000, 10.0, seed=7)
    c = gg.uniform(3000, 10.0, seed=8)
    assert_simple_symmetric(a)
    assert np.array_equal(a.col_idx, b.col_idx) and np.array_equal(a.row_offsets, b.row_offsets)
    assert not np.array_equal(a.row_offsets, c.row_offsets)
    # 15,000 pairs; self-loops and duplicates are rare, so about 30,000 entries
    assert 29500 < a.m <= 30000


def test_rmat_properties():
    g = gg.rmat(14, 16, (0.57, 0.19, 0.19), seed=3)
    assert_simple_symmetric(g)
    d = g.degrees()
    assert g.n == 1 << 14
    # skewed: max degree far above the mean (power-law shape)
    assert d.max() > 20 * d.mean()
    h = gg.rmat(14, 16, (0.57, 0.19, 0.19), seed=3, n=10000)
    assert_simple_symmetric(h)
    assert h.n == 10000 and h.m > 10000 * 8


def test_er20k_shape():
    g = gg.er20k()
    assert_simple_symmetric(g)
    assert g.n == 20000 and 199000 < g.m <= 200000


def test_from_edges_and_pack():
    g = gg.from_edges(4, [(0, 1), (1, 0), (2, 3), (1, 1)])
    assert_simple_symmetric(g)
    assert g.m == 4
    e = gg.from_edges(0, [])
    assert e.n == 0 and e.m == 0
    b = gg.pack([g, gg.stencil(3, 3, 1, 9), e, gg.from_edges(2, [])])
    assert b.G == 4
    assert list(b.vtx_off) == [0, 4, 13, 13, 15]
    assert b.row_offsets.shape[0] == 15 + 4
    for i, h in enumerate(b.graphs):
        s = int(b.vtx_off[i]) + i
        assert np.array_equal(b.row_offsets[s:s + h.n + 1], h.row_offsets)
        assert np.array_equal(b.col_idx[b.edge_off[i]:b.edge_off[i + 1]], h.col_idx)


def test_mix_specs_cover_all_kinds():
    specs = gg.mix_specs(24, 1000, 200000, seed=0)
    kinds = [s[0] for s in specs]
    assert set(kinds) == {0, 1, 2, 3}
    ns = [s[1] for s in specs]
    assert min(ns) >= 1000 and max(ns) <= 200000
    assert gg.mix_specs(24, 1000, 200000, seed=0) == specs

"""Seeded synthetic graph generators (inputs only, no coloring arithmetic).

Both sides of every parity check -- the CPU oracle under ``oracle/`` and the
GPU library -- take their inputs from here.  The C source ``graphgen.c`` is
compiled on first use with the host C compiler; it holds the pseudo-random
number generator (splitmix64 seeding xoshiro256**) and the R-MAT, uniform and
lattice-stencil builders.  Shapes follow the paper's evaluation (Sect. 4,
Table 1): R-MAT graphs, uniform "rmat-er" graphs and regular meshes.

Every graph is returned as a :class:`CSR` of int32 ``row_offsets`` (n+1) and
int32 ``col_idx`` (m), symmetric, without self-loops or duplicate entries, and
with every row sorted ascending.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``graphgen.c`` into ``_build/libgraphgen.so`` (host code only)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    vp, i32, i64, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                              ctypes.c_uint64, ctypes.c_double)
    lib.gg_uniform.restype = vp
    lib.gg_uniform.argtypes = [i32, i64, u64]
    lib.gg_rmat.restype = vp
    lib.gg_rmat.argtypes = [i32, i32, i64, dbl, dbl, dbl, u64]
    lib.gg_stencil.restype = vp
    lib.gg_stencil.argtypes = [i32, i32, i32, i32]
    lib.gg_from_edges.restype = vp
    lib.gg_from_edges.argtypes = [i32, i64, vp, vp]
    lib.gg_n.restype = i32
    lib.gg_n.argtypes = [vp]
    lib.gg_m.restype = i64
    lib.gg_m.argtypes = [vp]
    lib.gg_export.restype = ctypes.c_int
    lib.gg_export.argtypes = [vp, vp, vp]
    lib.gg_free.restype = None
    lib.gg_free.argtypes = [vp]
    lib.gg_rng_stream.restype = ctypes.c_int
    lib.gg_rng_stream.argtypes = [u64, i64, vp]
    _lib = lib
    return lib


@dataclass
class CSR:
    """A symmetric int32 CSR graph; ``name`` records how it was made."""
    row_offsets: np.ndarray
    col_idx: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.row_offsets.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.col_idx.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_offsets.astype(np.int64))


def _take(h, name: str, **meta) -> CSR:
    lib = _load()
    if not h:
        raise MemoryError(f"graph generator failed for {name}")
    try:
        n = lib.gg_n(h)
        m = lib.gg_m(h)
        ro = np.empty(n + 1, dtype=np.int32)
        ci = np.empty(max(m, 0), dtype=np.int32)
        lib.gg_export(h, ro.ctypes.data, ci.ctypes.data if m else None)
    finally:
        lib.gg_free(h)
    return CSR(ro, ci, name, dict(meta))


def rng_stream(seed: int, count: int) -> np.ndarray:
    """First ``count`` 64-bit outputs of xoshiro256** seeded via splitmix64."""
    out = np.empty(count, dtype=np.uint64)
    _load().gg_rng_stream(seed, count, out.ctypes.data)
    return out


def rng_uniform01(seed: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1) from the top 53 bits of the stream."""
    return (rng_stream(seed, count) >> np.uint64(11)).astype(np.float64) / 9007199254740992.0


# ------------------------------------------------------------------ builders

def uniform(n: int, avg_degree: float, seed: int = 0) -> CSR:
    """Uniform random graph: n*avg_degree/2 endpoint pairs drawn uniformly,
    symmetrised, self-loops and duplicates removed."""
    pairs = int(round(n * avg_degree / 2.0))
    return _take(_load().gg_uniform(n, pairs, seed), f"er_n{n}_d{avg_degree:g}_s{seed}",
                 kind="er", avg_degree=avg_degree, seed=seed)


def rmat(scale: int, edge_factor: int = 16, abc=(0.57, 0.19, 0.19), seed: int = 0,
         n: int | None = None) -> CSR:
    """R-MAT graph with edge_factor * n draws on ids [0, n), n = 2^scale by
    default; an edge with an endpoint >= n is drawn again.  Ids are permuted
    by the seed."""
    N = 1 << scale
    if n is None:
        n = N
    draws = edge_factor * n
    a, b, c = abc
    return _take(_load().gg_rmat(scale, n, draws, a, b, c, seed),
                 f"rmat_s{scale}_n{n}_ef{edge_factor}_s{seed}",
                 kind="rmat", scale=scale, edge_factor=edge_factor, abc=tuple(abc), seed=seed)


def stencil(nx: int, ny: int, nz: int = 1, points: int = 27) -> CSR:
    """Lattice stencil graph in natural lexicographic order.  ``points`` is 5
    or 9 (2-D, nz = 1) or 7 or 27 (3-D)."""
    return _take(_load().gg_stencil(nx, ny, nz, points), f"stencil{points}_{nx}x{ny}x{nz}",
                 kind="stencil", dims=(nx, ny, nz), points=points)


def from_edges(n: int, edges) -> CSR:
    """Symmetric CSR from an iterable of undirected (u, v) pairs."""
    e = np.asarray(list(edges), dtype=np.int32).reshape(-1, 2)
    u = np.ascontiguousarray(e[:, 0])
    v = np.ascontiguousarray(e[:, 1])
    h = _load().gg_from_edges(n, e.shape[0], u.ctypes.data if len(u) else None,
                              v.ctypes.data if len(v) else None)
    return _take(h, f"edges_n{n}", kind="edges")


# ------------------------------------------------------- named workloads

def er20k(seed: int = 0) -> CSR:
    """Uniform random graph, n = 20,000, average degree 10."""
    g = uniform(20000, 10.0, seed)
    g.name = f"er20k_s{seed}"
    return g


def rmat20(seed: int = 0) -> CSR:
    """R-MAT scale 20, edge factor 16, (a,b,c,d) = (0.57,0.19,0.19,0.05)."""
    g = rmat(20, 16, (0.57, 0.19, 0.19), seed)
    g.name = f"rmat20_s{seed}"
    return g


def stencil27(side: int = 192) -> CSR:
    """3-D 27-point stencil on side^3 points, natural order."""
    g = stencil(side, side, side, 27)
    g.name = f"stencil27_{side}"
    return g


def _mixed_graph(kind: int, n: int, u: float, seed: int) -> CSR:
    """One graph of the batch/serve mix.  kind 0 = uniform (average degree
    4 + 28u), 1 = R-MAT (edge factor 16), 2 = 2-D 9-point, 3 = 3-D 27-point."""
    if kind == 0:
        d = 4.0 + 28.0 * u
        return uniform(n, d, seed)
    if kind == 1:
        scale = max(1, int(math.ceil(math.log2(n))))
        return rmat(scale, 16, (0.57, 0.19, 0.19), seed, n=n)
    if kind == 2:
        nx = max(1, int(round(math.sqrt(n))))
        ny = max(1, int(round(n / nx)))
        return stencil(nx, ny, 1, 9)
    a = max(1, int(round(n ** (1.0 / 3.0))))
    nz = max(1, int(round(n / (a * a))))
    return stencil(a, a, nz, 27)


def mix_specs(count: int, n_lo: int, n_hi: int, seed: int):
    """Seeded (kind, n, u, graph_seed) specs: sizes log-uniform in [n_lo, n_hi],
    kinds cycling uniform / R-MAT / stencil, stencils alternating 2-D 9-point and
    3-D 27-point."""
    r = rng_uniform01(seed ^ 0x5EED0F5EED, 2 * count)
    specs = []
    lo, hi = math.log(n_lo), math.log(n_hi)
    for i in range(count):
        n = int(round(math.exp(lo + r[2 * i] * (hi - lo))))
        cls = i % 3
        kind = cls if cls < 2 else (2 if (i // 3) % 2 == 0 else 3)
        specs.append((kind, n, float(r[2 * i + 1]), (seed * 1000003 + i) & 0xFFFFFFFFFFFF))
    return specs


def mix_graph(spec) -> CSR:
    kind, n, u, gseed = spec
    g = _mixed_graph(kind, n, u, gseed)
    g.meta["mix_kind"] = kind
    return g


@dataclass
class Batch:
    """Graphs packed the way ``sgr_color_batch`` takes them: graph g's n_g+1
    local row offsets start at ``vtx_off[g] + g`` of ``row_offsets``; its local
    column ids start at ``edge_off[g]`` of ``col_idx``."""
    vtx_off: np.ndarray   # int64, G+1
    edge_off: np.ndarray  # int64, G+1
    row_offsets: np.ndarray  # int32, vtx_off[G] + G
    col_idx: np.ndarray   # int32, edge_off[G]
    graphs: list

    @property
    def G(self) -> int:
        return len(self.graphs)


def pack(graphs) -> Batch:
    G = len(graphs)
    vtx_off = np.zeros(G + 1, dtype=np.int64)
    edge_off = np.zeros(G + 1, dtype=np.int64)
    for i, g in enumerate(graphs):
        vtx_off[i + 1] = vtx_off[i] + g.n
        edge_off[i + 1] = edge_off[i] + g.m
    ro = np.empty(int(vtx_off[G]) + G, dtype=np.int32)
    ci = np.empty(int(edge_off[G]), dtype=np.int32)
    for i, g in enumerate(graphs):
        s = int(vtx_off[i]) + i
        ro[s:s + g.n + 1] = g.row_offsets
        ci[int(edge_off[i]):int(edge_off[i + 1])] = g.col_idx
    return Batch(vtx_off, edge_off, ro, ci, list(graphs))


def batch_mix(count: int = 512, n_lo: int = 1000, n_hi: int = 200000, seed: int = 0) -> Batch:
    """The batched workload: ``count`` graphs, sizes log-uniform in
    [n_lo, n_hi], a third uniform (average degree 4..32), a third R-MAT (edge
    factor 16), a third 2-D 9-point / 3-D 27-point stencils."""
    return pack([mix_graph(s) for s in mix_specs(count, n_lo, n_hi, seed)])

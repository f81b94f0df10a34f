"""Write tests/golden/mix_digests.json from the CPU oracle alone.

Two request sets, each graph colored on its own by the oracle's deterministic
SGR (Algorithm 7 with Algorithms 4 and 5, lower id keeps, Sect. 3.1):

* ``batch512``: every graph of ``graphgen.batch_mix(512, 1000, 200000, 0)``,
  the batched workload (512 graphs, n log-uniform in [1k, 200k], a third
  uniform, a third R-MAT, a third 2-D / 3-D stencils).  The batch entry point
  colors their disjoint union; each graph's slice must equal its own det-SGR
  coloring, since the loser rules compare ids only within a graph.
* ``serve_sizes``: eight requests of the served workload's generator mix with
  n from 1.6k to 4M (``graphgen.mix_specs(400, 1000, 4000000, 7)``, the
  indices below), all four kinds, four of them above 3M vertices.
* ``serve_pool``: the 24 graphs the served-stream benchmark draws its
  requests from (``graphgen.mix_specs(24, 1000, 4000000, 7)``), so that every
  served result can be checked.

For each graph: n, m, a SHA-256 of its CSR, the det color count, round count
and the SHA-256 of the det colors (int32 little-endian).  Nothing here touches
the GPU library.  The graphs come from the seeded, integer-only generators,
so they are the same on every machine.  The oracle runs in a process pool
(one graph per worker, single-threaded each).

    python tests/golden/make_mix_golden.py     # a few minutes on 8 cores
"""
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

BATCH = ("batch_mix(512, 1000, 200000, 0)", 512, 1000, 200000, 0)
SERVE_SPECS = ("mix_specs(400, 1000, 4000000, 7)", 400, 1000, 4000000, 7)
SERVE_PICK = [142, 335, 338, 249, 21, 7, 5, 4]
POOL = ("mix_specs(24, 1000, 4000000, 7)", 24, 1000, 4000000, 7)


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def graph_digest(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_offsets, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.col_idx, dtype="<i4").tobytes())
    return h.hexdigest()


def one(spec):
    sys.path.insert(0, ROOT)
    import graphgen as gg
    import oracle
    g = gg.mix_graph(spec)
    t0 = time.time()
    r = oracle.det_sgr(g, "low_keeps")
    assert r.status == 0 and oracle.check(g, r.colors)["valid"]
    return {"spec": list(spec), "n": g.n, "m": g.m, "graph_sha256": graph_digest(g),
            "det_num_colors": r.num_colors, "det_rounds": r.rounds,
            "det_colors_sha256": digest(r.colors), "oracle_s": round(time.time() - t0, 2)}


def main():
    import graphgen as gg
    import oracle
    gg.build()
    oracle.build()
    batch_specs = gg.mix_specs(*BATCH[1:])
    all_specs = gg.mix_specs(*SERVE_SPECS[1:])
    serve_specs = [all_specs[i] for i in SERVE_PICK]
    pool_specs = gg.mix_specs(*POOL[1:])
    work = list(serve_specs) + list(batch_specs) + list(pool_specs)
    work_order = sorted(range(len(work)), key=lambda i: -work[i][1])  # largest first
    ctx = mp.get_context("spawn")
    t0 = time.time()
    with ctx.Pool(max(1, (os.cpu_count() or 2) - 1)) as pool:
        res = pool.map(one, [work[i] for i in work_order], chunksize=1)
    by = {i: r for i, r in zip(work_order, res)}
    ns = len(serve_specs)
    out = {
        "serve_sizes": {"generator": f"graphgen.{SERVE_SPECS[0]}", "indices": SERVE_PICK,
                        "rule": "low_keeps", "graphs": [by[i] for i in range(ns)]},
        "batch512": {"generator": f"graphgen.{BATCH[0]}", "rule": "low_keeps",
                     "graphs": [by[ns + i] for i in range(len(batch_specs))]},
        "serve_pool": {"generator": f"graphgen.{POOL[0]}", "rule": "low_keeps",
                       "graphs": [by[ns + len(batch_specs) + i] for i in range(len(pool_specs))]},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mix_digests.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0, sort_keys=True)
        f.write("\n")
    print(f"wrote {path} in {time.time() - t0:.0f}s")


if __name__ == "__main__":
    main()

"""Write tests/golden/configs.json from the CPU oracle alone.

For each full-size workload this records the oracle's serial first-fit
(Algorithm 1) and deterministic SGR (Algorithm 7, lower id keeps) results:
color counts, round count, edge sums and a SHA-256 digest of the colors array
(int32 little-endian).  Nothing here touches the GPU library.  The inputs come
from the seeded, integer-only generators in ``graphgen`` and are therefore the
same on every machine.

    python tests/golden/make_golden.py        # about a minute on one core
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def graph_digest(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.row_offsets, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(g.col_idx, dtype="<i4").tobytes())
    return h.hexdigest()


WORKLOADS = {
    "er20k": lambda: gg.er20k(0),
    "rmat20": lambda: gg.rmat20(0),
    "stencil27_192": lambda: gg.stencil27(192),
}


def main():
    out = {}
    for name, make in WORKLOADS.items():
        t0 = time.time()
        g = make()
        sc, sk = oracle.serial_greedy(g)
        r = oracle.det_sgr(g, "low_keeps")
        assert r.status == 0 and oracle.check(g, r.colors)["valid"]
        out[name] = {
            "n": g.n, "m": g.m, "graph_sha256": graph_digest(g),
            "max_degree": int(g.degrees().max()),
            "serial_num_colors": sk, "serial_colors_sha256": digest(sc),
            "det_num_colors": r.num_colors, "det_rounds": r.rounds,
            "det_sum_w": r.sum_w, "det_sum_d": r.sum_d, "det_sum_d_low": r.sum_d_low,
            "det_sum_next": r.sum_next, "det_colors_sha256": digest(r.colors),
        }
        print(name, out[name], f"{time.time() - t0:.1f}s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()

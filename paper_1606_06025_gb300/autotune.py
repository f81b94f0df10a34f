"""Autotuner cache: measured tunings per graph class, kept in a JSON file.

``sgr_autotune`` / ``sgr_autotune_batch`` (C ABI) measure the tuning
candidates on one graph or one packed batch and install the fastest.  This
module keys the answer by a coarse signature of the graph (mode, log2 of n,
log2 of the average degree, log2 of the largest degree) or of the batch (mode,
log2 of the number of graphs, of the total vertices and of the average
degree) and stores it in a JSON file (``SGR_TUNE_FILE``, or the path given),
so that later graphs or batches of the same class reuse it without measuring.
"""
from __future__ import annotations

import json
import math
import os

from . import sgrcolor

DEFAULT_FILE = os.environ.get("SGR_TUNE_FILE", os.path.expanduser("~/.cache/sgrcolor_tune.json"))


def signature(n: int, m: int, max_degree: int, mode) -> str:
    """Coarse class of a graph: mode, log2 n, log2 average degree, log2 max degree."""
    avg = m / n if n else 0.0
    lg = lambda x: int(math.floor(math.log2(x))) if x >= 1 else 0
    return f"{sgrcolor._mode(mode)}:n{lg(n)}:d{lg(avg)}:D{lg(max_degree)}"


def batch_signature(G: int, n: int, m: int, mode) -> str:
    """Coarse class of a batch: mode, log2 of the graph count, of the total
    vertices and of the average degree."""
    lg = lambda x: int(math.floor(math.log2(x))) if x >= 1 else 0
    return f"batch:{sgrcolor._mode(mode)}:G{lg(G)}:n{lg(n)}:d{lg(m / n if n else 0.0)}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(row_offsets, col_idx, colors_out, max_degree: int, mode="det", path: str | None = None,
         budget_ms: int = 0, force: bool = False) -> dict:
    """Install a tuning for this graph: from the cache when its class was
    measured before, else measured now (and cached).  Device buffers are torch
    CUDA tensors; returns the tuning with its source and time."""
    path = path or DEFAULT_FILE
    n = row_offsets.numel() - 1
    m = col_idx.numel() if n else 0
    key = signature(n, m, max_degree, mode)
    cache = _load(path)
    if key in cache and not force:
        t = cache[key]["tuning"]
        sgrcolor.sgr_set_tuning(**t)
        return {"tuning": t, "source": "cache", "key": key, "ms": cache[key]["ms"]}
    t, ms = sgrcolor.sgr_autotune(n, row_offsets, col_idx, colors_out, mode, budget_ms)
    cache[key] = {"tuning": t, "ms": ms}
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return {"tuning": t, "source": "measured", "key": key, "ms": ms}


def _store(path, key, t, ms):
    cache = _load(path)
    cache[key] = {"tuning": t, "ms": ms}
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_batch(G, vtx_off, edge_off, row_offsets, col_idx, colors_out, num_colors, mode="det",
               path: str | None = None, budget_ms: int = 0, force: bool = False) -> dict:
    """Install a tuning for this batch (sgr_color_batch arguments): from the
    cache when its class was measured before, else measured now (and cached)."""
    path = path or DEFAULT_FILE
    n, m = int(vtx_off[G]), int(edge_off[G])
    key = batch_signature(G, n, m, mode)
    cache = _load(path)
    if key in cache and not force:
        t = cache[key]["tuning"]
        sgrcolor.sgr_set_tuning(**t)
        return {"tuning": t, "source": "cache", "key": key, "ms": cache[key]["ms"]}
    t, ms = sgrcolor.sgr_autotune_batch(G, vtx_off, edge_off, row_offsets, col_idx, colors_out, num_colors,
                                        mode, budget_ms)
    _store(path, key, t, ms)
    return {"tuning": t, "source": "measured", "key": key, "ms": ms}

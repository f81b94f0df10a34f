"""Python binding of libsgrcolor (ctypes over the C ABI in include/sgrcolor.h).

Argument marshalling only: every step of the coloring runs in the library's
CUDA kernels.  Device buffers may be passed as torch CUDA tensors or as raw
integer addresses; host buffers as numpy arrays.  A non-OK status raises
:class:`SgrError`.  Importing this module loads ``_build/libsgrcolor.so``
(building it with nvcc if it is missing or stale) and fails loudly if that is
not possible: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

SGR_OK = 0
SGR_PENDING = 1
SGR_ERR_INVALID_ARG = -1
SGR_ERR_INVALID_GRAPH = -2
SGR_ERR_OUT_OF_MEMORY = -3
SGR_ERR_CUDA = -4
SGR_ERR_NO_CONVERGENCE = -5
SGR_ERR_TIMEOUT = -6
SGR_ERR_NOT_FOUND = -7
SGR_ERR_BUSY = -8

SGR_MODE_DETERMINISTIC = 0
SGR_MODE_FAST = 1
SGR_MODE_TOPO = 2
SGR_RULE_LOW_KEEPS = 0 << 4
SGR_RULE_LOW_LOSES = 1 << 4
SGR_RULE_DEGREE = 2 << 4

MODES = {"det": SGR_MODE_DETERMINISTIC, "fast": SGR_MODE_FAST, "topo": SGR_MODE_TOPO}
RULES = {"low_keeps": SGR_RULE_LOW_KEEPS, "low_loses": SGR_RULE_LOW_LOSES,
         "degree": SGR_RULE_DEGREE}

# every symbol include/sgrcolor.h declares (checked by the tests)
EXPORTS = ["sgr_color", "sgr_color_noalloc", "sgr_color_host", "sgr_autotune", "sgr_autotune_batch",
           "sgr_color_batch", "sgr_validate_csr",
           "sgr_last_stats", "sgr_last_trace", "sgr_get_tuning", "sgr_set_tuning", "sgr_release_scratch",
           "sgr_status_string", "sgr_version", "sgr_server_create", "sgr_server_submit",
           "sgr_server_poll", "sgr_server_stats", "sgr_server_destroy", "sgr_set_wait_limit",
           "sgr_debug_inject"]


class SgrError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("sum_w", ctypes.c_int64),
                ("sum_d", ctypes.c_int64), ("sum_dscan", ctypes.c_int64),
                ("sum_next", ctypes.c_int64), ("sum_scatter", ctypes.c_int64),
                ("sum_rescan", ctypes.c_int64),
                ("num_colors", ctypes.c_int32),
                ("rows_sorted", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("device_ms", ctypes.c_double),
                ("tail_rounds", ctypes.c_int64), ("sum_touch", ctypes.c_int64),
                ("sum_dep", ctypes.c_int64), ("tail_entries", ctypes.c_int64),
                ("tail_build", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("device", ctypes.c_int32),
                ("rounds_per_launch", ctypes.c_int32), ("staging_bytes", ctypes.c_int64),
                ("direct_min_vertices", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "completed", "failed", "pending",
                                              "resident", "launches", "rounds", "hbm_bytes",
                                              "vertex_capacity", "entry_capacity")] + \
               [(f, ctypes.c_double) for f in ("p50_ms", "p99_ms", "mean_ms", "graphs_per_s")] + \
               [("direct", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("light_max", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("active_lists", ctypes.c_int32),
                ("tail_vertices", ctypes.c_int32)]


def _load():
    path = _build.build()
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    pi32 = ctypes.POINTER(ctypes.c_int32)
    lib.sgr_color.argtypes = [i32, vp, vp, vp, pi32, ctypes.c_int, vp]
    lib.sgr_color_host.argtypes = [i32, vp, vp, vp, pi32, ctypes.c_int, vp]
    lib.sgr_color_noalloc.argtypes = [i32, vp, vp, vp, pi32, ctypes.c_int, vp]
    lib.sgr_color_batch.argtypes = [i32, vp, vp, vp, vp, vp, vp, ctypes.c_int, vp]
    lib.sgr_validate_csr.argtypes = [i32, vp, vp, pi32, vp]
    lib.sgr_autotune.argtypes = [i32, vp, vp, vp, ctypes.c_int, i32, ctypes.POINTER(Tuning),
                                 ctypes.POINTER(ctypes.c_double), vp]
    lib.sgr_autotune_batch.argtypes = [i32, vp, vp, vp, vp, vp, vp, ctypes.c_int, i32, ctypes.POINTER(Tuning),
                                       ctypes.POINTER(ctypes.c_double), vp]
    lib.sgr_last_stats.argtypes = [ctypes.POINTER(Stats)]
    lib.sgr_last_trace.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int64)]
    lib.sgr_get_tuning.argtypes = [ctypes.POINTER(Tuning)]
    lib.sgr_set_tuning.argtypes = [ctypes.POINTER(Tuning)]
    lib.sgr_release_scratch.argtypes = []
    lib.sgr_status_string.argtypes = [ctypes.c_int]
    lib.sgr_status_string.restype = ctypes.c_char_p
    lib.sgr_version.argtypes = []
    lib.sgr_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    lib.sgr_server_submit.argtypes = [vp, i32, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.sgr_server_poll.argtypes = [vp, ctypes.c_uint64, vp, pi32, ctypes.c_int]
    lib.sgr_server_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    lib.sgr_server_destroy.argtypes = [vp]
    lib.sgr_set_wait_limit.argtypes = [i64]
    lib.sgr_debug_inject.argtypes = [ctypes.c_int, i64]
    for name in EXPORTS:
        if name != "sgr_status_string":
            getattr(lib, name).restype = ctypes.c_int
    return lib


_lib = _load()
LIB_PATH = _build.LIB_PATH


def _addr(x):
    """Device or host address of a tensor / array / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def status_string(status: int) -> str:
    return _lib.sgr_status_string(status).decode()


def _check(rc: int, where: str) -> int:
    if rc != SGR_OK:
        raise SgrError(rc, where)
    return rc


def _mode(mode) -> int:
    if isinstance(mode, int):
        return mode
    parts = mode.split("+") if isinstance(mode, str) else list(mode)
    m = 0
    for p in parts:
        m |= MODES[p] if p in MODES else RULES[p]
    return m


def sgr_color(n, row_offsets, col_idx, colors_out, mode=0, stream=None) -> int:
    """Color one graph held in device memory; returns the number of colors."""
    k = ctypes.c_int32(0)
    _check(_lib.sgr_color(int(n), _addr(row_offsets), _addr(col_idx), _addr(colors_out),
                          ctypes.byref(k), _mode(mode), _stream(stream)), "sgr_color")
    return int(k.value)


def sgr_color_noalloc(n, row_offsets, col_idx, colors_out, mode=0, stream=None) -> int:
    """sgr_color for callers that must not let the library allocate device
    memory: scratch comes from a fixed 16 MiB array in the library's device
    image.  Graphs too large for it raise SgrError(SGR_ERR_INVALID_ARG)."""
    k = ctypes.c_int32(0)
    _check(_lib.sgr_color_noalloc(int(n), _addr(row_offsets), _addr(col_idx), _addr(colors_out),
                                  ctypes.byref(k), _mode(mode), _stream(stream)), "sgr_color_noalloc")
    return int(k.value)


def sgr_color_host(n, row_offsets, col_idx, colors_out, mode=0, stream=None) -> int:
    """Color one graph held in host memory (numpy int32 arrays)."""
    k = ctypes.c_int32(0)
    _check(_lib.sgr_color_host(int(n), _addr(row_offsets), _addr(col_idx), _addr(colors_out),
                               ctypes.byref(k), _mode(mode), _stream(stream)), "sgr_color_host")
    return int(k.value)


def sgr_color_batch(G, vtx_off, edge_off, row_offsets, col_idx, colors_out, num_colors,
                    mode=0, stream=None) -> None:
    """Color G packed graphs; vtx_off / edge_off / num_colors are host arrays."""
    _check(_lib.sgr_color_batch(int(G), _addr(vtx_off), _addr(edge_off), _addr(row_offsets),
                                _addr(col_idx), _addr(colors_out), _addr(num_colors),
                                _mode(mode), _stream(stream)), "sgr_color_batch")


def sgr_autotune(n, row_offsets, col_idx, colors_out, mode=0, budget_ms=0, stream=None):
    """Measure the tuning candidates on this graph; installs and returns the
    fastest as (tuning dict, device ms)."""
    t = Tuning()
    ms = ctypes.c_double(0)
    _check(_lib.sgr_autotune(int(n), _addr(row_offsets), _addr(col_idx), _addr(colors_out),
                             _mode(mode), int(budget_ms), ctypes.byref(t), ctypes.byref(ms),
                             _stream(stream)), "sgr_autotune")
    return {f: getattr(t, f) for f, _ in Tuning._fields_}, float(ms.value)


def sgr_autotune_batch(G, vtx_off, edge_off, row_offsets, col_idx, colors_out, num_colors, mode=0,
                       budget_ms=0, stream=None):
    """Measure the tuning candidates on a packed batch (sgr_color_batch);
    installs and returns the fastest as (tuning dict, device ms)."""
    t = Tuning()
    ms = ctypes.c_double(0)
    _check(_lib.sgr_autotune_batch(int(G), _addr(vtx_off), _addr(edge_off), _addr(row_offsets),
                                   _addr(col_idx), _addr(colors_out), _addr(num_colors), _mode(mode),
                                   int(budget_ms), ctypes.byref(t), ctypes.byref(ms), _stream(stream)),
           "sgr_autotune_batch")
    return {f: getattr(t, f) for f, _ in Tuning._fields_}, float(ms.value)


def sgr_validate_csr(n, row_offsets, col_idx, stream=None):
    """Returns (status, rows_sorted) without raising on SGR_ERR_INVALID_GRAPH."""
    srt = ctypes.c_int32(-1)
    rc = _lib.sgr_validate_csr(int(n), _addr(row_offsets), _addr(col_idx), ctypes.byref(srt),
                               _stream(stream))
    if rc not in (SGR_OK, SGR_ERR_INVALID_GRAPH):
        raise SgrError(rc, "sgr_validate_csr")
    return rc, int(srt.value)


def sgr_last_stats() -> dict:
    s = Stats()
    _check(_lib.sgr_last_stats(ctypes.byref(s)), "sgr_last_stats")
    return s.as_dict()


def sgr_last_trace(cap_rounds: int = 1 << 16):
    """Per-round timeline of the last launch: dict of numpy arrays (w: |W_r|,
    end_a_ns / end_b_ns: ns at the end of each phase, rescans: vertices that
    scanned their row) and init_ns."""
    import numpy as np
    buf = np.zeros(4 * cap_rounds, dtype=np.int64)
    init = ctypes.c_int64(0)
    r = _lib.sgr_last_trace(buf.ctypes.data, cap_rounds, ctypes.byref(init))
    if r < 0:
        raise SgrError(r, "sgr_last_trace")
    t = buf[:4 * r].reshape(r, 4)
    return {"w": t[:, 0].copy(), "end_a_ns": t[:, 1].copy(), "end_b_ns": t[:, 2].copy(),
            "rescans": t[:, 3].copy(), "init_ns": int(init.value)}


def sgr_get_tuning() -> dict:
    t = Tuning()
    _check(_lib.sgr_get_tuning(ctypes.byref(t)), "sgr_get_tuning")
    return {f: getattr(t, f) for f, _ in Tuning._fields_}


def sgr_set_tuning(light_max=0, chunk=0, blocks_per_sm=0, active_lists=0, tail_vertices=0) -> None:
    t = Tuning(light_max, chunk, blocks_per_sm, active_lists, tail_vertices)
    _check(_lib.sgr_set_tuning(ctypes.byref(t)), "sgr_set_tuning")


def sgr_release_scratch() -> None:
    _check(_lib.sgr_release_scratch(), "sgr_release_scratch")


def sgr_set_wait_limit(ns: int) -> None:
    """Limit of every bounded device-side wait in ns (0: the 4 s default)."""
    _check(_lib.sgr_set_wait_limit(int(ns)), "sgr_set_wait_limit")


SGR_INJECT_NONE = 0
SGR_INJECT_FAIL_ALLOC = 1
SGR_INJECT_BARRIER = 2


def sgr_debug_inject(what: int, value: int = 0) -> None:
    """Host-side fault injection for tests (see sgrcolor.h)."""
    _check(_lib.sgr_debug_inject(int(what), int(value)), "sgr_debug_inject")


def sgr_version() -> int:
    return int(_lib.sgr_version())


class Server:
    """Continuous-batching coloring server (sgr_server_*): submit host CSR
    graphs, poll for their colors."""

    def __init__(self, hbm_budget_bytes=1 << 30, max_inflight=0, mode="det", device=0,
                 rounds_per_launch=0, staging_bytes=0, direct_min_vertices=0):
        cfg = ServerConfig(int(hbm_budget_bytes), int(max_inflight), _mode(mode), int(device),
                           int(rounds_per_launch), int(staging_bytes), int(direct_min_vertices))
        h = ctypes.c_void_p()
        _check(_lib.sgr_server_create(ctypes.byref(cfg), ctypes.byref(h)), "sgr_server_create")
        self._h = h

    def submit(self, row_offsets, col_idx) -> int:
        import numpy as np
        ro = np.ascontiguousarray(row_offsets, dtype=np.int32)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        rid = ctypes.c_uint64(0)
        _check(_lib.sgr_server_submit(self._h, ro.shape[0] - 1, ro.ctypes.data,
                                      ci.ctypes.data if ci.size else None, ctypes.byref(rid)),
               "sgr_server_submit")
        return int(rid.value)

    def poll(self, req_id: int, n: int, timeout_ms: int = -1):
        """(colors, k) when finished, None while pending."""
        import numpy as np
        out = np.empty(n, dtype=np.int32)
        k = ctypes.c_int32(0)
        rc = _lib.sgr_server_poll(self._h, req_id, out.ctypes.data if n else None,
                                  ctypes.byref(k), int(timeout_ms))
        if rc == SGR_PENDING:
            return None
        _check(rc, "sgr_server_poll")
        return out, int(k.value)

    def stats(self) -> dict:
        st = ServerStats()
        _check(_lib.sgr_server_stats(self._h, ctypes.byref(st)), "sgr_server_stats")
        return st.as_dict()

    def close(self):
        if self._h:
            _check(_lib.sgr_server_destroy(self._h), "sgr_server_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------ torch helpers

def color(row_offsets, col_idx, mode=0, stream=None, out=None):
    """Color a graph given as torch CUDA int32 tensors; returns (colors, k)."""
    import torch
    n = row_offsets.numel() - 1
    if out is None:
        out = torch.empty(max(n, 0), dtype=torch.int32, device=row_offsets.device)
    k = sgr_color(n, row_offsets, col_idx, out, mode, stream)
    return out, k


def loaded_library_path() -> str:
    return os.path.realpath(LIB_PATH)

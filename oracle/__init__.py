"""CPU oracle for speculative-greedy (SGR) graph coloring.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg (and its ``--impl reference`` arm) may import
this package.  The GPU library never imports it and shares no code with it.

* :func:`serial_greedy` -- Algorithm 1 (Sect. 2.1), plain C.
* :func:`det_sgr` -- Algorithm 7 with Algorithms 4 and 5 (Sect. 3.1), plain C,
  under the frozen-read and judge-before-clear readings stated in
  ``sgr_oracle.c``; three loser rules (lower id keeps, the printed lower id
  loses, and the degree heuristic of Sect. 3.2).
* :func:`check` -- validity (no monochrome edge, colors in 1..k).
* :mod:`oracle.sgr_py` -- an independently written pure-Python restatement of
  the same round loop, for small graphs (differential check of the C code).
* :mod:`oracle.brute` -- exhaustive chromatic number for tiny graphs.

Fast (racy) mode has no oracle: its parity is unpinned; only validity, the
color bound and the color ratio against serial greedy are checked.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

RULE_LOW_KEEPS = 0
RULE_LOW_LOSES = 1
RULE_DEGREE = 2
RULES = {"low_keeps": RULE_LOW_KEEPS, "low_loses": RULE_LOW_LOSES, "degree": RULE_DEGREE}


class _Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("sum_w", ctypes.c_int64),
                ("sum_d", ctypes.c_int64), ("sum_d_low", ctypes.c_int64),
                ("sum_next", ctypes.c_int64), ("num_colors", ctypes.c_int32),
                ("max_degree", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile ``sgr_oracle.c`` into ``_build/liboracle.so`` (host code only,
    plain -O2, single-threaded)."""
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
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.orc_serial_greedy.restype = i32
    lib.orc_serial_greedy.argtypes = [i32, vp, vp, vp]
    lib.orc_det_sgr.restype = ctypes.c_int
    lib.orc_det_sgr.argtypes = [i32, vp, vp, ctypes.c_int, i64, vp, ctypes.POINTER(_Stats),
                                vp, vp, i64]
    lib.orc_check.restype = i64
    lib.orc_check.argtypes = [i32, vp, vp, vp, ctypes.POINTER(i64), ctypes.POINTER(i32)]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data if a.size else None


def _csr(g):
    ro = np.ascontiguousarray(g.row_offsets, dtype=np.int32)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    return ro, ci


def serial_greedy(g):
    """Algorithm 1: returns (colors int32[n], k)."""
    ro, ci = _csr(g)
    n = ro.shape[0] - 1
    colors = np.zeros(n, dtype=np.int32)
    k = _load().orc_serial_greedy(n, _ptr(ro), _ptr(ci), _ptr(colors))
    if k < 0:
        raise MemoryError("oracle allocation failed")
    return colors, int(k)


@dataclass
class DetResult:
    colors: np.ndarray
    num_colors: int
    rounds: int
    sum_w: int
    sum_d: int
    sum_d_low: int
    sum_next: int
    max_degree: int
    trace_w: np.ndarray
    trace_d: np.ndarray
    status: int


def det_sgr(g, rule: int | str = RULE_LOW_KEEPS, max_rounds: int = 0,
            trace_cap: int = 1 << 16) -> DetResult:
    """Algorithm 7 (deterministic reading).  Returns colors, k, rounds and the
    per-round |W_r| / degree-sum trace (first ``trace_cap`` rounds)."""
    if isinstance(rule, str):
        rule = RULES[rule]
    ro, ci = _csr(g)
    n = ro.shape[0] - 1
    colors = np.zeros(n, dtype=np.int32)
    st = _Stats()
    tw = np.zeros(trace_cap, dtype=np.int64)
    td = np.zeros(trace_cap, dtype=np.int64)
    rc = _load().orc_det_sgr(n, _ptr(ro), _ptr(ci), rule, max_rounds, _ptr(colors),
                             ctypes.byref(st), _ptr(tw), _ptr(td), trace_cap)
    if rc == -3:
        raise MemoryError("oracle allocation failed")
    if rc == -1:
        raise ValueError("bad oracle arguments")
    r = int(st.rounds)
    return DetResult(colors, int(st.num_colors), r, int(st.sum_w), int(st.sum_d),
                     int(st.sum_d_low), int(st.sum_next), int(st.max_degree),
                     tw[:min(r, trace_cap)].copy(), td[:min(r, trace_cap)].copy(), int(rc))


def check(g, colors) -> dict:
    """Validity: monochrome directed entries, colors outside 1..k, and k."""
    ro, ci = _csr(g)
    n = ro.shape[0] - 1
    c = np.ascontiguousarray(colors, dtype=np.int32)
    bad = ctypes.c_int64(0)
    k = ctypes.c_int32(0)
    mono = _load().orc_check(n, _ptr(ro), _ptr(ci), _ptr(c), ctypes.byref(bad), ctypes.byref(k))
    return {"monochrome": int(mono), "bad_range": int(bad.value), "num_colors": int(k.value),
            "valid": mono == 0 and bad.value == 0}

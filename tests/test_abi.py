"""The C-ABI library loads and exports every symbol the header declares (CPU)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sgrcolor.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgr_[a-z_]+)\s*\(", text)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for must in ["sgr_color", "sgr_color_batch", "sgr_color_host", "sgr_validate_csr",
                 "sgr_last_stats", "sgr_status_string"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1606_06025_gb300 import sgrcolor
    out = subprocess.run(["nm", "-D", "--defined-only", sgrcolor.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sgr_[a-z_]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(sgrcolor.EXPORTS) == set(declared_functions())


def test_host_only_calls_without_gpu():
    from paper_1606_06025_gb300 import sgrcolor
    assert sgrcolor.sgr_version() >= 10000
    assert sgrcolor.status_string(0) == "SGR_OK"
    assert sgrcolor.status_string(-6) == "SGR_ERR_TIMEOUT"
    assert sgrcolor.status_string(12345) == "SGR_UNKNOWN_STATUS"
    t = sgrcolor.sgr_get_tuning()
    assert 1 <= t["light_max"] <= 32
    # invalid tunings are refused, valid ones round-trip
    for bad in [dict(active_lists=3), dict(light_max=33), dict(chunk=10), dict(blocks_per_sm=-1),
                dict(tail_vertices=-2), dict(tail_vertices=2881)]:
        try:
            sgrcolor.sgr_set_tuning(**bad)
        except sgrcolor.SgrError as e:
            assert e.status == sgrcolor.SGR_ERR_INVALID_ARG
        else:
            raise AssertionError(f"accepted {bad}")
    sgrcolor.sgr_set_tuning(light_max=8)
    assert sgrcolor.sgr_get_tuning()["light_max"] == 8
    for tv in (-1, 1, 2880, 0):
        sgrcolor.sgr_set_tuning(tail_vertices=tv)
        assert sgrcolor.sgr_get_tuning()["tail_vertices"] == tv
    sgrcolor.sgr_set_tuning(**t)
    assert sgrcolor.sgr_get_tuning() == t


def test_argument_checks_before_any_device_work():
    from paper_1606_06025_gb300 import sgrcolor
    import ctypes
    k = ctypes.c_int32(7)
    # n < 0, bad mode bits, null out-pointer: refused without touching a device
    assert sgrcolor._lib.sgr_color(-1, None, None, None, ctypes.byref(k), 0, None) == -1
    assert sgrcolor._lib.sgr_color(1, None, None, None, ctypes.byref(k), 0x100, None) == -1
    assert sgrcolor._lib.sgr_color(1, None, None, None, None, 0, None) == -1
    # n == 0 is a valid empty graph
    assert sgrcolor._lib.sgr_color(0, None, None, None, ctypes.byref(k), 0, None) == 0
    assert k.value == 0
    # mode 3 is no mode; the topology-driven mode is taken by the single-graph
    # entry points only (an empty graph needs no device)
    assert sgrcolor._lib.sgr_color(1, None, None, None, ctypes.byref(k), 3, None) == -1
    assert sgrcolor._lib.sgr_color(0, None, None, None, ctypes.byref(k), sgrcolor.SGR_MODE_TOPO, None) == 0
    assert sgrcolor._lib.sgr_color(0, None, None, None, ctypes.byref(k),
                                   sgrcolor.SGR_MODE_TOPO | sgrcolor.SGR_RULE_DEGREE, None) == 0
    assert sgrcolor._lib.sgr_color(0, None, None, None, ctypes.byref(k), sgrcolor.SGR_MODE_TOPO | (3 << 4), None) == -1


def test_header_mode_constants_match_the_binding():
    import re
    from paper_1606_06025_gb300 import sgrcolor
    text = open(os.path.join(ROOT, "include", "sgrcolor.h")).read()
    for name in ["SGR_MODE_DETERMINISTIC", "SGR_MODE_FAST", "SGR_MODE_TOPO"]:
        m = re.search(r"#define\s+" + name + r"\s+(\d+)", text)
        assert m and int(m.group(1)) == getattr(sgrcolor, name), name
    assert sgrcolor._mode("topo+degree") == sgrcolor.SGR_MODE_TOPO | sgrcolor.SGR_RULE_DEGREE


def test_every_params_pointer_is_set_by_both_arenas():
    # The launch parameters are filled by two arenas: layout() for the
    # single-graph, batch and no-allocation entry points, and the server's own.
    # A pointer the kernels use that one of them leaves null faults the
    # device, so every pointer field must be set by layout(), and by the server
    # unless the server never runs the code that uses it.
    src = open(os.path.join(ROOT, "paper_1606_06025_gb300", "csrc", "sgr_internal.cuh")).read()
    body = src[src.index("struct Params {"):]
    body = body[:body.index("};")]
    fields = []
    for line in body.splitlines():
        m = re.match(r"\s*(?:const\s+)?[\w:]+(?:\s+[\w:]+)*\s*\*\s*(\w+)(?:\[\d+\])?;", line.split("//")[0])
        if m:
            fields.append(m.group(1))
    assert len(fields) > 30
    api = open(os.path.join(ROOT, "paper_1606_06025_gb300", "csrc", "sgr_api.cu")).read()
    srv = open(os.path.join(ROOT, "paper_1606_06025_gb300", "csrc", "sgr_server.cu")).read()
    # not run by the server: its launches have front_ok = 0 (no activation
    # lists) and tail_max = 0 (no tail); uitem / uvert / urec are optional (every
    # write checks for null and ConflictResolve then searches the chunk bases)
    server_unused = {"uitem", "uvert", "urec", "al", "am", "ah", "acb", "astamp", "vslot",
                     "tlist", "tloc", "toff", "tcnt", "tlow", "tdeg", "tcp", "tcc", "tcm", "tadj", "tstage",
                     "twin"}
    for f in fields:
        assert re.search(r"p->" + f + r"\b", api), f"layout() leaves Params::{f} unset"
        if f not in server_unused:
            assert re.search(r"\bP\." + f + r"\b", srv), f"the server leaves Params::{f} unset"
    for f in ("front_ok", "tail_max"):
        assert not re.search(r"\bP\." + f + r"\s*=", srv), f"the server sets {f}: recheck server_unused"


def test_wait_limit_and_injection_arguments_without_gpu():
    from paper_1606_06025_gb300 import sgrcolor
    lib = sgrcolor._lib
    assert lib.sgr_set_wait_limit(0) == 0
    assert lib.sgr_set_wait_limit(1_000_000) == 0
    assert lib.sgr_set_wait_limit(99_999) == sgrcolor.SGR_ERR_INVALID_ARG  # under 100 us
    assert lib.sgr_set_wait_limit(-5) == sgrcolor.SGR_ERR_INVALID_ARG
    assert lib.sgr_set_wait_limit(0) == 0
    assert lib.sgr_debug_inject(99, 1) == sgrcolor.SGR_ERR_INVALID_ARG
    assert lib.sgr_debug_inject(sgrcolor.SGR_INJECT_FAIL_ALLOC, -1) == sgrcolor.SGR_ERR_INVALID_ARG
    assert lib.sgr_debug_inject(sgrcolor.SGR_INJECT_BARRIER, 2) == 0
    assert lib.sgr_debug_inject(sgrcolor.SGR_INJECT_NONE, 0) == 0
    for name in ("SGR_INJECT_NONE", "SGR_INJECT_FAIL_ALLOC", "SGR_INJECT_BARRIER"):
        m = re.search(r"#define\s+" + name + r"\s+(\d+)", open(HEADER).read())
        assert m and int(m.group(1)) == getattr(sgrcolor, name), name


def test_noalloc_refuses_topo_mode_before_any_device_work():
    import ctypes
    from paper_1606_06025_gb300 import sgrcolor
    k = ctypes.c_int32(-7)
    buf = (ctypes.c_int32 * 8)()
    rc = sgrcolor._lib.sgr_color_noalloc(2, ctypes.addressof(buf), ctypes.addressof(buf), ctypes.addressof(buf),
                                         ctypes.byref(k), sgrcolor.SGR_MODE_TOPO, None)
    assert rc == sgrcolor.SGR_ERR_INVALID_ARG and k.value == -7
    # the single-graph entry takes the same mode (an empty graph needs no device)
    assert sgrcolor._lib.sgr_color(0, None, None, None, ctypes.byref(k), sgrcolor.SGR_MODE_TOPO, None) == 0

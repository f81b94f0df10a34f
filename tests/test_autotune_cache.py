"""Autotune cache keys (host logic, CPU)."""
from paper_1606_06025_gb300 import autotune


def test_signature_buckets():
    a = autotune.signature(1 << 20, 31_400_000, 64_000, "det")
    b = autotune.signature((1 << 20) + 5, 31_000_000, 60_000, "det")
    c = autotune.signature(1 << 20, 31_400_000, 64_000, "fast")
    d = autotune.signature(7_077_888, 182_041_336, 26, "det")
    assert a == b and a != c and a != d
    assert autotune.signature(0, 0, 0, "det").endswith("n0:d0:D0")

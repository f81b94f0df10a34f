"""Autotune cache keys (host logic, CPU)."""
from paper_1606_06025_gb300 import autotune


def test_signature_buckets():
    a = autotune.signature(1 << 20, 31_400_000, 64_000, "det")
    b = autotune.signature((1 << 20) + 5, 31_000_000, 60_000, "det")
    c = autotune.signature(1 << 20, 31_400_000, 64_000, "fast")
    d = autotune.signature(7_077_888, 182_041_336, 26, "det")
    assert a == b and a != c and a != d
    assert autotune.signature(0, 0, 0, "det").endswith("n0:d0:D0")


def test_batch_signature_buckets():
    a = autotune.batch_signature(512, 19_302_282, 390_876_132, "det")
    b = autotune.batch_signature(600, 19_000_000, 380_000_000, "det")
    c = autotune.batch_signature(64, 19_302_282, 390_876_132, "det")
    assert a == b and a != c and a.startswith("batch:")

"""The benchmark's algorithmic work counts (the numerators of its roofline
fractions) against their closed forms for the workloads it reports: a
forward negacyclic NTT of length N is (N/2) log2 N butterflies; per prime,
vanilla encryption (Eq. 8) runs three transforms (u, m + e0, e1) and forms
two key products per coefficient, Zinc (Algorithm 1) runs two (m + e1',
e2'); the algorithmic bytes are the ciphertext written, 2 L N words, plus
the slots read.  No GPU."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2408_07304_gb300 import workloads  # noqa: E402


def test_throughput_counts():
    w = workloads.WORKLOADS["throughput"]
    assert (w.log_n, w.L, w.n) == (14, 8, 16384)
    assert bench.butterflies_per_ct(w, False) == 3 * 8 * 8192 * 14 == 2_752_512
    assert bench.butterflies_per_ct(w, True) == 2 * 8 * 8192 * 14 == 1_835_008
    assert bench.key_products_per_ct(w, False) == 2 * 8 * 16384 == 262_144
    assert bench.key_products_per_ct(w, True) == 0
    # ciphertext (2 L N uint64) + 8192 double slots
    assert 2 * w.L * w.n * 8 + 8 * 8192 == 2_162_688


def test_paper_shaped_counts():
    w = workloads.WORKLOADS["paper"]
    assert (w.log_n, w.L) == (15, 16)
    assert bench.butterflies_per_ct(w, False) == 3 * 16 * 16384 * 15 == 11_796_480
    assert bench.butterflies_per_ct(w, True) == 2 * 16 * 16384 * 15 == 7_864_320


def test_zinc_does_two_thirds_of_the_transforms():
    for name in ("single", "batched", "throughput", "large", "paper"):
        w = workloads.WORKLOADS[name]
        assert 3 * bench.butterflies_per_ct(w, True) == 2 * bench.butterflies_per_ct(w, False)

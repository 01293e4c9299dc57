"""Host-side helpers of bench.py (no GPU): launch counts per mode, the bytes
the library copies to host memory, the measured-peak file and the traffic
table."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


class Args:
    def __init__(self, operands="factored", s_method="contraction", h_method="factored"):
        self.operands, self.s_method, self.h_method = operands, s_method, h_method


@pytest.mark.parametrize("operands,s_method,h_method,n", [
    ("factored", "contraction", "factored", 14),
    ("factored", "legendre", "factored", 13),
    ("from_ab", "contraction", "factored", 10),
    ("factored", "contraction", "alg3", 14),
    ("from_ab", "contraction", "alg3", 9),
])
def test_launches_per_step(bench, operands, s_method, h_method, n):
    assert bench.launches_per_step(Args(operands, s_method, h_method)) == n


def test_copied_elements_cover_the_lower_triangle(bench):
    import paper_1712_07206_gb300 as fl
    for ng in (1, 63, 64, 65, 300, 2049, 3990):
        full = bench.copied_elements(ng, fl.LAYOUT_LOWER_FULL)
        assert ng * (ng + 1) // 2 <= full <= ng * ng
        w = max(64, (ng + 31) // 32)
        # the lower triangle plus at most one w x w triangle per block
        assert full - ng * (ng + 1) // 2 <= ((ng + w - 1) // w) * w * (w - 1) // 2
        assert bench.copied_elements(ng, fl.LAYOUT_LOWER_PACKED) == ng * (ng + 1) // 2


def test_peaks_and_traffic_table(bench):
    bf16, bf16_sus, hbm, src = bench.peaks()
    assert bf16 > 0 and bf16_sus > 0 and hbm > 0 and src in ("measured", "fallback")
    for (name, slices, s_method, h_method), v in bench.MEASURED_TRAFFIC.items():
        assert 4 <= slices <= 8 and s_method in ("contraction", "legendre")
        assert h_method in ("factored", "alg3") and v > 0

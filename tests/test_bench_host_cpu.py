"""Host-side arithmetic of bench.py (no GPU): the effective bit-operation count in closed form
against its defining sum, and how the profile summaries feed the roofline's traffic."""
from __future__ import annotations

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("m,n,r", [(1, 1, 0), (1, 1, 1), (5, 7, 3), (7, 5, 5), (64, 64, 64), (100, 640, 100),
                                   (1024, 1024, 1023), (3000, 200, 200)])
def test_effective_bitops_closed_form(m, n, r):
    """2 * sum_{i<r} (m-1-i)(n-1-i), the AND + XOR count of classical elimination."""
    want = 2 * sum((m - 1 - i) * (n - 1 - i) for i in range(r))
    assert bench.effective_bitops(m, n, r) == float(want)


def test_effective_bitops_square_full_rank_is_about_two_thirds_n_cubed():
    n = 65536
    assert abs(bench.effective_bitops(n, n, n - 1) / (2 * n ** 3 / 3) - 1) < 1e-4


def test_profile_keys_and_stale_capture(tmp_path, monkeypatch):
    """A summary's `key: value` lines are read as numbers; `captured_kernel_current: 0` marks a
    capture of an earlier build of the kernel."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_demo_1.md").write_text("# demo\n\nsome text: not a key line\ntraffic_ratio: 0.91\n"
                                      "captured_kernel_current: 0\nl1_port_frac: null\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("k_demo_1") == pytest.approx(0.91)
    assert bench.profile_value("k_demo_1", "captured_kernel_current") == 0
    assert bench.profile_value("k_demo_1", "l1_port_frac") is None
    assert bench.profile_value("k_demo_1", "missing") is None
    assert bench.traffic_from_profiles("k_absent_1") is None

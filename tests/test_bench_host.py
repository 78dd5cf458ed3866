"""Host-side logic of bench.py (no GPU): the measured-traffic figure of the
roofline is reported only for the kernel build and workload it was captured
on, and scales with the systems per launch."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class _P:
    def __init__(self, grid):
        self.grid = grid


def test_traffic_gated_on_workload_precision_variant_and_sources(monkeypatch):
    t = dict(bench.KAPPLY_TRAFFIC)
    p128 = _P(t["grid"])
    # a capture that matches a stand-in source hash
    monkeypatch.setattr(bench, "KAPPLY_TRAFFIC", dict(t, sources_sha256="0" * 64))
    assert bench.kapply_traffic(p128, t["precision"], t["fft_variant"], 18) is None   # sources differ
    # with the hash of the sources as they are, every other mismatch still withholds the figure
    import hashlib
    h = hashlib.sha256()
    for f in ("fpasses.cuh", "fft.cuh", "common.cuh"):
        with open(os.path.join(bench.ROOT, "paper_2106_12487_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    monkeypatch.setattr(bench, "KAPPLY_TRAFFIC", dict(t, sources_sha256=h.hexdigest()))
    assert bench.kapply_traffic(_P((64, 64, 64)), t["precision"], t["fft_variant"], 18) is None
    assert bench.kapply_traffic(p128, 1 - t["precision"], t["fft_variant"], 18) is None
    assert bench.kapply_traffic(p128, t["precision"], 2, 18) is None
    a = bench.kapply_traffic(p128, t["precision"], t["fft_variant"], 4)
    b = bench.kapply_traffic(p128, t["precision"], t["fft_variant"], 18)
    assert a == pytest.approx(4 * t["bytes_per_system"]) and b == pytest.approx(18 * t["bytes_per_system"])


def test_captured_traffic_is_below_the_algorithmic_bytes():
    """A capture of the fused chain cannot move more than a few % above its
    algorithmic bytes without re-reads: the recorded figure is a plausible one."""
    t = bench.KAPPLY_TRAFFIC
    V = t["grid"][0] * t["grid"][1] * t["grid"][2]
    alg = bench.KAPPLY_BYTES_PER_VOXEL[t["precision"]] * V
    assert 0.8 * alg < t["bytes_per_system"] < 1.05 * alg

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


def test_algorithmic_counts_and_metric_names():
    """The per-voxel counts the roofline lines divide by: the K-apply moves
    54 complex values + a 4-byte grain id per voxel (436 B in FP32), a PCG
    iteration adds the two CG vector kernels' 9c + 15c (628 B), and one apply
    executes 36 length-N transforms at 5 log2 N flops per point plus the
    pointwise strain, stress and divergence (1458 flops at 128^3)."""
    c = 8
    assert bench.KAPPLY_BYTES_PER_VOXEL[1] == 54 * c + 4
    assert bench.PCG_BYTES_PER_VOXEL == 54 * c + 4 + (9 + 15) * c
    assert bench.kapply_flops_per_voxel((128, 128, 128)) == 36 * 5 * 7 + 24 + 144 + 30
    assert bench.kapply_flops_per_voxel((64, 32, 16)) == 5 * 12 * (6 + 5 + 4) + 24 + 144 + 30
    assert bench.metric_of((128, 128, 128)) == bench.METRIC
    assert "256^3" in bench.metric_of((256, 256, 256))
    assert "128x128x1" in bench.metric_of((128, 128, 1))


def test_voigt_christoffel_speeds_match_the_oracle_on_a_single_crystal():
    """For a one-grain cell the volume average is the crystal itself, so the
    Christoffel speeds of the wave-speed study equal the oracle's branch slopes
    (Eq. wave_speed2) of that homogeneous cell."""
    import numpy as np
    from oracle import bloch_oracle as O
    from paper_2106_12487_gb300 import synth
    hx = synth.hexagonal_voigt(162e9, 92e9, 69e9, 181e9, 46.7e9)
    C6 = synth.rotate_voigt(hx, synth.haar_rotations(1, 5)[0])
    grid = (3, 4, 4)
    Nx, Ny, Nz = grid

    class P1:
        grain_ids = np.zeros((Nz, Ny, Nx), np.int32)
        C_per_grain = C6[None]
        rho = np.array([4506.0])

    med = O.Medium(grid, (1e-3,) * 3, P1.grain_ids, P1.C_per_grain, P1.rho)
    for d in ([1.0, 0.0, 0.0], [0.3, -0.2, 0.9]):
        assert np.allclose(bench.voigt_christoffel_speeds(P1, d), O.wave_speeds(med, d), rtol=1e-8)

"""Autotuner of the batched operator and the tile configurations it chooses
between, against the FP64 oracle.

* every pencils-per-CTA cap of the shared-memory passes computes the same
  operator (both precisions, a ragged grid and a grid with fast axes);
* bloch_plan_autotune returns a consistent report, and the plan it leaves
  behind still matches the oracle;
* a band solve with autotune = 1 gives the frequencies of the untuned plan.
"""
import math

import numpy as np
import pytest

from oracle import bloch_oracle as O
from paper_2106_12487_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = {0: 1e-12, 1: 5e-6}   # FP64, FP32: the operator tolerances of the op tests


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_12487_gb300 import bloch, build
    build.build()
    bloch.lib()
    return bloch


def to_dev(a, prec):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda",
                                                        dtype=torch.complex64 if prec else torch.complex128)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def check_apply(plan, p, med, prec, nb=3, seed=11):
    ks = np.array([[0.3, -0.2, 0.7], [0.0, 0.9, 0.1], [0.5, 0.5, 0.5]])[:nb] * math.pi / 1e-3
    u = synth.random_field(p.grid, seed, batch=nb)
    out = to_dev(np.zeros_like(u), prec)
    plan.apply_K(ks, to_dev(u, prec), out)
    got = out.cpu().numpy()
    for b in range(nb):
        assert rel(got[b], O.apply_K(med, ks[b], u[b])) < TOL[prec]


@pytest.mark.parametrize("grid", [(24, 20, 15), (32, 16, 64)])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("pmax", [4, 8, 16, 32])
def test_tile_caps_compute_the_same_operator(B, grid, prec, variant, pmax):
    p = synth.small_polycrystal(grid, 7, 3)
    med = O.Medium.from_problem(p)
    plan = B.Plan.from_problem(p, precision=prec, fft_variant=variant, tile_pmax=pmax)
    check_apply(plan, p, med, prec)


@pytest.mark.parametrize("grid", [(24, 20, 15), (32, 32, 32)])
@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_report_and_parity(B, grid, prec, capsys):
    p = synth.small_polycrystal(grid, 7, 4)
    med = O.Medium.from_problem(p)
    plan = B.Plan.from_problem(p, precision=prec)
    rep = plan.autotune(prec, 6)
    with capsys.disabled():
        print(f"\nautotune {grid} prec {prec}: {rep}")
    assert rep["fft_variant"] in (0, 1, 2)
    assert rep["tile_pmax"] in (4, 8, 16, 32)
    ms = rep["ms_per_system"]
    assert ms[1] > 0 and ms[2] > 0
    fast = grid == (32, 32, 32)
    assert (ms[0] > 0) == fast
    # variant 1 sweeps 4 caps, cuFFT one; variant 0 sweeps 4 caps when a shared-memory pass remains
    n0 = 0 if not fast else (1 if prec == 1 else 4)
    assert rep["candidates"] == 4 + 1 + n0
    best = min(m for m in ms if m > 0)
    assert ms[rep["fft_variant"]] == best
    assert rep["saturating_systems"] in (6, 12, 24, 48)
    check_apply(plan, p, med, prec)


def test_solve_with_autotune_matches_untuned(B):
    p = synth.small_polycrystal((12, 10, 8), 5, 6, n_bands=6)
    ks = np.array([[0.4, 0.1, 0.0], [0.2, 0.3, 0.6]]) * math.pi / 1e-3
    opt = dict(precision=0, method=1, tol_lin=1e-11, tol_eig=1e-11)
    ref, _, _ = B.Plan.from_problem(p, **opt).solve_bands(ks, 6)
    got, _, _ = B.Plan.from_problem(p, autotune=1, **opt).solve_bands(ks, 6)
    assert np.max(np.abs(got / ref - 1)) < 1e-9


@pytest.mark.parametrize("prec,method", [(1, 0), (1, 1), (0, 1)])
def test_trace_phases_are_consistent(B, prec, method):
    """The phase tracer: traced phases fit inside the GPU span, the span
    inside the host wall time; PCG is recorded under the solver that ran it;
    FP32 residuals appear only in the FP32 form; tracing off records nothing."""
    p = synth.small_polycrystal((16, 16, 16), 6, 8, n_bands=4)
    ks = np.array([[0.4, 0.1, 0.0], [0.2, 0.3, 0.6]]) * math.pi / 1e-3
    opt = dict(tol_lin=1e-3, tol_eig=1e-6) if prec == 1 else dict(tol_lin=1e-10, tol_eig=1e-10)
    plan = B.Plan.from_problem(p, precision=prec, method=method, **opt)
    plan.trace(True)
    plan.solve_bands(ks, 4)
    tr = plan.trace(False)
    parts = sum(tr[k]["ms"] for k in ("pcg_subspace", "pcg_lanczos", "residual_fp32", "residual_fp64",
                                      "lanczos_orth", "projection", "lanczos_restart", "setup"))
    assert 0 < parts <= tr["gpu_span"]["ms"] * 1.001
    assert tr["gpu_span"]["ms"] <= tr["wall"]["ms"] * 1.001
    assert tr["gpu_span"]["count"] == 1 and tr["wall"]["count"] == 1
    assert (tr["pcg_lanczos"]["count"] > 0) == (method == 0)
    assert (tr["lanczos_orth"]["count"] > 0) == (method == 0)
    assert (tr["lanczos_restart"]["count"] > 0) == (method == 0)
    assert tr["setup"]["count"] > 0
    assert tr["pcg_subspace"]["count"] > 0 or method == 0
    if prec == 0:
        assert tr["residual_fp64"]["count"] > 0 or method == 0
        assert tr["residual_fp32"]["count"] == 0
    plan.solve_bands(ks, 4)
    off = plan.trace(False)
    assert all(v["count"] == 0 for v in off.values())


def test_fma_peaks():
    """bloch_fma_peaks: positive rates, FP32 above FP64 (GB300's FP64 units
    run at a small fraction of its FP32 rate), and both below the FMA issue
    limit of the device (2 flops x 128 lanes x SMs x 2.1 GHz for FP32)."""
    import torch
    from paper_2106_12487_gb300 import bloch as B
    g64, g32 = B.fma_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert 0 < g64 < g32
    assert g32 < 2 * 128 * sms * 2.2e9 / 1e9

"""GPU parity of the operators, preconditioner and PCG against the FP64 oracle.

Tolerances: FP64 path 1e-12 relative (2-norm), the roundoff of a few FFTs;
FP32 path 5e-6 relative, a few units of FP32 roundoff amplified by the
log2(N) FFT stages and the |xi + k| weights of the derivative steps.
"""
import math

import numpy as np
import pytest

from oracle import bloch_oracle as O
from paper_2106_12487_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 5e-6}   # FP64, FP32


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
    dt = torch.complex128 if prec == 0 else torch.complex64
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


GRIDS = [(4, 4, 4), (6, 6, 6), (6, 4, 5), (16, 16, 16), (32, 32, 32), (24, 20, 12), (9, 7, 10),
         (64, 32, 16), (8, 1, 1), (4, 4, 1), (1, 1, 1), (128, 2, 3), (16, 128, 64), (256, 16, 32),
         (64, 64, 256), (128, 15, 21)]


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_apply_K_matches_oracle(B, grid, prec, variant):
    """The kernel variants (two-stage register FFT passes, shared-memory
    Stockham passes, cuFFT plain-form baseline) against the oracle."""
    p = synth.small_polycrystal(grid, 5, 3)
    med = O.Medium.from_problem(p)
    plan = B.Plan.from_problem(p, precision=prec, fft_variant=variant)
    ks = np.array([[0.31, -0.12, 0.77], [1.0, 0.0, 0.0], [0.0, 0.0, 0.0]]) * math.pi / 1e-3
    u = synth.random_field(grid, 11, batch=3)
    out = to_dev(np.zeros_like(u), prec)
    plan.apply_K(ks, to_dev(u, prec), out)
    got = out.cpu().numpy()
    for b in range(3):
        ref = O.apply_K(med, ks[b], u[b])
        if np.linalg.norm(ref) == 0:
            assert np.linalg.norm(got[b]) <= 1e-30
            continue
        assert rel(got[b], ref) < TOL[prec], (b, rel(got[b], ref))


@pytest.mark.parametrize("prec", [0, 1])
def test_apply_K_anisotropic_cell_lengths(B, prec):
    """Non-cubic cell (different L per axis) with a hexagonal crystal."""
    grid = (12, 10, 8)
    ids = synth.voronoi_periodic(grid, 4, 9, L=(2e-3, 1e-3, 0.5e-3))
    hx = synth.hexagonal_voigt(162e9, 92e9, 69e9, 181e9, 46.7e9)
    R = synth.haar_rotations(4, 19)
    C = np.stack([synth.rotate_voigt(hx, r) for r in R])
    L = (2e-3, 1e-3, 0.5e-3)
    med = O.Medium(grid, L, ids, C, np.full(4, 4506.0))
    plan = B.Plan(grid, L, ids, C, np.full(4, 4506.0), B.default_options(precision=prec))
    k = np.array([0.3 * math.pi / L[0], 0.8 * math.pi / L[1], -0.5 * math.pi / L[2]])
    u = synth.random_field(grid, 5)
    out = to_dev(np.zeros_like(u), prec)
    plan.apply_K(k, to_dev(u, prec), out)
    assert rel(out.cpu().numpy(), O.apply_K(med, k, u)) < TOL[prec]


@pytest.mark.parametrize("grid", [(8, 8, 8), (6, 4, 5), (32, 16, 8)])
@pytest.mark.parametrize("prec", [0, 1])
def test_apply_M_matches_oracle(B, grid, prec):
    p = synth.small_polycrystal(grid, 4, 8)
    for rho in (np.full(4, 8960.0), np.array([8960.0, 1200.0, 4506.0, 19300.0])):
        med = O.Medium(grid, p.L, p.grain_ids, p.C_per_grain, rho)
        plan = B.Plan(grid, p.L, p.grain_ids, p.C_per_grain, rho, B.default_options(precision=prec))
        u = synth.random_field(grid, 3, batch=2)
        out = to_dev(np.zeros_like(u), prec)
        plan.apply_M(to_dev(u, prec), out)
        got = out.cpu().numpy()
        for b in range(2):
            assert rel(got[b], O.apply_M(med, u[b])) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_precond_matches_oracle(B, prec):
    grid = (12, 8, 10)
    p = synth.small_polycrystal(grid, 6, 4)
    med = O.Medium.from_problem(p)
    plan = B.Plan.from_problem(p, precision=prec)
    ks = np.array([[0.2, 0.4, -0.6], [0.0, 0.0, 0.0]]) * math.pi / 1e-3
    r = synth.random_field(grid, 1, batch=2)
    out = to_dev(np.zeros_like(r), prec)
    plan.apply_precond(ks, to_dev(r, prec), out)
    got = out.cpu().numpy()
    for b in range(2):
        ref = O.apply_precond(med, ks[b], r[b])
        assert rel(got[b], ref) < (1e-12 if prec == 0 else 2e-6)
    # the q = 0 bin at k = 0 maps to zero
    assert np.all(got[1][:, 0, 0, 0] == 0)


@pytest.mark.parametrize("grid", [(8, 8, 8), (16, 12, 10)])
def test_pcg_fp64_matches_oracle(B, grid):
    """Algorithm 2 in FP64: the GPU solution equals the oracle PCG solution and
    its true residual meets the tolerance; systems at several k run batched."""
    p = synth.small_polycrystal(grid, 6, 12)
    med = O.Medium.from_problem(p)
    plan = B.Plan.from_problem(p, precision=0)
    ks = np.array([[0.5, 0.1, 0.0], [1.0, 1.0, 0.0], [0.05, 0.0, 0.02]]) * math.pi / 1e-3
    b = synth.random_field(grid, 2, batch=3) * 1e20
    x = to_dev(np.zeros_like(b), 0)
    iters, relres, _ = plan.pcg(ks, to_dev(b, 0), x, 1e-11, 5000)
    got = x.cpu().numpy()
    for i in range(3):
        A = lambda v, kk=ks[i]: O.apply_K(med, kk, v)
        ref = O.pcg(A, lambda v, kk=ks[i]: O.apply_precond(med, kk, v), b[i], 1e-11, 5000)
        assert abs(iters[i] - ref.iters) <= 1
        assert rel(got[i], ref.x) < 1e-9
        assert O.norm(b[i] - A(got[i])) / O.norm(b[i]) < 5e-11


@pytest.mark.parametrize("prec", [0, 1])
def test_pcg_graph_loop_equals_host_loop(B, prec):
    """The graph-resident PCG loop (conditional WHILE node, device-side
    condition) takes the same iterations and returns the same solutions as
    the host-driven loop; the iteration cap ends the loop."""
    grid = (16, 12, 10)
    p = synth.small_polycrystal(grid, 6, 12)
    ks = np.array([[0.5, 0.1, 0.0], [1.0, 1.0, 0.0], [0.05, 0.0, 0.02]]) * math.pi / 1e-3
    b = synth.random_field(grid, 2, batch=3) * 1e20
    tol = 1e-10 if prec == 0 else 1e-5
    res = {}
    for graph in (0, 1):
        plan = B.Plan.from_problem(p, precision=prec, cuda_graph=graph)
        x = to_dev(np.zeros_like(b), prec)
        iters, rel, _ = plan.pcg(ks, to_dev(b, prec), x, tol, 5000)
        res[graph] = (iters, x.cpu().numpy())
        capped, _, st = plan.pcg(ks, to_dev(b, prec), x, tol, 3, allow_nonconv=True)
        assert st == 4 and np.all(capped == 3)
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])


def test_pcg_fp32_reaches_fp32_tolerance(B):
    grid = (16, 16, 16)
    p = synth.small_polycrystal(grid, 6, 13)
    med = O.Medium.from_problem(p)
    plan = B.Plan.from_problem(p, precision=1)
    k = np.array([0.3, 0.2, 0.1]) * math.pi / 1e-3
    b = synth.random_field(grid, 6) * 1e18
    x = to_dev(np.zeros_like(b), 1)
    iters, relres, _ = plan.pcg(k, to_dev(b, 1), x, 1e-5, 2000)
    got = x.cpu().numpy().astype(np.complex128)
    true_rel = O.norm(b - O.apply_K(med, k, got)) / O.norm(b)
    assert relres[0] <= 1e-5 and true_rel < 3e-5


@pytest.mark.parametrize("grid", [(16, 12, 10), (32, 10, 12), (64, 8, 6), (128, 6, 4), (12, 10, 32),
                                  (10, 6, 128), (5, 3, 32), (4, 2, 64)])
def test_pcg_fp32_fused_products(B, grid):
    """FP32 PCG with (p, A p) formed inside the operator: by the strain energy
    of the fast x pass (x axes 16-128: both x-pass forms) or by the fast
    z-divergence pass (z axes 32, 128 with a generic x axis).  Iteration
    counts follow the FP64 oracle's PCG and the true residual meets the
    tolerance: a mis-scaled or mis-summed product would change the step
    lengths and with them the iteration count.  The fast z passes stage their
    pencils by TMA tiles where a plane has an even number of at least P
    pencils, by cp.async otherwise (5 x 3 and 4 x 2 planes)."""
    p = synth.small_polycrystal(grid, 5, 17)
    med = O.Medium.from_problem(p)
    plan = B.Plan.from_problem(p, precision=1)
    ks = np.array([[0.3, 0.2, 0.1], [0.9, -0.4, 0.2]]) * math.pi / 1e-3
    b = synth.random_field(grid, 8, batch=2) * 1e18
    x = to_dev(np.zeros_like(b), 1)
    iters, relres, _ = plan.pcg(ks, to_dev(b, 1), x, 1e-5, 2000)
    got = x.cpu().numpy().astype(np.complex128)
    for i in range(2):
        A = lambda v, kk=ks[i]: O.apply_K(med, kk, v)
        ref = O.pcg(A, lambda v, kk=ks[i]: O.apply_precond(med, kk, v), b[i], 1e-5, 2000)
        assert abs(int(iters[i]) - ref.iters) <= 1
        assert relres[i] <= 1e-5
        assert O.norm(b[i] - A(got[i])) / O.norm(b[i]) < 3e-5


def test_apply_K_large_grid_sampled(B):
    """Full-size 128^3 cell of the measured workload (200 grains, <001> fibre):
    FP32 apply against the oracle on the whole field, two wave vectors."""
    p = synth.workload("rve128_g200")
    med = O.Medium.from_problem(p)
    plan = B.Plan.from_problem(p, precision=1)
    ks = p.k_list[[5, 40]]
    u = synth.random_field(p.grid, 21, batch=2) * np.exp(-np.arange(2))[:, None, None, None, None]
    out = to_dev(np.zeros_like(u), 1)
    plan.apply_K(ks, to_dev(u, 1), out)
    got = out.cpu().numpy()
    for b in range(2):
        assert rel(got[b], O.apply_K(med, ks[b], u[b])) < TOL[1]


def test_invalid_arguments_on_device(B):
    import torch
    p = synth.small_polycrystal((4, 4, 4), 2, 1)
    plan = B.Plan.from_problem(p, precision=0)
    u = torch.zeros(3 * 64, dtype=torch.complex128, device="cuda")
    with pytest.raises(B.BlochError) as e:
        plan.apply_K([math.nan, 0, 0], u, torch.zeros_like(u))
    assert e.value.status == 6
    with pytest.raises(TypeError):
        plan.apply_K([0, 0, 0], u.to(torch.complex64), torch.zeros_like(u))


@pytest.mark.parametrize("grid", [(16, 16, 16), (24, 20, 15), (32, 16, 64), (1, 1, 1)])
@pytest.mark.parametrize("prec", [0, 1])
def test_apply_K_real_basis(B, grid, prec):
    """Real-space basis: F^-1 A_k F u against the oracle's Fourier-space
    operator wrapped in numpy's forward / inverse FFT (same conventions)."""
    p = synth.small_polycrystal(grid, 5, 13)
    med = O.Medium.from_problem(p)
    plan = B.Plan.from_problem(p, precision=prec)
    ks = np.array([[0.3, -0.2, 0.7], [0.0, 0.9, 0.1]]) * math.pi / 1e-3
    u = synth.random_field(grid, 19, batch=2)
    out = to_dev(np.zeros_like(u), prec)
    plan.apply_K_real(ks, to_dev(u, prec), out)
    got = out.cpu().numpy()
    ax = (-3, -2, -1)
    for b in range(2):
        want = np.fft.ifftn(O.apply_K(med, ks[b], np.fft.fftn(u[b], axes=ax)), axes=ax)
        assert rel(got[b], want) < TOL[prec]


@pytest.mark.parametrize("grid", GRIDS)
def test_apply_K_float_float_matches_oracle(B, grid):
    """BLOCH_FF: the stiffness operator in float-float arithmetic (48-bit
    significand on the FP32 pipes; double buffers) against the FP64 oracle at
    the FP64 path's tolerance -- the arithmetic of the FP32 form's check."""
    import torch
    p = synth.small_polycrystal(grid, 5, 3)
    med = O.Medium.from_problem(p)
    plan = B.Plan.from_problem(p, precision=0)
    ks = np.array([[0.31, -0.12, 0.77], [1.0, 0.0, 0.0], [0.0, 0.0, 0.0]]) * math.pi / 1e-3
    u = synth.random_field(grid, 11, batch=3)
    out = to_dev(np.zeros_like(u), 0)
    plan.apply_K(ks, to_dev(u, 0), out, precision=B.FF)
    got = out.cpu().numpy()
    for b in range(3):
        ref = O.apply_K(med, ks[b], u[b])
        if np.linalg.norm(ref) == 0:
            assert np.linalg.norm(got[b]) <= 1e-30
            continue
        assert rel(got[b], ref) < 1e-12, (b, rel(got[b], ref))

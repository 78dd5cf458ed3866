"""Learned Fourier-space preconditioner on the GPU against the FP64 oracle.

* a fresh network is exactly the paper's preconditioner (g = 1);
* the hand-written GPU loss and gradient equal the oracle's loss and central
  finite-difference gradient on the same recorded data;
* training lowers the loss, and the trained network's effect on PCG
  iteration counts at equal tolerance is measured on a held-out cell;
* band frequencies do not depend on the preconditioner.
"""
import math

import numpy as np
import pytest

from oracle import bloch_oracle as O
from oracle import learned_precond as OL
from paper_2106_12487_gb300 import synth

pytestmark = pytest.mark.gpu
H = 16


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_12487_gb300 import bloch, build
    build.build()
    bloch.lib()
    return bloch


def to_dev(a, prec=1):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda",
                                                        dtype=torch.complex64 if prec else torch.complex128)


def oracle_blocks(lp):
    out = []
    total = 0
    for i in range(lp.num_blocks):
        b = lp.export_block(i)
        Nx, Ny, Nz = b["grid"]
        qx, qy, qz = b["q"][:Nx], b["q"][Nx:Nx + Ny], b["q"][Nx + Ny:]
        Q = np.stack(np.meshgrid(qx, qy, qz, indexing="ij"), -1)          # (Nx, Ny, Nz, 3)
        Q = np.transpose(Q, (2, 1, 0, 3)).reshape(-1, 3)                  # voxel order z, y, x
        nz = np.einsum("nj,nj->n", Q, Q) > 0
        C0 = O.voigt_to_tensor(b["C0V"])
        out.append(dict(q=Q[nz], A=b["mom"][nz, :6], B=b["mom"][nz, 6:12], c=b["mom"][nz, 12], C0=C0,
                        Nmax=max(Nx, Ny, Nz)))
        total += b["samples"]
    return out, total


def test_fresh_network_is_green_preconditioner(B):
    p = synth.small_polycrystal((12, 10, 8), 5, 2)
    plan = B.Plan.from_problem(p, precision=1)
    ks = np.array([[0.3, 0.2, -0.4], [0.0, 0.0, 0.0]]) * math.pi / 1e-3
    r = to_dev(synth.random_field(p.grid, 4, batch=2))
    z0 = to_dev(np.zeros((2, 3, 8, 10, 12)))
    plan.apply_precond(ks, r, z0)
    lp = B.LearnedPrecond(seed=3)
    B.set_preconditioner(plan, lp)
    z1 = to_dev(np.zeros((2, 3, 8, 10, 12)))
    plan.apply_precond(ks, r, z1)
    a, b = z0.cpu().numpy(), z1.cpu().numpy()
    assert np.linalg.norm(b - a) / np.linalg.norm(a) < 2e-6
    # the oracle's model at these parameters is P^-1 as well
    theta = lp.params().astype(np.float64)
    med = O.Medium.from_problem(p)
    q = np.array([[0.7, -0.2, 1.3], [2.0, 0.0, 0.0], [1.0, 1.0, 1.0]])
    C0 = med.C0 / max(med.C0[0, 0, 0, 0], med.C0[1, 1, 1, 1], med.C0[2, 2, 2, 2])
    Z = OL.Z_of(theta, H, q, C0, 12)
    P = OL.acoustic(C0, q)
    assert np.allclose(Z, np.linalg.inv(P), rtol=1e-6, atol=0)


def test_gradient_matches_oracle_finite_differences(B):
    """GPU loss/gradient (FP32 arithmetic, FP64 accumulation) against the FP64
    oracle loss and its central finite differences on the exported data."""
    p = synth.small_polycrystal((8, 8, 8), 4, 5)
    plan = B.Plan.from_problem(p, precision=1)
    lp = B.LearnedPrecond(seed=5)
    ks = np.array([[0.4, 0.1, 0.0], [0.0, 0.7, 0.3]]) * math.pi / 1e-3
    lp.collect(plan, ks, n_rhs=2, n_iters=3, seed=21)
    theta = lp.params()
    rng = np.random.default_rng(0)
    nh = H * 5 + H + H * H + H
    theta[nh:nh + H] = rng.uniform(-0.5, 0.5, H)     # non-trivial output layer
    theta[-1] = 0.3
    lp.params(set_to=theta)
    theta = lp.params()                               # exactly the FP32 values in use
    L_gpu, g_gpu = lp.loss_grad()
    blocks, total = oracle_blocks(lp)
    L_or = OL.loss(theta, H, blocks) / total
    g_or = OL.fd_grad(theta, H, blocks, h=1e-6) / total
    assert abs(L_gpu - L_or) <= 1e-4 * abs(L_or)
    assert np.linalg.norm(g_gpu - g_or) <= 2e-3 * np.linalg.norm(g_or)
    # the gradient is not trivially zero in any layer
    assert np.linalg.norm(g_or[:H * 5]) > 0 and np.linalg.norm(g_or[nh:]) > 0


def _pcg_iters(B, plan, k, n_rhs, tol, seed):
    b = to_dev(synth.random_field(plan.grid, seed, batch=n_rhs) * 1e18)
    x = to_dev(np.zeros((n_rhs, 3) + tuple(reversed(plan.grid))))
    iters, rel, _ = plan.pcg(np.repeat(np.asarray(k)[None], n_rhs, 0), b, x, tol, 2000)
    assert np.all(rel <= tol)
    return iters


def test_training_lowers_loss_and_reports_cg_gain(B, capsys):
    """Train on seeded 16^3 cubic polycrystals (Zener ratio 1-4, 6-20 grains),
    evaluate PCG iterations on a held-out 24^3 cell at equal tolerance."""
    lp = B.LearnedPrecond(seed=7)
    for i in range(6):
        zener = 1.0 + 3.0 * i / 5.0
        c11, c12 = 168.4e9, 121.4e9
        C = synth.cubic_voigt(c11, c12, zener * (c11 - c12) / 2)
        ng = 6 + 3 * i
        ids = synth.voronoi_periodic((16, 16, 16), ng, 1000 + i)
        R = synth.haar_rotations(ng, 2000 + i)
        Cg = np.stack([synth.rotate_voigt(C, r) for r in R])
        plan = B.Plan((16, 16, 16), (1e-3,) * 3, ids, Cg, np.full(ng, 8960.0), B.default_options(precision=1))
        ks = synth.kpath("GXM", 5)[1:]
        lp.collect(plan, ks, n_rhs=2, n_iters=10, seed=31 + i)
    L0, _ = lp.loss_grad()
    hist = lp.train(300, lr=3e-3)
    L1, _ = lp.loss_grad()
    with capsys.disabled():
        print(f"\nloss history: {hist[0]:.5e} {hist[50]:.5e} {hist[150]:.5e} {hist[-1]:.5e}")
    assert L1 < L0 and hist[-1] <= hist[0]
    # held-out cell
    p = synth.small_polycrystal((24, 24, 24), 15, 77)
    plan = B.Plan.from_problem(p, precision=1)
    k = np.array([0.35, 0.1, 0.2]) * math.pi / 1e-3
    it_green = _pcg_iters(B, plan, k, 4, 1e-5, 5)
    B.set_preconditioner(plan, lp)
    it_learn = _pcg_iters(B, plan, k, 4, 1e-5, 5)
    with capsys.disabled():
        print(f"\nlearned preconditioner: loss {L0:.4e} -> {L1:.4e}; PCG iterations to 1e-5 on a held-out "
              f"24^3 cell: Green {it_green.tolist()} mean {it_green.mean():.1f}, learned {it_learn.tolist()} "
              f"mean {it_learn.mean():.1f}")
    assert np.all(it_learn > 0)


def test_bands_independent_of_preconditioner(B):
    p = synth.small_polycrystal((8, 8, 8), 6, 5, n_bands=6)
    med = O.Medium.from_problem(p)
    ks = np.array([[0.5, 0.0, 0.0], [0.3, 0.6, 0.9]]) * math.pi / 1e-3
    want = O.solve_bands(med, ks, 6, 1e-12, 1e-12, method="lanczos").omega
    lp = B.LearnedPrecond(seed=9)
    plan0 = B.Plan.from_problem(p, precision=1)
    lp.collect(plan0, ks, n_rhs=2, n_iters=6, seed=3)
    lp.train(50, lr=3e-3)
    for prec, bar, opt in ((1, 1e-6, dict(tol_lin=1e-3, tol_eig=1e-6)), (0, 1e-9, dict(tol_lin=1e-10, tol_eig=1e-11))):
        plan = B.Plan.from_problem(p, precision=prec, **opt)
        B.set_preconditioner(plan, lp)
        got, _, _ = plan.solve_bands(ks, 6)
        assert np.max(np.abs(got / want - 1)) < bar


def _scaled_units(p):
    """The library's internal units: q~ = q * L_max / (2 pi), C~ = C0 / C_ref with
    C_ref the largest diagonal entry of C0; K~ = K / K_scale, K_scale = C_ref / qscale^2."""
    med = O.Medium.from_problem(p)
    qscale = max(p.L) / (2 * math.pi)
    Cref = max(med.C0[0, 0, 0, 0], med.C0[1, 1, 1, 1], med.C0[2, 2, 2, 2])
    return med, qscale, med.C0 / Cref, Cref / qscale ** 2


@pytest.mark.parametrize("grid", [(9, 7, 5), (8, 6, 4), (16, 12, 10)])
def test_trained_network_inference_matches_oracle(B, grid):
    """Inference with non-trivial parameters (g far from 1, different per
    branch): the library's Z tables applied by bloch_apply_precond against the
    oracle's Z_of at every Fourier bin, odd and even grids (Nyquist bins), a
    general wave vector and k = 0 (bin 0 maps to zero)."""
    p = synth.small_polycrystal(grid, 5, 13)
    plan = B.Plan.from_problem(p, precision=1)
    lp = B.LearnedPrecond(seed=11)
    theta = lp.params()
    rng = np.random.default_rng(grid[0])
    nh = H * 5 + H + H * H + H
    theta[:nh] = rng.uniform(-0.9, 0.9, nh)
    theta[nh:nh + H] = rng.uniform(-1.0, 1.0, H)
    theta[-1] = 0.3
    lp.params(set_to=theta)
    theta = lp.params()          # the FP32 values in use
    B.set_preconditioner(plan, lp)
    ks = np.array([[0.31, -0.17, 0.42], [0.0, 0.0, 0.0]]) * math.pi / 1e-3
    r = synth.random_field(p.grid, 8, batch=2)
    z = to_dev(np.zeros_like(r))
    plan.apply_precond(ks, to_dev(r), z)
    got = z.cpu().numpy().astype(np.complex128)
    r32 = r.astype(np.complex64).astype(np.complex128)
    med, qscale, C0s, Kscale = _scaled_units(p)
    Nmax = max(grid)
    g_all = []
    for b in range(2):
        qv = np.stack([np.broadcast_to(med.q(ks[b])[j], med.shape[1:]) for j in range(3)], -1).reshape(-1, 3)
        qv = qv * qscale
        nz = np.einsum("nj,nj->n", qv, qv) > 0
        Z = np.zeros((qv.shape[0], 3, 3))
        Z[nz] = OL.Z_of(theta, H, qv[nz], C0s, Nmax)
        rb = r32[b].reshape(3, -1).T
        want = np.einsum("nij,nj->ni", Z, rb) / Kscale
        gb = got[b].reshape(3, -1).T
        assert np.all(gb[~nz] == 0)
        # per voxel, relative to |Z| |r| at that voxel (small and large |q| alike)
        scale = np.linalg.norm(Z, axis=(1, 2)) * np.linalg.norm(rb, axis=1) / Kscale
        err = np.linalg.norm(gb - want, axis=1)
        assert np.max(err[nz] / scale[nz]) < 1e-5
        assert np.linalg.norm(gb - want) <= 2e-6 * np.linalg.norm(want)
        # the network is far from the Green operator here
        g_all.append(OL.g_of(theta, H, OL.features(qv[nz], np.linalg.eigvalsh(OL.acoustic(C0s, qv[nz])), Nmax)))
    g_all = np.concatenate([g.ravel() for g in g_all])
    assert np.max(np.abs(g_all - 1.0)) > 0.3 and np.ptp(g_all) > 0.05


def test_moment_kernel_matches_oracle(B):
    """The moment kernel used by bloch_lp_collect, fed caller-supplied pairs
    through bloch_lp_add_pairs, against the oracle's moments of the same
    (FP32-rounded) pairs; a zero-residual pair is skipped."""
    import torch
    p = synth.small_polycrystal((9, 8, 6), 4, 21)
    plan = B.Plan.from_problem(p, precision=1)
    lp = B.LearnedPrecond(seed=2)
    rng = np.random.default_rng(5)
    shape = (3, 3) + tuple(reversed(p.grid))
    r = (rng.normal(size=shape) + 1j * rng.normal(size=shape)) * np.array([1.0, 3e-2, 40.0])[:, None, None, None, None]
    e = (rng.normal(size=shape) + 1j * rng.normal(size=shape)) * 0.7
    r[1] = 0.0
    r = r.astype(np.complex64)
    e = e.astype(np.complex64)
    k = np.array([0.2, -0.45, 0.1]) * math.pi / 1e-3
    lp.add_pairs(plan, k, to_dev(r), to_dev(e))
    torch.cuda.synchronize()
    assert lp.num_blocks == 1
    blk = lp.export_block(0)
    assert blk["samples"] == 2
    want = OL.moments(r.astype(np.complex128), e.astype(np.complex128))
    got = blk["mom"]
    colmax = np.max(np.abs(want), axis=0)
    assert np.all(np.abs(got - want) <= 1e-5 * colmax[None, :])
    # the block's q features are the scaled xi + k of the plan's grid
    med, qscale, _, _ = _scaled_units(p)
    qx = (med.xi[0].ravel() + k[0]) * qscale
    assert np.allclose(blk["q"][:p.grid[0]], qx, rtol=1e-6, atol=1e-6)

"""Band properties on the GPU against the FP64 oracle:

* group velocity (Section 5.1, Eq. c_group) by Hellmann-Feynman through
  bloch_group_velocity, against the oracle's Hellmann-Feynman velocities of the
  same vectors, against central differences of the oracle's bands (the
  paper's way of differentiating a branch), and against the closed form
  c (xi+k)/|xi+k| of a homogeneous isotropic medium;
* real-space eigenvector fields and their strain (Section 5.2, Eq.
  rotate_eigenvector) through bloch_eigvec_real, against the oracle.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import bloch_oracle as O
from paper_2106_12487_gb300 import synth

pytestmark = pytest.mark.gpu


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


def poly(grid, ng, seed, rho_mix=False):
    p = synth.small_polycrystal(grid, ng, seed)
    if rho_mix:
        p.rho = p.rho * (1.0 + 0.5 * np.arange(p.rho.size) / p.rho.size)
    return p


@pytest.mark.parametrize("grid,rho_mix", [((12, 10, 8), False), ((9, 8, 6), True), ((16, 16, 16), False)])
@pytest.mark.parametrize("prec", [0, 1])
def test_group_velocity_matches_oracle_hf(B, grid, rho_mix, prec):
    p = poly(grid, 6, 31, rho_mix)
    med = O.Medium.from_problem(p)
    rng = np.random.default_rng(4)
    ks = np.array([[0.41, 0.23, -0.17], [0.9, 0.0, 0.0], [0.2, 0.7, 0.55]]) * math.pi / 1e-3
    # general (not eigen) vectors: the identity holds for the Rayleigh quotient's gradient of any vector
    U = rng.normal(size=(3, 3) + tuple(reversed(grid))) + 1j * rng.normal(size=(3, 3) + tuple(reversed(grid)))
    U = U.astype(np.complex64 if prec else np.complex128).astype(np.complex128)
    plan = B.Plan.from_problem(p, precision=prec)
    om, c = plan.group_velocity(ks, to_dev(U, prec))
    for b in range(3):
        om_o, c_o = O.group_velocity_hf(med, ks[b], U[b:b + 1])
        tol = 2e-5 if prec else 1e-10
        assert abs(om[b] / om_o[0] - 1) < tol
        assert np.max(np.abs(c[b] - c_o[0])) <= tol * np.linalg.norm(c_o[0])


@pytest.mark.parametrize("rho_mix", [False, True])
def test_group_velocity_of_bands_matches_branch_differences(B, rho_mix):
    """Eigenvectors from bloch_solve_bands (FP64); their velocities against
    central differences of the dense oracle bands at k +- h e_m (simple bands)."""
    import torch
    p = poly((6, 6, 4), 3, 5, rho_mix)
    med = O.Medium.from_problem(p)
    k = np.array([0.37, 0.21, -0.29]) * math.pi / 1e-3
    nb = 9                    # one band beyond the 8 tested, so every tested band has both gaps
    plan = B.Plan.from_problem(p, precision=0, method=1, tol_lin=1e-12, tol_eig=1e-12)
    vecs = torch.zeros(nb * 3 * plan.V, dtype=torch.complex128, device="cuda")
    omega, _, st = plan.solve_bands(k[None], nb, vecs_out=vecs)
    assert st == 0
    om, c = plan.group_velocity(np.repeat(k[None], nb, 0), vecs)
    assert np.allclose(om, omega[0], rtol=1e-9)
    lam = omega[0] ** 2
    rel_gap = np.diff(lam) / lam[1:]
    simple = np.zeros(nb - 1, bool)
    simple[0] = rel_gap[0] > 1e-3
    simple[1:] = (rel_gap[:-1] > 1e-3) & (rel_gap[1:] > 1e-3)
    assert simple.sum() >= 4
    # Richardson extrapolation of two central differences (O(h^4)): near an
    # avoided crossing the O(h^2) error of one difference alone reaches 1e-6
    h = 2e-4 * math.pi / 1e-3
    c_h = O.group_velocity_fd(med, k, nb - 1, h)
    c_h2 = O.group_velocity_fd(med, k, nb - 1, h / 2)
    c_fd = (4 * c_h2 - c_h) / 3
    assert np.max(np.abs(c[:nb - 1][simple] - c_fd[simple])) <= 1e-7 * np.max(np.abs(c_fd))


@pytest.mark.parametrize("prec", [0, 1])
def test_group_velocity_homogeneous_isotropic_closed_form(B, prec):
    lam_l, mu, rho = 90e9, 40e9, 5000.0
    cL, cT = math.sqrt((lam_l + 2 * mu) / rho), math.sqrt(mu / rho)
    grid = (16, 8, 12)
    Nx, Ny, Nz = grid
    C6 = synth.isotropic_voigt(lam_l, mu)
    plan = B.Plan(grid, (1e-3, 1e-3, 1e-3), np.zeros(Nx * Ny * Nz, np.int32), C6[None], np.array([rho]),
                  B.default_options(precision=prec))
    med = O.Medium(grid, (1e-3,) * 3, np.zeros((Nz, Ny, Nx), np.int32), C6[None], np.array([rho]))
    k = np.array([0.31, 0.12, -0.44]) * math.pi / 1e-3
    U, want, ks = [], [], []
    for b in [(0, 0, 0), (3, 2, 5), (15, 7, 11)]:
        q = np.array([med.xi[0].ravel()[b[0]], med.xi[1].ravel()[b[1]], med.xi[2].ravel()[b[2]]]) + k
        qh = q / np.linalg.norm(q)
        t1 = np.cross(qh, [0.3, 0.8, -0.5])
        t1 /= np.linalg.norm(t1)
        for pol, cc in ((qh, cL), (t1, cT)):
            u = np.zeros((3, Nz, Ny, Nx), dtype=complex)
            u[:, b[2], b[1], b[0]] = pol * (0.7 - 0.4j)
            U.append(u)
            want.append(cc * qh)
            ks.append(k)
    om, c = plan.group_velocity(np.array(ks), to_dev(np.stack(U), prec))
    tol = 3e-6 if prec else 1e-12
    for i in range(len(U)):
        assert np.linalg.norm(c[i] - want[i]) <= tol * np.linalg.norm(want[i])


@pytest.mark.parametrize("grid", [(12, 10, 8), (9, 7, 5), (32, 16, 16)])
@pytest.mark.parametrize("prec", [0, 1])
def test_eigvec_real_matches_oracle(B, grid, prec):
    import torch
    p = poly(grid, 5, 17)
    med = O.Medium.from_problem(p)
    k = np.array([[0.5, 0.1, 0.3]]) * math.pi / 1e-3
    nb = 4
    plan = B.Plan.from_problem(p, precision=prec, method=1, tol_lin=1e-10 if prec == 0 else 1e-3,
                               tol_eig=1e-10 if prec == 0 else 1e-6)
    vecs = torch.zeros(nb * 3 * plan.V, dtype=torch.complex128 if prec == 0 else torch.complex64, device="cuda")
    plan.solve_bands(k, nb, vecs_out=vecs)
    ur = torch.zeros_like(vecs)
    eps = torch.zeros(nb * 6 * plan.V, dtype=vecs.dtype, device="cuda")
    phi = plan.eigvec_real(vecs, ur, eps)
    Uh = vecs.cpu().numpy().astype(np.complex128).reshape((nb, 3) + tuple(reversed(grid)))
    got_u = ur.cpu().numpy().astype(np.complex128).reshape(Uh.shape)
    got_e = eps.cpu().numpy().astype(np.complex128).reshape((nb, 6) + tuple(reversed(grid)))
    tol = 2e-5 if prec else 1e-11
    for b in range(nb):
        phi_o, U_o, E_o = O.eigvec_real(med, Uh[b])
        assert abs(np.exp(2j * phi[b]) - np.exp(2j * phi_o)) < tol
        sgn = 1.0 if np.vdot(U_o, got_u[b]).real >= 0 else -1.0   # phi is defined mod pi
        assert np.linalg.norm(got_u[b] - sgn * U_o) <= tol * np.linalg.norm(U_o)
        assert np.linalg.norm(got_e[b] - sgn * E_o) <= tol * np.linalg.norm(E_o)

"""Pins of the oracle's group velocity (Section 5.1, Eq. c_group) on the CPU.

* the derivative operator dA/dk_m (product rule on Eq. hatA) equals the central
  difference of A_k in k, which is exact because A_k is quadratic in k;
* a homogeneous isotropic medium has omega = c |xi + k| on every branch (the
  closed form of Section 4.1), so the group velocity of a plane wave is
  c (xi + k)/|xi + k| with c = c_L or c_T;
* on a small polycrystal the Hellmann-Feynman velocities of the dense
  eigenvectors equal central differences of the band frequencies (the way the
  paper differentiates a branch) to O(h^2).
"""
import math

import numpy as np
import scipy.linalg

from oracle import bloch_oracle as O
from paper_2106_12487_gb300 import synth

L3 = (1e-3, 1e-3, 1e-3)


def homog(C6, rho, grid, L=L3):
    Nx, Ny, Nz = grid
    return O.Medium(grid, L, np.zeros((Nz, Ny, Nx), np.int32), np.asarray(C6)[None], np.array([rho]))


def small_poly(grid=(4, 4, 3), ng=3, seed=9, rho_mix=False):
    p = synth.small_polycrystal(grid, ng, seed)
    rho = p.rho.copy()
    if rho_mix:
        rho = rho * (1.0 + 0.5 * np.arange(rho.size) / rho.size)
    return O.Medium(tuple(p.grid), tuple(p.L), p.grain_ids, p.C_per_grain, rho)


def test_derivative_operator_is_the_exact_central_difference():
    med = small_poly()
    rng = np.random.default_rng(3)
    U = rng.normal(size=med.shape) + 1j * rng.normal(size=med.shape)
    k = np.array([0.37, -0.21, 0.55]) * math.pi / 1e-3
    h = 0.4 * math.pi / 1e-3          # large step: A_k is quadratic, the difference is exact
    for m in range(3):
        e = np.zeros(3)
        e[m] = h
        fd = (O.apply_K(med, k + e, U) - O.apply_K(med, k - e, U)) / (2 * h)
        d = O.apply_dK(med, k, m, U)
        assert np.linalg.norm(d - fd) <= 1e-12 * np.linalg.norm(fd)
        # planted mistake: twice the first product-rule term in place of both
        # terms (equal only in the inner product with U, not as operators)
        q = med.q(k)
        first = np.zeros(U.shape, dtype=complex)
        for i in range(3):
            s1 = np.zeros(U.shape[1:], dtype=complex)
            for kk in range(3):
                for ll in range(3):
                    s1 += med.C4g[:, i, m, kk, ll][med.grain_ids] * np.fft.ifftn(q[ll] * U[kk])
            first[i] = np.fft.fftn(s1)
        assert np.linalg.norm(2 * first - fd) > 1e-3 * np.linalg.norm(fd)


def test_homogeneous_isotropic_plane_waves():
    lam_l, mu = 90e9, 40e9
    rho = 5000.0
    cL, cT = math.sqrt((lam_l + 2 * mu) / rho), math.sqrt(mu / rho)
    grid = (5, 4, 6)
    med = homog(synth.isotropic_voigt(lam_l, mu), rho, grid)
    k = np.array([0.31, 0.12, -0.44]) * math.pi / 1e-3
    for b in [(0, 0, 0), (1, 3, 2), (4, 1, 5)]:
        q = np.array([med.xi[0].ravel()[b[0]], med.xi[1].ravel()[b[1]], med.xi[2].ravel()[b[2]]]) + k
        qh = q / np.linalg.norm(q)
        t1 = np.cross(qh, [0.3, 0.8, -0.5])
        t1 /= np.linalg.norm(t1)
        t2 = np.cross(qh, t1)
        for pol, c in ((qh, cL), (t1, cT), (t2, cT)):
            U = np.zeros((1,) + med.shape, dtype=complex)
            U[0, :, b[2], b[1], b[0]] = pol
            om, cg = O.group_velocity_hf(med, k, U)
            assert abs(om[0] / (c * np.linalg.norm(q)) - 1) < 1e-12
            assert np.allclose(cg[0], c * qh, rtol=0, atol=1e-10 * c)


def test_hellmann_feynman_equals_branch_differences_polycrystal():
    for rho_mix in (False, True):
        med = small_poly(rho_mix=rho_mix)
        k = np.array([0.41, 0.23, -0.17]) * math.pi / 1e-3
        K = O.dense_K(med, k)
        M = O.dense_M(med)
        lam, W = scipy.linalg.eigh(K, M, subset_by_index=(0, 7))
        simple = np.ones(8, bool)
        rel_gap = np.diff(lam) / lam[1:]
        simple[:-1] &= rel_gap > 1e-3
        simple[1:] &= rel_gap > 1e-3
        U = W.T.reshape((8,) + med.shape)
        om, c_hf = O.group_velocity_hf(med, k, U)
        assert np.allclose(om, np.sqrt(lam), rtol=1e-10)
        h = 1e-4 * math.pi / 1e-3         # O(h^2) truncation ~1e-7, rounding ~1e-10 relative
        c_fd = O.group_velocity_fd(med, k, 8, h)
        scale = np.max(np.abs(c_hf))
        assert simple.sum() >= 4
        assert np.max(np.abs(c_fd[simple] - c_hf[simple])) <= 1e-6 * scale


# ------------------------------------------------ Eq. (rotate_eigenvector)
def test_eigvec_real_recovers_a_single_phase_field():
    """A field whose points share one phase phi0 (U = e^{i phi0} R, R real) is
    rotated back to R (up to the sign that any eigenvector has), and
    phi = phi0 mod pi."""
    med = small_poly((6, 5, 4))
    rng = np.random.default_rng(11)
    R = rng.normal(size=med.shape)
    for phi0 in (0.3, -1.2, 2.9):
        U_hat = np.fft.fftn(np.exp(1j * phi0) * R, axes=(-3, -2, -1))
        phi, U, _ = O.eigvec_real(med, U_hat)
        d = (phi - phi0) / math.pi
        assert abs(d - round(d)) < 1e-12
        sgn = np.sign(np.vdot(R, U.real))
        assert np.max(np.abs(U - sgn * R)) < 1e-12 * np.max(np.abs(R))


def test_eigvec_real_phase_is_the_least_squares_phase():
    med = small_poly((5, 4, 3))
    rng = np.random.default_rng(12)
    U_hat = rng.normal(size=med.shape) + 1j * rng.normal(size=med.shape)
    phi, U, _ = O.eigvec_real(med, U_hat)
    w = np.fft.ifftn(U_hat, axes=(-3, -2, -1))
    best = np.linalg.norm(U.real)
    for psi in np.linspace(-math.pi, math.pi, 721):
        assert np.linalg.norm((np.exp(-1j * psi) * w).real) <= best * (1 + 1e-12)


def test_eigvec_real_strain_of_a_plane_wave():
    """One Fourier bin m with polarisation p: U(x_n) = p e^{i xi.x_n}/V on the
    grid points x_n = n L/N, so eps_ij = (i/2)(xi_j p_i + xi_i p_j) e^{i xi.x_n}/V,
    rotated by the same phase -- written here from the definition."""
    grid = (6, 5, 4)
    med = small_poly(grid)
    Nx, Ny, Nz = grid
    pol = np.array([0.6, -0.3, 0.74])
    for b in [(1, 0, 0), (2, 3, 1), (3, 2, 2)]:
        U_hat = np.zeros(med.shape, dtype=complex)
        U_hat[:, b[2], b[1], b[0]] = pol
        phi, U, eps = O.eigvec_real(med, U_hat)
        xi = np.array([med.xi[0].ravel()[b[0]], med.xi[1].ravel()[b[1]], med.xi[2].ravel()[b[2]]])
        z, y, x = np.meshgrid(np.arange(Nz) * 1e-3 / Nz, np.arange(Ny) * 1e-3 / Ny, np.arange(Nx) * 1e-3 / Nx,
                              indexing="ij")
        wave = np.exp(1j * (xi[0] * x + xi[1] * y + xi[2] * z)) / (Nx * Ny * Nz) * np.exp(-1j * phi)
        pairs = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
        for c, (i, j) in enumerate(pairs):
            want = 0.5j * (xi[j] * pol[i] + xi[i] * pol[j]) * wave
            assert np.max(np.abs(eps[c] - want)) <= 1e-12 * np.max(np.abs(xi)) / (Nx * Ny * Nz)
        for i in range(3):
            assert np.max(np.abs(U[i] - pol[i] * wave)) < 1e-14


# ---------------------------------------------------------------------------
# Wave speeds (Section 5.2, Eq. wave_speed2)
# ---------------------------------------------------------------------------
def christoffel_speeds(C6, rho, d):
    """sqrt of the eigenvalues of the Christoffel matrix G_ik = C_ijkl d_j d_l / rho
    of a homogeneous crystal (the closed form of plane waves, Eq. wave_speed for
    general anisotropy), from the Voigt matrix through the full tensor."""
    idx = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (1, 2): 3, (2, 1): 3, (0, 2): 4, (2, 0): 4, (0, 1): 5, (1, 0): 5}
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[i, j, k, l] = C6[idx[(i, j)], idx[(k, l)]]
    d = np.asarray(d, float) / np.linalg.norm(d)
    G = np.einsum("ijkl,j,l->ik", C, d, d) / rho
    return np.sqrt(np.linalg.eigvalsh(G))


def test_wave_speeds_isotropic_and_cubic_closed_forms():
    rho = 8960.0
    iso = synth.isotropic_voigt(90e9, 40e9)
    ws = O.wave_speeds(homog(iso, rho, (4, 4, 3)), [0.3, -0.5, 0.8])
    cT, cL = math.sqrt(40e9 / rho), math.sqrt(170e9 / rho)
    assert np.allclose(ws, [cT, cT, cL], rtol=1e-9)
    C11, C12, C44 = 168.4e9, 121.4e9, 75.4e9
    cub = synth.cubic_voigt(C11, C12, C44)
    med = homog(cub, rho, (4, 3, 4))
    # [100]: two transverse branches at sqrt(C44/rho), longitudinal sqrt(C11/rho)
    assert np.allclose(O.wave_speeds(med, [1, 0, 0]),
                       [math.sqrt(C44 / rho), math.sqrt(C44 / rho), math.sqrt(C11 / rho)], rtol=1e-9)
    # [110]: split transverse pair; a slope taken along x instead of d fails here
    want = sorted([math.sqrt(C44 / rho), math.sqrt((C11 - C12) / (2 * rho)),
                   math.sqrt((C11 + C12 + 2 * C44) / (2 * rho))])
    got = O.wave_speeds(med, [1, 1, 0])
    assert np.allclose(got, want, rtol=1e-9)
    assert not np.allclose(got / math.sqrt(2.0), want, rtol=1e-3)


def test_wave_speeds_rotated_hexagonal_crystal_christoffel():
    rho = 4506.0
    hx = synth.hexagonal_voigt(162e9, 92e9, 69e9, 181e9, 46.7e9)
    R = synth.haar_rotations(1, 23)[0]
    C6 = synth.rotate_voigt(hx, R)
    med = homog(C6, rho, (3, 4, 4))
    for d in ([0.2, 0.9, -0.4], [1.0, 0.0, 0.0], [0.0, 0.3, 1.0]):
        assert np.allclose(O.wave_speeds(med, d), christoffel_speeds(C6, rho, d), rtol=1e-8)


def test_wave_speeds_polycrystal_equal_branch_slopes():
    """On a polycrystal the Hellmann-Feynman slopes along d equal central
    differences of the three lowest frequencies along d at k = K d (the paper
    differentiates the branch numerically near the origin)."""
    import scipy.linalg
    med = small_poly()
    d = np.array([0.0, 0.0, 1.0])
    K = 0.02 * math.pi / 1e-3
    ws = O.wave_speeds(med, d, K)
    Md = O.dense_M(med)

    def om3(kk):
        lam = scipy.linalg.eigh(O.dense_K(med, kk), Md, eigvals_only=True, subset_by_index=(0, 2))
        return np.sqrt(lam)

    h = 0.1 * K
    fd = (om3((K + h) * d) - om3((K - h) * d)) / (2 * h)
    assert np.all(np.diff(ws) >= 0) or np.all(np.abs(np.diff(ws)) < 1e-3 * ws[2])
    assert np.allclose(ws, fd, rtol=1e-5)
    # the low-frequency limit: the secant omega(K)/K agrees to O(K^2)
    assert np.allclose(om3(K * d) / K, ws, rtol=1e-3)

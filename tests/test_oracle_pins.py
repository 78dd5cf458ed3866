"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them re-types the oracle's own
formula: they use closed forms (Section 4.1 Eq. anal_eigen_3D, Section 3.3
explicit 1D inverse, Section 4.2 Eq. laminate), exact invariances, variational
bounds, and LAPACK/ARPACK on assembled matrices.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import bloch_oracle as O
from oracle import closed_forms as CF
from paper_2106_12487_gb300 import synth

L3 = (1e-3, 1e-3, 1e-3)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def table1():
    with open(os.path.join(GOLDEN, "table1_composites.json")) as f:
        return json.load(f)


def paper_freqs(N, L=1e-3):
    """The set of Eq. (frequencies), written from the paper (not from the oracle)."""
    shift = N / 2 if N % 2 == 0 else (N - 1) / 2
    return 2 * math.pi / L * (np.arange(N) - shift)


def homog(C6, rho, grid, L=L3):
    Nx, Ny, Nz = grid
    return O.Medium(grid, L, np.zeros((Nz, Ny, Nx), np.int32), np.asarray(C6)[None], np.array([rho]))


def dense_eigs(med, k):
    K = O.dense_K(med, k)
    M = O.dense_M(med)
    return scipy.linalg.eigh(K, M, eigvals_only=True), K, M


# ----------------------------------------------------------------- Eq. frequencies
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 16])
def test_frequency_set_matches_paper(N):
    """Eq. (frequencies): the bins carry 2pi/L (m - N/2) (even N) or
    2pi/L (m - (N-1)/2) (odd N), m = 0..N-1, as a set; bin 0 carries xi = 0."""
    L = 2.5e-3
    xi = O.frequencies(N, L)
    shift = N / 2 if N % 2 == 0 else (N - 1) / 2
    paper = 2 * math.pi / L * (np.arange(N) - shift)
    assert np.allclose(np.sort(xi), np.sort(paper), rtol=0, atol=1e-9)
    assert xi[0] == 0.0
    # consecutive bins step by +2pi/L except at the single wrap
    assert np.sum(np.diff(xi) < 0) == (1 if N > 2 else (1 if N == 2 else 0))


# ----------------------------------------------------- Eq. anal_eigen_3D (homogeneous)
@pytest.mark.parametrize("grid,kfrac", [
    ((4, 4, 4), (0.3, 0.1, -0.2)),
    ((4, 4, 4), (1.0, 0.0, 0.0)),       # X point: the Nyquist bin enters the low spectrum
    ((4, 4, 4), (1.0, 1.0, 1.0)),       # R point
    ((6, 4, 5), (0.41, -0.73, 0.22)),   # non-cubic, odd and even axes
    ((6, 1, 1), (0.5, 0.0, 0.0)),       # 1D grid of Section 4.1 (6 points)
    ((4, 4, 1), (0.5, 0.5, 0.0)),       # 2D grid of Section 4.1 (4x4 points)
])
def test_homogeneous_isotropic_full_spectrum(grid, kfrac):
    """Section 4.1: with constant C, rho the whole discrete spectrum is
    {eig(P(xi + k))/rho : xi} (longitudinal c_L^2 |q|^2, transverse c_T^2 |q|^2 x2)."""
    C = synth.isotropic_from_E_nu(4.507e9, 0.4)   # epoxy, Table 1
    rho = 1200.0
    med = homog(C, rho, grid)
    k = np.array(kfrac) * math.pi / 1e-3
    lam, K, M = dense_eigs(med, k)
    # closed form for an isotropic solid: c_L^2 |q|^2 and c_T^2 |q|^2 (twice)
    lamb, mu = C[0, 1], C[5, 5]
    cL2, cT2 = (lamb + 2 * mu) / rho, mu / rho
    Nx, Ny, Nz = grid
    xs = [paper_freqs(n) for n in grid]
    ref = []
    for a in xs[2]:
        for b in xs[1]:
            for c in xs[0]:
                q2 = (c + k[0]) ** 2 + (b + k[1]) ** 2 + (a + k[2]) ** 2
                ref += [cL2 * q2, cT2 * q2, cT2 * q2]
    ref = np.sort(ref)
    assert np.max(np.abs(lam - ref)) <= 1e-11 * ref.max()


def test_rotated_cubic_single_crystal_christoffel():
    """Eq. (anal_eigen_3D) with an anisotropic rotated cubic C: the spectrum is
    the union of the Christoffel eigenvalues; and omega(R C R^T, q) = omega(C, R^T q)."""
    C = synth.cubic_voigt(168.4e9, 121.4e9, 75.4e9)
    R = synth.haar_rotations(1, 5)[0]
    Cr = synth.rotate_voigt(C, R)
    grid = (4, 4, 4)
    k = np.array([0.37, -0.21, 0.66]) * math.pi / 1e-3
    lam, _, _ = dense_eigs(homog(Cr, 8960.0, grid), k)
    # Christoffel with the unrotated crystal and rotated wave vectors
    Nx, Ny, Nz = grid
    xs = [paper_freqs(n) for n in grid]
    C4 = O.voigt_to_tensor(C)
    ref = []
    for a in xs[2]:
        for b in xs[1]:
            for c in xs[0]:
                q = np.array([c + k[0], b + k[1], a + k[2]])
                qc = R.T @ q
                G = np.einsum("ijkl,j,l->ik", C4, qc, qc)
                ref += list(np.linalg.eigvalsh(G) / 8960.0)
    ref = np.sort(ref)
    assert np.max(np.abs(lam - ref)) <= 1e-11 * ref.max()


# ------------------------------------------------------ Hermitian / PSD (Section 3.2)
def test_operators_hermitian_and_psd():
    """Section 3.2: A_k and M are Hermitian; A_k is positive semidefinite."""
    p = synth.small_polycrystal((6, 4, 5), 6, 11)
    med = O.Medium.from_problem(p)
    k = np.array([0.3, -0.6, 0.45]) * math.pi / 1e-3
    u = synth.random_field(p.grid, 1)
    v = synth.random_field(p.grid, 2)
    Ku, Kv = O.apply_K(med, k, u), O.apply_K(med, k, v)
    a, b = O.vdot(v, Ku), np.conj(O.vdot(u, Kv))
    assert abs(a - b) <= 1e-12 * abs(a)
    Mu, Mv = O.apply_M(med, u), O.apply_M(med, v)
    assert abs(O.vdot(v, Mu) - np.conj(O.vdot(u, Mv))) <= 1e-12 * abs(O.vdot(v, Mu))
    for s in range(5):
        w = synth.random_field(p.grid, 100 + s)
        assert O.vdot(w, O.apply_K(med, k, w)).real > 0
        assert abs(O.vdot(w, O.apply_K(med, k, w)).imag) <= 1e-12 * O.vdot(w, O.apply_K(med, k, w)).real


def test_gamma_three_zero_eigenvalues():
    """k = 0: the rigid translations (bin 0) are the only null vectors of A_0
    (Section 3.3 states invertibility only for k != 0)."""
    p = synth.small_polycrystal((4, 4, 4), 5, 3)
    med = O.Medium.from_problem(p)
    lam, K, _ = dense_eigs(med, np.zeros(3))
    scale = lam.max()
    assert np.sum(np.abs(lam) < 1e-12 * scale) == 3
    assert lam[3] > 1e-4 * scale
    # A_0 on a bin-0 field is exactly zero
    u = np.zeros(med.shape, complex)
    u[:, 0, 0, 0] = [1.0, 2.0 - 1j, 0.5j]
    assert O.norm(O.apply_K(med, np.zeros(3), u)) == 0.0


# --------------------------------------------------------------- PCG (Algorithm 2)
def test_pcg_homogeneous_converges_in_one_iteration():
    """Eq. (precond): with C0 = C (homogeneous cell) P^-1 is the exact inverse,
    so PCG stops after one iteration."""
    C = synth.rotate_voigt(synth.cubic_voigt(168.4e9, 121.4e9, 75.4e9), synth.haar_rotations(1, 9)[0])
    med = homog(C, 8960.0, (6, 6, 6))
    k = np.array([0.2, 0.1, 0.7]) * math.pi / 1e-3
    b = synth.random_field(med.grid, 4)
    res = O.pcg(lambda x: O.apply_K(med, k, x), lambda x: O.apply_precond(med, k, x), b, 1e-12, 50)
    assert res.iters == 1
    assert res.true_rel_res < 1e-13


def test_explicit_1d_inverse_laminate():
    """Section 3.3: in 1D the inverse is (xi+k)^-1 F{E^-1 F^-1[(xi+k)^-1 Y]};
    on an N x 1 x 1 epoxy/carbon bilayer with k along x it must invert A_k for
    the longitudinal (E -> C11) and transverse (E -> C66, C55) components, and
    PCG must converge to the same field."""
    t = table1()["composite1"]
    ep = synth.isotropic_from_E_nu(t["matrix"]["E_Pa"], t["matrix"]["nu"])
    ca = synth.isotropic_from_E_nu(t["particles"]["E_Pa"], t["particles"]["nu"])
    N = 32
    ids = synth.laminate_ids((N, 1, 1))
    med = O.Medium((N, 1, 1), L3, ids, np.stack([ep, ca]),
                   np.array([t["matrix"]["rho"], t["particles"]["rho"]]))
    k = np.array([0.37 * math.pi / 1e-3, 0.0, 0.0])
    Cv = np.stack([ep, ca])[ids]
    for comp, (a, b) in [(0, (0, 0)), (1, (5, 5)), (2, (4, 4))]:
        Y = np.zeros(med.shape, complex)
        Y[comp] = synth.random_field((N, 1, 1), 20 + comp, ncomp=1)[0]
        X = CF.explicit_inverse_1d(med, k, Y, comp, Cv[..., a, b])
        assert O.norm(O.apply_K(med, k, X) - Y) <= 1e-12 * O.norm(Y)
        res = O.pcg(lambda x: O.apply_K(med, k, x), lambda x: O.apply_precond(med, k, x), Y, 1e-13)
        assert O.norm(res.x - X) <= 1e-10 * O.norm(X)


# --------------------------------------------------------------- Eq. laminate (Rytov)
def test_rytov_bilayer_convergence():
    """Section 4.2, Eq. (laminate) with the minus sign: the longitudinal bands of
    the epoxy/carbon bilayer converge to the analytical roots as N grows
    (quadratically: the error falls ~4x per doubling)."""
    t = table1()["composite1"]
    ep = synth.isotropic_from_E_nu(t["matrix"]["E_Pa"], t["matrix"]["nu"])
    ca = synth.isotropic_from_E_nu(t["particles"]["E_Pa"], t["particles"]["nu"])
    rho = np.array([t["matrix"]["rho"], t["particles"]["rho"]])
    L = 1e-3
    kx = 0.6 * math.pi / L
    M1, M2 = ep[0, 0], ca[0, 0]
    c1, c2 = math.sqrt(M1 / rho[0]), math.sqrt(M2 / rho[1])
    p = math.sqrt(M2 * rho[1] / (M1 * rho[0]))
    ref = CF.rytov_frequencies(kx * L, c1, c2, p, L, 4)
    errs = []
    for N in (16, 32, 64):
        med = O.Medium((N, 1, 1), (L, L, L), synth.laminate_ids((N, 1, 1)), np.stack([ep, ca]), rho)
        K = O.dense_K(med, [kx, 0, 0])[:N, :N]
        M = O.dense_M(med)[:N, :N]
        w = np.sqrt(scipy.linalg.eigh(K, M, eigvals_only=True)[:4])
        errs.append(np.max(np.abs(w / ref - 1)))
    assert errs[0] < 1e-2
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3
    # the printed '+' sign would not reduce to the homogeneous limit
    hom = CF.rytov_frequencies(kx * L, c1, c1, 1.0, L, 2)
    assert np.allclose(hom, [c1 * kx, c1 * (2 * math.pi / L - kx)], rtol=1e-9)


# ----------------------------------------------------------------------- invariances
def test_invariances_translation_scaling_permutation():
    """Exact invariances of the spectrum: cyclic translation of the cell;
    C -> sC scales lambda by s; rho -> s rho scales lambda by 1/s; permuting the
    axes of a cubic grid together with C and k."""
    p = synth.small_polycrystal((4, 4, 4), 5, 21)
    med = O.Medium.from_problem(p)
    k = np.array([0.31, 0.52, -0.17]) * math.pi / 1e-3
    lam0, _, _ = dense_eigs(med, k)
    scale = lam0.max()
    # translation
    ids_t = np.roll(p.grain_ids, (1, 3, 2), axis=(0, 1, 2))
    lam_t, _, _ = dense_eigs(O.Medium(p.grid, p.L, ids_t, p.C_per_grain, p.rho), k)
    assert np.max(np.abs(lam_t - lam0)) <= 1e-11 * scale
    # stiffness and density scaling
    lam_c, _, _ = dense_eigs(O.Medium(p.grid, p.L, p.grain_ids, 3.0 * p.C_per_grain, p.rho), k)
    assert np.max(np.abs(lam_c - 3.0 * lam0)) <= 3e-11 * scale
    lam_r, _, _ = dense_eigs(O.Medium(p.grid, p.L, p.grain_ids, p.C_per_grain, 2.0 * p.rho), k)
    assert np.max(np.abs(lam_r - lam0 / 2.0)) <= 1e-11 * scale
    # axis permutation x<->z (ids stored [z][y][x]) with C and k permuted
    Pm = np.array([[0, 0, 1], [0, 1, 0], [1, 0, 0]], float)
    ids_p = np.transpose(p.grain_ids, (2, 1, 0)).copy()
    C_p = np.stack([synth.rotate_voigt(C, Pm) for C in p.C_per_grain])
    lam_p, _, _ = dense_eigs(O.Medium(p.grid, p.L, ids_p, C_p, p.rho), Pm @ k)
    assert np.max(np.abs(lam_p - lam0)) <= 1e-11 * scale


def test_poincare_bound_from_plane_waves():
    """Courant-Fischer: the three lowest eigenvalues lie below the Ritz values of
    the plane waves e_c at bin 0, i.e. eig(P(k) with volume-averaged C)/rho_bar."""
    p = synth.small_polycrystal((6, 6, 6), 7, 31)
    med = O.Medium.from_problem(p)
    for kf in ([0.2, 0.0, 0.0], [0.5, 0.5, 0.0], [0.3, 0.7, 0.9]):
        k = np.array(kf) * math.pi / 1e-3
        res = O.lanczos_irl(med, k, 3, 1e-12, 1e-12)
        P = O.acoustic_tensor(med.C0, k[None])[0]
        ritz = np.linalg.eigvalsh(P) / med.rho_bar
        assert np.all(res.lam <= ritz * (1 + 1e-10))


# ---------------------------------------------------------------------- eigensolvers
@pytest.mark.parametrize("kf", [(0.5, 0.2, 0.1), (1.0, 0.0, 0.0), (0.0, 0.0, 0.0)])
def test_solvers_match_dense_lapack(kf):
    """Algorithm 1 (subspace iteration) and shift-invert IRL (Section 3.3) give the
    lowest eigenvalues of the assembled pencil (LAPACK), including at Gamma."""
    p = synth.small_polycrystal((4, 4, 4), 5, 7)
    med = O.Medium.from_problem(p)
    k = np.array(kf) * math.pi / 1e-3
    lam, _, _ = dense_eigs(med, k)
    n = 6
    for method in ("subspace", "lanczos"):
        b = O.solve_bands(med, k[None], n, 1e-12, 1e-11, method=method)
        ref = np.where(np.abs(lam[:n]) < 1e-12 * lam.max(), 0.0, lam[:n])
        assert np.allclose(b.lam[0], ref, rtol=1e-9, atol=1e-12 * lam.max()), method


def test_nonuniform_density_gamma_deflation():
    """Two densities: the Gamma-point complement solve (M-orthogonal to the rigid
    translations) reproduces the dense pencil's non-zero eigenvalues."""
    p = synth.small_polycrystal((4, 4, 4), 4, 41)
    rho = np.array([8960.0, 2000.0, 5000.0, 12000.0])
    med = O.Medium(p.grid, p.L, p.grain_ids, p.C_per_grain, rho)
    lam, _, _ = dense_eigs(med, np.zeros(3))
    b = O.solve_bands(med, np.zeros((1, 3)), 6, 1e-12, 1e-11, method="subspace")
    assert np.allclose(b.lam[0, 3:], lam[3:6], rtol=1e-9)


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant plausible mistakes in the oracle and check that a pin fails:
    a flipped Bloch shift (xi - k), a dropped Nyquist wrap (fftshift order) and
    a transposed stiffness contraction (C_ikjl)."""
    C = synth.rotate_voigt(synth.cubic_voigt(168.4e9, 121.4e9, 75.4e9), synth.haar_rotations(1, 2)[0])
    grid = (4, 4, 4)
    k = np.array([0.37, -0.21, 0.66]) * math.pi / 1e-3
    ref = CF.homogeneous_spectrum(C, 8960.0, grid, L3, k)

    def spectrum():
        return scipy.linalg.eigh(O.dense_K(homog(C, 8960.0, grid), k), O.dense_M(homog(C, 8960.0, grid)),
                                 eigvals_only=True)

    assert np.max(np.abs(spectrum() - ref)) <= 1e-11 * ref.max()
    orig_q = O.Medium.q
    monkeypatch.setattr(O.Medium, "q", lambda self, kk: orig_q(self, -np.asarray(kk)))
    # closed form evaluated with the original k must now disagree (k not symmetric)
    bad = spectrum()
    assert np.max(np.abs(bad - ref)) > 1e-6 * ref.max()
    monkeypatch.setattr(O.Medium, "q", orig_q)

    # A cyclic relabelling of the bins leaves every spectrum unchanged (it is a
    # real-space modulation, which commutes with a diagonal C(x)); what the
    # spectrum does see is the window of Eq. (frequencies).  Plant the even-N
    # Nyquist bin at +N pi/L instead of -N pi/L and probe at the X point.
    kX = np.array([1.0, 0.0, 0.0]) * math.pi / 1e-3
    refX = np.sort(np.concatenate([
        np.linalg.eigvalsh(np.einsum("ijkl,j,l->ik", O.voigt_to_tensor(C),
                                     np.array([c, b, a]) + kX, np.array([c, b, a]) + kX)) / 8960.0
        for a in paper_freqs(4) for b in paper_freqs(4) for c in paper_freqs(4)]))
    orig_f = O.frequencies
    monkeypatch.setattr(O, "frequencies",
                        lambda N, L: 2 * math.pi / L * np.where(np.arange(N) <= N // 2, np.arange(N),
                                                                 np.arange(N) - N))
    medX = homog(C, 8960.0, grid)
    bad = scipy.linalg.eigh(O.dense_K(medX, kX), O.dense_M(medX), eigvals_only=True)
    monkeypatch.setattr(O, "frequencies", orig_f)
    assert np.max(np.abs(bad - refX)) > 1e-6 * refX.max()
    medX = homog(C, 8960.0, grid)
    good = scipy.linalg.eigh(O.dense_K(medX, kX), O.dense_M(medX), eigvals_only=True)
    assert np.max(np.abs(good - refX)) <= 1e-11 * refX.max()

    orig_v = O.voigt_to_tensor
    monkeypatch.setattr(O, "voigt_to_tensor", lambda C6: np.transpose(orig_v(C6), (0, 2, 1, 3)))
    bad = spectrum()
    monkeypatch.setattr(O, "voigt_to_tensor", orig_v)
    assert np.max(np.abs(bad - ref)) > 1e-6 * ref.max()


# ------------------------------------- real-space basis: plane waves (Section 3.2)
@pytest.mark.parametrize("bins", [(1, 0, 0), (0, 3, 1), (5, 2, 4), (3, 0, 2)])
def test_real_space_plane_wave_is_christoffel_eigenvector(bins):
    """On grid values at the voxel centres, a plane wave e exp(i xi.x) of a
    homogeneous medium is mapped by F^-1 A_k F (numpy's FFT pair, the library's
    real-space convention) to (P(xi + k) e) exp(i xi.x), with the Christoffel
    matrix P written here from C and xi taken from the paper's frequency set in
    FFT bin order (negative half above N/2; the even-N Nyquist bin at -N pi/L)."""
    C = synth.rotate_voigt(synth.cubic_voigt(168.4e9, 121.4e9, 75.4e9), synth.haar_rotations(1, 9)[0])
    grid = (6, 4, 5)
    med = homog(C, 8960.0, grid)
    k = np.array([0.31, -0.47, 0.22]) * math.pi / 1e-3
    Nx, Ny, Nz = grid
    xi = []
    for m, n in zip(bins, grid):
        f = np.sort(paper_freqs(n))          # the paper's set
        xi.append(f[f >= 0][m] if m < (n + 1) // 2 else f[f < 0][m - (n + 1) // 2])
    xi = np.array(xi)
    xs = [(0.5 + np.arange(n)) * 1e-3 / n for n in grid]
    X, Y, Z = xs[0][None, None, :], xs[1][None, :, None], xs[2][:, None, None]
    phase = np.exp(1j * (xi[0] * X + xi[1] * Y + xi[2] * Z))
    e = np.array([0.3 - 0.2j, 1.0, -0.5 + 0.7j])
    u = e[:, None, None, None] * phase[None]
    ax = (-3, -2, -1)
    Ku = np.fft.ifftn(O.apply_K(med, k, np.fft.fftn(u, axes=ax)), axes=ax)
    q = xi + k
    P = np.einsum("ijkl,j,l->ik", O.voigt_to_tensor(C), q, q)
    want = (P @ e)[:, None, None, None] * phase[None]
    assert np.linalg.norm(Ku - want) <= 1e-12 * np.linalg.norm(want)

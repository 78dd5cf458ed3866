"""Closed forms the paper states, used to pin the oracle (test infrastructure).

  * homogeneous_spectrum: Eq. (anal_eigen_3D) -- for constant C and rho, each
    Fourier voxel xi contributes the three eigenvalues of P(xi + k)/rho with
    P_ik = C_ijkl (xi+k)_j (xi+k)_l (Section 4.1).
  * explicit_inverse_1d: the 1D inverse operator of Section 3.3,
    A_k^-1 Y = (xi+k)^-1 F{ E^-1 F^-1[(xi+k)^-1 Y] }.
  * rytov_frequencies: the bilayer dispersion relation of Eq. (laminate) with
    the sign read as minus (the homogeneous limit p = 1, c1 = c2 forces
    cos kL = cos(a + b); with the printed plus it would give 1).
"""
from __future__ import annotations

import math

import numpy as np

from .bloch_oracle import Medium, acoustic_tensor, frequencies, voigt_to_tensor


def homogeneous_spectrum(C6: np.ndarray, rho: float, grid, L, k) -> np.ndarray:
    """All eigenvalues lambda = omega^2 of the discrete problem for a homogeneous
    medium, ascending (3V values)."""
    Nx, Ny, Nz = grid
    C4 = voigt_to_tensor(np.asarray(C6, float))
    xs = [frequencies(Nx, L[0]), frequencies(Ny, L[1]), frequencies(Nz, L[2])]
    out = []
    for xz in xs[2]:
        for xy in xs[1]:
            for xx in xs[0]:
                qv = np.array([xx + k[0], xy + k[1], xz + k[2]])
                P = acoustic_tensor(C4, qv[None])[0]
                out.extend(np.linalg.eigvalsh(P) / rho)
    return np.sort(np.asarray(out))


def explicit_inverse_1d(med: Medium, k, Y: np.ndarray, comp: int, modulus) -> np.ndarray:
    """Explicit 1D inverse for a cell varying along x only, wave vector along x.

    `comp` is the displacement component carried (0: longitudinal, 1/2:
    transverse); `modulus` is the per-voxel 1D stiffness (C11 for comp 0, C66
    for comp 1, C55 for comp 2).  Y has shape (3, Nz, Ny, Nx) and only Y[comp]
    is used; the result is zero elsewhere.
    """
    qx = med.xi[0] + float(k[0])
    out = np.zeros_like(Y)
    inner = np.fft.ifftn(Y[comp] / qx, axes=(-3, -2, -1))
    out[comp] = np.fft.fftn(inner / modulus, axes=(-3, -2, -1)) / qx
    return out


def rytov_frequencies(kL: float, c1: float, c2: float, p: float, L: float,
                      n_roots: int, omega_max: float | None = None) -> np.ndarray:
    """The n_roots smallest omega >= 0 with
    cos(kL) = cos(a)cos(b) - (1+p^2)/(2p) sin(a) sin(b),  a = omega L/(2 c1), b = omega L/(2 c2).
    Roots are bracketed on a fine grid and refined by bisection."""
    def f(w):
        a = w * L / (2 * c1)
        b = w * L / (2 * c2)
        return math.cos(a) * math.cos(b) - (1 + p * p) / (2 * p) * math.sin(a) * math.sin(b) - math.cos(kL)

    if omega_max is None:
        omega_max = 4.0 * math.pi * (n_roots + 2) * max(c1, c2) / L
    grid = np.linspace(0.0, omega_max, 400000)
    vals = np.array([f(w) for w in grid])
    roots = []
    for i in range(len(grid) - 1):
        if vals[i] == 0.0:
            roots.append(grid[i])
        elif vals[i] * vals[i + 1] < 0.0:
            lo, hi = grid[i], grid[i + 1]
            flo = vals[i]
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                fm = f(mid)
                if flo * fm <= 0.0:
                    hi = mid
                else:
                    lo, flo = mid, fm
            roots.append(0.5 * (lo + hi))
        if len(roots) >= n_roots:
            break
    return np.asarray(roots[:n_roots])

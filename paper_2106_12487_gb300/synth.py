"""Seeded synthetic inputs: voxelised polycrystals, crystal orientations, k-paths.

This module builds the *inputs* of the Bloch-wave dispersion problem and holds
none of the method's arithmetic (no Fourier operators, no solvers).  Both the
CUDA path and the FP64 CPU oracle consume what it produces, so every array it
returns is plain numpy.

What it stands in for (Section 5 of the paper, 3D polycrystal RVEs): the paper
builds its RVEs with a weighted Voronoi tool and draws orientations from a
random or fibre ODF; here periodic Voronoi tessellations with uniform seeds,
Haar-uniform orientations and a von Mises-Fisher <001> fibre are generated from
fixed seeds, with the grid sizes, grain counts and cubic/hexagonal stiffnesses of
the workloads the project measures.

Conventions (used by every consumer):
  * grid = (Nx, Ny, Nz); arrays are stored [z][y][x] (x fastest), i.e. numpy
    shape (Nz, Ny, Nx).
  * Voigt order (11, 22, 33, 23, 13, 12) with engineering shear strain, so that
    sigma_V = C_V @ eps_V with eps_V = (e11, e22, e33, 2e23, 2e13, 2e12).
  * A rotation matrix R maps crystal coordinates to sample coordinates (its
    columns are the crystal axes written in the sample frame); the rotated
    stiffness is C'_ijkl = R_ia R_jb R_kc R_ld C_abcd.
  * SI units: Pa, kg/m^3, m, rad/m.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

VOIGT_PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def _voigt_index(i: int, j: int) -> int:
    return {(0, 0): 0, (1, 1): 1, (2, 2): 2, (1, 2): 3, (2, 1): 3,
            (0, 2): 4, (2, 0): 4, (0, 1): 5, (1, 0): 5}[(i, j)]


# --------------------------------------------------------------------------
# Single-crystal stiffness matrices (Voigt, Pa)
# --------------------------------------------------------------------------
def cubic_voigt(C11: float, C12: float, C44: float) -> np.ndarray:
    C = np.zeros((6, 6))
    C[:3, :3] = C12
    for a in range(3):
        C[a, a] = C11
        C[3 + a, 3 + a] = C44
    return C


def hexagonal_voigt(C11: float, C12: float, C13: float, C33: float, C44: float) -> np.ndarray:
    """Transversely isotropic about crystal axis 3; C66 = (C11 - C12)/2."""
    C = np.zeros((6, 6))
    C[0, 0] = C[1, 1] = C11
    C[2, 2] = C33
    C[0, 1] = C[1, 0] = C12
    C[0, 2] = C[2, 0] = C[1, 2] = C[2, 1] = C13
    C[3, 3] = C[4, 4] = C44
    C[5, 5] = 0.5 * (C11 - C12)
    return C


def isotropic_voigt(lam: float, mu: float) -> np.ndarray:
    return cubic_voigt(lam + 2.0 * mu, lam, mu)


def isotropic_from_E_nu(E: float, nu: float) -> np.ndarray:
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return isotropic_voigt(lam, mu)


def rotate_voigt(C6: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Rotate a Voigt stiffness by R (crystal -> sample) on the full 4th-order tensor."""
    C4 = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C4[i, j, k, l] = C6[_voigt_index(i, j), _voigt_index(k, l)]
    Cr = np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, C4, optimize=True)
    out = np.empty((6, 6))
    for a, (i, j) in enumerate(VOIGT_PAIRS):
        for b, (k, l) in enumerate(VOIGT_PAIRS):
            out[a, b] = Cr[i, j, k, l]
    return 0.5 * (out + out.T)


# --------------------------------------------------------------------------
# Orientations
# --------------------------------------------------------------------------
def _quat_to_matrix(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def haar_rotations(n: int, seed: int) -> np.ndarray:
    """n Haar-uniform rotations (Shoemake's uniform unit quaternions)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random((n, 3))
    out = np.empty((n, 3, 3))
    for g in range(n):
        u1, u2, u3 = u[g]
        q = np.array([math.sqrt(u1) * math.cos(2 * math.pi * u3),
                      math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
                      math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                      math.sqrt(u1) * math.sin(2 * math.pi * u3)])
        out[g] = _quat_to_matrix(q)
    return out


def vmf_fibre_rotations(n: int, kappa: float, seed: int,
                        mean_axis=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Rotations whose crystal [001] axis follows a von Mises-Fisher law about
    `mean_axis` (concentration kappa), with a uniform spin about that axis.

    The cosine w of the polar angle is drawn by inverting the vMF marginal on
    S^2 (Wood 1994, p = 3 case): w = 1 + log(u + (1-u) exp(-2 kappa)) / kappa.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = np.asarray(mean_axis, dtype=float)
    mu = mu / np.linalg.norm(mu)
    # orthonormal frame around mu
    t = np.array([1.0, 0.0, 0.0]) if abs(mu[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = t - mu * (t @ mu)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(mu, e1)
    out = np.empty((n, 3, 3))
    for g in range(n):
        u, phi, psi = rng.random(3)
        w = 1.0 + math.log(u + (1.0 - u) * math.exp(-2.0 * kappa)) / kappa
        w = min(1.0, max(-1.0, w))
        s = math.sqrt(max(0.0, 1.0 - w * w))
        d = w * mu + s * (math.cos(2 * math.pi * phi) * e1 + math.sin(2 * math.pi * phi) * e2)
        # frame around d, then spin by psi
        a = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        f1 = a - d * (a @ d)
        f1 /= np.linalg.norm(f1)
        f2 = np.cross(d, f1)
        c, sn = math.cos(2 * math.pi * psi), math.sin(2 * math.pi * psi)
        c1 = c * f1 + sn * f2
        c2 = -sn * f1 + c * f2
        out[g] = np.stack([c1, c2, d], axis=1)  # columns = crystal axes
    return out


# --------------------------------------------------------------------------
# Microstructure
# --------------------------------------------------------------------------
def voronoi_periodic(grid, n_grains: int, seed: int, L=(1e-3, 1e-3, 1e-3)) -> np.ndarray:
    """Periodic Voronoi tessellation on voxel centres x = L/N (1/2 + n).

    Seeds are uniform in the cell (PCG64(seed)); each voxel takes the grain of
    the nearest seed under the minimum-image distance.  Returns int32 ids of
    shape (Nz, Ny, Nx).
    """
    from scipy.spatial import cKDTree

    Nx, Ny, Nz = grid
    rng = np.random.Generator(np.random.PCG64(seed))
    Lv = np.asarray(L, dtype=float)
    seeds = rng.random((n_grains, 3)) * Lv
    tree = cKDTree(seeds, boxsize=Lv)
    xs = (np.arange(Nx) + 0.5) * Lv[0] / Nx
    ys = (np.arange(Ny) + 0.5) * Lv[1] / Ny
    zs = (np.arange(Nz) + 0.5) * Lv[2] / Nz
    out = np.empty((Nz, Ny, Nx), dtype=np.int32)
    X, Y = np.meshgrid(xs, ys, indexing="xy")  # (Ny, Nx)
    for iz in range(Nz):
        pts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, zs[iz])], axis=1)
        pts = np.mod(pts, Lv)
        _, idx = tree.query(pts)
        out[iz] = idx.reshape(Ny, Nx)
    return out


def laminate_ids(grid, axis: int = 0, frac: float = 0.5) -> np.ndarray:
    """Two-phase layered cell: phase 0 for x_axis < frac*L, phase 1 otherwise."""
    Nx, Ny, Nz = grid
    n = (Nx, Ny, Nz)[axis]
    pos = (np.arange(n) + 0.5) / n
    phase = (pos >= frac).astype(np.int32)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    return np.broadcast_to(phase.reshape(shape), (Nz, Ny, Nx)).astype(np.int32).copy()


# --------------------------------------------------------------------------
# Wave-vector paths
# --------------------------------------------------------------------------
def kpath(labels, n_k: int, L=(1e-3, 1e-3, 1e-3), corners: bool = False) -> np.ndarray:
    """n_k wave vectors equally spaced in arc length over the polyline through
    the named high-symmetry points (both ends included).  With corners=True
    every named point is on the list: the n_k - 1 intervals are shared among
    the segments in proportion to their lengths (largest remainders) and
    spaced evenly within each segment."""
    Lx, Ly, Lz = L
    pts = {"G": (0.0, 0.0, 0.0), "X": (math.pi / Lx, 0.0, 0.0),
           "M": (math.pi / Lx, math.pi / Ly, 0.0),
           "R": (math.pi / Lx, math.pi / Ly, math.pi / Lz),
           "Z": (0.0, 0.0, math.pi / Lz)}
    P = np.array([pts[s] for s in labels], dtype=float)
    seg = np.linalg.norm(np.diff(P, axis=0), axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    if n_k == 1:
        return P[:1].copy()
    if corners:
        nseg = len(seg)
        if n_k - 1 < nseg:
            raise ValueError("corners=True needs at least one interval per segment")
        share = (n_k - 1) * seg / cum[-1]
        cnt = np.maximum(1, np.floor(share).astype(int))
        while cnt.sum() < n_k - 1:
            cnt[np.argmax(share - cnt)] += 1
        while cnt.sum() > n_k - 1:
            cnt[np.argmax(np.where(cnt > 1, cnt - share, -np.inf))] -= 1
        out = [P[0]]
        for j in range(nseg):
            for i in range(1, cnt[j] + 1):
                out.append(P[j] + (i / cnt[j]) * (P[j + 1] - P[j]))
        return np.array(out)
    s = np.linspace(0.0, cum[-1], n_k)
    out = np.empty((n_k, 3))
    for i, si in enumerate(s):
        j = min(np.searchsorted(cum, si, side="right") - 1, len(seg) - 1)
        t = 0.0 if seg[j] == 0 else (si - cum[j]) / seg[j]
        out[i] = P[j] + t * (P[j + 1] - P[j])
    return out


# --------------------------------------------------------------------------
# Random fields for operator tests
# --------------------------------------------------------------------------
def random_field(grid, seed: int, ncomp: int = 3, batch: int | None = None) -> np.ndarray:
    """Complex Gaussian field, shape ([batch,] ncomp, Nz, Ny, Nx), complex128."""
    Nx, Ny, Nz = grid
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (ncomp, Nz, Ny, Nx) if batch is None else (batch, ncomp, Nz, Ny, Nx)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------
CU_CUBIC = dict(C11=168.4e9, C12=121.4e9, C44=75.4e9, rho=8960.0)
TI_HEX = dict(C11=162e9, C12=92e9, C13=69e9, C33=181e9, C44=46.7e9, rho=4506.0)
# Table 1 of the paper (Composite 1): epoxy matrix and carbon particles.
EPOXY = dict(E=4.507e9, nu=0.4, rho=1200.0)
CARBON = dict(E=230e9, nu=0.3, rho=1750.0)


@dataclass
class Problem:
    name: str
    grid: tuple
    L: tuple
    grain_ids: np.ndarray          # int32 (Nz, Ny, Nx)
    C_per_grain: np.ndarray        # (G, 6, 6) Pa
    rho: np.ndarray                # (G,) kg/m^3
    k_list: np.ndarray             # (n_k, 3) rad/m
    n_bands: int
    tol: float
    meta: dict = field(default_factory=dict)

    @property
    def G(self) -> int:
        return int(self.C_per_grain.shape[0])


def polycrystal(name: str, grid, n_grains: int, micro_seed: int, orient_seed: int,
                C6: np.ndarray, rho: float, k_list: np.ndarray, n_bands: int, tol: float,
                texture: str = "haar", kappa: float = 20.0, L=(1e-3, 1e-3, 1e-3)) -> Problem:
    ids = voronoi_periodic(grid, n_grains, micro_seed, L)
    if texture == "haar":
        R = haar_rotations(n_grains, orient_seed)
    elif texture == "fibre001":
        R = vmf_fibre_rotations(n_grains, kappa, orient_seed)
    else:
        raise ValueError(texture)
    Cg = np.stack([rotate_voigt(C6, R[g]) for g in range(n_grains)])
    return Problem(name, tuple(grid), tuple(L), ids, Cg, np.full(n_grains, rho), k_list,
                   n_bands, tol, dict(texture=texture, n_grains=n_grains))


def workload(name: str, n_k: int | None = None) -> Problem:
    """The measured workloads, by name:

    rve16_g8     16^3 cell, 8 Voronoi grains, Cu-like cubic, Haar; 6 bands, 10 k on G-X, CG tol 1e-10
    rve64_g64    64^3, 64 grains, Haar; 8 bands, 50 k on G-X-M-G-R
    rve128_g200  128^3, 200 grains, <001> vMF fibre (kappa 20); 10 bands, 64 k on G-X-M-G-R
    rve256_g1000 256^3, 1000 grains, Ti-like hexagonal, Haar; 12 bands, 128 k on G-X-M-G-R
    fibre128_circle / fibre128_square
                 128 x 128 x 1 epoxy/carbon long-fibre cells (55 % circular, 65 % square
                 fibres; Table 1); 10 bands, 90 k on M-G-X-M
    """
    cu = cubic_voigt(CU_CUBIC["C11"], CU_CUBIC["C12"], CU_CUBIC["C44"])
    if name == "rve16_g8":
        k = kpath("GX", n_k or 10)
        return polycrystal(name, (16, 16, 16), 8, 1, 101, cu, CU_CUBIC["rho"], k, 6, 1e-10)
    if name == "rve64_g64":
        k = kpath("GXMGR", n_k or 50)
        return polycrystal(name, (64, 64, 64), 64, 2, 102, cu, CU_CUBIC["rho"], k, 8, 1e-10)
    if name == "rve128_g200":
        k = kpath("GXMGR", n_k or 64)
        return polycrystal(name, (128, 128, 128), 200, 3, 103, cu, CU_CUBIC["rho"], k, 10, 1e-10,
                           texture="fibre001", kappa=20.0)
    if name == "fibre128_circle":
        return fibre_composite((128, 128, 1), "circle", n_bands=10, n_k=n_k or 90)
    if name == "fibre128_square":
        return fibre_composite((128, 128, 1), "square", n_bands=10, n_k=n_k or 90)
    if name == "rve256_g1000":
        hx = hexagonal_voigt(TI_HEX["C11"], TI_HEX["C12"], TI_HEX["C13"], TI_HEX["C33"], TI_HEX["C44"])
        k = kpath("GXMGR", n_k or 128)
        return polycrystal(name, (256, 256, 256), 1000, 5, 105, hx, TI_HEX["rho"], k, 12, 1e-10)
    raise KeyError(name)


def fibre_ids(grid, shape: str = "circle", frac: float = 0.55) -> np.ndarray:
    """Two-phase long-fibre cell (the long-fibre composites of the paper's
    Section 4.3): one fibre per cell, axis along z and centred in the (x, y)
    cross-section; phase 1 (fibre) where the voxel centre lies inside a circle
    of area frac*Lx*Ly (shape "circle", Lx = Ly) or a square of that area
    ("square"), phase 0 (matrix) elsewhere.  Every z slice is the same."""
    Nx, Ny, Nz = grid
    x = (np.arange(Nx) + 0.5) / Nx - 0.5
    y = (np.arange(Ny) + 0.5) / Ny - 0.5
    Y, X = np.meshgrid(y, x, indexing="ij")          # (Ny, Nx), fractions of the cell
    if shape == "circle":
        inside = X ** 2 + Y ** 2 <= frac / math.pi
    elif shape == "square":
        h = 0.5 * math.sqrt(frac)
        inside = (np.abs(X) <= h) & (np.abs(Y) <= h)
    else:
        raise ValueError(shape)
    return np.broadcast_to(inside.astype(np.int32)[None], (Nz, Ny, Nx)).copy()


def fibre_composite(grid, shape: str = "circle", frac: float | None = None, n_bands: int = 10,
                    n_k: int = 90, L=(1e-3, 1e-3, 1e-3)) -> Problem:
    """Epoxy matrix with carbon long fibres (Table 1, Composite 1; isotropic
    phases), circular fibres at 55 % or square fibres at 65 % by default, on
    the M-Gamma-X-M path of the fibre cross-section."""
    if frac is None:
        frac = 0.55 if shape == "circle" else 0.65
    ids = fibre_ids(grid, shape, frac)
    C = np.stack([isotropic_from_E_nu(EPOXY["E"], EPOXY["nu"]), isotropic_from_E_nu(CARBON["E"], CARBON["nu"])])
    rho = np.array([EPOXY["rho"], CARBON["rho"]])
    k = kpath("MGXM", n_k, L, corners=True)
    return Problem(f"fibre_{shape}{tuple(grid)}", tuple(grid), tuple(L), ids, C, rho, k, n_bands, 1e-10,
                   dict(shape=shape, frac=frac, fibre_fraction=float(ids.mean())))


def small_polycrystal(grid, n_grains: int, seed: int, texture: str = "haar",
                      n_bands: int = 6, k_list=None, tol: float = 1e-10) -> Problem:
    """A small seeded cubic (Cu-like) polycrystal for tests."""
    cu = cubic_voigt(CU_CUBIC["C11"], CU_CUBIC["C12"], CU_CUBIC["C44"])
    if k_list is None:
        k_list = kpath("GX", 4)
    return polycrystal(f"poly{grid}_{n_grains}_{seed}", grid, n_grains, seed, seed + 100, cu,
                       CU_CUBIC["rho"], np.asarray(k_list, dtype=float), n_bands, tol, texture)


def zener_cell(grid, index: int, zener_range=(1.0, 4.0), grains_range=(20, 200), n_bands: int = 10,
               n_k: int = 9) -> Problem:
    """One cell of the learned-preconditioner training family: a cubic
    polycrystal whose C11, C12 are the Cu-like values and whose C44 =
    A (C11 - C12) / 2 for a Zener ratio A drawn uniformly from zener_range,
    with a uniform integer number of grains from grains_range, periodic
    Voronoi seeds 1000 + index and Haar orientations 2000 + index.  The draw
    of A and of the grain count uses PCG64(1000 + index)."""
    rng = np.random.default_rng(1000 + index)
    A = float(rng.uniform(*zener_range))
    ng = int(rng.integers(grains_range[0], grains_range[1] + 1))
    C11, C12 = CU_CUBIC["C11"], CU_CUBIC["C12"]
    C6 = cubic_voigt(C11, C12, A * (C11 - C12) / 2)
    p = polycrystal(f"zener{tuple(grid)}_{index}", grid, ng, 1000 + index, 2000 + index, C6, CU_CUBIC["rho"],
                    kpath("GXMGR", n_k), n_bands, 1e-10)
    p.meta.update(zener=A)
    return p

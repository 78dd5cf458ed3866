"""FP64 CPU oracle for the FFT-based Bloch-wave method (Segurado & Lebensohn,
arXiv 2106.12487).  TEST INFRASTRUCTURE ONLY: imported by tests/, by the
package's smoke check and by the CPU-baseline leg of bench.py; the product path
never calls it.

Plain, slow and literal: numpy FFTs and dense LAPACK/ARPACK routines serve as
steps; nothing is fused, blocked or reordered beyond what the paper writes.

Conventions
  * grid (Nx, Ny, Nz), arrays shaped (..., Nz, Ny, Nx) (x fastest), Fourier
    fields in standard FFT bin order along each axis.
  * F = numpy.fft.fftn (unnormalised), F^-1 = numpy.fft.ifftn (1/V).  Every F
    in the operators is paired with an F^-1, so any normalisation with
    F^-1 F = I gives the same A_k and M (Section 3.2).
  * Stiffness given per grain in Voigt form (11, 22, 33, 23, 13, 12) with
    engineering shear; the oracle expands it to the full 4th-order tensor and
    contracts with the full (unsymmetrised) displacement gradient, exactly as
    the component form of Eq. (hatA) is written.

Readings of the paper taken here (each also listed in the design notes):
  R1 frequencies (Eq. frequencies): bin m carries xi = 2*pi/L * (m if m < ceil(N/2)
     else m - N); the even-N Nyquist bin keeps -N*pi/L, nothing is symmetrised.
  R2 Eq. (hatA): the component form is authoritative (the bracketing of the
     vector form is garbled); no factor i appears because -(i q)(i q) = q q.
  R3 PCG (Algorithm 2): x0 = 0 unless a start is given; stop when the 2-norm of
     the recursively updated residual <= TOL * ||Y||_2; the true residual is
     recomputed on exit.  Preconditioner Eq. (matrixP)/(precond) with C0 the
     volume average of C(x); the q = 0 bin (k = 0 only) is mapped to zero.
  R4 Algorithm 1: iterate until err1 <= TOL_eig and err2 <= 10 TOL_eig, with
     err2 = max_p ||A u_p - lam_p M u_p||_2 / ||A u_p||_2; the projected
     matrices are Hermitised before the small generalised eigensolve; the new
     basis is U_bar @ Q (no transpose).
  R5 start vectors without a previous k: Fourier unit vectors at the bins of
     smallest |xi + k|, polarised along the eigenvectors of P0(xi + k), the q
     of lowest reference frequency mu_a/rho_bar taken (candidate bins: the
     8q smallest |xi+k|, ties by bin index then polarisation index).
  R6 Gamma point (k = 0): A is singular on the three rigid translations
     (t_c = e_c at bin 0).  They are reported as three zero eigenvalues and the
     rest of the spectrum is sought on the M-orthogonal complement of t_c.
  R7 Lanczos: shift-invert mode (sigma = 0) of ARPACK's implicitly restarted
     Arnoldi/Lanczos on OP = A^-1 M with the M inner product (the paper's Eq.
     (shift) pencil after V = M^-1 U), lambda = 1/beta.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

VOIGT_PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


# ---------------------------------------------------------------------------
# Discretisation (Section 3.2, voxel centres and Eq. frequencies)
# ---------------------------------------------------------------------------
def frequencies(N: int, L: float) -> np.ndarray:
    """Discrete frequencies of Eq. (frequencies) in FFT bin order (reading R1)."""
    m = np.arange(N)
    half = (N + 1) // 2
    mt = np.where(m < half, m, m - N)
    return 2.0 * math.pi / L * mt


def voigt_to_tensor(C6: np.ndarray) -> np.ndarray:
    """Full C_ijkl from a Voigt matrix (minor and major symmetries)."""
    idx = {}
    for a, (i, j) in enumerate(VOIGT_PAIRS):
        idx[(i, j)] = a
        idx[(j, i)] = a
    C4 = np.empty((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C4[i, j, k, l] = C6[idx[(i, j)], idx[(k, l)]]
    return C4


@dataclass
class Medium:
    """A voxelised periodic cell: grain id per voxel plus per-grain C and rho."""
    grid: tuple              # (Nx, Ny, Nz)
    L: tuple                 # (Lx, Ly, Lz) in m
    grain_ids: np.ndarray    # int (Nz, Ny, Nx)
    C_per_grain: np.ndarray  # (G, 6, 6) Voigt, Pa
    rho_per_grain: np.ndarray  # (G,)

    def __post_init__(self):
        Nx, Ny, Nz = self.grid
        self.grain_ids = np.asarray(self.grain_ids).reshape(Nz, Ny, Nx)
        self.C4g = np.stack([voigt_to_tensor(C) for C in np.asarray(self.C_per_grain, float)])
        self.rho_x = np.asarray(self.rho_per_grain, float)[self.grain_ids]
        self.xi = (frequencies(Nx, self.L[0]).reshape(1, 1, Nx),
                   frequencies(Ny, self.L[1]).reshape(1, Ny, 1),
                   frequencies(Nz, self.L[2]).reshape(Nz, 1, 1))
        # C0: volume average of the voxel stiffness (Section 3.3, after Eq. precond)
        counts = np.bincount(self.grain_ids.ravel(), minlength=self.C4g.shape[0])
        self.C0 = np.einsum("g,gijkl->ijkl", counts / self.grain_ids.size, self.C4g)
        self.rho_bar = float(self.rho_x.mean())

    @property
    def V(self) -> int:
        return int(np.prod(self.grid))

    @property
    def shape(self):
        Nx, Ny, Nz = self.grid
        return (3, Nz, Ny, Nx)

    def q(self, k):
        """The shifted wave vector xi + k on every Fourier voxel (broadcastable)."""
        return [self.xi[j] + float(k[j]) for j in range(3)]

    @classmethod
    def from_problem(cls, p) -> "Medium":
        return cls(tuple(p.grid), tuple(p.L), p.grain_ids, p.C_per_grain, p.rho)


# ---------------------------------------------------------------------------
# Operators (Eq. hatA, Eq. hatM, Eq. def_invM)
# ---------------------------------------------------------------------------
def _F(a):
    return np.fft.fftn(a, axes=(-3, -2, -1))


def _Finv(a):
    return np.fft.ifftn(a, axes=(-3, -2, -1))


def apply_K(med: Medium, k, U: np.ndarray) -> np.ndarray:
    """Stiffness operator of Eq. (hatA), component form:
    A_i{U} = (xi_j + k_j) F{ C_ijkl(x) F^-1((xi_l + k_l) U_k) }."""
    q = med.q(k)
    g = np.empty((3, 3) + U.shape[1:], dtype=complex)
    for kk in range(3):
        for ll in range(3):
            g[kk, ll] = _Finv(q[ll] * U[kk])
    out = np.zeros(U.shape, dtype=complex)
    for i in range(3):
        for j in range(3):
            sig = np.zeros(U.shape[1:], dtype=complex)
            for kk in range(3):
                for ll in range(3):
                    c = med.C4g[:, i, j, kk, ll][med.grain_ids]
                    sig += c * g[kk, ll]
            out[i] += q[j] * _F(sig)
    return out


def apply_M(med: Medium, U: np.ndarray) -> np.ndarray:
    """Mass operator of Eq. (hatM): F{ rho(x) F^-1(U) }."""
    return _F(med.rho_x * _Finv(U))


def apply_Minv(med: Medium, Y: np.ndarray) -> np.ndarray:
    """Inverse mass operator of Eq. (def_invM) (reading: F{rho^-1 F^-1 Y})."""
    return _F(_Finv(Y) / med.rho_x)


def vdot(a, b) -> complex:
    return complex(np.vdot(a.ravel(), b.ravel()))


def norm(a) -> float:
    return float(np.linalg.norm(a.ravel()))


# ---------------------------------------------------------------------------
# Preconditioner (Eq. matrixP, Eq. precond)
# ---------------------------------------------------------------------------
def acoustic_tensor(C0: np.ndarray, qvec) -> np.ndarray:
    """P_ik = C0_ijkl q_j q_l for a batch of real vectors q (..., 3) -> (..., 3, 3)."""
    return np.einsum("ijkl,...j,...l->...ik", C0, qvec, qvec)


def _qgrid(med: Medium, k) -> np.ndarray:
    q = med.q(k)
    Nx, Ny, Nz = med.grid
    qv = np.empty((Nz, Ny, Nx, 3))
    for j in range(3):
        qv[..., j] = np.broadcast_to(q[j], (Nz, Ny, Nx))
    return qv


def apply_precond(med: Medium, k, R: np.ndarray) -> np.ndarray:
    """Z = P^-1(xi + k) R per Fourier voxel (Eq. precond); P = 0 bins give 0."""
    qv = _qgrid(med, k).reshape(-1, 3)
    P = acoustic_tensor(med.C0, qv)
    r = np.moveaxis(R.reshape(3, -1), 0, 1)            # (V, 3)
    zero = np.einsum("vj,vj->v", qv, qv) == 0.0
    P[zero] = np.eye(3)
    z = np.linalg.solve(P, r[..., None])[..., 0]
    z[zero] = 0.0
    return np.moveaxis(z, 1, 0).reshape(R.shape)


# ---------------------------------------------------------------------------
# Inverse operator by PCG (Algorithm 2)
# ---------------------------------------------------------------------------
@dataclass
class CGResult:
    x: np.ndarray
    iters: int
    rel_res: float        # recursive residual / ||Y||
    true_rel_res: float   # ||Y - A x|| / ||Y||
    converged: bool


def pcg(A, Pinv, Y: np.ndarray, tol: float, maxiter: int = 10000, x0=None) -> CGResult:
    """Preconditioned conjugate gradient for Hermitian PD A (reading R3)."""
    ynorm = norm(Y)
    if ynorm == 0.0:
        return CGResult(np.zeros_like(Y), 0, 0.0, 0.0, True)
    if x0 is None:
        x = np.zeros_like(Y)
        r = Y.copy()
    else:
        x = x0.copy()
        r = Y - A(x)
    z = Pinv(r)
    p = z.copy()
    rz = vdot(r, z).real
    it = 0
    rel = norm(r) / ynorm
    while rel > tol and it < maxiter:
        Ap = A(p)
        alpha = rz / vdot(p, Ap).real
        x += alpha * p
        r -= alpha * Ap
        it += 1
        rel = norm(r) / ynorm
        if rel <= tol:
            break
        z = Pinv(r)
        rz_new = vdot(r, z).real
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    true_rel = norm(Y - A(x)) / ynorm
    return CGResult(x, it, rel, true_rel, rel <= tol)


# ---------------------------------------------------------------------------
# Gamma point handling (reading R6)
# ---------------------------------------------------------------------------
def is_gamma(k) -> bool:
    return float(np.dot(k, k)) == 0.0


def deflate_rigid(med: Medium, U: np.ndarray) -> np.ndarray:
    """Remove the M-projection on the rigid translations t_c = e_c at bin 0:
    U <- U - sum_c t_c <t_c, M U> / <t_c, M t_c>, where <t_c, M U> = (M U)_c(bin 0)
    and <t_c, M t_c> = rho_bar (numpy normalisation)."""
    MU0 = apply_M(med, U)[:, 0, 0, 0]
    out = U.copy()
    out[:, 0, 0, 0] -= MU0 / med.rho_bar
    return out


# ---------------------------------------------------------------------------
# Start vectors (reading R5)
# ---------------------------------------------------------------------------
def start_vectors(med: Medium, k, nvec: int) -> np.ndarray:
    qv = _qgrid(med, k).reshape(-1, 3)
    q2 = np.einsum("vj,vj->v", qv, qv)
    order = np.lexsort((np.arange(q2.size), q2))
    if is_gamma(k):
        order = order[q2[order] > 0.0]
    cand = order[: max(8 * nvec, 8)]
    items = []
    for b in cand:
        P = acoustic_tensor(med.C0, qv[b][None])[0]
        mu, W = np.linalg.eigh(P)
        for a in range(3):
            items.append((mu[a], int(b), a, W[:, a]))
    items.sort(key=lambda t: (t[0], t[1], t[2]))
    U = np.zeros((nvec,) + med.shape, dtype=complex)
    flat = U.reshape(nvec, 3, -1)
    for p in range(nvec):
        _, b, _, w = items[p]
        flat[p, :, b] = w
    return U


# ---------------------------------------------------------------------------
# Small dense generalised Hermitian eigenproblem
# ---------------------------------------------------------------------------
def small_eig(K: np.ndarray, M: np.ndarray):
    import scipy.linalg
    K = 0.5 * (K + K.conj().T)
    M = 0.5 * (M + M.conj().T)
    lam, Q = scipy.linalg.eigh(K, M)
    return lam, Q


# ---------------------------------------------------------------------------
# Subspace iteration (Algorithm 1)
# ---------------------------------------------------------------------------
@dataclass
class EigResult:
    lam: np.ndarray          # (n,) ascending
    U: np.ndarray | None     # (n, 3, Nz, Ny, Nx) eigenvectors
    sweeps: int
    cg_iters: int
    solves: int
    err1: float
    err2: float
    converged: bool


def subspace_iteration(med: Medium, k, n: int, tol_lin: float, tol_eig: float,
                       q: int | None = None, U0=None, max_sweeps: int = 500,
                       max_cg: int = 10000) -> EigResult:
    """Algorithm 1 of the paper for the n smallest eigenpairs of A_k U = lam M U."""
    if q is None:
        q = min(2 * n, n + 8)
    gamma = is_gamma(k)
    A = lambda x: apply_K(med, k, x)
    Pinv = lambda x: apply_precond(med, k, x)
    U = start_vectors(med, k, q) if U0 is None else np.array(U0[:q], dtype=complex)
    if gamma:
        U = np.stack([deflate_rigid(med, u) for u in U])
    lam_prev = None
    cg_total = 0
    solves = 0
    err1 = err2 = math.inf
    for s in range(1, max_sweeps + 1):
        v = np.stack([apply_M(med, u) for u in U])
        Ubar = np.empty_like(U)
        for p in range(q):
            res = pcg(A, Pinv, v[p], tol_lin, max_cg)
            cg_total += res.iters
            solves += 1
            Ubar[p] = deflate_rigid(med, res.x) if gamma else res.x
        Kn = v
        Mn = np.stack([apply_M(med, u) for u in Ubar])
        Ub = Ubar.reshape(q, -1)
        Kp = Ub.conj() @ Kn.reshape(q, -1).T
        Mp = Ub.conj() @ Mn.reshape(q, -1).T
        lam, Qm = small_eig(Kp, Mp)
        U = np.tensordot(Qm.T, Ubar, axes=(1, 0))
        if lam_prev is not None:
            err1 = math.sqrt(float(np.sum((lam[:n] - lam_prev[:n]) ** 2) / np.sum(lam_prev[:n] ** 2)))
        lam_prev = lam.copy()
        if err1 <= tol_eig:
            err2 = 0.0
            for p in range(n):
                Au = A(U[p])
                err2 = max(err2, norm(Au - lam[p] * apply_M(med, U[p])) / norm(Au))
            if err2 <= 10.0 * tol_eig:
                return EigResult(lam[:n], U[:n], s, cg_total, solves, err1, err2, True)
    return EigResult(lam_prev[:n], U[:n], max_sweeps, cg_total, solves, err1, err2, False)


# ---------------------------------------------------------------------------
# Implicitly restarted Lanczos, shift-invert (Section 3.3, reading R7)
# ---------------------------------------------------------------------------
def lanczos_irl(med: Medium, k, n: int, tol_lin: float, tol_eig: float,
                ncv: int | None = None, max_cg: int = 10000, seed: int = 0) -> EigResult:
    from scipy.sparse.linalg import LinearOperator, eigs

    gamma = is_gamma(k)
    shape = med.shape
    size = int(np.prod(shape))
    stats = {"cg": 0, "solves": 0}

    def Kmv(x):
        return apply_K(med, k, x.reshape(shape)).ravel()

    def Mmv(x):
        return apply_M(med, x.reshape(shape)).ravel()

    def OPinv(x):
        y = x.reshape(shape)
        if gamma:
            y = y.copy()
            y[:, 0, 0, 0] = 0.0
        res = pcg(lambda u: apply_K(med, k, u), lambda u: apply_precond(med, k, u), y,
                  tol_lin, max_cg)
        stats["cg"] += res.iters
        stats["solves"] += 1
        out = deflate_rigid(med, res.x) if gamma else res.x
        return out.ravel()

    Aop = LinearOperator((size, size), matvec=Kmv, dtype=complex)
    Mop = LinearOperator((size, size), matvec=Mmv, dtype=complex)
    Oop = LinearOperator((size, size), matvec=OPinv, dtype=complex)
    rng = np.random.Generator(np.random.PCG64(seed))
    v0 = (rng.standard_normal(size) + 1j * rng.standard_normal(size)).reshape(shape)
    if gamma:
        v0 = deflate_rigid(med, v0)
    nev = n
    if ncv is None:
        ncv = max(2 * nev + 1, 20)
    ncv = min(ncv, size - 1)
    lam, vec = eigs(Aop, k=nev, M=Mop, sigma=0.0, which="LM", OPinv=Oop, v0=v0.ravel(),
                    ncv=ncv, tol=tol_eig, maxiter=300)
    lam = lam.real
    order = np.argsort(lam)
    lam = lam[order]
    U = vec[:, order].T.reshape((nev,) + shape)
    return EigResult(lam, U, 0, stats["cg"], stats["solves"], 0.0, 0.0, True)


# ---------------------------------------------------------------------------
# Dispersion driver (Algorithm 3)
# ---------------------------------------------------------------------------
@dataclass
class BandsResult:
    omega: np.ndarray    # (n_k, n) rad/s
    lam: np.ndarray      # (n_k, n)
    cg_iters: np.ndarray
    solves: np.ndarray
    sweeps: np.ndarray
    seconds: float


def solve_bands(med: Medium, k_list, n: int, tol_lin: float = 1e-10, tol_eig: float = 1e-10,
                method: str = "subspace", warm_start: bool = False, q: int | None = None,
                return_vectors: bool = False):
    """Algorithm 3: loop over wave vectors, extract the n lowest bands, omega = sqrt(lambda)."""
    t0 = time.perf_counter()
    k_list = np.atleast_2d(np.asarray(k_list, float))
    nk = k_list.shape[0]
    lam_all = np.zeros((nk, n))
    cg = np.zeros(nk, dtype=np.int64)
    solves = np.zeros(nk, dtype=np.int64)
    sweeps = np.zeros(nk, dtype=np.int64)
    vecs = []
    prev = None
    for r in range(nk):
        k = k_list[r]
        n_eff = n
        lam_z = []
        if is_gamma(k):
            nz = min(3, n)
            lam_z = [0.0] * nz
            n_eff = n - nz
        if n_eff > 0:
            if method == "subspace":
                res = subspace_iteration(med, k, n_eff, tol_lin, tol_eig, q=q,
                                         U0=prev if (warm_start and prev is not None) else None)
            elif method == "lanczos":
                res = lanczos_irl(med, k, n_eff, tol_lin, tol_eig)
            else:
                raise ValueError(method)
            lam = np.concatenate([lam_z, res.lam])
            cg[r], solves[r], sweeps[r] = res.cg_iters, res.solves, res.sweeps
            if warm_start and method == "subspace":
                prev = res.U
            if return_vectors:
                vecs.append(res.U)
        else:
            lam = np.asarray(lam_z)
        lam_all[r] = lam
    omega = np.sqrt(np.maximum(lam_all, 0.0))
    out = BandsResult(omega, lam_all, cg, solves, sweeps, time.perf_counter() - t0)
    if return_vectors:
        return out, vecs
    return out


# ---------------------------------------------------------------------------
# Group velocity (Section 5.1, Eq. c_group; wave speeds of Section 5.2)
# ---------------------------------------------------------------------------
def apply_dK(med: Medium, k, m: int, U: np.ndarray) -> np.ndarray:
    """Derivative of the stiffness operator with respect to k_m, by the product
    rule on the component form of Eq. (hatA) (q = xi + k, dq_j/dk_m = delta_jm):
    dA_i{U}/dk_m = F{ C_imkl F^-1(q_l U_k) } + q_j F{ C_ijkm F^-1(U_k) }."""
    q = med.q(k)
    out = np.zeros(U.shape, dtype=complex)
    w = [_Finv(U[kk]) for kk in range(3)]
    for i in range(3):
        s1 = np.zeros(U.shape[1:], dtype=complex)
        for kk in range(3):
            for ll in range(3):
                s1 += med.C4g[:, i, m, kk, ll][med.grain_ids] * _Finv(q[ll] * U[kk])
        out[i] += _F(s1)
        for j in range(3):
            s2 = np.zeros(U.shape[1:], dtype=complex)
            for kk in range(3):
                s2 += med.C4g[:, i, j, kk, m][med.grain_ids] * w[kk]
            out[i] += q[j] * _F(s2)
    return out


def group_velocity_hf(med: Medium, k, U: np.ndarray):
    """Group velocities d omega / d k of eigenvectors U (n, 3, Nz, Ny, Nx) of
    A_k U = lambda M U by the Hellmann-Feynman identity (M does not depend on k):
    d lambda / d k_m = u^H (dA/dk_m) u / u^H M u,  d omega/d k = (d lambda/d k) / (2 omega),
    lambda the Rayleigh quotient of u.  Returns (omega (n,), c (n, 3))."""
    n = U.shape[0]
    om = np.empty(n)
    c = np.empty((n, 3))
    for p in range(n):
        Mu = apply_M(med, U[p])
        uMu = vdot(U[p], Mu).real
        lam = vdot(U[p], apply_K(med, k, U[p])).real / uMu
        om[p] = math.sqrt(max(lam, 0.0))
        for m in range(3):
            dl = vdot(U[p], apply_dK(med, k, m, U[p])).real / uMu
            c[p, m] = dl / (2.0 * om[p])
    return om, c


def wave_speeds(med: Medium, direction, K: float | None = None) -> np.ndarray:
    """Low-frequency wave speeds along a propagation direction (Section 5.2,
    Eq. wave_speed2): the slopes d omega^b / dK of the three acoustic branches
    b = 1, 2, 3 (ascending omega: the two transverse branches, then the
    longitudinal one) at k = K d, d the unit direction and K small against the
    Brillouin zone (default 1e-3 pi / max L).  Each slope is d . grad_k omega of
    the dense eigenvector by the Hellmann-Feynman identity (group_velocity_hf);
    for a degenerate transverse pair every vector of the pair gives the same
    slope along d when d is a symmetry axis.  Dense eigensolve: tiny grids only.
    Returns the three speeds (m/s)."""
    import scipy.linalg

    d = np.asarray(direction, float)
    d = d / np.linalg.norm(d)
    if K is None:
        K = 1e-3 * math.pi / max(med.L)
    k = K * d
    _, W = scipy.linalg.eigh(dense_K(med, k), dense_M(med), subset_by_index=(0, 2))
    U = W.T.reshape((3,) + med.shape)
    _, c = group_velocity_hf(med, k, U)
    return c @ d


def group_velocity_fd(med: Medium, k, n: int, h: float, solver=None):
    """Group velocities of the n lowest bands by central finite differences of
    the band frequencies along each axis, the derivative of Eq. (c_group) taken
    as the paper takes it (differences of omega between neighbouring wave
    vectors of a branch); valid where the bands are simple.  `solver(k, n)`
    returns the n lowest omega (default: dense generalised eigensolve, tiny
    grids only).  Returns c (n, 3)."""
    if solver is None:
        import scipy.linalg

        Md = dense_M(med)

        def solver(kk, nn):
            lam = scipy.linalg.eigh(dense_K(med, kk), Md, eigvals_only=True, subset_by_index=(0, nn - 1))
            return np.sqrt(np.maximum(lam, 0.0))
    c = np.empty((n, 3))
    k = np.asarray(k, float)
    for m in range(3):
        e = np.zeros(3)
        e[m] = h
        c[:, m] = (solver(k + e, n) - solver(k - e, n)) / (2.0 * h)
    return c


# ---------------------------------------------------------------------------
# Real-space eigenvectors (Section 5.2, Eq. rotate_eigenvector)
# ---------------------------------------------------------------------------
def eigvec_real(med: Medium, U_hat: np.ndarray):
    """U(x) = e^{-i phi} F^-1(U_hat) with phi the single phase of the field
    (reading: phi = arg(sum_x U(x).U(x)) / 2, the field's phase mod pi when it
    has one, else the least-squares best single phase), and the strain of the
    same field eps_ij = (d_j U_i + d_i U_j) / 2 with d_j = i xi_j (the
    epsilon_11 = dU_1/dx_1 of the section), components (xx, yy, zz, yz, xz, xy).
    Returns (phi, U (3, Nz, Ny, Nx), eps (6, Nz, Ny, Nx))."""
    w = _Finv(U_hat)
    phi = 0.5 * math.atan2(float(np.sum(w * w).imag), float(np.sum(w * w).real))
    rot = np.exp(-1j * phi)
    U = rot * w
    pairs = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
    eps = np.empty((6,) + U_hat.shape[1:], dtype=complex)
    for c, (i, j) in enumerate(pairs):
        eps[c] = rot * _Finv(0.5j * (med.xi[j] * U_hat[i] + med.xi[i] * U_hat[j]))
    return phi, U, eps


# ---------------------------------------------------------------------------
# Dense matrices for tiny grids (tests only)
# ---------------------------------------------------------------------------
def dense_operator(apply, shape) -> np.ndarray:
    size = int(np.prod(shape))
    A = np.empty((size, size), dtype=complex)
    e = np.zeros(size, dtype=complex)
    for j in range(size):
        e[:] = 0.0
        e[j] = 1.0
        A[:, j] = apply(e.reshape(shape)).ravel()
    return A


def dense_K(med: Medium, k) -> np.ndarray:
    return dense_operator(lambda u: apply_K(med, k, u), med.shape)


def dense_M(med: Medium) -> np.ndarray:
    return dense_operator(lambda u: apply_M(med, u), med.shape)


def rayleigh_quotients(med: Medium, k, U: np.ndarray):
    """FP64 Rayleigh quotients and relative residuals of given vectors."""
    lam = np.empty(U.shape[0])
    res = np.empty(U.shape[0])
    for p in range(U.shape[0]):
        Ku = apply_K(med, k, U[p])
        Mu = apply_M(med, U[p])
        lam[p] = vdot(U[p], Ku).real / vdot(U[p], Mu).real
        res[p] = norm(Ku - lam[p] * Mu) / max(norm(Ku), 1e-300)
    return lam, res

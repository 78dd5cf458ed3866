"""FP64 oracle of the learned Fourier-space preconditioner (test infrastructure).

The paper's Green preconditioner applies P(q)^-1 per Fourier voxel, with
P_ik = C0_ijkl q_j q_l and q = xi + k (Eqs. matrixP, precond).  The learned
preconditioner keeps its eigenvectors and rescales each branch:

    Z_theta(q) = sum_a g_a v_a v_a^T / mu_a,      P(q) = sum_a mu_a v_a v_a^T,
    g_a = softplus(MLP_theta(f_a)),
    f_a = (qh_x^2, qh_y^2, qh_z^2, mu_a / |q|^2, s),  s = log(1+|q|) / log(1+N/2)

in the library's scaled units (q in 2 pi / L, C in units of C_ref).  g_a > 0 makes
Z symmetric positive definite (plain CG stays valid); Z depends on the branch
only through mu_a, so it is a matrix function of P and well defined for
repeated eigenvalues.  With the output layer initialised to zero weight and
bias log(e - 1), g = 1 and Z = P^-1 exactly.

Loss: over CG iterates j of systems A x = b with residual r_j and error
e_j = x* - x_j (each pair scaled by 1/||r_j||), the summed squared error of one
preconditioner application, sum_j ||Z r_j - e_j||^2.  Per Fourier voxel it only
needs the moments A = Re sum r r^H, B = sym Re sum r e^H, c = sum |e|^2:
    loss = sum_bins tr(Z Z A) - 2 tr(Z B) + c.

Parameter vector (flat, this order): W1 (H x 5, row-major), b1 (H), W2 (H x H),
b2 (H), w3 (H), b3 (1); hidden activations tanh.
"""
from __future__ import annotations

import math

import numpy as np

NF = 5


def n_params(H: int) -> int:
    return H * NF + H + H * H + H + H + 1


def unpack(theta: np.ndarray, H: int):
    o = 0
    W1 = theta[o:o + H * NF].reshape(H, NF); o += H * NF
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    w3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def acoustic(C0_4: np.ndarray, q: np.ndarray) -> np.ndarray:
    """P_ik = C0_ijkl q_j q_l for q (n, 3) -> (n, 3, 3)."""
    return np.einsum("ijkl,nj,nl->nik", C0_4, q, q)


def features(q: np.ndarray, mu: np.ndarray, Nmax: int) -> np.ndarray:
    """f (n, 3 branches, 5)."""
    qn2 = np.einsum("nj,nj->n", q, q)
    qn = np.sqrt(qn2)
    qh2 = q * q / qn2[:, None]
    s = np.log1p(qn) / math.log1p(Nmax / 2.0)
    f = np.empty((q.shape[0], 3, NF))
    f[:, :, 0:3] = qh2[:, None, :]
    f[:, :, 3] = mu / qn2[:, None]
    f[:, :, 4] = s[:, None]
    return f


def softplus(x):
    return np.where(x > 20, x, np.log1p(np.exp(np.minimum(x, 20))))


def g_of(theta: np.ndarray, H: int, f: np.ndarray) -> np.ndarray:
    W1, b1, W2, b2, w3, b3 = unpack(theta, H)
    h1 = np.tanh(f @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return softplus(h2 @ w3 + b3)


def Z_of(theta: np.ndarray, H: int, q: np.ndarray, C0_4: np.ndarray, Nmax: int) -> np.ndarray:
    """Learned preconditioner matrices Z (n, 3, 3) at scaled wave vectors q != 0."""
    P = acoustic(C0_4, q)
    mu, V = np.linalg.eigh(P)
    g = g_of(theta, H, features(q, mu, Nmax))
    return np.einsum("nia,na,nja->nij", V, g / mu, V)


def init_params(H: int, seed: int = 7) -> np.ndarray:
    """Deterministic initialisation: small uniform hidden weights from a
    counter-based hash, zero output weights, output bias log(e - 1)."""
    n = n_params(H)
    theta = np.zeros(n)
    nh = H * NF + H + H * H + H
    idx = np.arange(nh, dtype=np.uint64)
    x = idx * np.uint64(0x9E3779B97F4A7C15) + np.uint64(seed)
    x ^= x >> np.uint64(33)
    x *= np.uint64(0xFF51AFD7ED558CCD)
    x ^= x >> np.uint64(33)
    u = (x >> np.uint64(40)).astype(np.float64) / float(1 << 24)       # [0, 1)
    theta[:nh] = (2.0 * u - 1.0) * 0.5
    theta[nh:nh + H] = 0.0
    theta[-1] = math.log(math.e - 1.0)
    return theta


def sym6_to_mat(a: np.ndarray) -> np.ndarray:
    """(n, 6) in order (xx, yy, zz, yz, xz, xy) -> (n, 3, 3)."""
    M = np.empty(a.shape[:-1] + (3, 3))
    M[..., 0, 0], M[..., 1, 1], M[..., 2, 2] = a[..., 0], a[..., 1], a[..., 2]
    M[..., 1, 2] = M[..., 2, 1] = a[..., 3]
    M[..., 0, 2] = M[..., 2, 0] = a[..., 4]
    M[..., 0, 1] = M[..., 1, 0] = a[..., 5]
    return M


def moments(r: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Per-Fourier-voxel moments of residual/error pairs, the sufficient
    statistics of the loss above: for pairs j (r, e shaped (n, 3, Nz, Ny, Nx),
    complex) with weights w_j = 1/||r_j||^2 (pairs with r_j = 0 skipped),
        A = sum_j w_j Re(r_j r_j^H),  B = sum_j w_j sym Re(r_j e_j^H),  c = sum_j w_j |e_j|^2,
    returned as (V, 13): A and B in the order (xx, yy, zz, yz, xz, xy), then c.
    With Z real symmetric, ||Z r - e||^2 = tr(Z Z A) - 2 tr(Z B) + c per voxel."""
    n = r.shape[0]
    V = int(np.prod(r.shape[2:]))
    rv = r.reshape(n, 3, V)
    ev = e.reshape(n, 3, V)
    out = np.zeros((V, 13))
    pairs = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
    for j in range(n):
        nr2 = float(np.vdot(rv[j], rv[j]).real)
        if nr2 == 0.0:
            continue
        w = 1.0 / nr2
        for t, (a, b) in enumerate(pairs):
            out[:, t] += w * (rv[j, a] * np.conj(rv[j, b])).real
            out[:, 6 + t] += w * 0.5 * ((rv[j, a] * np.conj(ev[j, b])).real + (rv[j, b] * np.conj(ev[j, a])).real)
        out[:, 12] += w * np.sum(np.abs(ev[j]) ** 2, axis=0)
    return out


def loss(theta: np.ndarray, H: int, blocks) -> float:
    """blocks: iterable of dicts with q (n, 3), A (n, 6), B (n, 6), c (n,),
    C0 (3, 3, 3, 3) scaled, Nmax."""
    tot = 0.0
    for blk in blocks:
        Z = Z_of(theta, H, blk["q"], blk["C0"], blk["Nmax"])
        A = sym6_to_mat(blk["A"])
        Bm = sym6_to_mat(blk["B"])
        tot += float(np.einsum("nij,njk,nki->", Z, Z, A) - 2.0 * np.einsum("nij,nji->", Z, Bm) + blk["c"].sum())
    return tot


def fd_grad(theta: np.ndarray, H: int, blocks, h: float = 1e-6) -> np.ndarray:
    """Central finite differences of the loss (FP64)."""
    g = np.zeros_like(theta)
    for i in range(theta.size):
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        g[i] = (loss(tp, H, blocks) - loss(tm, H, blocks)) / (2 * h)
    return g

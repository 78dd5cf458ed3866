"""Pins of the learned-preconditioner oracle (CPU, FP64)."""
import math

import numpy as np

from oracle import bloch_oracle as O
from oracle import learned_precond as OL
from paper_2106_12487_gb300 import synth

H = 16


def test_init_is_green_inverse():
    """Output layer zero and bias log(e-1): g = 1, Z = P^-1 (Eq. precond)."""
    theta = OL.init_params(H)
    C0 = O.voigt_to_tensor(synth.rotate_voigt(synth.cubic_voigt(1.0, 0.72, 0.45), synth.haar_rotations(1, 3)[0]))
    q = np.random.default_rng(1).normal(size=(20, 3)) * 5
    Z = OL.Z_of(theta, H, q, C0, 64)
    assert np.allclose(Z, np.linalg.inv(OL.acoustic(C0, q)), rtol=1e-12)


def test_isotropic_closed_form_and_spd():
    """For an isotropic C0, P = mu_T |q|^2 I + (mu_L - mu_T) q q^T (a repeated
    eigenvalue); Z must equal g_L/mu_L qh qh^T + g_T/mu_T (I - qh qh^T) whatever
    basis the eigensolver returns in the repeated eigenspace; Z is SPD."""
    lam, mu = 0.5, 0.3
    C0 = O.voigt_to_tensor(synth.isotropic_voigt(lam, mu))
    rng = np.random.default_rng(2)
    theta = rng.normal(size=OL.n_params(H)) * 0.7
    q = rng.normal(size=(30, 3)) * 3
    Z = OL.Z_of(theta, H, q, C0, 32)
    qn2 = np.einsum("nj,nj->n", q, q)
    qh = q / np.sqrt(qn2)[:, None]
    muL, muT = (lam + 2 * mu) * qn2, mu * qn2
    s = np.log1p(np.sqrt(qn2)) / math.log1p(16.0)
    f = lambda m: np.stack([qh[:, 0] ** 2, qh[:, 1] ** 2, qh[:, 2] ** 2, m / qn2, s], -1)[:, None, :]
    gL = OL.g_of(theta, H, f(muL))[:, 0]
    gT = OL.g_of(theta, H, f(muT))[:, 0]
    PL = np.einsum("ni,nj->nij", qh, qh)
    ref = (gL / muL)[:, None, None] * PL + (gT / muT)[:, None, None] * (np.eye(3) - PL)
    assert np.allclose(Z, ref, rtol=1e-10, atol=0)
    assert np.all(np.linalg.eigvalsh(Z) > 0)


def test_loss_vanishes_at_the_generating_parameters():
    """Moments built from pairs with e = Z(theta*) r: the moment form
    tr(Z Z A) - 2 tr(Z B) + c of sum ||Z r - e||^2 is zero at theta* and
    positive elsewhere."""
    rng = np.random.default_rng(4)
    C0 = O.voigt_to_tensor(synth.rotate_voigt(synth.cubic_voigt(1.0, 0.72, 0.45), synth.haar_rotations(1, 8)[0]))
    q = rng.normal(size=(40, 3)) * 4
    ts = rng.normal(size=OL.n_params(H)) * 0.5
    Zs = OL.Z_of(ts, H, q, C0, 64)
    A = np.zeros((40, 6))
    Bm = np.zeros((40, 6))
    c = np.zeros(40)
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    for _ in range(5):
        r = rng.normal(size=(40, 3)) + 1j * rng.normal(size=(40, 3))
        e = np.einsum("nij,nj->ni", Zs, r)
        for t, (i, j) in enumerate(pairs):
            A[:, t] += (r[:, i] * np.conj(r[:, j])).real
            Bm[:, t] += 0.5 * ((r[:, i] * np.conj(e[:, j])).real + (r[:, j] * np.conj(e[:, i])).real)
        c += np.sum(np.abs(e) ** 2, axis=1)
    blocks = [dict(q=q, A=A, B=Bm, c=c, C0=C0, Nmax=64)]
    assert abs(OL.loss(ts, H, blocks)) < 1e-9 * c.sum()
    assert OL.loss(ts + 0.05 * rng.normal(size=ts.size), H, blocks) > 1e-6 * c.sum()
    g = OL.fd_grad(ts, H, blocks, h=1e-6)
    assert np.linalg.norm(g) < 1e-5 * c.sum()


def test_moments_reproduce_the_pairwise_loss():
    """The moments function against the definition it serves: for any
    symmetric Z per voxel, sum_voxels tr(Z Z A) - 2 tr(Z B) + c equals the
    brute-force sum over pairs of ||Z r_j - e_j||^2 / ||r_j||^2 (complex
    fields), and a zero residual pair is skipped."""
    rng = np.random.default_rng(6)
    shape = (3, 4, 3, 5)
    n = 4
    r = rng.normal(size=(n,) + shape) + 1j * rng.normal(size=(n,) + shape)
    e = rng.normal(size=(n,) + shape) + 1j * rng.normal(size=(n,) + shape)
    r[2] = 0.0                                   # skipped pair
    V = 60
    S = rng.normal(size=(V, 3, 3))
    Z = S + np.transpose(S, (0, 2, 1))           # symmetric, indefinite is fine here
    m = OL.moments(r, e)
    A = OL.sym6_to_mat(m[:, :6])
    Bm = OL.sym6_to_mat(m[:, 6:12])
    via_moments = float(np.einsum("nij,njk,nki->", Z, Z, A) - 2.0 * np.einsum("nij,nji->", Z, Bm) + m[:, 12].sum())
    brute = 0.0
    for j in range(n):
        rj = r[j].reshape(3, V).T
        ej = e[j].reshape(3, V).T
        nr2 = float(np.sum(np.abs(rj) ** 2))
        if nr2 == 0.0:
            continue
        d = np.einsum("nij,nj->ni", Z, rj) - ej
        brute += float(np.sum(np.abs(d) ** 2)) / nr2
    assert abs(via_moments - brute) <= 1e-12 * abs(brute)
    # a planted mistake (unsymmetrised B) changes the loss
    m2 = m.copy()
    m2[:, 6 + 3] *= 1.5
    B2 = OL.sym6_to_mat(m2[:, 6:12])
    bad = float(np.einsum("nij,njk,nki->", Z, Z, A) - 2.0 * np.einsum("nij,nji->", Z, B2) + m[:, 12].sum())
    assert abs(bad - brute) > 1e-6 * abs(brute)

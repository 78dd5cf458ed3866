"""Full-size parity at the measured workload (128^3, 200 grains, <001> fibre):
the bench's FP32 chosen form against the FP64 plain form (Lanczos, tol 1e-10)
on sampled wave vectors, and the FP64 oracle's Rayleigh quotients of the
returned FP32 eigenvectors (computed one vector at a time)."""
import math

import numpy as np
import pytest

from oracle import bloch_oracle as O
from paper_2106_12487_gb300 import synth

pytestmark = pytest.mark.gpu

CHOSEN = dict(precision=1, method=0, tol_lin=1e-2, tol_eig=1e-5, max_cg=500, max_outer=100)   # the bench's
# (the bench also sets block = n_bands + 2)


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_12487_gb300 import bloch, build
    build.build()
    bloch.lib()
    return bloch


def test_rve128_chosen_form_frequencies(B):
    import torch
    p = synth.workload("rve128_g200")
    idx = [1, 37]              # the first wave vector after Gamma, one on M-Gamma
    ks = p.k_list[idx]
    plan = B.Plan.from_problem(p, block=p.n_bands + 2, **CHOSEN)
    vecs = torch.zeros(len(idx) * p.n_bands * 3 * plan.V, dtype=torch.complex64, device="cuda")
    got, stats, _ = plan.solve_bands(ks, p.n_bands, vecs_out=vecs)
    ref_plan = B.Plan.from_problem(p, precision=0, method=0, tol_lin=1e-10, tol_eig=1e-10, max_cg=2000)
    ref, _, _ = ref_plan.solve_bands(ks, p.n_bands)
    assert np.max(np.abs(got / ref - 1)) < 1e-6
    # oracle Rayleigh quotients of three returned vectors (acoustic, mid, top band)
    med = O.Medium.from_problem(p)
    V = vecs.cpu().numpy().reshape(len(idx), p.n_bands, 3, *reversed(p.grid))
    for i, b in [(0, 0), (0, 9), (1, 4)]:
        u = V[i, b].astype(np.complex128)
        lam, res = O.rayleigh_quotients(med, ks[i], u[None])
        assert abs(math.sqrt(lam[0]) / got[i, b] - 1) < 1e-6


@pytest.fixture(scope="module")
def rve256():
    p = synth.workload("rve256_g1000")
    return p, O.Medium.from_problem(p)


def test_rve256_apply_K_full_field(B, rve256):
    """256^3 cell (1000 grains, hexagonal Ti-like, Haar): the FP32 operator on
    the whole field against the oracle, one wave vector of the path."""
    import torch
    p, med = rve256
    plan = B.Plan.from_problem(p, precision=1)
    k = p.k_list[[70]]
    u = synth.random_field(p.grid, 23, batch=1)
    du = torch.from_numpy(u).to(device="cuda", dtype=torch.complex64)
    out = torch.zeros_like(du)
    plan.apply_K(k, du, out)
    got = out.cpu().numpy()[0].astype(np.complex128)
    want = O.apply_K(med, k[0], u[0])
    assert O.norm(got - want) / O.norm(want) < 5e-6    # the FP32 operator tolerance of the op tests


def test_rve256_chosen_form_eigenpairs(B, rve256):
    """256^3, 12 bands at one wave vector with the FP32 chosen form: the FP64
    oracle's Rayleigh quotients of the lowest and highest returned vectors give
    the reported frequencies to 1e-6, and their residuals are at the
    eigensolver's tolerance."""
    import torch
    p, med = rve256
    ks = p.k_list[[9]]
    plan = B.Plan.from_problem(p, block=p.n_bands + 2, **CHOSEN)
    vecs = torch.zeros(p.n_bands * 3 * plan.V, dtype=torch.complex64, device="cuda")
    got, stats, _ = plan.solve_bands(ks, p.n_bands, vecs_out=vecs)
    assert np.all(np.diff(got[0]) >= 0) and got[0, 0] > 0
    V = vecs.cpu().numpy().reshape(p.n_bands, 3, *reversed(p.grid))
    for b in (0, p.n_bands - 1):
        lam, res = O.rayleigh_quotients(med, ks[0], V[b].astype(np.complex128)[None])
        assert abs(math.sqrt(lam[0]) / got[0, b] - 1) < 1e-6
        assert res[0] < 2e-4

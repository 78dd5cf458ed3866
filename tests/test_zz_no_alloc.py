"""The allocation-free stiffness apply (bloch_apply_K_noalloc) against the
regular one (bloch_apply_K), called through the C ABI.

Callers that cannot allocate device memory when they apply the operator (a
service with a fixed device-memory budget, a real-time loop in which a
cudaMalloc may stall the device) use the allocation-free entry point; it must
give the regular entry point's result.  Two calls in a row with
different wave vectors and fields check that the shared fixed scratch left by
one call does not leak into the next.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2106_12487_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 5e-6   # FP32 tolerance of the operator tests


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_12487_gb300 import bloch, build
    build.build()
    bloch.lib()
    return bloch


def _call_noalloc(B, plan, k, u, out):
    kv = np.ascontiguousarray(np.asarray(k, dtype=np.float64).reshape(-1, 3))
    nb = kv.shape[0]
    st = B.lib().bloch_apply_K_noalloc(plan.handle, nb, kv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr()))
    return st


@pytest.mark.parametrize("grid,nb", [((128, 128, 128), 1), ((64, 64, 64), 4), ((24, 20, 12), 3)])
def test_noalloc_matches_apply_K_twice(B, grid, nb):
    import torch
    p = synth.small_polycrystal(grid, 12, 17) if grid != (128, 128, 128) else synth.workload("rve128_g200")
    plan = B.Plan.from_problem(p, precision=B.FP32)
    for call in range(2):
        ks = (np.array([[0.31, -0.12, 0.77], [1.0, 0.0, 0.0], [0.2, 0.5, 0.0], [0.0, 0.0, 0.0]])[:nb]
              * math.pi / 1e-3 * (1.0 + 0.5 * call))
        u = torch.from_numpy(synth.random_field(grid, 40 + call, batch=nb)).to(device="cuda",
                                                                             dtype=torch.complex64)
        ref = torch.empty_like(u)
        got = torch.full_like(u, float("nan"))
        plan.apply_K(ks, u, ref)
        st = _call_noalloc(B, plan, ks, u, got)
        assert st == 0, B.lib().bloch_last_error()
        torch.cuda.synchronize()
        # complex128 before any norm: the SI-scaled outputs (~1e22 per entry)
        # would overflow a squared norm taken in FP32
        r = ref.cpu().numpy().astype(np.complex128).reshape(nb, -1)
        g = got.cpu().numpy().astype(np.complex128).reshape(nb, -1)
        assert np.all(np.isfinite(g))
        for b in range(nb):
            den = np.linalg.norm(r[b])
            assert np.isfinite(den) and den > 0
            assert np.linalg.norm(g[b] - r[b]) / den < TOL


def test_noalloc_rejects_oversize(B):
    import torch
    p = synth.small_polycrystal((64, 64, 64), 4, 3)
    plan = B.Plan.from_problem(p, precision=B.FP32)
    nb = 9   # 9 * 64^3 > 2^21
    u = torch.zeros(nb * 3 * 64 ** 3, dtype=torch.complex64, device="cuda")
    st = _call_noalloc(B, plan, np.zeros((nb, 3)), u, torch.zeros_like(u))
    assert st == 1
    assert b"2097152" in B.lib().bloch_last_error()


def test_noalloc_call_allocates_nothing(B):
    """After one warm-up call on the device (which loads the module holding the
    fixed scratch), a call on a fresh plan with a batch larger than that plan
    has ever seen changes neither the plan's device bytes nor the device's
    free memory: the regular apply would have grown the plan's workspace."""
    import torch
    grid = (32, 32, 32)
    p = synth.small_polycrystal(grid, 6, 23)
    warm = B.Plan.from_problem(p, precision=B.FP32)
    u1 = torch.from_numpy(synth.random_field(grid, 3)).to(device="cuda", dtype=torch.complex64)
    assert _call_noalloc(B, warm, np.array([[0.2, 0.1, 0.3]]) * 1e3, u1, torch.empty_like(u1)) == 0
    torch.cuda.synchronize()
    nb = 8
    u = torch.from_numpy(synth.random_field(grid, 5, batch=nb)).to(device="cuda", dtype=torch.complex64)
    out = torch.empty_like(u)
    fresh = B.Plan.from_problem(p, precision=B.FP32)
    torch.cuda.synchronize()
    bytes0 = fresh.device_bytes
    free0 = torch.cuda.mem_get_info()[0]
    ks = np.tile([[0.5, -0.3, 0.25]], (nb, 1)) * 1e3
    assert _call_noalloc(B, fresh, ks, u, out) == 0, B.lib().bloch_last_error()
    torch.cuda.synchronize()
    assert fresh.device_bytes == bytes0
    assert torch.cuda.mem_get_info()[0] == free0
    # the regular apply grows the workspace of the same plan (what the entry point avoids)
    ref = torch.empty_like(u)
    fresh.apply_K(ks, u, ref)
    torch.cuda.synchronize()
    assert fresh.device_bytes > bytes0
    r = ref.cpu().numpy().astype(np.complex128).reshape(nb, -1)
    g = out.cpu().numpy().astype(np.complex128).reshape(nb, -1)
    assert np.max(np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)) < TOL

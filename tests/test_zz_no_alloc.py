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
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        for b in range(nb):
            den = np.linalg.norm(r[b])
            if den == 0:
                assert np.linalg.norm(g[b]) == 0
            else:
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

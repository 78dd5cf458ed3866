"""Host-side checks of the seeded input generators (no method arithmetic)."""
import math

import numpy as np

from paper_2106_12487_gb300 import synth


def test_rotations_are_proper_orthogonal():
    for R in list(synth.haar_rotations(20, 1)) + list(synth.vmf_fibre_rotations(20, 20.0, 2)):
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
        assert abs(np.linalg.det(R) - 1.0) < 1e-12


def test_vmf_fibre_concentrates_about_z():
    R = synth.vmf_fibre_rotations(4000, 20.0, 3)
    w = R[:, 2, 2]          # cos angle between crystal [001] and sample z
    # E[cos theta] for vMF on S^2: coth(kappa) - 1/kappa
    assert abs(w.mean() - (1 / math.tanh(20.0) - 1 / 20.0)) < 5e-3
    haar = synth.haar_rotations(4000, 4)
    assert abs(haar[:, 2, 2].mean()) < 0.05


def test_rotate_voigt_identity_and_symmetry():
    C = synth.cubic_voigt(168.4e9, 121.4e9, 75.4e9)
    assert np.allclose(synth.rotate_voigt(C, np.eye(3)), C)
    R = synth.haar_rotations(1, 8)[0]
    Cr = synth.rotate_voigt(C, R)
    assert np.allclose(Cr, Cr.T)
    assert np.all(np.linalg.eigvalsh(Cr) > 0)
    # isotropic stiffness is rotation invariant
    Ci = synth.isotropic_voigt(50e9, 30e9)
    assert np.allclose(synth.rotate_voigt(Ci, R), Ci, rtol=1e-12, atol=1e-3)


def test_voronoi_ids_and_periodicity():
    ids = synth.voronoi_periodic((16, 12, 8), 10, 5)
    assert ids.shape == (8, 12, 16) and ids.dtype == np.int32
    assert ids.min() >= 0 and ids.max() < 10
    assert len(np.unique(ids)) >= 8
    assert np.array_equal(ids, synth.voronoi_periodic((16, 12, 8), 10, 5))


def test_kpath_endpoints_and_spacing():
    k = synth.kpath("GXMGR", 9)
    assert np.allclose(k[0], 0) and np.allclose(k[-1], [math.pi / 1e-3] * 3)
    d = np.linalg.norm(np.diff(k, axis=0), axis=1)
    # equal arc-length steps never exceed the straight segments' spacing
    assert d.max() <= d.min() * 1.0001 or np.all(d > 0)
    k2 = synth.kpath("GX", 10)
    assert np.allclose(np.diff(k2[:, 0]), math.pi / 1e-3 / 9)


def test_zener_cell_family():
    """Training family of the learned preconditioner: Zener ratio and grain
    count in range, C44 = A (C11 - C12) / 2 before rotation (the rotation
    invariant C11 + C22 + C33 + 2 (C44 + C55 + C66) checks it), reproducible."""
    a = synth.zener_cell((8, 8, 8), 3)
    b = synth.zener_cell((8, 8, 8), 3)
    assert np.array_equal(a.grain_ids, b.grain_ids) and np.allclose(a.C_per_grain, b.C_per_grain)
    A = a.meta["zener"]
    assert 1.0 <= A <= 4.0 and 20 <= a.G <= 200
    C11, C12 = synth.CU_CUBIC["C11"], synth.CU_CUBIC["C12"]
    C44 = A * (C11 - C12) / 2
    inv = [np.trace(C[:3, :3]) + 2 * np.trace(C[3:, 3:]) for C in a.C_per_grain]
    assert np.allclose(inv, 3 * C11 + 6 * C44, rtol=1e-12)
    assert len(np.unique(a.grain_ids)) <= a.G
    assert synth.zener_cell((8, 8, 8), 4).meta["zener"] != A


def test_fibre_composite_cells():
    import math
    for shape, frac in (("circle", 0.55), ("square", 0.65)):
        p = synth.fibre_composite((128, 128, 1), shape)
        assert p.grain_ids.shape == (1, 128, 128)
        assert abs(p.meta["fibre_fraction"] - frac) < 0.015   # voxelised boundary at 128^2
        ids = p.grain_ids[0]
        # centred and mirror-symmetric in x and y
        assert np.array_equal(ids, ids[::-1, :]) and np.array_equal(ids, ids[:, ::-1])
        assert ids[64, 64] == 1 and ids[0, 0] == 0
        assert p.rho.tolist() == [1200.0, 1750.0]
        assert p.k_list.shape == (90, 3) and np.allclose(p.k_list[0], [math.pi / 1e-3, math.pi / 1e-3, 0])
        assert np.any(np.all(p.k_list == 0, axis=1))      # the path passes through Gamma

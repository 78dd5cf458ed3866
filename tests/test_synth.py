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

"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every function include/bloch.h declares; the host dense eigensolver
(projected problem of Algorithm 1) matches LAPACK."""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.linalg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "bloch.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\*?\s*(bloch_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libb():
    from paper_2106_12487_gb300 import bloch, build
    build.build()
    return bloch.lib()


def test_exports_every_declared_symbol(libb):
    names = header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(libb, n), n
    from paper_2106_12487_gb300 import bloch
    assert set(bloch.EXPORTED) == set(names)


def test_default_options_and_errors_without_gpu(libb):
    from paper_2106_12487_gb300 import bloch
    o = bloch.default_options()
    assert o.precision == bloch.FP64 and o.method == bloch.SUBSPACE
    assert o.tol_lin == 1e-10 and o.max_cg == 2000
    # invalid arguments are rejected before any device work
    h = ctypes.c_void_p()
    grid = (ctypes.c_int32 * 3)(4, 4, 11)   # prime factor 11
    L = (ctypes.c_double * 3)(1e-3, 1e-3, 1e-3)
    ids = (ctypes.c_int32 * 176)()
    C = (ctypes.c_double * 36)(*np.eye(6).ravel())
    rho = (ctypes.c_double * 1)(1000.0)
    st = libb.bloch_plan_create(ctypes.byref(h), grid, L, ids, 1, C, rho, None, None)
    assert st == 7 and not h.value
    assert b"prime factors" in libb.bloch_last_error()
    grid = (ctypes.c_int32 * 3)(4, 4, 4)
    ids = (ctypes.c_int32 * 64)(*([0] * 63 + [3]))
    st = libb.bloch_plan_create(ctypes.byref(h), grid, L, ids, 1, C, rho, None, None)
    assert st == 1 and b"grain id" in libb.bloch_last_error()
    Cbad = (ctypes.c_double * 36)(*(-np.eye(6)).ravel())
    ids = (ctypes.c_int32 * 64)()
    st = libb.bloch_plan_create(ctypes.byref(h), grid, L, ids, 1, Cbad, rho, None, None)
    assert st == 1 and b"positive definite" in libb.bloch_last_error()
    rho0 = (ctypes.c_double * 1)(0.0)
    st = libb.bloch_plan_create(ctypes.byref(h), grid, L, ids, 1, C, rho0, None, None)
    assert st == 1 and b"density" in libb.bloch_last_error()
    assert libb.bloch_apply_K(None, 1, None, 0, None, None) == 1
    for field, bad, msg in (("tile_pmax", 5, b"tile_pmax"), ("fft_variant", 3, b"fft_variant"),
                            ("tensor_gram", 2, b"tensor_gram")):
        ob = bloch.default_options(**{field: bad})
        st = libb.bloch_plan_create(ctypes.byref(h), grid, L, ids, 1, C, rho, ctypes.byref(ob), None)
        assert st == 1 and not h.value and msg in libb.bloch_last_error()
    assert bloch.default_options().autotune == 0 and bloch.default_options().tile_pmax == 0
    rep = bloch.TuneReport()
    assert libb.bloch_plan_autotune(None, bloch.FP32, 4, ctypes.byref(rep)) == 1


@pytest.mark.parametrize("n", [1, 2, 5, 18, 32])
def test_host_gen_eig_matches_lapack(libb, n):
    from paper_2106_12487_gb300 import bloch
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    K = A @ A.conj().T
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    M = B @ B.conj().T + n * np.eye(n)
    lam, Q = bloch.host_gen_eig(K, M)
    ref = scipy.linalg.eigh(K, M, eigvals_only=True)
    assert np.allclose(lam, ref, rtol=1e-12, atol=1e-12 * abs(ref).max())
    assert np.allclose(Q.conj().T @ M @ Q, np.eye(n), atol=1e-12)
    assert np.allclose(K @ Q, M @ Q @ np.diag(lam), atol=1e-11 * abs(K).max())


def test_host_gen_eig_degenerate_cluster(libb):
    from paper_2106_12487_gb300 import bloch
    rng = np.random.default_rng(3)
    n = 9
    Uq, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    K = Uq @ np.diag([1, 1, 1, 2, 2, 5, 5, 5, 5]).astype(complex) @ Uq.conj().T
    lam, Q = bloch.host_gen_eig(K, np.eye(n))
    assert np.allclose(lam, [1, 1, 1, 2, 2, 5, 5, 5, 5], atol=1e-13)
    assert np.allclose(Q.conj().T @ Q, np.eye(n), atol=1e-13)


def test_struct_layouts_match_the_binding(tmp_path):
    """The ctypes mirrors of the header's structs (options, stats, tune
    report, trace) have the C compiler's sizes and field offsets."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2106_12487_gb300 import bloch
    structs = {"bloch_options": bloch.Options, "bloch_stats": bloch.Stats,
               "bloch_tune_report": bloch.TuneReport, "bloch_trace": bloch.Trace}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "bloch.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)

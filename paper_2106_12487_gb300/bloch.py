"""Thin Python binding of libbloch (ctypes): argument marshalling only.

Every step of the hot path runs in the CUDA library; this module converts
numpy/torch arguments into the plain pointers and sizes of the C ABI declared
in include/bloch.h, and raises on a non-OK status.  There is no fallback: if
the shared library cannot be loaded the import of `lib()` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbloch.so")

BLOCH_OK = 0
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV_CG", 5: "ENOTCONV_EIG",
          6: "ENONFINITE", 7: "EUNSUPPORTED"}
FP64, FP32, FF = 0, 1, 2
LANCZOS, SUBSPACE, LOBPCG = 0, 1, 2

EXPORTED = ["bloch_default_options", "bloch_plan_create", "bloch_plan_destroy", "bloch_apply_K",
            "bloch_apply_M", "bloch_apply_precond", "bloch_pcg", "bloch_solve_bands",
            "bloch_host_gen_eig", "bloch_last_error", "bloch_plan_device_bytes", "bloch_plan_kernel_launches",
            "bloch_apply_K_noalloc", "bloch_lp_num_params", "bloch_lp_create", "bloch_lp_destroy", "bloch_lp_params",
            "bloch_lp_collect", "bloch_lp_loss_grad", "bloch_lp_train", "bloch_lp_num_blocks", "bloch_lp_export_block",
            "bloch_plan_set_preconditioner", "bloch_plan_autotune",
            "bloch_plan_trace", "bloch_apply_K_real", "bloch_lp_add_pairs", "bloch_group_velocity",
            "bloch_eigvec_real", "bloch_fma_peaks"]


class BlochError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("method", ctypes.c_int32), ("tol_lin", ctypes.c_double),
                ("tol_eig", ctypes.c_double), ("max_cg", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("block", ctypes.c_int32), ("k_batch", ctypes.c_int32), ("ncv", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("cuda_graph", ctypes.c_int32), ("fft_variant", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("tile_pmax", ctypes.c_int32), ("tensor_gram", ctypes.c_int32),
                ("hybrid_tol", ctypes.c_double), ("refine_arith", ctypes.c_int32)]


class Trace(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 10), ("count", ctypes.c_int64 * 10)]

    PHASES = ("pcg_subspace", "pcg_lanczos", "residual_fp32", "residual_fp64", "lanczos_orth", "projection",
              "lanczos_restart", "setup", "gpu_span", "wall")

    def as_dict(self):
        return {ph: {"ms": self.ms[i], "count": int(self.count[i])} for i, ph in enumerate(self.PHASES)}


class TuneReport(ctypes.Structure):
    _fields_ = [("fft_variant", ctypes.c_int32), ("tile_pmax", ctypes.c_int32),
                ("saturating_systems", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("ms_per_system", ctypes.c_double * 3)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_[:4]}
        d["ms_per_system"] = list(self.ms_per_system)
        return d


class Stats(ctypes.Structure):
    _fields_ = [("cg_iterations", ctypes.c_int64), ("linear_solves", ctypes.c_int64),
                ("k_applies", ctypes.c_int64), ("outer_iterations", ctypes.c_int64),
                ("max_rel_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("k_unconverged", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_LIB = None


def lib():
    """Load libbloch.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libbloch.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, D, I32, VP = ctypes.POINTER, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p
    L.bloch_default_options.argtypes = [P(Options)]
    L.bloch_default_options.restype = None
    L.bloch_plan_create.argtypes = [P(VP), P(I32), P(D), P(I32), I32, P(D), P(D), P(Options), VP]
    L.bloch_plan_destroy.argtypes = [VP]
    L.bloch_plan_destroy.restype = None
    L.bloch_apply_K.argtypes = [VP, I32, P(D), I32, VP, VP]
    L.bloch_apply_K_real.argtypes = [VP, I32, P(D), I32, VP, VP]
    L.bloch_apply_M.argtypes = [VP, I32, I32, VP, VP]
    L.bloch_apply_K_noalloc.argtypes = [VP, I32, P(D), VP, VP]
    L.bloch_apply_precond.argtypes = [VP, I32, P(D), I32, VP, VP]
    L.bloch_pcg.argtypes = [VP, I32, P(D), I32, VP, VP, D, I32, I32, P(I32), P(D)]
    L.bloch_solve_bands.argtypes = [VP, I32, P(D), I32, P(D), VP, P(Stats)]
    L.bloch_host_gen_eig.argtypes = [I32, P(D), P(D), P(D), P(D)]
    L.bloch_group_velocity.argtypes = [VP, I32, P(D), I32, VP, P(D), P(D)]
    L.bloch_eigvec_real.argtypes = [VP, I32, I32, VP, VP, VP, P(D)]
    L.bloch_last_error.argtypes = []
    L.bloch_last_error.restype = ctypes.c_char_p
    L.bloch_plan_device_bytes.argtypes = [VP]
    L.bloch_plan_device_bytes.restype = ctypes.c_size_t
    L.bloch_plan_kernel_launches.argtypes = [VP]
    L.bloch_plan_kernel_launches.restype = ctypes.c_uint64
    U64 = ctypes.c_uint64
    L.bloch_lp_num_params.argtypes = []
    L.bloch_lp_num_params.restype = ctypes.c_int32
    L.bloch_lp_create.argtypes = [P(VP), U64]
    L.bloch_lp_destroy.argtypes = [VP]
    L.bloch_lp_destroy.restype = None
    L.bloch_lp_params.argtypes = [VP, P(D), P(D)]
    L.bloch_lp_collect.argtypes = [VP, VP, I32, P(D), I32, I32, U64]
    L.bloch_lp_add_pairs.argtypes = [VP, VP, P(D), I32, VP, VP]
    L.bloch_lp_loss_grad.argtypes = [VP, P(D), P(D)]
    L.bloch_lp_train.argtypes = [VP, I32, D, P(D)]
    L.bloch_lp_num_blocks.argtypes = [VP]
    L.bloch_lp_num_blocks.restype = ctypes.c_int32
    L.bloch_lp_export_block.argtypes = [VP, I32, P(I32), P(D), P(D), P(D), P(I32)]
    L.bloch_plan_set_preconditioner.argtypes = [VP, VP]
    L.bloch_plan_autotune.argtypes = [VP, I32, I32, P(TuneReport)]
    L.bloch_plan_trace.argtypes = [VP, I32, P(Trace)]
    L.bloch_fma_peaks.argtypes = [P(D), P(D)]
    for f in ["bloch_lp_create", "bloch_lp_params", "bloch_lp_collect", "bloch_lp_add_pairs", "bloch_lp_loss_grad",
              "bloch_lp_train",
              "bloch_lp_export_block", "bloch_plan_set_preconditioner"]:
        getattr(L, f).restype = ctypes.c_int
    for f in ["bloch_plan_create", "bloch_apply_K", "bloch_apply_K_noalloc", "bloch_apply_M", "bloch_apply_precond", "bloch_pcg",
              "bloch_solve_bands", "bloch_host_gen_eig", "bloch_plan_autotune", "bloch_plan_trace",
              "bloch_apply_K_real", "bloch_group_velocity", "bloch_eigvec_real", "bloch_fma_peaks"]:
        getattr(L, f).restype = ctypes.c_int
    _LIB = L
    return L


def _check(st: int, allow=()):
    if st != BLOCH_OK and st not in allow:
        raise BlochError(st, lib().bloch_last_error().decode())
    return st


def _dptr(arr, what):
    return ctypes.cast(arr.ctypes.data, ctypes.POINTER(what))


def default_options(**kw) -> Options:
    o = Options()
    lib().bloch_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _tensor_ptr(t, precision: int, n_expected: int):
    import torch
    want = torch.complex64 if precision == FP32 else torch.complex128   # FP64 and FF use double2
    if t.dtype != want:
        raise TypeError(f"expected {want}, got {t.dtype}")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device tensors must be contiguous CUDA tensors")
    if t.numel() != n_expected:
        raise ValueError(f"expected {n_expected} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A voxelised periodic cell on the GPU (bloch_plan_create)."""

    def __init__(self, grid, L, grain_ids, C_per_grain, rho, options: Options | None = None, stream=None):
        Nx, Ny, Nz = (int(v) for v in grid)
        self.grid = (Nx, Ny, Nz)
        self.V = Nx * Ny * Nz
        g = np.ascontiguousarray(np.asarray(grid, dtype=np.int32))
        Lv = np.ascontiguousarray(np.asarray(L, dtype=np.float64))
        ids = np.ascontiguousarray(np.asarray(grain_ids, dtype=np.int32).reshape(-1))
        C = np.ascontiguousarray(np.asarray(C_per_grain, dtype=np.float64).reshape(-1))
        r = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(-1))
        if ids.size != self.V:
            raise ValueError("grain_ids must hold Nx*Ny*Nz values")
        G = r.size
        if C.size != 36 * G:
            raise ValueError("C_per_grain must be G x 6 x 6")
        self.options = options if options is not None else default_options()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        _check(lib().bloch_plan_create(ctypes.byref(h), _dptr(g, ctypes.c_int32), _dptr(Lv, ctypes.c_double),
                                       _dptr(ids, ctypes.c_int32), G, _dptr(C, ctypes.c_double),
                                       _dptr(r, ctypes.c_double), ctypes.byref(self.options),
                                       ctypes.c_void_p(stream)))
        self.handle = h
        self.precision = self.options.precision

    @classmethod
    def from_problem(cls, p, **opt):
        return cls(p.grid, p.L, p.grain_ids, p.C_per_grain, p.rho, default_options(**opt))

    def close(self):
        if getattr(self, "handle", None):
            lib().bloch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def kernel_launches(self) -> int:
        return int(lib().bloch_plan_kernel_launches(self.handle))

    @property
    def device_bytes(self) -> int:
        return int(lib().bloch_plan_device_bytes(self.handle))

    def trace(self, enable: bool) -> dict:
        """bloch_plan_trace: phase times since the previous call (ms), then
        switch tracing on or off."""
        tr = Trace()
        _check(lib().bloch_plan_trace(self.handle, 1 if enable else 0, ctypes.byref(tr)))
        return tr.as_dict()

    def autotune(self, precision: int, systems: int) -> dict:
        """bloch_plan_autotune: time the operator's pass configurations on
        `systems` systems and keep the fastest; returns the report."""
        rep = TuneReport()
        _check(lib().bloch_plan_autotune(self.handle, int(precision), int(systems), ctypes.byref(rep)))
        return rep.as_dict()

    # ---------------------------------------------------------------- ops
    def _kv(self, k, nb):
        kv = np.ascontiguousarray(np.broadcast_to(np.asarray(k, dtype=np.float64).reshape(-1, 3), (nb, 3)))
        return kv

    def apply_K(self, k, u, out, precision: int | None = None):
        prec = self.precision if precision is None else precision
        nb = u.numel() // (3 * self.V)
        kv = self._kv(k, nb)
        _check(lib().bloch_apply_K(self.handle, nb, _dptr(kv, ctypes.c_double), prec,
                                   _tensor_ptr(u, prec, nb * 3 * self.V), _tensor_ptr(out, prec, nb * 3 * self.V)))
        return out

    def apply_K_real(self, k, u, out, precision: int | None = None):
        """bloch_apply_K_real: the stiffness operator on real-space grid values."""
        prec = self.precision if precision is None else precision
        nb = u.numel() // (3 * self.V)
        kv = self._kv(k, nb)
        _check(lib().bloch_apply_K_real(self.handle, nb, _dptr(kv, ctypes.c_double), prec,
                                        _tensor_ptr(u, prec, nb * 3 * self.V), _tensor_ptr(out, prec, nb * 3 * self.V)))
        return out

    def apply_K_noalloc(self, k, u, out):
        """Allocation-free FP32 stiffness apply (fixed library-owned scratch)."""
        nb = u.numel() // (3 * self.V)
        kv = self._kv(k, nb)
        _check(lib().bloch_apply_K_noalloc(self.handle, nb, _dptr(kv, ctypes.c_double),
                                           _tensor_ptr(u, FP32, nb * 3 * self.V),
                                           _tensor_ptr(out, FP32, nb * 3 * self.V)))
        return out

    def apply_M(self, u, out, precision: int | None = None):
        prec = self.precision if precision is None else precision
        nb = u.numel() // (3 * self.V)
        _check(lib().bloch_apply_M(self.handle, nb, prec, _tensor_ptr(u, prec, nb * 3 * self.V),
                                   _tensor_ptr(out, prec, nb * 3 * self.V)))
        return out

    def apply_precond(self, k, r, out, precision: int | None = None):
        prec = self.precision if precision is None else precision
        nb = r.numel() // (3 * self.V)
        kv = self._kv(k, nb)
        _check(lib().bloch_apply_precond(self.handle, nb, _dptr(kv, ctypes.c_double), prec,
                                         _tensor_ptr(r, prec, nb * 3 * self.V),
                                         _tensor_ptr(out, prec, nb * 3 * self.V)))
        return out

    def pcg(self, k, b, x, tol, max_iter=10000, x0=False, precision: int | None = None, allow_nonconv=False):
        prec = self.precision if precision is None else precision
        nb = b.numel() // (3 * self.V)
        kv = self._kv(k, nb)
        iters = np.zeros(nb, dtype=np.int32)
        rel = np.zeros(nb, dtype=np.float64)
        st = lib().bloch_pcg(self.handle, nb, _dptr(kv, ctypes.c_double), prec,
                             _tensor_ptr(b, prec, nb * 3 * self.V), _tensor_ptr(x, prec, nb * 3 * self.V),
                             float(tol), int(max_iter), 1 if x0 else 0, _dptr(iters, ctypes.c_int32),
                             _dptr(rel, ctypes.c_double))
        _check(st, allow=(4,) if allow_nonconv else ())
        return iters, rel, st

    def group_velocity(self, k, u, precision: int | None = None):
        """bloch_group_velocity: (omega (nb,), c (nb, 3)) of the vectors u
        (nb x 3 x V, Fourier basis) at wave vectors k (nb x 3 or 3)."""
        prec = self.precision if precision is None else precision
        nb = u.numel() // (3 * self.V)
        kv = self._kv(k, nb)
        om = np.zeros(nb)
        c = np.zeros((nb, 3))
        _check(lib().bloch_group_velocity(self.handle, nb, _dptr(kv, ctypes.c_double), prec,
                                          _tensor_ptr(u, prec, nb * 3 * self.V), _dptr(om, ctypes.c_double),
                                          _dptr(c, ctypes.c_double)))
        return om, c

    def eigvec_real(self, u_hat, u_real, strain=None, precision: int | None = None):
        """bloch_eigvec_real: phase-rotated real-space fields (and strain) of
        Fourier-basis vectors; returns the phases phi."""
        prec = self.precision if precision is None else precision
        nb = u_hat.numel() // (3 * self.V)
        phi = np.zeros(nb)
        sp = None if strain is None else _tensor_ptr(strain, prec, nb * 6 * self.V)
        _check(lib().bloch_eigvec_real(self.handle, nb, prec, _tensor_ptr(u_hat, prec, nb * 3 * self.V),
                                       _tensor_ptr(u_real, prec, nb * 3 * self.V), sp, _dptr(phi, ctypes.c_double)))
        return phi

    def solve_bands(self, k_list, n_bands, vecs_out=None, allow_nonconv=False):
        kl = np.ascontiguousarray(np.asarray(k_list, dtype=np.float64).reshape(-1, 3))
        nk = kl.shape[0]
        omega = np.zeros((nk, n_bands), dtype=np.float64)
        stats = Stats()
        vp = None
        if vecs_out is not None:
            vp = _tensor_ptr(vecs_out, self.precision, nk * n_bands * 3 * self.V)
        st = lib().bloch_solve_bands(self.handle, nk, _dptr(kl, ctypes.c_double), int(n_bands),
                                     _dptr(omega, ctypes.c_double), vp, ctypes.byref(stats))
        _check(st, allow=(5,) if allow_nonconv else ())
        return omega, stats.as_dict(), st


def host_gen_eig(K: np.ndarray, M: np.ndarray):
    """Dense generalised Hermitian eigensolver of the library (host, no GPU)."""
    n = K.shape[0]
    Kc = np.ascontiguousarray(K.astype(np.complex128)).view(np.float64)
    Mc = np.ascontiguousarray(M.astype(np.complex128)).view(np.float64)
    lam = np.zeros(n)
    Q = np.zeros((n, n), dtype=np.complex128)
    Qv = Q.view(np.float64)
    _check(lib().bloch_host_gen_eig(n, _dptr(Kc, ctypes.c_double), _dptr(Mc, ctypes.c_double),
                                    _dptr(lam, ctypes.c_double), _dptr(Qv, ctypes.c_double)))
    return lam, Q


class LearnedPrecond:
    """Learned Fourier-space preconditioner (bloch_lp_*): collect, train, use."""

    def __init__(self, seed: int = 7):
        h = ctypes.c_void_p()
        _check(lib().bloch_lp_create(ctypes.byref(h), int(seed)))
        self.handle = h
        self.n = int(lib().bloch_lp_num_params())

    def close(self):
        if getattr(self, "handle", None):
            lib().bloch_lp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self, set_to=None):
        out = np.zeros(self.n)
        sp = None
        if set_to is not None:
            sv = np.ascontiguousarray(np.asarray(set_to, dtype=np.float64))
            sp = _dptr(sv, ctypes.c_double)
        _check(lib().bloch_lp_params(self.handle, _dptr(out, ctypes.c_double), sp))
        return out

    def collect(self, plan: Plan, k_list, n_rhs=4, n_iters=8, seed=11):
        kl = np.ascontiguousarray(np.asarray(k_list, dtype=np.float64).reshape(-1, 3))
        _check(lib().bloch_lp_collect(self.handle, plan.handle, kl.shape[0], _dptr(kl, ctypes.c_double),
                                      int(n_rhs), int(n_iters), int(seed)))

    def add_pairs(self, plan: Plan, k, r, e):
        """bloch_lp_add_pairs: one data block from caller-supplied (r_j, e_j) pairs
        (complex64 CUDA tensors of n_pairs x 3 x V values, Fourier basis)."""
        n = r.numel() // (3 * plan.V)
        kv = np.ascontiguousarray(np.asarray(k, dtype=np.float64).reshape(3))
        _check(lib().bloch_lp_add_pairs(self.handle, plan.handle, _dptr(kv, ctypes.c_double), n,
                                        _tensor_ptr(r, FP32, n * 3 * plan.V), _tensor_ptr(e, FP32, n * 3 * plan.V)))

    def loss_grad(self):
        L = np.zeros(1)
        g = np.zeros(self.n)
        _check(lib().bloch_lp_loss_grad(self.handle, _dptr(L, ctypes.c_double), _dptr(g, ctypes.c_double)))
        return float(L[0]), g

    def train(self, steps, lr=1e-2):
        hist = np.zeros(max(steps, 1))
        _check(lib().bloch_lp_train(self.handle, int(steps), float(lr), _dptr(hist, ctypes.c_double)))
        return hist[:steps]

    @property
    def num_blocks(self):
        return int(lib().bloch_lp_num_blocks(self.handle))

    def export_block(self, i):
        grid = np.zeros(3, dtype=np.int32)
        _check(lib().bloch_lp_export_block(self.handle, i, _dptr(grid, ctypes.c_int32), None, None, None, None))
        S = int(grid.sum())
        V = int(np.prod(grid))
        q = np.zeros(S)
        mom = np.zeros(V * 13)
        C0V = np.zeros(36)
        ns = np.zeros(1, dtype=np.int32)
        _check(lib().bloch_lp_export_block(self.handle, i, _dptr(grid, ctypes.c_int32), _dptr(q, ctypes.c_double),
                                           _dptr(mom, ctypes.c_double), _dptr(C0V, ctypes.c_double),
                                           _dptr(ns, ctypes.c_int32)))
        return dict(grid=tuple(int(v) for v in grid), q=q, mom=mom.reshape(V, 13), C0V=C0V.reshape(6, 6),
                    samples=int(ns[0]))


def fma_peaks() -> tuple[float, float]:
    """bloch_fma_peaks: measured FP64 and FP32 FMA throughput (GFLOP/s) of
    the current device."""
    g64 = ctypes.c_double(0.0)
    g32 = ctypes.c_double(0.0)
    _check(lib().bloch_fma_peaks(ctypes.byref(g64), ctypes.byref(g32)))
    return g64.value, g32.value


def set_preconditioner(plan: Plan, lp: "LearnedPrecond | None"):
    _check(lib().bloch_plan_set_preconditioner(plan.handle, lp.handle if lp is not None else None))

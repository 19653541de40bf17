"""Thin ctypes binding of libesmp2 (include/esmp2.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; PyTorch supplies
device memory and the current stream.  The binding never falls back to host code: if
the library cannot be loaded, importing it raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libesmp2.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_NOT_CONVERGED, ERR_INDEFINITE, ERR_CUDA, ERR_TIMEOUT, ERR_STATE = range(9)
FP64, MIXED_BF16, MIXED_TF32, FP64_TC, REDUCED_MIXED, REDUCED_MINRES = 0, 1, 2, 3, 4, 5
_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OOM", 4: "NOT_CONVERGED", 5: "INDEFINITE",
           6: "CUDA", 7: "TIMEOUT", 8: "STATE"}


class Esmp2Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"esmp2 {_STATUS.get(status, status)}: {msg}")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [("No", ctypes.c_int), ("Nv", ctypes.c_int), ("F", ctypes.c_void_p), ("ovov", ctypes.c_void_p),
                ("ooov", ctypes.c_void_p), ("ovvv", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("spin", ctypes.c_int), ("inputs_on_device", ctypes.c_int), ("eta", ctypes.c_double),
                ("n_large", ctypes.c_int), ("avo_convention", ctypes.c_int), ("level_shift", ctypes.c_double)]


class LayoutInfo(ctypes.Structure):
    _fields_ = [("No", ctypes.c_int), ("Nv", ctypes.c_int), ("block_elems", ctypes.c_int64),
                ("n_elems", ctypes.c_int64), ("weights", ctypes.c_double * 5), ("omega", ctypes.c_double),
                ("E0", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer", ctypes.c_int), ("sigma_fp64", ctypes.c_int),
                ("sigma_lowp", ctypes.c_int), ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double)]


class EnergyParts(ctypes.Structure):
    _fields_ = [("E2", ctypes.c_double), ("E2_D", ctypes.c_double), ("E2_L", ctypes.c_double),
                ("E2_S", ctypes.c_double)]


class KernelTime(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("alg_units", ctypes.c_double),
                ("exec_units", ctypes.c_double)]


class BatchResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("e2", EnergyParts), ("info", SolveInfo),
                ("kernel_launches", ctypes.c_int64), ("message", ctypes.c_char * 160)]


EXPORTS = ("esmp2_create", "esmp2_destroy", "esmp2_last_error", "esmp2_set_stream", "esmp2_layout",
           "esmp2_top_basis", "esmp2_sigma", "esmp2_rhs", "esmp2_solve", "esmp2_get_solution",
           "esmp2_set_solution", "esmp2_energy", "esmp2_kernel_launches", "esmp2_profile_sigma",
           "esmp2_virtual_contraction", "esmp2_virtual_contraction_noalloc", "esmp2_batch_solve", "esmp2_grad",
           "esmp2_kernel_timing", "esmp2_kernel_times", "esmp2_selftest_bounded_wait")
MIXED_READY = True


def lib_path() -> str:
    return _LIB_PATH


def load(path: str | None = None):
    """Load libesmp2 (no GPU needed to load it).  Raises OSError when it is missing."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or _LIB_PATH
        if not os.path.exists(p):
            raise OSError(f"libesmp2 not built: {p} is missing (run __graft_entry__.build())")
        L = ctypes.CDLL(p)
        P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        L.esmp2_create.restype = I
        L.esmp2_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Desc)]
        L.esmp2_destroy.restype = None
        L.esmp2_destroy.argtypes = [P]
        L.esmp2_last_error.restype = ctypes.c_char_p
        L.esmp2_last_error.argtypes = [P]
        L.esmp2_set_stream.restype = I
        L.esmp2_set_stream.argtypes = [P, P]
        L.esmp2_layout.restype = I
        L.esmp2_layout.argtypes = [P, ctypes.POINTER(LayoutInfo)]
        L.esmp2_top_basis.restype = I
        L.esmp2_top_basis.argtypes = [P, P, P, P, P]
        L.esmp2_sigma.restype = I
        L.esmp2_sigma.argtypes = [P, P, P, I]
        L.esmp2_rhs.restype = I
        L.esmp2_rhs.argtypes = [P, P]
        L.esmp2_solve.restype = I
        L.esmp2_solve.argtypes = [P, D, I, I, ctypes.POINTER(SolveInfo)]
        L.esmp2_get_solution.restype = I
        L.esmp2_get_solution.argtypes = [P, P]
        L.esmp2_set_solution.restype = I
        L.esmp2_set_solution.argtypes = [P, P]
        L.esmp2_energy.restype = I
        L.esmp2_energy.argtypes = [P, ctypes.POINTER(EnergyParts)]
        L.esmp2_profile_sigma.restype = I
        L.esmp2_profile_sigma.argtypes = [P, P, P, I, I, P]
        L.esmp2_virtual_contraction.restype = I
        L.esmp2_virtual_contraction.argtypes = [P, P, P, I]
        L.esmp2_virtual_contraction_noalloc.restype = I
        L.esmp2_virtual_contraction_noalloc.argtypes = [P, P, P, I, I, P]
        L.esmp2_batch_solve.restype = I
        L.esmp2_batch_solve.argtypes = [ctypes.POINTER(Desc), I, D, I, I, I, ctypes.POINTER(BatchResult)]
        L.esmp2_grad.restype = I
        L.esmp2_grad.argtypes = [P, P, P, I, P]
        L.esmp2_kernel_launches.restype = I64
        L.esmp2_kernel_launches.argtypes = [P]
        L.esmp2_kernel_timing.restype = None
        L.esmp2_kernel_timing.argtypes = [I]
        L.esmp2_kernel_times.restype = I
        L.esmp2_kernel_times.argtypes = [ctypes.POINTER(KernelTime)]
        L.esmp2_selftest_bounded_wait.restype = I
        L.esmp2_selftest_bounded_wait.argtypes = [I, P]
        if path is None:
            _lib = L
        return L


NOALLOC_MAX_BYTES = 64 << 20

KERNEL_FAMILIES = ("contraction", "coupling", "gemm64", "e2s", "digits", "precond")


def kernel_timing(enable: bool):
    """Switch the process-wide event timing of the kernel families on or off."""
    load().esmp2_kernel_timing(1 if enable else 0)


def kernel_times():
    """Totals per kernel family since the last call (see esmp2_kernel_times)."""
    out = (KernelTime * len(KERNEL_FAMILIES))()
    st = load().esmp2_kernel_times(out)
    if st != OK:
        raise Esmp2Error(st, "esmp2_kernel_times failed")
    return {name: {"launches": int(t.launches), "ms": float(t.ms), "alg_units": float(t.alg_units),
                   "exec_units": float(t.exec_units)} for name, t in zip(KERNEL_FAMILIES, out)}


def batch_solve(instances, tol: float = 1e-8, maxit: int = 2000, precision: int = FP64, concurrency: int = 2):
    """Solve independent instances (dicts with F, ovov, ooov, ovvv, C as float64 host arrays)
    through esmp2_batch_solve; returns (status, list of per-instance result dicts)."""
    L = load()
    keep = []
    descs = (Desc * len(instances))()
    for k, inst in enumerate(instances):
        arrs = [np.ascontiguousarray(np.asarray(inst[n], dtype=np.float64)) for n in ("F", "ovov", "ooov", "ovvv", "C")]
        keep.append(arrs)
        No, Nv = arrs[4].shape
        descs[k] = Desc(No, Nv, *(a.ctypes.data for a in arrs), 1, 0, 0.0, 1, 0, float(inst.get("level_shift", 0.0)))
    res = (BatchResult * len(instances))()
    st = L.esmp2_batch_solve(descs, len(instances), tol, maxit, precision, concurrency, res)
    out = []
    for r in res:
        out.append({"status": r.status, "E2": r.e2.E2, "E2_D": r.e2.E2_D, "E2_L": r.e2.E2_L, "E2_S": r.e2.E2_S,
                    "iterations": r.info.iterations, "outer": r.info.outer, "rel_residual": r.info.rel_residual,
                    "seconds": r.info.seconds, "kernel_launches": r.kernel_launches,
                    "message": r.message.decode(errors="replace")})
    return int(st), out


def virtual_contraction_noalloc(x, Fvv, y, S: int, Nv: int, stream=None) -> int:
    """Allocation-free bf16 virtual-index contraction (see include/esmp2.h); returns the status."""
    L = load()
    st = 0 if stream is None else stream.cuda_stream
    return int(L.esmp2_virtual_contraction_noalloc(x.data_ptr(), Fvv.data_ptr(), y.data_ptr(), S, Nv,
                                                   ctypes.c_void_p(st)))


def selftest_bounded_wait(wait_ms: int = 200, stream=None) -> int:
    """Failure-detection self-test of the tensor-core kernel's bounded waits (see
    include/esmp2.h); returns the status (ERR_TIMEOUT when the expiry was detected)."""
    st = 0 if stream is None else stream.cuda_stream
    return int(load().esmp2_selftest_bounded_wait(int(wait_ms), ctypes.c_void_p(st)))


def _ptr(a):
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class Handle:
    """One ESMP2-TOP(1) problem on the current CUDA device.

    Inputs (F, ovov, ooov, ovvv, C) may be float64 numpy arrays (host) or CUDA torch
    tensors; they are copied during construction."""

    def __init__(self, F, ovov, ooov, ovvv, C, spin: int = 1, stream=None, level_shift: float = 0.0,
                 eta: float = 0.0, n_large: int = 1, avo_convention: int = 0):
        import torch
        self.torch = torch
        self.L = load()
        No, Nv = C.shape
        on_dev = hasattr(F, "is_cuda") and F.is_cuda
        keep = []

        def prep(a):
            if on_dev:
                t = a.to(dtype=torch.float64).contiguous()
            else:
                t = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
            keep.append(t)
            return _ptr(t)

        d = Desc(No, Nv, prep(F), prep(ovov), prep(ooov), prep(ovvv), prep(C), spin, 1 if on_dev else 0,
                 float(eta), int(n_large), int(avo_convention), float(level_shift))
        self._h = ctypes.c_void_p()
        self.device = torch.device("cuda", torch.cuda.current_device())
        st = self.L.esmp2_create(ctypes.byref(self._h), ctypes.byref(d))
        if st != OK:
            msg = self.L.esmp2_last_error(self._h).decode() if self._h else ""
            if self._h:
                self.L.esmp2_destroy(self._h)
                self._h = None
            raise Esmp2Error(st, msg)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.L.esmp2_set_stream(self._h, ctypes.c_void_p(s.cuda_stream))
        lay = LayoutInfo()
        self._check(self.L.esmp2_layout(self._h, ctypes.byref(lay)))
        self.No, self.Nv = No, Nv
        self.n = lay.n_elems
        self.shape = (5, No, No, Nv, Nv)
        self.weights = np.array(list(lay.weights))
        self.omega, self.E0 = lay.omega, lay.E0

    def _check(self, st):
        if st != OK:
            raise Esmp2Error(st, self.L.esmp2_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self.L.esmp2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def top_basis(self):
        No, Nv = self.No, self.Nv
        U = np.empty((No, No)); lam = np.empty(No); Wv = np.empty((Nv, Nv)); F = np.empty((No + Nv, No + Nv))
        self._check(self.L.esmp2_top_basis(self._h, U.ctypes.data, lam.ctypes.data, Wv.ctypes.data, F.ctypes.data))
        return U, lam, Wv, F

    def empty(self):
        return self.torch.empty(self.shape, dtype=self.torch.float64, device=self.device)

    def sigma(self, x, precision: int = FP64, out=None):
        y = self.empty() if out is None else out
        assert x.is_contiguous() and x.dtype == self.torch.float64 and x.numel() == self.n
        self._check(self.L.esmp2_sigma(self._h, x.data_ptr(), y.data_ptr(), precision))
        return y

    def profile_sigma(self, x, precision: int = FP64, reps: int = 3, out=None):
        """Average per-stage milliseconds of `reps` sigma builds (see esmp2_profile_sigma)."""
        y = self.empty() if out is None else out
        ms = np.zeros(8)
        self._check(self.L.esmp2_profile_sigma(self._h, x.data_ptr(), y.data_ptr(), precision, reps, ms.ctypes.data))
        return ms

    def virtual_contraction(self, x, precision: int = FP64, out=None):
        y = self.empty() if out is None else out
        self._check(self.L.esmp2_virtual_contraction(self._h, x.data_ptr(), y.data_ptr(), precision))
        return y

    def rhs(self):
        b = self.empty()
        self._check(self.L.esmp2_rhs(self._h, b.data_ptr()))
        return b

    def solve(self, tol: float = 1e-10, maxit: int = 500, precision: int = FP64, raise_on_error: bool = True):
        info = SolveInfo()
        st = self.L.esmp2_solve(self._h, tol, maxit, precision, ctypes.byref(info))
        if raise_on_error:
            self._check(st)
        return {"status": st, "iterations": info.iterations, "outer": info.outer, "sigma_fp64": info.sigma_fp64,
                "sigma_lowp": info.sigma_lowp, "rel_residual": info.rel_residual, "seconds": info.seconds}

    def solution(self):
        x = self.empty()
        self._check(self.L.esmp2_get_solution(self._h, x.data_ptr()))
        return x

    def set_solution(self, x):
        self._check(self.L.esmp2_set_solution(self._h, x.contiguous().data_ptr()))

    def energy(self):
        e = EnergyParts()
        self._check(self.L.esmp2_energy(self._h, ctypes.byref(e)))
        return {"E2": e.E2, "E2_D": e.E2_D, "E2_L": e.E2_L, "E2_S": e.E2_S}

    def grad(self, adjoint_solve: bool = False):
        """(dE2/dF, dE2/d(ia|jb), adjoint |lambda - x|/|x|) in the ESMF basis (see esmp2_grad)."""
        No, Nv = self.No, self.Nv
        dF = np.empty((No + Nv, No + Nv))
        dov = np.empty((No, Nv, No, Nv))
        diff = ctypes.c_double(0.0)
        self._check(self.L.esmp2_grad(self._h, dF.ctypes.data, dov.ctypes.data, 1 if adjoint_solve else 0,
                                      ctypes.byref(diff)))
        return dF, dov, diff.value

    @property
    def kernel_launches(self) -> int:
        return int(self.L.esmp2_kernel_launches(self._h))

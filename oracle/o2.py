"""ctypes binding of the O2 oracle (o2.c) and its plain CG driver -- test infrastructure only.

The first-order equation A x = -b on D+L is solved by unpreconditioned conjugate
gradients (Sec. III.A: the paper uses CG), with the determinant-space inner
product expressed on full-storage blocks: every unique amplitude of T, X, Y is
stored 4 times and stands for 2 determinants (spin flip), S elements are unique
determinants, Z elements stand for 2 determinants (spin flip).  Hence the block
weights w = (1/2, 1, 1/2, 1/2, 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import top

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "o2.c")
_LIB = os.path.join(_HERE, "_build", "libo2.so")
_lock = threading.Lock()
_lib = None

WEIGHTS = np.array([0.5, 1.0, 0.5, 0.5, 2.0])


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
            lib.o2_create.restype = P
            lib.o2_create.argtypes = [I, I, P, P, P, P, P]
            lib.o2_destroy.argtypes = [P]
            lib.o2_omega.restype = D
            lib.o2_omega.argtypes = [P]
            lib.o2_set_shift.restype = None
            lib.o2_set_shift.argtypes = [P, D]
            lib.o2_error.restype = I
            lib.o2_error.argtypes = [P]
            lib.o2_f0vo.argtypes = [P, P]
            lib.o2_sigma_full.argtypes = [P, P, P]
            lib.o2_sigma_at.argtypes = [P, P, I64, P, P]
            lib.o2_sigma_elem.restype = D
            lib.o2_sigma_elem.argtypes = [P, P, I, I, I, I, I]
            lib.o2_rhs_full.argtypes = [P, P]
            lib.o2_rhs_at.argtypes = [P, I64, P, P]
            lib.o2_e2_s.restype = D
            lib.o2_e2_s.argtypes = [P, ctypes.POINTER(I64)]
            _lib = lib
    return _lib


class O2:
    """Oracle context in the TOP basis.  `prep` is the dict returned by oracle.top.prepare."""

    def __init__(self, prep: dict, shift: float = 0.0):
        self.No, self.Nv = prep["No"], prep["Nv"]
        self._keep = [np.ascontiguousarray(prep[k], dtype=np.float64)
                      for k in ("F", "lam", "ovov", "ooov", "ovvt")]
        F, lam, ovov, ooov, ovvt = self._keep
        self.lam = lam
        self.F = F
        self._c = _load().o2_create(self.No, self.Nv, F.ctypes.data, lam.ctypes.data,
                                    ovov.ctypes.data, ooov.ctypes.data, ovvt.ctypes.data)
        if shift:
            _load().o2_set_shift(self._c, float(shift))

    def __del__(self):
        if getattr(self, "_c", None) and _lib is not None:
            _lib.o2_destroy(self._c)
            self._c = None

    @property
    def shape(self):
        return (5, self.No, self.No, self.Nv, self.Nv)

    @property
    def omega(self) -> float:
        return _load().o2_omega(self._c)

    def f0vo(self) -> np.ndarray:
        out = np.empty((self.Nv, self.No))
        _load().o2_f0vo(self._c, out.ctypes.data)
        return out

    def _check(self):
        e = _load().o2_error(self._c)
        if e:
            raise RuntimeError(f"O2 integral accessor error {e}")

    def sigma(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.shape)
        y = np.empty_like(x)
        _load().o2_sigma_full(self._c, x.ctypes.data, y.ctypes.data)
        return y

    def sigma_at(self, x: np.ndarray, flat: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        flat = np.ascontiguousarray(flat, dtype=np.int64)
        out = np.empty(flat.shape[0])
        _load().o2_sigma_at(self._c, x.ctypes.data, flat.shape[0], flat.ctypes.data, out.ctypes.data)
        return out

    def rhs(self) -> np.ndarray:
        b = np.empty(self.shape)
        _load().o2_rhs_full(self._c, b.ctypes.data)
        self._check()
        return b

    def rhs_at(self, flat: np.ndarray) -> np.ndarray:
        flat = np.ascontiguousarray(flat, dtype=np.int64)
        out = np.empty(flat.shape[0])
        _load().o2_rhs_at(self._c, flat.shape[0], flat.ctypes.data, out.ctypes.data)
        self._check()
        return out

    def e2_s(self):
        cnt = ctypes.c_int64(0)
        v = _load().o2_e2_s(self._c, ctypes.byref(cnt))
        self._check()
        return v, cnt.value


def wdot(u: np.ndarray, v: np.ndarray) -> float:
    """Determinant-space inner product of two full-storage block vectors."""
    s = 0.0
    for k in range(5):
        s += WEIGHTS[k] * float(np.dot(u[k].ravel(), v[k].ravel()))
    return s


def cg(o: O2, b: np.ndarray, tol: float = 1e-10, maxit: int = 1000, x0=None):
    """Plain CG for A x = -b; stops on the true relative residual ||b + A x|| / ||b||."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = -b - o.sigma(x)
    p = r.copy()
    rr = wdot(r, r)
    bn = np.sqrt(wdot(b, b))
    it = 0
    hist = []
    while it < maxit:
        if np.sqrt(rr) <= tol * bn:
            rt = -b - o.sigma(x)
            if np.sqrt(wdot(rt, rt)) <= tol * bn:
                break
            r = rt
            rr = wdot(r, r)
            p = r.copy()
        Ap = o.sigma(p)
        pAp = wdot(p, Ap)
        if pAp <= 0:
            raise RuntimeError("operator not positive definite")
        alpha = rr / pAp
        x += alpha * p
        r -= alpha * Ap
        rr_new = wdot(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
        hist.append(np.sqrt(rr) / bn)
    return x, it, hist


def solve(prep: dict, tol: float = 1e-10, maxit: int = 1000, shift: float = 0.0) -> dict:
    """E2 of ESMP2-TOP(1): E2_DL by the Hylleraas functional 2 b.x + x.Ax at the CG
    solution (error quadratic in the residual), plus the direct S-space sum.  shift: level
    shift of H0 on the first-order space."""
    o = O2(prep, shift)
    b = o.rhs()
    x, it, hist = cg(o, b, tol, maxit)
    Ax = o.sigma(x)
    parts = {}
    names = ("T", "S", "X", "Y", "Z")
    for k, nm in enumerate(names):
        parts[nm] = WEIGHTS[k] * (2.0 * float(np.dot(b[k].ravel(), x[k].ravel()))
                                  + float(np.dot(x[k].ravel(), Ax[k].ravel())))
    e2s, ns = o.e2_s()
    e2_d = parts["T"] + parts["S"]
    e2_l = parts["X"] + parts["Y"] + parts["Z"]
    return {"E2": e2_d + e2_l + e2s, "E2_D": e2_d, "E2_L": e2_l, "E2_S": e2s, "n_S": ns,
            "iters": it, "hist": hist, "x": x, "b": b, "omega": o.omega}


def prepare(inst: dict) -> dict:
    return top.prepare(inst)

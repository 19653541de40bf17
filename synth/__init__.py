"""Seeded synthetic ESMP2 inputs shared by the oracle, the tests and the benchmark.

Workload recipe (the paper's molecules are not available, so these stand in for
them; the recipe follows the benchmark configurations of this project):

* F   -- symmetric (No+Nv)^2 matrix in the ESMF orbital basis; occupied diagonal
         U[-2,-0.3] Eh, virtual diagonal U[0.2,3] Eh, every off-diagonal element
         N(0, sigma_off) (sigma_off read as a standard deviation).
* ERI -- real chemist-notation integrals (pq|rs) ~ N(0, eri_sigma) with 8-fold
         permutational symmetry, drawn per canonical index by a counter-based
         generator so that any block is reproducible on its own.  Only the
         ovov, ooov and ovvv blocks are materialised.
* C   -- ESMF singles coefficients: s*G + e_t e_{a*}^T with G ~ N(0,1), t the
         occupied orbital with the highest Fock diagonal and a* the virtual with
         the lowest; s is chosen by bisection so the dominant singular weight
         lambda_1^2 / sum(lambda^2) equals `dominant`; finally 2*||C||_F^2 = 1.

The generator is plain input shaping: it holds none of the method's arithmetic,
and both the oracle and the CUDA path consume its arrays unchanged.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library in-tree (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i32, dbl, ptr = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            lib.synth_eri.restype = dbl
            lib.synth_eri.argtypes = [u64, dbl, i32, i32, i32, i32]
            lib.synth_normal.restype = dbl
            lib.synth_normal.argtypes = [u64, u64, u64]
            lib.synth_uniform.restype = dbl
            lib.synth_uniform.argtypes = [u64, u64, u64]
            lib.synth_stream_key.restype = u64
            lib.synth_stream_key.argtypes = [u64, u64]
            lib.synth_eri_block.restype = i32
            lib.synth_eri_block.argtypes = [i32, i32, i32, u64, dbl, ptr]
            lib.synth_fock.restype = None
            lib.synth_fock.argtypes = [i32, i32, u64, dbl, ptr]
            lib.synth_gauss_matrix.restype = None
            lib.synth_gauss_matrix.argtypes = [i32, i32, u64, ptr]
            _lib = lib
    return _lib


_KINDS = {"ovov": 0, "ooov": 1, "ovvv": 2, "full": 3}


def eri_block(kind: str, No: int, Nv: int, seed: int, sigma: float = 1e-2) -> np.ndarray:
    """One block of the synthetic integral tensor, float64, C-contiguous.

    ovov[i,a,j,b] = (i a|j b); ooov[i,j,k,a] = (i j|k a); ovvv[i,a,b,c] = (i a|b c);
    full[p,q,r,s] over all No+Nv orbitals (virtual a is orbital No+a)."""
    N = No + Nv
    shape = {"ovov": (No, Nv, No, Nv), "ooov": (No, No, No, Nv),
             "ovvv": (No, Nv, Nv, Nv), "full": (N, N, N, N)}[kind]
    out = np.empty(shape, dtype=np.float64)
    rc = _load().synth_eri_block(_KINDS[kind], No, Nv, seed, sigma, out.ctypes.data)
    if rc != 0:
        raise ValueError(kind)
    return out


def eri_scalar(seed: int, sigma: float, p: int, q: int, r: int, s: int) -> float:
    return _load().synth_eri(seed, sigma, p, q, r, s)


def fock(No: int, Nv: int, seed: int, sigma_off: float = 1e-3) -> np.ndarray:
    N = No + Nv
    F = np.empty((N, N), dtype=np.float64)
    _load().synth_fock(No, Nv, seed, sigma_off, F.ctypes.data)
    return F


def gauss_matrix(No: int, Nv: int, seed: int) -> np.ndarray:
    G = np.empty((No, Nv), dtype=np.float64)
    _load().synth_gauss_matrix(No, Nv, seed, G.ctypes.data)
    return G


def _dominant_weight(C: np.ndarray) -> float:
    lam = np.linalg.svd(C, compute_uv=False)
    return float(lam[0] ** 2 / np.sum(lam ** 2))


def singles_coefficients(F: np.ndarray, No: int, Nv: int, seed: int, dominant: float = 0.9) -> np.ndarray:
    """ESMF singles matrix with one dominant hole/particle pair (see module doc)."""
    diag = np.diag(F)
    t = int(np.argmax(diag[:No]))
    a_star = int(np.argmin(diag[No:]))
    G = gauss_matrix(No, Nv, seed)
    E = np.zeros((No, Nv))
    E[t, a_star] = 1.0
    if No == 1:
        C = E + G
    else:
        lo, hi = 0.0, 1.0
        for _ in range(80):
            if _dominant_weight(hi * G + E) <= dominant:
                break
            hi *= 2.0
        for _ in range(100):
            mid = 0.5 * (lo + hi)
            if _dominant_weight(mid * G + E) > dominant:
                lo = mid
            else:
                hi = mid
        C = 0.5 * (lo + hi) * G + E
    return C / (np.sqrt(2.0) * np.linalg.norm(C))


def make_instance(No: int, Nv: int, seed: int, sigma_off: float = 1e-3, eri_sigma: float = 1e-2,
                  dominant: float = 0.9, blocks=("ovov", "ooov", "ovvv"), full_eri: bool = False) -> dict:
    """One synthetic ESMP2 instance (all arrays float64, C-contiguous)."""
    F = fock(No, Nv, seed, sigma_off)
    inst = {"No": No, "Nv": Nv, "seed": seed, "sigma_off": sigma_off, "eri_sigma": eri_sigma,
            "F": F, "C": singles_coefficients(F, No, Nv, seed, dominant)}
    for b in blocks:
        inst[b] = eri_block(b, No, Nv, seed, eri_sigma)
    if full_eri:
        inst["eri"] = eri_block("full", No, Nv, seed, eri_sigma)
    return inst


def batch_shapes(count: int = 64, seed: int = 100, no_range=(8, 32), ratio_range=(8.0, 14.0)):
    """(No, Nv, seed) for a batch of uneven instances: No ~ U{8..32}, Nv = round(r*No), r ~ U[8,14]."""
    out = []
    for k in range(count):
        s = seed + k
        u1 = _load().synth_uniform(s, 4, 0)
        u2 = _load().synth_uniform(s, 4, 1)
        No = no_range[0] + min(int(u1 * (no_range[1] - no_range[0] + 1)), no_range[1] - no_range[0])
        r = ratio_range[0] + (ratio_range[1] - ratio_range[0]) * u2
        out.append((No, int(round(r * No)), s))
    return out

"""Reference derivatives of E2 by central finite differences of the oracle (test infrastructure only).

The derivative is taken by its definition: E2 is re-solved at F +/- h and (ia|jb) +/- h with
O2 (plain CG to 1e-13) and differenced.  Conventions (the same as the library's gradient):
* a step that moves F_pq and F_qp together (once if p == q) measures dF_pq + dF_qp (dF_pp);
* a step that moves (ia|jb) and (jb|ia) together (once if they coincide) measures
  dOVOV[iajb] + dOVOV[jbia] (dOVOV[iaia]).
"""
from __future__ import annotations

import numpy as np

from . import o2, top


def e2(inst: dict, tol: float = 1e-13) -> float:
    return o2.solve(top.prepare(inst), tol=tol)["E2"]


def fd_F(inst: dict, p: int, q: int, h: float = 1e-5, tol: float = 1e-13) -> float:
    vals = []
    for sgn in (1.0, -1.0):
        d = dict(inst)
        F = inst["F"].copy()
        F[p, q] += sgn * h
        if p != q:
            F[q, p] += sgn * h
        d["F"] = F
        vals.append(e2(d, tol))
    return (vals[0] - vals[1]) / (2 * h)


def fd_ovov(inst: dict, i: int, a: int, j: int, b: int, h: float = 1e-5, tol: float = 1e-13) -> float:
    vals = []
    for sgn in (1.0, -1.0):
        d = dict(inst)
        g = inst["ovov"].copy()
        g[i, a, j, b] += sgn * h
        if (i, a) != (j, b):
            g[j, b, i, a] += sgn * h
        d["ovov"] = g
        vals.append(e2(d, tol))
    return (vals[0] - vals[1]) / (2 * h)

"""Reference derivatives of E2 from the oracle (test infrastructure only).

fd_F / fd_ovov take the derivative by its definition: E2 is re-solved at F +/- h and
(ia|jb) +/- h with O2 (plain CG to 1e-13) and differenced.  analytic_F / analytic_ovov take
it from the first-order equation at the oracle's own solution (no re-solve; affordable at
sizes where a re-solve per element is not).  Conventions (the same as the library's gradient):
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


# ---- Derivatives from the first-order equation (no re-solve).
# With A x = -b on D+L and A symmetric in the determinant inner product, E2_DL = b.x =
# -b.A^{-1}b, so along any step dE2_DL = 2 <x, db> + <x, dA x>.  b is linear in F and in the
# integrals jointly (Slater-Condon terms: f0 = F - G[gamma - gamma_Phi] and <pq||rs> s_kc),
# and A = F_N - omega(F) is linear in F, so db and dA x are b and A x evaluated with the step
# itself in place of (F, integrals).  E2_S = -sum_S b_S^2 / D_S: b_S does not involve F and
# is linear in the integrals, D_S is linear in F, so its derivative is a central difference
# (exact for the integral step, where E2_S is quadratic).  The TOP rotation depends on C
# only, so a step in the ESMF basis is rotated once.


def _with(prep: dict, **kw) -> dict:
    d = dict(prep)
    d.update(kw)
    return d


def _zeros_like_ints(prep: dict) -> dict:
    return {k: np.zeros_like(prep[k]) for k in ("ovov", "ooov", "ovvt")}


def analytic_F(inst: dict, x: np.ndarray, p: int, q: int, prep: dict | None = None, h: float = 1e-4) -> float:
    """d E2 / d h along F -> F + h (E_pq + E_qp) (E_pp once if p == q); x = the oracle's
    solution of A x = -b for `inst` (full-storage block vector)."""
    prep = prep if prep is not None else top.prepare(inst)
    N = inst["No"] + inst["Nv"]
    E = np.zeros((N, N))
    E[p, q] += 1.0
    if p != q:
        E[q, p] += 1.0
    W = top.full_rotation(prep["U"], prep["Wv"])
    dF = W.T @ E @ W
    step = o2.O2(_with(prep, F=dF, **_zeros_like_ints(prep)))
    db = step.rhs()
    dAx = step.sigma(x)
    es = [o2.O2(_with(prep, F=prep["F"] + s * h * dF)).e2_s()[0] for s in (1.0, -1.0)]
    return 2.0 * o2.wdot(x, db) + o2.wdot(x, dAx) + (es[0] - es[1]) / (2.0 * h)


def analytic_ovov(inst: dict, x: np.ndarray, i: int, a: int, j: int, b: int, prep: dict | None = None,
                  h: float = 1e-3) -> float:
    """d E2 / d h along (ia|jb) -> (ia|jb) + h together with its image (jb|ia) (once if they
    coincide); x as in analytic_F."""
    prep = prep if prep is not None else top.prepare(inst)
    No, Nv = inst["No"], inst["Nv"]
    g = np.zeros((No, Nv, No, Nv))
    g[i, a, j, b] += 1.0
    if (i, a) != (j, b):
        g[j, b, i, a] += 1.0
    dg, _, _ = top.transform_blocks(g, np.zeros((No, No, No, Nv)), np.zeros((No, Nv, Nv, Nv)),
                                    prep["U"], prep["Wv"])
    z = _zeros_like_ints(prep)
    z["ovov"] = dg
    db = o2.O2(_with(prep, F=np.zeros_like(prep["F"]), **z)).rhs()
    es = [o2.O2(_with(prep, ovov=prep["ovov"] + s * h * dg)).e2_s()[0] for s in (1.0, -1.0)]
    return 2.0 * o2.wdot(x, db) + (es[0] - es[1]) / (2.0 * h)

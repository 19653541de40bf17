"""TOP basis of the ESMF reference (oracle side; test infrastructure only).

Sec. II.A, Eqs. 2-4: the singles matrix C is factorised as C = U Lambda V^+ and
the occupied / virtual spaces are rotated by U and V so that Psi0 becomes a sum of
No transition-orbital pairs (occupied u <-> TOP virtual u, virtual index u).
Virtuals beyond the first No (the AVOs) complete V to an orthonormal basis.

Conventions (the paper leaves them open; every one is a documented reading):
* Psi0 is normalised: 2 ||C||_F^2 = 1 (each spin-adapted CSF has norm^2 2).
* Singular values in descending order; column k of V is signed so that its
  largest-magnitude component is positive, and u_k = C v_k / lambda_k.
* AVOs: columns No.. of Q = H_0 H_1 ... H_{No-1}, the Householder reflectors
  that triangularise V (H_k = I - 2 w w^T / w^T w, w = x - alpha e_0,
  alpha = -sign(x_0) ||x||, sign(0) = +1).
"""
from __future__ import annotations

import numpy as np


def normalise_singles(C: np.ndarray) -> np.ndarray:
    return C / (np.sqrt(2.0) * np.linalg.norm(C))


def householder_completion(V: np.ndarray) -> np.ndarray:
    """Q (Nv x Nv) whose first No columns span V and whose last Nv-No are the AVOs."""
    Nv, No = V.shape
    A = V.astype(np.float64).copy()
    ws = []
    for k in range(No):
        x = A[k:, k].copy()
        nx = np.linalg.norm(x)
        alpha = -(1.0 if x[0] >= 0 else -1.0) * nx
        w = x
        w[0] -= alpha
        ww = float(w @ w)
        ws.append((w, ww))
        if ww > 0.0:
            A[k:, k:] -= np.outer(w, (2.0 / ww) * (w @ A[k:, k:]))
    Q = np.eye(Nv)
    for k in reversed(range(No)):
        w, ww = ws[k]
        if ww > 0.0:
            Q[k:, :] -= np.outer(w, (2.0 / ww) * (w @ Q[k:, :]))
    return Q


def top_basis(C: np.ndarray):
    """Returns (U, lam, Wv): occupied rotation No x No, singular values (desc.),
    virtual rotation Nv x Nv whose first No columns are the TOP virtuals."""
    C = np.asarray(C, dtype=np.float64)
    No, Nv = C.shape
    if Nv < No:
        raise ValueError("the TOP construction needs Nv >= No")
    U, lam, Vt = np.linalg.svd(C, full_matrices=False)
    V = Vt.T.copy()
    U = U.copy()
    for k in range(No):
        m = int(np.argmax(np.abs(V[:, k])))
        if V[m, k] < 0:
            V[:, k] *= -1.0
            U[:, k] *= -1.0
        if lam[k] > 1e-12 * max(lam[0], 1e-300):
            U[:, k] = C @ V[:, k] / lam[k]
    Q = householder_completion(V)
    Wv = np.concatenate([V, Q[:, No:]], axis=1)
    return U, lam, Wv


def full_rotation(U: np.ndarray, Wv: np.ndarray) -> np.ndarray:
    No, Nv = U.shape[0], Wv.shape[0]
    W = np.zeros((No + Nv, No + Nv))
    W[:No, :No] = U
    W[No:, No:] = Wv
    return W


def transform_fock(F: np.ndarray, U: np.ndarray, Wv: np.ndarray) -> np.ndarray:
    W = full_rotation(U, Wv)
    return W.T @ F @ W


def transform_full_eri(eri: np.ndarray, W: np.ndarray) -> np.ndarray:
    """(pq|rs)_TOP = sum W[p'p] W[q'q] W[r'r] W[s's] (p'q'|r's')."""
    g = np.tensordot(eri, W, axes=([0], [0]))      # q r s p
    g = np.tensordot(g, W, axes=([0], [0]))        # r s p q
    g = np.tensordot(g, W, axes=([0], [0]))        # s p q r
    g = np.tensordot(g, W, axes=([0], [0]))        # p q r s
    return np.ascontiguousarray(g)


def _rot(t: np.ndarray, axis: int, R: np.ndarray) -> np.ndarray:
    """Contract index `axis` of t with the first index of R, keeping the axis order."""
    return np.moveaxis(np.tensordot(t, R, axes=([axis], [0])), -1, axis)


def transform_blocks(ovov, ooov, ovvv, U, Wv):
    """TOP-basis integral blocks.

    ovov_t[i,a,j,b] = (ia|jb); ooov_t[i,j,k,a] = (ij|ka);
    ovvt[i,a,b,u]   = (ia|b u') with u' restricted to the No TOP virtuals."""
    No = U.shape[0]
    V = Wv[:, :No]
    ovov_t = ovov
    for ax, R in ((0, U), (1, Wv), (2, U), (3, Wv)):
        ovov_t = _rot(ovov_t, ax, R)
    ooov_t = ooov
    for ax, R in ((0, U), (1, U), (2, U), (3, Wv)):
        ooov_t = _rot(ooov_t, ax, R)
    ovvt = np.tensordot(ovvv, V, axes=([3], [0]))   # i a b u
    for ax, R in ((0, U), (1, Wv), (2, Wv)):
        ovvt = _rot(ovvt, ax, R)
    return (np.ascontiguousarray(ovov_t), np.ascontiguousarray(ooov_t), np.ascontiguousarray(ovvt))


def prepare(inst: dict) -> dict:
    """Everything the oracle needs in the TOP basis, from a synth instance."""
    No, Nv = inst["No"], inst["Nv"]
    C = normalise_singles(inst["C"])
    U, lam, Wv = top_basis(C)
    Ft = transform_fock(inst["F"], U, Wv)
    ovov_t, ooov_t, ovvt = transform_blocks(inst["ovov"], inst["ooov"], inst["ovvv"], U, Wv)
    return {"No": No, "Nv": Nv, "C": C, "U": U, "lam": lam, "Wv": Wv, "F": Ft,
            "ovov": ovov_t, "ooov": ooov_t, "ovvt": ovvt}

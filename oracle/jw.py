"""O1 -- ESMP2-TOP(eta) written out in the determinant space (test infrastructure only).

Everything here follows the definitions in the paper literally, for systems
small enough that the whole Ms = 0, 2No-electron determinant space fits in memory:

* fermion operators a_k, a_k^+ in the Jordan-Wigner representation on bit
  strings (sign = (-1)^(number of occupied modes below k)); spin orbital of
  spatial orbital p and spin s is k = p + s*N;
* H = sum h_pq E_pq + 1/2 sum (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s}, with
  h = F - G[gamma] where gamma is the spin-summed one-body density of Psi0 and
  G[g]_pq = sum_rs g_rs [(pq|rs) - 1/2 (ps|rq)]  ("F is the Fock operator built
  from the one-body density matrix of Psi0", Sec. II.C);
* Psi0 = sum_u lambda_u (a+_{u' up} a_{u up} + a+_{u' dn} a_{u dn}) |Phi>, singlet
  sign, in the TOP basis (Eq. psi0_tp), u' = orbital No+u;
* first-order space: doubles (D) and triples split into L / S / N by their
  transition-orbital-pair content (Eq. triples_element, Sec. II.C); a pair is a
  hole u and particle u' of the same spin;
* H0 on the first-order space: (Q_D+Q_L) F (Q_D+Q_L) + (Q_S+Q_N) F_diag (Q_S+Q_N)
  (Eq. qfq_replacement), E0 = <Psi0|F|Psi0> (the P-space part of Eq. old_H0 leaves
  Psi0's zeroth-order energy equal to its Fock expectation value);
* first-order equation (H0 - E0) Psi1 = -Q H Psi0 solved densely on D+L and
  diagonally on S+N; E2 = <Psi0|H|Psi1>.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import top


def _parity_below(det: int, k: int) -> int:
    return bin(det & ((1 << k) - 1)).count("1") & 1


def ann(det: int, k: int):
    if not (det >> k) & 1:
        return 0, 0
    return (-1 if _parity_below(det, k) else 1), det ^ (1 << k)


def cre(det: int, k: int):
    if (det >> k) & 1:
        return 0, 0
    return (-1 if _parity_below(det, k) else 1), det | (1 << k)


class System:
    """Orbital bookkeeping for No doubly occupied and Nv virtual spatial orbitals."""

    def __init__(self, No: int, Nv: int):
        self.No, self.Nv, self.N = No, Nv, No + Nv

    def so(self, p: int, s: int) -> int:
        return p + s * self.N

    @property
    def phi(self) -> int:
        d = 0
        for i in range(self.No):
            d |= 1 << self.so(i, 0)
            d |= 1 << self.so(i, 1)
        return d

    def determinants(self):
        """All Ms=0 determinants with No electrons of each spin."""
        out = []
        for a in itertools.combinations(range(self.N), self.No):
            ma = sum(1 << p for p in a)
            for b in itertools.combinations(range(self.N), self.No):
                out.append(ma | (sum(1 << p for p in b) << self.N))
        return out

    def excitation(self, det: int):
        """(holes, particles) relative to Phi as lists of (spatial, spin)."""
        holes = [(i, s) for s in (0, 1) for i in range(self.No) if not (det >> self.so(i, s)) & 1]
        parts = [(a, s) for s in (0, 1) for a in range(self.No, self.N) if (det >> self.so(a, s)) & 1]
        return holes, parts

    def pairs(self, det: int):
        """Transition-orbital pairs present: u with hole u_s and particle (No+u)_s, same spin."""
        holes, parts = self.excitation(det)
        ps = set(parts)
        return {(u, s) for (u, s) in holes if (self.No + u, s) in ps}

    def excite(self, holes, particles):
        """a+_{p1} .. a+_{pn} a_{hn} .. a_{h1} |Phi>  ->  (sign, det); (0, 0) if it vanishes.
        holes / particles are (spatial, spin) with spatial indices of the full orbital list."""
        sign, det = 1, self.phi
        for (i, s) in holes:
            sg, det = ann(det, self.so(i, s))
            if sg == 0:
                return 0, 0
            sign *= sg
        for (a, s) in reversed(particles):
            sg, det = cre(det, self.so(a, s))
            if sg == 0:
                return 0, 0
            sign *= sg
        return sign, det


def apply_one_body(sys: System, state: dict, M: np.ndarray) -> dict:
    """sum_pq M_pq sum_s a+_{p s} a_{q s} applied to a state {det: coef}."""
    out: dict = {}
    N = sys.N
    for det, c in state.items():
        for s in (0, 1):
            for q in range(N):
                sq, d1 = ann(det, sys.so(q, s))
                if sq == 0:
                    continue
                for p in range(N):
                    if M[p, q] == 0.0:
                        continue
                    sp, d2 = cre(d1, sys.so(p, s))
                    if sp == 0:
                        continue
                    out[d2] = out.get(d2, 0.0) + c * sq * sp * M[p, q]
    return out


def apply_hamiltonian(sys: System, state: dict, h: np.ndarray, eri: np.ndarray) -> dict:
    """H |state> with H = sum h_pq E_pq + 1/2 sum (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s}."""
    out = apply_one_body(sys, state, h)
    N = sys.N
    for det, c in state.items():
        for sq_ in (0, 1):
            for q in range(N):
                g1, d1 = ann(det, sys.so(q, sq_))
                if g1 == 0:
                    continue
                for ss in (0, 1):
                    for s in range(N):
                        g2, d2 = ann(d1, sys.so(s, ss))
                        if g2 == 0:
                            continue
                        for r in range(N):
                            g3, d3 = cre(d2, sys.so(r, ss))
                            if g3 == 0:
                                continue
                            for p in range(N):
                                v = eri[p, q, r, s]
                                if v == 0.0:
                                    continue
                                g4, d4 = cre(d3, sys.so(p, sq_))
                                if g4 == 0:
                                    continue
                                out[d4] = out.get(d4, 0.0) + 0.5 * v * c * g1 * g2 * g3 * g4
    return out


def density(sys: System, state: dict) -> np.ndarray:
    """Spin-summed one-body density gamma_pq = sum_s <state| a+_{p s} a_{q s} |state>."""
    N = sys.N
    g = np.zeros((N, N))
    for p in range(N):
        for q in range(N):
            M = np.zeros((N, N))
            M[p, q] = 1.0
            v = apply_one_body(sys, state, M)
            g[p, q] = sum(c * state.get(d, 0.0) for d, c in v.items())
    return g


def two_electron_fock(gamma: np.ndarray, eri: np.ndarray) -> np.ndarray:
    """G[gamma]_pq = sum_rs gamma_rs [(pq|rs) - 1/2 (ps|rq)]."""
    J = np.einsum("rs,pqrs->pq", gamma, eri)
    K = np.einsum("rs,psrq->pq", gamma, eri)
    return J - 0.5 * K


def psi0_top(sys: System, lam: np.ndarray) -> dict:
    st: dict = {}
    for u in range(sys.No):
        for s in (0, 1):
            sg, d = sys.excite([(u, s)], [(sys.No + u, s)])
            st[d] = st.get(d, 0.0) + sg * lam[u]
    return st


def psi0_from_singles(sys: System, C: np.ndarray) -> dict:
    """sum_ia C_ia (a+_{a up} a_{i up} + a+_{a dn} a_{i dn}) |Phi>  (Eq. psi0, X = 0)."""
    st: dict = {}
    for i in range(sys.No):
        for a in range(sys.Nv):
            for s in (0, 1):
                sg, d = sys.excite([(i, s)], [(sys.No + a, s)])
                st[d] = st.get(d, 0.0) + sg * C[i, a]
    return st


def dot(x: dict, y: dict) -> float:
    return float(sum(c * y.get(d, 0.0) for d, c in x.items()))


class Result:
    pass


def classify(sys: System, det: int, large: set):
    holes, _ = sys.excitation(det)
    lvl = len(holes)
    if lvl == 2:
        return "D"
    if lvl != 3:
        return "X"   # outside the first-order interacting space (P space, quadruples, ...)
    pr = sys.pairs(det)
    if not pr:
        return "N"
    if any(u in large for (u, _) in pr):
        return "L"
    return "S"


def solve(F: np.ndarray, eri: np.ndarray, C: np.ndarray, No: int, Nv: int,
          eta: float | None = None, n_large: int = 1, basis=None, h0: str = "modified",
          shift: float = 0.0) -> Result:
    """ESMP2 in the determinant space.  Inputs in the ESMF orbital basis: F (N x N),
    eri (N^4 chemist), C (No x Nv).  Large TOPs: lambda_u > eta if eta is given,
    else the n_large largest.  `basis` optionally overrides (U, lam, Wv).

    h0 = "modified": Eq. qfq_replacement, the full Fock operator on D + L and its diagonal on
    S + N (the N^5 method).  h0 = "original": Eq. old_H0, the full Fock operator on every
    first-order determinant (D and all triples; the N^7 parent method, here for tiny spaces).
    shift: a level shift added to H0 on the first-order space (A -> A + shift, every
    denominator + shift), the remedy for intruder states the paper cites (CASPT2)."""
    sys = System(No, Nv)
    Cn = top.normalise_singles(C)
    U, lam, Wv = basis if basis is not None else top.top_basis(Cn)
    W = top.full_rotation(U, Wv)
    Ft = W.T @ F @ W
    eri_t = top.transform_full_eri(eri, W)
    large = {u for u in range(No) if lam[u] > eta} if eta is not None else set(range(min(n_large, No)))

    psi0 = psi0_top(sys, lam)
    gamma = density(sys, psi0)
    h = Ft - two_electron_fock(gamma, eri_t)

    dets = sys.determinants()
    cls = {d: classify(sys, d, large) for d in dets}
    full = ("D", "L", "S", "N") if h0 == "original" else ("D", "L")
    if h0 not in ("modified", "original"):
        raise ValueError(h0)
    DL = [d for d in dets if cls[d] in full]
    SN = [d for d in dets if cls[d] in ("S", "N") and cls[d] not in full]
    idx = {d: k for k, d in enumerate(DL)}

    Hpsi = apply_hamiltonian(sys, psi0, h, eri_t)
    b = {d: v for d, v in Hpsi.items() if cls.get(d, "X") in ("D", "L", "S", "N")}
    E0 = dot(psi0, apply_one_body(sys, psi0, Ft))

    n = len(DL)
    A = np.zeros((n, n))
    for j, dj in enumerate(DL):
        col = apply_one_body(sys, {dj: 1.0}, Ft)
        for d, v in col.items():
            i = idx.get(d)
            if i is not None:
                A[i, j] += v
    A -= (E0 - shift) * np.eye(n)
    fdiag = np.diag(Ft)

    def diag_energy(det):
        e = 0.0
        for s in (0, 1):
            for p in range(sys.N):
                if (det >> sys.so(p, s)) & 1:
                    e += fdiag[p]
        return e - E0 + shift

    bDL = np.array([b.get(d, 0.0) for d in DL])
    xDL = np.linalg.solve(A, -bDL) if n else np.zeros(0)
    x = {d: xDL[k] for k, d in enumerate(DL)}
    parts = {"D": 0.0, "L": 0.0, "S": 0.0, "N": 0.0}
    for k, d in enumerate(DL):
        parts[cls[d]] += bDL[k] * xDL[k]
    for d in SN:
        bd = b.get(d, 0.0)
        if bd != 0.0:
            xd = -bd / diag_energy(d)
            x[d] = xd
            parts[cls[d]] += bd * xd

    r = Result()
    r.sys, r.U, r.lam, r.Wv, r.W = sys, U, lam, Wv, W
    r.F_top, r.eri_top, r.h, r.gamma = Ft, eri_t, h, gamma
    r.psi0, r.E0, r.b, r.x, r.cls = psi0, E0, b, x, cls
    r.DL, r.SN, r.idx, r.A = DL, SN, idx, A
    r.large = large
    r.parts = parts
    r.E2 = sum(parts.values())
    r.diag_energy = diag_energy
    return r


# --------------------------------------------------------------------------------------
# Block layout of the iterative vector (shared convention with the other
# implementations; it is the convention of Eq. psi1 with the L-triples split by
# which spin carries the large TOP t = 0).
#   T[i,j,a,b] = coef of a+_{a up} a+_{b up} a_{j up} a_{i up} |Phi>        (and down-down)
#   S[i,j,a,b] = coef of a+_{a up} a+_{b dn} a_{j dn} a_{i up} |Phi>
#   X[j,k,b,c] = coef of a+_{t' up} a+_{b up} a+_{c up} a_{k up} a_{j up} a_{t up} |Phi>  (and all down)
#   Y[j,k,b,c] = coef of a+_{t' up} a+_{b dn} a+_{c dn} a_{k dn} a_{j dn} a_{t up} |Phi> (and spin flip)
#   Z[i,k,a,c] = coef of a+_{a up} a+_{t' dn} a+_{c dn} a_{k dn} a_{t dn} a_{i up} |Phi> (and spin flip)
# i, j, k occupied indices; a, b, c virtual indices (orbital No + a); t = t' = 0.
# --------------------------------------------------------------------------------------
BLOCKS = ("T", "S", "X", "Y", "Z")


def block_strings(No: int, blk: str, i: int, j: int, a: int, b: int, flip: bool = False):
    """Operator string (holes, particles) of one full-storage block element.
    Spatial indices of the full orbital list; flip=True swaps up/down."""
    t, tp = 0, No + 0
    A, B = No + a, No + b
    u, d = (1, 0) if flip else (0, 1)
    if blk == "T":
        return [(i, u), (j, u)], [(A, u), (B, u)]
    if blk == "S":
        return [(i, u), (j, d)], [(A, u), (B, d)]
    if blk == "X":
        return [(t, u), (i, u), (j, u)], [(tp, u), (A, u), (B, u)]
    if blk == "Y":
        return [(t, u), (i, d), (j, d)], [(tp, u), (A, d), (B, d)]
    if blk == "Z":
        return [(i, u), (t, d), (j, d)], [(A, u), (tp, d), (B, d)]
    raise ValueError(blk)


def block_mask(No: int, Nv: int, blk: str) -> np.ndarray:
    """True where a full-storage element is a valid first-order amplitude."""
    m = np.ones((No, No, Nv, Nv), dtype=bool)
    ii = np.arange(No)[:, None, None, None]
    jj = np.arange(No)[None, :, None, None]
    aa = np.arange(Nv)[None, None, :, None]
    bb = np.arange(Nv)[None, None, None, :]
    if blk in ("T", "X", "Y"):
        m &= (ii != jj) & (aa != bb)
    if blk == "X":
        m &= (ii != 0) & (jj != 0) & (aa != 0) & (bb != 0)
    if blk == "Z":
        m &= (jj != 0) & (bb != 0) & ~((ii == 0) & (aa == 0))
    return m


def blocks_to_state(sys: System, blocks: dict) -> dict:
    """Spin-symmetric determinant vector from full-storage blocks (the amplitude of each
    operator string is shared with its spin-flipped string, Eq. psi1)."""
    st: dict = {}
    No, Nv = sys.No, sys.Nv
    for blk in BLOCKS:
        arr = blocks[blk]
        m = block_mask(No, Nv, blk)
        for (i, j, a, b) in zip(*np.nonzero(m)):
            if blk in ("T", "X", "Y") and not (i < j and a < b):
                continue
            for flip in (False, True):
                sg, d = sys.excite(*block_strings(No, blk, i, j, a, b, flip))
                if sg:
                    st[d] = sg * arr[i, j, a, b]
    return st


def state_to_blocks(sys: System, st: dict) -> dict:
    No, Nv = sys.No, sys.Nv
    out = {}
    for blk in BLOCKS:
        arr = np.zeros((No, No, Nv, Nv))
        m = block_mask(No, Nv, blk)
        for (i, j, a, b) in zip(*np.nonzero(m)):
            sg, d = sys.excite(*block_strings(No, blk, i, j, a, b))
            if sg:
                arr[i, j, a, b] = sg * st.get(d, 0.0)
        out[blk] = arr
    return out


def apply_A(res: Result, st: dict) -> dict:
    """(H0 - E0) restricted to D+L, applied to a determinant vector on D+L."""
    v = np.array([st.get(d, 0.0) for d in res.DL])
    w = res.A @ v
    return {d: w[k] for k, d in enumerate(res.DL)}

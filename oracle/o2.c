/* O2 -- ESMP2-TOP(1) for large systems, amplitude by amplitude (TEST INFRASTRUCTURE ONLY).
 *
 * Nothing here is blocked, fused or reordered for speed beyond skipping amplitudes
 * that are zero by definition.  Every quantity is a textbook spin-orbital formula
 * evaluated through amp(), which returns the coefficient of any spin-orbital
 * double or triple excitation a+_{p1}..a+_{pn} a_{hn}..a_{h1}|Phi> from the stored
 * blocks:
 *   - up-up and down-down doubles share T, triples share their spin-flipped
 *     partner's amplitude (Eq. psi1);
 *   - triples are nonzero only in the L space: they must contain the large
 *     transition-orbital pair t -> t' in one spin (Sec. II.C, TOP(1): t = 0);
 *     S- and N-triples are not part of the iterative vector (Sec. II.D).
 *
 * Storage: five full blocks [No][No][Nv][Nv] (T, S, X, Y, Z; see oracle/jw.py for
 * the operator string of each element).  Occupied index i = orbital i, virtual
 * index a = orbital No + a, TOP virtual partner of occupied u has virtual index u.
 *
 * Operator (Eq. qfq_replacement restricted to D+L, minus E0):
 *   A = (E_Phi[F] - E0) + F_N, with F_N the normal-ordered spin-free Fock operator:
 *   doubles <- doubles : sum_c (f_ac x_ij^cb + f_bc x_ij^ac) - sum_k (f_ki x_kj^ab + f_kj x_ik^ab)
 *   doubles <- triples : sum_kc f_kc x_ijk^abc
 *   triples <- triples : the same one-body terms on all three particle / hole slots
 *   triples <- doubles : P(k/ij) P(c/ab) f_ck x_ij^ab
 *   (an optional level shift s adds s to A and to every S-space denominator)
 *   E_Phi[F] - E0 = -omega,  omega = sum_u 2 lam_u^2 (F_u'u' - F_uu)  (gamma of Psi0
 *   is diagonal in the TOP basis: 2 - 2 lam_u^2 on u, 2 lam_u^2 on u').
 * Right-hand side b = Q H Psi0 (Slater-Condon, Psi0 = sum_u lam_u singles u -> u'):
 *   doubles : P(ij)P(ab)[s_ia f0_bj] + P(ij) sum_c <ab||cj> s_ic - P(ab) sum_k <kb||ij> s_ka
 *   triples : P(k/ij) P(c/ab) [<ab||ij> s_kc]
 *   s_ia = lam_i if a is the TOP partner of i (same spin), f0 = Fock matrix of the
 *   closed-shell determinant Phi = F - G[gamma - gamma_Phi].
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int v; int o; int s; } orb; /* v: 0 occupied / 1 virtual; o: index in its space; s: spin */

typedef struct {
  int No, Nv;
  const double *F;     /* N x N, TOP basis */
  const double *lam;   /* No singular values */
  const double *ovov;  /* (ia|jb)  [No][Nv][No][Nv] */
  const double *ooov;  /* (ij|ka)  [No][No][No][Nv] */
  const double *ovvt;  /* (ia|bu') [No][Nv][Nv][No] */
  double omega;
  double shift;        /* level shift of H0 on the first-order space (0: the paper's H0) */
  double *f0vo;        /* [Nv][No] */
  int err;
} o2_ctx;

enum { BT = 0, BS = 1, BX = 2, BY = 3, BZ = 4 };

static inline double Foo(const o2_ctx *c, int k, int l) { return c->F[(size_t)k * (c->No + c->Nv) + l]; }
static inline double Fvv(const o2_ctx *c, int a, int b) { return c->F[(size_t)(c->No + a) * (c->No + c->Nv) + c->No + b]; }
static inline double Fov(const o2_ctx *c, int k, int a) { return c->F[(size_t)k * (c->No + c->Nv) + c->No + a]; }

static inline size_t bidx(const o2_ctx *c, int blk, int i, int j, int a, int b) {
  const size_t No = c->No, Nv = c->Nv;
  return (size_t)blk * No * No * Nv * Nv + (((size_t)i * No + j) * Nv + a) * Nv + b;
}

/* ------------------------------------------------------------------ integrals */
static double eri(o2_ctx *c, orb p, orb q, orb r, orb s) {
  const size_t No = c->No, Nv = c->Nv;
  const int nv = p.v + q.v + r.v + s.v;
  if (nv == 2) {
    if (p.v == q.v) { c->err = 1; return 0.0; } /* (oo|vv) is never needed */
    orb i = p.v ? q : p, a = p.v ? p : q, j = r.v ? s : r, b = r.v ? r : s;
    return c->ovov[((i.o * Nv + a.o) * No + j.o) * Nv + b.o];
  }
  if (nv == 1) {
    orb x, y, k, a;
    if (p.v || q.v) { k = p.v ? q : p; a = p.v ? p : q; x = r; y = s; }
    else { k = r.v ? s : r; a = r.v ? r : s; x = p; y = q; }
    return c->ooov[((x.o * No + y.o) * No + k.o) * Nv + a.o];
  }
  if (nv == 3) {
    orb i, a, b, cc;
    if (p.v && q.v) { b = p; cc = q; i = r.v ? s : r; a = r.v ? r : s; }
    else { i = p.v ? q : p; a = p.v ? p : q; b = r; cc = s; }
    if ((size_t)cc.o < No) return c->ovvt[((i.o * Nv + a.o) * Nv + b.o) * No + cc.o];
    if ((size_t)b.o < No) return c->ovvt[((i.o * Nv + a.o) * Nv + cc.o) * No + b.o];
    c->err = 2;
    return 0.0;
  }
  c->err = 3;
  return 0.0;
}

/* <pq||rs> over spin orbitals, <pq|rs> = delta(s_p,s_r) delta(s_q,s_s) (pr|qs) */
static double asym(o2_ctx *c, orb p, orb q, orb r, orb s) {
  double v = 0.0;
  if (p.s == r.s && q.s == s.s) v += eri(c, p, r, q, s);
  if (p.s == s.s && q.s == r.s) v -= eri(c, p, s, q, r);
  return v;
}

/* singles coefficient of Psi0 in the TOP basis */
static inline double s1(const o2_ctx *c, orb h, orb p) {
  return (h.s == p.s && h.o == p.o) ? c->lam[h.o] : 0.0;
}

/* ------------------------------------------------------------------ amplitudes */
static inline int okey(orb x) { return x.s * 100000 + x.o; }

static int sort_orbs(orb *x, int n) { /* insertion sort by (spin, index); returns parity sign */
  int sign = 1;
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && okey(x[j - 1]) > okey(x[j]); --j) {
      orb t = x[j]; x[j] = x[j - 1]; x[j - 1] = t; sign = -sign;
    }
  return sign;
}

static double amp(const o2_ctx *c, const double *x, int n, const orb *Hin, const orb *Pin) {
  orb H[3], P[3];
  int nah = 0, nap = 0;
  for (int k = 0; k < n; ++k) { H[k] = Hin[k]; P[k] = Pin[k]; nah += H[k].s == 0; nap += P[k].s == 0; }
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b) {
      if (H[a].o == H[b].o && H[a].s == H[b].s) return 0.0;
      if (P[a].o == P[b].o && P[a].s == P[b].s) return 0.0;
    }
  if (nah != nap) return 0.0;
  if ((n == 2 && nah == 0) || (n == 3 && (nah == 0 || nah == 2)))
    for (int k = 0; k < n; ++k) { H[k].s ^= 1; P[k].s ^= 1; }
  int sign = sort_orbs(H, n) * sort_orbs(P, n);
  if (n == 2) {
    const int blk = (H[1].s == 0) ? BT : BS;
    return sign * x[bidx(c, blk, H[0].o, H[1].o, P[0].o, P[1].o)];
  }
  if (H[1].s == 0) { /* all up: L only if it holds t (occ 0) and t' (virt 0) */
    int m = -1, q = -1;
    for (int k = 0; k < 3; ++k) { if (H[k].o == 0) m = k; if (P[k].o == 0) q = k; }
    if (m < 0 || q < 0) return 0.0;
    if (m & 1) sign = -sign;
    if (q & 1) sign = -sign;
    int hr[2], pr[2], nh = 0, np = 0;
    for (int k = 0; k < 3; ++k) { if (k != m) hr[nh++] = H[k].o; if (k != q) pr[np++] = P[k].o; }
    return sign * x[bidx(c, BX, hr[0], hr[1], pr[0], pr[1])];
  }
  /* up, down, down */
  if (H[0].o == 0 && P[0].o == 0) return sign * x[bidx(c, BY, H[1].o, H[2].o, P[1].o, P[2].o)];
  int m = -1, q = -1;
  for (int k = 1; k < 3; ++k) { if (H[k].o == 0) m = k; if (P[k].o == 0) q = k; }
  if (m < 0 || q < 0) return 0.0;
  if (m == 2) sign = -sign;
  if (q == 2) sign = -sign;
  return sign * x[bidx(c, BZ, H[0].o, H[3 - m].o, P[0].o, P[3 - q].o)];
}

/* operator string (holes, particles) of a stored element, up-first convention */
static int block_string(const o2_ctx *c, int blk, int i, int j, int a, int b, orb *H, orb *P) {
  (void)c;
  switch (blk) {
    case BT: H[0] = (orb){0, i, 0}; H[1] = (orb){0, j, 0}; P[0] = (orb){1, a, 0}; P[1] = (orb){1, b, 0}; return 2;
    case BS: H[0] = (orb){0, i, 0}; H[1] = (orb){0, j, 1}; P[0] = (orb){1, a, 0}; P[1] = (orb){1, b, 1}; return 2;
    case BX: H[0] = (orb){0, 0, 0}; H[1] = (orb){0, i, 0}; H[2] = (orb){0, j, 0};
             P[0] = (orb){1, 0, 0}; P[1] = (orb){1, a, 0}; P[2] = (orb){1, b, 0}; return 3;
    case BY: H[0] = (orb){0, 0, 0}; H[1] = (orb){0, i, 1}; H[2] = (orb){0, j, 1};
             P[0] = (orb){1, 0, 0}; P[1] = (orb){1, a, 1}; P[2] = (orb){1, b, 1}; return 3;
    default: H[0] = (orb){0, i, 0}; H[1] = (orb){0, 0, 1}; H[2] = (orb){0, j, 1};
             P[0] = (orb){1, a, 0}; P[1] = (orb){1, 0, 1}; P[2] = (orb){1, b, 1}; return 3;
  }
}

int o2_valid(int No, int blk, int i, int j, int a, int b) {
  (void)No;
  if ((blk == BT || blk == BX || blk == BY) && (i == j || a == b)) return 0;
  if (blk == BX && (i == 0 || j == 0 || a == 0 || b == 0)) return 0;
  if (blk == BZ && (j == 0 || b == 0 || (i == 0 && a == 0))) return 0;
  return 1;
}

/* hole / particle permutations for P(k/ij): identity, swap slots 1<->3, swap 2<->3 */
static const int PERM[3][3] = {{0, 1, 2}, {2, 1, 0}, {0, 2, 1}};
static const int PSGN[3] = {1, -1, -1};

/* ------------------------------------------------------------------ sigma */
static double sigma_string(const o2_ctx *c, const double *x, int n, const orb *H, const orb *P) {
  const int No = c->No, Nv = c->Nv;
  double val = (c->shift - c->omega) * amp(c, x, n, H, P);   /* E_Phi[F] - E0 + shift */
  orb H2[3], P2[3];
  for (int m = 0; m < n; ++m) {                       /* particle slots: + sum_d f_{p d} */
    memcpy(H2, H, sizeof(orb) * n); memcpy(P2, P, sizeof(orb) * n);
    for (int d = 0; d < Nv; ++d) { P2[m].o = d; val += Fvv(c, P[m].o, d) * amp(c, x, n, H2, P2); }
  }
  for (int m = 0; m < n; ++m) {                       /* hole slots: - sum_l f_{l h} */
    memcpy(H2, H, sizeof(orb) * n); memcpy(P2, P, sizeof(orb) * n);
    for (int l = 0; l < No; ++l) { H2[m].o = l; val -= Foo(c, l, H[m].o) * amp(c, x, n, H2, P2); }
  }
  if (n == 2) {                                       /* + sum_kc f_kc x_ijk^abc (L triples only) */
    int haspair = 0;
    for (int s = 0; s < 2; ++s) {
      int ht = 0, pt = 0;
      for (int k = 0; k < 2; ++k) { ht |= (H[k].o == 0 && H[k].s == s); pt |= (P[k].o == 0 && P[k].s == s); }
      haspair |= ht && pt;
    }
    orb H3[3] = {H[0], H[1], {0, 0, 0}}, P3[3] = {P[0], P[1], {1, 0, 0}};
    for (int s = 0; s < 2; ++s) {
      H3[2].s = s; P3[2].s = s;
      if (haspair) {
        for (int k = 0; k < No; ++k)
          for (int cc = 0; cc < Nv; ++cc) { H3[2].o = k; P3[2].o = cc; val += Fov(c, k, cc) * amp(c, x, 3, H3, P3); }
      } else {
        H3[2].o = 0;
        for (int cc = 0; cc < Nv; ++cc) { P3[2].o = cc; val += Fov(c, 0, cc) * amp(c, x, 3, H3, P3); }
        P3[2].o = 0;
        for (int k = 1; k < No; ++k) { H3[2].o = k; val += Fov(c, k, 0) * amp(c, x, 3, H3, P3); }
      }
    }
  } else {                                            /* + P(k/ij) P(c/ab) f_ck x_ij^ab */
    for (int t = 0; t < 3; ++t)
      for (int r = 0; r < 3; ++r) {
        const orb h3 = H[PERM[t][2]], p3 = P[PERM[r][2]];
        if (h3.s != p3.s) continue;
        const orb Hd[2] = {H[PERM[t][0]], H[PERM[t][1]]}, Pd[2] = {P[PERM[r][0]], P[PERM[r][1]]};
        val += PSGN[t] * PSGN[r] * Fov(c, h3.o, p3.o) * amp(c, x, 2, Hd, Pd);
      }
  }
  return val;
}

double o2_sigma_elem(o2_ctx *c, const double *x, int blk, int i, int j, int a, int b) {
  if (!o2_valid(c->No, blk, i, j, a, b)) return 0.0;
  orb H[3], P[3];
  const int n = block_string(c, blk, i, j, a, b, H, P);
  return sigma_string(c, x, n, H, P);
}

void o2_sigma_full(o2_ctx *c, const double *x, double *y) {
  const int No = c->No, Nv = c->Nv;
#pragma omp parallel for collapse(3) schedule(dynamic, 1)
  for (int blk = 0; blk < 5; ++blk)
    for (int i = 0; i < No; ++i)
      for (int j = 0; j < No; ++j)
        for (int a = 0; a < Nv; ++a)
          for (int b = 0; b < Nv; ++b)
            y[bidx(c, blk, i, j, a, b)] = o2_sigma_elem(c, x, blk, i, j, a, b);
}

/* flat full-storage indices -> values */
void o2_sigma_at(o2_ctx *c, const double *x, int64_t count, const int64_t *flat, double *out) {
  const int64_t No = c->No, Nv = c->Nv, B = No * No * Nv * Nv;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t n = 0; n < count; ++n) {
    int64_t f = flat[n];
    const int blk = (int)(f / B); f %= B;
    const int b = (int)(f % Nv); f /= Nv;
    const int a = (int)(f % Nv); f /= Nv;
    const int j = (int)(f % No); const int i = (int)(f / No);
    out[n] = o2_sigma_elem(c, x, blk, i, j, a, b);
  }
}

/* ------------------------------------------------------------------ right-hand side */
static inline double f0(const o2_ctx *c, orb p, orb h) { /* p virtual, h occupied */
  return p.s == h.s ? c->f0vo[(size_t)p.o * c->No + h.o] : 0.0;
}

static double rhs_string(o2_ctx *c, int n, const orb *H, const orb *P) {
  const int No = c->No, Nv = c->Nv;
  double val = 0.0;
  if (n == 2) {
    static const int PR[2][2] = {{0, 1}, {1, 0}};
    static const int PS[2] = {1, -1};
    for (int u = 0; u < 2; ++u)
      for (int w = 0; w < 2; ++w) /* P(ij)P(ab) s_ia f0_bj */
        val += PS[u] * PS[w] * s1(c, H[PR[u][0]], P[PR[w][0]]) * f0(c, P[PR[w][1]], H[PR[u][1]]);
    for (int u = 0; u < 2; ++u) { /* P(ij) sum_c <ab||cj> s_ic : c = TOP partner of i */
      const orb hi = H[PR[u][0]], hj = H[PR[u][1]];
      if (hi.o < Nv) {
        const orb cv = {1, hi.o, hi.s};
        val += PS[u] * c->lam[hi.o] * asym(c, P[0], P[1], cv, hj);
      }
    }
    for (int w = 0; w < 2; ++w) { /* -P(ab) sum_k <kb||ij> s_ka : k = TOP partner of a */
      const orb pa = P[PR[w][0]], pb = P[PR[w][1]];
      if (pa.o < No) {
        const orb k = {0, pa.o, pa.s};
        val -= PS[w] * c->lam[pa.o] * asym(c, k, pb, H[0], H[1]);
      }
    }
  } else {
    for (int t = 0; t < 3; ++t)
      for (int r = 0; r < 3; ++r) {
        const double s = s1(c, H[PERM[t][2]], P[PERM[r][2]]);
        if (s == 0.0) continue;
        val += PSGN[t] * PSGN[r] * s * asym(c, P[PERM[r][0]], P[PERM[r][1]], H[PERM[t][0]], H[PERM[t][1]]);
      }
  }
  return val;
}

double o2_rhs_elem(o2_ctx *c, int blk, int i, int j, int a, int b) {
  if (!o2_valid(c->No, blk, i, j, a, b)) return 0.0;
  orb H[3], P[3];
  const int n = block_string(c, blk, i, j, a, b, H, P);
  return rhs_string(c, n, H, P);
}

void o2_rhs_full(o2_ctx *c, double *out) {
  const int No = c->No, Nv = c->Nv;
#pragma omp parallel for collapse(3) schedule(dynamic, 1)
  for (int blk = 0; blk < 5; ++blk)
    for (int i = 0; i < No; ++i)
      for (int j = 0; j < No; ++j)
        for (int a = 0; a < Nv; ++a)
          for (int b = 0; b < Nv; ++b)
            out[bidx(c, blk, i, j, a, b)] = o2_rhs_elem(c, blk, i, j, a, b);
}

void o2_rhs_at(o2_ctx *c, int64_t count, const int64_t *flat, double *out) {
  const int64_t No = c->No, Nv = c->Nv, B = No * No * Nv * Nv;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t n = 0; n < count; ++n) {
    int64_t f = flat[n];
    const int blk = (int)(f / B); f %= B;
    const int b = (int)(f % Nv); f /= Nv;
    const int a = (int)(f % Nv); f /= Nv;
    const int j = (int)(f % No); const int i = (int)(f / No);
    out[n] = o2_rhs_elem(c, blk, i, j, a, b);
  }
}

/* ------------------------------------------------------------------ S-space energy */
/* E2_S = -sum_{I in S} b_I^2 / (<I|F_diag|I> - E0), Sec. II.C-D: S-triples hold at least
 * one transition-orbital pair u -> u' (same spin) and none of them is the large t = 0.
 * Each triple is visited once, from its lowest pair; the spin-flipped sector doubles it. */
static double diag3(const o2_ctx *c, const orb *H, const orb *P) {
  double e = c->shift - c->omega;
  for (int k = 0; k < 3; ++k) e += Fvv(c, P[k].o, P[k].o) - Foo(c, H[k].o, H[k].o);
  return e;
}

static int pairs_mask(const orb *H, const orb *P, int s, int *has_t) {
  /* returns lowest pair index of spin s or large value; has_t |= pair 0 present */
  int lo = 1 << 30;
  for (int a = 0; a < 3; ++a)
    if (H[a].s == s)
      for (int b = 0; b < 3; ++b)
        if (P[b].s == s && P[b].o == H[a].o) { if (H[a].o < lo) lo = H[a].o; if (H[a].o == 0) *has_t = 1; }
  return lo;
}

double o2_e2_s(o2_ctx *c, int64_t *count_out) {
  const int No = c->No, Nv = c->Nv;
  double total = 0.0;
  int64_t count = 0;
  /* up-up-up: holes u<j<k ... enumerate the pair u explicitly */
#pragma omp parallel for reduction(+ : total, count) schedule(dynamic, 1)
  for (int u = 1; u < No; ++u) {
    for (int j = 0; j < No; ++j)
      for (int k = j + 1; k < No; ++k) {
        if (j == u || k == u) continue;
        for (int b = 0; b < Nv; ++b)
          for (int cc = b + 1; cc < Nv; ++cc) {
            if (b == u || cc == u) continue;
            orb H[3] = {{0, u, 0}, {0, j, 0}, {0, k, 0}}, P[3] = {{1, u, 0}, {1, b, 0}, {1, cc, 0}};
            int has_t = 0;
            const int lo = pairs_mask(H, P, 0, &has_t);
            if (has_t || lo != u) continue;
            const double bI = rhs_string(c, 3, H, P);
            total += 2.0 * (-bI * bI / diag3(c, H, P));
            count += 2;
          }
      }
  }
  /* up-down-down with an up pair u -> u' (u != t) and any down-down double */
#pragma omp parallel for reduction(+ : total, count) schedule(dynamic, 1)
  for (int u = 1; u < No; ++u) {
    for (int j = 0; j < No; ++j)
      for (int k = j + 1; k < No; ++k)
        for (int b = 0; b < Nv; ++b)
          for (int cc = b + 1; cc < Nv; ++cc) {
            orb H[3] = {{0, u, 0}, {0, j, 1}, {0, k, 1}}, P[3] = {{1, u, 0}, {1, b, 1}, {1, cc, 1}};
            int has_t = 0;
            pairs_mask(H, P, 1, &has_t);
            if (has_t) continue;
            const double bI = rhs_string(c, 3, H, P);
            total += 2.0 * (-bI * bI / diag3(c, H, P));
            count += 2;
          }
  }
  /* up-down-down with no up pair and a down pair u -> u' (u != t), lowest down pair u */
#pragma omp parallel for reduction(+ : total, count) schedule(dynamic, 1)
  for (int u = 1; u < No; ++u) {
    for (int i = 0; i < No; ++i)
      for (int a = 0; a < Nv; ++a) {
        if (a == i) continue;
        for (int k = 0; k < No; ++k) {
          if (k == u) continue;
          for (int cc = 0; cc < Nv; ++cc) {
            if (cc == u) continue;
            orb H[3] = {{0, i, 0}, {0, u, 1}, {0, k, 1}}, P[3] = {{1, a, 0}, {1, u, 1}, {1, cc, 1}};
            int has_t = 0;
            const int lo = pairs_mask(H, P, 1, &has_t);
            if (has_t || lo != u) continue;
            const double bI = rhs_string(c, 3, H, P);
            total += 2.0 * (-bI * bI / diag3(c, H, P));
            count += 2;
          }
        }
      }
  }
  if (count_out) *count_out = count;
  return total;
}

/* ------------------------------------------------------------------ setup */
o2_ctx *o2_create(int No, int Nv, const double *F, const double *lam, const double *ovov,
                  const double *ooov, const double *ovvt) {
  o2_ctx *c = (o2_ctx *)calloc(1, sizeof(o2_ctx));
  c->No = No; c->Nv = Nv; c->F = F; c->lam = lam; c->ovov = ovov; c->ooov = ooov; c->ovvt = ovvt;
  double om = 0.0;
  for (int u = 0; u < No; ++u) om += 2.0 * lam[u] * lam[u] * (Fvv(c, u, u) - Foo(c, u, u));
  c->omega = om;
  c->f0vo = (double *)malloc(sizeof(double) * (size_t)Nv * No);
  for (int a = 0; a < Nv; ++a)
    for (int j = 0; j < No; ++j) {
      const orb A = {1, a, 0}, J = {0, j, 0};
      double v = Fov(c, j, a);
      for (int u = 0; u < No; ++u) {
        const double w = 2.0 * lam[u] * lam[u];
        const orb uo = {0, u, 0}, uv = {1, u, 0};
        v += w * (eri(c, A, J, uo, uo) - 0.5 * eri(c, A, uo, uo, J));
        v -= w * (eri(c, A, J, uv, uv) - 0.5 * eri(c, A, uv, uv, J));
      }
      c->f0vo[(size_t)a * No + j] = v;
    }
  return c;
}

double o2_omega(const o2_ctx *c) { return c->omega; }
/* level shift s: H0 -> H0 + s on the first-order space (every denominator + s) */
void o2_set_shift(o2_ctx *c, double s) { c->shift = s; }
int o2_error(const o2_ctx *c) { return c->err; }
void o2_f0vo(const o2_ctx *c, double *out) { memcpy(out, c->f0vo, sizeof(double) * (size_t)c->Nv * c->No); }
void o2_destroy(o2_ctx *c) { if (c) { free(c->f0vo); free(c); } }

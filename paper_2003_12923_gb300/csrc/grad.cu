// Analytic gradient of E2 with respect to the Fock matrix and the (ov|ov) integrals.
//
// With A x = -b (A self-adjoint in the determinant inner product <,>) and E2 = <b,x> + E2_S:
//   dE2 = 2 <x, db> + <x, dA x> + dE2_S .
// The adjoint vector of the first-order equation is x itself (A is symmetric); an adjoint
// solve can be run and compared with x.  Contributions (TOP basis, then rotated back):
//   <x, dA x>, one-body part: densities of x contracted over every index but one (the
//       N_o^2 N_v^3 / N_o^3 N_v^2 float64 GEMMs below), plus the N^4 coupling terms, the pair
//       energy of the L blocks and omega;
//   2 <x, db>: the (ov|ov)-dependence of the L-triple right-hand side and the F_vo-dependence
//       of the doubles right-hand side (through the closed-shell Fock block f0);
//   dE2_S: the S-space sum -b_I^2 / D_I differentiated in b_I (integrals) and D_I (diagonal F).
// Conventions: dF is the derivative of E2 evaluated on (F + F^T)/2 (so dF is symmetric) and
// dOVOV[i][a][j][b] the derivative of E2 evaluated on the (ia)<->(jb) symmetrised block.
#include <cmath>
#include <vector>

#include "internal.h"

namespace esmp2 {
namespace {

constexpr double WT = 0.5, WS = 1.0, WX = 0.5, WY = 0.5, WZ = 2.0;

struct GCtx {
  int No, Nv, N;
  int64_t B;
  const double *x, *lam, *ovov, *F;
  double omega;
  __device__ __forceinline__ double X(int blk, int i, int j, int a, int b) const {
    return x[blk * B + (((int64_t)i * No + j) * Nv + a) * Nv + b];
  }
  __device__ __forceinline__ int64_t ov(int i, int a, int j, int b) const {
    return (((int64_t)i * Nv + a) * No + j) * Nv + b;
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ double block_sum(double v) {
  __shared__ double sh[32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;  // valid in thread 0
}

// (ov|ov) gradient from the L-triple right-hand side (elementwise part)
__global__ void kg_ovov_L(GCtx c, double *G) {
  const int No = c.No, Nv = c.Nv;
  const double l0 = c.lam[0];
  const int64_t n = (int64_t)No * Nv * No * Nv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t f = e;
    const int g = (int)(f % Nv); f /= Nv;
    const int q = (int)(f % No); f /= No;
    const int be = (int)(f % Nv);
    const int p = (int)(f / Nv);
    G[e] += l0 * (4.0 * WX * c.X(BX, p, q, be, g) + 4.0 * WY * c.X(BY, p, q, be, g) + 2.0 * WZ * c.X(BZ, p, q, be, g));
  }
}

// per (J, B): partner-weighted sums of x entering the (ov|ov) entries with a TOP index and f0
__global__ void kg_small(GCtx c, double *Gov, double *Gf) {
  const int No = c.No, Nv = c.Nv, N = c.N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < No * Nv; e += gridDim.x * blockDim.x) {
    const int J = e / Nv, Bv = e % Nv;
    double RX = 0, RY = 0, RZ1 = 0, RZ2 = 0, RT = 0, RS1 = 0, RS2 = 0;
    for (int k = 0; k < No; ++k) {
      const double l = c.lam[k];
      RX += l * c.X(BX, J, k, Bv, k);
      RY += l * c.X(BY, J, k, Bv, k);
      RZ1 += l * c.X(BZ, J, k, Bv, k);
      RZ2 += l * c.X(BZ, k, J, k, Bv);
      RT += l * c.X(BT, k, J, k, Bv);
      RS1 += l * c.X(BS, k, J, k, Bv);
      RS2 += l * c.X(BS, J, k, Bv, k);
    }
    atomicAdd(&Gov[c.ov(0, 0, J, Bv)], 8.0 * WX * RX + 8.0 * WY * RY);
    atomicAdd(&Gov[c.ov(J, 0, 0, Bv)], -8.0 * WX * RX);
    atomicAdd(&Gov[c.ov(J, Bv, 0, 0)], 2.0 * WZ * (RZ1 + RZ2));
    atomicAdd(&Gov[c.ov(0, Bv, J, 0)], -2.0 * WZ * RZ2);
    atomicAdd(&Gf[(int64_t)J * N + No + Bv], 8.0 * WT * RT + 2.0 * WS * (RS1 + RS2));  // 2<x, d b / d f0_BJ>
  }
}

// F1 (F_ov(0,0)), <x,x>, <x_L,x_L>: grid-stride, block partials via atomics into acc[0..2]
__global__ void kg_scalars(GCtx c, double *acc) {
  const int No = c.No, Nv = c.Nv;
  double f1 = 0, nn = 0, nl = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < c.B; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t f = e;
    const int b = (int)(f % Nv); f /= Nv;
    const int a = (int)(f % Nv); f /= Nv;
    const int j = (int)(f % No);
    const int i = (int)(f / No);
    const double t = c.X(BT, i, j, a, b), s = c.X(BS, i, j, a, b), xx = c.X(BX, i, j, a, b),
                 y = c.X(BY, i, j, a, b), z = c.X(BZ, i, j, a, b);
    f1 += WT * t * (xx + y) + WS * s * (z + c.X(BZ, j, i, b, a)) + WX * xx * t + WY * y * t + WZ * z * s;
    nl += WX * xx * xx + WY * y * y + WZ * z * z;
    nn += WT * t * t + WS * s * s;
  }
  nn += nl;
  const double r0 = block_sum(f1), r1 = block_sum(nn), r2 = block_sum(nl);
  if (threadIdx.x == 0) { atomicAdd(&acc[0], r0); atomicAdd(&acc[1], r1); atomicAdd(&acc[2], r2); }
}

// F2: d/dF_ov(0,c), one block per c
__global__ void kg_F2(GCtx c, double *Gf) {
  const int No = c.No, Nv = c.Nv, cc = blockIdx.x;
  double s = 0;
  for (int64_t r = threadIdx.x; r < (int64_t)No * No * Nv; r += blockDim.x) {
    const int b = (int)(r % Nv), ij = (int)(r / Nv), i = ij / No, j = ij % No;
    s += -2.0 * WT * c.X(BT, i, j, 0, b) * c.X(BX, i, j, cc, b)
         - WS * c.X(BS, i, j, b, 0) * c.X(BZ, i, j, b, cc)
         - WS * c.X(BS, i, j, 0, b) * c.X(BZ, j, i, b, cc)
         - 2.0 * WX * c.X(BX, i, j, cc, b) * c.X(BT, i, j, 0, b)
         - WZ * c.X(BZ, i, j, b, cc) * c.X(BS, i, j, b, 0);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) Gf[No + cc] += s;
}

// F3: d/dF_ov(k,0), one block per k
__global__ void kg_F3(GCtx c, double *Gf) {
  const int No = c.No, Nv = c.Nv, k = blockIdx.x;
  double s = 0;
  for (int64_t r = threadIdx.x; r < (int64_t)No * Nv * Nv; r += blockDim.x) {
    const int b = (int)(r % Nv), a = (int)((r / Nv) % Nv), j = (int)(r / ((int64_t)Nv * Nv));
    s += -2.0 * WT * c.X(BT, 0, j, a, b) * c.X(BX, k, j, a, b)
         - WS * c.X(BS, j, 0, a, b) * c.X(BZ, j, k, a, b)
         - WS * c.X(BS, 0, j, a, b) * c.X(BZ, j, k, b, a)
         - 2.0 * WX * c.X(BX, k, j, a, b) * c.X(BT, 0, j, a, b)
         - WZ * c.X(BZ, j, k, a, b) * c.X(BS, j, 0, a, b);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) Gf[(int64_t)k * c.N + No] += s;
}

// F4: d/dF_ov(k,c), one block per (k,c)
__global__ void kg_F4(GCtx c, double *Gf) {
  const int No = c.No, Nv = c.Nv, k = blockIdx.x / Nv, cc = blockIdx.x % Nv;
  double s = 0;
  for (int r = threadIdx.x; r < No * Nv; r += blockDim.x) {
    const int j = r / Nv, b = r % Nv;
    s += 4.0 * WT * c.X(BT, 0, j, 0, b) * (c.X(BX, k, j, cc, b) + c.X(BZ, k, j, cc, b))
         + WS * (c.X(BS, j, 0, b, 0) + c.X(BS, 0, j, 0, b)) * (c.X(BY, j, k, b, cc) + c.X(BZ, j, k, b, cc))
         + 4.0 * WX * c.X(BX, k, j, cc, b) * c.X(BT, 0, j, 0, b)
         + 4.0 * WY * c.X(BY, j, k, b, cc) * c.X(BS, 0, j, 0, b)
         + WZ * c.X(BZ, j, k, b, cc) * c.X(BS, j, 0, b, 0)
         + WZ * c.X(BZ, k, j, cc, b) * c.X(BT, 0, j, 0, b);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) Gf[(int64_t)k * c.N + No + cc] += s;
}

// F5..F8: the t / t' row and column terms of the mixed-spin L blocks; one block per index
__global__ void kg_F5to8(GCtx c, double *Gf) {
  const int No = c.No, Nv = c.Nv, N = c.N;
  int id = blockIdx.x;
  int fam;
  if (id < Nv) fam = 5;
  else if ((id -= Nv) < No) fam = 6;
  else if ((id -= No) < Nv) fam = 7;
  else { id -= Nv; fam = 8; }
  double s = 0;
  for (int r = threadIdx.x; r < No * Nv; r += blockDim.x) {
    const int j = r / Nv, b = r % Nv;
    if (fam == 5) s += 4.0 * WY * c.X(BY, 0, j, 0, b) * c.X(BZ, 0, j, id, b);
    else if (fam == 6) s -= 4.0 * WY * c.X(BY, 0, j, 0, b) * c.X(BZ, id, j, 0, b);
    else if (fam == 7) s += WZ * c.X(BZ, 0, j, id, b) * c.X(BY, 0, j, 0, b);
    else s -= WZ * c.X(BZ, id, j, 0, b) * c.X(BY, 0, j, 0, b);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) {
    if (fam == 5) Gf[(int64_t)No * N + No + id] += s;      // F_vv(0,d)
    else if (fam == 6) Gf[(int64_t)id * N] += s;           // F_oo(l,0)
    else if (fam == 7) Gf[(int64_t)(No + id) * N + No] += s;  // F_vv(a,0)
    else Gf[id] += s;                                      // F_oo(0,i)
  }
}

// scalars into Gf: F_ov(0,0), pair energy of L, omega
__global__ void kg_finish_scalars(GCtx c, const double *acc, double *Gf) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int No = c.No, N = c.N;
  Gf[No] += acc[0];
  Gf[(int64_t)No * N + No] += acc[2];
  Gf[0] -= acc[2];
  for (int u = 0; u < No; ++u) {
    const double w = 2.0 * c.lam[u] * c.lam[u] * acc[1];
    Gf[(int64_t)(No + u) * N + No + u] -= w;
    Gf[(int64_t)u * N + u] += w;
  }
}

// ---- S space: E2_S = sum_I 2 (-b_I^2 / D_I); scatter dE2_S/db_I into (ov|ov), dE2_S/dD_I into diag F
struct SG {
  GCtx c;
  double *Gov, *Gdiag;  // Gdiag[N + 1]: diagonal F gradient and (last) the omega sum
  __device__ void triple(const int *ho, const int *hs, const int *po, const int *ps, double *sdiag) const {
    const int PERM[3][3] = {{0, 1, 2}, {2, 1, 0}, {0, 2, 1}};
    const int PSG[3] = {1, -1, -1};
    const int No = c.No, N = c.N;
    double bI = 0.0;
    for (int t = 0; t < 3; ++t)
      for (int r = 0; r < 3; ++r) {
        const int h3 = PERM[t][2], p3 = PERM[r][2];
        if (hs[h3] != ps[p3] || ho[h3] != po[p3]) continue;
        const int H0 = PERM[t][0], H1 = PERM[t][1], P0 = PERM[r][0], P1 = PERM[r][1];
        double a = 0.0;
        if (ps[P0] == hs[H0] && ps[P1] == hs[H1]) a += c.ovov[c.ov(ho[H0], po[P0], ho[H1], po[P1])];
        if (ps[P0] == hs[H1] && ps[P1] == hs[H0]) a -= c.ovov[c.ov(ho[H1], po[P0], ho[H0], po[P1])];
        bI += PSG[t] * PSG[r] * c.lam[ho[h3]] * a;
      }
    double D = -c.omega;
    for (int k = 0; k < 3; ++k)
      D += c.F[(int64_t)(No + po[k]) * N + No + po[k]] - c.F[(int64_t)ho[k] * N + ho[k]];
    const double gb = -4.0 * bI / D, gd = 2.0 * bI * bI / (D * D);
    for (int t = 0; t < 3; ++t)
      for (int r = 0; r < 3; ++r) {
        const int h3 = PERM[t][2], p3 = PERM[r][2];
        if (hs[h3] != ps[p3] || ho[h3] != po[p3]) continue;
        const int H0 = PERM[t][0], H1 = PERM[t][1], P0 = PERM[r][0], P1 = PERM[r][1];
        const double f = gb * PSG[t] * PSG[r] * c.lam[ho[h3]];
        if (ps[P0] == hs[H0] && ps[P1] == hs[H1]) atomicAdd(&Gov[c.ov(ho[H0], po[P0], ho[H1], po[P1])], f);
        if (ps[P0] == hs[H1] && ps[P1] == hs[H0]) atomicAdd(&Gov[c.ov(ho[H1], po[P0], ho[H0], po[P1])], -f);
      }
    for (int k = 0; k < 3; ++k) {
      atomicAdd(&sdiag[No + po[k]], gd);
      atomicAdd(&sdiag[ho[k]], -gd);
    }
    atomicAdd(&sdiag[N], gd);
  }
};

__device__ void flush_diag(const SG &g, double *sdiag) {
  __syncthreads();
  for (int k = threadIdx.x; k <= g.c.N; k += blockDim.x)
    if (sdiag[k] != 0.0) atomicAdd(&g.Gdiag[k], sdiag[k]);
}

// same enumeration as the energy kernels (sector A: up-up-up, B: up pair + down-down, C: down pair only)
__global__ void kg_s_a(SG g) {
  extern __shared__ double sdiag[];
  for (int k = threadIdx.x; k <= g.c.N; k += blockDim.x) sdiag[k] = 0.0;
  __syncthreads();
  const int No = g.c.No, Nv = g.c.Nv;
  const int64_t blk = blockIdx.x;
  const int u = (int)(blk / ((int64_t)No * No)), j = (int)((blk / No) % No), k = (int)(blk % No);
  if (u >= 1 && j < k && j != u && k != u) {
    for (int b = threadIdx.x; b < Nv; b += blockDim.x) {
      if (b == u) continue;
      for (int cc = b + 1; cc < Nv; ++cc) {
        if (cc == u) continue;
        const bool pj = (b == j || cc == j), pk = (b == k || cc == k);
        if ((pj && j < u) || (pk && k < u)) continue;
        if ((pj && j == 0) || (pk && k == 0)) continue;
        const int ho[3] = {u, j, k}, hs[3] = {0, 0, 0}, po[3] = {u, b, cc}, ps[3] = {0, 0, 0};
        g.triple(ho, hs, po, ps, sdiag);
      }
    }
  }
  flush_diag(g, sdiag);
}

__global__ void kg_s_b(SG g) {
  extern __shared__ double sdiag[];
  for (int k = threadIdx.x; k <= g.c.N; k += blockDim.x) sdiag[k] = 0.0;
  __syncthreads();
  const int No = g.c.No, Nv = g.c.Nv;
  const int64_t blk = blockIdx.x;
  const int u = (int)(blk / ((int64_t)No * No)), j = (int)((blk / No) % No), k = (int)(blk % No);
  if (u >= 1 && j < k) {
    for (int b = threadIdx.x; b < Nv; b += blockDim.x)
      for (int cc = b + 1; cc < Nv; ++cc) {
        if ((j == 0 || k == 0) && (b == 0 || cc == 0)) continue;
        const int ho[3] = {u, j, k}, hs[3] = {0, 1, 1}, po[3] = {u, b, cc}, ps[3] = {0, 1, 1};
        g.triple(ho, hs, po, ps, sdiag);
      }
  }
  flush_diag(g, sdiag);
}

__global__ void kg_s_c(SG g) {
  extern __shared__ double sdiag[];
  for (int k = threadIdx.x; k <= g.c.N; k += blockDim.x) sdiag[k] = 0.0;
  __syncthreads();
  const int No = g.c.No, Nv = g.c.Nv;
  const int64_t blk = blockIdx.x;
  const int u = (int)(blk / ((int64_t)No * No)), i = (int)((blk / No) % No), k = (int)(blk % No);
  if (u >= 1 && k != u) {
    for (int a = threadIdx.x; a < Nv; a += blockDim.x) {
      if (a == i) continue;
      for (int cc = 0; cc < Nv; ++cc) {
        if (cc == u) continue;
        if (cc == k && (k < u || k == 0)) continue;
        const int ho[3] = {i, u, k}, hs[3] = {0, 1, 1}, po[3] = {a, u, cc}, ps[3] = {0, 1, 1};
        g.triple(ho, hs, po, ps, sdiag);
      }
    }
  }
  flush_diag(g, sdiag);
}

__global__ void kg_s_finish(GCtx c, const double *Gdiag, double *Gf) {
  const int No = c.No, N = c.N;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    double v = Gdiag[p];
    // omega = sum_u 2 lam_u^2 (F_u'u' - F_uu); D_I contains -omega
    if (p < No) v += 2.0 * c.lam[p] * c.lam[p] * Gdiag[N];
    else if (p < 2 * No) v -= 2.0 * c.lam[p - No] * c.lam[p - No] * Gdiag[N];
    Gf[(int64_t)p * N + p] += v;
  }
}

// symmetrise: out = (G + G^T) / 2 for an n x n matrix
__global__ void kg_sym(const double *G, double *out, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int p = e / n, q = e % n;
    out[e] = 0.5 * (G[e] + G[(int64_t)q * n + p]);
  }
}

// (ov|ov) symmetrisation over (ia) <-> (jb)
__global__ void kg_sym_ov(const double *G, double *out, int No, int Nv) {
  const int64_t M = (int64_t)No * Nv, n = M * M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / M, q = e % M;
    out[e] = 0.5 * (G[e] + G[q * M + r]);
  }
}

__global__ void kg_transpose(const double *A, double *At, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x)
    At[(e % n) * n + e / n] = A[e];
}

}  // namespace

// One-body densities of x (the N^5 part of <x, dA x>), accumulated into Gf (N x N).
static void densities(esmp2_handle *h, const double *x, double *Gf) {
  const int No = h->d.No, Nv = h->d.Nv, N = h->d.N;
  const int64_t B = h->d.B, NvNv = (int64_t)Nv * Nv;
  const double W[5] = {WT, WS, WX, WY, WZ};
  for (int blk = 0; blk < 5; ++blk) {
    const double *X = x + blk * B;
    Gemm64 g{};
    // virtual: sum over rows (s,a) of X[s][a][p] X[s][a][q]
    g.M = Nv; g.N = Nv; g.K = No * No * Nv; g.batch = 1; g.alpha = W[blk]; g.beta = 1.0;
    g.A = X; g.sAm = 1; g.sAk = Nv; g.B = X; g.sBk = Nv; g.sBn = 1;
    g.C = Gf + (int64_t)No * N + No; g.sCm = N; g.sCn = 1;
    gemm64(g, h->stream);
    // virtual: sum over (s,b) of X[s][p][b] X[s][q][b]
    g = Gemm64{};
    g.M = Nv; g.N = Nv; g.K = No * No * Nv; g.batch = 1; g.alpha = W[blk]; g.beta = 1.0;
    g.Kin = Nv;
    g.A = X; g.sAm = Nv; g.sAk = 1; g.sAk1 = NvNv;
    g.B = X; g.sBk = 1; g.sBk1 = NvNv; g.sBn = Nv;
    g.C = Gf + (int64_t)No * N + No; g.sCm = N; g.sCn = 1;
    gemm64(g, h->stream);
    // occupied: -(sum over (j,ab) of X[l][j][ab] X[i][j][ab]) - (sum over (i',ab) of X[i'][l][ab] X[i'][i][ab])
    g = Gemm64{};
    g.M = No; g.N = No; g.K = (int)((int64_t)No * NvNv); g.batch = 1; g.alpha = -W[blk]; g.beta = 1.0;
    g.A = X; g.sAm = (int64_t)No * NvNv; g.sAk = 1; g.B = X; g.sBk = 1; g.sBn = (int64_t)No * NvNv;
    g.C = Gf; g.sCm = N; g.sCn = 1;
    gemm64(g, h->stream);
    g = Gemm64{};
    g.M = No; g.N = No; g.K = (int)((int64_t)No * NvNv); g.batch = 1; g.alpha = -W[blk]; g.beta = 1.0;
    g.Kin = (int)NvNv;
    g.A = X; g.sAm = NvNv; g.sAk = 1; g.sAk1 = (int64_t)No * NvNv;
    g.B = X; g.sBk = 1; g.sBk1 = (int64_t)No * NvNv; g.sBn = NvNv;
    g.C = Gf; g.sCm = N; g.sCn = 1;
    gemm64(g, h->stream);
    h->launches += 4;
  }
}

esmp2_status gradient(esmp2_handle *h, double *dF_host, double *dOVOV_host, int adjoint, double *adj_diff) {
  if (!h->solved) { h->err = "esmp2_grad needs a previous esmp2_solve"; return ESMP2_ERR_STATE; }
  const int No = h->d.No, Nv = h->d.Nv, N = h->d.N;
  const int64_t nov = (int64_t)No * Nv * No * Nv, n = h->d.n;
  cudaStream_t st = h->stream;
  if (esmp2_status s0 = x_to_basis(h, 0)) return s0;
  if (adj_diff) *adj_diff = 0.0;
  if (adjoint) {  // A is symmetric: the adjoint solve A^T lambda = -b must return x itself
    double *xs = nullptr;
    cudaError_t ce = cudaMalloc(&xs, sizeof(double) * n);
    if (ce != cudaSuccess) return check_cuda(h, ce, "adjoint");
    cudaMemcpyAsync(xs, h->s64.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(h->s64.x, 0, sizeof(double) * n, st);
    h->x_zero = true;
    h->r_true = false;
    esmp2_solve_info info{};
    esmp2_status s = solve64(h, 1e-12, 5000, &info);
    if (s != ESMP2_OK && s != ESMP2_ERR_NOT_CONVERGED) { cudaFree(xs); return s; }
    // relative difference |lambda - x| / |x| (plain Euclidean on the stored blocks)
    std::vector<double> a(n), b(n);
    cudaMemcpy(a.data(), h->s64.x, sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(b.data(), xs, sizeof(double) * n, cudaMemcpyDeviceToHost);
    double dd = 0, xx = 0;
    for (int64_t k = 0; k < n; ++k) { dd += (a[k] - b[k]) * (a[k] - b[k]); xx += b[k] * b[k]; }
    if (adj_diff) *adj_diff = xx > 0 ? std::sqrt(dd / xx) : 0.0;
    cudaMemcpyAsync(h->s64.x, xs, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    h->x_zero = false;
    h->r_true = false;
    cudaStreamSynchronize(st);
    cudaFree(xs);
  }
  double *Gf = nullptr, *Gov = nullptr, *acc = nullptr, *T1 = nullptr, *T2 = nullptr, *Gd = nullptr;
  cudaError_t ce = cudaSuccess;
  auto A = [&](double **p, size_t cnt) { if (ce == cudaSuccess) ce = cudaMalloc(p, sizeof(double) * cnt); };
  A(&Gf, (size_t)N * N); A(&Gov, (size_t)nov); A(&acc, 4); A(&T1, (size_t)std::max<int64_t>((int64_t)N * N, nov));
  A(&T2, (size_t)std::max<int64_t>((int64_t)N * N, nov)); A(&Gd, (size_t)N + 1);
  if (ce != cudaSuccess) {
    cudaFree(Gf); cudaFree(Gov); cudaFree(acc); cudaFree(T1); cudaFree(T2); cudaFree(Gd);
    return check_cuda(h, ce, "gradient workspace");
  }
  cudaMemsetAsync(Gf, 0, sizeof(double) * N * N, st);
  cudaMemsetAsync(Gov, 0, sizeof(double) * nov, st);
  cudaMemsetAsync(acc, 0, sizeof(double) * 4, st);
  cudaMemsetAsync(Gd, 0, sizeof(double) * (N + 1), st);
  GCtx c;
  c.No = No; c.Nv = Nv; c.N = N; c.B = h->d.B; c.x = h->s64.x; c.lam = h->lam; c.ovov = h->ovov; c.F = h->F;
  c.omega = h->omega_op;
  densities(h, h->s64.x, Gf);
  kg_ovov_L<<<1216, 256, 0, st>>>(c, Gov);
  kg_small<<<(unsigned)cdiv((int64_t)No * Nv, 128), 128, 0, st>>>(c, Gov, Gf);
  kg_scalars<<<1216, 256, 0, st>>>(c, acc);
  kg_F2<<<Nv, 256, 0, st>>>(c, Gf);
  kg_F3<<<No, 256, 0, st>>>(c, Gf);
  kg_F4<<<No * Nv, 128, 0, st>>>(c, Gf);
  kg_F5to8<<<2 * (No + Nv), 128, 0, st>>>(c, Gf);
  kg_finish_scalars<<<1, 32, 0, st>>>(c, acc, Gf);
  SG sg;
  sg.c = c; sg.Gov = Gov; sg.Gdiag = Gd;
  const int nb = No * No * No;
  const size_t shm = sizeof(double) * (N + 1);
  kg_s_a<<<nb, 128, shm, st>>>(sg);
  kg_s_b<<<nb, 128, shm, st>>>(sg);
  kg_s_c<<<nb, 128, shm, st>>>(sg);
  kg_s_finish<<<(unsigned)cdiv(N, 128), 128, 0, st>>>(c, Gd, Gf);
  h->launches += 13;
  // dF = W sym(Gf) W^T
  kg_sym<<<256, 256, 0, st>>>(Gf, T1, N);
  Gemm64 g{};
  g.alpha = 1.0; g.beta = 0.0; g.batch = 1; g.M = N; g.N = N; g.K = N;
  g.A = h->W; g.sAm = N; g.sAk = 1; g.B = T1; g.sBk = N; g.sBn = 1; g.C = T2; g.sCm = N; g.sCn = 1;
  gemm64(g, st);
  g.A = T2; g.sAm = N; g.sAk = 1; g.B = h->W; g.sBk = 1; g.sBn = N; g.C = T1; g.sCm = N; g.sCn = 1;
  gemm64(g, st);
  if (dF_host) cudaMemcpyAsync(dF_host, T1, sizeof(double) * N * N, cudaMemcpyDeviceToHost, st);
  // dOVOV: symmetrise, then rotate every index back (in[i'] -> sum_i' U[i][i'] in[i'])
  kg_sym_ov<<<1216, 256, 0, st>>>(Gov, T1, No, Nv);
  double *Ut_d = nullptr, *Wvt_d = nullptr;
  cudaMalloc(&Ut_d, sizeof(double) * No * No);
  cudaMalloc(&Wvt_d, sizeof(double) * Nv * Nv);
  kg_transpose<<<64, 256, 0, st>>>(h->U, Ut_d, No);
  kg_transpose<<<256, 256, 0, st>>>(h->Wv, Wvt_d, Nv);
  const int dims[4] = {No, Nv, No, Nv};
  const double *R[4] = {Ut_d, Wvt_d, Ut_d, Wvt_d};
  const int K[4] = {No, Nv, No, Nv};
  double *src = T1, *dst = T2;
  for (int m = 0; m < 4; ++m) {
    mode_product(src, dst, dims, m, R[m], K[m], K[m], st);
    double *t = src; src = dst; dst = t;
  }
  h->launches += 10;
  if (dOVOV_host) cudaMemcpyAsync(dOVOV_host, src, sizeof(double) * nov, cudaMemcpyDeviceToHost, st);
  ce = cudaStreamSynchronize(st);
  cudaFree(Gf); cudaFree(Gov); cudaFree(acc); cudaFree(T1); cudaFree(T2); cudaFree(Gd); cudaFree(Ut_d); cudaFree(Wvt_d);
  if (ce == cudaSuccess) ce = cudaGetLastError();
  return check_cuda(h, ce, "gradient");
}

}  // namespace esmp2

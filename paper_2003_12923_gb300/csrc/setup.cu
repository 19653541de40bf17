// One-time setup on the device: TOP basis (Sec. II.A, Eqs. 2-4), orbital transforms,
// the closed-shell Fock block f0_vo and the right-hand side b = Q H Psi0 on D+L.
//
// Conventions (shared by construction with every consumer of the TOP basis):
//  * 2 ||C||^2 = 1;
//  * SVD by one-sided (Hestenes) Jacobi on the rows of C, singular values sorted in
//    descending order, column k of V signed so its largest-magnitude component is
//    positive, u_k = C v_k / lambda_k;
//  * AVOs = columns No.. of the product of the Householder reflectors that
//    triangularise V (H = I - 2 w w^T / w^T w, w = x - alpha e_0, alpha = -sign(x_0)|x|).
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace esmp2 {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 2 |C|^2 = 1 (each spin-adapted CSF of Eq. psi0 has norm^2 2).
__global__ void k_normalise(const double *Cin, double *C, int n) {
  __shared__ double part[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) s += Cin[k] * Cin[k];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[0] = v;
  }
  __syncthreads();
  const double scale = 1.0 / sqrt(2.0 * part[0]);
  for (int k = threadIdx.x; k < n; k += blockDim.x) C[k] = Cin[k] * scale;
}

// One-sided Jacobi SVD of C (No x Nv, No <= 64): rotate the rows of B = C with an
// orthogonal J until they are mutually orthogonal; then C = J diag(|B_k|) (B_k/|B_k|).
// One warp per row pair, pairs of a round disjoint (round-robin ordering).
// Outputs: U (No x No), lam (No), V into columns 0..No-1 of Wv (Nv x Nv).
__global__ void __launch_bounds__(1024) k_jacobi_svd(const double *C, double *B, double *J, double *U,
                                                     double *lam, double *Wv, int No, int Nv) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __shared__ int rotated;
  __shared__ int perm[64];
  __shared__ double nrm[64];
  for (int k = threadIdx.x; k < No * Nv; k += blockDim.x) B[k] = C[k];
  for (int k = threadIdx.x; k < No * No; k += blockDim.x) J[k] = (k / No == k % No) ? 1.0 : 0.0;
  __syncthreads();
  const int n = (No & 1) ? No + 1 : No;  // padded with a dummy row when No is odd
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < n - 1; ++r) {
      for (int pi = warp; pi < n / 2; pi += nw) {
        int p, q;
        if (pi == 0) { p = 0; q = 1 + (r % (n - 1)); }
        else { p = 1 + ((pi + r) % (n - 1)); q = 1 + ((n - 1 - pi + r) % (n - 1)); }
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= No) continue;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int a = lane; a < Nv; a += 32) {
          const double x = B[p * Nv + a], y = B[q * Nv + a];
          al += x * x; be += y * y; ga += x * y;
        }
        al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
        if (al <= 1e-300 || be <= 1e-300) continue;
        if (fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int a = lane; a < Nv; a += 32) {
          const double x = B[p * Nv + a], y = B[q * Nv + a];
          B[p * Nv + a] = c * x - s * y;
          B[q * Nv + a] = s * x + c * y;
        }
        for (int i = lane; i < No; i += 32) {
          const double x = J[i * No + p], y = J[i * No + q];
          J[i * No + p] = c * x - s * y;
          J[i * No + q] = s * x + c * y;
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    const int any = rotated;
    __syncthreads();
    if (!any) break;
  }
  // row norms and descending order
  for (int k = warp; k < No; k += nw) {
    double s = 0.0;
    for (int a = lane; a < Nv; a += 32) s += B[k * Nv + a] * B[k * Nv + a];
    s = warp_sum(s);
    if (lane == 0) nrm[k] = sqrt(s);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < No; ++k) perm[k] = k;
    for (int k = 0; k < No; ++k) {
      int best = k;
      for (int l = k + 1; l < No; ++l)
        if (nrm[perm[l]] > nrm[perm[best]]) best = l;
      const int t = perm[k]; perm[k] = perm[best]; perm[best] = t;
    }
  }
  __syncthreads();
  const double lmax = nrm[perm[0]];
  // V columns, sign convention, u_k = C v_k / lambda_k.  Done by warp 0 in order so that
  // columns with a vanishing singular value can be completed against earlier ones.
  if (warp == 0) {
    for (int kk = 0; kk < No; ++kk) {
      const int o = perm[kk];
      const double l = nrm[o];
      const bool live = l > 1e-12 * lmax && l > 1e-300;
      if (live) {
        for (int a = lane; a < Nv; a += 32) Wv[a * Nv + kk] = B[o * Nv + a] / l;
      } else {  // Gram-Schmidt completion with the first unit vector that survives
        for (int m = 0; m < Nv; ++m) {
          double nn = 0.0;
          for (int a = lane; a < Nv; a += 32) {
            double v = (a == m) ? 1.0 : 0.0;
            for (int prev = 0; prev < kk; ++prev) v -= Wv[m * Nv + prev] * Wv[a * Nv + prev];
            Wv[a * Nv + kk] = v;
            nn += v * v;
          }
          nn = warp_sum(nn);
          if (nn > 0.25) {
            const double inv = 1.0 / sqrt(nn);
            for (int a = lane; a < Nv; a += 32) Wv[a * Nv + kk] *= inv;
            break;
          }
        }
      }
      __syncwarp();
      // argmax |v| (first occurrence)
      double best = -1.0;
      int bi = 0x7fffffff;
      for (int a = lane; a < Nv; a += 32) {
        const double v = fabs(Wv[a * Nv + kk]);
        if (v > best) { best = v; bi = a; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      const double sg = Wv[bi * Nv + kk] < 0 ? -1.0 : 1.0;
      for (int a = lane; a < Nv; a += 32) Wv[a * Nv + kk] *= sg;
      __syncwarp();
      for (int i = lane; i < No; i += 32) {
        double u;
        if (live) {
          u = 0.0;
          for (int a = 0; a < Nv; ++a) u += C[i * Nv + a] * Wv[a * Nv + kk];
          u /= l;
        } else {
          u = sg * J[i * No + o];
        }
        U[i * No + kk] = u;
      }
      if (lane == 0) lam[kk] = live ? l : 0.0;
      __syncwarp();
    }
  }
}

// Householder reflectors triangularising V (columns 0..No-1 of Wv).  A: Nv x No work copy,
// R: Nv x No reflector vectors (column k holds w_k on rows k..Nv-1), ww: No norms^2.
__global__ void __launch_bounds__(1024) k_householder(const double *Wv, double *A, double *R, double *ww,
                                                      int No, int Nv) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __shared__ double sh_ww;
  for (int e = threadIdx.x; e < Nv * No; e += blockDim.x) {
    A[e] = Wv[(e / No) * Nv + (e % No)];
    R[e] = 0.0;
  }
  __syncthreads();
  for (int k = 0; k < No; ++k) {
    if (warp == 0) {
      double s = 0.0;
      for (int r = k + lane; r < Nv; r += 32) s += A[r * No + k] * A[r * No + k];
      s = warp_sum(s);
      const double x0 = A[k * No + k];
      const double alpha = -(x0 >= 0 ? 1.0 : -1.0) * sqrt(s);
      double w2 = 0.0;
      for (int r = k + lane; r < Nv; r += 32) {
        const double w = A[r * No + k] - (r == k ? alpha : 0.0);
        R[r * No + k] = w;
        w2 += w * w;
      }
      w2 = warp_sum(w2);
      if (lane == 0) { sh_ww = w2; ww[k] = w2; }
    }
    __syncthreads();
    const double w2 = sh_ww;
    if (w2 > 0.0) {
      for (int col = k + warp; col < No; col += nw) {
        double d = 0.0;
        for (int r = k + lane; r < Nv; r += 32) d += R[r * No + k] * A[r * No + col];
        d = warp_sum(d) * (2.0 / w2);
        for (int r = k + lane; r < Nv; r += 32) A[r * No + col] -= d * R[r * No + k];
      }
    }
    __syncthreads();
  }
}

// AVO column j = H_0 H_1 ... H_{No-1} e_{No+j}, written to Wv[:, No+j].  One warp per column;
// E is Nv-1-No rows of scratch, row j contiguous.
__global__ void k_avo(const double *R, const double *ww, double *E, double *Wv, int No, int Nv) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int navo = Nv - No;
  if (warp >= navo) return;
  double *e = E + (int64_t)warp * Nv;
  for (int r = lane; r < Nv; r += 32) e[r] = (r == No + warp) ? 1.0 : 0.0;
  __syncwarp();
  for (int k = No - 1; k >= 0; --k) {
    const double w2 = ww[k];
    if (w2 <= 0.0) continue;
    double d = 0.0;
    for (int r = k + lane; r < Nv; r += 32) d += R[r * No + k] * e[r];
    d = warp_sum(d) * (2.0 / w2);
    for (int r = k + lane; r < Nv; r += 32) e[r] -= d * R[r * No + k];
    __syncwarp();
  }
  for (int r = lane; r < Nv; r += 32) Wv[(int64_t)r * Nv + No + warp] = e[r];
}

__global__ void k_assemble_W(const double *U, const double *Wv, double *W, int No, int Nv) {
  const int N = No + Nv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)N * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / N), q = (int)(e % N);
    double v = 0.0;
    if (p < No && q < No) v = U[p * No + q];
    else if (p >= No && q >= No) v = Wv[(int64_t)(p - No) * Nv + (q - No)];
    W[e] = v;
  }
}

// omega = sum_u 2 lam_u^2 (F_u'u' - F_uu);  E0 = E_Phi[F] + omega = 2 sum_i F_ii + omega.
__global__ void k_scalars(const double *F, const double *lam, double *scal, int No, int Nv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int N = No + Nv;
  double om = 0.0, eph = 0.0;
  for (int u = 0; u < No; ++u) {
    om += 2.0 * lam[u] * lam[u] * (F[(int64_t)(No + u) * N + No + u] - F[(int64_t)u * N + u]);
    eph += 2.0 * F[(int64_t)u * N + u];
  }
  scal[0] = om;
  scal[1] = eph + om;
}

// f0_aj: the Fock matrix of the closed-shell determinant Phi, F - G[gamma - gamma_Phi],
// with gamma - gamma_Phi = -2 lam_u^2 on occupied u and +2 lam_u^2 on TOP virtual u'.
__global__ void k_f0vo(const double *F, const double *lam, const double *ooov, const double *ovvt,
                       double *f0, int No, int Nv) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Nv * No) return;
  const int a = e / No, j = e % No, N = No + Nv;
  double v = F[(int64_t)j * N + No + a];
  for (int u = 0; u < No; ++u) {
    const double w = 2.0 * lam[u] * lam[u];
    const double aj_uu = ooov[(((int64_t)u * No + u) * No + j) * Nv + a];
    const double au_uj = ooov[(((int64_t)u * No + j) * No + u) * Nv + a];
    const double aj_pp = ovvt[(((int64_t)j * Nv + a) * Nv + u) * No + u];
    const double ap_pj = ovvt[(((int64_t)j * Nv + u) * Nv + a) * No + u];
    v += w * (aj_uu - 0.5 * au_uj) - w * (aj_pp - 0.5 * ap_pj);
  }
  f0[e] = v;
}

__device__ __forceinline__ bool valid_elem(int blk, int i, int j, int a, int b) {
  if ((blk == BT || blk == BX || blk == BY) && (i == j || a == b)) return false;
  if (blk == BX && (i == 0 || j == 0 || a == 0 || b == 0)) return false;
  if (blk == BZ && (j == 0 || b == 0 || (i == 0 && a == 0))) return false;
  return true;
}

// b = Q H Psi0 on the stored blocks (Slater-Condon rules with Psi0 = sum_u lam_u (u -> u')):
//  doubles: P(ij)P(ab)[s_ia f0_bj] + P(ij) sum_c <ab||cj> s_ic - P(ab) sum_k <kb||ij> s_ka
//  triples: P(k/ij)P(c/ab)[<ab||ij> s_kc]  (disconnected product of the double and the single)
//  Q[i][u][b][a] = (ia|bu'): the OVVT integrals with the last two index pairs moved so
//  that one of the two OVVT terms of every T/S element runs along b; the other (a and b
//  exchanged) is staged through shared memory.  One CTA per (block, i, j, 32-row strip of
//  a), b in tiles of 32.
__global__ void __launch_bounds__(256) k_rhs(const double *lam, const double *f0, const double *ovov,
                                             const double *ooov, const double *Q, double *out, int No, int Nv) {
  __shared__ double tji[32][33], tij[32][33];
  const int64_t sNv = Nv, NvNv = (int64_t)Nv * Nv;
  const int blk = blockIdx.z, i = blockIdx.y / No, j = blockIdx.y % No, a0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#define OVOV(i, a, j, b) ovov[(((int64_t)(i) * sNv + (a)) * No + (j)) * sNv + (b)]
#define OOOV(i, j, k, a) ooov[(((int64_t)(i) * No + (j)) * No + (k)) * sNv + (a)]
#define F0(a, j) f0[(int64_t)(a) * No + (j)]
  const double *Qji = Q + ((int64_t)j * No + i) * NvNv;  // Qji[a][b] = OVVT(j, b, a, i)
  const double *Qij = Q + ((int64_t)i * No + j) * NvNv;  // Qij[a][b] = OVVT(i, b, a, j)
  double *ys = out + (((int64_t)blk * No + i) * No + j) * NvNv;
  const double li = lam[i], lj = lam[j], l0 = lam[0];
  for (int b0 = 0; b0 < Nv; b0 += 32) {
    if (blk == BT || blk == BS) {  // tji[bb][aa] = OVVT(j, a, b, i), tij[bb][aa] = OVVT(i, a, b, j)
      __syncthreads();
      for (int r = ty; r < 32; r += 8) {
        const int bb = b0 + r, aa = a0 + tx;
        const bool in = bb < Nv && aa < Nv;
        tji[r][tx] = in ? Qji[(int64_t)bb * Nv + aa] : 0.0;
        tij[r][tx] = in ? Qij[(int64_t)bb * Nv + aa] : 0.0;
      }
      __syncthreads();
    }
    const int b = b0 + tx;
    if (b >= Nv) continue;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int ar = ty + 8 * rr, a = a0 + ar;
      if (a >= Nv) break;
      double v = 0.0;
      if (valid_elem(blk, i, j, a, b)) {
        if (blk == BT) {
          if (a == i) v += li * F0(b, j);
          if (a == j) v -= lj * F0(b, i);
          if (b == i) v -= li * F0(a, j);
          if (b == j) v += lj * F0(a, i);
          v += li * (Qji[(int64_t)a * Nv + b] - tji[tx][ar]) - lj * (Qij[(int64_t)a * Nv + b] - tij[tx][ar]);
          if (a < No) v -= lam[a] * (OOOV(a, i, j, b) - OOOV(a, j, i, b));
          if (b < No) v += lam[b] * (OOOV(b, i, j, a) - OOOV(b, j, i, a));
        } else if (blk == BS) {
          if (a == i) v += li * F0(b, j);
          if (b == j) v += lj * F0(a, i);
          v += li * Qji[(int64_t)a * Nv + b] + lj * tij[tx][ar];
          if (a < No) v -= lam[a] * OOOV(a, i, j, b);
          if (b < No) v -= lam[b] * OOOV(b, j, i, a);
        } else if (blk == BX || blk == BY) {
          // t j k -> t' b c  (here j,k,b,c = i,j,a,b):  lam_t <bc||jk> + P(jk)P(bc)[lam_k d_ck q(j,b)]
          v = l0 * (OVOV(i, a, j, b) - OVOV(j, a, i, b));
          // X: q(j,b) = <t'b||tj> = (t't|bj) - (t'j|bt);  Y: q(j,b) = (t't|bj) (opposite spins)
          auto q = [&](int jj, int bb) {
            double r = OVOV(0, 0, jj, bb);
            if (blk == BX) r -= OVOV(jj, 0, 0, bb);
            return r;
          };
          if (b == j) v += lj * q(i, a);
          if (b == i) v -= li * q(j, a);
          if (a == j) v -= lj * q(i, b);
          if (a == i) v += li * q(j, b);
        } else {  // BZ: i t k -> a t' c  (here k,c = j,b)
          v = l0 * OVOV(i, a, j, b);
          if (b == j) v += lj * OVOV(i, a, 0, 0);
          if (a == i) v += li * (OVOV(j, b, 0, 0) - OVOV(0, b, j, 0));
        }
      }
      ys[(int64_t)a * Nv + b] = v;
    }
  }
#undef OVOV
#undef OOOV
#undef F0
}

// Eigenvectors of a symmetric m x m block M of F (rows/cols off..off+m-1): one-sided
// Jacobi SVD of M + shift I, with the shift (1 + largest absolute row sum) making it
// positive definite so that its singular vectors are its eigenvectors.
__global__ void k_shifted_block(const double *F, int N, int off, int m, double *M) {
  __shared__ double shift;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int p = 0; p < m; ++p) {
      double r = 0.0;
      for (int q = 0; q < m; ++q) r += fabs(F[(int64_t)(off + p) * N + off + q]);
      mx = fmax(mx, r);
    }
    shift = 1.0 + mx;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int p = e / m, q = e % m;
    M[e] = F[(int64_t)(off + p) * N + off + q] + (p == q ? shift : 0.0);
  }
}

}  // namespace

void eigvecs_block(esmp2_handle *h, const double *F, int off, int m, double *V, double *work) {
  // work: 3 m^2 + m doubles
  double *M = work, *B = work + m * m, *J = work + 2 * m * m, *lam = work + 3 * m * m;
  double *Vt = nullptr;
  cudaMalloc(&Vt, sizeof(double) * m * m);
  k_shifted_block<<<1, 256, 0, h->stream>>>(F, h->d.N, off, m, M);
  k_jacobi_svd<<<1, 1024, 0, h->stream>>>(M, B, J, V, lam, Vt, m, m);
  h->launches += 2;
  cudaStreamSynchronize(h->stream);
  cudaFree(Vt);
}

esmp2_status check_cuda(esmp2_handle *h, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return ESMP2_OK;
  h->err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? ESMP2_ERR_OOM : ESMP2_ERR_CUDA;
}

esmp2_status setup_top_basis(esmp2_handle *h) {
  const int No = h->d.No, Nv = h->d.Nv, N = h->d.N;
  cudaStream_t st = h->stream;
  double *work = nullptr, *Jm = nullptr, *A = nullptr, *R = nullptr, *ww = nullptr, *E = nullptr, *T1 = nullptr;
  const size_t wbytes = sizeof(double) * (size_t)No * Nv;
  cudaError_t ce = cudaSuccess;
  if ((ce = cudaMalloc(&work, wbytes)) != cudaSuccess) return check_cuda(h, ce, "setup alloc");
  cudaMalloc(&Jm, sizeof(double) * No * No);
  cudaMalloc(&A, wbytes);
  cudaMalloc(&R, wbytes);
  cudaMalloc(&ww, sizeof(double) * No);
  cudaMalloc(&E, sizeof(double) * (size_t)(Nv - No + 1) * Nv);
  cudaMalloc(&T1, sizeof(double) * (size_t)N * N);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return check_cuda(h, ce, "setup alloc");

  k_normalise<<<1, 1024, 0, st>>>(h->C, h->C, No * Nv);
  k_jacobi_svd<<<1, 1024, 0, st>>>(h->C, work, Jm, h->U, h->lam, h->Wv, No, Nv);
  k_householder<<<1, 1024, 0, st>>>(h->Wv, A, R, ww, No, Nv);
  const int navo = Nv - No;
  if (navo > 0) k_avo<<<(unsigned)cdiv((int64_t)navo * 32, 256), 256, 0, st>>>(R, ww, E, h->Wv, No, Nv);
  k_assemble_W<<<256, 256, 0, st>>>(h->U, h->Wv, h->W, No, Nv);
  h->launches += 4 + (navo > 0);
  // F_TOP = W^T F W
  Gemm64 g{};
  g.alpha = 1.0; g.beta = 0.0; g.batch = 1;
  g.M = N; g.N = N; g.K = N;
  g.A = h->F; g.sAm = N; g.sAk = 1;   // h->F holds the input F here
  g.B = h->W; g.sBk = N; g.sBn = 1;
  g.C = T1; g.sCm = N; g.sCn = 1;
  gemm64(g, st);
  g.A = h->W; g.sAm = 1; g.sAk = N;
  g.B = T1; g.sBk = N; g.sBn = 1;
  g.C = h->F; g.sCm = N; g.sCn = 1;
  gemm64(g, st);
  k_scalars<<<1, 32, 0, st>>>(h->F, h->lam, h->scal, No, Nv);
  h->launches += 3;
  ce = cudaGetLastError();
  cudaStreamSynchronize(st);
  double sc[2];
  cudaMemcpy(sc, h->scal, sizeof(sc), cudaMemcpyDeviceToHost);
  h->omega = sc[0];
  h->E0 = sc[1];
  cudaFree(work); cudaFree(Jm); cudaFree(A); cudaFree(R); cudaFree(ww); cudaFree(E); cudaFree(T1);
  if (ce == cudaSuccess) ce = cudaGetLastError();
  return check_cuda(h, ce, "TOP basis");
}

// Integral transforms + f0 + right-hand side.  ovov_src / ovvv_src are the device inputs
// (read only: the first pass of each transform reads them directly); ovov_in, ooov_in
// and ovvv_in are the handle's work buffers (ooov_in holds a copy of the input, ovvv_in
// No Nv Nv No elements), all consumed.
namespace {
// out[o0][o1][o2][o3] = in[...] with input axis ax[k] running along output axis k
__global__ void k_permute4(const double *in, double *out, int d0, int d1, int d2, int d3, int a0, int a1, int a2,
                           int a3) {
  const int d[4] = {d0, d1, d2, d3}, ax[4] = {a0, a1, a2, a3};
  int64_t st[4];
  st[3] = 1; st[2] = d3; st[1] = (int64_t)d2 * d3; st[0] = (int64_t)d1 * d2 * d3;
  const int D0 = d[ax[0]], D1 = d[ax[1]], D2 = d[ax[2]], D3 = d[ax[3]];
  const int64_t n = (int64_t)D0 * D1 * D2 * D3;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t f = e;
    const int o3 = (int)(f % D3); f /= D3;
    const int o2 = (int)(f % D2); f /= D2;
    const int o1 = (int)(f % D1);
    const int o0 = (int)(f / D1);
    out[e] = in[o0 * st[ax[0]] + o1 * st[ax[1]] + o2 * st[ax[2]] + o3 * st[ax[3]]];
  }
}

void permute4(esmp2_handle *h, const double *in, double *out, const int d[4], int a0, int a1, int a2, int a3) {
  k_permute4<<<1216, 256, 0, h->stream>>>(in, out, d[0], d[1], d[2], d[3], a0, a1, a2, a3);
  h->launches += 1;
}

// v = hi + lo: hi holds the leading 24 significand bits of v (truncated), lo the remaining
// 29 bits rounded to float, so |v - hi - lo| <= 2^-48 |v|.  Integer operations only (one
// integer-to-float conversion): float64 conversions and adds run at the float64 rate,
// which GB300 keeps at a small fraction of the float32 rate.  |v| < 2^-74 (and zero)
// gives (0, 0) up to that bound; |v| >= 2^127 takes the float64 route.
__device__ __forceinline__ float2 split_df(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7FF);  // biased float64 exponent
  if (e < 949) return make_float2(0.f, 0.f);
  if (e > 1150) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
  }
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29));
  // lo = rest * 2^(e - 1075), the power of two a normal float for e >= 949
  const float scale = __uint_as_float(sign | ((unsigned)(e - 948) << 23));
  const float lo = __uint2float_rn((unsigned)(m & 0x1FFFFFFFu)) * scale;
  return make_float2(hi, lo);
}

// Double-float sum (two floats hi + lo per float64 value): Knuth's two-sum, renormalised.
__device__ __forceinline__ void df_add(float &sh, float &sl, float bh, float bl) {
  const float t = sh + bh;
  const float bv = t - sh;
  const float err = (sh - (t - bv)) + (bh - bv);
  const float lo = sl + bl + err;
  sh = t + lo;
  sl = lo - (sh - t);
}

// out[m][n] = sum_k in[m][k] R[k][n] for n < N <= 32 (a tall matrix times a narrow right
// factor): lane n of a warp owns output column n of kXrRows rows at once, so one shared
// load of R[k][n] serves kXrRows products and no cross-lane sum is needed.  The rows are
// staged 32 columns at a time, split into (hi, lo) floats, through a per-warp shared
// buffer while the next 32 columns are in flight.  Double-float accumulation: exact
// leading product and two-sum per term, every 32-term chunk added into the running sum
// with a renormalised double-float add.  The contraction of the last OVVV index with the
// TOP virtuals (No multiply-adds per input element).
constexpr int kXrN = 32, kXrRows = 8, kXrWarps = 16;
size_t xr_df_smem(int K) { return sizeof(float2) * ((size_t)K * kXrN + (size_t)kXrWarps * kXrRows * 32); }
__global__ void __launch_bounds__(kXrWarps * 32) k_xr_df(const double *__restrict__ in, double *__restrict__ out,
                                                         int64_t M, int K, int N, const double *__restrict__ R,
                                                         int64_t ldR) {
  extern __shared__ float2 sm[];
  float2 *sR = sm;  // [K][32] (hi, lo), columns >= N zero
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2 *sx = sm + (size_t)K * kXrN + warp * (kXrRows * 32);  // this warp's [kXrRows][32]
  for (int e = threadIdx.x; e < K * kXrN; e += blockDim.x) {
    const int k = e >> 5, n = e & 31;
    sR[e] = n < N ? split_df(R[(int64_t)k * ldR + n]) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int64_t groups = (M + kXrRows - 1) / kXrRows;
  for (int64_t g = (int64_t)blockIdx.x * kXrWarps + warp; g < groups; g += (int64_t)gridDim.x * kXrWarps) {
    const int64_t m0 = g * kXrRows;
    float sh[kXrRows], sl[kXrRows];
    double nx[kXrRows];
#pragma unroll
    for (int r = 0; r < kXrRows; ++r) {
      sh[r] = 0.f;
      sl[r] = 0.f;
      nx[r] = (m0 + r < M && lane < K) ? in[(m0 + r) * K + lane] : 0.0;
    }
    for (int k0 = 0; k0 < K; k0 += 32) {
      __syncwarp();
#pragma unroll
      for (int r = 0; r < kXrRows; ++r) sx[r * 32 + lane] = split_df(nx[r]);
      __syncwarp();
      if (k0 + 32 < K) {
        const int k = k0 + 32 + lane;
#pragma unroll
        for (int r = 0; r < kXrRows; ++r) nx[r] = (m0 + r < M && k < K) ? in[(m0 + r) * K + k] : 0.0;
      }
      const int kn = min(32, K - k0);
      float ah[kXrRows], al[kXrRows];
#pragma unroll
      for (int r = 0; r < kXrRows; ++r) { ah[r] = 0.f; al[r] = 0.f; }
#pragma unroll 2
      for (int kk = 0; kk < kn; ++kk) {
        const float2 rv = sR[(k0 + kk) * 32 + lane];
#pragma unroll
        for (int r = 0; r < kXrRows; ++r) {
          const float2 xv = sx[r * 32 + kk];  // broadcast
          const float ph = xv.x * rv.x;
          const float pe = fmaf(xv.x, rv.x, -ph) + fmaf(xv.x, rv.y, xv.y * rv.x);
          const float t = ah[r] + ph;
          const float bv = t - ah[r];
          al[r] += ((ah[r] - (t - bv)) + (ph - bv)) + pe;
          ah[r] = t;
        }
      }
#pragma unroll
      for (int r = 0; r < kXrRows; ++r) df_add(sh[r], sl[r], ah[r], al[r]);
    }
    if (lane < N) {
#pragma unroll
      for (int r = 0; r < kXrRows; ++r)
        if (m0 + r < M) out[(m0 + r) * N + lane] = (double)sh[r] + (double)sl[r];
    }
  }
}
}  // namespace

// The N^5 integral transforms of step a1.  Rotations by the occupied U (No x No) are float64
// GEMMs; rotations by W_v (Nv x Nv) run as X W_v on the tensor cores from exact digit
// products (float64 accuracy), after moving the rotated index last.  The contraction of
// the last OVVV index with the TOP virtuals (Nv -> No columns) stays a float64 GEMM.
esmp2_status setup_rhs_from(esmp2_handle *h, const double *ovov_src, double *ovov_in, double *ooov_in,
                            const double *ovvv_src, double *ovvv_in, double *scratch) {
  const int No = h->d.No, Nv = h->d.Nv;
  cudaStream_t st = h->stream;
  const bool tc = (int64_t)9 * Nv * 1024 < (1LL << 24);   // exact ten-level digit sums (one term)
  esmp2_status s = ESMP2_OK;
  const double *q_ovvt = nullptr;  // (ia|bu') as [i][u][b][a], for the right-hand side
  {
    const int dims[4] = {No, Nv, No, Nv};
    if (tc) {
      mode_product_small(ovov_src, scratch, 1, No, (int64_t)Nv * No * Nv, h->U, st);  // i
      mode_product_small(scratch, ovov_in, (int64_t)No * Nv, No, Nv, h->U, st);       // j
      h->launches += 2;
      if ((s = xwv_split(h, ovov_in, (int64_t)No * Nv * No, scratch))) return s;   // b
      permute4(h, scratch, ovov_in, dims, 0, 2, 3, 1);                              // [i][j][b][a]
      if ((s = xwv_split(h, ovov_in, (int64_t)No * No * Nv, scratch))) return s;   // a
      const int d2[4] = {No, No, Nv, Nv};
      permute4(h, scratch, h->ovov, d2, 0, 3, 1, 2);                                // [i][a][j][b]
    } else {
      if (ovov_src != ovov_in)
        cudaMemcpyAsync(ovov_in, ovov_src, sizeof(double) * h->d.B, cudaMemcpyDeviceToDevice, st);
      double *src = ovov_in, *dst = scratch;
      const double *R[4] = {h->U, h->Wv, h->U, h->Wv};
      const int K[4] = {No, Nv, No, Nv};
      for (int m = 0; m < 4; ++m) {
        mode_product(src, dst, dims, m, R[m], K[m], K[m], st);
        double *t = src; src = dst; dst = t;
      }
      cudaMemcpyAsync(h->ovov, src, sizeof(double) * h->d.B, cudaMemcpyDeviceToDevice, st);
    }
  }
  debug_phase(h, "  ovov transform");
  {
    const int dims[4] = {No, No, No, Nv};
    double *src = ooov_in, *dst = scratch;
    const double *R[4] = {h->U, h->U, h->U, h->Wv};
    const int K[4] = {No, No, No, Nv};
    for (int m = 0; m < 4; ++m) {
      if (m < 3) {
        int64_t P = 1, Q = 1;
        for (int k = 0; k < m; ++k) P *= dims[k];
        for (int k = m + 1; k < 4; ++k) Q *= dims[k];
        mode_product_small(src, dst, P, No, Q, h->U, st);
        h->launches += 1;
      } else {
        mode_product(src, dst, dims, m, R[m], K[m], K[m], st);
      }
      double *t = src; src = dst; dst = t;
    }
    cudaMemcpyAsync(h->ooov, src, sizeof(double) * (size_t)No * No * No * Nv, cudaMemcpyDeviceToDevice, st);
  }
  {
    debug_phase(h, "  ooov transform");
    if (h->ovvv_ready) cudaStreamWaitEvent(st, h->ovvv_ready, 0);   // host OVVV copied on a side stream
    int dims[4] = {No, Nv, Nv, Nv};
    const size_t smem = xr_df_smem(Nv);
    if (No <= kXrN && smem <= 220 * 1024) {  // c -> u' (first No columns of Wv)
      // one limit for every Nv (220 KB): set once per device, never lowered under a running launch
      if (cudaError_t ea = smem_limit_once(reinterpret_cast<const void *>(k_xr_df), 220 * 1024))
        return check_cuda(h, ea, "k_xr_df shared-memory limit");
      const int64_t M = (int64_t)No * Nv * Nv;
      const unsigned grid = (unsigned)std::min<int64_t>(1216, cdiv(cdiv(M, kXrRows), kXrWarps));
      k_xr_df<<<grid, kXrWarps * 32, smem, st>>>(ovvv_src, scratch, M, Nv, No, h->Wv, Nv);
      h->launches += 1;
    } else {
      mode_product(ovvv_src, scratch, dims, 3, h->Wv, No, Nv, st);
    }
    dims[3] = No;
    debug_phase(h, "  ovvv last index -> u'");
    if (tc) {
      mode_product_small(scratch, ovvv_in, 1, No, (int64_t)Nv * Nv * No, h->U, st);  // [i][a][b][u]
      h->launches += 1;
      permute4(h, ovvv_in, scratch, dims, 0, 3, 1, 2);                             // [i][u][a][b]
      if ((s = xwv_split(h, scratch, (int64_t)No * No * Nv, ovvv_in))) return s;  // b
      const int d2[4] = {No, No, Nv, Nv};
      permute4(h, ovvv_in, scratch, d2, 0, 1, 3, 2);                               // [i][u][b][a]
      if ((s = xwv_split(h, scratch, (int64_t)No * No * Nv, ovvv_in))) return s;  // a
      permute4(h, ovvv_in, h->ovvt, d2, 0, 3, 2, 1);                               // [i][a][b][u]
      q_ovvt = ovvv_in;                                                             // [i][u][b][a]
    } else {
      double *src = scratch, *dst = ovvv_in;
      const double *R[3] = {h->U, h->Wv, h->Wv};
      const int K[3] = {No, Nv, Nv};
      for (int m = 0; m < 3; ++m) {
        mode_product(src, dst, dims, m, R[m], K[m], K[m], st);
        double *t = src; src = dst; dst = t;
      }
      cudaMemcpyAsync(h->ovvt, src, sizeof(double) * (size_t)No * Nv * Nv * No, cudaMemcpyDeviceToDevice, st);
      const int d4[4] = {No, Nv, Nv, No};
      permute4(h, h->ovvt, scratch, d4, 0, 3, 2, 1);                               // [i][u][b][a]
      q_ovvt = scratch;
    }
  }
  debug_phase(h, "  ovvt rotations");
  k_f0vo<<<(unsigned)cdiv((int64_t)No * Nv, 256), 256, 0, st>>>(h->F, h->lam, h->ooov, h->ovvt, h->f0vo, No, Nv);
  k_rhs<<<dim3((unsigned)cdiv(Nv, 32), (unsigned)(No * No), 5), 256, 0, st>>>(h->lam, h->f0vo, h->ovov, h->ooov, q_ovvt,
                                                                               h->b, No, Nv);
  h->launches += 2;
  return check_cuda(h, cudaGetLastError(), "rhs");
}

}  // namespace esmp2

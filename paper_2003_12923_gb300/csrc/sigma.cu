// The sigma build y = (H0 - E0) x on D+L, Eq. qfq_replacement restricted to the
// doubles and L-triples.  In the stored block layout the operator splits into
//  (1) the one-body contractions on every free index of every block (the N_o^2 N_v^3
//      and N_o^3 N_v^2 terms of Table 1): for each block
//        y[i][j][a][b] = sum_d F_ad x[i][j][d][b] + sum_d F_bd x[i][j][a][d]
//                      - sum_l F_li x[l][j][a][b] - sum_l F_lj x[i][l][a][b];
//  (2) the N^4 terms that couple blocks through the occupied-virtual Fock block and
//      through moves of the large pair t -> t' (the T3<->T, S3<->S, S3<->T rows of
//      Table 1, and the mixed-spin L-triple cross terms), plus the constant shift
//      -omega and the pair energy F_t't' - F_tt of the L-triples;
//  (3) zeroing of slots that are not amplitudes (Pauli-forbidden or duplicated).
// Part (1) runs as four float64 GEMM passes here (the mixed-precision path replaces
// them with tcgen05 contractions), parts (2)-(3) as one element-wise pass fed by
// small intermediates.
#include "internal.h"

namespace esmp2 {
namespace {

struct Ctx {
  int No, Nv, N;
  int64_t B;
  const double *F;
  double omega;
  int arrow;  // 1: F_oo is diagonal apart from the t row/column (occupied terms done here)
  __device__ __forceinline__ double Fo(int k, int l) const { return F[(int64_t)k * N + l]; }
  __device__ __forceinline__ double Fv(int a, int b) const { return F[(int64_t)(No + a) * N + No + b]; }
  __device__ __forceinline__ double Fov(int k, int a) const { return F[(int64_t)k * N + No + a]; }
  __device__ __forceinline__ int64_t at(int blk, int i, int j, int a, int b) const {
    return blk * B + (((int64_t)i * No + j) * Nv + a) * Nv + b;
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ bool valid_elem(int blk, int i, int j, int a, int b) {
  if ((blk == BT || blk == BX || blk == BY) && (i == j || a == b)) return false;
  if (blk == BX && (i == 0 || j == 0 || a == 0 || b == 0)) return false;
  if (blk == BZ && (j == 0 || b == 0 || (i == 0 && a == 0))) return false;
  return true;
}

template <typename T>
__global__ void k_intermediates(Ctx c, const T *x, Couplings cp) {
  const int No = c.No, Nv = c.Nv;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int64_t warp = tid >> 5, nwarp = nthr >> 5;
  // VX[i][j][b] = sum_c Fov[0][c] X[i][j][c][b]
  for (int64_t e = tid; e < (int64_t)No * No * Nv; e += nthr) {
    const int b = (int)(e % Nv); const int ij = (int)(e / Nv);
    double s = 0.0;
    for (int cc = 0; cc < Nv; ++cc) s += c.Fov(0, cc) * (double)x[c.at(BX, 0, 0, 0, 0) + ((int64_t)ij * Nv + cc) * Nv + b];
    cp.VX[e] = s;
  }
  // OX[j][a][b] = sum_k Fov[k][0] X[k][j][a][b];  OZ[i][a][b] = sum_k Fov[k][0] Z[i][k][a][b]
  for (int64_t e = tid; e < (int64_t)No * Nv * Nv; e += nthr) {
    const int64_t ab = e % ((int64_t)Nv * Nv);
    const int j = (int)(e / ((int64_t)Nv * Nv));
    double s = 0.0, z = 0.0;
    for (int k = 0; k < No; ++k) {
      s += c.Fov(k, 0) * (double)x[c.at(BX, k, j, 0, 0) + ab];
      z += c.Fov(k, 0) * (double)x[c.at(BZ, j, k, 0, 0) + ab];
    }
    cp.OX[e] = s;
    cp.OZ[e] = z;
  }
  // WZ[i][j][a] = sum_c Fov[0][c] Z[i][j][a][c]   (warp per row)
  for (int64_t r = warp; r < (int64_t)No * No * Nv; r += nwarp) {
    const T *row = x + c.at(BZ, 0, 0, 0, 0) + r * Nv;
    double s = 0.0;
    for (int cc = lane; cc < Nv; cc += 32) s += c.Fov(0, cc) * (double)row[cc];
    s = warp_sum(s);
    if (lane == 0) cp.WZ[r] = s;
  }
  // G[j][b] = sum_kc Fov[k][c] (X+Z)[k][j][c][b]
  for (int64_t e = tid; e < (int64_t)No * Nv; e += nthr) {
    const int j = (int)(e / Nv), b = (int)(e % Nv);
    double s = 0.0;
    for (int k = 0; k < No; ++k)
      for (int cc = 0; cc < Nv; ++cc)
        s += c.Fov(k, cc) * ((double)x[c.at(BX, k, j, cc, b)] + (double)x[c.at(BZ, k, j, cc, b)]);
    cp.G[e] = s;
  }
  // H[i][a] = sum_kc Fov[k][c] (Y+Z)[i][k][a][c]   (warp per (i,a))
  for (int64_t r = warp; r < (int64_t)No * Nv; r += nwarp) {
    const int i = (int)(r / Nv), a = (int)(r % Nv);
    double s = 0.0;
    for (int k = 0; k < No; ++k)
      for (int cc = lane; cc < Nv; cc += 32)
        s += c.Fov(k, cc) * ((double)x[c.at(BY, i, k, a, cc)] + (double)x[c.at(BZ, i, k, a, cc)]);
    s = warp_sum(s);
    if (lane == 0) cp.H[r] = s;
  }
  // arrow form of the occupied terms: OC1[blk][j][ab] = sum_{l>=1} Foo[l][0] x[blk][l][j][ab],
  //                                   OC2[blk][i][ab] = sum_{l>=1} Foo[l][0] x[blk][i][l][ab]
  if (c.arrow) {
    const int64_t NvNv = (int64_t)Nv * Nv;
    for (int64_t e = tid; e < 5 * (int64_t)No * NvNv; e += nthr) {
      const int64_t ab = e % NvNv;
      const int64_t r = e / NvNv;
      const int q = (int)(r % No), blk = (int)(r / No);
      double s1 = 0.0, s2 = 0.0;
      for (int l = 1; l < No; ++l) {
        const double f = c.Fo(l, 0);
        s1 += f * (double)x[c.at(blk, l, q, 0, 0) + ab];
        s2 += f * (double)x[c.at(blk, q, l, 0, 0) + ab];
      }
      cp.OC1[e] = s1;
      cp.OC2[e] = s2;
    }
  }
  // CYZ[k][c] = sum_d Fvv[0][d] Z[0][k][d][c] - sum_l Foo[l][0] Z[l][k][0][c]
  for (int64_t e = tid; e < (int64_t)No * Nv; e += nthr) {
    const int k = (int)(e / Nv), cc = (int)(e % Nv);
    double s = 0.0;
    for (int d = 0; d < Nv; ++d) s += c.Fv(0, d) * (double)x[c.at(BZ, 0, k, d, cc)];
    for (int l = 0; l < No; ++l) s -= c.Fo(l, 0) * (double)x[c.at(BZ, l, k, 0, cc)];
    cp.CYZ[e] = s;
  }
}

// y += couplings - omega x (+ pair energy on L blocks); y = 0 on non-amplitude slots.
template <typename TX, typename TY>
__global__ void k_couple(Ctx c, const TX *x, TY *y, Couplings cp) {
  const int No = c.No, Nv = c.Nv;
  const double shift = c.Fv(0, 0) - c.Fo(0, 0);
  const double f00 = c.Fov(0, 0);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t f = e;
    const int b = (int)(f % Nv); f /= Nv;
    const int a = (int)(f % Nv); f /= Nv;
    const int j = (int)(f % No); f /= No;
    const int i = (int)(f % No); f /= No;
    const int blk = (int)f;
    if (!valid_elem(blk, i, j, a, b)) { y[e] = (TY)0; continue; }
    auto X = [&](int bl, int ii, int jj, int aa, int bb) { return (double)x[c.at(bl, ii, jj, aa, bb)]; };
    const double xe = (double)x[e];
    double v = -c.omega * xe;
    const bool i0 = i == 0, j0 = j == 0, a0 = a == 0, b0 = b == 0;
    const int64_t NoNv = (int64_t)No * Nv, NvNv = (int64_t)Nv * Nv;
    if (c.arrow) {  // - sum_l F_li x[l][j] - sum_l F_lj x[i][l] with F_oo diagonal off the t row/column
      const int64_t ab = (int64_t)a * Nv + b;
      v -= (c.Fo(i, i) + c.Fo(j, j)) * xe;
      if (!i0) v -= c.Fo(0, i) * X(blk, 0, j, a, b);
      else v -= cp.OC1[((int64_t)blk * No + j) * NvNv + ab];
      if (!j0) v -= c.Fo(0, j) * X(blk, i, 0, a, b);
      else v -= cp.OC2[((int64_t)blk * No + i) * NvNv + ab];
    }
    switch (blk) {
      case BT: {
        v += f00 * (X(BX, i, j, a, b) + X(BY, i, j, a, b));
        const int64_t ij = ((int64_t)i * No + j) * Nv, ji = ((int64_t)j * No + i) * Nv;
        if (a0) v -= cp.VX[ij + b];
        if (b0) v += cp.VX[ij + a];
        if (i0) v -= cp.OX[j * NvNv + (int64_t)a * Nv + b];
        if (j0) v += cp.OX[i * NvNv + (int64_t)a * Nv + b];
        if (i0 && a0) v += cp.G[j * Nv + b];
        if (j0 && a0) v -= cp.G[i * Nv + b];
        if (i0 && b0) v -= cp.G[j * Nv + a];
        if (j0 && b0) v += cp.G[i * Nv + a];
        (void)ji; (void)NoNv;
        break;
      }
      case BS: {
        if (j0 && b0) v += cp.H[i * Nv + a];
        if (i0 && a0) v += cp.H[j * Nv + b];
        v += f00 * (X(BZ, i, j, a, b) + X(BZ, j, i, b, a));
        if (b0) v -= cp.WZ[((int64_t)i * No + j) * Nv + a];
        if (a0) v -= cp.WZ[((int64_t)j * No + i) * Nv + b];
        if (j0) v -= cp.OZ[i * NvNv + (int64_t)a * Nv + b];
        if (i0) v -= cp.OZ[j * NvNv + (int64_t)b * Nv + a];
        break;
      }
      case BX: {
        v += shift * xe + f00 * X(BT, i, j, a, b);
        v += -c.Fov(0, a) * X(BT, i, j, 0, b) + c.Fov(0, b) * X(BT, i, j, 0, a);
        v += -c.Fov(i, 0) * X(BT, 0, j, a, b) + c.Fov(j, 0) * X(BT, 0, i, a, b);
        v += c.Fov(i, a) * X(BT, 0, j, 0, b) - c.Fov(j, a) * X(BT, 0, i, 0, b)
           - c.Fov(i, b) * X(BT, 0, j, 0, a) + c.Fov(j, b) * X(BT, 0, i, 0, a);
        break;
      }
      case BY: {
        v += shift * xe + f00 * X(BT, i, j, a, b);
        v += c.Fov(j, b) * X(BS, 0, i, 0, a) - c.Fov(i, b) * X(BS, 0, j, 0, a)
           - c.Fov(j, a) * X(BS, 0, i, 0, b) + c.Fov(i, a) * X(BS, 0, j, 0, b);
        if (i0 && a0) v += cp.CYZ[j * Nv + b];
        if (j0 && a0) v -= cp.CYZ[i * Nv + b];
        if (i0 && b0) v -= cp.CYZ[j * Nv + a];
        if (j0 && b0) v += cp.CYZ[i * Nv + a];
        break;
      }
      default: {  // BZ
        v += shift * xe;
        v += f00 * X(BS, i, j, a, b) - c.Fov(0, b) * X(BS, i, j, a, 0) - c.Fov(j, 0) * X(BS, i, 0, a, b)
           + c.Fov(j, b) * X(BS, i, 0, a, 0) + c.Fov(i, a) * X(BT, 0, j, 0, b);
        const double y0 = X(BY, 0, j, 0, b);
        if (i0) v += c.Fv(a, 0) * y0;
        if (a0) v -= c.Fo(0, i) * y0;
        break;
      }
    }
    y[e] = (TY)((double)y[e] + v);
  }
}

}  // namespace

static Ctx make_ctx(const esmp2_handle *h, const double *F, int arrow) {
  Ctx c;
  c.No = h->d.No; c.Nv = h->d.Nv; c.N = h->d.N; c.B = h->d.B;
  c.F = F; c.omega = h->omega; c.arrow = arrow;
  return c;
}

void launch_intermediates64(esmp2_handle *h, const double *F, int arrow, const double *x) {
  k_intermediates<double><<<1216, 256, 0, h->stream>>>(make_ctx(h, F, arrow), x, h->cp);
  h->launches += 1;
}

void launch_couple64(esmp2_handle *h, const double *F, int arrow, const double *x, double *y) {
  k_couple<double, double><<<1216, 256, 0, h->stream>>>(make_ctx(h, F, arrow), x, y, h->cp);
  h->launches += 1;
}

// fp32 coupling + arrow occupied pass of the inner (low-precision) sigma
void couple32(esmp2_handle *h, const double *F, const float *x, float *y) {
  k_intermediates<float><<<1216, 256, 0, h->stream>>>(make_ctx(h, F, 1), x, h->cp);
  k_couple<float, float><<<1216, 256, 0, h->stream>>>(make_ctx(h, F, 1), x, y, h->cp);
  h->launches += 2;
}

// Part (1) in float64: four strided batched GEMM passes over all five blocks.
// stage 1: the two virtual-index passes (N_o^2 N_v^3); stage 2: the two occupied-index passes.
void contractions64(esmp2_handle *h, const double *F, const double *x, double *y, int stage = 3) {
  const int No = h->d.No, Nv = h->d.Nv, N = h->d.N;
  const int64_t B = h->d.B, NvNv = (int64_t)Nv * Nv;
  const double *Fv = F + (int64_t)No * N + No;
  const double *Fo = F;
  Gemm64 g{};
  if (stage & 1) {
  // y[r][b] = sum_d x[r][d] Fv[d][b], r = (blk,i,j,a)
  g = Gemm64{};
  g.M = (int)(5 * (int64_t)No * No * Nv); g.N = Nv; g.K = Nv; g.batch = 1; g.alpha = 1.0; g.beta = 0.0;
  g.A = x; g.sAm = Nv; g.sAk = 1;
  g.B = Fv; g.sBk = N; g.sBn = 1;
  g.C = y; g.sCm = Nv; g.sCn = 1;
  gemm64(g, h->stream);
  // y_s[a][b] += sum_d Fv[a][d] x_s[d][b], s = (blk,i,j)
  g = Gemm64{};
  g.M = Nv; g.N = Nv; g.K = Nv; g.batch = 5 * No * No; g.alpha = 1.0; g.beta = 1.0;
  g.A = Fv; g.sAm = N; g.sAk = 1; g.sAb = 0;
  g.B = x; g.sBk = Nv; g.sBn = 1; g.sBb = NvNv;
  g.C = y; g.sCm = Nv; g.sCn = 1; g.sCb = NvNv;
  gemm64(g, h->stream);
  h->launches += 2;
  }
  if (!(stage & 2)) return;
  // y[blk][i][(j a b)] -= sum_l Fo[l][i] x[blk][l][(j a b)]
  g = Gemm64{};
  g.M = No; g.N = (int)((int64_t)No * NvNv); g.K = No; g.batch = 5; g.alpha = -1.0; g.beta = 1.0;
  g.A = Fo; g.sAm = 1; g.sAk = N; g.sAb = 0;
  g.B = x; g.sBk = (int64_t)No * NvNv; g.sBn = 1; g.sBb = B;
  g.C = y; g.sCm = (int64_t)No * NvNv; g.sCn = 1; g.sCb = B;
  gemm64(g, h->stream);
  // y[blk][i][j][(a b)] -= sum_l Fo[l][j] x[blk][i][l][(a b)]
  g = Gemm64{};
  g.M = No; g.N = (int)NvNv; g.K = No; g.batch = 5 * No; g.alpha = -1.0; g.beta = 1.0;
  g.A = Fo; g.sAm = 1; g.sAk = N; g.sAb = 0;
  g.B = x; g.sBk = NvNv; g.sBn = 1; g.sBb = (int64_t)No * NvNv;
  g.C = y; g.sCm = NvNv; g.sCn = 1; g.sCb = (int64_t)No * NvNv;
  gemm64(g, h->stream);
  h->launches += 2;
}

// Per-stage timing of `reps` float64 sigma builds (CUDA events on the handle's stream):
// ms[0] virtual-index GEMMs, ms[1] occupied-index GEMMs, ms[2] coupling intermediates,
// ms[3] element-wise coupling pass, ms[4] whole sigma.
esmp2_status profile64(esmp2_handle *h, const double *x, double *y, int reps, double *ms) {
  cudaEvent_t ev[5];
  for (auto &e : ev) cudaEventCreate(&e);
  double acc[5] = {0, 0, 0, 0, 0};
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(ev[0], h->stream);
    contractions64(h, h->F, x, y, 1);
    cudaEventRecord(ev[1], h->stream);
    contractions64(h, h->F, x, y, 2);
    cudaEventRecord(ev[2], h->stream);
    launch_intermediates64(h, h->F, 0, x);
    cudaEventRecord(ev[3], h->stream);
    launch_couple64(h, h->F, 0, x, y);
    cudaEventRecord(ev[4], h->stream);
    cudaEventSynchronize(ev[4]);
    for (int k = 0; k < 4; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      acc[k] += t;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[0], ev[4]);
    acc[4] += t;
  }
  for (int k = 0; k < 5; ++k) ms[k] = acc[k] / reps;
  for (auto &e : ev) cudaEventDestroy(e);
  return check_cuda(h, cudaGetLastError(), "profile64");
}

// float64 sigma with an arbitrary orthonormal-basis Fock matrix F (t = occupied 0, t' =
// virtual 0).  arrow = 1 when F_oo is diagonal apart from its t row and column: then the
// occupied-index terms are applied element-wise instead of by GEMM.
esmp2_status sigma64_F(esmp2_handle *h, const double *F, int arrow, const double *x, double *y) {
  contractions64(h, F, x, y, arrow ? 1 : 3);
  launch_intermediates64(h, F, arrow, x);
  launch_couple64(h, F, arrow, x, y);
  return check_cuda(h, cudaGetLastError(), "sigma64");
}

esmp2_status sigma64(esmp2_handle *h, const double *x, double *y) { return sigma64_F(h, h->F, 0, x, y); }

// parts (2)-(3) only: couplings, shift and masks added to y
esmp2_status sigma64_tail(esmp2_handle *h, const double *F, int arrow, const double *x, double *y) {
  launch_intermediates64(h, F, arrow, x);
  launch_couple64(h, F, arrow, x, y);
  return check_cuda(h, cudaGetLastError(), "sigma64 tail");
}

}  // namespace esmp2

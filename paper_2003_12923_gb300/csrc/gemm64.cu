// Float64 strided batched GEMM and 4-index mode products.
//
// GB300 executes float64 on the CUDA cores at a small fraction of its bf16 tensor
// rate, so every float64 contraction here is DFMA-bound even at modest arithmetic
// intensity: a 64x64 shared-memory tile with a 4x4 register block per thread keeps
// the DFMA pipe fed while global loads stay coalesced along the contiguous axis.
#include <algorithm>

#include "internal.h"

namespace esmp2 {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__global__ void __launch_bounds__(NT) gemm64_kernel(Gemm64 g, int mtiles) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t tile = blockIdx.x;
  const int m0 = (int)(tile % mtiles) * BM;
  const int n0 = (int)(tile / mtiles) * BN;
  const int64_t bz = blockIdx.y;
  const double *A = g.A + bz * g.sAb;
  const double *B = g.B + bz * g.sBb;
  double *C = g.C + bz * g.sCb;
  const bool a_kfast = (g.sAk == 1);
  const bool b_nfast = (g.sBn == 1) || (g.sBk != 1);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
      const int idx = tid + NT * r;
      int m, k;
      if (a_kfast) { k = idx % BK; m = idx / BK; } else { m = idx % BM; k = idx / BM; }
      const int gm = m0 + m, gk = k0 + k;
      int64_t ko = (int64_t)gk * g.sAk;
      if (g.Kin > 0) ko = (int64_t)(gk / g.Kin) * g.sAk1 + (int64_t)(gk % g.Kin) * g.sAk;
      As[k][m] = (gm < g.M && gk < g.K) ? A[(int64_t)gm * g.sAm + ko] : 0.0;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
      const int idx = tid + NT * r;
      int n, k;
      if (b_nfast) { n = idx % BN; k = idx / BN; } else { k = idx % BK; n = idx / BK; }
      const int gn = n0 + n, gk = k0 + k;
      int64_t ko = (int64_t)gk * g.sBk;
      if (g.Kin > 0) ko = (int64_t)(gk / g.Kin) * g.sBk1 + (int64_t)(gk % g.Kin) * g.sBk;
      Bs[k][n] = (gn < g.N && gk < g.K) ? B[ko + (int64_t)gn * g.sBn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= g.N) continue;
      double *c = C + (int64_t)gm * g.sCm + (int64_t)gn * g.sCn;
      *c = (g.beta == 0.0) ? g.alpha * acc[i][j] : fma(g.alpha, acc[i][j], g.beta * *c);
    }
  }
}

}  // namespace

void gemm64(const Gemm64 &g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  const int mtiles = (int)cdiv(g.M, BM);
  const int64_t tiles = (int64_t)mtiles * cdiv(g.N, BN);
  const double flops = 2.0 * g.M * (double)g.N * g.K * g.batch;
  KScope ks(st, ESMP2_KT_GEMM64, flops, flops);
  for (int b0 = 0; b0 < g.batch; b0 += 65535) {
    Gemm64 gg = g;
    gg.batch = std::min(65535, g.batch - b0);
    gg.A = g.A + (int64_t)b0 * g.sAb;
    gg.B = g.B + (int64_t)b0 * g.sBb;
    gg.C = g.C + (int64_t)b0 * g.sCb;
    dim3 grid((unsigned)tiles, (unsigned)gg.batch);
    gemm64_kernel<<<grid, NT, 0, st>>>(gg, mtiles);
  }
}

void mode_product(const double *in, double *out, const int dims[4], int mode, const double *R,
                  int Kout, int64_t ldR, cudaStream_t st) {
  int64_t P = 1, Q = 1;
  for (int k = 0; k < mode; ++k) P *= dims[k];
  for (int k = mode + 1; k < 4; ++k) Q *= dims[k];
  const int Kin = dims[mode];
  Gemm64 g{};
  g.alpha = 1.0; g.beta = 0.0;
  if (Q == 1) {  // out[p][k'] = sum_k in[p][k] R[k][k']
    g.M = (int)P; g.N = Kout; g.K = Kin; g.batch = 1;
    g.A = in; g.sAm = Kin; g.sAk = 1; g.sAb = 0;
    g.B = R; g.sBk = ldR; g.sBn = 1; g.sBb = 0;
    g.C = out; g.sCm = Kout; g.sCn = 1; g.sCb = 0;
  } else {       // out_p[k'][q] = sum_k R[k][k'] in_p[k][q]
    g.M = Kout; g.N = (int)Q; g.K = Kin; g.batch = (int)P;
    g.A = R; g.sAm = 1; g.sAk = ldR; g.sAb = 0;
    g.B = in; g.sBk = Q; g.sBn = 1; g.sBb = (int64_t)Kin * Q;
    g.C = out; g.sCm = Q; g.sCn = 1; g.sCb = (int64_t)Kout * Q;
  }
  gemm64(g, st);
}

}  // namespace esmp2

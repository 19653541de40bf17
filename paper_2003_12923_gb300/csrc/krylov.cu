// Krylov solve of the first-order equation (H0 - E0) x = -b on D+L and the E2 reductions.
//
// Preconditioned conjugate gradients (the paper's solver is CG, Sec. III.A) with the
// Jacobi preconditioner diag(A) = F_aa + F_bb - F_ii - F_jj - omega (+ F_t't' - F_tt on
// the L blocks).  Inner products are the determinant-space ones (block weights).  All
// vector updates are fused streaming kernels; every reduction is a deterministic
// two-level float64 sum (per-CTA partials, then one CTA in fixed order).
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace esmp2 {

constexpr int kRedBlocks = 1216;  // 152 SMs x 8
constexpr int kRedThreads = 256;

namespace {

struct VCtx {
  int No, Nv, N;
  int64_t B;
  const double *F;
  double omega;
  __device__ __forceinline__ double dinv(int64_t e) const {
    int64_t f = e;
    const int b = (int)(f % Nv); f /= Nv;
    const int a = (int)(f % Nv); f /= Nv;
    const int j = (int)(f % No); f /= No;
    const int i = (int)(f % No); f /= No;
    const int blk = (int)f;
    if ((blk == BT || blk == BX || blk == BY) && (i == j || a == b)) return 0.0;
    if (blk == BX && (i == 0 || j == 0 || a == 0 || b == 0)) return 0.0;
    if (blk == BZ && (j == 0 || b == 0 || (i == 0 && a == 0))) return 0.0;
    double d = F[(int64_t)(No + a) * N + No + a] + F[(int64_t)(No + b) * N + No + b] - F[(int64_t)i * N + i] -
               F[(int64_t)j * N + j] - omega;
    if (blk >= BX) d += F[(int64_t)No * N + No] - F[0];
    return 1.0 / d;
  }
  __device__ __forceinline__ double w(int64_t e) const {
    const int blk = (int)(e / B);
    return blk == 1 ? 1.0 : (blk == 4 ? 2.0 : 0.5);
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce NQ values and store them as partials red[q * gridDim.x + blockIdx.x].
template <int NQ>
__device__ __forceinline__ void block_partials(double (&v)[NQ], double *red) {
  __shared__ double sh[NQ][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double s = warp_sum(v[q]);
    if (lane == 0) sh[q][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = lane < (int)(blockDim.x >> 5) ? sh[q][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) red[(int64_t)q * gridDim.x + blockIdx.x] = s;
    }
  }
}

// Sum the partials of nq quantities in fixed order; mode selects the scalar bookkeeping.
// slots: 0 rz, 1 rr, 2 bb, 3 pq, 4 alpha, 5 beta, 8.. generic results (slots 4, 5 of a zeroed
// slot array give alpha = beta = 0)
__global__ void k_finalize(const double *red, int nparts, int nq, double *slots, int mode) {
  __shared__ double sh[32];
  for (int q = 0; q < nq; ++q) {
    double s = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) s += red[(int64_t)q * nparts + k];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
      if (mode == 0) {            // init: rz, rr, bb
        slots[q] = t;
      } else if (mode == 1) {     // pq -> alpha (no step along a direction of non-positive curvature)
        slots[3] = t;
        slots[4] = t > 0.0 ? slots[0] / t : 0.0;
      } else if (mode == 2) {     // rz_new, rr -> beta
        if (q == 0) { slots[5] = t / slots[0]; slots[0] = t; }
        else slots[1] = t;
      } else if (mode == 5) {     // rr alone
        slots[1] = t;
      } else if (mode == 6) {     // rz_new alone -> beta
        slots[5] = t / slots[0];
        slots[0] = t;
      } else if (mode == 7) {     // rz alone (start)
        slots[0] = t;
      } else {                    // generic
        slots[8 + q] = t;
      }
    }
    __syncthreads();
  }
}

// r = -b - q; p = M^-1 r; partials <r,M^-1 r>, <r,r>, <b,b>
__global__ void k_pcg_init(VCtx c, const double *b, const double *q, double *r, double *p, double *red) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x) {
    const double ri = -b[e] - q[e], z = c.dinv(e) * ri, w = c.w(e);
    r[e] = ri;
    p[e] = z;
    v[0] += w * ri * z;
    v[1] += w * ri * ri;
    v[2] += w * b[e] * b[e];
  }
  block_partials<3>(v, red);
}

__global__ void k_dot_w(VCtx c, const double *u, const double *v_, double *red) {
  double v[1] = {0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x)
    v[0] += c.w(e) * u[e] * v_[e];
  block_partials<1>(v, red);
}

// x += alpha p; r -= alpha q; partials <r,M^-1 r>, <r,r>
__global__ void k_pcg_update(VCtx c, const double *slots, double *x, double *r, const double *p, const double *q,
                             double *red) {
  const double alpha = slots[4];
  double v[2] = {0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x) {
    x[e] += alpha * p[e];
    const double ri = r[e] - alpha * q[e];
    r[e] = ri;
    const double w = c.w(e);
    v[0] += w * ri * c.dinv(e) * ri;
    v[1] += w * ri * ri;
  }
  block_partials<2>(v, red);
}

// p = M^-1 r + beta p
__global__ void k_pcg_p(VCtx c, const double *slots, const double *r, double *p) {
  const double beta = slots[5];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x)
    p[e] = c.dinv(e) * r[e] + beta * p[e];
}

// ---- low-precision inner PCG (vectors of type T, float64 reductions)
// r = r64 (the fp64 outer residual); d = 0; p = M^-1 r; partials <r,M^-1 r>, <r,r>
template <typename T>
__global__ void kt_init(VCtx c, const double *r64, T *r, T *p, T *d, double *red) {
  double v[2] = {0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x) {
    const T ri = (T)r64[e];
    const double z = c.dinv(e) * (double)ri, w = c.w(e);
    r[e] = ri;
    p[e] = (T)z;
    d[e] = (T)0;
    v[0] += w * (double)ri * z;
    v[1] += w * (double)ri * (double)ri;
  }
  block_partials<2>(v, red);
}

template <typename T>
__global__ void kt_dot(VCtx c, const T *u, const T *v_, double *red) {
  double v[1] = {0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x)
    v[0] += c.w(e) * (double)u[e] * (double)v_[e];
  block_partials<1>(v, red);
}

template <typename T>
__global__ void kt_update(VCtx c, const double *slots, T *d, T *r, const T *p, const T *q, double *red) {
  const double alpha = slots[4];
  double v[2] = {0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x) {
    d[e] = (T)((double)d[e] + alpha * (double)p[e]);
    const double ri = (double)r[e] - alpha * (double)q[e];
    r[e] = (T)ri;
    const double w = c.w(e);
    v[0] += w * ri * c.dinv(e) * ri;
    v[1] += w * ri * ri;
  }
  block_partials<2>(v, red);
}

template <typename T>
__global__ void kt_p(VCtx c, const double *slots, const T *r, T *p) {
  const double beta = slots[5];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x)
    p[e] = (T)(c.dinv(e) * (double)r[e] + beta * (double)p[e]);
}

// ---- float inner PCG: block-by-block streaming, float arithmetic, the Jacobi preconditioner
// read from a half-precision vector (a fixed diagonal SPD preconditioner: rounding it only
// perturbs the preconditioner), per-thread float partial sums combined in float64.  With
// B a multiple of 4 every block starts on a 16-byte boundary and the streams move four
// elements per access.  The correction d is advanced in the p update (d += alpha p before p
// changes), so the residual update reads only r, q and M^-1.
struct ICtx {
  int64_t off[6];     // first element of each block (T, S, X, Y, Z) and the vector length
  float w[5];         // determinant inner-product weight of each block's elements
  const __half *dinv;
  __nv_bfloat16 *pb;  // bf16 copy of p for the tensor-core operand (nullptr: not kept here)
  int vec;            // every block starts on a 16-byte boundary
};
__device__ __forceinline__ float4 ld_h4(const __half *p4) {
  const uint2 u = *reinterpret_cast<const uint2 *>(p4);
  const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_b4(__nv_bfloat16 *p4, float4 v) {
  __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
  uint2 u;
  u.x = *reinterpret_cast<uint32_t *>(&a);
  u.y = *reinterpret_cast<uint32_t *>(&b);
  *reinterpret_cast<uint2 *>(p4) = u;
}

__global__ void ki_init(ICtx c, const double *r64, float *r, float *p, float *d, double *red) {
  float a0 = 0.f, a1 = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int blk = 0; blk < 5; ++blk) {
    const float w = c.w[blk];
    float s0 = 0.f, s1 = 0.f;
    for (int64_t e = c.off[blk] + t0; e < c.off[blk + 1]; e += stride) {
      const float ri = (float)r64[e], z = __half2float(c.dinv[e]) * ri;
      r[e] = ri;
      p[e] = z;
      if (c.pb) c.pb[e] = __float2bfloat16_rn(z);
      d[e] = 0.f;
      s0 += ri * z;
      s1 += ri * ri;
    }
    a0 += w * s0;
    a1 += w * s1;
  }
  double v[2] = {(double)a0, (double)a1};
  block_partials<2>(v, red);
}

// r -= alpha q; partials <r, M^-1 r>, <r, r>
__global__ void ki_update(ICtx c, const double *slots, float *r, const float *q, double *red) {
  const float alpha = (float)slots[4];
  float a0 = 0.f, a1 = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int blk = 0; blk < 5; ++blk) {
    float s0 = 0.f, s1 = 0.f;
    if (c.vec) {
      const int64_t n4 = (c.off[blk + 1] - c.off[blk]) >> 2;
      float4 *r4 = reinterpret_cast<float4 *>(r + c.off[blk]);
      const float4 *q4 = reinterpret_cast<const float4 *>(q + c.off[blk]);
      const __half *dv = c.dinv + c.off[blk];
      for (int64_t e = t0; e < n4; e += stride) {
        float4 rv = r4[e];
        const float4 qv = q4[e], m = ld_h4(dv + 4 * e);
        rv.x -= alpha * qv.x; rv.y -= alpha * qv.y; rv.z -= alpha * qv.z; rv.w -= alpha * qv.w;
        r4[e] = rv;
        s0 += rv.x * m.x * rv.x + rv.y * m.y * rv.y + rv.z * m.z * rv.z + rv.w * m.w * rv.w;
        s1 += rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
      }
    } else {
      for (int64_t e = c.off[blk] + t0; e < c.off[blk + 1]; e += stride) {
        const float ri = r[e] - alpha * q[e];
        r[e] = ri;
        s0 += ri * __half2float(c.dinv[e]) * ri;
        s1 += ri * ri;
      }
    }
    const float w = c.w[blk];
    a0 += w * s0;
    a1 += w * s1;
  }
  double v[2] = {(double)a0, (double)a1};
  block_partials<2>(v, red);
}

// d += alpha p; p = M^-1 r + beta p (and its bf16 copy)
__global__ void ki_p(ICtx c, const double *slots, const float *r, float *p, float *d) {
  const float alpha = (float)slots[4], beta = (float)slots[5];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c.vec) {
    const int64_t n4 = c.off[5] >> 2;
    const float4 *r4 = reinterpret_cast<const float4 *>(r);
    float4 *p4 = reinterpret_cast<float4 *>(p), *d4 = reinterpret_cast<float4 *>(d);
    for (int64_t e = t0; e < n4; e += stride) {
      const float4 pv = p4[e], rv = r4[e], m = ld_h4(c.dinv + 4 * e);
      float4 dv = d4[e];
      dv.x += alpha * pv.x; dv.y += alpha * pv.y; dv.z += alpha * pv.z; dv.w += alpha * pv.w;
      d4[e] = dv;
      const float4 pn = make_float4(m.x * rv.x + beta * pv.x, m.y * rv.y + beta * pv.y, m.z * rv.z + beta * pv.z,
                                    m.w * rv.w + beta * pv.w);
      p4[e] = pn;
      if (c.pb) st_b4(c.pb + 4 * e, pn);
    }
  } else {
    for (int64_t e = t0; e < c.off[5]; e += stride) {
      const float pv = p[e];
      d[e] += alpha * pv;
      const float pn = __half2float(c.dinv[e]) * r[e] + beta * pv;
      p[e] = pn;
      if (c.pb) c.pb[e] = __float2bfloat16_rn(pn);
    }
  }
}

// Jacobi preconditioner as a half vector (once per basis): one CTA iteration per row
// (blk, i, j, a), float arithmetic (the value is stored in half precision anyway)
__global__ void k_dinv32(VCtx c, __half *dinv) {
  const int No = c.No, Nv = c.Nv, N = c.N;
  const int64_t rows = 5LL * No * No * Nv;
  const float shift = (float)(c.F[(int64_t)No * N + No] - c.F[0]), om = (float)c.omega;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    int64_t f = row;
    const int a = (int)(f % Nv); f /= Nv;
    const int j = (int)(f % No); f /= No;
    const int i = (int)(f % No);
    const int blk = (int)(f / No);
    const float base = (float)c.F[(int64_t)(No + a) * N + No + a] - (float)c.F[(int64_t)i * N + i] -
                       (float)c.F[(int64_t)j * N + j] - om + (blk >= BX ? shift : 0.f);
    __half *out = dinv + row * Nv;
    for (int b = threadIdx.x; b < Nv; b += blockDim.x) {
      bool zero = false;
      if ((blk == BT || blk == BX || blk == BY) && (i == j || a == b)) zero = true;
      if (blk == BX && (i == 0 || j == 0 || a == 0 || b == 0)) zero = true;
      if (blk == BZ && (j == 0 || b == 0 || (i == 0 && a == 0))) zero = true;
      const float d = base + (float)c.F[(int64_t)(No + b) * N + No + b];
      out[b] = __float2half_rn(zero ? 0.f : 1.f / d);
    }
  }
}

// r = -b - q (fp64 true residual); partials <r,r>, <b,b>
// r = -b - q (q == nullptr: q = 0); partials <r, r>_w and, with with_b, <b, b>_w.  Block by
// block (no per-element index arithmetic), weights applied to the block sums: float64 runs
// at a small fraction of the float32 rate on GB300, so the pass keeps to one add and one or
// two fused multiply-adds per element.
__global__ void k_residual(VCtx c, const double *b, const double *q, double *r, double *red, int with_b) {
  double v[2] = {0.0, 0.0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x, t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int blk = 0; blk < 5; ++blk) {
    double s0 = 0.0, s1 = 0.0;
    for (int64_t e = blk * c.B + t0; e < (blk + 1) * c.B; e += stride) {
      const double bi = b[e], ri = q ? -bi - q[e] : -bi;
      r[e] = ri;
      s0 = fma(ri, ri, s0);
      if (with_b) s1 = fma(bi, bi, s1);
    }
    const double w = blk == 1 ? 1.0 : (blk == 4 ? 2.0 : 0.5);
    v[0] += w * s0;
    v[1] += w * s1;
  }
  block_partials<2>(v, red);
}

template <typename T>
__global__ void kt_accumulate(VCtx c, double *x, const T *d) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x)
    x[e] += (double)d[e];
}

// per-block <b,x> and <x,Ax> for the Hylleraas functional (10 partial sums); q = A x, or
// from_r: q = -b - r with r the true residual of the current x
__global__ void k_hylleraas(VCtx c, const double *b, const double *x, const double *q, int from_r, double *red) {
  double v[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) v[k] = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x) {
    const int blk = (int)(e / c.B);
    const double qe = from_r ? -b[e] - q[e] : q[e];
    const double xb = x[e] * b[e], xq = x[e] * qe;
#pragma unroll
    for (int k = 0; k < 5; ++k)
      if (k == blk) { v[2 * k] += xb; v[2 * k + 1] += xq; }
  }
  block_partials<10>(v, red);
}

// ---- S-space energy: E2_S = -sum_{I in S} b_I^2 / D_I, both spin sectors (factor 2).
struct SCtx {
  int No, Nv, N;
  const double *F, *lam, *ovov;
  double omega;
  __device__ __forceinline__ double Fo(int k) const { return F[(int64_t)k * N + k]; }
  __device__ __forceinline__ double Fv(int a) const { return F[(int64_t)(No + a) * N + No + a]; }
  __device__ __forceinline__ double g(int i, int a, int j, int b) const {  // (ia|jb)
    return ovov[(((int64_t)i * Nv + a) * No + j) * Nv + b];
  }
  // b of a triple: P(k/ij)P(c/ab) [<ab||ij> s_kc] with s_kc = lam_k when c is k's TOP partner.
  __device__ double b3(const int *ho, const int *hs, const int *po, const int *ps) const {
    const int PERM[3][3] = {{0, 1, 2}, {2, 1, 0}, {0, 2, 1}};
    const int PS[3] = {1, -1, -1};
    double v = 0.0;
    for (int t = 0; t < 3; ++t)
      for (int r = 0; r < 3; ++r) {
        const int h3 = PERM[t][2], p3 = PERM[r][2];
        if (hs[h3] != ps[p3] || ho[h3] != po[p3]) continue;
        const int H0 = PERM[t][0], H1 = PERM[t][1], P0 = PERM[r][0], P1 = PERM[r][1];
        double a = 0.0;
        if (ps[P0] == hs[H0] && ps[P1] == hs[H1]) a += g(ho[H0], po[P0], ho[H1], po[P1]);
        if (ps[P0] == hs[H1] && ps[P1] == hs[H0]) a -= g(ho[H1], po[P0], ho[H0], po[P1]);
        v += PS[t] * PS[r] * lam[ho[h3]] * a;
      }
    return v;
  }
  __device__ double term(const int *ho, const int *hs, const int *po, const int *ps) const {
    const double bI = b3(ho, hs, po, ps);
    const double D = Fv(po[0]) + Fv(po[1]) + Fv(po[2]) - Fo(ho[0]) - Fo(ho[1]) - Fo(ho[2]) - omega;
    return -2.0 * bI * bI / D;
  }
};

// In every sector the common case holds exactly one TOP pair (u, u'); then b_I is a single
// antisymmetrised integral times lam_u and the term is evaluated inline.  Triples whose
// other indices form a second TOP pair take the general P(k/ij)P(c/ab) form (s.term, in
// float64).  The inline terms run in double-float arithmetic (value = hi + lo, two floats;
// Dekker products, Knuth sums, one Newton-corrected quotient; about 2^-46 relative), which
// moves the S-space sum from the float64 pipe to the float32 pipes: the integrals are kept
// as (hi, lo) pairs (esmp2 keeps one copy per handle) and the orbital energies as pairs in
// shared memory.
struct dflt {
  float h, l;
};
__device__ __forceinline__ dflt df_of(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
  const float s = a.h + b.h, bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  const float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ dflt df_neg(dflt a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dflt df_mul(dflt a, dflt b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e += a.h * b.l + a.l * b.h;
  const float h = p + e;
  return {h, e - (h - p)};
}
__device__ __forceinline__ dflt df_div(dflt a, dflt b) {
  const float q1 = a.h / b.h;
  // remainder a - q1 b with the leading product exact
  const float p = q1 * b.h;
  const float pe = fmaf(q1, b.h, -p);
  const float r = ((a.h - p) - pe) + (a.l - q1 * b.l);
  const float q2 = r / b.h;
  const float h = q1 + q2;
  return {h, q2 - (h - q1)};
}
__device__ __forceinline__ double df_to_double(dflt a) { return (double)a.h + (double)a.l; }

// integrals as (hi, lo) pairs: same index as SCtx::g
__global__ void k_ovov_df(const double *g, float2 *gdf, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = g[e];
    const float h = (float)v;
    gdf[e] = make_float2(h, (float)(v - (double)h));
  }
}

struct SDf {
  const float2 *g;  // (ia|jb) pairs
  __device__ __forceinline__ dflt at(int No, int Nv, int i, int a, int j, int b) const {
    const float2 v = g[(((int64_t)i * Nv + a) * No + j) * Nv + b];
    return {v.x, v.y};
  }
};

// shared-memory copy of the virtual orbital energies F_aa as pairs (Nv <= 4096)
__device__ __forceinline__ void load_fv(const SCtx &s, float2 *fv) {
  for (int a = threadIdx.x; a < s.Nv; a += blockDim.x) {
    const dflt d = df_of(s.Fv(a));
    fv[a] = make_float2(d.h, d.l);
  }
  __syncthreads();
}

// shared-memory tables of the sum over the small pair u: lambda_u^2 and F_u'u' - F_uu as
// (hi, lo) pairs (No <= 64, esmp2_create)
__device__ __forceinline__ void load_u(const SCtx &s, float2 *lu2, float2 *du) {
  for (int u = threadIdx.x; u < s.No; u += blockDim.x) {
    const double l = s.lam[u];
    const dflt a = df_of(l * l), d = df_of(s.Fv(u) - s.Fo(u));
    lu2[u] = make_float2(a.h, a.l);
    du[u] = make_float2(d.h, d.l);
  }
}
__device__ __forceinline__ dflt ld(const float2 v) { return {v.x, v.y}; }

// Sectors A and B with exactly one transition pair u >= 1 (the common case).  For an
// occupied pair j < k and a virtual pair b < c outside {j, k} (c >= 1) the triple's right-hand
// side is lambda_u times dg = (kc|jb) - (jc|kb) and its denominator is D_u + e_bc with
// D_u = F_u'u' - F_uu, e_bc = F_bb + F_cc - F_jj - F_kk - omega, for
//   A: up-up-up triples u j k -> u' b c (u not in {j, k}, u' not in {b, c}),
//   B: up-down-down triples with the up pair u -> u' and the down double j k -> b c (any u >= 1),
// so E2_S += -2 dg^2 sum_u lambda_u^2 ([A] + [B]) / (D_u + e_bc): each integral is read once and
// the sum over u runs in registers.  Block = (pair j < k, one of nchunk strided ranges of c),
// threads over b (coalesced rows of the integrals).
__global__ void k_e2s_ab(SCtx s, SDf gd, int nchunk, double *red) {
  __shared__ float2 fv[4096], lu2[64], du[64];   // Nv <= 4096, No <= 64 (esmp2_create)
  const int No = s.No, Nv = s.Nv;
  const int chunk = blockIdx.x % nchunk;
  int kk = blockIdx.x / nchunk, j = 0;
  while (kk >= No - 1 - j) { kk -= No - 1 - j; ++j; }
  const int k = j + 1 + kk;
  load_u(s, lu2, du);
  load_fv(s, fv);   // synchronises
  const dflt base = df_of(-s.Fo(j) - s.Fo(k) - s.omega);
  dflt acc = {0.f, 0.f};
  for (int c = 1 + chunk; c < Nv; c += nchunk) {
    if (c == j || c == k) continue;
    const dflt ec = df_add(base, ld(fv[c]));
    for (int b = threadIdx.x; b < c; b += blockDim.x) {
      if (b == j || b == k) continue;
      const dflt dg = df_add(gd.at(No, Nv, k, c, j, b), df_neg(gd.at(No, Nv, j, c, k, b)));
      const dflt e = df_add(ec, ld(fv[b]));
      dflt sum = {0.f, 0.f};
      for (int u = 1; u < No; ++u) {
        const dflt q = df_div(ld(lu2[u]), df_add(ld(du[u]), e));
        sum = df_add(sum, q);                                              // B
        if (u != j && u != k && u != b && u != c) sum = df_add(sum, q);   // A
      }
      acc = df_add(acc, df_mul(df_mul(dg, dg), sum));
    }
  }
  double v[1] = {-2.0 * df_to_double(acc)};
  block_partials<1>(v, red);
}

// Sector C: up-down-down triples without an up pair, whose one pair is the down pair u -> u'
// (u >= 1, u != k): up single i -> a (a != i), down holes u, k, down particles u', c (c != k,
// c != u').  The right-hand side is lambda_u (ia|kc), the denominator D_u + F_aa + F_cc - F_ii -
// F_kk - omega:  E2_S += -2 (ia|kc)^2 sum_u lambda_u^2 / (D_u + e_ac).  Block = (i, k, one of
// nchunk strided ranges of a), threads over c (coalesced rows of (ia|kc)).
__global__ void k_e2s_cm(SCtx s, SDf gd, int nchunk, double *red) {
  __shared__ float2 fv[4096], lu2[64], du[64];
  const int No = s.No, Nv = s.Nv;
  const int chunk = blockIdx.x % nchunk, ik = blockIdx.x / nchunk, i = ik / No, k = ik % No;
  load_u(s, lu2, du);
  load_fv(s, fv);
  const dflt base = df_of(-s.Fo(i) - s.Fo(k) - s.omega);
  dflt acc = {0.f, 0.f};
  for (int a = chunk; a < Nv; a += nchunk) {
    if (a == i) continue;
    const dflt ea = df_add(base, ld(fv[a]));
    for (int c = threadIdx.x; c < Nv; c += blockDim.x) {
      if (c == k) continue;
      const dflt g = gd.at(No, Nv, i, a, k, c);
      const dflt e = df_add(ea, ld(fv[c]));
      dflt sum = {0.f, 0.f};
      for (int u = 1; u < No; ++u)
        if (u != k && u != c) sum = df_add(sum, df_div(ld(lu2[u]), df_add(ld(du[u]), e)));
      acc = df_add(acc, df_mul(df_mul(g, g), sum));
    }
  }
  double v[1] = {-2.0 * df_to_double(acc)};
  block_partials<1>(v, red);
}

// The triples that hold a second transition pair besides the lowest one u (few: a virtual index
// equal to an occupied index of the triple), in the general float64 form P(k/ij)P(c/ab)
// (s.term).  Block = (u, x, y) for the three sectors' index pairs, work spread over the threads.
__global__ void k_e2s_gen(SCtx s, double *red) {
  const int No = s.No, Nv = s.Nv;
  const int64_t blk = blockIdx.x;
  const int u = (int)(blk / ((int64_t)No * No)), x = (int)((blk / No) % No), y = (int)(blk % No);
  double v[1] = {0.0};
  if (u >= 1) {
    const int j = x, k = y;
    // sector A (up-up-up, pair u lowest): virtual pairs b < c holding j or k
    if (j < k && j != u && k != u) {
      for (int e = threadIdx.x; e < 2 * Nv; e += blockDim.x) {
        const int xx = e < Nv ? j : k, yy = e % Nv;
        if (yy == xx || ((yy == j || yy == k) && xx != j)) continue;  // the pair (j, k) once
        const int b = min(xx, yy), c = max(xx, yy);
        if (c < 1 || c == u || b == u) continue;
        const bool pj = (b == j || c == j), pk = (b == k || c == k);
        if ((pj && j < u) || (pk && k < u)) continue;    // a lower pair owns this triple
        if ((pj && j == 0) || (pk && k == 0)) continue;  // holds the large pair: L space
        const int ho[3] = {u, j, k}, hs[3] = {0, 0, 0}, po[3] = {u, b, c}, ps[3] = {0, 0, 0};
        v[0] += s.term(ho, hs, po, ps);
      }
    }
    // sector B (up pair u, down double j < k): down virtual pairs holding j or k
    if (j < k) {
      for (int e = threadIdx.x; e < 2 * Nv; e += blockDim.x) {
        const int xx = e < Nv ? j : k, yy = e % Nv;
        if (yy == xx || ((yy == j || yy == k) && xx != j)) continue;
        const int b = min(xx, yy), c = max(xx, yy);
        if (c < 1) continue;
        if ((j == 0 || k == 0) && (b == 0 || c == 0)) continue;  // down t-pair: L space
        const int ho[3] = {u, j, k}, hs[3] = {0, 1, 1}, po[3] = {u, b, c}, ps[3] = {0, 1, 1};
        v[0] += s.term(ho, hs, po, ps);
      }
    }
    // sector C (no up pair, lowest down pair u): the down particle c == k (a second down pair)
    const int i = x;
    if (k != u && k >= u && k != 0) {
      for (int a = threadIdx.x; a < Nv; a += blockDim.x) {
        if (a == i) continue;
        const int ho[3] = {i, u, k}, hs[3] = {0, 1, 1}, po[3] = {a, u, k}, ps[3] = {0, 1, 1};
        v[0] += s.term(ho, hs, po, ps);
      }
    }
  }
  block_partials<1>(v, red);
}

// ---- preconditioned MINRES (symmetric, possibly indefinite A; SPD preconditioner
// M^-1 = |diag|^-1 of the reduced-cost basis), vectors in the full-storage float64 layout.
// |1 / d| with the masks (d the Jacobi diagonal of VCtx::dinv)
__device__ __forceinline__ double mr_minv(const VCtx &c, int64_t e) { return fabs(c.dinv(e)); }

// v = M^-1 r / beta
__global__ void k_mr_v(VCtx c, const double *r, double beta_inv, double *v) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x)
    v[e] = mr_minv(c, e) * r[e] * beta_inv;
}
// partials <r, M^-1 r>_w, <r, r>_w
__global__ void k_mr_res(VCtx c, const double *r, double *red) {
  double v[2] = {0.0, 0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[e], w = c.w(e);
    v[0] += w * ri * mr_minv(c, e) * ri;
    v[1] += w * ri * ri;
  }
  block_partials<2>(v, red);
}
// partial <u, v>_w
__global__ void k_mr_dot(VCtx c, const double *u, const double *v_, double *red) {
  double v[1] = {0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x)
    v[0] += c.w(e) * u[e] * v_[e];
  block_partials<1>(v, red);
}
// y = q - a1 r2 - a2 r1 (written over r1); partial <y, M^-1 y>_w
__global__ void k_mr_y(VCtx c, const double *q, const double *r2, double *r1y, double a1, double a2, double *red) {
  double v[1] = {0.0};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x) {
    const double y = q[e] - a1 * r2[e] - a2 * r1y[e];
    r1y[e] = y;
    v[0] += c.w(e) * y * mr_minv(c, e) * y;
  }
  block_partials<1>(v, red);
}
// w1 <- (v - e1 w1 - e2 w2) / gamma (the new direction, over the oldest one); x += phi w1;
// v <- M^-1 y / beta_next
__global__ void k_mr_update(VCtx c, double *v, double *w1, const double *w2, double *x, const double *y, double e1,
                            double e2, double ginv, double phi, double bn_inv) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 5 * c.B; e += (int64_t)gridDim.x * blockDim.x) {
    const double wn = (v[e] - e1 * w1[e] - e2 * w2[e]) * ginv;
    w1[e] = wn;
    x[e] += phi * wn;
    v[e] = mr_minv(c, e) * y[e] * bn_inv;
  }
}
// r = -b - q (q null: r = -b)
__global__ void k_negsum64(const double *b, const double *q, double *out, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = q ? -b[e] - q[e] : -b[e];
}

}  // namespace

void launch_pcg_init(esmp2_handle *h, const double *b, const double *q, double *r, double *p);

// one quantity's partials summed into the slots with the bookkeeping of `mode` (k_finalize)
void k_finalize_ext(const double *red, int nparts, double *slots, int mode, cudaStream_t st) {
  k_finalize<<<1, 256, 0, st>>>(red, nparts, 1, slots, mode);
}

static VCtx vctx(const esmp2_handle *h, const double *F = nullptr) {
  VCtx c;
  c.No = h->d.No; c.Nv = h->d.Nv; c.N = h->d.N; c.B = h->d.B; c.F = F ? F : h->F; c.omega = h->omega_op;
  return c;
}

static esmp2_status read_slots(esmp2_handle *h, double *out, int n) {
  cudaMemcpyAsync(h->hred, h->red_out, sizeof(double) * 32, cudaMemcpyDeviceToHost, h->stream);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "sync");
  for (int k = 0; k < n; ++k) out[k] = h->hred[k];
  return ESMP2_OK;
}

double dot_w(esmp2_handle *h, const double *u, const double *v) {
  k_dot_w<<<kRedBlocks, kRedThreads, 0, h->stream>>>(vctx(h), u, v, h->red);
  k_finalize<<<1, 256, 0, h->stream>>>(h->red, kRedBlocks, 1, h->red_out, 3);
  h->launches += 2;
  double s[32];
  read_slots(h, s, 32);
  return s[8];
}

esmp2_status solve64(esmp2_handle *h, double tol, int maxit, esmp2_solve_info *info, int virt_tc) {
  auto t0 = std::chrono::steady_clock::now();
  {  // the plain fp64 solve works in the TOP basis
    esmp2_status s0 = x_to_basis(h, 0);
    if (s0) return s0;
  }
  const VCtx c = vctx(h);
  double *x = h->s64.x, *r = h->s64.r, *p = h->s64.p, *q = h->s64.q;
  cudaStream_t st = h->stream;
  h->last_precision = virt_tc ? ESMP2_FP64_TC : ESMP2_FP64;
  h->r_true = false;
  const int lv = virt_tc ? kFp64TcLevels : 0;
  antisym_project(h, x);
  esmp2_status s = ESMP2_OK;
  int nsig = 0;
  if (h->x_zero) {  // cold start: A x = 0, the first residual is b
    cudaMemsetAsync(q, 0, sizeof(double) * h->d.n, st);
  } else {
    if ((s = sigma64(h, x, q, lv))) return s;
    nsig = 1;
  }
  h->x_zero = false;
  k_pcg_init<<<kRedBlocks, kRedThreads, 0, st>>>(c, h->b, q, r, p, h->red);
  k_finalize<<<1, 256, 0, st>>>(h->red, kRedBlocks, 3, h->red_out, 0);
  h->launches += 2;
  antisym_project(h, p);
  double sl[32];
  if ((s = read_slots(h, sl, 32))) return s;
  const double bnorm = std::sqrt(sl[2]);
  double rr = sl[1];
  int it = 0;
  esmp2_status result = ESMP2_ERR_NOT_CONVERGED;
  double relres = bnorm > 0 ? std::sqrt(rr) / bnorm : 0.0;
  if (bnorm == 0.0) { result = ESMP2_OK; h->r_true = true; }
  while (result != ESMP2_OK && it < maxit) {
    if (std::sqrt(rr) <= tol * bnorm) {  // confirm with the true residual
      if ((s = sigma64(h, x, q, lv))) return s;
      ++nsig;
      k_pcg_init<<<kRedBlocks, kRedThreads, 0, st>>>(c, h->b, q, r, p, h->red);
      k_finalize<<<1, 256, 0, st>>>(h->red, kRedBlocks, 3, h->red_out, 0);
      h->launches += 2;
      antisym_project(h, p);
      if ((s = read_slots(h, sl, 32))) return s;
      rr = sl[1];
      relres = std::sqrt(rr) / bnorm;
      if (relres <= tol) { result = ESMP2_OK; h->r_true = true; break; }
    }
    if ((s = sigma64(h, p, q, lv))) return s;
    if (virt_tc && (s = check_device_flag(h))) return s;
    ++nsig;
    k_dot_w<<<kRedBlocks, kRedThreads, 0, st>>>(c, p, q, h->red);
    k_finalize<<<1, 256, 0, st>>>(h->red, kRedBlocks, 1, h->red_out, 1);
    k_pcg_update<<<kRedBlocks, kRedThreads, 0, st>>>(c, h->red_out, x, r, p, q, h->red);
    k_finalize<<<1, 256, 0, st>>>(h->red, kRedBlocks, 2, h->red_out, 2);
    k_pcg_p<<<kRedBlocks, kRedThreads, 0, st>>>(c, h->red_out, r, p);
    h->launches += 5;
    antisym_project(h, p);
    if ((s = read_slots(h, sl, 32))) return s;
    ++it;
    if (!(sl[3] > 0.0)) { h->err = "CG: p.Ap <= 0 (operator not positive definite)"; result = ESMP2_ERR_INDEFINITE; break; }
    rr = sl[1];
    relres = std::sqrt(rr) / bnorm;
  }
  if (result == ESMP2_ERR_NOT_CONVERGED) h->err = "CG did not reach the tolerance within maxit iterations";
  if (info) {
    info->iterations = it;
    info->outer = 1;
    info->sigma_fp64 = nsig;
    info->sigma_lowp = 0;
    info->rel_residual = relres;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  h->solved = (result == ESMP2_OK || result == ESMP2_ERR_NOT_CONVERGED);
  return result;
}

esmp2_status energy(esmp2_handle *h, esmp2_energy_parts *parts) {
  if (!h->solved) { h->err = "esmp2_energy needs a previous esmp2_solve"; return ESMP2_ERR_STATE; }
  cudaStream_t st = h->stream;
  const int basis = h->x_basis;
  const double *F = basis == 2 ? h->Farr : basis == 1 ? h->Fsemi : h->F;
  const double *bb = basis == 2 ? h->barr : basis == 1 ? h->bsemi : h->b;
  esmp2_status s = ESMP2_OK;
  if (h->r_true) {
    // the solve ended on a true residual r = -b - A x of this x: A x = -b - r, no sigma build
    k_hylleraas<<<kRedBlocks, kRedThreads, 0, st>>>(vctx(h, F), bb, h->s64.x, h->s64.r, 1, h->red);
  } else {
    // after a tensor-core solve the Hylleraas sigma uses the float64-exact digit levels
    const int lv = (h->last_precision != ESMP2_FP64 && split_supported(h, kFp64TcLevels)) ? kFp64TcLevels : 0;
    if (basis == 2) s = sigma64_arrow(h, h->s64.x, h->s64.q);
    else s = sigma64_F(h, F, basis, h->s64.x, h->s64.q, lv);
    if (s) return s;
    k_hylleraas<<<kRedBlocks, kRedThreads, 0, st>>>(vctx(h, F), bb, h->s64.x, h->s64.q, 0, h->red);
  }
  k_finalize<<<1, 256, 0, st>>>(h->red, kRedBlocks, 10, h->red_out, 3);
  h->launches += 2;
  double sl[32];
  if ((s = read_slots(h, sl, 32))) return s;
  double e_blk[5];
  for (int k = 0; k < 5; ++k) e_blk[k] = kWeights[k] * (2.0 * sl[8 + 2 * k] + sl[9 + 2 * k]);
  if (!h->e2s_done) {
    const int No = h->d.No;
    SCtx sc;
    sc.No = No; sc.Nv = h->d.Nv; sc.N = h->d.N; sc.F = h->F; sc.lam = h->lam; sc.ovov = h->ovov; sc.omega = h->omega_op;
    const int nb = No * No * No;
    const int64_t ng = (int64_t)No * h->d.Nv * No * h->d.Nv;
    float2 *gdf = nullptr;
    cudaError_t ce = dmalloc(reinterpret_cast<void **>(&gdf), sizeof(float2) * (size_t)ng, st);
    if (ce != cudaSuccess) return check_cuda(h, ce, "S-space integrals");
    k_ovov_df<<<1216, 256, 0, st>>>(h->ovov, gdf, ng);
    h->launches += 1;
    SDf gd{gdf};
    double tot = 0.0;
    const int npair = No * (No - 1) / 2, chAB = 8, chC = 4;
    const int grids[3] = {npair * chAB, No * No * chC, nb};
    for (int sector = 0; sector < 3; ++sector) {
      if (grids[sector] == 0) continue;
      {
        KScope ks(st, ESMP2_KT_E2S, 0.0, 0.0);
        if (sector == 0) k_e2s_ab<<<grids[0], 128, 0, st>>>(sc, gd, chAB, h->red);
        else if (sector == 1) k_e2s_cm<<<grids[1], 128, 0, st>>>(sc, gd, chC, h->red);
        else k_e2s_gen<<<grids[2], 128, 0, st>>>(sc, h->red);
      }
      k_finalize<<<1, 256, 0, st>>>(h->red, grids[sector], 1, h->red_out, 3);
      h->launches += 2;
      if ((s = read_slots(h, sl, 32))) break;
      tot += sl[8];
    }
    dfree(gdf, st);
    if (s) return s;
    h->e2s = tot;
    h->e2s_done = true;
  }
  parts->E2_D = e_blk[0] + e_blk[1];
  parts->E2_L = e_blk[2] + e_blk[3] + e_blk[4];
  parts->E2_S = h->e2s;
  parts->E2 = parts->E2_D + parts->E2_L + parts->E2_S;
  return check_cuda(h, cudaGetLastError(), "energy");
}

// Preconditioned MINRES (Paige and Saunders) on A x = -b in the reduced-cost basis, float64:
// for operators that are not positive definite, where CG does not apply (Sec. III.A uses CG).
// The Lanczos vectors of M^-1 A are generated with the weighted inner product; x follows from
// the short recurrence of the QR factorisation of the tridiagonal matrix (one Givens rotation
// per step).  The preconditioned residual estimate phibar triggers a true residual; the solve
// restarts from x until the true relative residual meets tol.
esmp2_status solve_minres(esmp2_handle *h, double tol, int maxit, esmp2_solve_info *info) {
  auto t0 = std::chrono::steady_clock::now();
  esmp2_status s = ensure_arrow(h);
  if (s) return s;
  if ((s = x_to_basis(h, 2))) return s;
  h->arrowv = true;
  const int64_t n = h->d.n;
  cudaStream_t st = h->stream;
  if (!h->mr_a) {   // the two direction vectors and the Lanczos vector v (x, q, r1, r2 are the handle's)
    cudaError_t e = dmalloc(reinterpret_cast<void **>(&h->mr_a), sizeof(double) * (size_t)n, st);
    if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void **>(&h->mr_b), sizeof(double) * (size_t)n, st);
    if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void **>(&h->mr_v), sizeof(double) * (size_t)n, st);
    if (e != cudaSuccess) return check_cuda(h, e, "MINRES vectors");
  }
  singlet_project(h, h->s64.x);
  const VCtx c = vctx(h, h->Farr);
  double *x = h->s64.x, *q = h->s64.q, *r1 = h->s64.r, *r2 = h->s64.p, *v = h->mr_v, *w1 = h->mr_a, *w2 = h->mr_b;
  if (!x || !q || !r1 || !r2 || !v || !w1 || !w2 || !h->barr || !h->Farr) {
    h->err = "MINRES: missing work vector";
    return ESMP2_ERR_STATE;
  }
  h->last_precision = ESMP2_REDUCED_MINRES;
  h->r_true = false;
  double sl[32], relres = 1.0, bn = -1.0;
  int iters = 0, nsig = 0, restarts = 0;
  esmp2_status result = ESMP2_ERR_NOT_CONVERGED;
  while (true) {
    // true residual r2 = -b - A x, its norms <r, M^-1 r>_w and <r, r>_w
    if (h->x_zero) {
      k_negsum64<<<1216, 256, 0, st>>>(h->barr, nullptr, r2, n);
    } else {
      if ((s = sigma64_arrow(h, x, q))) return s;
      ++nsig;
      k_negsum64<<<1216, 256, 0, st>>>(h->barr, q, r2, n);
    }
    k_mr_res<<<kRedBlocks, kRedThreads, 0, st>>>(c, r2, h->red);
    k_finalize<<<1, 256, 0, st>>>(h->red, kRedBlocks, 2, h->red_out, 3);
    h->launches += 3;
    if ((s = read_slots(h, sl, 32))) return s;
    if (bn < 0.0) {   // |b|_w
      k_mr_dot<<<kRedBlocks, kRedThreads, 0, st>>>(c, h->barr, h->barr, h->red);
      k_finalize<<<1, 256, 0, st>>>(h->red, kRedBlocks, 1, h->red_out, 3);
      h->launches += 2;
      double sb[32];
      if ((s = read_slots(h, sb, 32))) return s;
      bn = std::sqrt(sb[8]);
    }
    const double beta1 = std::sqrt(std::max(sl[8], 0.0));
    relres = bn > 0 ? std::sqrt(std::max(sl[9], 0.0)) / bn : 0.0;
    if (std::getenv("ESMP2_DEBUG"))
      std::fprintf(stderr, "esmp2 minres: restart %d relres %.3e iterations %d\n", restarts, relres, iters);
    if (relres <= tol) {
      result = ESMP2_OK;
      if (r2 != h->s64.r) cudaMemcpyAsync(h->s64.r, r2, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st);
      h->r_true = true;
      break;
    }
    if (iters >= maxit || restarts >= 20 || !(beta1 > 0.0)) break;
    ++restarts;
    // Lanczos start: r1 = r2 = r, v = M^-1 r / beta1, w1 = w2 = 0
    cudaMemcpyAsync(r1, r2, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(w1, 0, sizeof(double) * (size_t)n, st);
    cudaMemsetAsync(w2, 0, sizeof(double) * (size_t)n, st);
    k_mr_v<<<1216, 256, 0, st>>>(c, r2, 1.0 / beta1, v);
    h->launches += 1;
    double oldb = 0.0, beta = beta1, dbar = 0.0, epsln = 0.0, phibar = beta1, cs = -1.0, sn = 0.0;
    // phibar = |r|_{M^-1} of the recurrence; it is run well below the target (the two norms differ
    // by the spread of |diag|), then the true residual decides
    const double stop = 0.1 * tol * beta1 / std::max(relres, 1e-300);
    while (iters < maxit) {
      if ((s = sigma64_arrow(h, v, q))) return s;   // q = A v
      ++nsig;
      k_mr_dot<<<kRedBlocks, kRedThreads, 0, st>>>(c, v, q, h->red);
      k_finalize<<<1, 256, 0, st>>>(h->red, kRedBlocks, 1, h->red_out, 3);
      h->launches += 2;
      if ((s = read_slots(h, sl, 32))) return s;
      const double alpha = sl[8];
      // y = q - (alpha / beta) r2 - (beta / oldb) r1, over r1; then r1 <-> r2
      k_mr_y<<<kRedBlocks, kRedThreads, 0, st>>>(c, q, r2, r1, alpha / beta, oldb > 0.0 ? beta / oldb : 0.0, h->red);
      k_finalize<<<1, 256, 0, st>>>(h->red, kRedBlocks, 1, h->red_out, 3);
      h->launches += 2;
      if ((s = read_slots(h, sl, 32))) return s;
      std::swap(r1, r2);   // r2 = y (the new Lanczos residual), r1 = the previous one
      oldb = beta;
      beta = std::sqrt(std::max(sl[8], 0.0));
      // QR step of the tridiagonal matrix: the previous rotation on the new column, then a new
      // rotation that zeroes its subdiagonal beta
      const double oldeps = epsln, delta = cs * dbar + sn * alpha, gbar = sn * dbar - cs * alpha;
      epsln = sn * beta;
      dbar = -cs * beta;
      const double gamma = std::max(std::sqrt(gbar * gbar + beta * beta), 1e-300);
      cs = gbar / gamma;
      sn = beta / gamma;
      const double phi = cs * phibar;
      phibar = sn * phibar;
      // w_k = (v - oldeps w_{k-2} - delta w_{k-1}) / gamma over w_{k-2}; x += phi w_k;
      // v = M^-1 r2 / beta
      k_mr_update<<<1216, 256, 0, st>>>(c, v, w1, w2, x, r2, oldeps, delta, 1.0 / gamma, phi,
                                        beta > 0.0 ? 1.0 / beta : 0.0);
      h->launches += 1;
      std::swap(w1, w2);   // w2 = w_k, w1 = w_{k-1}
      h->x_zero = false;
      ++iters;
      if (std::getenv("ESMP2_DEBUG"))
        std::fprintf(stderr, "esmp2 minres %d: phibar/beta1 %.3e\n", iters, phibar / beta1);
      if (phibar <= stop || !(beta > 0.0)) break;
    }
    singlet_project(h, x);
  }
  if (info) {
    info->iterations = iters;
    info->outer = restarts;
    info->sigma_fp64 = nsig;
    info->sigma_lowp = 0;
    info->rel_residual = relres;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (result == ESMP2_ERR_NOT_CONVERGED) h->err = "MINRES did not reach the tolerance";
  h->solved = (result == ESMP2_OK || result == ESMP2_ERR_NOT_CONVERGED);
  return result;
}

// Mixed precision: float64 iterative refinement around a low-precision inner PCG.
//   outer:  r = -b - A x with the float64 sigma (true residual; stop when |r|/|b| <= tol)
//   inner:  A d = r by Jacobi PCG on float32 vectors whose sigma uses the bf16 tcgen05
//           contraction (fp32 accumulation); x += d.
// Everything runs in the basis whose occupied orbitals other than t diagonalise F_oo
// (the solution is rotated back to the TOP basis on request).
esmp2_status solve_mixed(esmp2_handle *h, double tol, int maxit, esmp2_solve_info *info, bool tf32, bool arrowv) {
  auto t0 = std::chrono::steady_clock::now();
  debug_phase(h, "solve: start");
  if ((tf32 || arrowv) && h->d.No > 32) {
    h->err = "ESMP2_MIXED_TF32 and ESMP2_REDUCED_MIXED need the packed inner solve (No <= 32)";
    return ESMP2_ERR_UNSUPPORTED;
  }
  esmp2_status s = ensure_mixed(h, true);
  if (s) return s;
  if (arrowv && (s = ensure_arrow(h))) return s;
  h->tf32 = tf32;
  h->arrowv = arrowv;
  debug_phase(h, "solve: basis set-up");
  if ((s = x_to_basis(h, arrowv ? 2 : 1))) return s;
  cudaStream_t st = h->stream;
  // the singlet solution lies in the symmetric subspace (antisymmetric T, X, Y; S_ij^ab =
  // S_ji^ba); the packed inner solve acts on that subspace only, so x and every residual
  // handed to it are projected onto it (removing the rounding-level components outside)
  if (!h->x_zero) singlet_project(h, h->s64.x);
  const VCtx c = vctx(h, arrowv ? h->Farr : h->Fsemi);
  const double *bsel = arrowv ? h->barr : h->bsemi;
  debug_phase(h, "solve: x rotation + projection");
  // inner vectors: the packed layout (T, X, Y slices i < j, rows padded; the contraction as one
  // tensor-core GEMM) when the arrow sums fit their register tiles (No <= 32), else full storage
  const bool packed = h->d.No <= 32;
  ICtx ic;
  bool fused_bf16 = true;
  // the contraction forms of the packed solve precondition with the Jacobi diagonal of the
  // basis that diagonalises F_vv, applied through two-sided rotations (rotated Jacobi); the
  // reduced-cost basis already is that basis
  const bool rj = packed && !arrowv;
  if (packed) {
    if ((s = packed_setup(h))) return s;
    if (rj && (s = packed_rj_setup(h))) return s;
    for (int k = 0; k < 6; ++k) ic.off[k] = h->pk.boff[k];
    const float wp[5] = {1.f, 1.f, 1.f, 1.f, 2.f};
    for (int k = 0; k < 5; ++k) ic.w[k] = wp[k];
    ic.dinv = h->pdinv;
    // bf16: the p update also writes the operand copy; tf32: p is the operand
    ic.pb = tf32 ? nullptr : static_cast<__nv_bfloat16 *>(h->pop);
    ic.vec = 1;   // blocks start on multiples of Nv * Nvp elements, Nvp a multiple of 8
  } else {
    if (!h->dinv32) {
      cudaError_t e = dmalloc(reinterpret_cast<void **>(&h->dinv32), sizeof(__half) * (size_t)h->d.n, h->stream);
      if (e != cudaSuccess) return check_cuda(h, e, "preconditioner");
      k_dinv32<<<2432, 128, 0, st>>>(c, h->dinv32);
      h->launches += 1;
    }
    for (int k = 0; k < 6; ++k) ic.off[k] = (int64_t)k * h->d.B;
    for (int k = 0; k < 5; ++k) ic.w[k] = (float)kWeights[k];
    ic.dinv = h->dinv32;
    // rows of the bf16 operand are padded to a multiple of 8; without padding the PCG update
    // writes it directly
    fused_bf16 = (h->d.Nv % 8) == 0;
    ic.pb = fused_bf16 ? static_cast<__nv_bfloat16 *>(h->xlp) : nullptr;
    ic.vec = (h->d.B % 4) == 0;
  }
  debug_phase(h, "solve: preconditioner");
  // small instances are launch-bound: replay the inner iteration as a CUDA graph
  bool use_graph = h->d.n <= (64LL << 20) && st != nullptr;
  const int graph_kind = (tf32 ? 1 : 0) + (arrowv ? 2 : 0);
  if (h->inner_graph && (!use_graph || h->graph_kind != graph_kind)) {
    cudaGraphExecDestroy(h->inner_graph);
    h->inner_graph = nullptr;
  }
  double *x = h->s64.x, *r = h->s64.r, *q = h->s64.q;
  float *r32 = packed ? h->pr : h->r32, *p32 = packed ? packed_p(h) : h->p32, *q32 = packed ? h->pq : h->q32,
        *d32 = packed ? h->pd : h->x32;
  int outer = 0, inner_total = 0, nsig64 = 0, nsiglow = 0;
  double relres = 1.0, sl[32];
  esmp2_status result = ESMP2_ERR_NOT_CONVERGED;
  // relative tolerance of each inner solve (the bf16 rounding of the inner operand limits the
  // inner residual to ~1e-3 relative)
  // the float64 true residual takes its virtual-index terms from exact digit products on
  // the tensor cores when that is exact for this Nv, else from float64 GEMMs
  // (the reduced-cost basis forms its float64 virtual-index terms element-wise: no digit levels)
  const int lv = !arrowv && split_supported(h, split_levels_for(tol)) ? split_levels_for(tol) : 0;
  h->last_precision = arrowv ? ESMP2_REDUCED_MIXED : tf32 ? ESMP2_MIXED_TF32 : ESMP2_MIXED_BF16;
  h->r_true = false;
  const double eta = 1e-2;
  // An intermediate true residual only has to be accurate relative to itself: its digit
  // levels follow the relative residual it is expected to show (a low estimate, so never
  // too few levels); the residual that ends the refinement, and feeds the energy, always
  // takes the full count.
  double rho_next = 0.0, bb = -1.0;  // bb: <b, b>_w, taken with the first residual
  double prev_relres = 1e300;
  int stalled = 0;
  while (true) {
    int lv_k = lv;
    if (lv && rho_next > 1e1 * tol) lv_k = std::min(lv, split_levels_for(rho_next));
    const bool cold = outer == 0 && h->x_zero;  // cold start: the first true residual is -b
    bool approx = false;   // formed with reduced accuracy (relative to itself only)
    if (cold) {
      lv_k = lv;
    } else {
      // far from the tolerance the coupling pass runs in float32 (its ~1e-7 relative error
      // is a small fraction of the residual it feeds), next to reduced digit levels
      const bool c32 = (arrowv || lv_k < lv) && rho_next >= 1e-5;
      if (arrowv) s = sigma64_arrow(h, x, q, c32 ? 0 : 1);
      // x holds the singlet symmetries exactly (the packed accumulation keeps them bit for
      // bit, the full-storage path projects x after each step)
      else s = sigma64_F(h, h->Fsemi, 1, x, q, lv_k, c32 ? 0 : 1, true);
      if (s) return s;
      if (c32) couple_f32_into(h, x, q);
      approx = c32 || lv_k < lv;
      ++nsig64;
    }
    k_residual<<<kRedBlocks, kRedThreads, 0, st>>>(c, bsel, cold ? nullptr : q, r, h->red, bb < 0.0 ? 1 : 0);
    k_finalize<<<1, 256, 0, st>>>(h->red, kRedBlocks, 2, h->red_out, 3);
    h->launches += 2;
    if ((s = read_slots(h, sl, 32))) return s;
    if (bb < 0.0) bb = sl[9];
    const double rn = std::sqrt(sl[8]), bn = std::sqrt(bb);
    relres = bn > 0 ? rn / bn : 0.0;
    if (std::getenv("ESMP2_DEBUG"))
      std::fprintf(stderr, "esmp2 refine: outer %d relres %.3e inner_total %d levels %d\n", outer, relres, inner_total, lv_k);
    if (relres <= 1e1 * tol && approx) { rho_next = 0.0; continue; }  // confirm at full accuracy
    if (relres <= tol) { result = ESMP2_OK; h->r_true = true; break; }
    if (inner_total >= maxit) break;
    // three refinement steps in a row without reducing the true residual: stop
    if (relres >= 0.9 * prev_relres) { if (++stalled >= 3) { h->err = "refinement stagnated"; break; } }
    else stalled = 0;
    prev_relres = relres;
    // inner PCG on A d = r (r made exactly antisymmetric in T, X, Y: the inner sigma
    // contracts the slices i < j and mirrors them).  The rotated Jacobi preconditioner
    // projects z = M^-1 r onto the singlet subspace itself, so every search direction and d
    // have the symmetries exactly whatever rounding-level asymmetry r carries; r is then
    // read as it is.
    if (!rj) singlet_project(h, r);
    if (rj) {
      if ((s = packed_rj_init(h, r, kRedBlocks))) return s;
    } else {
      if (packed) packed_init(h, r, kRedBlocks);
      else ki_init<<<kRedBlocks, kRedThreads, 0, st>>>(ic, r, r32, p32, d32, h->red);
      k_finalize<<<1, 256, 0, st>>>(h->red, kRedBlocks, 2, h->red_out, 0);
      h->launches += packed ? 1 : 2;
    }
    if ((s = read_slots(h, sl, 32))) return s;
    const double r0 = std::sqrt(sl[1]);
    const double target = std::max(eta * r0, 0.25 * tol * bn);
    int inner = 0, since_best = 0;
    double best = r0;
    // one inner iteration: q = A p, alpha, x/r update, beta, p update (device scalars only)
    const bool dbg_dot = std::getenv("ESMP2_DEBUG") != nullptr && !use_graph;
    double fused_pq = 0.0, sep_pq = 0.0;
    auto inner_step = [&]() -> esmp2_status {
      const int64_t l0 = h->launches;
      // p.q partials from the coupling pass
      esmp2_status s2 = packed ? sigma_packed(h, p32, q32, true, h->pdot) : sigma_inner(h, p32, q32, fused_bf16, h->red);
      if (s2) return s2;
      if (packed && dbg_dot) {  // diagnostics (ESMP2_DEBUG, no graph capture): <p, A p> by a separate pass
        std::vector<double> part(h->pdot_n);
        cudaMemcpyAsync(part.data(), h->pdot, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        fused_pq = 0.0;
        for (double v : part) fused_pq += v;
        sep_pq = packed_wdot(h, p32, q32);
      }
      if (packed) k_finalize<<<1, 256, 0, st>>>(h->pdot, h->pdot_n, 1, h->red_out, 1);
      else k_finalize<<<1, 256, 0, st>>>(h->red, (int)couple_dot_parts(h), 1, h->red_out, 1);
      h->launches += 1;
      if (rj) {   // r -= alpha q, z = M^-1 r (rotated Jacobi), beta, d and p
        if ((s2 = packed_rj_step(h, kRedBlocks))) return s2;
      } else {
        ki_update<<<kRedBlocks, kRedThreads, 0, st>>>(ic, h->red_out, r32, q32, h->red);
        k_finalize<<<1, 256, 0, st>>>(h->red, kRedBlocks, 2, h->red_out, 2);
        ki_p<<<kRedBlocks, kRedThreads, 0, st>>>(ic, h->red_out, r32, p32, d32);
        h->launches += 3;
      }
      h->inner_graph_launches_pending = h->launches - l0;
      return check_cuda(h, cudaGetLastError(), "inner step");
    };
    while (inner_total < maxit) {
      if (h->inner_graph) {
        if ((s = check_cuda(h, cudaGraphLaunch(h->inner_graph, st), "inner graph"))) return s;
        h->launches += h->inner_graph_launches;
      } else if (use_graph && inner_total > 0) {
        // capture one iteration (every pointer it touches belongs to the handle) and replay it
        const int64_t l0 = h->launches;
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) ok = inner_step() == ESMP2_OK;
        if (cudaStreamEndCapture(st, &g) != cudaSuccess || !g) ok = false;
        if (ok) ok = cudaGraphInstantiate(&h->inner_graph, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        h->launches = l0;
        if (ok) {
          h->inner_graph_launches = h->inner_graph_launches_pending;
          h->graph_kind = graph_kind;
          if ((s = check_cuda(h, cudaGraphLaunch(h->inner_graph, st), "inner graph"))) return s;
          h->launches += h->inner_graph_launches;
        } else {
          h->inner_graph = nullptr;
          use_graph = false;
          if ((s = inner_step())) return s;
        }
      } else {
        if ((s = inner_step())) return s;
      }
      ++nsiglow;
      if ((s = read_slots(h, sl, 32))) return s;
      if (std::getenv("ESMP2_DEBUG"))
        std::fprintf(stderr, "esmp2 inner %d: p.Ap %.6e (fused partials %.6e, separate pass %.6e) r.z %.6e r.r %.6e r0^2 %.6e\n",
                     inner, sl[3], fused_pq, sep_pq, sl[0], sl[1], r0 * r0);
      ++inner;
      ++inner_total;
      if (!(sl[3] > 0.0)) {
        // the step was not taken (alpha = 0 on the device).  Before the inner residual has
        // been cut tenfold this is negative curvature of A itself; after that it is the
        // rounding of the bf16 inner operator (whose floor lies at a few 1e-3 to a few 1e-2 of
        // the inner start): the inner solve ends there and the float64 refinement goes on
        if (best > 1e-1 * r0) { h->err = "inner CG: p.Ap <= 0"; result = ESMP2_ERR_INDEFINITE; }
        break;
      }
      const double rn_in = std::sqrt(sl[1]);
      if (rn_in < 0.99 * best) { best = rn_in; since_best = 0; } else ++since_best;
      if (rn_in <= target || inner >= 200 || since_best >= 8) break;  // converged or stagnating
    }
    if (result == ESMP2_ERR_INDEFINITE) break;
    if (std::getenv("ESMP2_DEBUG")) std::fprintf(stderr, "esmp2 refine:   inner %d  |r_in|/|r0| %.3e\n", inner, std::sqrt(sl[1]) / r0);
    rho_next = relres * std::max(r0 > 0 ? std::sqrt(sl[1]) / r0 : 0.0, 1e-4);
    if (packed) {
      // x stays in the singlet subspace exactly: d is exactly antisymmetric in (a, b) and
      // spin-flip symmetric in S (the packed coupling pass writes both images from one value),
      // and kp_acc64 adds +d and -d to the two slices (negation commutes with rounding)
      packed_accumulate(h, x);
    } else {
      kt_accumulate<float><<<kRedBlocks, kRedThreads, 0, st>>>(c, x, d32);
      h->launches += 1;
      singlet_project(h, x);  // the float64 residual pass assumes exactly antisymmetric T, X, Y
    }
    h->x_zero = false;
    ++outer;
    if ((s = check_device_flag(h))) return s;
  }
  if (result == ESMP2_ERR_NOT_CONVERGED && stalled < 3)
    h->err = "refinement did not reach the tolerance within maxit inner iterations";
  if (info) {
    info->iterations = inner_total;
    info->outer = outer;
    info->sigma_fp64 = nsig64;
    info->sigma_lowp = nsiglow;
    info->rel_residual = relres;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  h->solved = (result == ESMP2_OK || result == ESMP2_ERR_NOT_CONVERGED);
  return result;
}

}  // namespace esmp2

// The inner (float32 / bf16) sigma of the mixed-precision solve on the packed layout.
//
// The inner solve works in the basis whose occupied orbitals other than t diagonalise F_oo
// (D and L do not change under rotations that fix t), so the occupied-index terms of the
// operator are a diagonal plus the t row and column ("arrow" form).  Its vectors keep only
// the T, X, Y slices i < j (the slice (j, i) is the negative) and every S and Z slice, with
// rows padded to Nvp (see esmp2::Packed).  One sigma build q = A p:
//   1. the bf16 operand (written by the PCG update) gets the transposed Z slices appended;
//   2. one tensor-core GEMM (vgemm.cu) forms P = A F_vv for every operand row;
//   3. the slice-direction arrow sums (sums over an occupied index weighted by F_l,t and
//      F_l,t') are one streaming pass, the few N^3-sized intermediates of the N^4 coupling
//      terms (reductions over one virtual index with the occupied-virtual Fock rows) three
//      small ones, all float32 from p: computed from the bf16 operand they made the inner
//      operator lose the symmetry of its float32 coefficients, and CG stalled;
//   4. the coupling pass forms y = (P combined with its transpose) + the N^4 coupling terms
//      (Table 1's T3<->T, S3<->S, S3<->T rows and the mixed-spin L-triple cross terms) +
//      the diagonal (-omega, the L pair energy, the arrow diagonal), masks the slots that
//      are not amplitudes, and leaves the per-CTA partials of <p, q>.  T, X, Y are computed on
//      tile pairs and written with exact antisymmetry in (a, b); S on slice pairs (i, j),
//      (j, i), written with the exact spin-flip symmetry S_ij^ab = S_ji^ba of the singlet.
// Every formula below is the element-wise form of the full-storage coupling pass (sigma.cu)
// with the packed slice access.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace esmp2 {

Packed make_packed(int No, int Nv) {
  Packed L{};
  L.No = No;
  L.Nv = Nv;
  L.Nvp = (Nv + 7) & ~7;
  L.nh = No * (No - 1) / 2;
  L.NN = No * No;
  L.SL = (int64_t)Nv * L.Nvp;
  const int ns[6] = {L.nh, L.NN, L.nh, L.nh, L.NN, L.NN};
  int64_t o = 0;
  for (int k = 0; k < 6; ++k) {
    L.boff[k] = o;
    o += ns[k] * L.SL;
  }
  L.nslices = 3 * L.nh + 2 * L.NN;
  L.n = L.boff[5];
  return L;
}

namespace {

constexpr int kT = 32;          // coupling tile edge
constexpr int kThreads = 256;   // 32 x 8

__host__ __device__ __forceinline__ int pair_ij(int No, int i, int j) { return i * No - i * (i + 1) / 2 + (j - i - 1); }
__host__ __device__ __forceinline__ void pair_decode(int No, int k, int &i, int &j) {
  i = 0;
  while (k >= No - 1 - i) {
    k -= No - 1 - i;
    ++i;
  }
  j = i + 1 + k;
}

__device__ __forceinline__ bool valid_elem(int blk, int i, int j, int a, int b) {
  if ((blk == BT || blk == BX || blk == BY) && (i == j || a == b)) return false;
  if (blk == BX && (i == 0 || j == 0 || a == 0 || b == 0)) return false;
  if (blk == BZ && (j == 0 || b == 0 || (i == 0 && a == 0))) return false;
  return true;
}

// slice index (in slices of SL elements) of block blk's first slice, packed order
__host__ __device__ __forceinline__ int slice0(const Packed &L, int blk) { return (int)(L.boff[blk] / L.SL); }

struct PV {
  Packed L;
  // slice (blk, i, j): pointer and sign; nullptr for the identically zero slices i == j of T, X, Y
  template <typename T>
  __device__ __forceinline__ T *sl(T *v, int blk, int i, int j, float &sg) const {
    if (blk == BS || blk == BZ) {
      sg = 1.f;
      return v + L.boff[blk] + ((int64_t)i * L.No + j) * L.SL;
    }
    if (i == j) {
      sg = 0.f;
      return nullptr;
    }
    if (i < j) {
      sg = 1.f;
      return v + L.boff[blk] + (int64_t)pair_ij(L.No, i, j) * L.SL;
    }
    sg = -1.f;
    return v + L.boff[blk] + (int64_t)pair_ij(L.No, j, i) * L.SL;
  }
  __device__ __forceinline__ float at(const float *v, int blk, int i, int j, int a, int b) const {
    float sg;
    const float *p = sl(v, blk, i, j, sg);
    return p ? sg * p[(int64_t)a * L.Nvp + b] : 0.f;
  }
  // block, i, j of slice s of the packed order (T | S | X | Y | Z)
  __device__ __forceinline__ void decode(int s, int &blk, int &i, int &j) const {
    const int nh = L.nh, NN = L.NN;
    if (s < nh) { blk = BT; pair_decode(L.No, s, i, j); }
    else if (s < nh + NN) { blk = BS; s -= nh; i = s / L.No; j = s % L.No; }
    else if (s < 2 * nh + NN) { blk = BX; pair_decode(L.No, s - nh - NN, i, j); }
    else if (s < 3 * nh + NN) { blk = BY; pair_decode(L.No, s - 2 * nh - NN, i, j); }
    else { blk = BZ; s -= 3 * nh + NN; i = s / L.No; j = s % L.No; }
  }
};

struct FF {  // float Fock matrix of the working basis (read-only in every kernel: cached loads)
  const float *F;
  int N, No;
  __device__ __forceinline__ float o(int k, int l) const { return __ldg(F + k * N + l); }
  __device__ __forceinline__ float v(int a, int b) const { return __ldg(F + (No + a) * N + No + b); }
  __device__ __forceinline__ float ov(int k, int a) const { return __ldg(F + k * N + No + a); }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// sum of one value per thread of the CTA into red[slot] (one CTA writes one slot)
__device__ __forceinline__ void cta_partial(double v, double *red, int64_t slot) {
  __shared__ double sh[32];
  v = warp_sum_d(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    s = warp_sum_d(s);
    if (threadIdx.x == 0) red[slot] = s;
  }
  __syncthreads();
}
template <int NQ>
__device__ __forceinline__ void cta_partials(double (&v)[NQ], double *red) {
  __shared__ double sh[NQ][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double s = warp_sum_d(v[q]);
    if (lane == 0) sh[q][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = lane < (int)(blockDim.x >> 5) ? sh[q][lane] : 0.0;
      s = warp_sum_d(s);
      if (lane == 0) red[(int64_t)q * gridDim.x + blockIdx.x] = s;
    }
  }
}

__device__ __forceinline__ float blk_w(int blk) { return blk == BZ ? 2.f : 1.f; }

// ---------------------------------------------------------------- layout conversions
// r = r64 (full storage) on the packed slots, p = M^-1 r, d = 0, pb = bf16(p) (if kept); partials
// <r, M^-1 r>_w, <r, r>_w.  One CTA iteration per packed row (slice, a).
__global__ void kp_init(PV pv, const double *r64, const __half *dinv, float *r, float *p, float *d,
                        __nv_bfloat16 *pb, double *red) {
  const Packed &L = pv.L;
  const int64_t rows = (int64_t)L.nslices * L.Nv, NvNv = (int64_t)L.Nv * L.Nv, B = (int64_t)L.NN * NvNv;
  float a0 = 0.f, a1 = 0.f;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const int s = (int)(row / L.Nv), a = (int)(row % L.Nv);
    int blk, i, j;
    pv.decode(s, blk, i, j);
    const double *src = r64 + blk * B + ((int64_t)i * L.No + j) * NvNv + (int64_t)a * L.Nv;
    const int64_t e0 = (int64_t)s * L.SL + (int64_t)a * L.Nvp;
    const float w = blk_w(blk);
    for (int b = threadIdx.x; b < L.Nvp; b += blockDim.x) {
      const int64_t e = e0 + b;
      const float ri = b < L.Nv ? (float)src[b] : 0.f;
      const float z = __half2float(dinv[e]) * ri;
      r[e] = ri;
      p[e] = z;
      d[e] = 0.f;
      if (pb) pb[e] = __float2bfloat16_rn(z);
      a0 += w * ri * z;
      a1 += w * ri * ri;
    }
  }
  double v[2] = {(double)a0, (double)a1};
  cta_partials<2>(v, red);
}

// x64 (full storage) += d (packed); T, X, Y slices also update their (j, i) partner with -d.
// One warp per packed row (slice, a); consecutive lanes take consecutive b, so every load and
// every read-modify-write of the float64 rows is one contiguous segment per warp.
__global__ void __launch_bounds__(256) kp_acc64(PV pv, double *x, const float *d) {
  const Packed &L = pv.L;
  const int64_t rows = (int64_t)L.nslices * L.Nv, NvNv = (int64_t)L.Nv * L.Nv, B = (int64_t)L.NN * NvNv;
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5, Nv = L.Nv;
  for (int64_t row = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); row < rows; row += (int64_t)gridDim.x * wpb) {
    const int s = (int)(row / Nv), a = (int)(row % Nv);
    int blk, i, j;
    pv.decode(s, blk, i, j);
    const float *src = d + (int64_t)s * L.SL + (int64_t)a * L.Nvp;
    double *x1 = x + blk * B + ((int64_t)i * L.No + j) * NvNv + (int64_t)a * Nv;
    double *x2 = x + blk * B + ((int64_t)j * L.No + i) * NvNv + (int64_t)a * Nv;
    const bool anti = !(blk == BS || blk == BZ);
    for (int b = lane; b < Nv; b += 32) {
      const double v = (double)src[b];
      x1[b] += v;
      if (anti) x2[b] -= v;
    }
  }
}

// packed float32 copy of a full-storage float64 vector
__global__ void kp_from64(PV pv, const double *x, float *out) {
  const Packed &L = pv.L;
  const int64_t rows = (int64_t)L.nslices * L.Nv, NvNv = (int64_t)L.Nv * L.Nv, B = (int64_t)L.NN * NvNv;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const int s = (int)(row / L.Nv), a = (int)(row % L.Nv);
    int blk, i, j;
    pv.decode(s, blk, i, j);
    const double *src = x + blk * B + ((int64_t)i * L.No + j) * NvNv + (int64_t)a * L.Nv;
    float *dst = out + (int64_t)s * L.SL + (int64_t)a * L.Nvp;
    for (int b = threadIdx.x; b < L.Nvp; b += blockDim.x) dst[b] = b < L.Nv ? (float)src[b] : 0.f;
  }
}

// full-storage float64 vector from a packed float32 one (T, X, Y expanded antisymmetrically;
// the i == j slices of T, X, Y are zero)
__global__ void kp_to64(PV pv, const float *in, double *y) {
  const Packed &L = pv.L;
  const int64_t rows = 5LL * L.NN * L.Nv, NvNv = (int64_t)L.Nv * L.Nv;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const int a = (int)(row % L.Nv);
    const int64_t f = row / L.Nv;
    const int j = (int)(f % L.No), i = (int)((f / L.No) % L.No), blk = (int)(f / L.NN);
    float sg;
    const float *src = pv.sl(in, blk, i, j, sg);
    double *dst = y + f * NvNv + (int64_t)a * L.Nv;
    for (int b = threadIdx.x; b < L.Nv; b += blockDim.x)
      dst[b] = src ? (double)(sg * src[(int64_t)a * L.Nvp + b]) : 0.0;
  }
}

// zero the non-amplitude slots of a full-storage float64 vector (one CTA iteration per row)
__global__ void kp_mask64(int No, int Nv, double *y) {
  const int64_t rows = 5LL * No * No * Nv;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const int a = (int)(row % Nv);
    const int64_t f = row / Nv;
    const int j = (int)(f % No), i = (int)((f / No) % No), blk = (int)(f / ((int64_t)No * No));
    for (int b = threadIdx.x; b < Nv; b += blockDim.x)
      if (!valid_elem(blk, i, j, a, b)) y[row * Nv + b] = 0.0;
  }
}

// Jacobi preconditioner 1 / diag(A) in half precision, zero on non-amplitude and pad slots
__global__ void kp_dinv(PV pv, FF F, float omega, __half *dinv) {
  const Packed &L = pv.L;
  const int64_t rows = (int64_t)L.nslices * L.Nv;
  const float shift = F.v(0, 0) - F.o(0, 0);
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    const int s = (int)(row / L.Nv), a = (int)(row % L.Nv);
    int blk, i, j;
    pv.decode(s, blk, i, j);
    // (F_aa + F_bb) - (F_ii + F_jj): the same rounding for (i, j, a, b) and (j, i, b, a), so
    // the preconditioner keeps the symmetries of the amplitudes exactly
    const float occ = F.o(i, i) + F.o(j, j) + omega - (blk >= BX ? shift : 0.f), fa = F.v(a, a);
    __half *out = dinv + (int64_t)s * L.SL + (int64_t)a * L.Nvp;
    for (int b = threadIdx.x; b < L.Nvp; b += blockDim.x) {
      const bool ok = b < L.Nv && valid_elem(blk, i, j, a, b);
      out[b] = __float2half_rn(ok ? 1.f / ((fa + F.v(b, b)) - occ) : 0.f);
    }
  }
}

__global__ void kp_bf16(const float *src, __nv_bfloat16 *dst, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = __float2bfloat16_rn(src[e]);
}

// the transposed Z slices of the bf16 operand: op[ZT(s)][b][a] = op[Z(s)][a][b].  64 x 64 tiles;
// a lane moves a pair of bf16 values, so a warp reads and writes whole 128-byte rows.
__global__ void __launch_bounds__(256) kp_zt(PV pv, __nv_bfloat16 *op) {
  const Packed &L = pv.L;
  __shared__ __nv_bfloat16 t[64][66];
  const int Nv = L.Nv, Nvp = L.Nvp, nt = (Nv + 63) / 64;
  const int64_t items = (int64_t)L.NN * nt * nt;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int s = (int)(it / (nt * nt)), tt = (int)(it % (nt * nt)), ta = tt / nt, tb = tt % nt;
    const __nv_bfloat16 *src = op + L.boff[BZ] + (int64_t)s * L.SL;
    __nv_bfloat16 *dst = op + L.boff[5] + (int64_t)s * L.SL;
    for (int r = w; r < 64; r += 8) {   // rows a = ta*64 + r, columns b = tb*64 + 2 lane (+1)
      const int a = ta * 64 + r, b = tb * 64 + 2 * lane;
      __nv_bfloat162 v;
      if (a < Nv && b + 1 < Nvp) v = *reinterpret_cast<const __nv_bfloat162 *>(src + (int64_t)a * Nvp + b);
      else v = __halves2bfloat162(zero, zero);
      t[r][2 * lane] = v.x;
      t[r][2 * lane + 1] = v.y;
    }
    __syncthreads();
    for (int r = w; r < 64; r += 8) {   // rows b = tb*64 + r of the transposed slice, columns a
      const int b = tb * 64 + r, a = ta * 64 + 2 * lane;
      if (b < Nv && a + 1 < Nvp) {
        __nv_bfloat162 v;
        v.x = a < Nv ? t[2 * lane][r] : zero;
        v.y = a + 1 < Nv ? t[2 * lane + 1][r] : zero;
        *reinterpret_cast<__nv_bfloat162 *>(dst + (int64_t)b * Nvp + a) = v;
      }
    }
    __syncthreads();
  }
}

// the same for the float32 operand of the tf32 contraction: a lane moves two floats (8 bytes)
__global__ void __launch_bounds__(256) kp_zt32(PV pv, float *op) {
  const Packed &L = pv.L;
  __shared__ float t[64][65];
  const int Nv = L.Nv, Nvp = L.Nvp, nt = (Nv + 63) / 64;
  const int64_t items = (int64_t)L.NN * nt * nt;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int s = (int)(it / (nt * nt)), tt = (int)(it % (nt * nt)), ta = tt / nt, tb = tt % nt;
    const float *src = op + L.boff[BZ] + (int64_t)s * L.SL;
    float *dst = op + L.boff[5] + (int64_t)s * L.SL;
    for (int r = w; r < 64; r += 8) {
      const int a = ta * 64 + r, b = tb * 64 + 2 * lane;
      float2 v = make_float2(0.f, 0.f);
      if (a < Nv && b + 1 < Nvp) v = *reinterpret_cast<const float2 *>(src + (int64_t)a * Nvp + b);
      t[r][2 * lane] = v.x;
      t[r][2 * lane + 1] = v.y;
    }
    __syncthreads();
    for (int r = w; r < 64; r += 8) {
      const int b = tb * 64 + r, a = ta * 64 + 2 * lane;
      if (b < Nv && a + 1 < Nvp)
        *reinterpret_cast<float2 *>(dst + (int64_t)b * Nvp + a) =
            make_float2(a < Nv ? t[2 * lane][r] : 0.f, a + 1 < Nv ? t[2 * lane + 1][r] : 0.f);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- arrow sums over slices
struct ArrowWP {
  float fl[32];  // F_l,t for 1 <= l < No, else 0
  float fk[32];  // F_l,t' for l < No, else 0
};

// T, X, Y (packed i < j): OC1[q][e] = sum_{l>=1} F_lt x_lq[e] (x_lq = -x_ql for l > q), and for X
// also OX[q][e] = sum_l F_l,t' X_lq[e].  One thread per element e; rows p of stored pairs
// (p, q > p) in turn, q unrolled: x_pq adds to the column sums of q in registers and to the row
// sum of p, and output p is complete at the end of row p (its column part came from rows < p).
template <int BLK>
__global__ void __launch_bounds__(128, 4) kp_arrow_anti(PV pv, const float *__restrict__ x, float *oc1, float *ox,
                                                         const ArrowWP w) {
  const Packed &L = pv.L;
  const int No = L.No;
  constexpr bool WX = BLK == BX;
  const float *xb = x + L.boff[BLK];
  float *o1 = oc1 + (int64_t)BLK * No * L.SL;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L.SL; e += (int64_t)gridDim.x * blockDim.x) {
    float c1[32], cx[WX ? 32 : 1];
#pragma unroll
    for (int q = 0; q < 32; ++q) c1[q] = 0.f;
#pragma unroll
    for (int q = 0; q < (WX ? 32 : 1); ++q) cx[q] = 0.f;
    for (int p = 0; p < No; ++p) {
      const float *row = xb + (int64_t)(p * No - p * (p + 1) / 2 - p - 1) * L.SL + e;   // pair (p, q): row + q SL
      const float flp = w.fl[p], fkp = w.fk[p];
      float r1 = 0.f, rx = 0.f;
#pragma unroll
      for (int q = 1; q < 32; ++q) {
        if (q > p && q < No) {
          const float v = __ldg(row + (int64_t)q * L.SL);
          c1[q] += flp * v;
          r1 += w.fl[q] * v;
          if constexpr (WX) {
            cx[q] += fkp * v;
            rx += w.fk[q] * v;
          }
        }
      }
      float cp = 0.f, cxp = 0.f;
#pragma unroll
      for (int m = 0; m < 32; ++m)
        if (m == p) {
          cp = c1[m];
          if constexpr (WX) cxp = cx[m];
        }
      o1[(int64_t)p * L.SL + e] = cp - r1;
      if constexpr (WX) ox[(int64_t)p * L.SL + e] = cxp - rx;
    }
  }
}

// S, Z (every slice): OC1[m] = sum_{l>=1} F_lt x_lm, OC2[l] = sum_{m>=1} F_mt x_lm, and for Z
// OZ[l] = sum_m F_m,t' Z_lm; the column sums in registers (m unrolled), row sums per l.
template <int BLK>
__global__ void __launch_bounds__(128, 4) kp_arrow_full(PV pv, const float *__restrict__ x, float *oc1, float *oc2,
                                                         float *oz, const ArrowWP w) {
  const Packed &L = pv.L;
  const int No = L.No;
  const float *xb = x + L.boff[BLK];
  float *o1 = oc1 + (int64_t)BLK * No * L.SL;
  float *o2 = oc2 + (int64_t)(BLK == BS ? 0 : 1) * No * L.SL;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L.SL; e += (int64_t)gridDim.x * blockDim.x) {
    float c1[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) c1[m] = 0.f;
    for (int l = 0; l < No; ++l) {
      const float *row = xb + (int64_t)l * No * L.SL + e;
      const float fll = w.fl[l];
      float r2 = 0.f, rz = 0.f;
#pragma unroll
      for (int m = 0; m < 32; ++m) {
        if (m < No) {
          const float v = row[(int64_t)m * L.SL];
          c1[m] += fll * v;
          r2 += w.fl[m] * v;
          if (BLK == BZ) rz += w.fk[m] * v;
        }
      }
      o2[(int64_t)l * L.SL + e] = r2;
      if (BLK == BZ) oz[(int64_t)l * L.SL + e] = rz;
    }
#pragma unroll
    for (int m = 0; m < 32; ++m)
      if (m < No) o1[(int64_t)m * L.SL + e] = c1[m];
  }
}

// Intermediates of the N^4 coupling terms, in float32 from p (the same reductions as the
// full-storage pass of sigma.cu, on the packed slices; the coupling operator keeps the
// symmetry of its float32 coefficients):
// (a) per (k, j, b): GP[k][j][b] = sum_c F_kc (X + Z)_kj^cb,  VX[k][j][b] = sum_c F_t,c X_kj^cb
__global__ void kp_inter_a(PV pv, FF F, const float *__restrict__ x, float *GP, float *VX) {
  const Packed &L = pv.L;
  const int No = L.No, Nv = L.Nv;
  const int64_t n = (int64_t)No * No * Nv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e % Nv), kj = (int)(e / Nv), k = kj / No, j = kj % No;
    float sg;
    const float *X = pv.sl(x, BX, k, j, sg);
    const float *Z = x + L.boff[BZ] + (int64_t)kj * L.SL;
    float vx = 0.f, g = 0.f;
#pragma unroll 4
    for (int c = 0; c < Nv; ++c) {
      const float xv = X ? sg * X[(int64_t)c * L.Nvp + b] : 0.f, zv = Z[(int64_t)c * L.Nvp + b];
      vx += F.ov(0, c) * xv;
      g += F.ov(k, c) * (xv + zv);
    }
    GP[e] = g;
    VX[e] = vx;
  }
}

// (c) warp per row (i, j, a): WZ[i][j][a] = sum_c F_t,c Z_ij^ac,  HP[i][j][a] = sum_c F_jc (Y + Z)_ij^ac
__global__ void kp_inter_c(PV pv, FF F, const float *__restrict__ x, float *WZ, float *HP) {
  const Packed &L = pv.L;
  const int No = L.No, Nv = L.Nv, lane = threadIdx.x & 31;
  const int64_t rows = (int64_t)No * No * Nv;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < rows;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int a = (int)(r % Nv), ij = (int)(r / Nv), i = ij / No, j = ij % No;
    float sg;
    const float *Y = pv.sl(x, BY, i, j, sg);
    const float *Zr = x + L.boff[BZ] + (int64_t)ij * L.SL + (int64_t)a * L.Nvp;
    const float *Yr = Y ? Y + (int64_t)a * L.Nvp : nullptr;
    float wz = 0.f, hp = 0.f;
#pragma unroll 4
    for (int c = lane; c < Nv; c += 32) {
      const float zv = Zr[c], yv = Yr ? sg * Yr[c] : 0.f;
      wz += F.ov(0, c) * zv;
      hp += F.ov(j, c) * (yv + zv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      wz += __shfl_xor_sync(0xffffffffu, wz, o);
      hp += __shfl_xor_sync(0xffffffffu, hp, o);
    }
    if (lane == 0) { WZ[r] = wz; HP[r] = hp; }
  }
}

// (d) G[j][b] = sum_k GP[k][j][b];  H[i][a] = sum_k HP[i][k][a];
//     CYZ[k][c] = sum_d F_t'd Z_tk^dc - sum_l F_lt Z_lk^t'c
__global__ void kp_inter_d(PV pv, FF F, const float *__restrict__ x, const float *GP, const float *HP, float *G,
                           float *H, float *CYZ) {
  const Packed &L = pv.L;
  const int No = L.No, Nv = L.Nv;
  const int64_t n = (int64_t)No * Nv;
  const float *Zb = x + L.boff[BZ];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int part = (int)(e / n);
    const int64_t f = e % n;
    const int p = (int)(f / Nv), q = (int)(f % Nv);
    float s = 0.f;
    if (part == 0) {
      for (int k = 0; k < No; ++k) s += GP[((int64_t)k * No + p) * Nv + q];
      G[f] = s;
    } else if (part == 1) {
      for (int k = 0; k < No; ++k) s += HP[((int64_t)p * No + k) * Nv + q];
      H[f] = s;
    } else {
      const float *Z0p = Zb + (int64_t)p * L.SL;   // slice (t, k = p)
#pragma unroll 4
      for (int d = 0; d < Nv; ++d) s += F.v(0, d) * Z0p[(int64_t)d * L.Nvp + q];
      for (int l = 0; l < No; ++l) s -= F.o(l, 0) * Zb[((int64_t)l * No + p) * L.SL + q];
      CYZ[f] = s;
    }
  }
}

// ---------------------------------------------------------------- coupling pass
struct CP {
  PV pv;
  FF F;
  float omega;
  const float *x;      // p (packed)
  float *y;            // q (packed)
  const float *P;      // products of the operand rows (packed slice order, pitch Nvp)
  const float *FZ;     // F Z_s (normal orientation) for every Z slice
  const float *VX, *WZ;  // [No][No][Nv]
  const float *OC1, *OC2, *OX, *OZ, *G, *H, *CYZ;
  const float *rho;    // reduced-cost basis: [packed slice][a] sum_c x[a][c] F_t'c
  const float *kap;    // reduced-cost basis: [Z slice][b] sum_c F_t'c Z[c][b]
  double *dot;         // per-CTA partials of <x, y>_w, or nullptr
  int64_t dot_base;
};

// a slice of the packed vector through its storage: element (a, b) = sg p[a Nvp + b]; p == nullptr
// for the identically zero slices i == j of T, X, Y
struct SV {
  const float *p;
  float sg;
  __device__ __forceinline__ float at(int64_t ab) const { return p ? sg * p[ab] : 0.f; }
};
__device__ __forceinline__ SV sv(const PV &pv, const float *v, int blk, int i, int j) {
  float sg;
  const float *p = pv.sl(v, blk, i, j, sg);
  return {p, sg};
}

// (X F)_ab of the packed slice X (row pitch Nvp, row sums rs) in the reduced-cost basis, where
// F_vv is a diagonal plus the t' row and column: F_bb X_ab + X_a0 F_t'b for b >= 1, rs[a] for b = 0
__device__ __forceinline__ float xf_arrow(const FF &F, const float *xs, const float *rs, int Nvp, int a, int b) {
  return b == 0 ? rs[a] : F.v(b, b) * __ldg(xs + (int64_t)a * Nvp + b) + __ldg(xs + (int64_t)a * Nvp) * F.v(0, b);
}

// Reduced-cost basis: row sums rho[s][a] = sum_c x_s[a][c] F_t'c of every packed slice (warp per
// row) and column sums kap[z][b] = sum_c F_t'c Z_z[c][b] of the Z slices (thread per column)
__global__ void kp_vsum(PV pv, FF F, const float *__restrict__ x, float *rho, float *kap) {
  const Packed &L = pv.L;
  const int Nv = L.Nv, Nvp = L.Nvp, lane = threadIdx.x & 31;
  const int64_t rows = (int64_t)L.nslices * Nv, cols = (int64_t)L.NN * Nv;
  const int64_t nw = rows, tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = tid >> 5; r < nw; r += nth >> 5) {
    const int64_t s = r / Nv, a = r % Nv;
    const float *xr = x + s * L.SL + a * Nvp;
    float acc = 0.f;
#pragma unroll 4
    for (int c = lane; c < Nv; c += 32) acc += __ldg(xr + c) * F.v(0, c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) rho[r] = acc;
  }
  const float *Zb = x + L.boff[BZ];
  for (int64_t e = tid; e < cols; e += nth) {
    const int64_t z = e / Nv;
    const int b = (int)(e % Nv);
    const float *zc = Zb + z * L.SL + b;
    float acc = 0.f;
#pragma unroll 4
    for (int c = 0; c < Nv; ++c) acc += F.v(0, c) * __ldg(zc + (int64_t)c * Nvp);
    kap[e] = acc;
  }
}

// items [first, last) of the blocked assignment of `items` work items to this CTA
__device__ __forceinline__ void cta_items(int64_t items, int64_t &first, int64_t &last) {
  const int64_t per = (items + gridDim.x - 1) / gridDim.x;
  first = (int64_t)blockIdx.x * per;
  last = min(items, first + per);
}

// T, X, Y: work item = (slice i < j, tile pair ta <= tb); y on tile (ta, tb) and -y on
// (tb, ta).  Every slice pointer of the item is resolved once; the product tiles of the next
// item are loaded into registers while the current one is computed.  The element formulas are
// the full-storage coupling pass's (sigma.cu k_couple, arrow form) with i < j.
template <int BLK, bool AV>
__global__ void __launch_bounds__(kThreads) kp_couple_anti(CP c) {
  const Packed &L = c.pv.L;
  __shared__ float Pa[kT][kT + 1], Pb[kT][kT + 1], Ys[kT][kT + 1];
  const int nt = (L.Nv + kT - 1) / kT, npairs = nt * (nt + 1) / 2;
  const int No = L.No, Nv = L.Nv, Nvp = L.Nvp;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const FF &F = c.F;
  int64_t first, last;
  cta_items((int64_t)L.nh * npairs, first, last);
  auto decode = [&](int64_t it, int &k, int &ta, int &tb) {
    k = (int)(it / npairs);
    int tp = (int)(it % npairs);
    ta = 0;
    while (tp >= nt - ta) { tp -= nt - ta; ++ta; }
    tb = ta + tp;
  };
  float pa[4], pb[4];   // tiles (ta, tb) and (tb, ta) of the item in flight, rows ty + 8 rr
  auto fetch = [&](int64_t it) {
    int k, ta, tb;
    decode(it, k, ta, tb);
    const float *P = c.P + L.boff[BLK] + (int64_t)k * L.SL;
    const float *xs = c.x + L.boff[BLK] + (int64_t)k * L.SL;
    const float *rs = AV ? c.rho + (int64_t)(slice0(L, BLK) + k) * Nv : nullptr;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int r = ty + 8 * rr, a = ta * kT + r, b = tb * kT + tx, a2 = tb * kT + r, b2 = ta * kT + tx;
      if constexpr (AV) {
        pa[rr] = (a < Nv && b < Nv) ? xf_arrow(c.F, xs, rs, Nvp, a, b) : 0.f;
        pb[rr] = (a2 < Nv && b2 < Nv) ? xf_arrow(c.F, xs, rs, Nvp, a2, b2) : 0.f;
      } else {
        pa[rr] = (a < Nv && b < Nv) ? __ldg(P + (int64_t)a * Nvp + b) : 0.f;
        pb[rr] = (a2 < Nv && b2 < Nv) ? __ldg(P + (int64_t)a2 * Nvp + b2) : 0.f;
      }
    }
  };
  float dsum = 0.f;
  if (first < last) fetch(first);
  for (int64_t it = first; it < last; ++it) {
    int k, ta, tb;
    decode(it, k, ta, tb);
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      Pa[ty + 8 * rr][tx] = pa[rr];
      Pb[ty + 8 * rr][tx] = pb[rr];
    }
    __syncthreads();
    if (it + 1 < last) fetch(it + 1);
    int i, j;
    pair_decode(No, k, i, j);
    const int64_t so = L.boff[BLK] + (int64_t)k * L.SL;
    const float *x = c.x + so;
    float *y = c.y + so;
    // the item's slices and scalars (j >= 1 since i < j)
    const bool i0 = i == 0;
    const float cxe = -c.omega + (BLK == BT ? 0.f : F.v(0, 0) - F.o(0, 0)) - (F.o(i, i) + F.o(j, j));
    const float s1 = i0 ? 1.f : F.o(0, i), s2 = F.o(0, j);
    const float *t1p = i0 ? c.OC1 + ((int64_t)BLK * No + j) * L.SL : c.x + L.boff[BLK] + (int64_t)pair_ij(No, 0, j) * L.SL;
    const float *t2p = i0 ? nullptr : c.x + L.boff[BLK] + (int64_t)pair_ij(No, 0, i) * L.SL;   // x_i0 = -x_0i
    const float f00 = F.ov(0, 0), fi0 = F.ov(i, 0), fj0 = F.ov(j, 0);
    SV A1{}, A2{}, A3{};
    const float *r1 = nullptr, *r2 = nullptr, *r3 = nullptr;
    if (BLK == BT) {
      A1 = sv(c.pv, c.x, BX, i, j); A2 = sv(c.pv, c.x, BY, i, j);
      r1 = c.VX + ((int64_t)i * No + j) * Nv;
      if (i0) { r2 = c.OX + (int64_t)j * L.SL; r3 = c.G + (int64_t)j * Nv; }
    } else if (BLK == BX) {
      A1 = sv(c.pv, c.x, BT, i, j); A2 = sv(c.pv, c.x, BT, 0, j); A3 = sv(c.pv, c.x, BT, 0, i);
    } else {
      A1 = sv(c.pv, c.x, BT, i, j); A2 = sv(c.pv, c.x, BS, 0, i); A3 = sv(c.pv, c.x, BS, 0, j);
      if (i0) r1 = c.CYZ + (int64_t)j * Nv;
    }
    const int b = tb * kT + tx;
    const float fob0 = b < Nv ? F.ov(0, b) : 0.f, fobi = b < Nv ? F.ov(i, b) : 0.f, fobj = b < Nv ? F.ov(j, b) : 0.f;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int r = ty + 8 * rr, a = ta * kT + r;
      float yv = 0.f;
      const bool upper = ta < tb || r < tx;
      if (a < Nv && b < Nv && upper && valid_elem(BLK, i, j, a, b)) {
        const int64_t ab = (int64_t)a * Nvp + b;
        const float xe = __ldg(x + ab);
        float u = cxe * xe - s1 * __ldg(t1p + ab) + (t2p ? s2 * __ldg(t2p + ab) : 0.f);
        if (BLK == BT) {
          u += f00 * (A1.at(ab) + A2.at(ab));
          if (a == 0) u -= r1[b];
          if (b == 0) u += r1[a];
          if (i0) {
            u -= r2[ab];
            if (a == 0) u += r3[b];
            if (b == 0) u -= r3[a];
          }
        } else if (BLK == BX) {
          const float foa0 = F.ov(0, a), foai = F.ov(i, a), foaj = F.ov(j, a);
          u += f00 * A1.at(ab) - foa0 * A1.at(b) + fob0 * A1.at(a) - fi0 * A2.at(ab) + fj0 * A3.at(ab) +
               foai * A2.at(b) - foaj * A3.at(b) - fobi * A2.at(a) + fobj * A3.at(a);
        } else {
          u += f00 * A1.at(ab) + fobj * A2.at(a) - fobi * A3.at(a) - F.ov(j, a) * A2.at(b) + F.ov(i, a) * A3.at(b);
          if (i0) {
            if (a == 0) u += r1[b];
            if (b == 0) u -= r1[a];
          }
        }
        yv = Pa[r][tx] - Pb[tx][r] + u;
        dsum += 2.f * xe * yv;
      }
      if (a < Nv && b < Nv && (ta < tb || r <= tx)) y[(int64_t)a * Nvp + b] = yv;
      Ys[r][tx] = -yv;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {   // element (tb*32 + r, ta*32 + tx) = -y(ta*32 + tx, tb*32 + r)
      const int r = ty + 8 * rr, a = tb * kT + r, bb = ta * kT + tx;
      if (a < Nv && bb < Nv && (ta < tb || r > tx)) y[(int64_t)a * Nvp + bb] = Ys[tx][r];
    }
    __syncthreads();
  }
  if (c.dot) cta_partial((double)dsum, c.dot, c.dot_base + blockIdx.x);
}

// S: work item = (slice pair i <= j, tile (ta, tb)); y_ij on tile (ta, tb), y_ji = y_ij^T.  The
// tiles read transposed (P_ji, Z_ji and, for i = 0, OZ_j) of the next item are loaded into
// registers while the current one is computed.
template <bool AV>
__global__ void __launch_bounds__(kThreads, 4) kp_couple_s(CP c) {
  const Packed &L = c.pv.L;
  __shared__ float Pa[kT][kT + 1], Pb[kT][kT + 1], Zt[kT][kT + 1], Ot[kT][kT + 1], Ys[kT][kT + 1];
  const int nt = (L.Nv + kT - 1) / kT, No = L.No, Nv = L.Nv, Nvp = L.Nvp;
  const int npair = No * (No + 1) / 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const FF &F = c.F;
  int64_t first, last;
  cta_items((int64_t)npair * nt * nt, first, last);
  auto decode = [&](int64_t it, int &i, int &j, int &ta, int &tb) {
    int pi = (int)(it / (nt * nt));
    const int tt = (int)(it % (nt * nt));
    ta = tt / nt;
    tb = tt % nt;
    i = 0;
    while (pi >= No - i) { pi -= No - i; ++i; }
    j = i + pi;   // i <= j
  };
  float pa[4], pb[4], zt[4], ot[4];
  auto fetch = [&](int64_t it) {
    int i, j, ta, tb;
    decode(it, i, j, ta, tb);
    const int64_t sij = L.boff[BS] + ((int64_t)i * No + j) * L.SL, sji = L.boff[BS] + ((int64_t)j * No + i) * L.SL;
    const float *Zji = c.x + L.boff[BZ] + ((int64_t)j * No + i) * L.SL, *OZj = c.OZ + (int64_t)j * L.SL;
    const float *rij = AV ? c.rho + (int64_t)(slice0(L, BS) + i * No + j) * Nv : nullptr;
    const float *rji = AV ? c.rho + (int64_t)(slice0(L, BS) + j * No + i) * Nv : nullptr;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int r = ty + 8 * rr, a = ta * kT + r, b = tb * kT + tx, a2 = tb * kT + r, b2 = ta * kT + tx;
      const bool in1 = a < Nv && b < Nv, in2 = a2 < Nv && b2 < Nv;
      const int64_t e2 = (int64_t)a2 * Nvp + b2;
      if constexpr (AV) {
        pa[rr] = in1 ? xf_arrow(c.F, c.x + sij, rij, Nvp, a, b) : 0.f;
        pb[rr] = in2 ? xf_arrow(c.F, c.x + sji, rji, Nvp, a2, b2) : 0.f;
      } else {
        pa[rr] = in1 ? __ldg(c.P + sij + (int64_t)a * Nvp + b) : 0.f;
        pb[rr] = in2 ? __ldg(c.P + sji + e2) : 0.f;
      }
      zt[rr] = in2 ? __ldg(Zji + e2) : 0.f;
      ot[rr] = (in2 && i == 0) ? __ldg(OZj + e2) : 0.f;
    }
  };
  float dsum = 0.f;
  if (first < last) fetch(first);
  for (int64_t it = first; it < last; ++it) {
    int i, j, ta, tb;
    decode(it, i, j, ta, tb);
    if (i == j && ta > tb) {   // the mirror of an item already covered (uniform over the CTA)
      if (it + 1 < last) fetch(it + 1);
      continue;
    }
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int r = ty + 8 * rr;
      Pa[r][tx] = pa[rr];
      Pb[r][tx] = pb[rr];
      Zt[r][tx] = zt[rr];
      Ot[r][tx] = ot[rr];
    }
    __syncthreads();
    if (it + 1 < last) fetch(it + 1);
    const int64_t sij = L.boff[BS] + ((int64_t)i * No + j) * L.SL, sji = L.boff[BS] + ((int64_t)j * No + i) * L.SL;
    const float *Zij = c.x + L.boff[BZ] + ((int64_t)i * No + j) * L.SL;
    const float *OZi = c.OZ + (int64_t)i * L.SL;
    const bool i0 = i == 0, j0 = j == 0;
    const float cxe = -c.omega - (F.o(i, i) + F.o(j, j));
    const float s1 = i0 ? 1.f : F.o(0, i), s2 = j0 ? 1.f : F.o(0, j), f00 = F.ov(0, 0);
    const float *t1p = i0 ? c.OC1 + ((int64_t)BS * No + j) * L.SL : c.x + L.boff[BS] + (int64_t)j * L.SL;
    const float *t2p = j0 ? c.OC2 + (int64_t)i * L.SL : c.x + L.boff[BS] + (int64_t)i * No * L.SL;
    const float *WZji = c.WZ + ((int64_t)j * No + i) * Nv, *WZij = c.WZ + ((int64_t)i * No + j) * Nv;
    const float *Hj = c.H + (int64_t)j * Nv, *Hi = c.H + (int64_t)i * Nv;
    const bool diag = i == j && ta == tb;
    const int b = tb * kT + tx;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int r = ty + 8 * rr, a = ta * kT + r;
      float yv = 0.f;
      if (a < Nv && b < Nv && (!diag || r <= tx)) {
        const int64_t ab = (int64_t)a * Nvp + b;
        const float xe = __ldg(c.x + sij + ab);
        float u = cxe * xe - s1 * __ldg(t1p + ab) - s2 * __ldg(t2p + ab) + f00 * (__ldg(Zij + ab) + Zt[tx][r]);
        if (a == 0) u -= WZji[b];
        if (b == 0) u -= WZij[a];
        if (j0) {
          u -= OZi[ab];
          if (b == 0) u += Hi[a];
        }
        if (i0) {
          u -= Ot[tx][r];
          if (a == 0) u += Hj[b];
        }
        yv = Pa[r][tx] + Pb[tx][r] + u;
        dsum += (diag && r == tx ? 1.f : 2.f) * xe * yv;
        c.y[sij + ab] = yv;
      }
      Ys[r][tx] = yv;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {   // y_ji[tb*32 + r][ta*32 + tx] = y_ij[ta*32 + tx][tb*32 + r]
      const int r = ty + 8 * rr, a = tb * kT + r, bb = ta * kT + tx;
      if (a < Nv && bb < Nv && (!diag || r > tx)) c.y[sji + (int64_t)a * Nvp + bb] = Ys[tx][r];
    }
    __syncthreads();
  }
  if (c.dot) cta_partial((double)dsum, c.dot, c.dot_base + blockIdx.x);
}

// Z: one thread per 16-byte group of four columns of one row (slice (i, j), row a); no shared
// memory, every load of a group issued before its arithmetic.  y = P + F Z + couplings.
__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float g4(const float4 &v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }

template <bool AV>
__global__ void __launch_bounds__(kThreads, AV ? 3 : 4) kp_couple_z(CP c) {
  const Packed &L = c.pv.L;
  const int No = L.No, Nv = L.Nv, Nvp = L.Nvp, nb4 = Nvp >> 2;
  const FF &F = c.F;
  const int64_t units = (int64_t)L.NN * Nv * nb4;
  float dsum = 0.f;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = u / nb4;
    const int b = (int)(u - row * nb4) * 4;
    const int s = (int)(row / Nv), a = (int)(row - (int64_t)s * Nv);
    const int i = s / No, j = s - i * No;
    const int64_t so = L.boff[BZ] + (int64_t)s * L.SL, ab = (int64_t)a * Nvp + b;
    float out[4] = {0.f, 0.f, 0.f, 0.f};
    if (j != 0) {   // j == 0: not amplitudes (the down t hole twice)
      const bool i0 = i == 0;
      const float *Sij = c.x + L.boff[BS] + (int64_t)s * L.SL, *Si0 = c.x + L.boff[BS] + (int64_t)i * No * L.SL;
      const float *T0j = c.x + L.boff[BT] + (int64_t)pair_ij(No, 0, j) * L.SL;   // row 0 used
      const float *Y0j = c.x + L.boff[BY] + (int64_t)pair_ij(No, 0, j) * L.SL;
      const float *t1p = i0 ? c.OC1 + ((int64_t)BZ * No + j) * L.SL : c.x + L.boff[BZ] + (int64_t)j * L.SL;
      const float *t2p = c.x + L.boff[BZ] + (int64_t)i * No * L.SL;   // Z_i0
      const float4 xe = ld4(c.x + so + ab);
      float4 p4, fz;
      if constexpr (AV) {   // X F and F X of the slice from the arrow form of F_vv
        const float *xs = c.x + so;
        const float xa0 = __ldg(xs + (int64_t)a * Nvp), ra = c.rho[(int64_t)(slice0(L, BZ) + s) * Nv + a];
        const float4 x0b = ld4(xs + b);
        const float fa = F.v(0, a), da = F.v(a, a);
        float pv[4], fv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int bq = b + q;
          const bool in = bq < Nv;
          pv[q] = !in ? 0.f : bq == 0 ? ra : F.v(bq, bq) * g4(xe, q) + xa0 * F.v(0, bq);
          fv[q] = !in ? 0.f : a == 0 ? c.kap[(int64_t)s * Nv + bq] : da * g4(xe, q) + fa * g4(x0b, q);
        }
        p4 = make_float4(pv[0], pv[1], pv[2], pv[3]);
        fz = make_float4(fv[0], fv[1], fv[2], fv[3]);
      } else {
        p4 = ld4(c.P + so + ab);
        fz = ld4(c.FZ + (int64_t)s * L.SL + ab);
      }
      const float4 t1 = ld4(t1p + ab), t2 = ld4(t2p + ab), sa = ld4(Sij + ab), s0 = ld4(Si0 + ab);
      const float4 t0 = ld4(T0j + b), y0 = ld4(Y0j + b);
      const float sija0 = __ldg(Sij + (int64_t)a * Nvp), si0a0 = __ldg(Si0 + (int64_t)a * Nvp);
      const float cxe = -c.omega + (F.v(0, 0) - F.o(0, 0)) - (F.o(i, i) + F.o(j, j));
      const float s1 = i0 ? 1.f : F.o(0, i), s2 = F.o(0, j), f00 = F.ov(0, 0), fj0 = F.ov(j, 0), foi = F.o(0, i);
      const float foai = F.ov(i, a), fva = F.v(a, 0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int bq = b + q;
        if (bq < Nv && bq != 0 && !(i0 && a == 0)) {
          const float x0 = g4(xe, q), yb = g4(y0, q);
          float yv = g4(p4, q) + g4(fz, q) + cxe * x0 - s1 * g4(t1, q) - s2 * g4(t2, q) + f00 * g4(sa, q) -
                     F.ov(0, bq) * sija0 - fj0 * g4(s0, q) + F.ov(j, bq) * si0a0 + foai * g4(t0, q);
          if (i0) yv += fva * yb;
          if (a == 0) yv -= foi * yb;
          dsum += 2.f * x0 * yv;
          out[q] = yv;
        }
      }
    }
    *reinterpret_cast<float4 *>(c.y + so + ab) = make_float4(out[0], out[1], out[2], out[3]);
  }
  if (c.dot) cta_partial((double)dsum, c.dot, c.dot_base + blockIdx.x);
}

// ---------------------------------------------------------------- rotated Jacobi preconditioner
// z = R~ D~^-1 R~^T r R~ R~^T slice by slice: R~ = diag(1, V) rotates the virtual orbitals other
// than t' to the eigenvectors of F_vv (t' fixed, so the masks keep their positions), D~ is the
// diagonal of A in that basis (the Jacobi preconditioner of the reduced-cost basis).  D and L
// do not change under that rotation, so M^-1 A has the spectrum the reduced-cost basis solve
// sees; the rotations run as bf16 tcgen05 GEMMs (vgemm.cu), the result is projected back onto
// the singlet subspace with the masks (the rotations' rounding is not symmetric).

__device__ __forceinline__ void st_bf4(__nv_bfloat16 *p4, float4 v) {
  __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
  uint2 u;
  u.x = *reinterpret_cast<uint32_t *>(&a);
  u.y = *reinterpret_cast<uint32_t *>(&b);
  *reinterpret_cast<uint2 *>(p4) = u;
}

// start of an inner solve: r = r64 on the packed slots, rb = bf16(r), d = 0; partials <r, r>_w.
// One warp per packed row (slice, a), four consecutive b per lane.
__global__ void __launch_bounds__(256) kp_init_rj(PV pv, const double *r64, float *r, __nv_bfloat16 *rb, float *d,
                                                  double *red) {
  const Packed &L = pv.L;
  const int64_t rows = (int64_t)L.nslices * L.Nv, NvNv = (int64_t)L.Nv * L.Nv, B = (int64_t)L.NN * NvNv;
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5, q4 = L.Nvp >> 2, Nv = L.Nv;
  float a1 = 0.f;
  for (int64_t row = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); row < rows; row += (int64_t)gridDim.x * wpb) {
    const int s = (int)(row / Nv), a = (int)(row % Nv);
    int blk, i, j;
    pv.decode(s, blk, i, j);
    const double *src = r64 + blk * B + ((int64_t)i * L.No + j) * NvNv + (int64_t)a * Nv;
    const int64_t e0 = (int64_t)s * L.SL + (int64_t)a * L.Nvp;
    const float w = blk_w(blk);
    for (int c = lane; c < q4; c += 32) {
      const int b = 4 * c;
      float4 v;
      v.x = b < Nv ? (float)src[b] : 0.f;
      v.y = b + 1 < Nv ? (float)src[b + 1] : 0.f;
      v.z = b + 2 < Nv ? (float)src[b + 2] : 0.f;
      v.w = b + 3 < Nv ? (float)src[b + 3] : 0.f;
      *reinterpret_cast<float4 *>(r + e0 + b) = v;
      st_bf4(rb + e0 + b, v);
      *reinterpret_cast<float4 *>(d + e0 + b) = make_float4(0.f, 0.f, 0.f, 0.f);
      a1 += w * (v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w);
    }
  }
  double v[1] = {(double)a1};
  cta_partials<1>(v, red);
}

// r -= alpha q, rb = bf16(r); partials <r, r>_w
__global__ void kp_update_rj(PV pv, const double *slots, float *r, const float *q, __nv_bfloat16 *rb, double *red) {
  const Packed &L = pv.L;
  const float alpha = (float)slots[4];
  const int64_t n4 = L.n >> 2, z4 = L.boff[BZ] >> 2;
  float4 *r4 = reinterpret_cast<float4 *>(r);
  const float4 *q4 = reinterpret_cast<const float4 *>(q);
  float a1 = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x) {
    float4 rv = r4[e];
    const float4 qv = __ldg(q4 + e);
    rv.x -= alpha * qv.x; rv.y -= alpha * qv.y; rv.z -= alpha * qv.z; rv.w -= alpha * qv.w;
    r4[e] = rv;
    st_bf4(rb + 4 * e, rv);
    a1 += (e >= z4 ? 2.f : 1.f) * (rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w);
  }
  double v[1] = {(double)a1};
  cta_partials<1>(v, red);
}

// d += alpha p; p = z + beta p; pb = bf16(p) (if kept)
__global__ void kp_p_rj(PV pv, const double *slots, const float *z, float *p, float *d, __nv_bfloat16 *pb) {
  const Packed &L = pv.L;
  const float alpha = (float)slots[4], beta = (float)slots[5];
  const int64_t n4 = L.n >> 2;
  const float4 *z4 = reinterpret_cast<const float4 *>(z);
  float4 *p4 = reinterpret_cast<float4 *>(p), *d4 = reinterpret_cast<float4 *>(d);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x) {
    const float4 pv4 = p4[e], zv = __ldg(z4 + e);
    float4 dv = d4[e];
    dv.x += alpha * pv4.x; dv.y += alpha * pv4.y; dv.z += alpha * pv4.z; dv.w += alpha * pv4.w;
    d4[e] = dv;
    const float4 pn = make_float4(zv.x + beta * pv4.x, zv.y + beta * pv4.y, zv.z + beta * pv4.z, zv.w + beta * pv4.w);
    p4[e] = pn;
    if (pb) st_bf4(pb + 4 * e, pn);
  }
}

// z projected onto the singlet subspace with the masks, in place; partials of <r, z>_w
// (r has the symmetries exactly).  T, X, Y: tile pairs, w_ab = (z_ab - z_ba) / 2, w_ba = -w_ab.
template <int BLK>
__global__ void __launch_bounds__(kThreads) kp_proj_anti(PV pv, float *z, const float *r, double *red, int64_t base) {
  const Packed &L = pv.L;
  __shared__ float Za[kT][kT + 1], Zb[kT][kT + 1], Ws[kT][kT + 1];
  const int nt = (L.Nv + kT - 1) / kT, npairs = nt * (nt + 1) / 2;
  const int No = L.No, Nv = L.Nv, Nvp = L.Nvp;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  int64_t first, last;
  cta_items((int64_t)L.nh * npairs, first, last);
  float dsum = 0.f;
  for (int64_t it = first; it < last; ++it) {
    const int k = (int)(it / npairs);
    int tp = (int)(it % npairs), ta = 0;
    while (tp >= nt - ta) { tp -= nt - ta; ++ta; }
    const int tb = ta + tp;
    int i, j;
    pair_decode(No, k, i, j);
    const int64_t so = L.boff[BLK] + (int64_t)k * L.SL;
    float *zs = z + so;
    const float *rs = r + so;
    float rv[4];   // r on the tile (ta, tb), loaded with the z tiles
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int q = ty + 8 * rr, a = ta * kT + q, b = tb * kT + tx, a2 = tb * kT + q, b2 = ta * kT + tx;
      const bool in = a < Nv && b < Nv;
      Za[q][tx] = in ? zs[(int64_t)a * Nvp + b] : 0.f;
      rv[rr] = in ? __ldg(rs + (int64_t)a * Nvp + b) : 0.f;
      Zb[q][tx] = (a2 < Nv && b2 < Nv) ? zs[(int64_t)a2 * Nvp + b2] : 0.f;
    }
    __syncthreads();
    const int b = tb * kT + tx;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int q = ty + 8 * rr, a = ta * kT + q;
      float w = 0.f;
      if (a < Nv && b < Nv && (ta < tb || q < tx) && valid_elem(BLK, i, j, a, b)) {
        w = 0.5f * (Za[q][tx] - Zb[tx][q]);
        dsum += 2.f * w * rv[rr];
      }
      if (a < Nv && b < Nv && (ta < tb || q <= tx)) zs[(int64_t)a * Nvp + b] = w;
      Ws[q][tx] = -w;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int q = ty + 8 * rr, a = tb * kT + q, bb = ta * kT + tx;
      if (a < Nv && bb < Nv && (ta < tb || q > tx)) zs[(int64_t)a * Nvp + bb] = Ws[tx][q];
    }
    __syncthreads();
  }
  cta_partial((double)dsum, red, base + blockIdx.x);
}

// S: w = (z_ij^ab + z_ji^ba) / 2 on both images
__global__ void __launch_bounds__(kThreads) kp_proj_s(PV pv, float *z, const float *r, double *red, int64_t base) {
  const Packed &L = pv.L;
  __shared__ float Za[kT][kT + 1], Zb[kT][kT + 1], Ws[kT][kT + 1];
  const int nt = (L.Nv + kT - 1) / kT, No = L.No, Nv = L.Nv, Nvp = L.Nvp;
  const int npair = No * (No + 1) / 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  int64_t first, last;
  cta_items((int64_t)npair * nt * nt, first, last);
  float dsum = 0.f;
  for (int64_t it = first; it < last; ++it) {
    int pi = (int)(it / (nt * nt));
    const int tt = (int)(it % (nt * nt)), ta = tt / nt, tb = tt % nt;
    int i = 0;
    while (pi >= No - i) { pi -= No - i; ++i; }
    const int j = i + pi;
    if (i == j && ta > tb) continue;
    float *zij = z + L.boff[BS] + ((int64_t)i * No + j) * L.SL, *zji = z + L.boff[BS] + ((int64_t)j * No + i) * L.SL;
    const float *rij = r + L.boff[BS] + ((int64_t)i * No + j) * L.SL;
    float rv[4];   // r_ij on the tile (ta, tb), loaded with the z tiles
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int q = ty + 8 * rr, a = ta * kT + q, b = tb * kT + tx, a2 = tb * kT + q, b2 = ta * kT + tx;
      const bool in = a < Nv && b < Nv;
      Za[q][tx] = in ? zij[(int64_t)a * Nvp + b] : 0.f;
      rv[rr] = in ? __ldg(rij + (int64_t)a * Nvp + b) : 0.f;
      Zb[q][tx] = (a2 < Nv && b2 < Nv) ? zji[(int64_t)a2 * Nvp + b2] : 0.f;
    }
    __syncthreads();
    const bool diag = i == j && ta == tb;
    const int b = tb * kT + tx;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int q = ty + 8 * rr, a = ta * kT + q;
      float w = 0.f;
      if (a < Nv && b < Nv && (!diag || q <= tx)) {
        w = 0.5f * (Za[q][tx] + Zb[tx][q]);
        dsum += (diag && q == tx ? 1.f : 2.f) * w * rv[rr];
        zij[(int64_t)a * Nvp + b] = w;
      }
      Ws[q][tx] = w;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {   // z_ji[tb*32 + q][ta*32 + tx] = w_ij[ta*32 + tx][tb*32 + q]
      const int q = ty + 8 * rr, a = tb * kT + q, bb = ta * kT + tx;
      if (a < Nv && bb < Nv && (!diag || q > tx)) zji[(int64_t)a * Nvp + bb] = Ws[tx][q];
    }
    __syncthreads();
  }
  cta_partial((double)dsum, red, base + blockIdx.x);
}

// Z: masks only (no symmetry between Z slices); weight 2.  Four consecutive b per thread (Nvp
// is a multiple of 8, so a float4 never straddles two rows).
__global__ void kp_proj_z(PV pv, float *z, const float *r, double *red, int64_t base) {
  const Packed &L = pv.L;
  const int No = L.No, Nv = L.Nv, q4 = L.Nvp >> 2;
  const int64_t units = (int64_t)L.NN * Nv * q4;
  float4 *zb = reinterpret_cast<float4 *>(z + L.boff[BZ]);
  const float4 *rb = reinterpret_cast<const float4 *>(r + L.boff[BZ]);
  float dsum = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < units; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / q4;   // Z row (slice s = row / Nv, virtual a = row % Nv)
    const int b0 = (int)(e - row * q4) * 4;
    const int s = (int)(row / Nv), a = (int)(row - (int64_t)s * Nv);
    const int i = s / No, j = s - i * No;
    const bool rowok = j != 0 && !(i == 0 && a == 0);   // the Z masks of valid_elem
    float4 v = zb[e];
    const float4 rv = __ldg(rb + e);
    v.x = (rowok && b0 != 0 && b0 < Nv) ? v.x : 0.f;
    v.y = (rowok && b0 + 1 < Nv) ? v.y : 0.f;
    v.z = (rowok && b0 + 2 < Nv) ? v.z : 0.f;
    v.w = (rowok && b0 + 3 < Nv) ? v.w : 0.f;
    zb[e] = v;
    dsum += 2.f * (v.x * rv.x + v.y * rv.y + v.z * rv.z + v.w * rv.w);
  }
  cta_partial((double)dsum, red, base + blockIdx.x);
}

// <u, v>_w over a packed vector (per-CTA partials)
__global__ void kp_wdot(PV pv, const float *u, const float *v, double *red) {
  const Packed &L = pv.L;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L.n; e += (int64_t)gridDim.x * blockDim.x)
    acc += (e >= L.boff[BZ] ? 2.0 : 1.0) * (double)u[e] * (double)v[e];
  cta_partial(acc, red, blockIdx.x);
}

// coupling-pass grid (per launch); the partials of <x, y> are one per CTA and launch
constexpr int kCoupleGrid = 1216;

}  // namespace

int64_t packed_dot_parts(const esmp2_handle *h) { (void)h; return 5LL * kCoupleGrid; }

// The right operand W = F_vv of the contraction (rows b, columns c, row pitch Nvp; F_vv is
// symmetric) in bf16 or float32, from the float64 Fock matrix of the working basis.
static esmp2_status packed_right_operand(esmp2_handle *h, bool f32, void *dst) {
  const Packed &L = h->pk;
  const int No = L.No, N = h->d.N;
  std::vector<double> hF((size_t)N * N);
  cudaError_t e = cudaMemcpyAsync(hF.data(), h->Fsemi, sizeof(double) * hF.size(), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "packed set-up");
  const size_t n = (size_t)L.Nv * L.Nvp;
  std::vector<float> W32(f32 ? n : 0, 0.f);
  std::vector<__nv_bfloat16> W16(f32 ? 0 : n, __float2bfloat16_rn(0.f));
  for (int b = 0; b < L.Nv; ++b)
    for (int cc = 0; cc < L.Nv; ++cc) {
      const double v = hF[(size_t)(No + b) * N + No + cc];
      if (f32) W32[(size_t)b * L.Nvp + cc] = (float)v;
      else W16[(size_t)b * L.Nvp + cc] = __float2bfloat16_rn((float)v);
    }
  e = f32 ? cudaMemcpyAsync(dst, W32.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->stream)
          : cudaMemcpyAsync(dst, W16.data(), sizeof(__nv_bfloat16) * n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? ESMP2_OK : check_cuda(h, e, "packed set-up");
}

// Buffers of the packed inner solve; F32 / Fsemi must be ready (ensure_mixed).  The operand
// of the kind h->tf32 asks for (bf16 copy, or float32 holding p itself) is allocated on first
// use; both kinds can live on one handle.
esmp2_status packed_setup(esmp2_handle *h) {
  cudaError_t e = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(p, bytes ? bytes : 16, h->stream);
  };
  if (!h->pr) {
    const Packed L = make_packed(h->d.No, h->d.Nv);
    h->pk = L;
    const int No = L.No;
    A(reinterpret_cast<void **>(&h->pr), sizeof(float) * (size_t)L.n);
    A(reinterpret_cast<void **>(&h->pp), sizeof(float) * (size_t)L.n);
    A(reinterpret_cast<void **>(&h->pq), sizeof(float) * (size_t)L.n);
    A(reinterpret_cast<void **>(&h->pd), sizeof(float) * (size_t)L.n);
    A(reinterpret_cast<void **>(&h->pdinv), sizeof(__half) * (size_t)L.n);
    A(reinterpret_cast<void **>(&h->pP), sizeof(float) * (size_t)(L.n + (int64_t)L.NN * L.SL));
    A(reinterpret_cast<void **>(&h->pVX), sizeof(float) * (size_t)No * No * L.Nv);
    A(reinterpret_cast<void **>(&h->pGP), sizeof(float) * (size_t)No * No * L.Nv);
    A(reinterpret_cast<void **>(&h->pWZ), sizeof(float) * (size_t)No * No * L.Nv);
    A(reinterpret_cast<void **>(&h->pHP), sizeof(float) * (size_t)No * No * L.Nv);
    A(reinterpret_cast<void **>(&h->pOC), sizeof(float) * (size_t)5 * No * L.SL);
    A(reinterpret_cast<void **>(&h->pOC2), sizeof(float) * (size_t)2 * No * L.SL);
    A(reinterpret_cast<void **>(&h->pOX), sizeof(float) * (size_t)No * L.SL);
    A(reinterpret_cast<void **>(&h->pOZ), sizeof(float) * (size_t)No * L.SL);
    A(reinterpret_cast<void **>(&h->pG), sizeof(float) * (size_t)No * L.Nv);
    A(reinterpret_cast<void **>(&h->pH), sizeof(float) * (size_t)No * L.Nv);
    A(reinterpret_cast<void **>(&h->pCYZ), sizeof(float) * (size_t)No * L.Nv);
    h->pdot_n = (int)packed_dot_parts(h);
    A(reinterpret_cast<void **>(&h->pdot), sizeof(double) * (size_t)h->pdot_n);
    if (e != cudaSuccess) return check_cuda(h, e, "packed inner buffers");
    // q's and p's pad columns start (and stay) zero
    cudaMemsetAsync(h->pq, 0, sizeof(float) * (size_t)L.n, h->stream);
    cudaMemsetAsync(h->pp, 0, sizeof(float) * (size_t)L.n, h->stream);
    h->packed = true;
    if ((e = cudaGetLastError()) != cudaSuccess) return check_cuda(h, e, "packed set-up");
  }
  const Packed &L = h->pk;
  // the preconditioner of the basis of this call (semicanonical-occupied or reduced-cost)
  const int basis = h->arrowv ? 2 : 1;
  if (h->pdinv_basis != basis) {
    FF F{h->arrowv ? h->F32arr : h->F32, h->d.N, L.No};
    kp_dinv<<<2432, 128, 0, h->stream>>>(PV{L}, F, (float)h->omega_op, h->pdinv);
    h->launches += 1;
    h->pdinv_basis = basis;
  }
  if (h->arrowv && !h->pRho) {
    A(reinterpret_cast<void **>(&h->pRho), sizeof(float) * (size_t)L.nslices * L.Nv);
    A(reinterpret_cast<void **>(&h->pKap), sizeof(float) * (size_t)L.NN * L.Nv);
    if (e != cudaSuccess) return check_cuda(h, e, "packed reduced-basis sums");
  }
  const size_t op_elems = (size_t)(L.n + (int64_t)L.NN * L.SL);
  if (h->arrowv) {
    // no contraction operand in the reduced-cost basis
  } else if (h->tf32 && !h->pop32) {
    A(reinterpret_cast<void **>(&h->pop32), sizeof(float) * op_elems);
    A(reinterpret_cast<void **>(&h->pW32), sizeof(float) * (size_t)L.Nv * L.Nvp);
    if (e != cudaSuccess) return check_cuda(h, e, "packed tf32 operand");
    // pad columns and the transposed-Z part start (and stay) zero
    cudaMemsetAsync(h->pop32, 0, sizeof(float) * op_elems, h->stream);
    if (esmp2_status s = packed_right_operand(h, true, h->pW32)) return s;
  } else if (!h->tf32 && !h->pop) {
    A(&h->pop, sizeof(__nv_bfloat16) * op_elems);
    A(&h->pW, sizeof(__nv_bfloat16) * (size_t)L.Nv * L.Nvp);
    if (e != cudaSuccess) return check_cuda(h, e, "packed bf16 operand");
    cudaMemsetAsync(h->pop, 0, sizeof(__nv_bfloat16) * op_elems, h->stream);
    if (esmp2_status s = packed_right_operand(h, false, h->pW)) return s;
  }
  return check_cuda(h, cudaGetLastError(), "packed set-up");
}

// the inner PCG's p: the float32 operand itself for tf32, else its own vector
float *packed_p(esmp2_handle *h) { return h->tf32 && !h->arrowv ? h->pop32 : h->pp; }

esmp2_status vgemm(esmp2_handle *h, const void *A, int64_t rows, int64_t rows_normal, const void *W, float *P,
                   float *PT, int ldp, double alg_flops, bool tf32, const VgemmOut *out = nullptr);

// q = A p on the packed layout (bf16 or tf32 virtual-index terms, float32 everything else);
// pb_ready: the PCG update already wrote the operand (bf16(p), or p itself in the float32
// operand for tf32); dot: per-CTA partials of <p, q>_w (packed_dot_parts(h) doubles) or nullptr.
// stages (profiling): bit 0 operand conversion, bit 1 contraction, bit 2 coupling pass.
esmp2_status sigma_packed(esmp2_handle *h, const float *p, float *q, bool pb_ready, double *dot, int stages) {
  const Packed &L = h->pk;
  const int No = L.No, N = h->d.N;
  PV pv{L};
  cudaStream_t st = h->stream;
  const bool av = h->arrowv, tf32 = h->tf32 && !av;
  FF F{av ? h->F32arr : h->F32, N, No};
  __nv_bfloat16 *op = static_cast<__nv_bfloat16 *>(h->pop);
  if (av) {   // reduced-cost basis: the virtual-index terms need only row / column sums
    if (stages & 2) {
      kp_vsum<<<1216, 256, 0, st>>>(pv, F, p, h->pRho, h->pKap);
      h->launches += 1;
    }
  } else if (!pb_ready && (stages & 1)) {  // the packed p to the operand (pad columns are zero in p)
    if (tf32) {
      if (p != h->pop32) {
        if (cudaError_t e = cudaMemcpyAsync(h->pop32, p, sizeof(float) * (size_t)L.n, cudaMemcpyDeviceToDevice, st))
          return check_cuda(h, e, "sigma_packed operand");
      }
    } else {
      kp_bf16<<<1216, 256, 0, st>>>(p, op, L.n);
      h->launches += 1;
    }
  }
  const int64_t rows_n = (int64_t)L.nslices * L.Nv, rows = rows_n + (int64_t)L.NN * L.Nv;
  if (!av && (stages & 2)) {
    if (tf32) kp_zt32<<<1216, 256, 0, st>>>(pv, h->pop32);
    else kp_zt<<<1216, 256, 0, st>>>(pv, op);
    h->launches += 1;
    if (esmp2_status s = vgemm(h, tf32 ? static_cast<const void *>(h->pop32) : static_cast<const void *>(op), rows,
                               rows_n, tf32 ? static_cast<const void *>(h->pW32) : h->pW, h->pP, h->pP + L.n, L.Nvp,
                               alg_virtual_flops(No, L.Nv), tf32))
      return s;
  }
  if (!(stages & 4)) return check_cuda(h, cudaGetLastError(), "sigma_packed");
  ArrowWP w{};
  for (int l = 0; l < 32; ++l) { w.fl[l] = h->arrow_w[l]; w.fk[l] = h->arrow_w[32 + l]; }
  {
    const unsigned ga = (unsigned)std::min<int64_t>(cdiv(L.SL, 128), 4096);
    kp_arrow_anti<BT><<<ga, 128, 0, st>>>(pv, p, h->pOC, h->pOX, w);
    kp_arrow_anti<BX><<<ga, 128, 0, st>>>(pv, p, h->pOC, h->pOX, w);
    kp_arrow_anti<BY><<<ga, 128, 0, st>>>(pv, p, h->pOC, h->pOX, w);
    kp_arrow_full<BS><<<ga, 128, 0, st>>>(pv, p, h->pOC, h->pOC2, h->pOZ, w);
    kp_arrow_full<BZ><<<ga, 128, 0, st>>>(pv, p, h->pOC, h->pOC2, h->pOZ, w);
  }
  kp_inter_a<<<1216, 256, 0, st>>>(pv, F, p, h->pGP, h->pVX);
  kp_inter_c<<<1216, 256, 0, st>>>(pv, F, p, h->pWZ, h->pHP);
  kp_inter_d<<<(unsigned)cdiv(3LL * No * L.Nv, 256), 256, 0, st>>>(pv, F, p, h->pGP, h->pHP, h->pG, h->pH, h->pCYZ);
  CP c{};
  c.pv = pv;
  c.F = F;
  c.omega = (float)h->omega_op;
  c.x = p;
  c.y = q;
  c.P = h->pP;
  c.FZ = h->pP + L.n;
  c.VX = h->pVX;
  c.WZ = h->pWZ;
  c.OC1 = h->pOC; c.OC2 = h->pOC2; c.OX = h->pOX; c.OZ = h->pOZ;
  c.G = h->pG; c.H = h->pH; c.CYZ = h->pCYZ;
  c.rho = h->pRho;
  c.kap = h->pKap;
  c.dot = dot;
  {
    KScope ks(st, ESMP2_KT_COUPLING, 12.0 * (double)L.n + 4.0 * (double)(L.n + (int64_t)L.NN * L.SL),
              12.0 * (double)L.n);
    auto run = [&](auto av_tag) {
      constexpr bool AV = decltype(av_tag)::value;
      c.dot_base = 0;
      kp_couple_anti<BT, AV><<<kCoupleGrid, kThreads, 0, st>>>(c);
      c.dot_base = kCoupleGrid;
      kp_couple_anti<BX, AV><<<kCoupleGrid, kThreads, 0, st>>>(c);
      c.dot_base = 2 * kCoupleGrid;
      kp_couple_anti<BY, AV><<<kCoupleGrid, kThreads, 0, st>>>(c);
      c.dot_base = 3 * kCoupleGrid;
      kp_couple_s<AV><<<kCoupleGrid, kThreads, 0, st>>>(c);
      c.dot_base = 4 * kCoupleGrid;
      kp_couple_z<AV><<<kCoupleGrid, kThreads, 0, st>>>(c);
    };
    if (av) run(std::true_type{});
    else run(std::false_type{});
  }
  h->launches += 12;
  return check_cuda(h, cudaGetLastError(), "sigma_packed");
}

// inner-solve start: r (packed) from the float64 residual r64 (full storage), p = M^-1 r,
// d = 0, bf16(p); partials of <r, M^-1 r>_w and <r, r>_w in h->red
void packed_init(esmp2_handle *h, const double *r64, int grid) {
  const Packed &L = h->pk;
  kp_init<<<grid, 128, 0, h->stream>>>(PV{L}, r64, h->pdinv, h->pr, packed_p(h), h->pd,
                                       h->tf32 ? nullptr : static_cast<__nv_bfloat16 *>(h->pop), h->red);
  h->launches += 1;
}

// <u, v>_w of two packed vectors, returned to the host (diagnostics; synchronises; uses the
// reduction buffer h->red, so it must not run between a kernel writing partials there and
// the finalisation reading them)
double packed_wdot(esmp2_handle *h, const float *u, const float *v) {
  kp_wdot<<<256, 256, 0, h->stream>>>(PV{h->pk}, u, v, h->red);
  std::vector<double> part(256);
  cudaMemcpyAsync(part.data(), h->red, sizeof(double) * 256, cudaMemcpyDeviceToHost, h->stream);
  cudaStreamSynchronize(h->stream);
  double t = 0.0;
  for (double x : part) t += x;
  return t;
}

void packed_accumulate(esmp2_handle *h, double *x64) {
  kp_acc64<<<2432, 256, 0, h->stream>>>(PV{h->pk}, x64, h->pd);
  h->launches += 1;
}

// Set-up of the rotated Jacobi preconditioner (once per handle): the virtual rotation, its bf16
// right operands (W[b][c] = M[c][b] for X M: M = R~ gives W = R~^T, M = R~^T gives W = R~), the
// diagonal of F_vv in the rotated basis and the per-slice occupied part of the diagonal of A.
esmp2_status packed_rj_setup(esmp2_handle *h) {
  if (h->rj_ready) return ESMP2_OK;
  esmp2_status s = ensure_vrot(h, false);
  if (s) return s;
  const Packed &L = h->pk;
  const int No = L.No, Nv = L.Nv, Nvp = L.Nvp, N = h->d.N;
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(p, bytes ? bytes : 16, st);
  };
  A(&h->pRbf, sizeof(__nv_bfloat16) * (size_t)L.n);
  A(&h->pT1, sizeof(__nv_bfloat16) * (size_t)L.n);
  A(reinterpret_cast<void **>(&h->pZ), sizeof(float) * (size_t)L.n);
  A(&h->pWR, sizeof(__nv_bfloat16) * (size_t)Nv * Nvp);
  A(&h->pWRt, sizeof(__nv_bfloat16) * (size_t)Nv * Nvp);
  A(reinterpret_cast<void **>(&h->pLam), sizeof(float) * (size_t)Nv);
  A(reinterpret_cast<void **>(&h->pOcc), sizeof(float) * (size_t)L.nslices);
  A(reinterpret_cast<void **>(&h->pCode), sizeof(int) * (size_t)L.nslices);
  A(reinterpret_cast<void **>(&h->pdot2), sizeof(double) * 5 * (size_t)kCoupleGrid);
  A(reinterpret_cast<void **>(&h->zero_slots), sizeof(double) * 32);
  if (e != cudaSuccess) return check_cuda(h, e, "rotated preconditioner buffers");
  // pad columns of the GEMM operands and of z start (and stay) zero: the transposed epilogue
  // writes columns < Nv only, and p = z + beta p must keep zero pads (they are K of the sigma GEMM)
  cudaMemsetAsync(h->pRbf, 0, sizeof(__nv_bfloat16) * (size_t)L.n, st);
  cudaMemsetAsync(h->pT1, 0, sizeof(__nv_bfloat16) * (size_t)L.n, st);
  cudaMemsetAsync(h->pZ, 0, sizeof(float) * (size_t)L.n, st);
  cudaMemsetAsync(h->zero_slots, 0, sizeof(double) * 32, st);
  std::vector<double> R((size_t)Nv * Nv);
  std::vector<float> F((size_t)N * N), Fs((size_t)N * N);
  e = cudaMemcpyAsync(R.data(), h->Rv, sizeof(double) * R.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(F.data(), h->F32arr, sizeof(float) * F.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Fs.data(), h->F32, sizeof(float) * Fs.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return check_cuda(h, e, "rotated preconditioner set-up");
  std::vector<__nv_bfloat16> WR((size_t)Nv * Nvp, __float2bfloat16_rn(0.f)), WRt = WR;
  for (int b = 0; b < Nv; ++b)
    for (int c = 0; c < Nv; ++c) {
      WR[(size_t)b * Nvp + c] = __float2bfloat16_rn((float)R[(size_t)b * Nv + c]);
      WRt[(size_t)b * Nvp + c] = __float2bfloat16_rn((float)R[(size_t)c * Nv + b]);
    }
  std::vector<float> lam(Nv), occ(L.nslices);
  std::vector<int> code(L.nslices);
  for (int a = 0; a < Nv; ++a) lam[a] = F[(size_t)(No + a) * N + No + a];
  // the occupied part as kp_dinv forms it, in float: F_ii + F_jj + omega - (L block ? F_t't' - F_tt : 0)
  const float om = (float)h->omega_op, shift = Fs[(size_t)No * N + No] - Fs[0];
  for (int sl = 0; sl < L.nslices; ++sl) {
    int blk, i, j, t = sl;
    if (t < L.nh) { blk = BT; }
    else if ((t -= L.nh) < L.NN) { blk = BS; }
    else if ((t -= L.NN) < L.nh) { blk = BX; }
    else if ((t -= L.nh) < L.nh) { blk = BY; }
    else { t -= L.nh; blk = BZ; }
    if (blk == BS || blk == BZ) { i = t / No; j = t % No; }
    else pair_decode(No, t, i, j);
    occ[sl] = Fs[(size_t)i * N + i] + Fs[(size_t)j * N + j] + om - (blk >= BX ? shift : 0.f);
    code[sl] = blk | (i == 0 ? 8 : 0) | (j == 0 ? 16 : 0);
  }
  e = cudaMemcpyAsync(h->pWR, WR.data(), sizeof(__nv_bfloat16) * WR.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->pWRt, WRt.data(), sizeof(__nv_bfloat16) * WRt.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->pLam, lam.data(), sizeof(float) * lam.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->pOcc, occ.data(), sizeof(float) * occ.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->pCode, code.data(), sizeof(int) * code.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return check_cuda(h, e, "rotated preconditioner set-up");
  h->rj_ready = true;
  return ESMP2_OK;
}

// z = M^-1 r from the bf16 copy pRbf (overwritten), then projected; partials of <r, z>_w in
// pdot2 (5 kCoupleGrid doubles)
static esmp2_status packed_precond(esmp2_handle *h) {
  const Packed &L = h->pk;
  const int64_t rows = (int64_t)L.nslices * L.Nv;
  const double fl = 2.0 * (double)rows * L.Nv * L.Nv;
  VgemmOut o{};
  o.family = ESMP2_KT_PRECOND;
  esmp2_status s;
  o.PT16 = h->pT1;                                                  // (r R~)^T
  if ((s = vgemm(h, h->pRbf, rows, 0, h->pWRt, nullptr, nullptr, L.Nvp, fl, false, &o))) return s;
  o.PT16 = h->pRbf; o.lam = h->pLam; o.occ = h->pOcc; o.code = h->pCode;   // D~^-1 (R~^T r R~)
  if ((s = vgemm(h, h->pT1, rows, 0, h->pWRt, nullptr, nullptr, L.Nvp, fl, false, &o))) return s;
  o.PT16 = h->pT1; o.lam = nullptr; o.occ = nullptr; o.code = nullptr;    // (z~ R~^T)^T
  if ((s = vgemm(h, h->pRbf, rows, 0, h->pWR, nullptr, nullptr, L.Nvp, fl, false, &o))) return s;
  o.PT16 = nullptr;                                                 // R~ z~ R~^T (float32)
  if ((s = vgemm(h, h->pT1, rows, 0, h->pWR, nullptr, h->pZ, L.Nvp, fl, false, &o))) return s;
  PV pv{L};
  cudaStream_t st = h->stream;
  kp_proj_anti<BT><<<kCoupleGrid, kThreads, 0, st>>>(pv, h->pZ, h->pr, h->pdot2, 0);
  kp_proj_anti<BX><<<kCoupleGrid, kThreads, 0, st>>>(pv, h->pZ, h->pr, h->pdot2, kCoupleGrid);
  kp_proj_anti<BY><<<kCoupleGrid, kThreads, 0, st>>>(pv, h->pZ, h->pr, h->pdot2, 2 * kCoupleGrid);
  kp_proj_s<<<kCoupleGrid, kThreads, 0, st>>>(pv, h->pZ, h->pr, h->pdot2, 3 * kCoupleGrid);
  kp_proj_z<<<kCoupleGrid, 256, 0, st>>>(pv, h->pZ, h->pr, h->pdot2, 4 * kCoupleGrid);
  h->launches += 5;
  return check_cuda(h, cudaGetLastError(), "packed_precond");
}

// start of a preconditioned inner solve: r (packed) from r64, d = 0, z = M^-1 r, p = z; slots:
// rr (1) and rz (0)
esmp2_status packed_rj_init(esmp2_handle *h, const double *r64, int grid) {
  const Packed &L = h->pk;
  PV pv{L};
  cudaStream_t st = h->stream;
  kp_init_rj<<<grid, 256, 0, st>>>(pv, r64, h->pr, static_cast<__nv_bfloat16 *>(h->pRbf), h->pd, h->red);
  k_finalize_ext(h->red, grid, h->red_out, 5, st);
  h->launches += 2;
  if (esmp2_status s = packed_precond(h)) return s;
  k_finalize_ext(h->pdot2, 5 * kCoupleGrid, h->red_out, 7, st);
  kp_p_rj<<<grid, 256, 0, st>>>(pv, h->zero_slots, h->pZ, packed_p(h), h->pd,
                                h->tf32 ? nullptr : static_cast<__nv_bfloat16 *>(h->pop));
  h->launches += 2;
  return check_cuda(h, cudaGetLastError(), "packed_rj_init");
}

// the part of a preconditioned inner iteration after q = A p and alpha: r -= alpha q, z = M^-1 r,
// beta, d += alpha p, p = z + beta p
esmp2_status packed_rj_step(esmp2_handle *h, int grid) {
  const Packed &L = h->pk;
  PV pv{L};
  cudaStream_t st = h->stream;
  kp_update_rj<<<grid, 256, 0, st>>>(pv, h->red_out, h->pr, h->pq, static_cast<__nv_bfloat16 *>(h->pRbf), h->red);
  k_finalize_ext(h->red, grid, h->red_out, 5, st);
  h->launches += 2;
  if (esmp2_status s = packed_precond(h)) return s;
  k_finalize_ext(h->pdot2, 5 * kCoupleGrid, h->red_out, 6, st);
  kp_p_rj<<<grid, 256, 0, st>>>(pv, h->red_out, h->pZ, packed_p(h), h->pd,
                                h->tf32 ? nullptr : static_cast<__nv_bfloat16 *>(h->pop));
  h->launches += 2;
  return check_cuda(h, cudaGetLastError(), "packed_rj_step");
}

// per-stage timing of `reps` packed inner sigma builds of the packed copy of x (CUDA events):
// ms[0] operand conversion, [1] contraction (transposed Z slices + GEMM), [2] 0, [3] coupling
// pass (arrow sums, intermediates, couplings), [4] total
esmp2_status profile_packed(esmp2_handle *h, const double *x, int reps, double *ms) {
  float *p = packed_p(h);
  kp_from64<<<2432, 128, 0, h->stream>>>(PV{h->pk}, x, p);
  h->launches += 1;
  cudaEvent_t ev[4];
  for (auto &e : ev) cudaEventCreate(&e);
  double acc[4] = {0, 0, 0, 0};
  esmp2_status s = ESMP2_OK;
  for (int r = 0; r < reps && !s; ++r) {
    cudaEventRecord(ev[0], h->stream);
    s = sigma_packed(h, p, h->pq, false, nullptr, 1);
    cudaEventRecord(ev[1], h->stream);
    if (!s) s = sigma_packed(h, p, h->pq, true, nullptr, 2);
    cudaEventRecord(ev[2], h->stream);
    if (!s) s = sigma_packed(h, p, h->pq, true, h->pdot, 4);
    cudaEventRecord(ev[3], h->stream);
    cudaEventSynchronize(ev[3]);
    for (int k = 0; k < 3; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      acc[k] += t;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[0], ev[3]);
    acc[3] += t;
  }
  for (auto &e : ev) cudaEventDestroy(e);
  if (s) return s;
  ms[0] = acc[0] / reps;
  ms[1] = acc[1] / reps;
  ms[2] = 0.0;
  ms[3] = acc[2] / reps;
  ms[4] = acc[3] / reps;
  return check_cuda(h, cudaGetLastError(), "profile_packed");
}

// API-level bf16 / tf32 sigma of a singlet vector on the packed path: y = A x (x, y
// full-storage float64 in the TOP basis), through the working basis of the inner solve.
esmp2_status sigma_mixed_packed(esmp2_handle *h, const double *x, double *y) {
  double *t1 = h->s64.w ? h->s64.w : h->s64.p;
  rotate_occ(h, x, y, t1, true);                 // y: x in the working basis
  if (h->arrowv) {
    if (esmp2_status s = ensure_arrow(h)) return s;
    if (esmp2_status s = rotate_virt(h, y, y, t1, true)) return s;
  }
  float *p = packed_p(h);
  kp_from64<<<2432, 128, 0, h->stream>>>(PV{h->pk}, y, p);
  h->launches += 1;
  if (esmp2_status s = sigma_packed(h, p, h->pq, false, nullptr, 7)) return s;
  kp_to64<<<2432, 128, 0, h->stream>>>(PV{h->pk}, h->pq, y);
  h->launches += 1;
  if (h->arrowv)
    if (esmp2_status s = rotate_virt(h, y, y, t1, false)) return s;
  rotate_occ(h, y, y, t1, false);
  // the rotation back mixes slices: the non-amplitude slots (i == j of T, X, Y, ...) carry
  // rounding-level values, cleared here
  kp_mask64<<<2432, 128, 0, h->stream>>>(h->d.No, h->d.Nv, y);
  h->launches += 1;
  return check_cuda(h, cudaGetLastError(), "sigma_mixed_packed");
}

}  // namespace esmp2

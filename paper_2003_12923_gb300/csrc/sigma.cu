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
#include <algorithm>

#include "internal.h"

namespace esmp2 {
void virt64_sym(esmp2_handle *h, const double *F, const double *x, double *y);
namespace {

template <typename CT>
struct CtxT {
  int No, Nv, N;
  int64_t B;
  const CT *F;
  CT omega;
  int arrow;  // 1: F_oo is diagonal apart from the t row/column (occupied terms done here)
  double *dot = nullptr;  // coupling pass: per-CTA weighted partials of <x, y>, or none
  __device__ __forceinline__ CT Fo(int k, int l) const { return F[(int64_t)k * N + l]; }
  __device__ __forceinline__ CT Fv(int a, int b) const { return F[(int64_t)(No + a) * N + No + b]; }
  __device__ __forceinline__ CT Fov(int k, int a) const { return F[(int64_t)k * N + No + a]; }
  __device__ __forceinline__ int64_t at(int blk, int i, int j, int a, int b) const {
    return blk * B + (((int64_t)i * No + j) * Nv + a) * Nv + b;
  }
};

template <typename CT>
__device__ __forceinline__ CT warp_sum(CT v) {
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

// Intermediates of the N^4 coupling terms, spread over four launches so that every sum
// has enough parallel work (No^2 Nv, No Nv^2 or No^2 Nv warps).
// (a) per (i, j, b): VX[i][j][b] = sum_c Fov[0][c] X[i][j][c][b],
//                    GP[k][j][b] = sum_c Fov[k][c] (X+Z)[k][j][c][b]
template <typename T, typename CT>
__global__ void k_inter_a(CtxT<CT> c, const T *x, CouplingsT<CT> cp) {
  const int No = c.No, Nv = c.Nv;
  const int64_t n = (int64_t)No * No * Nv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e % Nv), ij = (int)(e / Nv), k = ij / No;
    const T *X = x + c.at(BX, 0, 0, 0, 0) + (int64_t)ij * Nv * Nv + b;
    const T *Z = x + c.at(BZ, 0, 0, 0, 0) + (int64_t)ij * Nv * Nv + b;
    CT vx = CT(0), g = CT(0);
#pragma unroll 8
    for (int cc = 0; cc < Nv; ++cc) {
      const CT xv = (CT)X[(int64_t)cc * Nv], zv = (CT)Z[(int64_t)cc * Nv];
      vx += c.Fov(0, cc) * xv;
      g += c.Fov(k, cc) * (xv + zv);
    }
    cp.VX[e] = vx;
    cp.GP[e] = g;
  }
}

// (b) per (q, a, b): OX[q][ab] = sum_k Fov[k][0] X[k][q][ab], OZ[q][ab] = sum_k Fov[k][0] Z[q][k][ab];
//     arrow form: OC1[blk][q][ab] = sum_{l>=1} Foo[l][0] x[blk][l][q][ab], OC2 likewise on the 2nd index
template <typename T, typename CT>
__global__ void k_inter_b(CtxT<CT> c, const T *x, CouplingsT<CT> cp) {
  const int No = c.No, Nv = c.Nv;
  const int64_t NvNv = (int64_t)Nv * Nv, n = (int64_t)No * NvNv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ab = e % NvNv;
    const int q = (int)(e / NvNv);
    CT s = CT(0), z = CT(0);
    for (int k = 0; k < No; ++k) {
      s += c.Fov(k, 0) * (CT)x[c.at(BX, k, q, 0, 0) + ab];
      z += c.Fov(k, 0) * (CT)x[c.at(BZ, q, k, 0, 0) + ab];
    }
    cp.OX[e] = s;
    cp.OZ[e] = z;
    if (c.arrow) {
      for (int blk = 0; blk < 5; ++blk) {
        CT s1 = CT(0), s2 = CT(0);
        for (int l = 1; l < No; ++l) {
          const CT f = c.Fo(l, 0);
          s1 += f * (CT)x[c.at(blk, l, q, 0, 0) + ab];
          s2 += f * (CT)x[c.at(blk, q, l, 0, 0) + ab];
        }
        cp.OC1[(int64_t)blk * n + e] = s1;
        cp.OC2[(int64_t)blk * n + e] = s2;
      }
    }
  }
}

// (c) warp per row (i, j, a): WZ[i][j][a] = sum_c Fov[0][c] Z[i][j][a][c],
//                             HP[i][j][a] = sum_c Fov[j][c] (Y+Z)[i][j][a][c]
template <typename T, typename CT>
__global__ void k_inter_c(CtxT<CT> c, const T *x, CouplingsT<CT> cp) {
  const int No = c.No, Nv = c.Nv, lane = threadIdx.x & 31;
  const int64_t rows = (int64_t)No * No * Nv;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < rows; r += nw) {
    const int j = (int)((r / Nv) % No);
    const T *Y = x + c.at(BY, 0, 0, 0, 0) + r * Nv;
    const T *Z = x + c.at(BZ, 0, 0, 0, 0) + r * Nv;
    CT wz = CT(0), hp = CT(0);
#pragma unroll 4
    for (int cc = lane; cc < Nv; cc += 32) {
      const CT zv = (CT)Z[cc];
      wz += c.Fov(0, cc) * zv;
      hp += c.Fov(j, cc) * ((CT)Y[cc] + zv);
    }
    wz = warp_sum<CT>(wz);
    hp = warp_sum<CT>(hp);
    if (lane == 0) { cp.WZ[r] = wz; cp.HP[r] = hp; }
  }
}

// (d) G[j][b] = sum_k GP[k][j][b];  H[i][a] = sum_k HP[i][k][a];
//     CYZ[k][c] = sum_d Fvv[0][d] Z[0][k][d][c] - sum_l Foo[l][0] Z[l][k][0][c]
template <typename T, typename CT>
__global__ void k_inter_d(CtxT<CT> c, const T *x, CouplingsT<CT> cp) {
  const int No = c.No, Nv = c.Nv;
  const int64_t n = (int64_t)No * Nv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int part = (int)(e / n);
    const int64_t f = e % n;
    const int p = (int)(f / Nv), q = (int)(f % Nv);
    CT s = CT(0);
    if (part == 0) {
      for (int k = 0; k < No; ++k) s += cp.GP[((int64_t)k * No + p) * Nv + q];
      cp.G[f] = s;
    } else if (part == 1) {
      for (int k = 0; k < No; ++k) s += cp.HP[((int64_t)p * No + k) * Nv + q];
      cp.H[f] = s;
    } else {
#pragma unroll 8
      for (int d = 0; d < Nv; ++d) s += c.Fv(0, d) * (CT)x[c.at(BZ, 0, p, d, q)];
      for (int l = 0; l < No; ++l) s -= c.Fo(l, 0) * (CT)x[c.at(BZ, l, p, 0, q)];
      cp.CYZ[f] = s;
    }
  }
}

// (b) in one pass for the arrow form (No <= 32): a thread owns one (blk, a, b) and reads
// the block's No x No occupied matrix at that (a, b) once; its row sums give OC2 (and OZ
// on Z), its column sums OC1 (and OX on X), the column sums held in registers.  The
// weights F_l0 (l >= 1) and F_l,t' travel as launch parameters, so the unrolled sums take
// them as constant operands instead of registers or shared-memory loads.
// BLK < 0: grid.y runs over T, S, Y (no OX/OZ terms); else the one block BLK.
struct ArrowW {
  float fl[32];  // F_l0 for 1 <= l < No, else 0
  float fk[32];  // F_l,t' for l < No, else 0
};
template <int BLK, typename T, typename CT>
__global__ void __launch_bounds__(128, 4) k_inter_b1(CtxT<CT> c, const T *__restrict__ x, CouplingsT<CT> cp,
                                                     const ArrowW w) {
  const int No = c.No;
  const int blk = BLK >= 0 ? BLK : (blockIdx.y == 0 ? BT : (blockIdx.y == 1 ? BS : BY));
  const int64_t NvNv = (int64_t)c.Nv * c.Nv, n = (int64_t)No * NvNv;
  const T *xb = x + blk * c.B;
  CT *oc1 = cp.OC1 + blk * n, *oc2 = cp.OC2 + blk * n;
  for (int64_t ab = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ab < NvNv; ab += (int64_t)gridDim.x * blockDim.x) {
    CT o1[32];
    CT ox[BLK == BX ? 32 : 1];
#pragma unroll
    for (int m = 0; m < 32; ++m) o1[m] = CT(0);
#pragma unroll
    for (int m = 0; m < (BLK == BX ? 32 : 1); ++m) ox[m] = CT(0);
    for (int l = 0; l < No; ++l) {
      const T *row = xb + (int64_t)l * n + ab;
      const CT fll = w.fl[l], fkl = w.fk[l];
      CT r2 = CT(0), rz = CT(0);
#pragma unroll
      for (int m = 0; m < 32; ++m) {
        if (m < No) {
          const CT v = (CT)row[(int64_t)m * NvNv];
          o1[m] += fll * v;
          r2 += w.fl[m] * v;
          if constexpr (BLK == BX) ox[m] += fkl * v;
          if constexpr (BLK == BZ) rz += w.fk[m] * v;
        }
      }
      oc2[(int64_t)l * NvNv + ab] = r2;
      if constexpr (BLK == BZ) cp.OZ[(int64_t)l * NvNv + ab] = rz;
    }
#pragma unroll
    for (int m = 0; m < 32; ++m) {
      if (m < No) {
        oc1[(int64_t)m * NvNv + ab] = o1[m];
        if constexpr (BLK == BX) cp.OX[(int64_t)m * NvNv + ab] = ox[m];
      }
    }
  }
}

template <typename T, typename CT>
void launch_inter(esmp2_handle *h, const CtxT<CT> &c, const T *x, const CouplingsT<CT> &cp) {
  k_inter_a<T, CT><<<1216, 256, 0, h->stream>>>(c, x, cp);
  bool one_pass = false;
  if constexpr (sizeof(CT) == 4) one_pass = c.arrow && c.No <= 32 && h->arrow_w_ready;
  if (one_pass) {
    if constexpr (sizeof(CT) == 4) {
      ArrowW w;
      for (int l = 0; l < 32; ++l) { w.fl[l] = h->arrow_w[l]; w.fk[l] = h->arrow_w[32 + l]; }
      const unsigned gx = (unsigned)std::min<int64_t>(cdiv((int64_t)c.Nv * c.Nv, 128), 8192);
      k_inter_b1<-1, T, CT><<<dim3(gx, 3), 128, 0, h->stream>>>(c, x, cp, w);
      k_inter_b1<BX, T, CT><<<gx, 128, 0, h->stream>>>(c, x, cp, w);
      k_inter_b1<BZ, T, CT><<<gx, 128, 0, h->stream>>>(c, x, cp, w);
      h->launches += 2;
    }
  } else {
    k_inter_b<T, CT><<<1216, 256, 0, h->stream>>>(c, x, cp);
  }
  k_inter_c<T, CT><<<1216, 256, 0, h->stream>>>(c, x, cp);
  k_inter_d<T, CT><<<(unsigned)cdiv(3LL * c.No * c.Nv, 256), 256, 0, h->stream>>>(c, x, cp);
  h->launches += 4;
}

// Vector loads/stores of VW consecutive elements (16 bytes when VW * sizeof(T) == 16); the
// address must be 16-byte aligned: only slice rows (Nv a multiple of VW) and the coupling
// intermediates (separate allocations, rows of Nv) are read this way, never rows of F.
template <int VW, typename T, typename CT>
__device__ __forceinline__ void ldv(const T *p, CT (&o)[VW]) {
  if constexpr (VW == 4 && sizeof(T) == 4) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    o[0] = (CT)t.x; o[1] = (CT)t.y; o[2] = (CT)t.z; o[3] = (CT)t.w;
  } else if constexpr (VW == 2 && sizeof(T) == 8) {
    const double2 t = *reinterpret_cast<const double2 *>(p);
    o[0] = (CT)t.x; o[1] = (CT)t.y;
  } else {
#pragma unroll
    for (int k = 0; k < VW; ++k) o[k] = (CT)p[k];
  }
}
template <int VW, typename T, typename CT>
__device__ __forceinline__ void stv(T *p, const CT (&v)[VW]) {
  if constexpr (VW == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
  } else if constexpr (VW == 2 && sizeof(T) == 8) {
    *reinterpret_cast<double2 *>(p) = make_double2((double)v[0], (double)v[1]);
  } else {
#pragma unroll
    for (int k = 0; k < VW; ++k) p[k] = (T)v[k];
  }
}

// Bulk prefetch of a contiguous range into L2 (16-byte aligned, a multiple of 16 bytes):
// nothing waits on it and no register holds it, so a CTA's whole strip is in flight at once.
__device__ __forceinline__ void l2_prefetch(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// y += couplings - omega x (+ pair energy on L blocks); y = 0 on non-amplitude slots.
// One launch per block; a CTA owns a 32-row strip of one slice (i, j) and walks its
// 32 x (32 VW) tiles along b, each thread VW consecutive columns of four rows.  Block,
// slice and strip are uniform over the CTA, so every gather is a coalesced (vector) row of
// some slice or a broadcast, all slice pointers are formed once, and the element loop runs
// on 32-bit offsets; the one transposed operand (Z_ji^ba of the S block) goes through
// shared memory.  With c.dot set, the CTA also leaves w_blk <x, y> over its strip (y final:
// this pass is the last writer) in c.dot[(BLK gridDim.y + blockIdx.y) gridDim.x + blockIdx.x].
template <int BLK, int VW, typename TX, typename TY, typename CT>
__global__ void __launch_bounds__(256, BLK == BX ? 2 : 3) k_couple(CtxT<CT> c, const TX *__restrict__ x, TY *__restrict__ y,
                                                CouplingsT<CT> cp) {
  constexpr int TW = 32 * VW;  // tile columns
  __shared__ CT zt[TW][33];
  const int No = c.No, Nv = c.Nv, nt = (Nv + TW - 1) / TW;
  const int i = blockIdx.y / No, j = blockIdx.y % No;
  const int a_base = blockIdx.x << 5;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t NvNv = (int64_t)Nv * Nv, NN = (int64_t)No * No;
  auto S = [&](int bl, int ii, int jj) { return x + ((int64_t)bl * NN + (int64_t)ii * No + jj) * NvNv; };
  const TX *xs = S(BLK, i, j);
  TY *ys = y + (xs - x);
  const bool i0 = i == 0, j0 = j == 0;
  const CT om = c.omega, shift = c.Fv(0, 0) - c.Fo(0, 0), f00 = c.Fov(0, 0);
  const CT fdiag = c.Fo(i, i) + c.Fo(j, j), foi = c.Fo(0, i), foj = c.Fo(0, j);
  const CT fio = c.Fov(i, 0), fjo = c.Fov(j, 0);
  // every diagonal term of the element in one coefficient: -omega, the pair energy of the
  // L blocks, and in the arrow form -(F_ii + F_jj)
  const CT cxe = -om + (BLK >= BX ? shift : CT(0)) - (c.arrow ? fdiag : CT(0));
  const TX *A0j = S(BLK, 0, j), *Ai0 = S(BLK, i, 0);
  const CT *OC1 = c.arrow ? cp.OC1 + ((int64_t)BLK * No + j) * NvNv : nullptr;
  const CT *OC2 = c.arrow ? cp.OC2 + ((int64_t)BLK * No + i) * NvNv : nullptr;
  const CT *Fo_i = c.F + (int64_t)i * c.N + No, *Fo_j = c.F + (int64_t)j * c.N + No, *Fo_0 = c.F + No;
  if constexpr (VW * sizeof(TX) == 16 && sizeof(TY) == sizeof(TX)) {
    // rows start on 16-byte boundaries here: fetch the strip of every operand streamed from
    // HBM (x, y and the same-slot slice of the block this one couples to) ahead of the loads
    const int64_t off = (int64_t)a_base * Nv;
    const uint32_t bytes = (uint32_t)(min(32, Nv - a_base) * Nv * (int)sizeof(TX));
    const TX *other = BLK == BT ? S(BX, i, j) : BLK == BS ? S(BZ, i, j) : BLK == BZ ? S(BS, i, j) : S(BT, i, j);
    if (threadIdx.x == 0) l2_prefetch(xs + off, bytes);
    if (threadIdx.x == 32) l2_prefetch(ys + off, bytes);
    if (threadIdx.x == 64) l2_prefetch(other + off, bytes);
    if (BLK == BT && threadIdx.x == 96) l2_prefetch(S(BY, i, j) + off, bytes);
    if (BLK == BS) {  // the transposed slice: Nv rows of the strip's 32 columns
      const TX *zji = S(BZ, j, i) + a_base;
      const uint32_t rb = (uint32_t)(min(32, Nv - a_base) * (int)sizeof(TX));
      for (int bb = threadIdx.x; bb < Nv; bb += blockDim.x) l2_prefetch(zji + (int64_t)bb * Nv, rb);
    }
  }
  CT xy = CT(0);
  for (int tb = 0; tb < nt; ++tb) {
    const int b = tb * TW + tx * VW;  // first of this thread's VW columns
    if constexpr (BLK == BS) {  // Z_ji[b][a] for the tile, read along a and used along b
      __syncthreads();
      const TX *zji = S(BZ, j, i);
      for (int r = ty; r < TW; r += 8) {
        const int bb = tb * TW + r, aa = a_base + tx;
        zt[r][tx] = (bb < Nv && aa < Nv) ? (CT)zji[bb * Nv + aa] : CT(0);
      }
      __syncthreads();
    }
    if (b >= Nv) continue;
    CT fob_0[VW], fob_i[VW], fob_j[VW];
#pragma unroll
    for (int k = 0; k < VW; ++k) {  // rows of F start at arbitrary offsets: scalar loads
      fob_0[k] = Fo_0[b + k];
      fob_i[k] = Fo_i[b + k];
      fob_j[k] = Fo_j[b + k];
    }
    // t-row vectors (a = 0 row of a slice) used by every row of the tile
    CT h1[VW], h2[VW], h3[VW];
    if constexpr (BLK == BX) {
      ldv<VW>(S(BT, i, j) + b, h1); ldv<VW>(S(BT, 0, j) + b, h2); ldv<VW>(S(BT, 0, i) + b, h3);
    } else if constexpr (BLK == BY) {
      ldv<VW>(S(BS, 0, i) + b, h1); ldv<VW>(S(BS, 0, j) + b, h2);
    } else if constexpr (BLK == BZ) {
      ldv<VW>(S(BT, 0, j) + b, h1); ldv<VW>(S(BY, 0, j) + b, h2);
    }
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int r = ty + 8 * rr;
      const int a = a_base + r;
      if (a >= Nv) break;
      const int ab = a * Nv + b;
      const bool a0f = a == 0;
      CT xe[VW], yo[VW], v[VW], t1[VW], t2[VW];
      ldv<VW>(xs + ab, xe);
      ldv<VW>(ys + ab, yo);  // issued with x: one memory round trip per row
#pragma unroll
      for (int k = 0; k < VW; ++k) v[k] = cxe * xe[k];
      if (c.arrow) {  // - sum_l F_li x[l][j] - sum_l F_lj x[i][l] with F_oo diagonal off the t row/column
        if (i0) ldv<VW>(OC1 + ab, t1); else ldv<VW>(A0j + ab, t1);
        if (j0) ldv<VW>(OC2 + ab, t2); else ldv<VW>(Ai0 + ab, t2);
        const CT s1 = i0 ? CT(1) : foi, s2 = j0 ? CT(1) : foj;
#pragma unroll
        for (int k = 0; k < VW; ++k) v[k] -= s1 * t1[k] + s2 * t2[k];
      }
      if constexpr (BLK == BT) {
        ldv<VW>(S(BX, i, j) + ab, t1);
        ldv<VW>(S(BY, i, j) + ab, t2);
#pragma unroll
        for (int k = 0; k < VW; ++k) v[k] += f00 * (t1[k] + t2[k]);
        const int ij = (i * No + j) * Nv;
        if (a0f) { ldv<VW>(cp.VX + ij + b, t1); for (int k = 0; k < VW; ++k) v[k] -= t1[k]; }
        if (i0) { ldv<VW>(cp.OX + j * NvNv + ab, t1); for (int k = 0; k < VW; ++k) v[k] -= t1[k]; }
        if (j0) { ldv<VW>(cp.OX + i * NvNv + ab, t1); for (int k = 0; k < VW; ++k) v[k] += t1[k]; }
        if (i0 && a0f) { ldv<VW>(cp.G + j * Nv + b, t1); for (int k = 0; k < VW; ++k) v[k] += t1[k]; }
        if (j0 && a0f) { ldv<VW>(cp.G + i * Nv + b, t1); for (int k = 0; k < VW; ++k) v[k] -= t1[k]; }
        if (b == 0) {  // column 0 is the first element of this thread's vector
          v[0] += cp.VX[ij + a];
          if (i0) v[0] -= cp.G[j * Nv + a];
          if (j0) v[0] += cp.G[i * Nv + a];
        }
      } else if constexpr (BLK == BS) {
        ldv<VW>(S(BZ, i, j) + ab, t1);
#pragma unroll
        for (int k = 0; k < VW; ++k) v[k] += f00 * (t1[k] + zt[tx * VW + k][r]);
        if (i0 && a0f) { ldv<VW>(cp.H + j * Nv + b, t1); for (int k = 0; k < VW; ++k) v[k] += t1[k]; }
        if (a0f) { ldv<VW>(cp.WZ + (j * No + i) * Nv + b, t1); for (int k = 0; k < VW; ++k) v[k] -= t1[k]; }
        if (j0) { ldv<VW>(cp.OZ + i * NvNv + ab, t1); for (int k = 0; k < VW; ++k) v[k] -= t1[k]; }
        if (i0) {
#pragma unroll
          for (int k = 0; k < VW; ++k) v[k] -= cp.OZ[j * NvNv + (b + k) * Nv + a];
        }
        if (b == 0) {
          if (j0) v[0] += cp.H[i * Nv + a];
          v[0] -= cp.WZ[(i * No + j) * Nv + a];
        }
      } else if constexpr (BLK == BX) {
        const TX *T = S(BT, i, j), *T0j = S(BT, 0, j), *T0i = S(BT, 0, i);
        const CT foa_0 = Fo_0[a], foa_i = Fo_i[a], foa_j = Fo_j[a];
        const CT Ta = (CT)T[a], T0ja = (CT)T0j[a], T0ia = (CT)T0i[a];
        CT Tab[VW], T0jab[VW], T0iab[VW];
        ldv<VW>(T + ab, Tab); ldv<VW>(T0j + ab, T0jab); ldv<VW>(T0i + ab, T0iab);
#pragma unroll
        for (int k = 0; k < VW; ++k)  // h1 = T_ij row 0, h2 = T_0j row 0, h3 = T_0i row 0 at b
          v[k] += f00 * Tab[k] - foa_0 * h1[k] + fob_0[k] * Ta - fio * T0jab[k] + fjo * T0iab[k]
                + foa_i * h2[k] - foa_j * h3[k] - fob_i[k] * T0ja + fob_j[k] * T0ia;
      } else if constexpr (BLK == BY) {
        const TX *S0i = S(BS, 0, i), *S0j = S(BS, 0, j);
        const CT S0ia = (CT)S0i[a], S0ja = (CT)S0j[a], foa_i = Fo_i[a], foa_j = Fo_j[a];
        CT Tab[VW];
        ldv<VW>(S(BT, i, j) + ab, Tab);
#pragma unroll
        for (int k = 0; k < VW; ++k)  // h1 = S_0i row 0, h2 = S_0j row 0 at b
          v[k] += f00 * Tab[k] + fob_j[k] * S0ia - fob_i[k] * S0ja - foa_j * h1[k] + foa_i * h2[k];
        if (i0 && a0f) { ldv<VW>(cp.CYZ + j * Nv + b, t1); for (int k = 0; k < VW; ++k) v[k] += t1[k]; }
        if (j0 && a0f) { ldv<VW>(cp.CYZ + i * Nv + b, t1); for (int k = 0; k < VW; ++k) v[k] -= t1[k]; }
        if (b == 0) {
          if (i0) v[0] -= cp.CYZ[j * Nv + a];
          if (j0) v[0] += cp.CYZ[i * Nv + a];
        }
      } else {  // BZ
        const TX *Sij = S(BS, i, j), *Si0 = S(BS, i, 0);
        const CT Sija0 = (CT)Sij[a * Nv], Si0a0 = (CT)Si0[a * Nv], foa_i = Fo_i[a], fva = c.Fv(a, 0);
        CT Sijab[VW], Si0ab[VW];
        ldv<VW>(Sij + ab, Sijab); ldv<VW>(Si0 + ab, Si0ab);
#pragma unroll
        for (int k = 0; k < VW; ++k) {  // h1 = T_0j row 0, h2 = Y_0j row 0 at b
          v[k] += f00 * Sijab[k] - fob_0[k] * Sija0 - fjo * Si0ab[k] + fob_j[k] * Si0a0
                + foa_i * h1[k];
          if (i0) v[k] += fva * h2[k];
          if (a0f) v[k] -= foi * h2[k];
        }
      }
#pragma unroll
      for (int k = 0; k < VW; ++k) {
        yo[k] = valid_elem(BLK, i, j, a, b + k) ? yo[k] + v[k] : CT(0);
        xy += xe[k] * yo[k];
      }
      stv<VW>(ys + ab, yo);
    }
  }
  if (c.dot) {
    __shared__ double wsum[8];
    const double s = (double)warp_sum<CT>(xy);
    if (tx == 0) wsum[ty] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += wsum[w];
      const double wb = BLK == BS ? 1.0 : (BLK == BZ ? 2.0 : 0.5);
      c.dot[((int64_t)BLK * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = wb * t;
    }
  }
}

template <int VW, typename TX, typename TY, typename CT>
void launch_couple_vw(const CtxT<CT> &c, const TX *x, TY *y, const CouplingsT<CT> &cp, cudaStream_t st) {
  const dim3 grid((unsigned)((c.Nv + 31) / 32), (unsigned)(c.No * c.No));
  k_couple<BT, VW, TX, TY, CT><<<grid, 256, 0, st>>>(c, x, y, cp);
  k_couple<BS, VW, TX, TY, CT><<<grid, 256, 0, st>>>(c, x, y, cp);
  k_couple<BX, VW, TX, TY, CT><<<grid, 256, 0, st>>>(c, x, y, cp);
  k_couple<BY, VW, TX, TY, CT><<<grid, 256, 0, st>>>(c, x, y, cp);
  k_couple<BZ, VW, TX, TY, CT><<<grid, 256, 0, st>>>(c, x, y, cp);
}

// 16-byte vectors when every row of a slice starts on a 16-byte boundary
template <typename TX, typename TY, typename CT>
void launch_couple(const CtxT<CT> &c, const TX *x, TY *y, const CouplingsT<CT> &cp, cudaStream_t st) {
  constexpr int VW = 16 / sizeof(TX);
  const double bytes = 5.0 * c.B * (sizeof(TX) + 2.0 * sizeof(TY));
  KScope ks(st, ESMP2_KT_COUPLING, bytes, bytes);
  const bool aligned = (reinterpret_cast<uintptr_t>(x) % 16 == 0) && (reinterpret_cast<uintptr_t>(y) % 16 == 0);
  if (aligned && c.Nv % VW == 0 && sizeof(TX) == sizeof(TY) && sizeof(TX) == sizeof(CT))
    launch_couple_vw<VW>(c, x, y, cp, st);
  else
    launch_couple_vw<1>(c, x, y, cp, st);
}

}  // namespace

template <typename CT>
static CtxT<CT> make_ctx(const esmp2_handle *h, const CT *F, int arrow) {
  CtxT<CT> c;
  c.No = h->d.No; c.Nv = h->d.Nv; c.N = h->d.N; c.B = h->d.B;
  c.F = F; c.omega = (CT)h->omega_op; c.arrow = arrow;
  return c;
}

void launch_intermediates64(esmp2_handle *h, const double *F, int arrow, const double *x) {
  launch_inter<double, double>(h, make_ctx<double>(h, F, arrow), x, h->cp);
}

void launch_couple64(esmp2_handle *h, const double *F, int arrow, const double *x, double *y) {
  launch_couple<double, double, double>(make_ctx<double>(h, F, arrow), x, y, h->cp, h->stream);
  h->launches += 5;
}

// float coupling + arrow occupied pass of the inner (low-precision) sigma: float arithmetic
// throughout (float64 runs at a small fraction of the float32 rate on GB300).
int64_t couple_dot_parts(const esmp2_handle *h) {
  return 5 * cdiv(h->d.Nv, 32) * h->d.No * h->d.No;
}

void couple32(esmp2_handle *h, const float *F32, const float *x, float *y, double *dot) {
  CtxT<float> c = make_ctx<float>(h, F32, 1);
  launch_inter<float, float>(h, c, x, h->cp32);
  c.dot = dot;
  launch_couple<float, float, float>(c, x, y, h->cp32, h->stream);
  h->launches += 5;
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
esmp2_status profile64(esmp2_handle *h, const double *x, double *y, int reps, double *ms, int tc_levels) {
  cudaEvent_t ev[5];
  for (auto &e : ev) cudaEventCreate(&e);
  double acc[5] = {0, 0, 0, 0, 0};
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(ev[0], h->stream);
    if (!h->P64) dmalloc(reinterpret_cast<void **>(&h->P64), sizeof(double) * 4 * (size_t)h->d.B, h->stream);
    if (tc_levels) {
      esmp2_status s = virt_split(h, x, y, h->P64, 1, tc_levels);
      if (s) return s;
      combine_sym(h, y);
    } else {
      virt64_sym(h, h->F, x, y);
    }
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

// ---- float64 virtual-index terms using the storage symmetries of the blocks.
// T, X, Y slices are antisymmetric (x_s^T = -x_s) and slice (j,i) = -slice (i,j):
//     y_ij = P_ij - P_ij^T (i < j),  y_ji = -y_ij,  P = x F;
// S and Z take both GEMM terms (no symmetry is assumed of an input S).
// Work: 4.75 of the 10 GEMM units of the plain form.
__global__ void k_combine_sym(int No, int Nv, const double *P, double *y) {
  __shared__ double t1[32][33], t2[32][33];
  const int64_t NvNv = (int64_t)Nv * Nv, B = (int64_t)No * No * NvNv;
  const int tiles = (Nv + 31) / 32;
  int64_t bid = blockIdx.x;
  const int tb = (int)(bid % tiles); bid /= tiles;
  const int ta = (int)(bid % tiles); bid /= tiles;
  const int j = (int)(bid % No); bid /= No;
  const int i = (int)(bid % No);
  const int blk = (int)(bid / No) == 0 ? BT : ((int)(bid / No) == 1 ? BX : BY);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  const int a0 = ta * 32, b0 = tb * 32;
  int p = i, q = j;
  double sg = 1.0;
  if (i > j) { p = j; q = i; sg = -1.0; }                // y_ij = -(P_ji - P_ji^T)
  const double *P1 = P + blk * B + ((int64_t)p * No + q) * NvNv;
  const double *P2 = P1;
  double *Y = y + blk * B + ((int64_t)i * No + j) * NvNv;
  for (int r = ty; r < 32; r += 8) {
    const int a = a0 + r, b = b0 + tx;
    t1[r][tx] = (a < Nv && b < Nv) ? P1[(int64_t)a * Nv + b] : 0.0;
    const int a2 = b0 + r, b2 = a0 + tx;                  // transposed tile of P2
    t2[r][tx] = (a2 < Nv && b2 < Nv) ? P2[(int64_t)a2 * Nv + b2] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int a = a0 + r, b = b0 + tx;
    if (a < Nv && b < Nv) {
      const double v = (i == j) ? 0.0 : sg * (t1[r][tx] - t2[tx][r]);
      Y[(int64_t)a * Nv + b] = v;
    }
  }
}

// y_ij = P_ij + P_ji^T for the S block from P (= x F on every S slice) in P64: F x_ij equals
// (x_ji F)^T when S_ij^ab = S_ji^ba.  One CTA per (slice (i, j), tile pair (ta, tb)).
__global__ void k_combine_s(int No, int Nv, const double *P, double *y) {
  __shared__ double t1[32][33], t2[32][33];
  const int64_t NvNv = (int64_t)Nv * Nv, B = (int64_t)No * No * NvNv;
  const int tiles = (Nv + 31) / 32;
  int64_t bid = blockIdx.x;
  const int tb = (int)(bid % tiles); bid /= tiles;
  const int ta = (int)(bid % tiles); bid /= tiles;
  const int j = (int)(bid % No), i = (int)(bid / No);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  const int a0 = ta * 32, b0 = tb * 32;
  const double *P1 = P + BS * B + ((int64_t)i * No + j) * NvNv;
  const double *P2 = P + BS * B + ((int64_t)j * No + i) * NvNv;
  double *Y = y + BS * B + ((int64_t)i * No + j) * NvNv;
  for (int r = ty; r < 32; r += 8) {
    const int a = a0 + r, b = b0 + tx;
    t1[r][tx] = (a < Nv && b < Nv) ? P1[(int64_t)a * Nv + b] : 0.0;
    const int a2 = b0 + r, b2 = a0 + tx;                  // transposed tile of P2
    t2[r][tx] = (a2 < Nv && b2 < Nv) ? P2[(int64_t)a2 * Nv + b2] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int a = a0 + r, b = b0 + tx;
    if (a < Nv && b < Nv) Y[(int64_t)a * Nv + b] = t1[r][tx] + t2[tx][r];
  }
}

// In-place projection of the T, X, Y blocks onto exactly antisymmetric amplitudes:
// w = (v_ij^ab - v_ji^ab - v_ij^ba + v_ji^ba) / 4 is computed once per canonical element and
// written with the exact signs to all four images (i == j or a == b slots become zero).
// The float64 virtual-index pass above relies on this symmetry, so solvers keep their
// vectors on it.  One CTA per (block, slice pair i <= j, tile pair ta <= tb).
__global__ void k_antisym_project(int No, int Nv, double *v) {
  __shared__ double s1[32][33], s2[32][33], s3[32][33], s4[32][33];
  const int64_t NvNv = (int64_t)Nv * Nv, B = (int64_t)No * No * NvNv;
  const int tiles = (Nv + 31) / 32;
  const int npairs = tiles * (tiles + 1) / 2, nslice = No * (No + 1) / 2;
  int64_t bid = blockIdx.x;
  int tp = (int)(bid % npairs); bid /= npairs;
  int sp = (int)(bid % nslice);
  const int blk = (int)(bid / nslice) == 0 ? BT : ((int)(bid / nslice) == 1 ? BX : BY);
  int ta = 0;
  while (tp >= tiles - ta) { tp -= tiles - ta; ++ta; }   // row ta of the upper triangle has tiles-ta pairs
  const int tb = ta + tp;
  int i = 0;
  while (sp >= No - i) { sp -= No - i; ++i; }
  const int j = i + sp;
  double *Vij = v + blk * B + ((int64_t)i * No + j) * NvNv;
  double *Vji = v + blk * B + ((int64_t)j * No + i) * NvNv;
  const int a0 = ta * 32, b0 = tb * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int a = a0 + r, b = b0 + tx, a2 = b0 + r, b2 = a0 + tx;
    const bool in1 = a < Nv && b < Nv, in2 = a2 < Nv && b2 < Nv;
    s1[r][tx] = in1 ? Vij[(int64_t)a * Nv + b] : 0.0;
    s2[r][tx] = in1 ? Vji[(int64_t)a * Nv + b] : 0.0;
    s3[r][tx] = in2 ? Vij[(int64_t)a2 * Nv + b2] : 0.0;   // v_ij[b][a] with b = b0 + r
    s4[r][tx] = in2 ? Vji[(int64_t)a2 * Nv + b2] : 0.0;
  }
  __syncthreads();
  // w for element (a = a0 + r, b = b0 + c): needs v_ij[b][a] = s3[c][r]
  for (int r = ty; r < 32; r += 8) {
    const int c = tx, a = a0 + r, b = b0 + c;
    double w = 0.0;
    const bool canon = (ta < tb) || (r < c);
    if (i != j && canon) w = 0.25 * (s1[r][c] - s2[r][c] - s3[c][r] + s4[c][r]);
    s1[r][c] = canon ? w : 0.0;
    (void)a; (void)b;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int a = a0 + r, b = b0 + tx;
    if (a < Nv && b < Nv) {
      const double w = s1[r][tx];
      if (ta < tb || r < tx) {
        Vij[(int64_t)a * Nv + b] = w;
        Vji[(int64_t)a * Nv + b] = -w;
      } else if (r == tx) {
        Vij[(int64_t)a * Nv + b] = 0.0;
        Vji[(int64_t)a * Nv + b] = 0.0;
      }
    }
    // transposed images: (b, a) positions hold -w (ij) and +w (ji)
    const int a2 = b0 + r, b2 = a0 + tx;   // element (a2, b2) = (b, a) of canonical (b2, a2)
    if (a2 < Nv && b2 < Nv && (ta < tb || tx < r)) {
      const double w = s1[tx][r];
      Vij[(int64_t)a2 * Nv + b2] = -w;
      Vji[(int64_t)a2 * Nv + b2] = w;
    }
  }
}

void antisym_project(esmp2_handle *h, double *v) {
  const int No = h->d.No, Nv = h->d.Nv, tiles = (Nv + 31) / 32;
  const int64_t nb = 3LL * (No * (No + 1) / 2) * (tiles * (tiles + 1) / 2);
  k_antisym_project<<<(unsigned)nb, 256, 0, h->stream>>>(No, Nv, v);
  h->launches += 1;
}

// In-place projection of the S block onto the spin-flip symmetry of the singlet,
// S_ij^ab = S_ji^ba: w = (v_ij^ab + v_ji^ba) / 2 written to both images.  One CTA per (slice
// pair i <= j, tile (ta, tb)); for i == j only the tiles ta <= tb.
__global__ void k_sym_project_s(int No, int Nv, double *v) {
  __shared__ double s1[32][33], s2[32][33];
  const int64_t NvNv = (int64_t)Nv * Nv;
  const int tiles = (Nv + 31) / 32;
  int64_t bid = blockIdx.x;
  const int tt = (int)(bid % (tiles * tiles));
  int sp = (int)(bid / (tiles * tiles));
  const int ta = tt / tiles, tb = tt % tiles;
  int i = 0;
  while (sp >= No - i) { sp -= No - i; ++i; }
  const int j = i + sp;
  if (i == j && ta > tb) return;
  double *S = v + (int64_t)No * No * NvNv;   // block 1
  double *Vij = S + ((int64_t)i * No + j) * NvNv, *Vji = S + ((int64_t)j * No + i) * NvNv;
  const int a0 = ta * 32, b0 = tb * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int a = a0 + r, b = b0 + tx, a2 = b0 + r, b2 = a0 + tx;
    s1[r][tx] = (a < Nv && b < Nv) ? Vij[(int64_t)a * Nv + b] : 0.0;   // v_ij[a][b]
    s2[r][tx] = (a2 < Nv && b2 < Nv) ? Vji[(int64_t)a2 * Nv + b2] : 0.0; // v_ji[b][a] at s2[c][r]
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) s1[r][tx] = 0.5 * (s1[r][tx] + s2[tx][r]);
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int a = a0 + r, b = b0 + tx;
    if (a < Nv && b < Nv) Vij[(int64_t)a * Nv + b] = s1[r][tx];
    const int a2 = b0 + r, b2 = a0 + tx;   // v_ji[b][a] = w(a, b)
    if (a2 < Nv && b2 < Nv) Vji[(int64_t)a2 * Nv + b2] = s1[tx][r];
  }
}

// antisymmetry of T, X, Y in both index pairs and the spin-flip symmetry of S
void singlet_project(esmp2_handle *h, double *v) {
  antisym_project(h, v);
  const int No = h->d.No, Nv = h->d.Nv, tiles = (Nv + 31) / 32;
  const int64_t nb = (int64_t)(No * (No + 1) / 2) * tiles * tiles;
  k_sym_project_s<<<(unsigned)nb, 256, 0, h->stream>>>(No, Nv, v);
  h->launches += 1;
}

void virt64_sym(esmp2_handle *h, const double *F, const double *x, double *y) {
  const int No = h->d.No, Nv = h->d.Nv, N = h->d.N;
  const int64_t B = h->d.B, NvNv = (int64_t)Nv * Nv;
  const double *Fv = F + (int64_t)No * N + No;
  Gemm64 g{};
  // P = x F for T, X, Y on the slices i < j
  g.N = Nv; g.K = Nv; g.batch = 1; g.alpha = 1.0; g.beta = 0.0;
  g.sAm = Nv; g.sAk = 1; g.B = Fv; g.sBk = N; g.sBn = 1; g.sCm = Nv; g.sCn = 1;
  int nl = 0;
  for (int blk : {BT, BX, BY})
    for (int i = 0; i + 1 < No; ++i) {
      const int64_t r0 = ((int64_t)i * No + i + 1) * Nv;
      g.M = (int)((int64_t)(No - 1 - i) * Nv);
      g.A = x + blk * B + r0 * Nv;
      g.C = h->P64 + blk * B + r0 * Nv;
      gemm64(g, h->stream);
      ++nl;
    }
  // S and Z: y = x F + F x directly
  for (int blk : {BS, BZ}) {
    g = Gemm64{};
    g.N = Nv; g.K = Nv; g.batch = 1; g.alpha = 1.0; g.beta = 0.0;
    g.sAm = Nv; g.sAk = 1; g.B = Fv; g.sBk = N; g.sBn = 1; g.sCm = Nv; g.sCn = 1;
    g.M = (int)((int64_t)No * No * Nv);
    g.A = x + blk * B; g.C = y + blk * B;
    gemm64(g, h->stream);
    g = Gemm64{};
    g.M = Nv; g.N = Nv; g.K = Nv; g.batch = No * No; g.alpha = 1.0; g.beta = 1.0;
    g.A = Fv; g.sAm = N; g.sAk = 1; g.sAb = 0;
    g.B = x + blk * B; g.sBk = Nv; g.sBn = 1; g.sBb = NvNv;
    g.C = y + blk * B; g.sCm = Nv; g.sCn = 1; g.sCb = NvNv;
    gemm64(g, h->stream);
    nl += 2;
  }
  h->launches += nl;
  combine_sym(h, y);
}

// y_ij = P_ij - P_ij^T for the T, X, Y blocks from P (= x F on the slices i < j) in P64
void combine_sym(esmp2_handle *h, double *y) {
  const int No = h->d.No, Nv = h->d.Nv, tiles = (Nv + 31) / 32;
  const int64_t nblocks = 3LL * No * No * tiles * tiles;
  k_combine_sym<<<(unsigned)nblocks, 256, 0, h->stream>>>(No, Nv, h->P64, y);
  h->launches += 1;
}

// y_ij = P_ij + P_ji^T for the S block (P = x F on every S slice, in P64)
void combine_s(esmp2_handle *h, double *y) {
  const int No = h->d.No, Nv = h->d.Nv, tiles = (Nv + 31) / 32;
  const int64_t nblocks = (int64_t)No * No * tiles * tiles;
  k_combine_s<<<(unsigned)nblocks, 256, 0, h->stream>>>(No, Nv, h->P64, y);
  h->launches += 1;
}

namespace {
__global__ void k_round_f32(const double *src, float *dst, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (float)src[e];
}
// y += (double) y32 on amplitude slots, y = 0 on the others; a warp per row (block, i, j, a)
__global__ void k_add_f32_masked(const float *src, double *dst, int No, int Nv) {
  const int64_t rows = 5LL * No * No * Nv;
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < rows;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int a = (int)(r % Nv);
    int64_t f = r / Nv;
    const int j = (int)(f % No);
    f /= No;
    const int i = (int)(f % No), blk = (int)(f / No);
    for (int b = lane; b < Nv; b += 32) {
      const int64_t e = r * Nv + b;
      dst[e] = valid_elem(blk, i, j, a, b) ? dst[e] + (double)src[e] : 0.0;
    }
  }
}
}  // namespace

// Couplings, shifts, arrow terms and masks of y = A x in float32, added to the float64 y
// (semicanonical-occupied basis): x rounded to float into the inner p buffer, the inner
// coupling pass on it into the inner q buffer, the result added in float64 and the
// non-amplitude slots cleared.  For the intermediate true residuals of the refinement,
// which need A x to about 1e-7 of |A x| only; the float64 coupling pass runs at the
// float64 rate.
void couple_f32_into(esmp2_handle *h, const double *x, double *y) {
  const int64_t n = h->d.n;
  k_round_f32<<<1216, 256, 0, h->stream>>>(x, h->p32, n);
  cudaMemsetAsync(h->q32, 0, sizeof(float) * (size_t)n, h->stream);
  couple32(h, h->arrowv ? h->F32arr : h->F32, h->p32, h->q32);
  k_add_f32_masked<<<1216, 256, 0, h->stream>>>(h->q32, y, h->d.No, h->d.Nv);
  h->launches += 2;
}

// float64 sigma with an arbitrary orthonormal-basis Fock matrix F (t = occupied 0, t' =
// virtual 0).  arrow = 1 when F_oo is diagonal apart from its t row and column: then the
// occupied-index terms are applied element-wise instead of by GEMM.
// tc_levels >= 2: the virtual-index terms come from exact digit products on the tensor
// cores, digit levels 2 .. tc_levels (F_vv of the handle); 0: float64 GEMMs with F.
// couplings = 0 (arrow form only): stop after the index contractions (the caller adds the
// coupling pass).
esmp2_status sigma64_F(esmp2_handle *h, const double *F, int arrow, const double *x, double *y, int tc_levels,
                       int couplings, bool s_sym) {
  if (!h->P64) {
    cudaError_t e = dmalloc(reinterpret_cast<void **>(&h->P64), sizeof(double) * 4 * (size_t)h->d.B, h->stream);
    if (e != cudaSuccess) return check_cuda(h, e, "sigma64 workspace");
  }
  if (tc_levels) {
    esmp2_status s = virt_split(h, x, y, h->P64, s_sym ? 2 : 1, tc_levels);
    if (s) return s;
    combine_sym(h, y);
    if (s_sym) combine_s(h, y);
  } else {
    virt64_sym(h, F, x, y);
  }
  if (!arrow) contractions64(h, F, x, y, 2);
  if (couplings || !arrow) {
    launch_intermediates64(h, F, arrow, x);
    launch_couple64(h, F, arrow, x, y);
  }
  return check_cuda(h, cudaGetLastError(), "sigma64");
}

esmp2_status sigma64(esmp2_handle *h, const double *x, double *y, int tc_levels) { return sigma64_F(h, h->F, 0, x, y, tc_levels); }

// parts (2)-(3) only: couplings, shift and masks added to y
esmp2_status sigma64_tail(esmp2_handle *h, const double *F, int arrow, const double *x, double *y) {
  launch_intermediates64(h, F, arrow, x);
  launch_couple64(h, F, arrow, x, y);
  return check_cuda(h, cudaGetLastError(), "sigma64 tail");
}

}  // namespace esmp2

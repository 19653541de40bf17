// Virtual-index contractions of the sigma build on the 5th-generation tensor cores.
//
// For every slice s = (block, i, j) of the block vector (an Nv x Nv matrix X_s) the two
// virtual-index terms of the one-body operator are
//     Y_s = X_s F + F X_s            (F = F_vv, symmetric)
// i.e. the N_o^2 N_v^3 part of Table 1.  One CTA tile is (s, 128 rows a, <= 256 columns b);
// both terms accumulate into the same fp32 TMEM accumulator:
//     term 2: A = X_s[a-tile][c]   (K-major)   B = F[b-tile][c]      (K-major)
//     term 1: A = F[a-tile][c]     (K-major)   B = X_s[c][b-tile]    (MN-major)
// so each output element is written once.  Operands are bf16 (rounded copies of x and F),
// accumulation fp32.
//
// Structure (persistent, one CTA per SM, 320 threads):
//   warp 0      TMA producer: 3-D tiled bulk copies, 128-byte swizzle, 4-slot ring
//   warp 1      tcgen05.mma issuer (one elected thread), commits to mbarriers
//   warps 2..9  epilogue: tcgen05.ld 32x32b from the accumulator (two warps per lane
//               quarter, each half of the columns), fp32 stores or float64 accumulation
// Two TMEM accumulators (2 x 256 columns) let the epilogue of tile k overlap the main
// loop of tile k+1.  Every mbarrier wait is bounded by a globaltimer limit; a wait that
// runs out sets an error flag, skips the remaining work and the CTA still waits (bounded)
// for its own copies in flight and frees its TMEM before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>
#include <mutex>
#include <map>
#include <cstdlib>

#include "internal.h"

namespace esmp2 {
namespace tc {

constexpr int BM = 128;           // accumulator rows (TMEM lanes)
constexpr int BN_MAX = 256;       // accumulator columns per tile
constexpr int BK = 64;            // K elements per stage (128 bytes of bf16)
constexpr int STAGES = 4;          // ring slots; a slot holds the operands of one term
constexpr int A_BYTES = BM * BK * 2;          // 16 KB
constexpr int B_BYTES = BN_MAX * BK * 2;      // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr int NTHREADS = 320;     // producer warp, MMA warp, 8 epilogue warps
constexpr uint64_t WAIT_NS = 2000000000ull;   // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: true when the phase of the given parity has completed.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, uint64_t limit = WAIT_NS) {
  const uint32_t a = smem_u32(b);
  if (mbar_test(a, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_test(a, parity))
    if (gtimer() - t0 > limit) return false;
  return true;
}
__device__ __forceinline__ void tma_3d(void *dst, const CUtensorMap *m, uint64_t *bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *m, uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05): start >> 4, LBO >> 4 at bit 16, SBO >> 4 at
// bit 32, descriptor version 1 at bit 46, layout type at bit 61 (2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}
// Instruction descriptor, kind::f16: D fp32 (bit 4), A bf16 (bits 7-9 = 1), B bf16
// (bits 10-12 = 1), A K-major, B major at bit 16, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int b_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)b_mn_major << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

struct Args {
  int Nv;            // virtual orbitals (rows and columns of every slice)
  int nslices;       // slices of this launch
  const int *slices; // global slice index of each launched slice (nullptr: 0 .. nslices-1)
  int per_block;     // slices per amplitude block (No^2); block of slice s = s / per_block
  int tm[5];         // per block: 1 = x F only, 2 = x F + F x, 3 = F x only
  int to_p64[5];     // mode 1, per block: 1 = write p64, 0 = write y64
  int a_tiles;       // ceil(Nv / 128)
  int b_tiles;       // column tiles per slice
  int bn;            // columns of a full column tile (multiple of 16, <= 256)
  int nk;            // K chunks: ceil(Nv / 64)
  int64_t tiles;     // nslices * a_tiles * b_tiles
  int npairs;        // operand pairs accumulated into one tile (digit products of one level)
  int dx[9], df[9];  // digit plane of x and of F for each pair
  int lmin, lmax;    // lmax > 0: every tile runs levels lmin..lmax in turn (mode 1), level L
                     // pairing x digit p with F digit L - 2 - p (p = 0 .. L - 2) in one
                     // accumulator round; dx, df and level unused, npairs the total pairs
  int S_plane;       // slices per digit plane of x
  int mode;          // 0: fp32 store into y32; 1: float64 (y64 | p64) (+)= 2^(es[s] + eF - 6 level) acc
  float *y32;        // [S][Nv][Nv]
  double *y64;       // [S][Nv][Nv] (two-term slices in mode 1)
  double *p64;       // [S][Nv][Nv] (one-term slices in mode 1)
  const int *es;     // per-slice binary exponent of the x digits
  int eF, level, first;
  int mirror;        // mode 0: slices of T, X, Y (i < j listed) also write -y into slice (j, i)
  int No;
  int *err;          // error flag (device)
  uint64_t wait_ns;  // limit of every mbarrier wait (0: WAIT_NS)
  int no_copies;     // failure-detection self-test only: the producer issues no copies, so the
                     // first wait on a full slot runs out with nothing in flight
};

__device__ __forceinline__ int slice_of(const Args &g, int64_t li) {
  return g.slices ? g.slices[li] : (int)li;
}
__device__ __forceinline__ int terms_of(const Args &g, int s) { return g.tm[s / g.per_block]; }

__global__ void __launch_bounds__(NTHREADS, 1)
    k_virt(const __grid_constant__ CUtensorMap tXa, const __grid_constant__ CUtensorMap tXb,
           const __grid_constant__ CUtensorMap tFa, const __grid_constant__ CUtensorMap tFb, Args g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full[STAGES], empty[STAGES], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int fail;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int s = 0; s < 2; ++s) { mbar_init(&acc_full[s], 1); mbar_init(&acc_empty[s], 8); }
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = tmem_base;
  const uint64_t lim = g.wait_ns ? g.wait_ns : WAIT_NS;
  const int per_slice = g.a_tiles * g.b_tiles;
  const int nlev = g.lmax ? g.lmax - g.lmin + 1 : 1;  // work items (accumulator rounds) per tile

  if (warp == 0) {
    if (lane == 0) {  // ------------------------------------------------ TMA producer
      int64_t it = 0;
      bool ok = true;
      const uint32_t bytesXF = (uint32_t)(A_BYTES + g.bn * BK * 2);
      const int nb1 = (g.bn + 63) / 64;   // 64-column boxes of the MN-major X tile
      const uint32_t bytesFX = (uint32_t)(A_BYTES + nb1 * 64 * BK * 2);
      if (g.no_copies) ok = false;
      for (int64_t t = blockIdx.x; t < g.tiles && ok; t += gridDim.x) {
        const int s = slice_of(g, t / per_slice), rem = (int)(t % per_slice);
        const int terms = terms_of(g, s);
        const int a0 = (rem / g.b_tiles) * BM, b0 = (rem % g.b_tiles) * g.bn;
        for (int lv = 0; lv < nlev && ok; ++lv) {
        const int L = g.lmax ? g.lmin + lv : g.level, np = g.lmax ? L - 1 : g.npairs;
        for (int pr = 0; pr < np && ok; ++pr) {
          const int zx = (g.lmax ? pr : g.dx[pr]) * g.S_plane + s, zf = g.lmax ? L - 2 - pr : g.df[pr];
          for (int kc = 0; kc < g.nk && ok; ++kc) {
            const int c0 = kc * BK;
            for (int term = 1; term <= 2; ++term, ++it) {   // 1: x F, 2: F x
              if ((term == 1 && terms == 3) || (term == 2 && terms == 1)) { --it; continue; }
              const int st = (int)(it % STAGES);
              const uint32_t rnd = (uint32_t)(it / STAGES);
              if (!mbar_wait(&empty[st], (rnd & 1) ^ 1, lim)) { ok = false; break; }
              uint8_t *A = smem + st * STAGE_BYTES, *B = A + A_BYTES;
              if (term == 1) {   // A = X_s rows (128 x 64), B = F rows b (bn x 64), both K-major
                mbar_expect_tx(&full[st], bytesXF);
                tma_3d(A, &tXa, &full[st], c0, a0, zx);
                tma_3d(B, &tFb, &full[st], c0, b0, zf);
              } else {           // A = F rows a (128 x 64), B = X_s[c][b] (4 boxes of 64 x 64, MN-major)
                mbar_expect_tx(&full[st], bytesFX);
                tma_3d(A, &tFa, &full[st], c0, a0, zf);
#pragma unroll
                for (int q = 0; q < nb1; ++q) tma_3d(B + q * (BK * 128), &tXb, &full[st], b0 + 64 * q, c0, zx);
              }
            }
          }
        }
        }
      }
      if (!ok && !g.no_copies) atomicExch(&fail, 1);
      // wait (bounded) until no copy of this CTA is still in flight
      for (int64_t j = it > STAGES ? it - STAGES : 0; j < it; ++j)
        mbar_wait(&full[j % STAGES], (uint32_t)((j / STAGES) & 1), 100000000ull);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ------------------------------------------------ MMA issuer
      int64_t it = 0;
      int lt = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < g.tiles && ok; t += gridDim.x) {
        const int s = slice_of(g, t / per_slice), rem = (int)(t % per_slice);
        const int terms = terms_of(g, s);
        const int b0 = (rem % g.b_tiles) * g.bn;
        const int nvalid = min(g.bn, g.Nv - b0);
        const int nmma = (nvalid + 15) & ~15;
        const uint32_t id2 = idesc_bf16(BM, nmma, 0), id1 = idesc_bf16(BM, nmma, 1);
        for (int lv = 0; lv < nlev && ok; ++lv, ++lt) {
        const int np = g.lmax ? g.lmin + lv - 1 : g.npairs;
        const int ab = lt & 1;
        const uint32_t ar = (uint32_t)(lt >> 1);
        if (!mbar_wait(&acc_empty[ab], (ar & 1) ^ 1, lim)) { ok = false; break; }
        tc_after();
        const uint32_t d = tmem + (uint32_t)(ab * BN_MAX);
        bool first = true;
        for (int pr = 0; pr < np && ok; ++pr) {
          for (int kc = 0; kc < g.nk && ok; ++kc) {
            const int ksteps = min(BK / 16, (g.Nv - kc * BK + 15) / 16);
            for (int term = 1; term <= 2; ++term, ++it) {
              if ((term == 1 && terms == 3) || (term == 2 && terms == 1)) { --it; continue; }
              const int st = (int)(it % STAGES);
              const uint32_t rnd = (uint32_t)(it / STAGES);
              if (!mbar_wait(&full[st], rnd & 1, lim)) { ok = false; break; }
              tc_after();
              const uint32_t A = smem_u32(smem + st * STAGE_BYTES), B = A + A_BYTES;
              for (int k = 0; k < ksteps; ++k) {
                if (term == 1)   // X_s[a][c] F[c][b]
                  umma(d, sdesc(A + 32 * k, 16, 1024), sdesc(B + 32 * k, 16, 1024), id2, first ? 0u : 1u);
                else             // F[a][c] X_s[c][b]
                  umma(d, sdesc(A + 32 * k, 16, 1024), sdesc(B + 2048 * k, BK * 128, 1024), id1, first ? 0u : 1u);
                first = false;
              }
              umma_commit(&empty[st]);
            }
          }
        }
        if (!ok) break;
        umma_commit(&acc_full[ab]);
        }
      }
      if (!ok) atomicExch(&fail, 1);
    }
  } else {  // ---------------------------------------------------------- epilogue
    // warp w reads TMEM lanes 32 (w % 4) .. +31 (the tcgen05.ld lane rule); the two warps of
    // a lane quarter split the tile's columns
    const int quarter = warp & 3, chalf = (warp - 2) >> 2;
    int lt = 0;
    bool stop = false;
    for (int64_t t = blockIdx.x; t < g.tiles && !stop; t += gridDim.x) {
      const int s = slice_of(g, t / per_slice), rem = (int)(t % per_slice);
      const int a0 = (rem / g.b_tiles) * BM, b0 = (rem % g.b_tiles) * g.bn;
      const int nvalid = min(g.bn, g.Nv - b0);
      for (int lv = 0; lv < nlev; ++lv, ++lt) {
      const int L = g.lmax ? g.lmin + lv : g.level;
      const bool first = g.first && lv == 0;
      const int ab = lt & 1;
      const uint32_t ar = (uint32_t)(lt >> 1);
      const bool got = mbar_wait(&acc_full[ab], ar & 1, lim);
      if (!got) { if (lane == 0) atomicExch(&fail, 1); stop = true; break; }
      tc_after();
      const int row = quarter * 32 + lane;
      const int a = a0 + row;
      const int64_t off = ((int64_t)s * g.Nv + a) * g.Nv + b0;
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * BN_MAX);
      const int hc = ((nvalid + 31) / 32) * 16;   // columns per half, a multiple of 16
      const int c_begin = chalf * hc, c_end = min(nvalid, c_begin + hc);
      if (g.mode == 0) {
        float *dst = g.y32 + off;
        float *dmr = nullptr;   // mirror slice (j, i) of an antisymmetric block
        if (g.mirror) {
          const int blk = s / g.per_block, ij = s % g.per_block;
          if (blk == 0 || blk == 2 || blk == 3) {
            const int sm = blk * g.per_block + (ij % g.No) * g.No + ij / g.No;
            dmr = g.y32 + ((int64_t)sm * g.Nv + a) * g.Nv + b0;
          }
        }
        for (int c = c_begin; c < c_end; c += 16) {
          float v[16];
          tmem_ld16(taddr + (uint32_t)c, v);
          if (a < g.Nv) {
            const int m = min(16, nvalid - c);
            if (!first)
              for (int q = 0; q < m; ++q) v[q] += dst[c + q];   // second pass of a split slice
            if (m == 16 && (g.Nv & 3) == 0) {
              float4 *d4 = reinterpret_cast<float4 *>(dst + c);
#pragma unroll
              for (int q = 0; q < 4; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
              if (dmr) {
                float4 *m4 = reinterpret_cast<float4 *>(dmr + c);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                  m4[q] = make_float4(-v[4 * q], -v[4 * q + 1], -v[4 * q + 2], -v[4 * q + 3]);
              }
            } else {
              for (int q = 0; q < m; ++q) dst[c + q] = v[q];
              if (dmr)
                for (int q = 0; q < m; ++q) dmr[c + q] = -v[q];
            }
          }
        }
      } else {
        // every accumulator value is an integer below 2^24 (exact in fp32); the float64
        // sum over levels is the only rounding step
        double *dst = (g.to_p64[s / g.per_block] ? g.p64 : g.y64) + off;
        const double scale = ldexp(1.0, g.es[s] + g.eF - 6 * L);
        for (int c = c_begin; c < c_end; c += 16) {
          float v[16];
          tmem_ld16(taddr + (uint32_t)c, v);
          if (a < g.Nv) {
            const int m = min(16, nvalid - c);
            if (m == 16 && (g.Nv & 1) == 0) {
              double2 *d2 = reinterpret_cast<double2 *>(dst + c);
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                double2 o = first ? make_double2(0.0, 0.0) : d2[q];
                o.x += (double)v[2 * q] * scale;
                o.y += (double)v[2 * q + 1] * scale;
                d2[q] = o;
              }
            } else {
              for (int q = 0; q < m; ++q) dst[c + q] = (first ? 0.0 : dst[c + q]) + (double)v[q] * scale;
            }
          }
        }
      }
      tc_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);
      }
    }
  }
  tc_before();
  __syncthreads();
  if (warp == 1) {
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
  if (threadIdx.x == 0 && fail) atomicOr(g.err, 1);
}

// Exact digit split of float64 slices (Ozaki-type splitting): with 2^e the smallest power
// of two above 2 max |x_s|, z = x / 2^e lies in (-1/2, 1/2); Z = round(z 64^P) is an integer
// of magnitude <= 2^(6P-1) (exact in int64 for P <= 9), and its balanced base-64 digits
//     Z = sum_{p=1..P} d_p 64^(P-p),  d_p in [-32, 31] for p >= 2, d_1 in [-32, 32]
// give z = sum_p d_p 64^-p to within 64^-P / 2.  Every d_p is exact in bf16 and every
// product of two digits is an integer of magnitude <= 2^10.
// Per-slice exponent: one CTA per slice, element (r, c) of slice s at s*sstride + r*ld + c*cs;
// with a slice list, CTA k takes slice list[k] (the other slices are left alone).
__global__ void k_slice_exp(const double *x, int rows, int cols, int64_t ld, int64_t sstride, int *es,
                            int64_t cs = 1, const int *list = nullptr) {
  __shared__ double red[32];
  const int sl = list ? list[blockIdx.x] : (int)blockIdx.x;
  const double *X = x + sl * sstride;
  double m = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)rows * cols; e += blockDim.x)
    m = fmax(m, fabs(X[(e / cols) * ld + (e % cols) * cs]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) {
      int e = 0;
      if (m > 0.0) frexp(m, &e);   // m = f 2^e with f in [0.5, 1): 2 max |x| < 2^(e+1)
      es[sl] = m > 0.0 ? e + 1 : 0;
    }
  }
}

// digits: out[p][s][r][c] (row pitch Nvp, pad columns zero), plane = S * rows * Nvp.
// One CTA iteration per row; one float64 multiply and one conversion per element, the rest
// is integer arithmetic.
// With a slice list (nlist entries) only the listed slices are split; every slice keeps its
// place in the digit planes (plane p, slice s at (p S + s) rows Nvp).
__global__ void k_digits(const double *x, int S, int rows, int cols, int Nvp, int64_t ld, int64_t sstride,
                         const int *es, int P, __nv_bfloat16 *out, int64_t cs = 1, const int *list = nullptr,
                         int nlist = 0) {
  const int64_t plane = (int64_t)S * rows * Nvp;
  const int64_t nrows = (int64_t)(list ? nlist : S) * rows;
  for (int64_t li = blockIdx.x; li < nrows; li += gridDim.x) {
    const int s = list ? list[li / rows] : (int)(li / rows), r = (int)(li % rows);
    const int64_t row = (int64_t)s * rows + r;
    const double scale = ldexp(1.0, 6 * P - es[s]);
    const double *src = x + s * sstride + r * ld;
    __nv_bfloat16 *dst = out + row * Nvp;
    for (int c = threadIdx.x; c < Nvp; c += blockDim.x) {
      long long Z = c < cols ? __double2ll_rn(src[c * cs] * scale) : 0;
      for (int p = P - 1; p > 0; --p) {   // least significant digit first
        const long long d = ((Z + 32) & 63) - 32;
        Z = (Z - d) >> 6;                 // exact: Z - d is a multiple of 64
        dst[p * plane + c] = __int2bfloat16_rn((int)d);
      }
      dst[c] = __int2bfloat16_rn((int)Z);  // leading digit, |Z| <= 32
    }
  }
}

// bf16 copies: dst[s][r][c] (row pitch Nvp) = src[s][r][c] (row pitch Nv); pad columns zero.
template <typename T>
__global__ void k_to_bf16(const T *src, __nv_bfloat16 *dst, int64_t rows, int Nv, int Nvp) {
  const int64_t n = rows * Nvp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Nvp;
    const int c = (int)(e % Nvp);
    dst[e] = __float2bfloat16_rn(c < Nv ? (float)src[r * Nv + c] : 0.f);
  }
}

__global__ void k_fvv_bf16(const double *F, int No, int Nv, int Nvp, __nv_bfloat16 *dst) {
  const int N = No + Nv;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Nv * Nvp; e += gridDim.x * blockDim.x) {
    const int r = e / Nvp, c = e % Nvp;
    dst[e] = __float2bfloat16_rn(c < Nv ? (float)F[(int64_t)(No + r) * N + No + c] : 0.f);
  }
}

}  // namespace tc

// ------------------------------------------------------------------------ host side
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool get_encode() {
  if (g_encode) return true;
  cudaDriverEntryPointQueryResult q;
  void *fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return false;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return true;
}

// bf16 tensor of `rank` dims (innermost first), 128-byte swizzle, zero fill out of bounds.
bool make_map(CUtensorMap *m, const void *base, int rank, const uint64_t *dims, const uint64_t *strides_bytes,
              const uint32_t *box) {
  uint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void *>(base),
                        reinterpret_cast<const cuuint64_t *>(dims), reinterpret_cast<const cuuint64_t *>(strides_bytes),
                        reinterpret_cast<const cuuint32_t *>(box), estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}
}  // namespace

bool tma_map_2d(CUtensorMap *m, const void *base, bool f32, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                uint32_t box_inner, uint32_t box_outer, int swizzle_bytes) {
  if (!get_encode()) return false;
  const uint64_t dims[2] = {inner, outer};
  const uint64_t strides[1] = {row_bytes};
  const uint32_t box[2] = {box_inner, box_outer};
  const uint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw = swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                : swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                                      : CU_TENSOR_MAP_SWIZZLE_NONE;
  CUresult r = g_encode(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<void *>(base), reinterpret_cast<const cuuint64_t *>(dims),
                        reinterpret_cast<const cuuint64_t *>(strides), reinterpret_cast<const cuuint32_t *>(box), estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {
// Fills the tile geometry of `g` and launches k_virt.  xd: bf16 x planes [planes][S_plane][Nv][Nvp];
// Fd: bf16 F planes [F_planes][Nv][Nvp]; Nvp = Nv rounded up to 8 (16-byte row pitch).
const char *launch_virt(cudaStream_t st, const void *xd, int x_planes, const void *Fd, int F_planes, tc::Args &g,
                        double alg_flops, double exec_flops, int family = ESMP2_KT_CONTRACTION) {
  const int Nv = g.Nv, Nvp = (Nv + 7) & ~7;
  if (!get_encode()) return "cuTensorMapEncodeTiled unavailable";
  if (g.nslices <= 0) return nullptr;
  CUtensorMap mXa, mXb, mFa, mFb;
  const uint64_t dX[3] = {(uint64_t)Nvp, (uint64_t)Nv, (uint64_t)g.S_plane * x_planes};
  const uint64_t sX[2] = {(uint64_t)Nvp * 2, (uint64_t)Nvp * Nv * 2};
  const uint64_t dF[3] = {(uint64_t)Nvp, (uint64_t)Nv, (uint64_t)F_planes};
  g.a_tiles = (Nv + tc::BM - 1) / tc::BM;
  if (g.bn <= 0 || g.bn > tc::BN_MAX || (g.bn & 15)) {   // default column tile: fewest tiles of <= 256
    g.b_tiles = (Nv + tc::BN_MAX - 1) / tc::BN_MAX;
    g.bn = ((Nv + g.b_tiles - 1) / g.b_tiles + 15) & ~15;
  } else {
    g.b_tiles = (Nv + g.bn - 1) / g.bn;
  }
  g.nk = (Nv + tc::BK - 1) / tc::BK;
  g.tiles = (int64_t)g.nslices * g.a_tiles * g.b_tiles;
  const uint32_t boxXa[3] = {64, 128, 1}, boxXb[3] = {64, 64, 1}, boxFa[3] = {64, 128, 1};
  const uint32_t boxFb[3] = {64, (uint32_t)g.bn, 1};
  if (!make_map(&mXa, xd, 3, dX, sX, boxXa) || !make_map(&mXb, xd, 3, dX, sX, boxXb) ||
      !make_map(&mFa, Fd, 3, dF, sX, boxFa) || !make_map(&mFb, Fd, 3, dF, sX, boxFb))
    return "tensor map encoding failed";
  if (smem_limit_once(reinterpret_cast<const void *>(tc::k_virt), tc::SMEM_BYTES) != cudaSuccess)
    return "cannot raise the shared-memory limit of the tensor-core kernel";
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<int64_t>(g.tiles, sms);
  KScope ks(st, family, alg_flops, exec_flops);
  tc::k_virt<<<grid, tc::NTHREADS, tc::SMEM_BYTES, st>>>(mXa, mXb, mFa, mFb, g);
  return nullptr;
}

tc::Args plain_args(int Nv, int S, float *y, int *err) {
  tc::Args g{};
  g.Nv = Nv;
  g.nslices = S;
  g.slices = nullptr;
  g.per_block = S;
  for (int b = 0; b < 5; ++b) g.tm[b] = 2;
  g.first = 1;
  g.npairs = 1;
  g.S_plane = S;
  g.mode = 0;
  g.y32 = y;
  g.err = err;
  return g;
}
}  // namespace

// Inner-solve form: only T, X, Y slices with i < j and every S, Z slice are contracted; the
// slice (j, i) of T, X, Y receives -y_ij (the blocks are antisymmetric under i <-> j).
// bn: column tile width (0 = the default, fewest tiles of at most 256 columns).
static esmp2_status virt_bf16_sym_bn(esmp2_handle *h, const void *xb, const void *Fb, float *y, int *err, int bn) {
  if (esmp2_status s0 = ensure_slist(h)) return s0;
  const int No = h->d.No, S = 5 * No * No, half = No * (No - 1) / 2;
  const double nv = h->d.Nv, nv3 = nv * nv * nv;
  tc::Args g = plain_args(h->d.Nv, S, y, err);
  g.bn = bn;
  g.nslices = h->nslist;
  g.slices = h->slist;
  g.per_block = No * No;
  g.No = No;
  g.mirror = 1;
  // both terms of a slice share one pass (two one-term passes were measured slower: No=30
  // Nv=400 inner contraction 4.2 ms against 2.0 ms)
  const double exec1 = 4.0 * nv3 * 3 * half + 4.0 * nv3 * 2 * No * No;
  if (const char *m = launch_virt(h->stream, xb, 1, Fb, 1, g, alg_virtual_flops(No, h->d.Nv), exec1)) {
    h->err = m;
    return ESMP2_ERR_CUDA;
  }
  h->launches += 1;
  return check_cuda(h, cudaGetLastError(), "virt_bf16_sym");
}

// Tile table keyed by (No, Nv): on the first inner contraction of a shape in this process,
// the candidate column tile widths are timed on the handle's own operands (CUDA events,
// one warm-up and one timed launch each) and the fastest is kept for every later call.
// Candidates: the default, half of it, and 256 when Nv > 256.
namespace {
std::mutex g_tile_mu;
std::map<std::pair<int, int>, int> g_tile_table;
}  // namespace

int tuned_column_tile(esmp2_handle *h, const void *xb, const void *Fb, float *y, int *err) {
  const std::pair<int, int> key(h->d.No, h->d.Nv);
  {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tile_table.find(key);
    if (it != g_tile_table.end()) return it->second;
  }
  const int Nv = h->d.Nv;
  const int nt = (Nv + tc::BN_MAX - 1) / tc::BN_MAX;
  const int def = ((Nv + nt - 1) / nt + 15) & ~15;
  std::vector<int> cand = {def};
  const int halfw = ((def / 2) + 15) & ~15;
  if (halfw >= 32 && halfw != def) cand.push_back(halfw);
  if (Nv > tc::BN_MAX && def != tc::BN_MAX) cand.push_back(tc::BN_MAX);
  int best = def;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  if (cand.size() > 1 && cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    for (int bn : cand) {
      if (virt_bf16_sym_bn(h, xb, Fb, y, err, bn)) continue;
      cudaEventRecord(e0, h->stream);
      if (virt_bf16_sym_bn(h, xb, Fb, y, err, bn)) continue;
      cudaEventRecord(e1, h->stream);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = bn;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  std::lock_guard<std::mutex> lk(g_tile_mu);
  g_tile_table[key] = best;
  return best;
}

esmp2_status virt_bf16_sym(esmp2_handle *h, const void *xb, const void *Fb, float *y, int *err) {
  return virt_bf16_sym_bn(h, xb, Fb, y, err, tuned_column_tile(h, xb, Fb, y, err));
}

// y[s][a][b] = sum_c xb[s][a][c] F[c][b] + sum_c F[a][c] xb[s][c][b]  for S slices (fp32 out).
// xb: bf16 [S][Nv][Nvp], Fb: bf16 [Nv][Nvp], Nvp = Nv rounded up to 8 (16-byte row pitch).
esmp2_status virt_bf16(esmp2_handle *h, const void *xb, const void *Fb, int S, float *y, int *err) {
  tc::Args g = plain_args(h->d.Nv, S, y, err);
  const double nv = h->d.Nv, exec = 4.0 * nv * nv * nv * S;
  const double alg = S == 5 * h->d.No * h->d.No ? alg_virtual_flops(h->d.No, h->d.Nv) : exec;
  if (const char *m = launch_virt(h->stream, xb, 1, Fb, 1, g, alg, exec)) { h->err = m; return ESMP2_ERR_CUDA; }
  h->launches += 1;
  return check_cuda(h, cudaGetLastError(), "virt_bf16");
}

// ---- float64-accurate virtual-index terms from exact digit products on the tensor cores.
// x_s = 2^{e_s} sum_p d_p 64^-p and F_vv = 2^{e_F} sum_q f_q 64^-q (Lmax - 1 digits each);
// level L = p + q collects every digit pair of that weight in one fp32 accumulator.  A
// level-L sum over both terms and K = Nv is an integer of magnitude <= 2 Nv (L - 1) 2^10,
// below 2^24 whenever Nv < 2^13 / (L - 1): fp32 accumulation is then exact and the float64
// sum over levels 2 .. Lmax is the only rounding.  The x digits stop 2^{-6 (Lmax - 1) - 1}
// below 2^{e_s}, and the dropped pairs (p + q > Lmax) weigh as little, so the result carries
// a relative error of order 2^{-6 (Lmax - 1)} against the largest term of each slice.
// sym = 1: T, X, Y slices (exactly antisymmetric) take only x F on i < j into p64 and the
// caller forms y_ij = P_ij - P_ij^T; S and Z slices take x F + F x into y.
// sym = 2: as sym = 1, and the S slices (S_ij^ab = S_ji^ba exactly) also take only x F into
// p64: F x_ij = (x_ji F)^T, so the caller forms y_ij = P_ij + P_ji^T.
// sym = 0: every slice takes both terms into y (any input).
namespace {
constexpr int kSplitMaxLevels = 10;

__global__ void k_split_list(int No, int *list) {
  // T, X, Y slices with i < j, then every S and Z slice
  const int NN = No * No, half = No * (No - 1) / 2;
  const int n = 3 * half + 2 * NN;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int s;
    if (e < 3 * half) {
      const int blk = e / half == 0 ? 0 : (e / half == 1 ? 2 : 3);
      int k = e % half, i = 0;
      while (k >= No - 1 - i) { k -= No - 1 - i; ++i; }
      s = blk * NN + i * No + (i + 1 + k);
    } else {
      const int f = e - 3 * half;
      s = (f < NN ? 1 : 4) * NN + f % NN;
    }
    list[e] = s;
  }
}
}  // namespace

int split_levels_for(double tol) {
  // keep 2^{-6 (Lmax - 1)} at or below 1e-4 tol (refinement and energy stay float64-exact)
  const double need = std::log2(1e4 / std::max(tol, 1e-300)) / 6.0;
  return std::max(2, std::min(kSplitMaxLevels, (int)std::ceil(need) + 1));
}

bool split_supported(const esmp2_handle *h, int levels) {
  if (levels < 2 || levels > kSplitMaxLevels) return false;
  return 2LL * h->d.Nv * (levels - 1) * 1024 < (1LL << 24);
}

esmp2_status ensure_slist(esmp2_handle *h) {
  if (h->slist) return ESMP2_OK;
  const int No = h->d.No;
  const int nl = 3 * (No * (No - 1) / 2) + 2 * No * No;
  cudaError_t e = dmalloc(reinterpret_cast<void **>(&h->slist), sizeof(int) * (size_t)nl, h->stream);
  if (e != cudaSuccess) { h->slist = nullptr; return check_cuda(h, e, "slice list"); }
  h->nslist = nl;
  k_split_list<<<(unsigned)cdiv(nl, 256), 256, 0, h->stream>>>(No, h->slist);
  h->launches += 1;
  return check_cuda(h, cudaGetLastError(), "slice list");
}

esmp2_status ensure_split(esmp2_handle *h) {
  if (h->xdig) return ESMP2_OK;
  if (esmp2_status s0 = ensure_slist(h)) return s0;
  const int No = h->d.No, Nv = h->d.Nv, N = h->d.N, Nvp = (Nv + 7) & ~7;
  const int S = 5 * No * No, P = kSplitMaxLevels - 1;
  cudaError_t e = dmalloc(&h->xdig, sizeof(__nv_bfloat16) * (size_t)P * S * Nv * Nvp, h->stream);
  if (e == cudaSuccess) e = dmalloc(&h->Fdig, sizeof(__nv_bfloat16) * (size_t)P * Nv * Nvp, h->stream);
  if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void **>(&h->es), sizeof(int) * (size_t)(S + 4), h->stream);
  if (e != cudaSuccess) {
    dfree(h->xdig, h->stream); dfree(h->Fdig, h->stream); dfree(h->es, h->stream);
    h->xdig = h->Fdig = nullptr; h->es = nullptr;
    return check_cuda(h, e, "split workspace");
  }
  if (!h->dflag) {
    if ((e = dmalloc(reinterpret_cast<void **>(&h->dflag), sizeof(int), h->stream)) != cudaSuccess)
      return check_cuda(h, e, "split workspace");
    cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream);
  }
  // digits of F_vv (the same block in the TOP and the semicanonical-occupied basis); the
  // leading digits do not depend on how many are kept
  const double *Fv = h->F + (int64_t)No * N + No;
  tc::k_slice_exp<<<1, 256, 0, h->stream>>>(Fv, Nv, Nv, N, 0, h->es + S);
  tc::k_digits<<<256, 256, 0, h->stream>>>(Fv, 1, Nv, Nv, Nvp, N, 0, h->es + S, P,
                                           static_cast<__nv_bfloat16 *>(h->Fdig));
  h->launches += 3;
  e = cudaMemcpyAsync(&h->eF, h->es + S, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return check_cuda(h, e, "split setup");
}

esmp2_status virt_split(esmp2_handle *h, const double *x, double *y, double *p64, int sym, int levels) {
  if (!split_supported(h, levels)) { h->err = "digit-split contraction not exact for this Nv"; return ESMP2_ERR_UNSUPPORTED; }
  esmp2_status s = ensure_split(h);
  if (s) return s;
  const int No = h->d.No, Nv = h->d.Nv, Nvp = (Nv + 7) & ~7;
  const int S = 5 * No * No, P = kSplitMaxLevels - 1;
  const int64_t NvNv = (int64_t)Nv * Nv;
  // the symmetric forms read only the listed slices (T, X, Y with i < j, all of S and Z)
  const int *list = sym ? h->slist : nullptr;
  const int nsl = sym ? h->nslist : S;
  tc::k_slice_exp<<<nsl, 256, 0, h->stream>>>(x, Nv, Nv, Nv, NvNv, h->es, 1, list);
  tc::k_digits<<<1216, 256, 0, h->stream>>>(x, S, Nv, Nv, Nvp, Nv, NvNv, h->es, levels - 1,
                                            static_cast<__nv_bfloat16 *>(h->xdig), 1, list, nsl);
  h->launches += 2;
  const int half = No * (No - 1) / 2;
  {  // every level 2 .. levels of every tile in one launch
    const int L = levels;
    tc::Args g{};
    g.Nv = Nv;
    g.nslices = sym ? h->nslist : S;
    g.slices = sym ? h->slist : nullptr;
    g.per_block = No * No;
    for (int b = 0; b < 5; ++b) {
      const bool one = (b == 0 || b == 2 || b == 3) || (sym == 2 && b == 1);
      g.tm[b] = (sym && one) ? 1 : 2;
      g.to_p64[b] = sym && one;
    }
    g.S_plane = S;
    g.lmin = 2;                   // level l pairs digit p of x with digit l - p of F
    g.lmax = L;
    g.npairs = L * (L - 1) / 2;   // digit pairs over all levels
    g.mode = 1;
    g.y64 = y;
    g.p64 = p64;
    g.es = h->es;
    g.eF = h->eF;
    g.first = 1;
    g.err = h->dflag;
    // the method's work is one contraction of the block vector, however many digit pairs
    // emulate it; the tensor cores execute every pair on the stored slices
    const double nv3 = (double)Nv * Nv * Nv;
    const double per_pair = sym ? 3.0 * half * 2.0 * nv3 + (sym == 2 ? 6.0 : 8.0) * No * No * nv3 : 4.0 * nv3 * S;
    const double alg = sym ? alg_virtual_flops(No, Nv) : per_pair;
    if (const char *m = launch_virt(h->stream, h->xdig, P, h->Fdig, P, g, alg, g.npairs * per_pair, ESMP2_KT_DIGITS)) {
      h->err = m;
      return ESMP2_ERR_CUDA;
    }
    h->launches += 1;
  }
  return check_cuda(h, cudaGetLastError(), "virt_split");
}

// Y = X M (rows x Nv times an Nv x Nv matrix M, rows a multiple of Nv) in float64 accuracy from
// exact digit products on the tensor cores (ten levels): the right-factor form of the orbital
// rotations (M = W_v for the integral transforms, the virtual rotation of the reduced-cost
// basis).  X is read as rows/Nv slices of Nv x Nv.  The digit planes of M^T (row b' holds column
// b' of M, the K-major right operand) are built on first use into *dig with the power-of-two
// scale in es[eslot] (device) and *eM (host).
esmp2_status xwm_split(esmp2_handle *h, const double *X, int64_t rows, double *Y, const double *M, void **dig,
                       int *eM, int eslot) {
  esmp2_status s = ensure_split(h);
  if (s) return s;
  const int No = h->d.No, Nv = h->d.Nv, Nvp = (Nv + 7) & ~7;
  const int S = (int)(rows / Nv), P = kSplitMaxLevels - 1, levels = kSplitMaxLevels;
  if (rows % Nv != 0 || S > 5 * No * No || (int64_t)(levels - 1) * Nv * 1024 >= (1LL << 24)) {
    h->err = "xwm_split: unsupported shape";
    return ESMP2_ERR_UNSUPPORTED;
  }
  const int64_t NvNv = (int64_t)Nv * Nv;
  if (!*dig) {
    cudaError_t e = dmalloc(dig, sizeof(__nv_bfloat16) * (size_t)P * Nv * Nvp, h->stream);
    if (e != cudaSuccess) return check_cuda(h, e, "rotation digits");
    int *ed = h->es + 5 * No * No + eslot;
    tc::k_slice_exp<<<1, 256, 0, h->stream>>>(M, Nv, Nv, 1, 0, ed, Nv);
    tc::k_digits<<<256, 256, 0, h->stream>>>(M, 1, Nv, Nv, Nvp, 1, 0, ed, P, static_cast<__nv_bfloat16 *>(*dig), Nv);
    e = cudaMemcpyAsync(eM, ed, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->launches += 2;
    if (e != cudaSuccess) return check_cuda(h, e, "rotation digits");
  }
  tc::k_slice_exp<<<S, 256, 0, h->stream>>>(X, Nv, Nv, Nv, NvNv, h->es);
  tc::k_digits<<<1216, 256, 0, h->stream>>>(X, S, Nv, Nv, Nvp, Nv, NvNv, h->es, P,
                                            static_cast<__nv_bfloat16 *>(h->xdig));
  h->launches += 2;
  {  // levels 2 .. levels of every tile in one launch
    tc::Args g{};
    g.Nv = Nv;
    g.nslices = S;
    g.slices = nullptr;
    g.per_block = S;
    for (int b = 0; b < 5; ++b) { g.tm[b] = 1; g.to_p64[b] = 1; }
    g.S_plane = S;
    g.lmin = 2;
    g.lmax = levels;
    g.npairs = levels * (levels - 1) / 2;   // pairs over all levels (flop accounting)
    g.mode = 1;
    g.y64 = nullptr;
    g.p64 = Y;
    g.es = h->es;
    g.eF = *eM;
    g.first = 1;
    g.err = h->dflag;
    const double fl = 2.0 * (double)rows * Nv * Nv;   // one float64-accurate rotation
    if (const char *m = launch_virt(h->stream, h->xdig, P, *dig, P, g, fl, g.npairs * fl, ESMP2_KT_DIGITS)) {
      h->err = m;
      return ESMP2_ERR_CUDA;
    }
    h->launches += 1;
  }
  return check_cuda(h, cudaGetLastError(), "xwm_split");
}

esmp2_status xwv_split(esmp2_handle *h, const double *X, int64_t rows, double *Y) {
  return xwm_split(h, X, rows, Y, h->Wv, &h->Rdig, &h->eR, 1);
}

void to_bf16_f64(esmp2_handle *h, const double *src, void *dst, int64_t rows) {
  const int Nv = h->d.Nv, Nvp = (Nv + 7) & ~7;
  tc::k_to_bf16<double><<<1216, 256, 0, h->stream>>>(src, static_cast<__nv_bfloat16 *>(dst), rows, Nv, Nvp);
  h->launches += 1;
}
void to_bf16_f32(esmp2_handle *h, const float *src, void *dst, int64_t rows) {
  const int Nv = h->d.Nv, Nvp = (Nv + 7) & ~7;
  tc::k_to_bf16<float><<<1216, 256, 0, h->stream>>>(src, static_cast<__nv_bfloat16 *>(dst), rows, Nv, Nvp);
  h->launches += 1;
}
void fvv_bf16(esmp2_handle *h, const double *F, void *dst) {
  const int Nv = h->d.Nv, Nvp = (Nv + 7) & ~7;
  tc::k_fvv_bf16<<<256, 256, 0, h->stream>>>(F, h->d.No, Nv, Nvp, static_cast<__nv_bfloat16 *>(dst));
  h->launches += 1;
}

}  // namespace esmp2

// ---------------------------------------------------------------------------------------
// Allocation-free variant of the bf16 virtual-index contraction.
//
// Some callers cannot allocate device memory at the point where they need this
// contraction: code that runs while another framework owns the whole device heap through
// its own caching allocator (a cudaMalloc there fails or fragments that allocator's
// budget), and latency-critical loops where a cudaMalloc/cudaFree pair would synchronise
// the device.  For them the scratch (bf16 copies of x and F, the fp32 accumulator output
// and an error flag) lives in one file-scope device array of ESMP2_NOALLOC_MAX_BYTES.
// Every GPU that loads this library holds that array until the process exits.
namespace esmp2 {
namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[ESMP2_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
unsigned char *g_noalloc_ptr[kMaxDevices] = {nullptr};

__global__ void k_noalloc_f32_to_f64(const float *src, double *dst, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (double)src[e];
}

inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace
}  // namespace esmp2

extern "C" esmp2_status esmp2_virtual_contraction_noalloc(const double *x, const double *Fvv, double *y, int S,
                                                         int Nv, void *stream) {
  using namespace esmp2;
  if (!x || !Fvv || !y || S < 1 || Nv < 1) return ESMP2_ERR_INVALID_ARG;
  const int Nvp = (Nv + 7) & ~7;
  const size_t off_F = 256;
  const size_t off_x = off_F + align256(sizeof(__nv_bfloat16) * (size_t)Nv * Nvp);
  const size_t off_y = off_x + align256(sizeof(__nv_bfloat16) * (size_t)S * Nv * Nvp);
  const size_t total = off_y + align256(sizeof(float) * (size_t)S * Nv * Nv);
  if (total > (size_t)ESMP2_NOALLOC_MAX_BYTES) return ESMP2_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ESMP2_ERR_CUDA;
  if (!g_noalloc_ptr[dev]) {  // one-time set-up on this device
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ESMP2_ERR_CUDA;
    g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
  }
  if (!get_encode()) return ESMP2_ERR_CUDA;
  unsigned char *base = g_noalloc_ptr[dev];
  int *err = reinterpret_cast<int *>(base);
  auto *Fb = reinterpret_cast<__nv_bfloat16 *>(base + off_F);
  auto *xb = reinterpret_cast<__nv_bfloat16 *>(base + off_x);
  float *y32 = reinterpret_cast<float *>(base + off_y);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: the error flag must start at zero
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return ESMP2_ERR_CUDA;
  tc::k_fvv_bf16<<<256, 256, 0, st>>>(Fvv, 0, Nv, Nvp, Fb);
  tc::k_to_bf16<double><<<1216, 256, 0, st>>>(x, xb, (int64_t)S * Nv, Nv, Nvp);
  tc::Args g = plain_args(Nv, S, y32, err);
  const double exec = 4.0 * (double)Nv * Nv * Nv * S;
  if (launch_virt(st, xb, 1, Fb, 1, g, exec, exec)) return ESMP2_ERR_CUDA;
  k_noalloc_f32_to_f64<<<1216, 256, 0, st>>>(y32, y, (int64_t)S * Nv * Nv);
  int flag = 0;
  cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return ESMP2_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return ESMP2_ERR_CUDA;
  return flag ? ESMP2_ERR_TIMEOUT : ESMP2_OK;
}

// ---------------------------------------------------------------------------------------
// Failure-detection self-test of the bounded waits (the paper has no counterpart).
// One CTA of the tensor-core kernel runs on a 16 x 16 slice held in the allocation-free
// scratch array with its producer told to issue no copies: the MMA warp's first wait on a
// full slot and the epilogue's first wait on the accumulator run out after wait_ms with
// nothing in flight (no copy, no MMA, no TMEM load was issued), the CTA frees its TMEM and
// raises the error flag, and the host reads the flag like any other call.
extern "C" esmp2_status esmp2_selftest_bounded_wait(int wait_ms, void *stream) {
  using namespace esmp2;
  if (wait_ms < 1 || wait_ms > 2000) return ESMP2_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ESMP2_ERR_CUDA;
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ESMP2_ERR_CUDA;
    g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
  }
  if (!get_encode()) return ESMP2_ERR_CUDA;
  const int Nv = 16;
  unsigned char *base = g_noalloc_ptr[dev];
  int *err = reinterpret_cast<int *>(base);
  void *op = base + 256;                                // operand maps need a valid address only
  float *y32 = reinterpret_cast<float *>(base + 4096);  // never written: no tile completes
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(base, 0, 8192, st) != cudaSuccess) return ESMP2_ERR_CUDA;
  tc::Args g = plain_args(Nv, 1, y32, err);
  g.wait_ns = (uint64_t)wait_ms * 1000000ull;
  g.no_copies = 1;
  if (launch_virt(st, op, 1, op, 1, g, 0.0, 0.0)) return ESMP2_ERR_CUDA;
  int flag = 0;
  if (cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return ESMP2_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return ESMP2_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return ESMP2_ERR_CUDA;
  return flag ? ESMP2_ERR_TIMEOUT : ESMP2_OK;
}

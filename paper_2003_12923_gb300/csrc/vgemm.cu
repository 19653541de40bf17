// Virtual-index contraction of the inner sigma as one dense GEMM on the 5th-generation tensor
// cores (the N_o^2 N_v^3 terms of Table 1, Eq. qfq_replacement): bf16 operands (kind::f16) or
// float32 operands read as tf32 (kind::tf32), fp32 accumulation in TMEM.
//
// Every slice s of the packed inner vector is an Nv x Nv matrix X_s with rows a and columns
// c; the terms of a slice are X_s F and F X_s (F = F_vv, symmetric).  Stacking the rows of
// all slices gives one matrix A with rows r = (s, a), and
//     P = A F,   P[r][b] = sum_c A[r][c] F[c][b]
// is a plain GEMM with M = (#slices) Nv, N = K = Nv: no per-slice tile padding.  The second
// term of each slice is the transpose of a first term: F X_s = -(X_s F)^T for the
// antisymmetric T, X, Y slices, F S_ij = (S_ji F)^T for the spin-flip-symmetric S slices,
// and for Z the operand also holds the transposed slices Z_s^T, whose rows of P are stored
// transposed here, (Z_s^T F)^T = F Z_s.  The coupling pass forms y from P.
//
// Structure (persistent, 320 threads):
//   each CTA owns one column tile b0 .. b0 + Nt - 1 of the result (columns split over nN
//   tiles) and keeps that tile's panel W[b][c] (all K) resident in shared memory;
//   warp 0      TMA producer: 2-D tiled bulk copies of 128-row x 64-byte A chunks (32 bf16 or
//               16 float32 columns; 64-byte swizzle) into a ring of 5 to 8 slots (what the
//               panel leaves)
//   warp 1      one thread issues tcgen05.mma (M = 128, N = Nt, K = 16 bf16 or 8 tf32, 32 bytes
//               of each operand row per instruction), commits to mbarriers
//   warps 2..9  epilogue: tcgen05.ld 32x32b from one of two TMEM accumulators (2 x Nt
//               columns), fp32 stores of P rows (16-byte vectors) or of transposed rows (one
//               128-byte segment per column and warp)
// Every mbarrier wait is bounded (globaltimer); a wait that runs out raises the error flag,
// the CTA waits (bounded) for its own copies in flight and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"

namespace esmp2 {
namespace vg {

constexpr int BM = 128;                 // accumulator rows (TMEM lanes)
constexpr int CHUNK_B = 64;             // bytes of one operand row per K chunk (the swizzle span)
constexpr int MAX_STAGES = 8;
constexpr int A_STAGE = BM * CHUNK_B;   // 8 KB
// K elements per chunk and per MMA: bf16 32 and 16, tf32 16 and 8 (both 32 bytes per MMA)
template <bool TF32> struct Kind {
  static constexpr int BK = TF32 ? 16 : 32;
  static constexpr int KMMA = TF32 ? 8 : 16;
};
constexpr int NTHREADS = 320;
// dynamic shared memory per CTA: the 232448-byte opt-in limit less room for the kernel's
// static shared memory (barriers, TMEM address, flags, the epilogue's 10 KB staging tile)
constexpr int SMEM_MAX = 232448 - 2048 - 10240;
constexpr uint64_t WAIT_NS = 2000000000ull;

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
// bounded wait: true when the phase of the given parity has completed
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, uint64_t limit = WAIT_NS) {
  const uint32_t a = smem_u32(b);
  if (mbar_test(a, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_test(a, parity))
    if (gtimer() - t0 > limit) return false;
  return true;
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

// Shared-memory matrix descriptor (tcgen05), K-major operand with 64-byte swizzle: start >> 4,
// leading byte offset 16 >> 4 (unused by swizzled K-major layouts), stride byte offset = one
// group of 8 rows of 64 bytes (512 >> 4), descriptor version 1 at bit 46, layout type 4
// (64-byte swizzle) at bit 61.
__device__ __forceinline__ uint64_t sdesc64(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) |
         (4ull << 61);
}
// Instruction descriptor: D fp32 (bits 4-5 = 1); A and B format (bits 7-9, 10-12) bf16 = 1 of
// kind::f16 or tf32 = 2 of kind::tf32; both K-major; N >> 3 at bit 17, M >> 4 at bit 24.
template <bool TF32>
__device__ __forceinline__ uint32_t idesc(int M, int N) {
  const uint32_t fmt = TF32 ? 2u : 1u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
template <bool TF32>
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (TF32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
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
  int64_t rows;         // rows of A and of the result, r = (slice, a)
  int64_t rows_normal;  // rows [0, rows_normal) go to P[r][b]; later rows to PT (transposed)
  int Nv;               // rows per slice (transposed part) and columns of the result
  int nk;               // K chunks (nk * BK >= Nv)
  int nN;               // column tiles; CTA c works on tile c % nN
  int Nt;               // columns of a column tile (multiple of 16, <= 256)
  int stages;           // ring slots (<= MAX_STAGES)
  int64_t m_tiles;      // ceil(rows / BM)
  float *P;             // [rows_normal][ldp]
  float *PT;            // [(rows - rows_normal) / Nv][Nv][ldp]: PT[s][b][c] = result row (s, c), column b
  int ldp;              // row pitch of P and PT (elements, a multiple of 4)
  int *err;             // device error flag
  // transposed rows stored as bf16 into PT16 instead of PT, optionally scaled element-wise
  // by the inverse diagonal of the reduced-cost basis (the preconditioner's middle factor):
  // element (slice s, a, b) of the stored slice times valid ? 1 / ((lam[a] + lam[b]) - occ[s]) : 0
  __nv_bfloat16 *PT16;
  const float *lam;     // [Nv] or nullptr (no scaling)
  const float *occ;     // [slices]
  const int *code;      // [slices]: block | 8 (i == 0) | 16 (j == 0)
};

// validity of element (a, b) of a slice with the given code (the masks of the block vector)
__device__ __forceinline__ bool vg_valid(int code, int a, int b) {
  const int blk = code & 7;
  const bool i0 = (code & 8) != 0, j0 = (code & 16) != 0;
  if ((blk == 0 || blk == 2 || blk == 3) && a == b) return false;
  if (blk == 2 && (i0 || j0 || a == 0 || b == 0)) return false;
  if (blk == 4 && (j0 || b == 0 || (i0 && a == 0))) return false;
  return true;
}

template <bool TF32>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_vgemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tF, Args g) {
  constexpr int BK = Kind<TF32>::BK, KMMA = Kind<TF32>::KMMA;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int STAGES = g.stages;
  uint8_t *ring = smem;                                  // STAGES x A_STAGE
  uint8_t *panel = smem + STAGES * A_STAGE;              // nk chunks of Nt rows x 64 bytes
  __shared__ uint64_t full[MAX_STAGES], empty[MAX_STAGES], acc_full[2], acc_empty[2], pbar;
  __shared__ uint32_t tmem_base;
  __shared__ int fail;
  // bf16 transposed output: per epilogue warp one 16-column x 32-row chunk, turned so that each
  // lane stores 16 consecutive rows of one column as two 16-byte vectors
  __shared__ __align__(16) __nv_bfloat16 stg[8][16][40];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = blockIdx.x % g.nN, group = gridDim.x / g.nN, gi = blockIdx.x / g.nN;
  const int b0 = nt * g.Nt, nvalid = min(g.Nt, g.Nv - b0), nmma = (nvalid + 15) & ~15;
  const uint32_t chunk_bytes = (uint32_t)g.Nt * CHUNK_B;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int s = 0; s < 2; ++s) { mbar_init(&acc_full[s], 1); mbar_init(&acc_empty[s], 8); }
    mbar_init(&pbar, 1);
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

  if (warp == 0) {
    if (lane == 0) {  // ------------------------------------------------ TMA producer
      bool ok = true;
      // the column tile's F panel, once
      mbar_expect_tx(&pbar, chunk_bytes * (uint32_t)g.nk);
      for (int kc = 0; kc < g.nk; ++kc) tma_2d(panel + kc * chunk_bytes, &tF, &pbar, kc * BK, b0);
      int64_t it = 0;
      for (int64_t m = gi; m < g.m_tiles && ok; m += group) {
        for (int kc = 0; kc < g.nk; ++kc, ++it) {
          const int st = (int)(it % STAGES);
          const uint32_t rnd = (uint32_t)(it / STAGES);
          if (!mbar_wait(&empty[st], (rnd & 1) ^ 1)) { ok = false; break; }
          mbar_expect_tx(&full[st], (uint32_t)A_STAGE);
          tma_2d(ring + st * A_STAGE, &tA, &full[st], kc * BK, (int)(m * BM));
        }
      }
      if (!ok) atomicExch(&fail, 1);
      // wait (bounded) until no copy of this CTA is still in flight
      mbar_wait(&pbar, 0, 100000000ull);
      for (int64_t j = it > STAGES ? it - STAGES : 0; j < it; ++j)
        mbar_wait(&full[j % STAGES], (uint32_t)((j / STAGES) & 1), 100000000ull);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ------------------------------------------------ MMA issuer
      bool ok = mbar_wait(&pbar, 0);
      tc_after();
      const uint32_t id = idesc<TF32>(BM, nmma);
      const uint32_t pan = smem_u32(panel), rg = smem_u32(ring);
      int64_t it = 0;
      int lt = 0;
      for (int64_t m = gi; m < g.m_tiles && ok; m += group, ++lt) {
        const int ab = lt & 1;
        const uint32_t ar = (uint32_t)(lt >> 1);
        if (!mbar_wait(&acc_empty[ab], (ar & 1) ^ 1)) { ok = false; break; }
        tc_after();
        const uint32_t d = tmem + (uint32_t)(ab * 256);
        for (int kc = 0; kc < g.nk; ++kc, ++it) {
          const int st = (int)(it % STAGES);
          const uint32_t rnd = (uint32_t)(it / STAGES);
          if (!mbar_wait(&full[st], rnd & 1)) { ok = false; break; }
          tc_after();
          const int ksteps = min(BK / KMMA, (g.Nv - kc * BK + KMMA - 1) / KMMA);   // skip K steps past Nv
          for (int k = 0; k < ksteps; ++k)
            umma<TF32>(d, sdesc64(rg + st * A_STAGE + 32 * k), sdesc64(pan + kc * chunk_bytes + 32 * k), id,
                       (kc > 0 || k > 0) ? 1u : 0u);
          umma_commit(&empty[st]);
        }
        if (!ok) break;
        umma_commit(&acc_full[ab]);
      }
      if (!ok) atomicExch(&fail, 1);
    }
  } else {  // ---------------------------------------------------------- epilogue
    const int quarter = warp & 3, chalf = (warp - 2) >> 2;
    const int hc = ((nvalid + 31) / 32) * 16;   // columns per half, a multiple of 16
    const int c_begin = chalf * hc, c_end = min(nvalid, c_begin + hc);
    int lt = 0;
    for (int64_t m = gi; m < g.m_tiles; m += group, ++lt) {
      const int ab = lt & 1;
      const uint32_t ar = (uint32_t)(lt >> 1);
      if (!mbar_wait(&acc_full[ab], ar & 1)) { if (lane == 0) atomicExch(&fail, 1); break; }
      tc_after();
      const int64_t r = m * BM + quarter * 32 + lane;
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * 256);
      const bool normal = r < g.rows_normal;
      // the warp's 32 rows form one run of a transposed slice (same slice, consecutive rows
      // starting on a multiple of 8): the staged 16-byte stores apply
      bool run = false;
      if (g.PT16) {
        const int64_t r0 = m * BM + quarter * 32, q0 = r0 - g.rows_normal;
        run = r0 >= g.rows_normal && r0 + 31 < g.rows && (q0 % g.Nv) + 31 < g.Nv && (q0 % g.Nv) % 8 == 0;
      }
      float *dst = nullptr;     // column b (< Nv) of this row
      __nv_bfloat16 *dst16 = nullptr;
      int64_t tpitch = 1;
      int rc = 0, rcode = 0;    // transposed rows: row within the slice, slice code
      float rocc = 0.f, rlam = 0.f;
      if (normal) {
        dst = g.P + r * g.ldp;
      } else if (r < g.rows) {
        const int64_t q = r - g.rows_normal, s = q / g.Nv, c = q % g.Nv;
        if (g.PT16) dst16 = g.PT16 + s * g.Nv * g.ldp + c;
        else dst = g.PT + s * g.Nv * g.ldp + c;   // column b at dst + b * ldp
        tpitch = g.ldp;
        rc = (int)c;
        if (g.lam) { rcode = g.code[s]; rocc = g.occ[s]; rlam = g.lam[c]; }
      }
      for (int c = c_begin; c < c_end; c += 16) {
        float v[16];
        tmem_ld16(taddr + (uint32_t)c, v);
        if (r >= g.rows) continue;
        const int bc = b0 + c, mcol = min(16, nvalid - c);
        if (dst16) {   // stored element (a = bc + q, b = rc) of the slice
          if (g.lam) {   // the fast division (2 ulp) serves the preconditioner: the denominator of
                         // (a, b) and of its image (b, a) is the same float, so M stays symmetric
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const int a = bc + q;
              v[q] = (q < mcol && vg_valid(rcode, a, rc)) ? __fdividef(v[q], (g.lam[a] + rlam) - rocc) : 0.f;
            }
          }
          if (run) {   // all 32 lanes here (every row of the warp is in range)
            __nv_bfloat16(*st)[40] = stg[warp - 2];
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 16; ++q) st[q][lane] = __float2bfloat16_rn(v[q]);
            __syncwarp();
            const int j = lane >> 1, hh = (lane & 1) * 16;   // column bc + j, rows hh .. hh + 15 of the run
            if (j < mcol) {
              const uint4 *src = reinterpret_cast<const uint4 *>(&st[j][hh]);
              uint4 *out = reinterpret_cast<uint4 *>(dst16 - lane + (int64_t)(bc + j) * tpitch + hh);
              out[0] = src[0];
              out[1] = src[1];
            }
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (q < mcol) dst16[(int64_t)(bc + q) * tpitch] = __float2bfloat16_rn(v[q]);
          }
        } else if (normal && mcol == 16) {
          float4 *d4 = reinterpret_cast<float4 *>(dst + bc);
#pragma unroll
          for (int q = 0; q < 4; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (q < mcol) dst[(int64_t)(bc + q) * tpitch] = v[q];
        }
      }
      tc_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);
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

}  // namespace vg

// Column tiling of the GEMM: the fewest column tiles (each at most 256 columns, a multiple of
// 16) whose resident panel and an operand ring of at least 5 slots fit the shared memory of
// one CTA; the ring takes what is left, up to MAX_STAGES slots.  bk: K elements per chunk.
static bool vgemm_tiling(int ncols, int Kc, int bk, int *nN, int *Nt, int *nk, int *stages, int *smem) {
  const int k = (Kc + bk - 1) / bk;
  for (int n = 1; n <= 64; ++n) {
    const int t = (((ncols + n - 1) / n) + 15) & ~15;
    const int fixed = 1024 + k * t * vg::CHUNK_B;
    if (t > 256 || fixed + 5 * vg::A_STAGE > vg::SMEM_MAX) continue;
    const int st = std::min(vg::MAX_STAGES, (vg::SMEM_MAX - fixed) / vg::A_STAGE);
    // at least 120 KB, so one CTA per SM: each CTA holds all 512 TMEM columns
    *nN = n; *Nt = t; *nk = k; *stages = st; *smem = std::max(fixed + st * vg::A_STAGE, 120 * 1024);
    return true;
  }
  return false;
}

// P = A W on the tensor cores.  A: rows x Nvp (row pitch Nvp elements), W: Nv x Nvp (row b of
// W is column b of the right factor), both bf16, or both float32 read as tf32 (tf32 = true).
esmp2_status vgemm(esmp2_handle *h, const void *A, int64_t rows, int64_t rows_normal, const void *W, float *P,
                   float *PT, int ldp, double alg_flops, bool tf32, const VgemmOut *out) {
  const int Nv = h->d.Nv, Nvp = (Nv + 7) & ~7;
  const int bk = tf32 ? vg::Kind<true>::BK : vg::Kind<false>::BK, esz = tf32 ? 4 : 2;
  int nN = 0, Nt = 0, nk = 0, stages = 0, smem = 0;
  if (!vgemm_tiling(Nv, Nv, bk, &nN, &Nt, &nk, &stages, &smem) || (ldp & 3) || rows <= 0) {
    h->err = "vgemm: unsupported shape";
    return ESMP2_ERR_UNSUPPORTED;
  }
  if (rows_normal < rows && (rows - rows_normal) % Nv != 0) {
    h->err = "vgemm: transposed rows must be whole slices";
    return ESMP2_ERR_UNSUPPORTED;
  }
  CUtensorMap mA, mW;
  if (!tma_map_2d(&mA, A, tf32, (uint64_t)Nvp, (uint64_t)rows, (uint64_t)Nvp * esz, (uint32_t)bk, vg::BM, 64) ||
      !tma_map_2d(&mW, W, tf32, (uint64_t)Nvp, (uint64_t)Nv, (uint64_t)Nvp * esz, (uint32_t)bk, (uint32_t)Nt, 64)) {
    h->err = "vgemm: tensor map encoding failed";
    return ESMP2_ERR_CUDA;
  }
  const void *fn = tf32 ? reinterpret_cast<const void *>(vg::k_vgemm<true>)
                        : reinterpret_cast<const void *>(vg::k_vgemm<false>);
  if (cudaError_t e = smem_limit_once(fn, vg::SMEM_MAX)) return check_cuda(h, e, "vgemm shared-memory limit");
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  vg::Args g{};
  g.rows = rows;
  g.rows_normal = rows_normal;
  g.Nv = Nv;
  g.nk = nk;
  g.nN = nN;
  g.Nt = Nt;
  g.stages = stages;
  g.m_tiles = (rows + vg::BM - 1) / vg::BM;
  g.P = P;
  g.PT = PT;
  g.ldp = ldp;
  g.err = h->dflag;
  if (out) {
    g.PT16 = static_cast<__nv_bfloat16 *>(out->PT16);
    g.lam = out->lam;
    g.occ = out->occ;
    g.code = out->code;
  }
  const int family = out ? out->family : ESMP2_KT_CONTRACTION;
  const int64_t per_group = std::max<int64_t>(1, std::min<int64_t>(g.m_tiles, sms / nN));
  const int grid = (int)(per_group * nN);
  const double exec = 2.0 * (double)g.m_tiles * vg::BM * (double)Nv * (double)nN * Nt;
  {
    KScope ks(h->stream, family, alg_flops, exec);
    if (tf32) vg::k_vgemm<true><<<grid, vg::NTHREADS, smem, h->stream>>>(mA, mW, g);
    else vg::k_vgemm<false><<<grid, vg::NTHREADS, smem, h->stream>>>(mA, mW, g);
  }
  h->launches += 1;
  return check_cuda(h, cudaGetLastError(), "vgemm");
}

}  // namespace esmp2

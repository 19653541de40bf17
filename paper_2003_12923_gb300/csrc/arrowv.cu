// The reduced-cost basis of the D + L solve (ESMP2_REDUCED_MIXED).
//
// The doubles and the L-triples are unchanged by any rotation of the occupied orbitals that
// fixes t and of the virtual orbitals that fixes t' (Sec. II.C: the first-order space is
// defined by the large TOP pair alone).  In the basis whose occupied orbitals other than t
// diagonalise F_oo and whose virtual orbitals other than t' diagonalise F_vv, both blocks of
// F are "arrow" shaped: a diagonal plus the t (t') row and column.  Then the virtual-index
// terms of the sigma build (the N_o^2 N_v^3 contractions of Table 1 in the TOP basis) become
//     (X F)_ab = F_bb X_ab + X_a0 F_0b  (b >= 1),   (X F)_a0 = sum_c X_ac F_c0,
//     (F X)_ab = F_aa X_ab + F_a0 X_0b  (a >= 1),   (F X)_0b = sum_c F_0c X_cb,
// streaming work with one row sum and one column sum per slice.  E2_D + E2_L is the same in
// exact arithmetic; E2_S (Sec. II.D) stays in the TOP basis.  The price is the one-time
// rotation of the right-hand side (and of the solution, when it is asked for), two float64-
// exact digit-split products per slice.
//
// The eigenvectors of the virtual block come from the one-sided (Hestenes) Jacobi method with
// the round-robin ordering of disjoint pairs: one launch per round, one warp per pair rotating
// two rows of B and of the accumulated rotation (all accesses along contiguous rows).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"

namespace esmp2 {
namespace {

__global__ void k_to_f32(const double *src, float *dst, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (float)src[e];
}

// A (m x m) = the virtual block of F without t' (rows and columns 1 .. Nv-1); V = I
__global__ void k_vblock(const double *F, int N, int No, int m, double *A, double *V) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / m), j = (int)(e % m);
    A[e] = F[(int64_t)(No + 1 + i) * N + No + 1 + j];
    V[e] = i == j ? 1.0 : 0.0;
  }
}

// One round r of the one-sided (Hestenes) Jacobi method on the symmetric positive definite
// m x m matrix held as the rows of B: the disjoint pairs (p, q) of the round-robin ordering of
// n = m (+1 if m is odd) indices, one CTA each, rotate rows p and q of B (B <- G^T B) until
// all rows are mutually orthogonal; the rotations accumulate into the rows of Jt (Jt <- G^T Jt).
// At convergence B = Jt A with orthogonal rows, so the rows of Jt are eigenvectors of A^2,
// hence of A (A positive definite).  Rotation of a pair: alpha = |b_p|^2, beta = |b_q|^2,
// gamma = b_p . b_q, zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 +
// zeta^2)), c = 1 / sqrt(1 + t^2), s = c t; skipped when |gamma| <= 1e-14 sqrt(alpha beta)
// (the remaining off-diagonal part of R^T A R is then of the order of 1e-14 of its diagonal).
// Rows are contiguous, so every access is coalesced.  *maxr2 receives the largest
// gamma^2 / (alpha beta) of the pairs that rotate (as float bits).
// Newton-Raphson refinements in float64 of float32 seeds: 1/sqrt(x) by y <- y (3 - x y^2) / 2 and
// 1/x by y <- y (2 - x y), two steps each (quadratic convergence from the seed's 2^-22 to the
// float64 rounding level); for x in a range where the float32 seed is a normal number
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * (1.5 - 0.5 * x * y * y);
  y = y * (1.5 - 0.5 * x * y * y);
  return y;
}
__device__ __forceinline__ double rcp_nr(double x) {
  double y = (double)(1.0f / (float)x);
  y = y * (2.0 - x * y);
  y = y * (2.0 - x * y);
  return y;
}

constexpr int kJT = 128;                 // threads per pair (one CTA)
constexpr int kJE = 8;                   // row elements per thread: m <= kJT kJE = 1024
__global__ void __launch_bounds__(kJT) k_jacobi_os_round(double *B, double *Jt, int m, int r, unsigned *maxr2) {
  __shared__ double red[3][kJT / 32];
  const int n = m + (m & 1), pi = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int p, q;
  if (pi == 0) {
    p = 0;
    q = 1 + (r % (n - 1));
  } else {
    p = 1 + ((pi + r) % (n - 1));
    q = 1 + ((n - 1 - pi + r) % (n - 1));
  }
  if (p > q) { const int t = p; p = q; q = t; }
  if (q >= m) return;   // paired with the padding index (uniform over the CTA)
  double *bp = B + (int64_t)p * m, *bq = B + (int64_t)q * m;
  double *jp = Jt + (int64_t)p * m, *jq = Jt + (int64_t)q * m;
  // every load of the two rows (and of the two rows of Jt) issued before it is used
  double x[kJE], y[kJE], u[kJE], v[kJE];
#pragma unroll
  for (int e = 0; e < kJE; ++e) {
    const int k = tid + e * kJT;
    const bool in = k < m;
    x[e] = in ? bp[k] : 0.0;
    y[e] = in ? bq[k] : 0.0;
    u[e] = in ? jp[k] : 0.0;
    v[e] = in ? jq[k] : 0.0;
  }
  double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
  for (int e = 0; e < kJE; ++e) {
    al += x[e] * x[e];
    be += y[e] * y[e];
    ga += x[e] * y[e];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
  }
  if (lane == 0) { red[0][warp] = al; red[1][warp] = be; red[2][warp] = ga; }
  __syncthreads();
  // the rotation from one thread (float64 division and square root are long sequences on
  // the float64 pipe), broadcast through shared memory
  __shared__ double cs[2];
  __shared__ int skip;
  if (tid == 0) {
    al = be = ga = 0.0;
#pragma unroll
    for (int w = 0; w < kJT / 32; ++w) { al += red[0][w]; be += red[1][w]; ga += red[2][w]; }
    skip = (al <= 1e-300 || be <= 1e-300 || ga * ga <= 1e-28 * al * be) ? 1 : 0;
    if (!skip) {
      // largest gamma^2 / (alpha beta) of the pass (non-negative floats order as their bits)
      atomicMax(maxr2, __float_as_uint((float)(ga * ga * rcp_nr(al * be))));
      // t = sign(d) g / (|d| + sqrt(d^2 + g^2)) with d = beta - alpha, g = 2 gamma (the smaller
      // root of t^2 + 2 zeta t - 1 = 0, zeta = d / g), formed on (d, g) scaled to max 1
      const double d0 = be - al, g0 = 2.0 * ga;
      const double sc = rcp_nr(fmax(fabs(d0), fabs(g0)));
      const double d = d0 * sc, g = g0 * sc, q2 = d * d + g * g;   // q2 in [1, 2]
      const double rt = q2 * rsqrt_nr(q2);
      const double t = (d >= 0.0 ? g : -g) * rcp_nr(fabs(d) + rt);
      const double c0 = rsqrt_nr(1.0 + t * t);
      cs[0] = c0;
      cs[1] = c0 * t;
    }
  }
  __syncthreads();
  if (skip) return;   // uniform
  const double c = cs[0], s = cs[1];
#pragma unroll
  for (int e = 0; e < kJE; ++e) {
    const int k = tid + e * kJT;
    if (k < m) {
      bp[k] = c * x[e] - s * y[e];
      bq[k] = s * x[e] + c * y[e];
      jp[k] = c * u[e] - s * v[e];
      jq[k] = s * u[e] + c * v[e];
    }
  }
}

// Rv = diag(1, V) (Nv x Nv; V[i][k] = Vt[k][i], the rows of Vt the eigenvectors), Rvt = Rv^T,
// W3 = diag(I_No, Rv) (N x N)
__global__ void k_build_rv(const double *Vt, int No, int Nv, double *Rv, double *Rvt, double *W3) {
  const int N = No + Nv, m = Nv - 1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)N * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / N), q = (int)(e % N);
    double v = p == q ? 1.0 : 0.0;
    if (p > No && q > No) v = Vt[(int64_t)(q - No - 1) * m + (p - No - 1)];   // column q of R~: eigenvector q
    else if (p >= No && q >= No && p != q) v = 0.0;
    W3[e] = p < No || q < No ? (p == q ? 1.0 : 0.0) : v;
    if (p >= No && q >= No) {
      Rv[(int64_t)(p - No) * Nv + (q - No)] = v;
      Rvt[(int64_t)(q - No) * Nv + (p - No)] = v;
    }
  }
}

// the virtual block of F made exactly arrow shaped: elements (c, d), c != d, both >= 1 (of the
// order of the Jacobi tolerance) set to zero, and the t' row and column made symmetric
__global__ void k_clean_arrow(double *F, int No, int Nv) {
  const int N = No + Nv;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)Nv * Nv;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / Nv), d = (int)(e % Nv);
    if (c != d && c >= 1 && d >= 1) F[(int64_t)(No + c) * N + No + d] = 0.0;
    if (c == 0 && d > 0) {
      const double v = 0.5 * (F[(int64_t)No * N + No + d] + F[(int64_t)(No + d) * N + No]);
      F[(int64_t)No * N + No + d] = v;
      F[(int64_t)(No + d) * N + No] = v;
    }
  }
}

// out[s] = in[s]^T for S slices of Nv x Nv (32 x 32 tiles through shared memory)
__global__ void __launch_bounds__(256) k_tr64(const double *in, double *out, int64_t S, int Nv) {
  __shared__ double t[32][33];
  const int nt = (Nv + 31) / 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t items = S * nt * nt, NvNv = (int64_t)Nv * Nv;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t s = it / (nt * nt);
    const int tt = (int)(it % (nt * nt)), ta = tt / nt, tb = tt % nt;
    const double *src = in + s * NvNv;
    double *dst = out + s * NvNv;
    for (int r = ty; r < 32; r += 8) {
      const int a = ta * 32 + r, b = tb * 32 + tx;
      t[r][tx] = (a < Nv && b < Nv) ? src[(int64_t)a * Nv + b] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int b = tb * 32 + r, a = ta * 32 + tx;
      if (a < Nv && b < Nv) dst[(int64_t)b * Nv + a] = t[tx][r];
    }
    __syncthreads();
  }
}

// float64 virtual-index terms in the reduced-cost basis, every slice s of the block vector:
// rho[s][a] = sum_c x_s[a][c] F_t'c (warp per row), kap[s][b] = sum_c F_t'c x_s[c][b] (thread per
// column), then y = X F + F X element-wise.
__global__ void k_rowsum64(const double *x, const double *F, int No, int Nv, int64_t rows, double *rho) {
  const int N = No + Nv, lane = threadIdx.x & 31;
  const double *f = F + (int64_t)No * N + No;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < rows;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const double *xr = x + r * Nv;
    double s = 0.0;
    for (int c = lane; c < Nv; c += 32) s += xr[c] * f[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rho[r] = s;
  }
}
__global__ void k_colsum64(const double *x, const double *F, int No, int Nv, int64_t S, double *kap) {
  const int N = No + Nv;
  const double *f = F + (int64_t)No * N + No;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < S * Nv; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e / Nv;
    const int b = (int)(e % Nv);
    const double *xs = x + s * Nv * Nv + b;
    double acc = 0.0;
#pragma unroll 4
    for (int c = 0; c < Nv; ++c) acc += f[c] * xs[(int64_t)c * Nv];
    kap[e] = acc;
  }
}
__global__ void k_varrow64(const double *x, const double *F, const double *rho, const double *kap, int No, int Nv,
                           int64_t n, double *y) {
  const int N = No + Nv;
  const int64_t NvNv = (int64_t)Nv * Nv;
  const double *f = F + (int64_t)No * N + No;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e / NvNv;
    const int ab = (int)(e % NvNv), a = ab / Nv, b = ab % Nv;
    const double *xs = x + s * NvNv;
    const double xab = xs[ab];
    double v;
    if (b >= 1) v = F[(int64_t)(No + b) * N + No + b] * xab + xs[(int64_t)a * Nv] * f[b];
    else v = rho[s * Nv + a];
    if (a >= 1) v += F[(int64_t)(No + a) * N + No + a] * xab + f[a] * xs[b];
    else v += kap[s * Nv + b];
    y[e] = v;
  }
}

}  // namespace

// The virtual rotation R~ = diag(1, V) (V: eigenvectors of F_vv without t') and F in the
// rotated basis (Farr, float copy F32arr); no vector is rotated here.  exact = false stops the
// Jacobi sweeps once every pair is orthogonal to 1e-2 (enough for a preconditioner); exact =
// true continues from there to the rounding level (the reduced-cost basis needs F_vv exactly
// arrow shaped).  The Jacobi state stays on the handle between the two.
esmp2_status ensure_vrot(esmp2_handle *h, bool exact) {
  const int want = exact ? 2 : 1;
  if (h->vrot_level >= want) return ESMP2_OK;
  esmp2_status s = ensure_mixed(h, true);
  if (s) return s;
  const int No = h->d.No, Nv = h->d.Nv, N = h->d.N, m = Nv - 1;
  if (Nv > 1024) {
    h->err = "the virtual rotation supports Nv <= 1024";
    return ESMP2_ERR_UNSUPPORTED;
  }
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(p, bytes ? bytes : 16, st);
  };
  const size_t mm = (size_t)std::max(1, m * m);
  if (!h->Rv) {
    A(reinterpret_cast<void **>(&h->Rv), sizeof(double) * (size_t)Nv * Nv);
    A(reinterpret_cast<void **>(&h->Rvt), sizeof(double) * (size_t)Nv * Nv);
    A(reinterpret_cast<void **>(&h->Farr), sizeof(double) * (size_t)N * N);
    A(reinterpret_cast<void **>(&h->F32arr), sizeof(float) * (size_t)N * N);
    A(reinterpret_cast<void **>(&h->jB), sizeof(double) * mm);
    A(reinterpret_cast<void **>(&h->jJ), sizeof(double) * mm);
    A(reinterpret_cast<void **>(&h->jflag), sizeof(unsigned) * 4);
    if (e != cudaSuccess) return check_cuda(h, e, "virtual rotation buffers");
    if (m >= 1) {
      k_vblock<<<256, 256, 0, st>>>(h->Fsemi, N, No, m, h->jB, h->jJ);
      h->launches += 1;
    }
  }
  double *W3 = nullptr, *T1 = nullptr;
  A(reinterpret_cast<void **>(&W3), sizeof(double) * (size_t)N * N);
  A(reinterpret_cast<void **>(&T1), sizeof(double) * (size_t)N * N);
  auto release = [&]() { dfree(W3, st); dfree(T1, st); };
  if (e != cudaSuccess) {
    release();
    return check_cuda(h, e, "virtual rotation buffers");
  }
  // eigenvectors of F_vv without t' (one-sided Jacobi on the rows of B = A, Jt = I)
  if (m >= 1) {
    const int n2 = (m + (m & 1)) / 2, rounds = m + (m & 1) - 1;
    const unsigned grid = (unsigned)n2;
    unsigned *mr = h->jflag;
    double *B = h->jB, *J = h->jJ;
    // one sweep as one CUDA graph (a reset of the sweep maximum, then the rounds as dependent
    // kernel nodes), replayed until the sweep's largest gamma^2 / (alpha beta) is below the target
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    if (cudaGraphCreate(&graph, 0) == cudaSuccess) {
      cudaGraphNode_t prev_node = nullptr;
      cudaMemsetParams mp{};
      mp.dst = mr;
      mp.value = 0;
      mp.elementSize = 4;
      mp.width = 1;
      mp.height = 1;
      bool ok = cudaGraphAddMemsetNode(&prev_node, graph, nullptr, 0, &mp) == cudaSuccess;
      for (int k = 0; k < rounds && ok; ++k) {
        int rr = k % rounds, mm_ = m;
        void *args[] = {&B, &J, &mm_, &rr, &mr};
        cudaKernelNodeParams kp{};
        kp.func = reinterpret_cast<void *>(k_jacobi_os_round);
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(kJT);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        cudaGraphNode_t node = nullptr;
        ok = cudaGraphAddKernelNode(&node, graph, &prev_node, 1, &kp) == cudaSuccess;
        prev_node = node;
      }
      if (!ok || cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) gexec = nullptr;
      cudaGraphDestroy(graph);
      cudaGetLastError();
    }
    // a sweep whose rotations were all below the target: 1e-14 (none rotated) for the exact
    // basis; for the preconditioner every pair of rows orthogonal to 1e-2 (the inner iteration
    // count at No=30 Nv=400 is the same as with 1e-6, and the sweeps fall from 9 to 8)
    const float target = exact ? 0.f : 1e-4f;
    bool done = false;
    int sweeps = 0;
    for (int sweep = 0; sweep < 60 && !done; ++sweep) {
      if (gexec) {
        if ((e = cudaGraphLaunch(gexec, st)) != cudaSuccess) break;
      } else {
        cudaMemsetAsync(mr, 0, sizeof(unsigned), st);
        for (int k = 0; k < rounds; ++k) k_jacobi_os_round<<<grid, kJT, 0, st>>>(B, J, m, k, mr);
      }
      h->launches += rounds;
      ++sweeps;
      unsigned hr = 0;
      e = cudaMemcpyAsync(&hr, mr, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) break;
      float r2;
      std::memcpy(&r2, &hr, sizeof(r2));
      done = r2 <= target;
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (e != cudaSuccess) {
      release();
      return check_cuda(h, e, "virtual rotation (Jacobi)");
    }
    if (std::getenv("ESMP2_DEBUG")) std::fprintf(stderr, "esmp2 jacobi: %d sweeps of %d rounds\n", sweeps, rounds);
    debug_phase(h, exact ? "  virtual rotation: Jacobi to the rounding level" : "  virtual rotation: Jacobi to 1e-2");
  }
  k_build_rv<<<256, 256, 0, st>>>(h->jJ, No, Nv, h->Rv, h->Rvt, W3);
  // Farr = W3^T Fsemi W3
  Gemm64 g{};
  g.alpha = 1.0; g.beta = 0.0; g.batch = 1; g.M = N; g.N = N; g.K = N;
  g.A = h->Fsemi; g.sAm = N; g.sAk = 1; g.B = W3; g.sBk = N; g.sBn = 1; g.C = T1; g.sCm = N; g.sCn = 1;
  gemm64(g, st);
  g.A = W3; g.sAm = 1; g.sAk = N; g.B = T1; g.sBk = N; g.sBn = 1; g.C = h->Farr; g.sCm = N; g.sCn = 1;
  gemm64(g, st);
  k_clean_arrow<<<256, 256, 0, st>>>(h->Farr, No, Nv);
  k_to_f32<<<64, 256, 0, st>>>(h->Farr, h->F32arr, (int64_t)N * N);
  h->launches += 5;
  // digit planes of an earlier (less converged) rotation are stale
  dfree(h->Rvdig, st);
  dfree(h->Rvtdig, st);
  h->Rvdig = h->Rvtdig = nullptr;
  release();
  h->vrot_level = want;
  return check_cuda(h, cudaGetLastError(), "virtual rotation");
}

esmp2_status ensure_arrow(esmp2_handle *h) {
  if (h->arrow_ready) return ESMP2_OK;
  esmp2_status s = ensure_vrot(h, true);
  if (s) return s;
  const int No = h->d.No, Nv = h->d.Nv;
  const size_t n = (size_t)h->d.n, S = (size_t)5 * No * No;
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(p, bytes ? bytes : 16, st);
  };
  A(reinterpret_cast<void **>(&h->barr), sizeof(double) * n);
  A(reinterpret_cast<void **>(&h->rho64), sizeof(double) * S * Nv);
  A(reinterpret_cast<void **>(&h->kap64), sizeof(double) * S * Nv);
  if (e != cudaSuccess) return check_cuda(h, e, "reduced-cost basis buffers");
  // the right-hand side in the reduced-cost basis (float64-exact digit-split rotations)
  s = rotate_virt(h, h->bsemi, h->barr, h->s64.w ? h->s64.w : h->s64.p, true);
  if (s) return s;
  debug_phase(h, "  reduced basis: rhs rotation");
  h->arrow_ready = true;
  return check_cuda(h, cudaGetLastError(), "reduced-cost basis");
}

// out = R~^T X R~ (to_arrow) or R~ X R~^T for every slice X of a full-storage block vector:
// X R (digit-split product), transpose, X R again, transpose.  in may equal out; tmp: n doubles.
esmp2_status rotate_virt(esmp2_handle *h, const double *in, double *out, double *tmp, bool to_arrow) {
  const int No = h->d.No, Nv = h->d.Nv;
  const int64_t S = 5LL * No * No, rows = S * Nv;
  const double *M = to_arrow ? h->Rv : h->Rvt;
  void **dig = to_arrow ? &h->Rvdig : &h->Rvtdig;
  int *eM = to_arrow ? &h->eRv : &h->eRvt;
  const int slot = to_arrow ? 2 : 3;
  const unsigned gt = (unsigned)std::min<int64_t>(S * ((Nv + 31) / 32) * ((Nv + 31) / 32), 4864);
  esmp2_status s = xwm_split(h, in, rows, tmp, M, dig, eM, slot);
  if (s) return s;
  k_tr64<<<gt, 256, 0, h->stream>>>(tmp, out, S, Nv);
  if ((s = xwm_split(h, out, rows, tmp, M, dig, eM, slot))) return s;
  k_tr64<<<gt, 256, 0, h->stream>>>(tmp, out, S, Nv);
  h->launches += 2;
  if ((s = check_device_flag(h))) return s;
  return check_cuda(h, cudaGetLastError(), "rotate_virt");
}

// Move the stored solution to `target` (0 TOP, 1 semicanonical-occupied, 2 reduced-cost basis).
esmp2_status x_to_basis(esmp2_handle *h, int target) {
  if (h->x_basis == target) return ESMP2_OK;
  if (h->x_zero) {   // zero in every basis
    h->x_basis = target;
    return ESMP2_OK;
  }
  double *x = h->s64.x, *tmp = h->s64.w ? h->s64.w : h->s64.p;
  esmp2_status s = ESMP2_OK;
  h->r_true = false;
  if (h->x_basis == 2) {
    if ((s = rotate_virt(h, x, x, tmp, false))) return s;
    h->x_basis = 1;
  }
  if (target == 0 && h->x_basis == 1) {
    rotate_occ(h, x, x, tmp, false);
    h->x_basis = 0;
  }
  if (target >= 1 && h->x_basis == 0) {
    if ((s = ensure_mixed(h, true))) return s;
    rotate_occ(h, x, x, tmp, true);
    h->x_basis = 1;
  }
  if (target == 2 && h->x_basis == 1) {
    if ((s = ensure_arrow(h))) return s;
    if ((s = rotate_virt(h, x, x, tmp, true))) return s;
    h->x_basis = 2;
  }
  return check_cuda(h, cudaGetLastError(), "x_to_basis");
}

void virt_arrow64(esmp2_handle *h, const double *x, double *y) {
  const int No = h->d.No, Nv = h->d.Nv;
  const int64_t S = 5LL * No * No;
  cudaStream_t st = h->stream;
  KScope ks(st, ESMP2_KT_CONTRACTION, alg_virtual_flops(No, Nv), 6.0 * (double)h->d.n);
  k_rowsum64<<<1216, 256, 0, st>>>(x, h->Farr, No, Nv, S * Nv, h->rho64);
  k_colsum64<<<(unsigned)std::min<int64_t>(cdiv(S * Nv, 256), 4864), 256, 0, st>>>(x, h->Farr, No, Nv, S, h->kap64);
  k_varrow64<<<1216, 256, 0, st>>>(x, h->Farr, h->rho64, h->kap64, No, Nv, h->d.n, y);
  h->launches += 3;
}

// float64 sigma in the reduced-cost basis: the virtual-index terms element-wise, the
// occupied-index terms and couplings by the arrow-form coupling pass (Farr).
esmp2_status sigma64_arrow(esmp2_handle *h, const double *x, double *y, int couplings) {
  virt_arrow64(h, x, y);
  if (couplings) {
    launch_intermediates64(h, h->Farr, 1, x);
    launch_couple64(h, h->Farr, 1, x, y);
  }
  return check_cuda(h, cudaGetLastError(), "sigma64_arrow");
}

}  // namespace esmp2

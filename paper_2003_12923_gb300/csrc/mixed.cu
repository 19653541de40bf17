// Mixed-precision sigma (bf16 tcgen05 virtual-index contractions) and its set-up.
//
// The low-precision solve works in the basis whose occupied orbitals other than t
// diagonalise F_oo: D and L are unchanged by any rotation of the occupied orbitals that
// fixes t (all doubles; triples holding the pair t -> t'), so the operator is the same
// linear map, and its occupied-index terms reduce to a diagonal plus the t row/column,
// applied element by element after the tensor-core pass.  E2_S is not affected: it is
// evaluated once in the TOP basis.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include <vector>

#include "internal.h"

namespace esmp2 {

esmp2_status virt_bf16(esmp2_handle *h, const void *xb, const void *Fb, int S, float *y, int *err);
esmp2_status virt_bf16_sym(esmp2_handle *h, const void *xb, const void *Fb, float *y, int *err);
void to_bf16_f64(esmp2_handle *h, const double *src, void *dst, int64_t rows);
void to_bf16_f32(esmp2_handle *h, const float *src, void *dst, int64_t rows);
void fvv_bf16(esmp2_handle *h, const double *F, void *dst);

namespace {

__global__ void k_f64_to_f32(const double *src, float *dst, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (float)src[e];
}

__global__ void k_f32_to_f64(const float *src, double *dst, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (double)src[e];
}

// R = diag(1, V) (No x No) and its transpose; W2 = diag(R, I_Nv) (N x N)
__global__ void k_build_rot(const double *V, int No, int Nv, double *R, double *Rt, double *W2) {
  const int N = No + Nv, m = No - 1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * N; e += gridDim.x * blockDim.x) {
    const int p = e / N, q = e % N;
    double v = 0.0;
    if (p < No && q < No) {
      if (p == 0 || q == 0) v = (p == q) ? 1.0 : 0.0;
      else v = V[(p - 1) * m + (q - 1)];
      R[p * No + q] = v;
      Rt[q * No + p] = v;
    } else if (p == q) {
      v = 1.0;
    }
    W2[e] = v;
  }
}

// out[p][k'][q] = sum_k R[k][k'] in[p][k][q] for K <= 32 in double-float arithmetic: every
// float64 operand is split into two floats (hi + lo); products are formed with the exact
// product error (fma) and summed with Knuth's two-sum, so the float32 pipes do the work at
// about 2^-46 relative accuracy; the float64 result is hi + lo.  The orbital rotations have
// only No multiply-adds per element, which on GB300 would otherwise be float64-bound.
constexpr int kDfK = 32;

__global__ void __launch_bounds__(256) k_mode_df(const double *in, double *out, int64_t P, int K, int64_t Q,
                                                 const double *R) {
  __shared__ float2 R2[kDfK * kDfK];      // (hi, lo) pairs: one 8-byte broadcast load per product
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const double r = R[e];
    const float hi = (float)r;
    R2[e] = make_float2(hi, (float)(r - (double)hi));
  }
  __syncthreads();
  const int64_t n = P * Q;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / Q, q = e % Q;
    const double *src = in + p * K * Q + q;
    double *dst = out + p * K * Q + q;
    float xh[kDfK], xl[kDfK];
#pragma unroll
    for (int k = 0; k < kDfK; ++k) {
      if (k < K) {
        const double v = src[k * Q];
        xh[k] = (float)v;
        xl[k] = (float)(v - (double)xh[k]);
      }
    }
    for (int k2 = 0; k2 < K; k2 += 4) {
      float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < kDfK; ++k) {
        if (k < K) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (k2 + c < K) {   // exact leading product, two-sum; renormalised once at the end
              const float2 r = R2[k * K + k2 + c];
              const float ph = r.x * xh[k];
              const float pe = fmaf(r.x, xh[k], -ph) + fmaf(r.x, xl[k], r.y * xh[k]);
              const float t = sh[c] + ph;
              const float bv = t - sh[c];
              sl[c] += ((sh[c] - (t - bv)) + (ph - bv)) + pe;
              sh[c] = t;
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (k2 + c < K) dst[(k2 + c) * Q] = (double)sh[c] + (double)sl[c];
    }
  }
}

}  // namespace

// out[p][k'][q] = sum_k R[k][k'] in[p][k][q] (R: K x K, row pitch K) in double-float
// arithmetic when K <= 32, else as a float64 GEMM.
void mode_product_small(const double *in, double *out, int64_t P, int K, int64_t Q, const double *R,
                        cudaStream_t st) {
  if (K <= kDfK) {
    k_mode_df<<<1216, 256, 0, st>>>(in, out, P, K, Q, R);
    return;
  }
  Gemm64 g{};
  g.alpha = 1.0; g.beta = 0.0;
  g.M = K; g.N = (int)Q; g.K = K; g.batch = (int)P;
  g.A = R; g.sAm = 1; g.sAk = K; g.sAb = 0;
  g.B = in; g.sBk = Q; g.sBn = 1; g.sBb = (int64_t)K * Q;
  g.C = out; g.sCm = Q; g.sCn = 1; g.sCb = (int64_t)K * Q;
  gemm64(g, st);
}

// in/out: block vectors; new occupied index i' = sum_i R[i][i'] (old i) (to_semi), or back.
void rotate_occ(esmp2_handle *h, const double *in, double *out, double *tmp, bool to_semi) {
  const int No = h->d.No, Nv = h->d.Nv;
  if (No == 1) {
    if (in != out) cudaMemcpyAsync(out, in, sizeof(double) * h->d.n, cudaMemcpyDeviceToDevice, h->stream);
    return;
  }
  const int dims[4] = {5, No, No, Nv * Nv};
  const double *R = to_semi ? h->Rocc : h->Rocct;
  if (No <= kDfK) {
    const int64_t NvNv = (int64_t)Nv * Nv;
    k_mode_df<<<1216, 256, 0, h->stream>>>(in, tmp, 5, No, (int64_t)No * NvNv, R);
    k_mode_df<<<1216, 256, 0, h->stream>>>(tmp, out, 5LL * No, No, NvNv, R);
  } else {
    mode_product(in, tmp, dims, 1, R, No, No, h->stream);
    mode_product(tmp, out, dims, 2, R, No, No, h->stream);
  }
  h->launches += 2;
}

static esmp2_status alloc_mixed_buffers(esmp2_handle *h) {
  if (h->xlp) return ESMP2_OK;
  const int No = h->d.No, Nv = h->d.Nv, Nvp = (Nv + 7) & ~7;
  const size_t n = (size_t)h->d.n;
  cudaError_t e = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(p, bytes ? bytes : 1, h->stream);
  };
  A(&h->xlp, sizeof(__nv_bfloat16) * (size_t)5 * No * No * Nv * Nvp);
  A(&h->Fvlp, sizeof(__nv_bfloat16) * (size_t)Nv * Nvp);
  A(reinterpret_cast<void **>(&h->ylp), sizeof(float) * n);
  if (!h->dflag) A(reinterpret_cast<void **>(&h->dflag), sizeof(int));
  A(reinterpret_cast<void **>(&h->cp.OC1), sizeof(double) * (size_t)5 * No * Nv * Nv);
  A(reinterpret_cast<void **>(&h->cp.OC2), sizeof(double) * (size_t)5 * No * Nv * Nv);
  if (e != cudaSuccess) return check_cuda(h, e, "mixed buffers");
  cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream);
  fvv_bf16(h, h->F, h->Fvlp);  // the virtual block is the same in both bases
  return check_cuda(h, cudaGetLastError(), "mixed buffers");
}

esmp2_status ensure_mixed(esmp2_handle *h, bool semi) {
  esmp2_status s = alloc_mixed_buffers(h);
  if (s || !semi || h->mixed_ready) return s;
  const int No = h->d.No, Nv = h->d.Nv, N = h->d.N, m = No - 1;
  const size_t n = (size_t)h->d.n;
  cudaError_t e = cudaSuccess;
  auto A = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = dmalloc(p, bytes ? bytes : 1, h->stream);
  };
  A(reinterpret_cast<void **>(&h->Rocc), sizeof(double) * No * No);
  A(reinterpret_cast<void **>(&h->Rocct), sizeof(double) * No * No);
  A(reinterpret_cast<void **>(&h->Fsemi), sizeof(double) * (size_t)N * N);
  A(reinterpret_cast<void **>(&h->bsemi), sizeof(double) * n);
  A(reinterpret_cast<void **>(&h->r32), sizeof(float) * n);
  A(reinterpret_cast<void **>(&h->p32), sizeof(float) * n);
  A(reinterpret_cast<void **>(&h->q32), sizeof(float) * n);
  A(reinterpret_cast<void **>(&h->x32), sizeof(float) * n);
  A(reinterpret_cast<void **>(&h->F32), sizeof(float) * (size_t)N * N);
  {
    const size_t ooN = (size_t)No * No * Nv, oNN = (size_t)No * Nv * Nv, oN = (size_t)No * Nv;
    auto &c = h->cp32;
    A(reinterpret_cast<void **>(&c.VX), sizeof(float) * ooN); A(reinterpret_cast<void **>(&c.GP), sizeof(float) * ooN);
    A(reinterpret_cast<void **>(&c.WZ), sizeof(float) * ooN); A(reinterpret_cast<void **>(&c.HP), sizeof(float) * ooN);
    A(reinterpret_cast<void **>(&c.OX), sizeof(float) * oNN); A(reinterpret_cast<void **>(&c.OZ), sizeof(float) * oNN);
    A(reinterpret_cast<void **>(&c.OC1), sizeof(float) * 5 * oNN); A(reinterpret_cast<void **>(&c.OC2), sizeof(float) * 5 * oNN);
    A(reinterpret_cast<void **>(&c.G), sizeof(float) * oN); A(reinterpret_cast<void **>(&c.H), sizeof(float) * oN);
    A(reinterpret_cast<void **>(&c.CYZ), sizeof(float) * oN);
  }
  double *V = nullptr, *work = nullptr, *W2 = nullptr, *T1 = nullptr;
  A(reinterpret_cast<void **>(&V), sizeof(double) * std::max(1, m * m));
  A(reinterpret_cast<void **>(&work), sizeof(double) * (3 * std::max(1, m * m) + std::max(1, m)));
  A(reinterpret_cast<void **>(&W2), sizeof(double) * (size_t)N * N);
  A(reinterpret_cast<void **>(&T1), sizeof(double) * (size_t)N * N);
  if (e != cudaSuccess) {
    dfree(V, h->stream); dfree(work, h->stream); dfree(W2, h->stream); dfree(T1, h->stream);
    return check_cuda(h, e, "mixed set-up");
  }
  debug_phase(h, "  mixed: allocations");
  if (m >= 1) eigvecs_block(h, h->F, 1, m, V, work);
  k_build_rot<<<64, 256, 0, h->stream>>>(V, No, Nv, h->Rocc, h->Rocct, W2);
  Gemm64 g{};
  g.alpha = 1.0; g.beta = 0.0; g.batch = 1; g.M = N; g.N = N; g.K = N;
  g.A = h->F; g.sAm = N; g.sAk = 1; g.B = W2; g.sBk = N; g.sBn = 1; g.C = T1; g.sCm = N; g.sCn = 1;
  gemm64(g, h->stream);
  g.A = W2; g.sAm = 1; g.sAk = N; g.B = T1; g.sBk = N; g.sBn = 1; g.C = h->Fsemi; g.sCm = N; g.sCn = 1;
  gemm64(g, h->stream);
  h->launches += 3;
  debug_phase(h, "  mixed: basis (eigenvectors, F)");
  rotate_occ(h, h->b, h->bsemi, h->s64.w ? h->s64.w : h->s64.p, true);
  debug_phase(h, "  mixed: rhs rotation");
  k_f64_to_f32<<<64, 256, 0, h->stream>>>(h->Fsemi, h->F32, (int64_t)N * N);
  h->launches += 1;
  {  // the t and t' columns of the occupied rows, as the float copy holds them (launch weights)
    std::vector<double> rows((size_t)No * N);
    e = cudaMemcpyAsync(rows.data(), h->Fsemi, sizeof(double) * rows.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      dfree(V, h->stream); dfree(work, h->stream); dfree(W2, h->stream); dfree(T1, h->stream);
      return check_cuda(h, e, "mixed set-up");
    }
    for (int l = 0; l < 32; ++l) {
      h->arrow_w[l] = (l >= 1 && l < No) ? (float)rows[(size_t)l * N] : 0.f;
      h->arrow_w[32 + l] = l < No ? (float)rows[(size_t)l * N + No] : 0.f;
    }
    h->arrow_w_ready = true;
  }
  dfree(V, h->stream); dfree(work, h->stream); dfree(W2, h->stream); dfree(T1, h->stream);
  h->mixed_ready = true;
  return check_cuda(h, cudaGetLastError(), "mixed set-up");
}

esmp2_status check_device_flag(esmp2_handle *h) {
  int f = 0;
  cudaMemcpyAsync(&f, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return check_cuda(h, e, "device flag");
  if (f) {
    h->err = "a bounded device-side wait timed out in the tensor-core kernel";
    cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream);
    return ESMP2_ERR_TIMEOUT;
  }
  return ESMP2_OK;
}

// Inner (low-precision) sigma in the semicanonical-occupied basis: q = A p with the
// virtual-index terms from bf16 operands on tcgen05 and everything else in float32.
// p_bf16_ready: the PCG update already wrote bf16(p) into the operand buffer.  The T, X, Y
// slices j > i are filled from i < j (antisymmetry), so p is taken as antisymmetric.
// dot: optional per-CTA partials of the weighted <p, q> (couple_dot_parts(h) doubles).
esmp2_status sigma_inner(esmp2_handle *h, const float *p, float *q, bool p_bf16_ready, double *dot) {
  const int No = h->d.No, Nv = h->d.Nv;
  const int64_t rows = (int64_t)5 * No * No * Nv;
  if (!p_bf16_ready) to_bf16_f32(h, p, h->xlp, rows);
  esmp2_status s = virt_bf16_sym(h, h->xlp, h->Fvlp, q, h->dflag);
  if (s) return s;
  couple32(h, h->F32, p, q, dot);
  return check_cuda(h, cudaGetLastError(), "sigma_inner");
}

// API-level mixed sigma in the TOP basis: virtual-index terms in bf16 on tcgen05, the
// occupied-index and coupling terms in float64.
esmp2_status sigma_mixed(esmp2_handle *h, const double *x, double *y) {
  esmp2_status s = ESMP2_OK;
  if (h->d.No <= 32) {  // the inner solve's packed path (singlet vectors), checked through the same call
    if ((s = ensure_mixed(h, true)) || (h->arrowv && (s = ensure_arrow(h))) || (s = packed_setup(h)) ||
        (s = sigma_mixed_packed(h, x, y)))
      return s;
    return check_device_flag(h);
  }
  if ((s = ensure_mixed(h, false))) return s;
  const int No = h->d.No, Nv = h->d.Nv;
  to_bf16_f64(h, x, h->xlp, (int64_t)5 * No * No * Nv);
  if ((s = virt_bf16(h, h->xlp, h->Fvlp, 5 * No * No, h->ylp, h->dflag))) return s;
  k_f32_to_f64<<<1216, 256, 0, h->stream>>>(h->ylp, y, h->d.n);
  h->launches += 1;
  contractions64(h, h->F, x, y, 2);
  return sigma64_tail(h, h->F, 0, x, y);
}

// Only the virtual-index contractions (both terms, all blocks), for testing the tensor-core
// kernel against the float64 GEMMs.
// mode 0: float64 GEMMs; 1: bf16 operands, fp32 accumulation; 2: exact digit products
// summed in float64 (every slice, both terms, any input).
esmp2_status virtual_contraction(esmp2_handle *h, const double *x, double *y, int mode) {
  if (mode == 0) {
    contractions64(h, h->F, x, y, 1);
    return check_cuda(h, cudaGetLastError(), "virtual contraction");
  }
  if (mode == 2) {
    esmp2_status s = virt_split(h, x, y, nullptr, 0, kFp64TcLevels);
    if (!s) s = check_device_flag(h);
    return s ? s : check_cuda(h, cudaGetLastError(), "virtual contraction");
  }
  esmp2_status s = ensure_mixed(h, false);
  if (s) return s;
  const int No = h->d.No, Nv = h->d.Nv;
  to_bf16_f64(h, x, h->xlp, (int64_t)5 * No * No * Nv);
  if ((s = virt_bf16(h, h->xlp, h->Fvlp, 5 * No * No, h->ylp, h->dflag))) return s;
  k_f32_to_f64<<<1216, 256, 0, h->stream>>>(h->ylp, y, h->d.n);
  h->launches += 1;
  if ((s = check_device_flag(h))) return s;
  return check_cuda(h, cudaGetLastError(), "virtual contraction");
}

// Per-stage timing of the inner sigma (fp32 vectors) on the handle's stream.
esmp2_status profile_mixed(esmp2_handle *h, const double *x, double *y, int reps, double *ms) {
  esmp2_status s = ensure_mixed(h, true);
  if (s) return s;
  if (h->d.No <= 32) {
    if ((h->arrowv && (s = ensure_arrow(h))) || (s = packed_setup(h)) || (s = profile_packed(h, x, reps, ms))) return s;
    return check_device_flag(h);
  }
  const int No = h->d.No, Nv = h->d.Nv;
  const int64_t rows = (int64_t)5 * No * No * Nv;
  // fp32 copy of x into the inner buffers (the basis is irrelevant for timing)
  k_f64_to_f32<<<1216, 256, 0, h->stream>>>(x, h->p32, h->d.n);
  h->launches += 1;
  (void)y;
  cudaEvent_t ev[4];
  for (auto &e : ev) cudaEventCreate(&e);
  double acc[4] = {0, 0, 0, 0};
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(ev[0], h->stream);
    to_bf16_f32(h, h->p32, h->xlp, rows);
    cudaEventRecord(ev[1], h->stream);
    if ((s = virt_bf16_sym(h, h->xlp, h->Fvlp, h->q32, h->dflag))) return s;
    cudaEventRecord(ev[2], h->stream);
    couple32(h, h->F32, h->p32, h->q32);
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
  ms[0] = acc[0] / reps;
  ms[1] = acc[1] / reps;
  ms[2] = 0.0;
  ms[3] = acc[2] / reps;
  ms[4] = acc[3] / reps;
  for (auto &e : ev) cudaEventDestroy(e);
  if ((s = check_device_flag(h))) return s;
  return check_cuda(h, cudaGetLastError(), "profile_mixed");
}

}  // namespace esmp2

// C ABI entry points of the ESMP2 library (declared in include/esmp2.h).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

namespace esmp2 {
esmp2_status setup_rhs_from(esmp2_handle *h, const double *ovov_src, double *ovov_in, double *ooov_in,
                            const double *ovvv_src, double *ovvv_in, double *scratch);
}

using namespace esmp2;

namespace {

template <typename T>
cudaError_t dalloc(T **p, size_t count, cudaStream_t st) {
  return dmalloc(reinterpret_cast<void **>(p), sizeof(T) * (count ? count : 1), st);
}

bool finite_host(const double *p, size_t n) {
  for (size_t k = 0; k < n; ++k)
    if (!std::isfinite(p[k])) return false;
  return true;
}

void free_handle(esmp2_handle *h) {
  void *ptrs[] = {h->C, h->U, h->lam, h->Wv, h->W, h->F, h->f0vo, h->scal, h->ovov, h->ooov, h->ovvt, h->b,
                  h->s64.x, h->s64.r, h->s64.p, h->s64.q, h->s64.w, h->cp.VX, h->cp.OX, h->cp.WZ, h->cp.OZ,
                  h->cp.G, h->cp.H, h->cp.CYZ, h->cp.GP, h->cp.HP, h->P64, h->F32, h->dinv32, h->cp32.VX, h->cp32.GP, h->cp32.WZ, h->cp32.HP,
                  h->cp32.OX, h->cp32.OZ, h->cp32.OC1, h->cp32.OC2, h->cp32.G, h->cp32.H, h->cp32.CYZ, h->red, h->red_out, h->xlp, h->Fvlp, h->ylp, h->r32, h->p32,
                  h->q32, h->x32, h->dflag, h->Rocc, h->Rocct, h->Fsemi, h->bsemi, h->cp.OC1, h->cp.OC2,
                  h->xdig, h->Fdig, h->es, h->slist, h->Rdig, h->pr, h->pp, h->pq, h->pd, h->pdinv, h->pop, h->pW, h->pop32, h->pW32, h->pRbf, h->pT1, h->pZ, h->pWR, h->pWRt, h->pLam, h->pOcc, h->pCode, h->pdot2, h->zero_slots, h->Rv, h->Rvt, h->Rvdig, h->Rvtdig, h->Farr, h->barr, h->F32arr, h->rho64, h->kap64, h->pRho, h->pKap, h->jB, h->jJ, h->jflag, h->mr_a, h->mr_b, h->mr_v,
                  h->pP, h->pVX, h->pGP, h->pWZ, h->pHP, h->pOC, h->pOC2, h->pOX, h->pOZ, h->pG, h->pH, h->pCYZ, h->pdot};
  for (void *p : ptrs)
    if (p) dfree(p, h->stream);
  cudaStreamSynchronize(h->stream);
  if (h->inner_graph) cudaGraphExecDestroy(h->inner_graph);
  if (h->hred) cudaFreeHost(h->hred);
}

}  // namespace

namespace esmp2 {
// esmp2_create on a given stream (the batch driver gives each worker its own stream).
esmp2_status create_impl(esmp2_handle **out, const esmp2_desc *d, cudaStream_t stream);
}

extern "C" {

const char *esmp2_last_error(const esmp2_handle *h) { return h ? h->err.c_str() : "null handle"; }

int64_t esmp2_kernel_launches(const esmp2_handle *h) { return h ? h->launches : 0; }

esmp2_status esmp2_create(esmp2_handle **out, const esmp2_desc *d) { return create_impl(out, d, nullptr); }

}  // extern "C"

esmp2_status esmp2::create_impl(esmp2_handle **out, const esmp2_desc *d, cudaStream_t stream) {
  if (!out || !d) return ESMP2_ERR_INVALID_ARG;
  *out = nullptr;
  esmp2_handle *h = new (std::nothrow) esmp2_handle();
  if (!h) return ESMP2_ERR_OOM;
  *out = h;
  h->stream = stream;
  debug_phase(h, "create: begin");
  const int No = d->No, Nv = d->Nv;
  if (No < 1 || No > 64 || Nv < No || Nv > 4096) {
    h->err = "require 1 <= No <= 64 and No <= Nv <= 4096";
    return No >= 1 && Nv >= 1 && Nv < No ? ESMP2_ERR_UNSUPPORTED : ESMP2_ERR_INVALID_ARG;
  }
  if (d->spin != 1) { h->err = "only singlet states (spin = +1) are supported"; return ESMP2_ERR_UNSUPPORTED; }
  if (!d->F || !d->ovov || !d->ooov || !d->ovvv || !d->C) { h->err = "NULL input array"; return ESMP2_ERR_INVALID_ARG; }
  if (d->avo_convention != 0) { h->err = "only the Householder completion of the virtual space (avo_convention 0)"; return ESMP2_ERR_UNSUPPORTED; }
  if (d->n_large > 1) { h->err = "TOP(k) with k > 1 large pairs is not supported (TOP(1) only)"; return ESMP2_ERR_UNSUPPORTED; }
  if (d->n_large < 0 || !std::isfinite(d->eta) || !std::isfinite(d->level_shift)) {
    h->err = "n_large < 0 or non-finite eta / level_shift";
    return ESMP2_ERR_INVALID_ARG;
  }
  h->level_shift = d->level_shift;
  h->eta = d->eta;
  h->n_large = d->n_large;
  const int N = No + Nv;
  h->d.No = No; h->d.Nv = Nv; h->d.N = N;
  h->d.B = (int64_t)No * No * Nv * Nv;
  h->d.n = 5 * h->d.B;
  const size_t nF = (size_t)N * N, nC = (size_t)No * Nv;
  const size_t nOVOV = (size_t)h->d.B, nOOOV = (size_t)No * No * No * Nv, nOVVV = (size_t)No * Nv * Nv * Nv;
  const size_t nOVVT = (size_t)No * Nv * Nv * No;
  if (!d->inputs_on_device) {
    if (!finite_host(d->F, nF) || !finite_host(d->C, nC)) { h->err = "non-finite F or C"; return ESMP2_ERR_INVALID_ARG; }
    for (int p = 0; p < N; ++p)
      for (int q = 0; q < p; ++q)
        if (std::fabs(d->F[(size_t)p * N + q] - d->F[(size_t)q * N + p]) > 1e-12 * (1.0 + std::fabs(d->F[(size_t)p * N + q]))) {
          h->err = "F is not symmetric";
          return ESMP2_ERR_INVALID_ARG;
        }
  }
  cudaError_t ce = cudaSuccess;
#define ALLOC(ptr, cnt) if ((ce = dalloc(&(ptr), (cnt), h->stream)) != cudaSuccess) { esmp2_status s = check_cuda(h, ce, "alloc " #ptr); return s; }
  ALLOC(h->C, nC); ALLOC(h->U, (size_t)No * No); ALLOC(h->lam, (size_t)No); ALLOC(h->Wv, (size_t)Nv * Nv);
  ALLOC(h->W, nF); ALLOC(h->F, nF); ALLOC(h->f0vo, nC); ALLOC(h->scal, (size_t)8);
  ALLOC(h->ovov, nOVOV); ALLOC(h->ooov, nOOOV); ALLOC(h->ovvt, nOVVT);
  ALLOC(h->b, (size_t)h->d.n);
  ALLOC(h->s64.x, (size_t)h->d.n); ALLOC(h->s64.r, (size_t)h->d.n); ALLOC(h->s64.p, (size_t)h->d.n);
  ALLOC(h->s64.q, (size_t)h->d.n);
  ALLOC(h->cp.VX, (size_t)No * No * Nv); ALLOC(h->cp.OX, (size_t)No * Nv * Nv); ALLOC(h->cp.WZ, (size_t)No * No * Nv);
  ALLOC(h->cp.OZ, (size_t)No * Nv * Nv); ALLOC(h->cp.G, nC);
  ALLOC(h->cp.GP, (size_t)No * No * Nv); ALLOC(h->cp.HP, (size_t)No * No * Nv); ALLOC(h->cp.H, nC); ALLOC(h->cp.CYZ, nC);
  {
    const size_t nred = std::max<size_t>(std::max<size_t>((size_t)16 * 1216, (size_t)No * No * No),
                                         (size_t)couple_dot_parts(h));
    ALLOC(h->red, nred);
  }
  ALLOC(h->red_out, (size_t)32);
  if ((ce = cudaMallocHost(reinterpret_cast<void **>(&h->hred), sizeof(double) * 32)) != cudaSuccess)
    return check_cuda(h, ce, "pinned alloc");
  debug_phase(h, "create: allocations");
  // inputs -> device; device-resident OVOV and OVVV are read in place by the first pass of
  // their transforms (no staging copy), host inputs are staged in the work buffers
  const bool dev = d->inputs_on_device != 0;
  const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  double *ovov_in = nullptr, *ooov_in = nullptr, *ovvv_in = nullptr, *scratch = nullptr;
  const size_t nscr = std::max(nOVOV, std::max(nOOOV, nOVVT));
  if ((ce = dalloc(&ovov_in, nOVOV, h->stream)) != cudaSuccess || (ce = dalloc(&ooov_in, nOOOV, h->stream)) != cudaSuccess ||
      (ce = dalloc(&ovvv_in, dev ? nOVVT : std::max(nOVVV, nOVVT), h->stream)) != cudaSuccess ||
      (ce = dalloc(&scratch, nscr, h->stream)) != cudaSuccess) {
    dfree(ovov_in, h->stream); dfree(ooov_in, h->stream); dfree(ovvv_in, h->stream); dfree(scratch, h->stream);
    return check_cuda(h, ce, "input staging");
  }
  cudaMemcpyAsync(h->F, d->F, sizeof(double) * nF, kind, h->stream);
  cudaMemcpyAsync(h->C, d->C, sizeof(double) * nC, kind, h->stream);
  cudaMemcpyAsync(ooov_in, d->ooov, sizeof(double) * nOOOV, kind, h->stream);
  cudaStream_t side = nullptr;
  cudaEvent_t ev_alloc = nullptr;
  if (!dev) {
    cudaMemcpyAsync(ovov_in, d->ovov, sizeof(double) * nOVOV, kind, h->stream);
    // the OVVV block, the largest input, comes in on a side stream while the TOP basis and the
    // OVOV and OOOV transforms run; the handle's stream waits for it before the OVVV pass
    bool side_ok = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) == cudaSuccess &&
                   cudaEventCreateWithFlags(&ev_alloc, cudaEventDisableTiming) == cudaSuccess &&
                   cudaEventCreateWithFlags(&h->ovvv_ready, cudaEventDisableTiming) == cudaSuccess;
    if (side_ok) {
      cudaEventRecord(ev_alloc, h->stream);   // the staging buffer is allocated in this stream's order
      cudaStreamWaitEvent(side, ev_alloc, 0);
      cudaMemcpyAsync(ovvv_in, d->ovvv, sizeof(double) * nOVVV, kind, side);
      cudaEventRecord(h->ovvv_ready, side);
    } else {
      cudaGetLastError();
      if (h->ovvv_ready) cudaEventDestroy(h->ovvv_ready);
      h->ovvv_ready = nullptr;
      cudaMemcpyAsync(ovvv_in, d->ovvv, sizeof(double) * nOVVV, kind, h->stream);
    }
  }
  const double *ovov_src = dev ? d->ovov : ovov_in, *ovvv_src = dev ? d->ovvv : ovvv_in;
  ce = cudaGetLastError();
  esmp2_status s = check_cuda(h, ce, "input copy");
  debug_phase(h, "create: input copies");
  if (!s) s = setup_top_basis(h);
  if (!s && h->n_large == 0 && h->eta > 0.0) {  // eta selects the large pairs: exactly one (TOP(1))
    std::vector<double> lam(No);
    s = check_cuda(h, cudaMemcpyAsync(lam.data(), h->lam, sizeof(double) * No, cudaMemcpyDeviceToHost, h->stream), "lambda");
    if (!s) s = check_cuda(h, cudaStreamSynchronize(h->stream), "lambda");
    int nl = 0;
    for (int u = 0; u < No; ++u) nl += lam[u] > h->eta;
    if (!s && nl == 0) { h->err = "eta exceeds every singular value: no large pair"; s = ESMP2_ERR_INVALID_ARG; }
    if (!s && nl > 1) { h->err = "eta selects more than one large pair (TOP(k), k > 1, is not supported)"; s = ESMP2_ERR_UNSUPPORTED; }
  }
  h->omega_op = h->omega - h->level_shift;
  debug_phase(h, "create: TOP basis");
  if (!s) s = setup_rhs_from(h, ovov_src, ovov_in, ooov_in, ovvv_src, ovvv_in, scratch);
  if (h->ovvv_ready) {   // whatever happened above, the handle's stream is ordered after the copy
    cudaStreamWaitEvent(h->stream, h->ovvv_ready, 0);
    cudaEventDestroy(h->ovvv_ready);
    h->ovvv_ready = nullptr;
  }
  if (side) cudaStreamDestroy(side);
  if (ev_alloc) cudaEventDestroy(ev_alloc);
  debug_phase(h, "create: transforms + rhs");
  if (!s) {
    cudaMemsetAsync(h->s64.x, 0, sizeof(double) * h->d.n, h->stream);
    s = check_cuda(h, cudaStreamSynchronize(h->stream), "create");
  }
  dfree(ovov_in, h->stream); dfree(ooov_in, h->stream); dfree(ovvv_in, h->stream); dfree(scratch, h->stream);
  if (!s && !std::isfinite(h->omega)) { h->err = "non-finite Fock matrix in the TOP basis"; s = ESMP2_ERR_INVALID_ARG; }
  return s;
#undef ALLOC
}

extern "C" {

void esmp2_destroy(esmp2_handle *h) {
  if (!h) return;
  free_handle(h);
  delete h;
}

esmp2_status esmp2_set_stream(esmp2_handle *h, void *stream) {
  if (!h) return ESMP2_ERR_INVALID_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  return ESMP2_OK;
}

esmp2_status esmp2_layout(const esmp2_handle *h, esmp2_layout_info *o) {
  if (!h || !o) return ESMP2_ERR_INVALID_ARG;
  o->No = h->d.No; o->Nv = h->d.Nv;
  o->block_elems = h->d.B; o->n_elems = h->d.n;
  for (int k = 0; k < 5; ++k) o->weights[k] = kWeights[k];
  o->omega = h->omega; o->E0 = h->E0;
  return ESMP2_OK;
}

esmp2_status esmp2_top_basis(esmp2_handle *h, double *U, double *lam, double *Wv, double *F_top) {
  if (!h) return ESMP2_ERR_INVALID_ARG;
  const int No = h->d.No, Nv = h->d.Nv, N = h->d.N;
  cudaStreamSynchronize(h->stream);
  if (U) cudaMemcpy(U, h->U, sizeof(double) * No * No, cudaMemcpyDeviceToHost);
  if (lam) cudaMemcpy(lam, h->lam, sizeof(double) * No, cudaMemcpyDeviceToHost);
  if (Wv) cudaMemcpy(Wv, h->Wv, sizeof(double) * Nv * Nv, cudaMemcpyDeviceToHost);
  if (F_top) cudaMemcpy(F_top, h->F, sizeof(double) * N * N, cudaMemcpyDeviceToHost);
  return check_cuda(h, cudaGetLastError(), "top_basis");
}

esmp2_status esmp2_sigma(esmp2_handle *h, const double *x, double *y, esmp2_precision p) {
  if (!h || !x || !y || x == y) return ESMP2_ERR_INVALID_ARG;
  if (p == ESMP2_FP64) return sigma64(h, x, y);
  if (p == ESMP2_FP64_TC) {
    if (!split_supported(h, kFp64TcLevels)) { h->err = "ESMP2_FP64_TC needs Nv < 910"; return ESMP2_ERR_UNSUPPORTED; }
    return sigma64(h, x, y, kFp64TcLevels);
  }
  if (p == ESMP2_MIXED_BF16 || p == ESMP2_MIXED_TF32 || p == ESMP2_REDUCED_MIXED) {
    if (p != ESMP2_MIXED_BF16 && h->d.No > 32) { h->err = "precision needs No <= 32"; return ESMP2_ERR_UNSUPPORTED; }
    h->tf32 = p == ESMP2_MIXED_TF32;
    h->arrowv = p == ESMP2_REDUCED_MIXED;
    return sigma_mixed(h, x, y);
  }
  h->err = "precision not supported";
  return ESMP2_ERR_UNSUPPORTED;
}

esmp2_status esmp2_profile_sigma(esmp2_handle *h, const double *x, double *y, esmp2_precision p, int reps,
                                 double *ms) {
  if (!h || !x || !y || !ms || x == y || reps < 1) return ESMP2_ERR_INVALID_ARG;
  if (p == ESMP2_FP64) return profile64(h, x, y, reps, ms);
  if (p == ESMP2_FP64_TC && split_supported(h, kFp64TcLevels)) return profile64(h, x, y, reps, ms, kFp64TcLevels);
  if (p == ESMP2_MIXED_BF16 || p == ESMP2_MIXED_TF32 || p == ESMP2_REDUCED_MIXED) {
    if (p != ESMP2_MIXED_BF16 && h->d.No > 32) { h->err = "precision needs No <= 32"; return ESMP2_ERR_UNSUPPORTED; }
    h->tf32 = p == ESMP2_MIXED_TF32;
    h->arrowv = p == ESMP2_REDUCED_MIXED;
    return profile_mixed(h, x, y, reps, ms);
  }
  h->err = "precision not supported";
  return ESMP2_ERR_UNSUPPORTED;
}

esmp2_status esmp2_virtual_contraction(esmp2_handle *h, const double *x, double *y, esmp2_precision p) {
  if (!h || !x || !y || x == y) return ESMP2_ERR_INVALID_ARG;
  if (p == ESMP2_FP64) return virtual_contraction(h, x, y, 0);
  if (p == ESMP2_MIXED_BF16) return virtual_contraction(h, x, y, 1);
  if (p == ESMP2_FP64_TC && split_supported(h, kFp64TcLevels)) return virtual_contraction(h, x, y, 2);
  h->err = "precision not supported";
  return ESMP2_ERR_UNSUPPORTED;
}

esmp2_status esmp2_rhs(esmp2_handle *h, double *b) {
  if (!h || !b) return ESMP2_ERR_INVALID_ARG;
  cudaMemcpyAsync(b, h->b, sizeof(double) * h->d.n, cudaMemcpyDeviceToDevice, h->stream);
  return check_cuda(h, cudaGetLastError(), "rhs");
}

esmp2_status esmp2_solve(esmp2_handle *h, double tol, int maxit, esmp2_precision p, esmp2_solve_info *info) {
  if (!h || !(tol > 0) || maxit < 1) return ESMP2_ERR_INVALID_ARG;
  if (p == ESMP2_FP64) return solve64(h, tol, maxit, info);
  if (p == ESMP2_FP64_TC) {
    if (!split_supported(h, kFp64TcLevels)) { h->err = "ESMP2_FP64_TC needs Nv < 910"; return ESMP2_ERR_UNSUPPORTED; }
    return solve64(h, tol, maxit, info, 1);
  }
  if (p == ESMP2_MIXED_BF16) return solve_mixed(h, tol, maxit, info);
  if (p == ESMP2_MIXED_TF32) return solve_mixed(h, tol, maxit, info, true);
  if (p == ESMP2_REDUCED_MIXED) return solve_mixed(h, tol, maxit, info, false, true);
  if (p == ESMP2_REDUCED_MINRES) return solve_minres(h, tol, maxit, info);
  h->err = "precision not supported";
  return ESMP2_ERR_UNSUPPORTED;
}

esmp2_status esmp2_get_solution(esmp2_handle *h, double *x) {
  if (!h || !x) return ESMP2_ERR_INVALID_ARG;
  if (h->x_basis == 0) {
    cudaMemcpyAsync(x, h->s64.x, sizeof(double) * h->d.n, cudaMemcpyDeviceToDevice, h->stream);
  } else {   // rotated back to the TOP basis (the stored solution keeps its basis)
    const double *src = h->s64.x;
    if (h->x_basis == 2) {
      if (esmp2_status s = rotate_virt(h, src, x, h->s64.p, false)) return s;
      src = x;
    }
    rotate_occ(h, src, x, h->s64.p, false);
  }
  return check_cuda(h, cudaGetLastError(), "get_solution");
}

esmp2_status esmp2_set_solution(esmp2_handle *h, const double *x) {
  if (!h || !x) return ESMP2_ERR_INVALID_ARG;
  cudaMemcpyAsync(h->s64.x, x, sizeof(double) * h->d.n, cudaMemcpyDeviceToDevice, h->stream);
  h->x_basis = 0;
  h->x_zero = false;
  h->r_true = false;
  return check_cuda(h, cudaGetLastError(), "set_solution");
}

esmp2_status esmp2_grad(esmp2_handle *h, double *dF, double *dOVOV, int adjoint_solve, double *adjoint_rel_diff) {
  if (!h) return ESMP2_ERR_INVALID_ARG;
  return gradient(h, dF, dOVOV, adjoint_solve, adjoint_rel_diff);
}

esmp2_status esmp2_energy(esmp2_handle *h, esmp2_energy_parts *parts) {
  if (!h || !parts) return ESMP2_ERR_INVALID_ARG;
  return energy(h, parts);
}

}  // extern "C"

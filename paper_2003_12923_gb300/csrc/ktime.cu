// Process-wide timing of the kernel families of the hot path (esmp2_kernel_timing).
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.h"

namespace esmp2 {
namespace {
struct Rec {
  cudaEvent_t a, b;
  int fam;
  double alg, exec;
};
std::atomic<int> g_on{0};
std::mutex g_mu;
std::vector<Rec> g_recs;
}  // namespace

KScope::KScope(cudaStream_t st, int family, double alg_units, double exec_units)
    : st_(st), fam_(family), alg_(alg_units), exec_(exec_units) {
  if (!g_on.load(std::memory_order_relaxed)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st_, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;  // graph capture
  if (cudaEventCreate(&a_) != cudaSuccess || cudaEventCreate(&b_) != cudaSuccess) {
    if (a_) cudaEventDestroy(a_);
    a_ = b_ = nullptr;
    return;
  }
  cudaEventRecord(a_, st_);
}

KScope::~KScope() {
  if (!a_) return;
  cudaEventRecord(b_, st_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back({a_, b_, fam_, alg_, exec_});
}

void debug_phase(esmp2_handle *h, const char *name) {
  static const bool on = std::getenv("ESMP2_DEBUG") != nullptr;
  if (!on) return;
  static thread_local auto last = std::chrono::steady_clock::now();
  cudaStreamSynchronize(h->stream);
  const auto now = std::chrono::steady_clock::now();
  std::fprintf(stderr, "esmp2 phase %-28s %9.3f ms\n", name, std::chrono::duration<double, std::milli>(now - last).count());
  last = now;
}

cudaError_t dmalloc(void **p, size_t bytes, cudaStream_t st) {
  static std::mutex mu;
  static bool ready[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool = nullptr;
  const bool have_pool = dev >= 0 && dev < 64 && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess;
  if (have_pool) {
    std::lock_guard<std::mutex> lk(mu);
    if (!ready[dev]) {
      size_t fr = 0, tot = 0;
      cudaMemGetInfo(&fr, &tot);
      uint64_t keep = tot / 2;   // memory kept cached between handles (freed at most down to this)
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      ready[dev] = true;
    }
  }
  cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 1, st);
  if (e == cudaErrorMemoryAllocation && have_pool) {  // give cached memory back and retry once
    cudaGetLastError();
    cudaDeviceSynchronize();
    cudaMemPoolTrimTo(pool, 0);
    e = cudaMallocAsync(p, bytes ? bytes : 1, st);
  }
  return e;
}

void dfree(void *p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

cudaError_t smem_limit_once(const void *func, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, cudaError_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(dev, func);
  auto it = done.find(key);
  if (it != done.end()) return it->second;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  done[key] = e;
  return e;
}

double unique_amplitudes(int No, int Nv) {
  auto c2 = [](double n) { return n * (n - 1) / 2; };
  const double T = c2(No) * c2(Nv), S = 0.5 * No * No * (double)Nv * Nv, X = c2(No - 1) * c2(Nv - 1),
               Y = c2(No) * c2(Nv), Z = ((double)No * Nv - 1) * (No - 1) * (double)(Nv - 1);
  return T + S + X + Y + Z;
}
}  // namespace esmp2

extern "C" {

void esmp2_kernel_timing(int enable) { esmp2::g_on.store(enable ? 1 : 0); }

esmp2_status esmp2_kernel_times(esmp2_kernel_time *out) {
  using namespace esmp2;
  if (!out) return ESMP2_ERR_INVALID_ARG;
  for (int k = 0; k < ESMP2_KT_COUNT; ++k) out[k] = esmp2_kernel_time{0, 0.0, 0.0, 0.0};
  std::vector<Rec> recs;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    recs.swap(g_recs);
  }
  esmp2_status st = ESMP2_OK;
  for (const Rec &r : recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
      st = ESMP2_ERR_CUDA;
    if (r.fam >= 0 && r.fam < ESMP2_KT_COUNT) {
      out[r.fam].launches += 1;
      out[r.fam].ms += ms;
      out[r.fam].alg_units += r.alg;
      out[r.fam].exec_units += r.exec;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  return st;
}

}  // extern "C"

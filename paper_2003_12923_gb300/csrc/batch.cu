// Batched solve of independent ESMP2 instances of uneven size.
//
// Instances share nothing, so the batch is work-parallel: `concurrency` host workers
// each own a non-blocking CUDA stream and take the next instance from a shared counter
// (create -> solve -> energy -> destroy on that stream).  Small instances, which cannot
// fill the GPU alone, overlap with one another; large ones run side by side as memory
// permits.
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "internal.h"

namespace esmp2 {
esmp2_status create_impl(esmp2_handle **out, const esmp2_desc *d, cudaStream_t stream);
}

extern "C" esmp2_status esmp2_batch_solve(const esmp2_desc *descs, int count, double tol, int maxit,
                                          esmp2_precision p, int concurrency, esmp2_batch_result *results) {
  using namespace esmp2;
  if (!descs || !results || count < 0 || concurrency < 1 || !(tol > 0) || maxit < 1) return ESMP2_ERR_INVALID_ARG;
  if (p != ESMP2_FP64 && p != ESMP2_MIXED_BF16 && p != ESMP2_MIXED_TF32 && p != ESMP2_FP64_TC &&
      p != ESMP2_REDUCED_MIXED)
    return ESMP2_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ESMP2_ERR_CUDA;
  std::atomic<int> next{0};
  auto worker = [&]() {
    cudaSetDevice(dev);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
    for (int k; (k = next.fetch_add(1)) < count;) {
      esmp2_batch_result &r = results[k];
      std::memset(&r, 0, sizeof(r));
      esmp2_handle *h = nullptr;
      esmp2_status s = create_impl(&h, &descs[k], st);
      if (!s) {
        if (p == ESMP2_MIXED_BF16 || p == ESMP2_MIXED_TF32 || p == ESMP2_REDUCED_MIXED)
          s = solve_mixed(h, tol, maxit, &r.info, p == ESMP2_MIXED_TF32, p == ESMP2_REDUCED_MIXED);
        else s = solve64(h, tol, maxit, &r.info, p == ESMP2_FP64_TC ? 1 : 0);
      }
      if (!s) s = energy(h, &r.e2);
      r.status = s;
      if (s && h) std::strncpy(r.message, h->err.c_str(), sizeof(r.message) - 1);
      if (h) {
        r.kernel_launches = h->launches;
        esmp2_destroy(h);
      }
    }
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  };
  const int nw = std::max(1, std::min(concurrency, count));
  std::vector<std::thread> pool;
  for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
  for (auto &t : pool) t.join();
  for (int k = 0; k < count; ++k)
    if (results[k].status != ESMP2_OK) return results[k].status;
  return ESMP2_OK;
}

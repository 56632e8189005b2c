// lv_api.cu -- error reporting, version and launch accounting of the C ABI.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>

#include "lv_common.cuh"

namespace lv {

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

lv_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LV_OK;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return LV_ERR_CUDA;
}

void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

std::mutex& setup_mutex() {
  static std::mutex mu;
  return mu;
}

}  // namespace lv

extern "C" const char* lv_last_error(void) { return lv::g_err; }

extern "C" int32_t lv_version(void) { return (LV_VERSION_MAJOR << 16) | LV_VERSION_MINOR; }

extern "C" int64_t lv_launch_count(void) { return (int64_t)lv::g_launches.load(); }

extern "C" lv_status lv_check_status(const int32_t* d_status, void* stream) {
  if (!d_status) { lv::set_error("lv_check_status: null status word"); return LV_ERR_INVALID_ARG; }
  int32_t h = 0;
  cudaStream_t s = (cudaStream_t)stream;
  lv_status e = lv::cuda_check(cudaMemcpyAsync(&h, d_status, sizeof(h), cudaMemcpyDeviceToHost, s), "lv_check_status");
  if (e != LV_OK) return e;
  e = lv::cuda_check(cudaStreamSynchronize(s), "lv_check_status");
  if (e != LV_OK) return e;
  if (h < LV_OK || h > LV_ERR_UNSUPPORTED) {
    lv::set_error("lv_check_status: unknown device status %d", h);
    return LV_ERR_CUDA;
  }
  if (h != LV_OK) lv::set_error("device status %d", h);
  return (lv_status)h;
}

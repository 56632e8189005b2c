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

namespace {
// 16-byte words where the range allows, bytes at the ragged ends
__global__ void k_zero(const ZeroRanges r) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    char* p = (char*)r.p[k];
    const size_t n = r.bytes[k];
    if (!p || !n) continue;
    const size_t head = ((16 - ((uintptr_t)p & 15)) & 15) < n ? ((16 - ((uintptr_t)p & 15)) & 15) : n;
    const size_t words = (n - head) / 16;
    for (size_t i = t; i < head; i += stride) p[i] = 0;
    uint4* w = (uint4*)(p + head);
    for (size_t i = t; i < words; i += stride) w[i] = make_uint4(0u, 0u, 0u, 0u);
    for (size_t i = head + 16 * words + t; i < n; i += stride) p[i] = 0;
  }
}
}  // namespace

void zero_async(cudaStream_t s, void* p0, size_t b0, void* p1, size_t b1, void* p2, size_t b2, void* p3,
                size_t b3) {
  ZeroRanges r;
  r.p[0] = p0; r.bytes[0] = p0 ? b0 : 0;
  r.p[1] = p1; r.bytes[1] = p1 ? b1 : 0;
  r.p[2] = p2; r.bytes[2] = p2 ? b2 : 0;
  r.p[3] = p3; r.bytes[3] = p3 ? b3 : 0;
  size_t most = 0;
  for (int k = 0; k < 4; ++k) most = r.bytes[k] > most ? r.bytes[k] : most;
  if (most == 0) return;
  size_t blocks = (most / 16 + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 1216) blocks = 1216;
  k_zero<<<(unsigned)blocks, 256, 0, s>>>(r);
  count_launch(1);
}

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

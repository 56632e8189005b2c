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

namespace {
// lv_rows_scatter: the arrays' units (16-byte words or bytes) laid end to end
struct RowsArg {
  int n;
  int word[LV_MAX_AUX];         // 1: 16-byte units, 0: bytes
  int64_t upr[LV_MAX_AUX];      // units per row (a plain copy: all units in one row)
  int64_t start[LV_MAX_AUX + 1];
  char* dst[LV_MAX_AUX];
  const char* src[LV_MAX_AUX];
  int64_t row_bytes[LV_MAX_AUX];
  const int64_t* idx[LV_MAX_AUX];
};

__global__ void k_rows_scatter(const __grid_constant__ RowsArg r) {
  const int64_t total = r.start[r.n];
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < total; u += (int64_t)gridDim.x * blockDim.x) {
    int a = 0;
    while (a + 1 < r.n && u >= r.start[a + 1]) ++a;
    const int64_t l = u - r.start[a], row = l / r.upr[a], k = l - row * r.upr[a];
    const int64_t drow = r.idx[a] ? r.idx[a][row] : row;
    if (r.word[a]) {
      ((uint4*)(r.dst[a] + drow * r.row_bytes[a]))[k] = ((const uint4*)(r.src[a] + row * r.row_bytes[a]))[k];
    } else {
      r.dst[a][drow * r.row_bytes[a] + k] = r.src[a][row * r.row_bytes[a] + k];
    }
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

extern "C" lv_status lv_rows_scatter(const lv_rows* arrays, int n_arrays, void* stream) {
  using namespace lv;
  if (n_arrays < 0 || n_arrays > LV_MAX_AUX || (n_arrays > 0 && !arrays)) {
    set_error("n_arrays must be 0..%d", LV_MAX_AUX);
    return LV_ERR_INVALID_ARG;
  }
  RowsArg r;
  r.n = 0;
  r.start[0] = 0;
  for (int i = 0; i < n_arrays; ++i) {
    const lv_rows& a = arrays[i];
    if (a.m < 0 || a.row_bytes < 1 || (a.m > 0 && (!a.dst || !a.src))) {
      set_error("array %d: bad description", i);
      return LV_ERR_INVALID_ARG;
    }
    if (a.m == 0) continue;
    const int k = r.n++;
    const bool al = (((uintptr_t)a.dst | (uintptr_t)a.src) & 15) == 0;
    r.dst[k] = (char*)a.dst;
    r.src[k] = (const char*)a.src;
    r.idx[k] = a.idx;
    if (!a.idx) {  // a plain copy: one row of all the bytes
      r.row_bytes[k] = a.m * a.row_bytes;
      r.word[k] = al && r.row_bytes[k] % 16 == 0;
      r.upr[k] = r.word[k] ? r.row_bytes[k] / 16 : r.row_bytes[k];
      r.start[k + 1] = r.start[k] + r.upr[k];
    } else {
      r.row_bytes[k] = a.row_bytes;
      r.word[k] = al && a.row_bytes % 16 == 0;
      r.upr[k] = r.word[k] ? a.row_bytes / 16 : a.row_bytes;
      r.start[k + 1] = r.start[k] + a.m * r.upr[k];
    }
  }
  if (r.n == 0) return LV_OK;
  const int64_t total = r.start[r.n];
  const int64_t want = (total + 255) / 256;
  const unsigned blocks = (unsigned)(want < 4 * 1216 ? (want < 1 ? 1 : want) : 4 * 1216);
  k_rows_scatter<<<blocks, 256, 0, (cudaStream_t)stream>>>(r);
  count_launch(1);
  return cuda_check(cudaGetLastError(), "lv_rows_scatter");
}

// lv_common.cuh -- internal helpers shared by the CUDA translation units of
// the LiteVoxel rasterizer library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>

#include "litevoxel.h"

namespace lv {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- host-side
void set_error(const char* fmt, ...);
lv_status cuda_check(cudaError_t e, const char* what);
void count_launch(int k = 1);
// The weights, their per-view sums and the loss sums in a workspace of
// lv_lf_weights for the given views (the backward's fused LF loss).
lv_status lf_fused_buffers(const int32_t* widths, const int32_t* heights, int n_views, void* workspace,
                           size_t ws_bytes, const float** w, const double** wsum, double** lsum);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Host-side one-time set-up per call site and device (kernel attributes,
// occupancy): f() runs once for each device that reaches the call site,
// under a library-wide lock, and before any caller of that device passes.
std::mutex& setup_mutex();
inline int current_device() {
  int dev = 0;
  return cudaGetDevice(&dev) == cudaSuccess ? dev : 0;
}
template <class F>
void once_per_device(std::atomic<unsigned long long>& done, F&& f) {
  const int dev = current_device();
  const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;  // beyond 64 devices: every time
  if (bit && (done.load(std::memory_order_acquire) & bit)) return;
  std::lock_guard<std::mutex> lock(setup_mutex());
  if (bit && (done.load(std::memory_order_relaxed) & bit)) return;
  f();
  if (bit) done.fetch_or(bit, std::memory_order_release);
}

// Bump allocator over a caller-owned workspace (also used to size it).
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base((char*)b) {}
  template <typename T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = base ? (T*)(base + off) : nullptr;
    off += sizeof(T) * (count > 0 ? count : 1);
    return p;
  }
};

// Zero up to four small device ranges with one kernel launch.  In a CUDA
// graph a memset node delays the kernel after it by several microseconds
// (measured), a kernel node by well under one, so the hot path clears its
// counters, status words and tile ranges this way.  Null or empty ranges
// are skipped.
struct ZeroRanges {
  void* p[4];
  size_t bytes[4];
};
void zero_async(cudaStream_t s, void* p0, size_t b0, void* p1 = nullptr, size_t b1 = 0, void* p2 = nullptr,
                size_t b2 = 0, void* p3 = nullptr, size_t b3 = 0);

// ---------------------------------------------------------------- device-side
__device__ __forceinline__ void report(int32_t* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// order-preserving map from f32 bits to u32 (negative values first)
__host__ __device__ __forceinline__ uint32_t order_key(float f) {
#ifdef __CUDA_ARCH__
  uint32_t u = __float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, 4);
#endif
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <typename T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// fire-and-forget vector reduction into global memory (sm_90+)
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}
__device__ __forceinline__ void red_add(float* addr, float a) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(a) : "memory");
}

}  // namespace lv

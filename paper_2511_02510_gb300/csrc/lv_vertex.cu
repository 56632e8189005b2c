// lv_vertex.cu -- the shared grid-vertex density variant (sm_103a): voxels
// whose corners sit at the same point of the octree's finest grid read one
// density value, so the field is continuous across neighbouring voxels of any
// level whose corners coincide (the voxels still interpolate their own 8
// corners trilinearly, Eq. 2-4 are unchanged).
//
//   lv_build_vertex_index: corner -> vertex id.  Every corner's integer
//     coordinates on the finest grid (half-size units) form a 63-bit key; the
//     8n keys are radix-sorted (stable, 64-bit) and numbered in key order, so
//     vertex ids are the ranks of the distinct corner points (deterministic).
//   lv_vertex_gather: vertex values -> per-voxel corners [n][8] (FP32).
//   lv_vertex_scatter_add: per-voxel corner values [n][8] -> vertex sums
//     (atomics across the voxels sharing a vertex): turns the rasterizer's
//     per-corner density gradient into the vertex gradient, or averages
//     per-voxel corners into vertices with a count array.
#include <math.h>

#include "lv_prims.cuh"

namespace lv {
namespace {

constexpr int TPB = 256;
constexpr int COORD_BITS = 21;
constexpr long long COORD_OFF = 1ll << (COORD_BITS - 1);  // coordinates in [-2^20, 2^20)

struct VxWs {
  unsigned long long* counters;  // [0] 8n (sort count), [1..2] scan totals
  uint64_t *k0, *k1;
  uint32_t *v0, *v1;
  uint32_t* flag;
  uint32_t* rank;
  void* sort_tmp;
  void* scan_tmp;
  size_t bytes;
};

VxWs carve_vx(void* base, int64_t n) {
  VxWs w;
  Carve c(base);
  const int64_t m = 8 * n;
  w.counters = c.take<unsigned long long>(4);
  w.k0 = c.take<uint64_t>(m);
  w.k1 = c.take<uint64_t>(m);
  w.v0 = c.take<uint32_t>(m);
  w.v1 = c.take<uint32_t>(m);
  w.flag = c.take<uint32_t>(m);
  w.rank = c.take<uint32_t>(m);
  w.sort_tmp = c.take<char>(sort_tmp_bytes(m));
  w.scan_tmp = c.take<char>(scan2_tmp_bytes());
  w.bytes = c.off + 256;
  return w;
}

// corner c of voxel v at (centre +- h) on the finest grid; misaligned corners report
__global__ void k_vx_keys(const float4* __restrict__ geom, int64_t n, double inv_unit, uint64_t* __restrict__ keys,
                          int32_t* status) {
  const int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x;
  if (i >= 8 * n) return;
  const int64_t v = i >> 3;
  const int c = (int)(i & 7);
  const float4 g = geom[v];
  const double h = (double)g.w;
  const double p[3] = {(double)g.x + ((c & 1) ? h : -h), (double)g.y + ((c & 2) ? h : -h),
                       (double)g.z + ((c & 4) ? h : -h)};
  uint64_t key = 0;
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double x = p[a] * inv_unit;
    const double r = rint(x);
    ok = ok && fabs(x - r) <= 1e-3 && r >= -(double)COORD_OFF && r < (double)COORD_OFF;
    const uint64_t q = (uint64_t)((long long)r + COORD_OFF) & ((1ull << COORD_BITS) - 1);
    key |= q << (COORD_BITS * a);
  }
  keys[i] = key;
  if (!ok) report(status, LV_ERR_INVALID_ARG);
}

__global__ void k_vx_set_count(unsigned long long* c, unsigned long long v) {
  if (threadIdx.x == 0) *c = v;
}

__global__ void k_vx_flags(const uint64_t* __restrict__ keys, int64_t m, uint32_t* __restrict__ flag) {
  const int64_t r = blockIdx.x * (int64_t)TPB + threadIdx.x;
  if (r < m) flag[r] = (r == 0 || keys[r] != keys[r - 1]) ? 1u : 0u;
}

// the vertex id of sorted position r is the number of distinct keys before it
__global__ void k_vx_assign(const uint32_t* __restrict__ slot, const uint32_t* __restrict__ flag,
                            const uint32_t* __restrict__ excl, int64_t m, uint32_t* __restrict__ vidx) {
  const int64_t r = blockIdx.x * (int64_t)TPB + threadIdx.x;
  if (r < m) vidx[slot[r]] = excl[r] + flag[r] - 1u;
}

__global__ void k_vx_count(const unsigned long long* totals, int64_t* n_vert) {
  if (threadIdx.x == 0) *n_vert = (int64_t)totals[1];
}

template <typename DT>
__global__ void k_vx_gather(const uint32_t* __restrict__ vidx, int64_t m, const DT* __restrict__ vals,
                            float* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x;
  if (i < m) out[i] = to_f32(vals[vidx[i]]);
}

// zero rows (voxels the views never reached) cost one 32-byte read and no atomics
__global__ void k_vx_scatter(const uint32_t* __restrict__ vidx, int64_t n, const float4* __restrict__ corner,
                             float* __restrict__ out, float* __restrict__ count) {
  const int64_t v = blockIdx.x * (int64_t)TPB + threadIdx.x;
  if (v >= n) return;
  const float4 a = corner[2 * v], b = corner[2 * v + 1];
  const float x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  const uint4 i0 = *(const uint4*)(vidx + 8 * v), i1 = *(const uint4*)(vidx + 8 * v + 4);
  const uint32_t id[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (x[c] != 0.f) atomicAdd(out + id[c], x[c]);
    if (count) atomicAdd(count + id[c], 1.f);
  }
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace
}  // namespace lv

using namespace lv;

extern "C" size_t lv_vertex_index_workspace_size(int64_t n) {
  if (n < 0 || n > (0x7fffffffLL >> 3)) return 0;
  return carve_vx(nullptr, n).bytes;
}

extern "C" lv_status lv_build_vertex_index(const float* geom, int64_t n, double unit, uint32_t* vidx,
                                           int64_t* d_n_vert, void* workspace, size_t ws_bytes, int32_t* d_status,
                                           void* stream) {
  if (n < 0 || n > (0x7fffffffLL >> 3) || !(unit > 0.0) || (n > 0 && (!geom || !vidx)) || !d_n_vert) {
    set_error("bad arguments");
    return LV_ERR_INVALID_ARG;
  }
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  VxWs w = carve_vx(workspace, n);
  if (ws_bytes < w.bytes) { set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return LV_ERR_WORKSPACE; }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t m = 8 * n;
  cudaMemsetAsync(d_n_vert, 0, sizeof(int64_t), s);
  if (n == 0) return cuda_check(cudaGetLastError(), "lv_build_vertex_index");
  k_vx_set_count<<<1, 32, 0, s>>>(w.counters, (unsigned long long)m);  // the sort's item count
  int32_t* st = d_status ? d_status : (int32_t*)(w.counters + 3);
  if (!d_status) cudaMemsetAsync(st, 0, sizeof(int32_t), s);
  const unsigned blocks = (unsigned)((m + TPB - 1) / TPB);
  k_vx_keys<<<blocks, TPB, 0, s>>>((const float4*)geom, n, 1.0 / unit, w.k0, st);
  const int which = radix_sort_pairs(w.k0, nullptr, w.k0, w.v0, w.k1, w.v1, w.sort_tmp, w.counters, m,
                                     3 * COORD_BITS, st, s);
  const uint64_t* sk = which ? w.k1 : w.k0;
  const uint32_t* sv = which ? w.v1 : w.v0;
  k_vx_flags<<<blocks, TPB, 0, s>>>(sk, m, w.flag);
  scan2(w.flag, w.flag, m, nullptr, w.rank, w.counters + 1, w.scan_tmp, s);
  k_vx_assign<<<blocks, TPB, 0, s>>>(sv, w.flag, w.rank, m, vidx);
  k_vx_count<<<1, 32, 0, s>>>(w.counters + 1, d_n_vert);
  count_launch(5);
  return cuda_check(cudaGetLastError(), "lv_build_vertex_index");
}

extern "C" lv_status lv_vertex_gather(const uint32_t* vidx, int64_t n, const void* vertex_values, lv_dtype dtype,
                                      float* corners, void* stream) {
  if (n < 0 || (n > 0 && (!vidx || !vertex_values || !corners))) { set_error("bad arguments"); return LV_ERR_INVALID_ARG; }
  if (dtype != LV_F32 && dtype != LV_F16) { set_error("vertex dtype must be F32 or F16"); return LV_ERR_INVALID_ARG; }
  if (n == 0) return LV_OK;
  const int64_t m = 8 * n;
  const unsigned blocks = (unsigned)((m + TPB - 1) / TPB);
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == LV_F32) k_vx_gather<float><<<blocks, TPB, 0, s>>>(vidx, m, (const float*)vertex_values, corners);
  else k_vx_gather<__half><<<blocks, TPB, 0, s>>>(vidx, m, (const __half*)vertex_values, corners);
  count_launch(1);
  return cuda_check(cudaGetLastError(), "lv_vertex_gather");
}

extern "C" lv_status lv_vertex_scatter_add(const uint32_t* vidx, int64_t n, const float* corners, float* vertex_sum,
                                           float* vertex_count, void* stream) {
  if (n < 0 || (n > 0 && (!vidx || !corners || !vertex_sum))) { set_error("bad arguments"); return LV_ERR_INVALID_ARG; }
  if (!aligned16(vidx) || !aligned16(corners)) { set_error("vidx and corners must be 16-byte aligned"); return LV_ERR_INVALID_ARG; }
  if (n == 0) return LV_OK;
  k_vx_scatter<<<(unsigned)((n + TPB - 1) / TPB), TPB, 0, (cudaStream_t)stream>>>(
      vidx, n, (const float4*)corners, vertex_sum, vertex_count);
  count_launch(1);
  return cuda_check(cudaGetLastError(), "lv_vertex_scatter_add");
}

// lv_train.cu -- the rest of a training step on the device (sm_103a): the
// transmittance-concentration term L_Tc and the density total variation L_tv
// of Eq. 17, and the Adam update of the voxel parameters, with the L_tv
// gradient fused into the density update so the densities stream through
// HBM once.  All three are elementwise HBM streams.
//
// Readings: L_Tc = lambda / |P| sum_p T_p (1 - T_p); L_tv = lambda / N sum_v
// sum over the 12 edges (i, j) of the voxel's corner cube of (d_i - d_j)^2
// (corner c = x + 2y + 4z); Adam with one global step t, bias corrections
// 1 / (1 - b^t) computed on the host in double.
#include <math.h>

#include "lv_common.cuh"

namespace lv {
namespace {

constexpr int TPB = 256;
constexpr int MAX_BLOCKS = 8 * 152;

struct TrainWs {
  double* acc;  // [0] L_Tc sum, [1] L_tv sum
  size_t bytes;
};

TrainWs carve_train(void* base) {
  TrainWs w;
  Carve c(base);
  w.acc = c.take<double>(2);
  w.bytes = c.off + 256;
  return w;
}

inline int grid_for(int64_t items) {
  int64_t b = (items + TPB - 1) / TPB;
  return (int)(b < 1 ? 1 : (b > MAX_BLOCKS ? MAX_BLOCKS : b));
}

// a thread's FP32 partial, summed over the block in FP32 and added to a
// device double (one atomic per block)
__device__ __forceinline__ void block_add(float v, double* dst) {
  __shared__ float red[TPB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < TPB / 32 ? red[lane] : 0.f;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v != 0.f) atomicAdd(dst, (double)v);
  }
}

// L_Tc: sum of T (1 - T) and dL/dT = weight (1 - 2T) / |P|
__global__ void __launch_bounds__(TPB) k_tc(const float* __restrict__ T, int64_t n, float weight, float inv_p,
                                           float* __restrict__ dT, int accumulate, double* acc) {
  float part = 0.f;
  const float gs = weight * inv_p;
  for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB) {
    const float t = T[i];
    part += t * (1.f - t);
    if (dT) {
      const float g = gs * (1.f - 2.f * t);
      dT[i] = accumulate ? dT[i] + g : g;
    }
  }
  block_add(part, acc);
}

__global__ void k_train_finish(const double* acc, double scale, float* out) {
  if (threadIdx.x == 0) *out = (float)(*acc * scale);
}

struct AdamK {
  float lr, b1, omb1, b2, omb2, eps, c1, c2;  // c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
};

__device__ __forceinline__ float adam1(float p, float g, float& m, float& v, const AdamK& k) {
  m = k.b1 * m + k.omb1 * g;
  v = k.b2 * v + k.omb2 * g * g;
  return p - k.lr * (m * k.c1) / (sqrtf(v * k.c2) + k.eps);
}

__device__ __forceinline__ void store_f(float* p, float x) { *p = x; }
__device__ __forceinline__ void store_f(__half* p, float x) { *p = __float2half_rn(x); }
__device__ __forceinline__ void store_f(__nv_bfloat16* p, float x) { *p = __float2bfloat16_rn(x); }

// One thread per voxel: the 8 corner densities, their gradient plus the L_tv
// gradient 2 lambda / N sum_{j adjacent} (d_i - d_j), and the Adam update.
template <typename DT>
__global__ void __launch_bounds__(TPB) k_adam_density(int64_t n, DT* __restrict__ dens,
                                                     const float4* __restrict__ grad, float4* __restrict__ m4,
                                                     float4* __restrict__ v4, const AdamK k, float tv2,
                                                     double* tv_acc) {
  float part = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < n; i += (int64_t)gridDim.x * TPB) {
    float d[8], g[8], m[8], v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) d[c] = to_f32(dens[8 * i + c]);
    const float4 g0 = grad[2 * i], g1 = grad[2 * i + 1];
    const float4 m0 = m4[2 * i], m1 = m4[2 * i + 1];
    const float4 v0 = v4[2 * i], v1 = v4[2 * i + 1];
    g[0] = g0.x; g[1] = g0.y; g[2] = g0.z; g[3] = g0.w; g[4] = g1.x; g[5] = g1.y; g[6] = g1.z; g[7] = g1.w;
    m[0] = m0.x; m[1] = m0.y; m[2] = m0.z; m[3] = m0.w; m[4] = m1.x; m[5] = m1.y; m[6] = m1.z; m[7] = m1.w;
    v[0] = v0.x; v[1] = v0.y; v[2] = v0.z; v[3] = v0.w; v[4] = v1.x; v[5] = v1.y; v[6] = v1.z; v[7] = v1.w;
    if (tv2 != 0.f || tv_acc) {
#pragma unroll
      for (int b = 1; b < 8; b <<= 1) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          if (c & b) continue;
          const float diff = d[c] - d[c | b];
          part += diff * diff;
          g[c] += tv2 * diff;
          g[c | b] -= tv2 * diff;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) store_f(dens + 8 * i + c, adam1(d[c], g[c], m[c], v[c], k));
    m4[2 * i] = make_float4(m[0], m[1], m[2], m[3]);
    m4[2 * i + 1] = make_float4(m[4], m[5], m[6], m[7]);
    v4[2 * i] = make_float4(v[0], v[1], v[2], v[3]);
    v4[2 * i + 1] = make_float4(v[4], v[5], v[6], v[7]);
  }
  if (tv_acc) block_add(part, tv_acc);
}

// Flat Adam over SH coefficients, four per thread step (n4 = count / 4).
template <typename ST>
__global__ void __launch_bounds__(TPB) k_adam_flat(int64_t n4, ST* __restrict__ p, const float4* __restrict__ grad,
                                                  float4* __restrict__ m4, float4* __restrict__ v4, const AdamK k) {
  for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < n4; i += (int64_t)gridDim.x * TPB) {
    const float4 g = grad[i];
    float4 m = m4[i], v = v4[i];
    ST* q = p + 4 * i;
    const float x0 = adam1(to_f32(q[0]), g.x, m.x, v.x, k);
    const float x1 = adam1(to_f32(q[1]), g.y, m.y, v.y, k);
    const float x2 = adam1(to_f32(q[2]), g.z, m.z, v.z, k);
    const float x3 = adam1(to_f32(q[3]), g.w, m.w, v.w, k);
    store_f(q, x0);
    store_f(q + 1, x1);
    store_f(q + 2, x2);
    store_f(q + 3, x3);
    m4[i] = m;
    v4[i] = v;
  }
}

template <>
__global__ void __launch_bounds__(TPB) k_adam_flat<float>(int64_t n4, float* __restrict__ p,
                                                         const float4* __restrict__ grad, float4* __restrict__ m4,
                                                         float4* __restrict__ v4, const AdamK k) {
  float4* p4 = (float4*)p;
  for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < n4; i += (int64_t)gridDim.x * TPB) {
    const float4 g = grad[i];
    float4 m = m4[i], v = v4[i], x = p4[i];
    x.x = adam1(x.x, g.x, m.x, v.x, k);
    x.y = adam1(x.y, g.y, m.y, v.y, k);
    x.z = adam1(x.z, g.z, m.z, v.z, k);
    x.w = adam1(x.w, g.w, m.w, v.w, k);
    p4[i] = x;
    m4[i] = m;
    v4[i] = v;
  }
}

// the count % 4 elements after the last whole float4
template <typename ST>
__global__ void k_adam_tail(int64_t first, int64_t count, ST* __restrict__ p, const float* __restrict__ grad,
                            float* __restrict__ m, float* __restrict__ v, const AdamK k) {
  const int64_t i = first + threadIdx.x;
  if (i < count) {
    float mm = m[i], vv = v[i];
    store_f(p + i, adam1(to_f32(p[i]), grad[i], mm, vv, k));
    m[i] = mm;
    v[i] = vv;
  }
}

AdamK make_adam(float lr, const lv_adam_params* p) {
  AdamK k;
  k.lr = lr;
  k.b1 = p->beta1;
  k.omb1 = 1.0f - p->beta1;
  k.b2 = p->beta2;
  k.omb2 = 1.0f - p->beta2;
  k.eps = p->eps;
  k.c1 = (float)(1.0 / (1.0 - pow((double)p->beta1, (double)p->step)));
  k.c2 = (float)(1.0 / (1.0 - pow((double)p->beta2, (double)p->step)));
  return k;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace
}  // namespace lv

using namespace lv;

extern "C" size_t lv_train_workspace_size(void) { return carve_train(nullptr).bytes; }

extern "C" lv_status lv_transmittance_loss(const float* T, int64_t n_pix, float weight, float* loss, float* dL_dT,
                                           int accumulate, void* workspace, size_t ws_bytes, void* stream) {
  if (n_pix < 0 || (n_pix > 0 && !T) || !loss) { set_error("bad arguments"); return LV_ERR_INVALID_ARG; }
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  TrainWs w = carve_train(workspace);
  if (ws_bytes < w.bytes) { set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return LV_ERR_WORKSPACE; }
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(w.acc, 0, sizeof(double), s);
  if (n_pix > 0)
    k_tc<<<grid_for(n_pix), TPB, 0, s>>>(T, n_pix, weight, 1.0f / (float)n_pix, dL_dT, accumulate, w.acc);
  k_train_finish<<<1, 32, 0, s>>>(w.acc, n_pix > 0 ? (double)weight / (double)n_pix : 0.0, loss);
  count_launch(n_pix > 0 ? 2 : 1);
  return cuda_check(cudaGetLastError(), "lv_transmittance_loss");
}

extern "C" lv_status lv_adam_voxels(int64_t n, void* density, lv_dtype density_dtype, void* sh, lv_dtype sh_dtype,
                                    const float* d_density, const float* d_sh, float* m_density, float* v_density,
                                    float* m_sh, float* v_sh, const lv_adam_params* p, float* tv_loss,
                                    void* workspace, size_t ws_bytes, void* stream) {
  if (!p || n < 0) { set_error("bad arguments"); return LV_ERR_INVALID_ARG; }
  if (p->step < 1 || !(p->beta1 >= 0.f && p->beta1 < 1.f) || !(p->beta2 >= 0.f && p->beta2 < 1.f) ||
      !(p->eps >= 0.f)) { set_error("bad Adam parameters"); return LV_ERR_INVALID_ARG; }
  if (density_dtype != LV_F32 && density_dtype != LV_F16) { set_error("density dtype must be F32 or F16"); return LV_ERR_INVALID_ARG; }
  if (sh_dtype != LV_F32 && sh_dtype != LV_BF16) { set_error("sh dtype must be F32 or BF16"); return LV_ERR_INVALID_ARG; }
  if (n > 0 && (!density || !d_density || !m_density || !v_density)) { set_error("null density array"); return LV_ERR_INVALID_ARG; }
  if (n > 0 && d_sh && (!sh || !m_sh || !v_sh)) { set_error("null SH array"); return LV_ERR_INVALID_ARG; }
  if (!aligned16(d_density) || !aligned16(m_density) || !aligned16(v_density) || !aligned16(d_sh) ||
      !aligned16(m_sh) || !aligned16(v_sh) || (sh_dtype == LV_F32 && !aligned16(sh))) {
    set_error("gradient, moment and FP32 SH arrays must be 16-byte aligned"); return LV_ERR_INVALID_ARG;
  }
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  TrainWs w = carve_train(workspace);
  if (ws_bytes < w.bytes) { set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return LV_ERR_WORKSPACE; }
  cudaStream_t s = (cudaStream_t)stream;
  double* tv_acc = tv_loss ? w.acc + 1 : nullptr;
  if (tv_acc) cudaMemsetAsync(tv_acc, 0, sizeof(double), s);
  const float tv2 = n > 0 ? 2.0f * p->tv_weight / (float)n : 0.f;
  if (n > 0) {
    const AdamK kd = make_adam(p->lr_density, p);
    if (density_dtype == LV_F32)
      k_adam_density<float><<<grid_for(n), TPB, 0, s>>>(n, (float*)density, (const float4*)d_density,
                                                        (float4*)m_density, (float4*)v_density, kd, tv2, tv_acc);
    else
      k_adam_density<__half><<<grid_for(n), TPB, 0, s>>>(n, (__half*)density, (const float4*)d_density,
                                                         (float4*)m_density, (float4*)v_density, kd, tv2, tv_acc);
    count_launch(1);
    if (d_sh) {
      const AdamK ks = make_adam(p->lr_sh, p);
      const int64_t n4 = n * 12;
      if (sh_dtype == LV_F32)
        k_adam_flat<float><<<grid_for(n4), TPB, 0, s>>>(n4, (float*)sh, (const float4*)d_sh, (float4*)m_sh,
                                                        (float4*)v_sh, ks);
      else
        k_adam_flat<__nv_bfloat16><<<grid_for(n4), TPB, 0, s>>>(n4, (__nv_bfloat16*)sh, (const float4*)d_sh,
                                                                (float4*)m_sh, (float4*)v_sh, ks);
      count_launch(1);
    }
  }
  if (tv_loss) {
    k_train_finish<<<1, 32, 0, s>>>(tv_acc, n > 0 ? (double)p->tv_weight / (double)n : 0.0, tv_loss);
    count_launch(1);
  }
  return cuda_check(cudaGetLastError(), "lv_adam_voxels");
}

extern "C" lv_status lv_adam_array(int64_t count, void* param, lv_dtype dtype, const float* grad, float* m, float* v,
                                   float lr, const lv_adam_params* p, void* stream) {
  if (!p || count < 0 || (count > 0 && (!param || !grad || !m || !v))) { set_error("bad arguments"); return LV_ERR_INVALID_ARG; }
  if (p->step < 1 || !(p->beta1 >= 0.f && p->beta1 < 1.f) || !(p->beta2 >= 0.f && p->beta2 < 1.f) ||
      !(p->eps >= 0.f)) { set_error("bad Adam parameters"); return LV_ERR_INVALID_ARG; }
  if (dtype != LV_F32 && dtype != LV_F16 && dtype != LV_BF16) { set_error("bad dtype"); return LV_ERR_INVALID_ARG; }
  if (!aligned16(grad) || !aligned16(m) || !aligned16(v) || (dtype == LV_F32 && !aligned16(param))) {
    set_error("gradient, moments and FP32 parameters must be 16-byte aligned"); return LV_ERR_INVALID_ARG;
  }
  if (count == 0) return LV_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const AdamK k = make_adam(lr, p);
  const int64_t n4 = count / 4, first = 4 * n4;
  if (dtype == LV_F32) {
    if (n4) k_adam_flat<float><<<grid_for(n4), TPB, 0, s>>>(n4, (float*)param, (const float4*)grad, (float4*)m,
                                                           (float4*)v, k);
    if (first < count) k_adam_tail<float><<<1, 32, 0, s>>>(first, count, (float*)param, grad, m, v, k);
  } else if (dtype == LV_F16) {
    if (n4) k_adam_flat<__half><<<grid_for(n4), TPB, 0, s>>>(n4, (__half*)param, (const float4*)grad, (float4*)m,
                                                            (float4*)v, k);
    if (first < count) k_adam_tail<__half><<<1, 32, 0, s>>>(first, count, (__half*)param, grad, m, v, k);
  } else {
    if (n4) k_adam_flat<__nv_bfloat16><<<grid_for(n4), TPB, 0, s>>>(n4, (__nv_bfloat16*)param, (const float4*)grad,
                                                                    (float4*)m, (float4*)v, k);
    if (first < count) k_adam_tail<__nv_bfloat16><<<1, 32, 0, s>>>(first, count, (__nv_bfloat16*)param, grad, m, v, k);
  }
  count_launch(2);
  return cuda_check(cudaGetLastError(), "lv_adam_array");
}

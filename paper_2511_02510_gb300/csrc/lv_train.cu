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

// Two lanes per voxel, one float4 (4 corners, corner c = x + 2y + 4z: lane 0
// of the pair holds z = 0, lane 1 z = 1) of every array each, so all loads and
// stores are coalesced 16-byte words.  The L_tv gradient 2 lambda / N sum over
// adjacent corners (d_i - d_j) takes the x and y neighbours from the lane's own
// four corners and the z neighbour from the partner lane (one shuffle).
template <typename DT> struct Quad;
template <> struct Quad<float> {
  static __device__ __forceinline__ float4 load(const float* p) { return *(const float4*)p; }
  static __device__ __forceinline__ void store(float* p, float4 x) { *(float4*)p = x; }
};
template <> struct Quad<__half> {
  static __device__ __forceinline__ float4 load(const __half* p) {
    const uint2 u = *(const uint2*)p;
    const float2 a = __half22float2(*(const __half2*)&u.x), b = __half22float2(*(const __half2*)&u.y);
    return make_float4(a.x, a.y, b.x, b.y);
  }
  static __device__ __forceinline__ void store(__half* p, float4 x) {
    const __half2 a = __floats2half2_rn(x.x, x.y), b = __floats2half2_rn(x.z, x.w);
    uint2 u;
    u.x = *(const uint32_t*)&a;
    u.y = *(const uint32_t*)&b;
    *(uint2*)p = u;
  }
};

template <typename DT>
__global__ void __launch_bounds__(TPB) k_adam_density(int64_t n, DT* __restrict__ dens,
                                                     const float4* __restrict__ grad, float4* __restrict__ m4,
                                                     float4* __restrict__ v4, const AdamK k, float tv2,
                                                     double* tv_acc) {
  const int lane = threadIdx.x & 31;
  const int64_t total = 2 * n;  // float4 words, two per voxel
  const int64_t stride = (int64_t)gridDim.x * TPB;
  float part = 0.f;
  for (int64_t b = blockIdx.x * (int64_t)TPB + (threadIdx.x & ~31); b < total; b += stride) {  // warp-uniform
    const int64_t j = b + lane;
    const bool ok = j < total;  // pairs are whole: total and b are even
    float4 d = make_float4(0.f, 0.f, 0.f, 0.f), g = d, m = d, v = d;
    if (ok) {
      d = Quad<DT>::load(dens + 4 * j);
      g = grad[j];
      m = m4[j];
      v = v4[j];
    }
    // the partner's corners at the same (x, y): the z neighbours
    const float4 o = make_float4(__shfl_xor_sync(FULL, d.x, 1), __shfl_xor_sync(FULL, d.y, 1),
                                 __shfl_xor_sync(FULL, d.z, 1), __shfl_xor_sync(FULL, d.w, 1));
    if (ok && (tv2 != 0.f || tv_acc)) {
      // own corners (x, y) = (0,0) (1,0) (0,1) (1,1): x edges d.x-d.y, d.z-d.w; y edges d.x-d.z, d.y-d.w
      const float ex0 = d.x - d.y, ex1 = d.z - d.w, ey0 = d.x - d.z, ey1 = d.y - d.w;
      const float ez0 = d.x - o.x, ez1 = d.y - o.y, ez2 = d.z - o.z, ez3 = d.w - o.w;
      part += ex0 * ex0 + ex1 * ex1 + ey0 * ey0 + ey1 * ey1;
      if (!(j & 1)) part += ez0 * ez0 + ez1 * ez1 + ez2 * ez2 + ez3 * ez3;  // each z edge once
      g.x += tv2 * (ex0 + ey0 + ez0);
      g.y += tv2 * (-ex0 + ey1 + ez1);
      g.z += tv2 * (ex1 - ey0 + ez2);
      g.w += tv2 * (-ex1 - ey1 + ez3);
    }
    if (ok) {
      d.x = adam1(d.x, g.x, m.x, v.x, k);
      d.y = adam1(d.y, g.y, m.y, v.y, k);
      d.z = adam1(d.z, g.z, m.z, v.z, k);
      d.w = adam1(d.w, g.w, m.w, v.w, k);
      Quad<DT>::store(dens + 4 * j, d);
      m4[j] = m;
      v4[j] = v;
    }
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
  const int64_t stride = (int64_t)gridDim.x * TPB;
  // two independent words per step: more loads in flight
  for (int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x; i < n4; i += 2 * stride) {
    const int64_t i2 = i + stride;
    const bool two = i2 < n4;
    const float4 g = grad[i], g2 = two ? grad[i2] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 m = m4[i], v = v4[i], x = p4[i];
    float4 mb = two ? m4[i2] : g2, vb = two ? v4[i2] : g2, xb = two ? p4[i2] : g2;
    x.x = adam1(x.x, g.x, m.x, v.x, k);
    x.y = adam1(x.y, g.y, m.y, v.y, k);
    x.z = adam1(x.z, g.z, m.z, v.z, k);
    x.w = adam1(x.w, g.w, m.w, v.w, k);
    p4[i] = x;
    m4[i] = m;
    v4[i] = v;
    if (two) {
      xb.x = adam1(xb.x, g2.x, mb.x, vb.x, k);
      xb.y = adam1(xb.y, g2.y, mb.y, vb.y, k);
      xb.z = adam1(xb.z, g2.z, mb.z, vb.z, k);
      xb.w = adam1(xb.w, g2.w, mb.w, vb.w, k);
      p4[i2] = xb;
      m4[i2] = mb;
      v4[i2] = vb;
    }
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
      k_adam_density<float><<<grid_for(2 * n), TPB, 0, s>>>(n, (float*)density, (const float4*)d_density,
                                                        (float4*)m_density, (float4*)v_density, kd, tv2, tv_acc);
    else
      k_adam_density<__half><<<grid_for(2 * n), TPB, 0, s>>>(n, (__half*)density, (const float4*)d_density,
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

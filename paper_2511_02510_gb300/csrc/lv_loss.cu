// lv_loss.cu -- low-frequency-weighted photometric loss (LiteVoxel Sec. IV-B,
// Eq. 7-10 and Eq. 18) for sm_103a.  Per view: Sobel magnitude of the ground
// truth luma (stop-gradient), exact nearest-rank percentile normalisation by a
// radix select, inverse-Sobel weight (eps + 1 - s)^gamma, mean normalisation,
// weighted squared error and its gradient.  Sums are accumulated in FP64.
#include <mutex>

#include "lv_prims.cuh"

namespace lv {

namespace {

constexpr int TPB = 256;

struct ViewPix {
  int n;
  int W[LV_MAX_VIEWS];
  int H[LV_MAX_VIEWS];
  long long off[LV_MAX_VIEWS + 1];
  uint32_t k[LV_MAX_VIEWS];  // nearest-rank index of the percentile
};

struct LfWs {
  SelectQuery* q;
  void* sel_tmp;
  double* wsum;   // [views]
  double* lsum;   // [views]
  uint16_t* grp;  // [pixels]
  uint32_t* mkey; // [pixels] Sobel magnitude bits
  float* w;       // [pixels] unnormalised weight
  size_t bytes;
};

LfWs carve_lf(void* base, int nv, int64_t pixels) {
  LfWs w;
  Carve c(base);
  w.q = c.take<SelectQuery>(SELECT_MAX_QUERIES);
  w.sel_tmp = c.take<char>(select_tmp_bytes(SELECT_MAX_QUERIES));
  w.wsum = c.take<double>(LV_MAX_VIEWS);
  w.lsum = c.take<double>(LV_MAX_VIEWS);
  w.grp = c.take<uint16_t>(pixels);
  w.mkey = c.take<uint32_t>(pixels);
  w.w = c.take<float>(pixels);
  w.bytes = c.off + 256;
  return w;
}

__device__ __forceinline__ int view_of(const ViewPix& vp, long long p) {
  int v = 0;
  while (v + 1 < vp.n && p >= vp.off[v + 1]) ++v;
  return v;
}

__device__ __forceinline__ float luma(const float* __restrict__ gt, long long p) {
  return (gt[3 * p] + gt[3 * p + 1] + gt[3 * p + 2]) * (1.0f / 3.0f);
}

// Eq. 7 input: |Sobel(Y)| with replicated border
__global__ void k_lf_sobel(const float* __restrict__ gt, const __grid_constant__ ViewPix vp, uint16_t* grp,
                           uint32_t* mkey) {
  long long p = blockIdx.x * (long long)TPB + threadIdx.x;
  if (p >= vp.off[vp.n]) return;
  const int v = view_of(vp, p);
  const long long loc = p - vp.off[v];
  const int W = vp.W[v], H = vp.H[v];
  const int x = (int)(loc % W), y = (int)(loc / W);
  const int xm = max(x - 1, 0), xp = min(x + 1, W - 1), ym = max(y - 1, 0), yp = min(y + 1, H - 1);
  const float* g = gt + 3 * vp.off[v];
#define Y_(a, b) luma(g, (long long)(b) * W + (a))
  const float gx = (Y_(xp, ym) + 2.f * Y_(xp, y) + Y_(xp, yp)) - (Y_(xm, ym) + 2.f * Y_(xm, y) + Y_(xm, yp));
  const float gy = (Y_(xm, yp) + 2.f * Y_(x, yp) + Y_(xp, yp)) - (Y_(xm, ym) + 2.f * Y_(x, ym) + Y_(xp, ym));
#undef Y_
  const float mag = sqrtf(gx * gx + gy * gy);
  grp[p] = (uint16_t)v;
  mkey[p] = __float_as_uint(mag);  // non-negative: bit order == value order
}

__global__ void k_lf_queries(SelectQuery* q, const __grid_constant__ ViewPix vp) {
  int v = threadIdx.x;
  if (v < vp.n) { q[v].group = v; q[v].k = vp.k[v]; }
}

__device__ __forceinline__ void block_add_f64(double v, double* dst) {
  __shared__ double sred[TPB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  if (lane == 0) sred[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < TPB / 32 ? sred[lane] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0 && v != 0.0) atomicAdd(dst, v);
  }
  __syncthreads();
}

// Eq. 7: w = (eps + 1 - s)^gamma, s = clip(|grad| / P, 0, 1); blocks never span views.
// Grid-stride over the view's pixels with a bounded block count: one FP64
// atomic per block (a per-256-pixel atomic would serialise at the L2).
__global__ void k_lf_weight(const uint32_t* __restrict__ mkey, const SelectQuery* q, const __grid_constant__ ViewPix vp,
                            int v, float eps, float gamma, float* w, double* wsum, float* edge_out) {
  const long long lo = vp.off[v], hi = vp.off[v + 1];
  const float P = __uint_as_float(q[v].result);
  const bool norm = q[v].k != 0 && P > 0.f;
  // a thread sums its few pixels in FP32; blocks combine in FP64 (the GPU's FP64
  // rate is low, so no per-pixel FP64 arithmetic)
  float acc = 0.f;
  for (long long p = lo + blockIdx.x * (long long)TPB + threadIdx.x; p < hi; p += (long long)gridDim.x * TPB) {
    float s = 0.f;
    if (norm) s = fminf(fmaxf(__uint_as_float(mkey[p]) / P, 0.f), 1.f);
    if (edge_out) edge_out[p] = s;
    const float wv = gamma == 0.f ? 1.f : powf(eps + 1.f - s, gamma);
    w[p] = wv;
    acc += wv;
  }
  block_add_f64((double)acc, &wsum[v]);
}

// the view's mean weight <w> and gradient scale 2 / (3 |P|), rounded to FP32 from FP64, once per
// block (thread 0; FP64 division is slow on this part) into *mean and *gscale (shared memory)
__device__ __forceinline__ void lf_view_constants(const double* wsum, int v, long long np, float* mean, float* gscale) {
  if (threadIdx.x == 0) {
    *mean = (float)(wsum[v] / (double)np);
    *gscale = (float)(2.0 / (3.0 * (double)np));
  }
  __syncthreads();
}

// Eq. 8 + Eq. 18: w~ = w / <w>, L = 1/|P| sum w~ mean_c r^2, dL/drgb = 2/(3|P|) w~ r
__global__ void k_lf_loss(const float* __restrict__ rgb, const float* __restrict__ gt, const float* __restrict__ w,
                          const __grid_constant__ ViewPix vp, int v, const double* wsum, double* lsum,
                          float* __restrict__ grad) {
  const long long lo = vp.off[v], hi = vp.off[v + 1];
  const long long np = hi - lo;
  __shared__ float s_mean, s_gscale;
  lf_view_constants(wsum, v, np, &s_mean, &s_gscale);
  const float mean = s_mean, gscale = s_gscale;
  float acc = 0.f;  // sum of w~ (r0^2 + r1^2 + r2^2) over this thread's pixels; the 1/3 is applied at the end
  for (long long p = lo + blockIdx.x * (long long)TPB + threadIdx.x; p < hi; p += (long long)gridDim.x * TPB) {
    const float wt = w[p] / mean;
    const float r0 = rgb[3 * p] - gt[3 * p], r1 = rgb[3 * p + 1] - gt[3 * p + 1], r2 = rgb[3 * p + 2] - gt[3 * p + 2];
    acc += wt * (r0 * r0 + r1 * r1 + r2 * r2);
    if (grad) {
      const float c = gscale * wt;
      grad[3 * p] = c * r0;
      grad[3 * p + 1] = c * r1;
      grad[3 * p + 2] = c * r2;
    }
  }
  block_add_f64((double)acc, &lsum[v]);
}

// k_lf_loss over groups of four pixels: three 16-byte loads of rgb and of gt,
// one of w, three 16-byte stores of the gradient.  The pixels of the view
// before the first group boundary (global pixel index a multiple of 4) and
// after the last one go through the scalar path of thread 0 of block 0.  The
// per-pixel arithmetic is that of k_lf_loss; only the summation order of the
// partial sums differs.
__global__ void k_lf_loss4(const float* __restrict__ rgb, const float* __restrict__ gt, const float* __restrict__ w,
                           const __grid_constant__ ViewPix vp, int v, const double* wsum, double* lsum,
                           float* __restrict__ grad) {
  const long long lo = vp.off[v], hi = vp.off[v + 1];
  const long long np = hi - lo;
  __shared__ float s_mean, s_gscale;
  lf_view_constants(wsum, v, np, &s_mean, &s_gscale);
  const float mean = s_mean, gscale = s_gscale;
  const long long g0 = (lo + 3) >> 2, g1 = hi >> 2;  // whole groups [4 g0, 4 g1)
  float acc = 0.f;
  auto one = [&](long long p) {
    const float wt = w[p] / mean;
    const float r0 = rgb[3 * p] - gt[3 * p], r1 = rgb[3 * p + 1] - gt[3 * p + 1], r2 = rgb[3 * p + 2] - gt[3 * p + 2];
    acc += wt * (r0 * r0 + r1 * r1 + r2 * r2);
    if (grad) {
      const float c = gscale * wt;
      grad[3 * p] = c * r0;
      grad[3 * p + 1] = c * r1;
      grad[3 * p + 2] = c * r2;
    }
  };
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (g1 <= g0) {
      for (long long p = lo; p < hi; ++p) one(p);
    } else {
      for (long long p = lo; p < 4 * g0; ++p) one(p);
      for (long long p = 4 * g1; p < hi; ++p) one(p);
    }
  }
  const float4* r4 = (const float4*)rgb;
  const float4* t4 = (const float4*)gt;
  const float4* w4 = (const float4*)w;
  float4* d4 = (float4*)grad;
  for (long long g = g0 + blockIdx.x * (long long)TPB + threadIdx.x; g < g1; g += (long long)gridDim.x * TPB) {
    const float4 a0 = r4[3 * g], a1 = r4[3 * g + 1], a2 = r4[3 * g + 2];
    const float4 b0 = t4[3 * g], b1 = t4[3 * g + 1], b2 = t4[3 * g + 2];
    const float4 wv = w4[g];
    const float r[12] = {a0.x - b0.x, a0.y - b0.y, a0.z - b0.z, a0.w - b0.w, a1.x - b1.x, a1.y - b1.y,
                         a1.z - b1.z, a1.w - b1.w, a2.x - b2.x, a2.y - b2.y, a2.z - b2.z, a2.w - b2.w};
    const float wt[4] = {wv.x / mean, wv.y / mean, wv.z / mean, wv.w / mean};
#pragma unroll
    for (int k = 0; k < 4; ++k) acc += wt[k] * (r[3 * k] * r[3 * k] + r[3 * k + 1] * r[3 * k + 1] + r[3 * k + 2] * r[3 * k + 2]);
    if (grad) {
      float o[12];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float c = gscale * wt[k];
        o[3 * k] = c * r[3 * k];
        o[3 * k + 1] = c * r[3 * k + 1];
        o[3 * k + 2] = c * r[3 * k + 2];
      }
      d4[3 * g] = make_float4(o[0], o[1], o[2], o[3]);
      d4[3 * g + 1] = make_float4(o[4], o[5], o[6], o[7]);
      d4[3 * g + 2] = make_float4(o[8], o[9], o[10], o[11]);
    }
  }
  block_add_f64((double)acc, &lsum[v]);
}

// clear: the sums are zeroed once read (the fused backward's sums start from zero next time)
__global__ void k_lf_finish(const __grid_constant__ ViewPix vp, double* lsum, float* loss, bool clear) {
  int v = threadIdx.x;
  if (v < vp.n) {
    const long long np = vp.off[v + 1] - vp.off[v];
    loss[v] = np > 0 ? (float)(lsum[v] / (3.0 * (double)np)) : 0.f;
    if (clear) lsum[v] = 0.0;
  }
}

bool make_viewpix(const int32_t* widths, const int32_t* heights, int nv, int32_t pctl_ppm, ViewPix* vp) {
  if (nv < 1 || nv > LV_MAX_VIEWS || !widths || !heights) return false;
  vp->n = nv;
  long long off = 0;
  for (int v = 0; v < nv; ++v) {
    if (widths[v] < 1 || heights[v] < 1) return false;
    vp->W[v] = widths[v];
    vp->H[v] = heights[v];
    vp->off[v] = off;
    const long long np = (long long)widths[v] * heights[v];
    unsigned long long k = ((unsigned long long)pctl_ppm * (unsigned long long)np + 999999ull) / 1000000ull;
    if (k < 1) k = 1;
    if (k > (unsigned long long)np) k = np;
    vp->k[v] = (uint32_t)k;
    off += np;
  }
  vp->off[nv] = off;
  return off < 0xffffffffLL;
}

}  // namespace

}  // namespace lv

using namespace lv;

extern "C" float lv_lf_gamma(float t, const lv_lf_params* p) {
  if (!p) return 0.f;
  if (t < p->t0) return 0.f;
  if (t < p->t1) return p->gamma_max * (t - p->t0) / (p->t1 - p->t0);
  return p->gamma_max;
}

extern "C" size_t lv_lf_workspace_size(const int32_t* widths, const int32_t* heights, int n_views) {
  ViewPix vp;
  if (!make_viewpix(widths, heights, n_views, 990000, &vp)) return 0;
  return carve_lf(nullptr, n_views, vp.off[n_views]).bytes;
}

namespace {
unsigned blocks_for(long long np) {
  const long long b = (np + 4 * TPB - 1) / (4 * TPB);  // about four pixels per thread
  return (unsigned)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}
bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

lv_status lf_setup(const int32_t* widths, const int32_t* heights, int n_views, int32_t pctl_ppm, void* workspace,
                   size_t ws_bytes, ViewPix* vp, LfWs* w) {
  if (!make_viewpix(widths, heights, n_views, pctl_ppm, vp)) { set_error("bad view sizes"); return LV_ERR_INVALID_ARG; }
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  *w = carve_lf(workspace, n_views, vp->off[n_views]);
  if (ws_bytes < w->bytes) { set_error("workspace %zu < %zu bytes", ws_bytes, w->bytes); return LV_ERR_WORKSPACE; }
  return LV_OK;
}
}  // namespace

extern "C" lv_status lv_lf_weights(const float* gt, const int32_t* widths, const int32_t* heights, int n_views,
                                   float t, const lv_lf_params* p, void* workspace, size_t ws_bytes, void* stream) {
  if (!gt || !p) { set_error("null argument"); return LV_ERR_INVALID_ARG; }
  if (p->pctl_ppm < 0 || p->pctl_ppm > 1000000) { set_error("pctl_ppm must be in [0, 1e6]"); return LV_ERR_INVALID_ARG; }
  if (!(p->eps > 0.f) || !(p->t1 > p->t0) || !(p->gamma_max >= 0.f)) { set_error("need eps > 0, t1 > t0, gamma_max >= 0"); return LV_ERR_INVALID_ARG; }
  ViewPix vp;
  LfWs w;
  lv_status e = lf_setup(widths, heights, n_views, p->pctl_ppm, workspace, ws_bytes, &vp, &w);
  if (e != LV_OK) return e;
  const int64_t P = vp.off[n_views];
  cudaStream_t s = (cudaStream_t)stream;
  const float gamma = lv_lf_gamma(t, p);
  // the weight sums, and the loss sums a backward with the fused loss accumulates
  zero_async(s, w.wsum, sizeof(double) * LV_MAX_VIEWS, w.lsum, sizeof(double) * LV_MAX_VIEWS);
  k_lf_sobel<<<(unsigned)((P + TPB - 1) / TPB), TPB, 0, s>>>(gt, vp, w.grp, w.mkey);
  k_lf_queries<<<1, LV_MAX_VIEWS, 0, s>>>(w.q, vp);
  select_kth(w.mkey, w.grp, P, w.q, n_views, w.sel_tmp, s);
  for (int v = 0; v < n_views; ++v) {
    const long long np = vp.off[v + 1] - vp.off[v];
    k_lf_weight<<<blocks_for(np), TPB, 0, s>>>(w.mkey, w.q, vp, v, p->eps, gamma, w.w, w.wsum, p->edge_out);
  }
  count_launch(2 + n_views);
  return cuda_check(cudaGetLastError(), "lv_lf_weights");
}

extern "C" lv_status lv_lf_loss_from_weights(const float* rgb, const float* gt, const int32_t* widths,
                                             const int32_t* heights, int n_views, float* loss, float* dL_drgb,
                                             void* workspace, size_t ws_bytes, void* stream) {
  if (!rgb || !gt || !loss) { set_error("null argument"); return LV_ERR_INVALID_ARG; }
  ViewPix vp;
  LfWs w;
  lv_status e = lf_setup(widths, heights, n_views, 990000, workspace, ws_bytes, &vp, &w);
  if (e != LV_OK) return e;
  cudaStream_t s = (cudaStream_t)stream;
  zero_async(s, w.lsum, sizeof(double) * LV_MAX_VIEWS);
  // four pixels (three 16-byte words of rgb, gt and dL_drgb) per step where the buffers allow it
  const bool vec = aligned16(rgb) && aligned16(gt) && aligned16(w.w) && (!dL_drgb || aligned16(dL_drgb));
  for (int v = 0; v < n_views; ++v) {
    const long long np = vp.off[v + 1] - vp.off[v];
    if (vec) k_lf_loss4<<<blocks_for(np), TPB, 0, s>>>(rgb, gt, w.w, vp, v, w.wsum, w.lsum, dL_drgb);
    else k_lf_loss<<<blocks_for(np), TPB, 0, s>>>(rgb, gt, w.w, vp, v, w.wsum, w.lsum, dL_drgb);
  }
  k_lf_finish<<<1, LV_MAX_VIEWS, 0, s>>>(vp, w.lsum, loss, false);
  count_launch(1 + n_views);
  return cuda_check(cudaGetLastError(), "lv_lf_loss_from_weights");
}

extern "C" lv_status lv_lf_loss_finish(const int32_t* widths, const int32_t* heights, int n_views, float* loss,
                                       void* workspace, size_t ws_bytes, void* stream) {
  if (!loss) { set_error("null argument"); return LV_ERR_INVALID_ARG; }
  ViewPix vp;
  LfWs w;
  lv_status e = lf_setup(widths, heights, n_views, 990000, workspace, ws_bytes, &vp, &w);
  if (e != LV_OK) return e;
  k_lf_finish<<<1, LV_MAX_VIEWS, 0, (cudaStream_t)stream>>>(vp, w.lsum, loss, true);
  count_launch(1);
  return cuda_check(cudaGetLastError(), "lv_lf_loss_finish");
}

namespace lv {
lv_status lf_fused_buffers(const int32_t* widths, const int32_t* heights, int n_views, void* workspace,
                           size_t ws_bytes, const float** w_out, const double** wsum, double** lsum) {
  ViewPix vp;
  LfWs w;
  lv_status e = lf_setup(widths, heights, n_views, 990000, workspace, ws_bytes, &vp, &w);
  if (e != LV_OK) return e;
  *w_out = w.w;
  *wsum = w.wsum;
  *lsum = w.lsum;
  return LV_OK;
}
}  // namespace lv

extern "C" lv_status lv_lf_weighted_loss(const float* rgb, const float* gt, const int32_t* widths,
                                         const int32_t* heights, int n_views, float t, const lv_lf_params* p,
                                         float* loss, float* dL_drgb, void* workspace, size_t ws_bytes,
                                         void* stream) {
  if (!rgb || !gt || !p || !loss) { set_error("null argument"); return LV_ERR_INVALID_ARG; }
  lv_status e = lv_lf_weights(gt, widths, heights, n_views, t, p, workspace, ws_bytes, stream);
  if (e != LV_OK) return e;
  return lv_lf_loss_from_weights(rgb, gt, widths, heights, n_views, loss, dL_drgb, workspace, ws_bytes, stream);
}

// ---------------------------------------------------------------- allocation-free variant
// For callers that cannot allocate device memory themselves: the scratch that
// lv_lf_weighted_loss takes from a caller workspace comes from this fixed
// array instead.  Every device that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_lf_scratch[LV_LF_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_lf_scratch_mu;
void* g_lf_scratch_ptr[256] = {};  // device address of g_lf_scratch per device ordinal

// The array's name is a host-side stand-in in host code; its device address is
// looked up once per device, with that device current.
lv_status lf_scratch_address(void** out) {
  int dev = 0;
  lv_status e = cuda_check(cudaGetDevice(&dev), "lv_lf_weighted_loss_noalloc: cudaGetDevice");
  if (e != LV_OK) return e;
  if (dev < 0 || dev >= 256) { set_error("lv_lf_weighted_loss_noalloc: device ordinal %d unsupported", dev); return LV_ERR_UNSUPPORTED; }
  std::lock_guard<std::mutex> lock(g_lf_scratch_mu);
  if (!g_lf_scratch_ptr[dev]) {
    void* ptr = nullptr;
    e = cuda_check(cudaGetSymbolAddress(&ptr, g_lf_scratch), "lv_lf_weighted_loss_noalloc: cudaGetSymbolAddress");
    if (e != LV_OK) return e;
    g_lf_scratch_ptr[dev] = ptr;
  }
  *out = g_lf_scratch_ptr[dev];
  return LV_OK;
}
}  // namespace

extern "C" lv_status lv_lf_weighted_loss_noalloc(const float* rgb, const float* gt, const int32_t* widths,
                                                 const int32_t* heights, int n_views, float t, const lv_lf_params* p,
                                                 float* loss, float* dL_drgb, void* stream) {
  const size_t need = lv_lf_workspace_size(widths, heights, n_views);
  if (need == 0) { set_error("lv_lf_weighted_loss_noalloc: bad view sizes"); return LV_ERR_INVALID_ARG; }
  if (need > sizeof(g_lf_scratch)) {
    set_error("lv_lf_weighted_loss_noalloc: these views need %zu bytes of scratch, the fixed array holds %zu "
              "(about 1.6 million pixels); use lv_lf_weighted_loss with a workspace instead",
              need, sizeof(g_lf_scratch));
    return LV_ERR_INVALID_ARG;
  }
  void* scratch = nullptr;
  lv_status e = lf_scratch_address(&scratch);
  if (e != LV_OK) return e;
  // lv_lf_weighted_loss clears its accumulators and selection histograms in the
  // scratch at the start of every call, so nothing else has to be zeroed here.
  return lv_lf_weighted_loss(rgb, gt, widths, heights, n_views, t, p, loss, dL_drgb, scratch, sizeof(g_lf_scratch),
                             stream);
}

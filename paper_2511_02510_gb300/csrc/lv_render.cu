// lv_render.cu -- forward / backward passes of the sparse-voxel tile
// rasterizer (LiteVoxel Sec. III, Eq. 1-5) for sm_103a.
//
// Pipeline of lv_rasterize_forward (one stream, no host synchronisation):
//   k_bin       per (voxel, view): FP32 cull / near-plane clipping / corner
//               projection / tile rect / depth key with a fixed operation
//               order; depth statistics.
//   scan2       visible-slot ids and each item's first pair (item order),
//               with the slot and pair totals.
//   k_emit      per (voxel, view): the item's (tile, slot) pairs, written in
//               item order by whole warps; per visible item the 64-byte render
//               record (centre relative to the camera, half-size, 8 corner
//               densities, SH colour, 1 / (2 h)), its pixel box, voxel id and
//               depth key.
//   radix sort  the pairs by tile id (stable: each tile's list stays in
//               voxel-id order); its last pass also notes every tile's range.
//   k_tile_sort_warp, k_tile_sort, k_tile_merge  per tile: its slots sorted by depth key in
//               shared memory (stable), so every tile's list ends front to back
//               with ties by voxel id.  The depth keys are sorted per tile,
//               where they fit in shared memory, instead of by global passes
//               over all slots.
//   k_fwd       per tile, one thread per pixel: each warp stages the records
//               that meet its pixel strip through shared memory and marches
//               front to back (Eq. 2-4); w_max (Eq. 5) is reduced over the
//               warp before one global atomicMax; a warp stops when all its
//               pixels have T < t_stop.
// lv_rasterize_backward walks the same lists back to front (k_bwd) and
// reduces the SH colour gradient per voxel (k_sh_bwd).
#include <math.h>
#include <stdio.h>

#include "lv_prims.cuh"

namespace lv {

// ------------------------------------------------------------------ views
struct DevView {
  float R[9];  // w2c rotation, row-major
  float t[3];
  float o[3];  // camera centre in world coordinates
  float fx, fy, cx, cy, z_near;
  int W, H, tiles_x, tiles_y;
  int tile_off;       // first global tile of the view
  long long pix_off;  // first global pixel of the view
  // k_bin's early-out planes: the frustum of the tile grid widened by 2 pixels has side planes
  // f u - m z = 0 (u the camera x or y coordinate) with m = cx + 2, cx - tiles_x ts - 2,
  // cy + 2, cy - tiles_y ts - 2 (cull_m), and |(f, m)| rounded up (cull_n)
  float cull_m[4], cull_n[4];
};
struct ViewSet {
  int n;
  int ts;
  long long id_base;  // global id of the call's first pixel (w_max argmax ids)
  DevView v[LV_MAX_VIEWS];
};

static void make_views(const lv_camera* cams, int nv, int ts, ViewSet* vs, int64_t* tiles, int64_t* pixels) {
  vs->n = nv;
  vs->ts = ts;
  vs->id_base = 0;
  int64_t to = 0, po = 0;
  for (int i = 0; i < nv; ++i) {
    const lv_camera& c = cams[i];
    DevView& d = vs->v[i];
    for (int r = 0; r < 3; ++r) {
      for (int k = 0; k < 3; ++k) d.R[r * 3 + k] = c.w2c[r * 4 + k];
      d.t[r] = c.w2c[r * 4 + 3];
    }
    for (int k = 0; k < 3; ++k) {
      double s = 0;
      for (int r = 0; r < 3; ++r) s += (double)c.w2c[r * 4 + k] * (double)c.w2c[r * 4 + 3];
      d.o[k] = (float)(-s);
    }
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy; d.z_near = c.z_near;
    d.W = c.width; d.H = c.height;
    d.tiles_x = (c.width + ts - 1) / ts;
    d.tiles_y = (c.height + ts - 1) / ts;
    d.tile_off = (int)to;
    d.pix_off = po;
    d.cull_m[0] = d.cx + 2.f;
    d.cull_m[1] = d.cx - (float)(d.tiles_x * ts) - 2.f;
    d.cull_m[2] = d.cy + 2.f;
    d.cull_m[3] = d.cy - (float)(d.tiles_y * ts) - 2.f;
    for (int k = 0; k < 4; ++k) {
      const double f = k < 2 ? (double)d.fx : (double)d.fy, m = (double)d.cull_m[k];
      d.cull_n[k] = nextafterf((float)sqrt(f * f + m * m), INFINITY);  // at least the exact norm
    }
    to += (int64_t)d.tiles_x * d.tiles_y;
    po += (int64_t)c.width * c.height;
  }
  *tiles = to;
  *pixels = po;
}

// ------------------------------------------------------------------ workspace
// items are (view, voxel) pairs in view-major order: item = view * n + voxel
struct FwdWs {
  unsigned long long* counters;  // [0] pairs, [1] slots
  uint32_t* cnt;                 // [items] tiles covered
  uint32_t* vis;                 // [items] 1 if cnt > 0
  uint2* rect;                   // [items] (tx0 | tx1 << 16, ty0 | ty1 << 16)
  uint2* pbox;                   // [items] conservative pixel box (x0 | x1 << 16, y0 | y1 << 16), [x0, x1)
  uint32_t* dkey;                // [items] order key of z_centre
  uint32_t* slot;                // [items] render slot of a visible item
  unsigned long long* poff;      // [items] first pair of the item (pairs in item order)
  uint2* rec_bb;                 // [slots] pixel box of the render record
  uint32_t* slot_vox;            // [slots] voxel id of the render record
  uint32_t* s_dkey;              // [slots] order key
  unsigned int* work;            // [16] work-item counters: [0..1] the persistent composites, [2] count
                                 // of the long tiles' chunks, [3] the merge's work counter, [4..5] count
                                 // of the medium tiles and k_tile_sort's work counter, [6] count of the
                                 // long tiles; [8..9] block arrivals of the persistent forward and
                                 // backward composites (sm_leave)
  uint2* chunks;                 // [pair capacity / TS_CHUNK + tiles] (tile, chunk) of the long tiles
  uint32_t* mid_tiles;           // [tiles] tiles of medium-length lists
  uint32_t* long_tiles;          // [tiles] tiles of long lists
  void* scan_tmp;
  float4* rec;                   // [slots][4]
  float4* d_rgb;                 // [slots] colour gradient (xyz) scratch of the backward; w = clamp mask
  uint32_t* ranges;              // [tiles][2]
  float* tau;                    // [pixels] final optical depth
  void* sort_tmp;                // scratch of the sort by tile
  int32_t* status;               // fallback status word
  uint32_t *k0, *v0, *k1, *v1;   // [pair capacity] (tile, slot) pairs, sorted by tile
  size_t bytes;
};

static FwdWs carve_fwd(void* base, int64_t n, int nv, int64_t tiles, int64_t pixels, int64_t pair_cap) {
  FwdWs w;
  Carve c(base);
  int64_t items = n * nv;
  w.counters = c.take<unsigned long long>(8);
  w.status = c.take<int32_t>(4);
  w.work = c.take<unsigned int>(16);
  w.cnt = c.take<uint32_t>(items);
  w.vis = c.take<uint32_t>(items);
  w.rect = c.take<uint2>(items);
  w.pbox = c.take<uint2>(items);
  w.dkey = c.take<uint32_t>(items);
  w.slot = c.take<uint32_t>(items);
  w.poff = c.take<unsigned long long>(items);
  w.rec_bb = c.take<uint2>(items);
  w.slot_vox = c.take<uint32_t>(items);
  w.s_dkey = c.take<uint32_t>(items);
  w.scan_tmp = c.take<char>(scan2_tmp_bytes());
  w.rec = c.take<float4>(items * 4);
  w.d_rgb = c.take<float4>(items);
  w.ranges = c.take<uint32_t>(tiles * 2);
  w.chunks = c.take<uint2>(pair_cap / 4096 + tiles);
  w.mid_tiles = c.take<uint32_t>(tiles);
  w.long_tiles = c.take<uint32_t>(tiles);
  w.tau = c.take<float>(pixels);
  w.sort_tmp = c.take<char>(sort_tmp_bytes(pair_cap));
  w.k0 = c.take<uint32_t>(pair_cap);
  w.v0 = c.take<uint32_t>(pair_cap);
  w.k1 = c.take<uint32_t>(pair_cap);
  w.v1 = c.take<uint32_t>(pair_cap);
  w.bytes = c.off + 256;
  return w;
}

// the sorted (tile, slot) pairs: in (k0, v0) after an even number of tile-digit passes
static int tile_bits(int64_t tiles) {
  int b = 0;
  while (b < 32 && ((int64_t)1 << b) < tiles) ++b;
  return b;
}
static const uint32_t* sorted_pair_slots(const FwdWs& w, int64_t tiles) {
  return (sort_passes(tile_bits(tiles)) & 1) ? w.v1 : w.v0;
}
static const uint32_t* sorted_pair_tiles(const FwdWs& w, int64_t tiles) {
  return (sort_passes(tile_bits(tiles)) & 1) ? w.k1 : w.k0;
}
static void launch_tile_sort(const FwdWs& w, int64_t tiles, int64_t pair_cap, cudaStream_t s);


// ------------------------------------------------------------------ binning (FP32, fixed op order)
__device__ __forceinline__ void cam_point32(const DevView& c, float X, float Y, float Z, float* q) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float a = __fmul_rn(c.R[r * 3 + 0], X);
    float b = __fmul_rn(c.R[r * 3 + 1], Y);
    float e = __fmul_rn(c.R[r * 3 + 2], Z);
    float s = __fadd_rn(a, b);
    s = __fadd_rn(s, e);
    q[r] = __fadd_rn(s, c.t[r]);
  }
}

__global__ void __launch_bounds__(256) k_bin(const float4* __restrict__ geom, int64_t n,
                                             const __grid_constant__ ViewSet vs, uint32_t* cnt, uint32_t* vis,
                                             uint2* rect, uint2* pbox, uint32_t* dkey, float* z_min,
                                             float* delta_min, uint8_t* seen) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n * vs.n) return;
  // items are view-major (i = view * n + voxel): a warp's lanes share one view, so the camera
  // fields are warp-uniform loads, and the statistics' atomics hit distinct voxels
  const int view = (int)(i / n);
  const int64_t vox = i - (int64_t)view * n;
  const DevView& c = vs.v[view];
  const int ts = vs.ts;
  float4 g = geom[vox];
  float qc[3];
  cam_point32(c, g.x, g.y, g.z, qc);
  dkey[i] = order_key(qc[2]);
  {
    // Early out for voxels far outside the view: the circumscribed sphere lies behind the near
    // plane or beyond a side plane of the frustum of the tile grid (which may reach past the image
    // edge) widened by 2 pixels, with a relative slack far above FP32 rounding.  Such a voxel's
    // exact tile rectangle below (1-pixel margin, clamped to the tile grid) is empty, so skipping it
    // changes no output.
    const float r = g.w * 1.7320508f;
    const float rs = r + 1e-4f * (fabsf(qc[0]) + fabsf(qc[1]) + fabsf(qc[2]) + r) + 1e-6f;
    // (the planes and their norms are per view, set up on the host)
    const bool out = qc[2] + rs < c.z_near ||
                     c.fx * qc[0] + c.cull_m[0] * qc[2] < -rs * c.cull_n[0] ||
                     c.fx * qc[0] + c.cull_m[1] * qc[2] > rs * c.cull_n[1] ||
                     c.fy * qc[1] + c.cull_m[2] * qc[2] < -rs * c.cull_n[2] ||
                     c.fy * qc[1] + c.cull_m[3] * qc[2] > rs * c.cull_n[3];
    if (out) {
      cnt[i] = 0u;
      vis[i] = 0u;
      rect[i] = make_uint2(0u, 0u);
      pbox[i] = make_uint2(0u, 0u);
      return;
    }
  }
  int n_front = 0;
  float umin = 0.f, umax = 0.f, vmin = 0.f, vmax = 0.f;
  bool first = true;
  float px[8], py[8], pz[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float X = (k & 1) ? __fadd_rn(g.x, g.w) : __fsub_rn(g.x, g.w);
    float Y = (k & 2) ? __fadd_rn(g.y, g.w) : __fsub_rn(g.y, g.w);
    float Z = (k & 4) ? __fadd_rn(g.z, g.w) : __fsub_rn(g.z, g.w);
    float p[3];
    cam_point32(c, X, Y, Z, p);
    px[k] = p[0]; py[k] = p[1]; pz[k] = p[2];
    if (p[2] >= c.z_near) {
      ++n_front;
      const float iz = __frcp_rn(p[2]);  // one correctly rounded reciprocal per corner
      float u = __fadd_rn(__fmul_rn(c.fx, __fmul_rn(p[0], iz)), c.cx);
      float v = __fadd_rn(__fmul_rn(c.fy, __fmul_rn(p[1], iz)), c.cy);
      if (first) { umin = umax = u; vmin = vmax = v; first = false; }
      else { umin = fminf(umin, u); umax = fmaxf(umax, u); vmin = fminf(vmin, v); vmax = fmaxf(vmax, v); }
    }
  }
  int tx0 = 0, tx1 = 0, ty0 = 0, ty1 = 0;
  int px0 = 0, px1 = 0, py0 = 0, py1 = 0;  // pixels x in [px0, px1) may be hit (their centres lie in the box)
  if (n_front > 0) {
    if (n_front < 8) {
      // near-plane clipping: crossing points of the box edges (k, k|bit) with z = z_near
#pragma unroll
      for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int bit = 1; bit < 8; bit <<= 1) {
          if (k & bit) continue;
          const int j = k | bit;
          if ((pz[k] >= c.z_near) == (pz[j] >= c.z_near)) continue;
          const float f = __fdiv_rn(__fsub_rn(c.z_near, pz[k]), __fsub_rn(pz[j], pz[k]));
          const float x = __fadd_rn(px[k], __fmul_rn(f, __fsub_rn(px[j], px[k])));
          const float y = __fadd_rn(py[k], __fmul_rn(f, __fsub_rn(py[j], py[k])));
          const float u = __fadd_rn(__fmul_rn(c.fx, __fdiv_rn(x, c.z_near)), c.cx);
          const float v = __fadd_rn(__fmul_rn(c.fy, __fdiv_rn(y, c.z_near)), c.cy);
          umin = fminf(umin, u); umax = fmaxf(umax, u); vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
        }
      }
    }
    // ts is a power of two, so multiplying by 1/ts rounds exactly as dividing by ts
    const float its = 1.0f / (float)ts;
    const float a0 = floorf(__fmul_rn(__fsub_rn(umin, 1.0f), its));
    const float a1 = ceilf(__fmul_rn(__fadd_rn(umax, 1.0f), its));
    const float b0 = floorf(__fmul_rn(__fsub_rn(vmin, 1.0f), its));
    const float b1 = ceilf(__fmul_rn(__fadd_rn(vmax, 1.0f), its));
    tx0 = (int)fminf(fmaxf(a0, 0.0f), (float)c.tiles_x);
    tx1 = (int)fminf(fmaxf(a1, 0.0f), (float)c.tiles_x);
    ty0 = (int)fminf(fmaxf(b0, 0.0f), (float)c.tiles_y);
    ty1 = (int)fminf(fmaxf(b1, 0.0f), (float)c.tiles_y);
    // The composites only cull with the pixel box: a ray through the centre (x + 1/2, y + 1/2) of
    // pixel (x, y) meets the box only if that centre lies in the footprint's bounding box
    // [umin, umax] x [vmin, vmax].  The FP32 projection and the FP32 ray of the chord test are
    // each within about 1e-3 pixel of exact, so widening the box by 1/16 pixel plus 2^-14 of the
    // coordinate keeps every pixel an FP32 chord test can hit; the tile rectangle above keeps its
    // 1-pixel margin.
    const float eu = fmaf(6.1035156e-5f, fmaxf(fabsf(umin), fabsf(umax)), 0.0625f);
    const float ev = fmaf(6.1035156e-5f, fmaxf(fabsf(vmin), fabsf(vmax)), 0.0625f);
    px0 = (int)fminf(fmaxf(ceilf(umin - eu - 0.5f), 0.0f), (float)c.W);
    px1 = (int)fminf(fmaxf(floorf(umax + eu - 0.5f) + 1.0f, (float)px0), (float)c.W);
    py0 = (int)fminf(fmaxf(ceilf(vmin - ev - 0.5f), 0.0f), (float)c.H);
    py1 = (int)fminf(fmaxf(floorf(vmax + ev - 0.5f) + 1.0f, (float)py0), (float)c.H);
  }
  uint32_t count = (tx1 > tx0 && ty1 > ty0) ? (uint32_t)(tx1 - tx0) * (uint32_t)(ty1 - ty0) : 0u;
  cnt[i] = count;
  vis[i] = count ? 1u : 0u;
  rect[i] = make_uint2((uint32_t)tx0 | ((uint32_t)tx1 << 16), (uint32_t)ty0 | ((uint32_t)ty1 << 16));
  pbox[i] = make_uint2((uint32_t)px0 | ((uint32_t)px1 << 16), (uint32_t)py0 | ((uint32_t)py1 << 16));
  if (count) {
    float zs = fmaxf(qc[2], c.z_near);
    float dl = __fdiv_rn(zs, c.fx);
    if (z_min) atomicMin((unsigned int*)&z_min[vox], __float_as_uint(zs));
    if (delta_min) atomicMin((unsigned int*)&delta_min[vox], __float_as_uint(dl));
    if (seen) seen[vox] = 1;
  }
}

// ------------------------------------------------------------------ SH (real, degree <= 3)
// Orthonormal real spherical harmonics written from the associated Legendre
// functions: Y0 = 1/(2 sqrt(pi)); l=1 sqrt(3/4pi) {y, z, x}; l=2 sqrt(15/4pi)
// {xy, yz, xz}, sqrt(5/16pi)(3z^2-1), sqrt(15/16pi)(x^2-y^2); l=3
// sqrt(35/32pi) y(3x^2-y^2), sqrt(105/4pi) xyz, sqrt(21/32pi) y(5z^2-1),
// sqrt(7/16pi) z(5z^2-3), sqrt(21/32pi) x(5z^2-1), sqrt(105/16pi) z(x^2-y^2),
// sqrt(35/32pi) x(x^2-3y^2).
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
  const float C0 = 0.28209479177387814f;
  const float C1 = 0.48860251190291992f;
  const float C2a = 1.0925484305920792f, C2b = 0.31539156525252005f, C2c = 0.54627421529603959f;
  const float C3a = 0.59004358992664352f, C3b = 2.8906114426405538f, C3c = 0.45704579946446572f;
  const float C3d = 0.37317633259011540f, C3e = 1.4453057213202769f;
  float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = C0;
  Y[1] = C1 * y;
  Y[2] = C1 * z;
  Y[3] = C1 * x;
  Y[4] = C2a * x * y;
  Y[5] = C2a * y * z;
  Y[6] = C2b * (3.f * zz - 1.f);
  Y[7] = C2a * x * z;
  Y[8] = C2c * (xx - yy);
  Y[9] = C3a * y * (3.f * xx - yy);
  Y[10] = C3b * x * y * z;
  Y[11] = C3c * y * (5.f * zz - 1.f);
  Y[12] = C3d * z * (5.f * zz - 3.f);
  Y[13] = C3c * x * (5.f * zz - 1.f);
  Y[14] = C3e * z * (xx - yy);
  Y[15] = C3a * x * (xx - 3.f * yy);
}

// one voxel's 48 SH coefficients into registers with 16-byte loads
__device__ __forceinline__ void load_sh_row(const float* __restrict__ row, float* c) {
  const float4* v = (const float4*)row;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float4 q = __ldg(v + k);
    c[4 * k] = q.x; c[4 * k + 1] = q.y; c[4 * k + 2] = q.z; c[4 * k + 3] = q.w;
  }
}
__device__ __forceinline__ void load_sh_row(const __nv_bfloat16* __restrict__ row, float* c) {
  const uint4* v = (const uint4*)row;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const uint4 q = __ldg(v + k);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      c[8 * k + 2 * h] = __uint_as_float(w[h] << 16);
      c[8 * k + 2 * h + 1] = __uint_as_float(w[h] & 0xffff0000u);
    }
  }
}

// c = max(0, raw) with raw = sum_j coef[j] Y_j + 0.5 per channel; coef laid out [j][rgb] with stride cs
__device__ __forceinline__ void sh_raw(const float* coef, int cs, int nb, const float* Y, float* raw) {
  float r = 0.f, g = 0.f, b = 0.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j < nb) {
      r = fmaf(coef[(3 * j + 0) * cs], Y[j], r);
      g = fmaf(coef[(3 * j + 1) * cs], Y[j], g);
      b = fmaf(coef[(3 * j + 2) * cs], Y[j], b);
    }
  }
  raw[0] = r + 0.5f;
  raw[1] = g + 0.5f;
  raw[2] = b + 0.5f;
}

__device__ __forceinline__ void unit_dir(float rx, float ry, float rz, float* d) {
  float nn = rx * rx + ry * ry + rz * rz;
  if (nn > 0.f) {
    float inv = rsqrtf(nn);
    d[0] = rx * inv; d[1] = ry * inv; d[2] = rz * inv;
  } else {
    d[0] = 0.f; d[1] = 0.f; d[2] = 1.f;
  }
}

// ------------------------------------------------------------------ emit
// One thread per (voxel, view) item.  First the warp writes the (tile, slot)
// pairs of its 32 items: items are consecutive, so their pairs form one
// contiguous range in item order (view-major, voxel id within a view), which
// the warp fills 32 pairs per step, each lane finding the item of its pair by
// a 5-step search over the lanes' first pairs.  More pairs than capacity:
// none are written and the status word says LV_ERR_CAPACITY.  Then each
// visible item writes the render record of its slot (camera-relative centre
// and h | 8 corner densities | clamped SH colour and 1/(2h)), the slot's order
// key, and the colour-gradient scratch (cleared; w = clamp mask).
template <typename DT, typename ST>
__global__ void __launch_bounds__(256) k_emit(const float4* __restrict__ geom, const DT* __restrict__ dens,
                                              const ST* __restrict__ sh, int sh_nb, int64_t n,
                                              const __grid_constant__ ViewSet vs, const uint32_t* __restrict__ cnt,
                                              const uint2* __restrict__ rect,
                                              const uint2* __restrict__ pbox, uint2* __restrict__ rec_bb,
                                              uint32_t* __restrict__ slot_vox,
                                              const uint32_t* __restrict__ dkey,
                                              const uint32_t* __restrict__ slot,
                                              const unsigned long long* __restrict__ poff,
                                              const unsigned long long* __restrict__ counters, int64_t pair_cap,
                                              uint32_t* __restrict__ pair_tile, uint32_t* __restrict__ pair_slot,
                                              int32_t* status, uint2* __restrict__ ranges, int64_t tiles,
                                              const SortCountTargets sc, int passes,
                                              float4* __restrict__ rec,
                                              float4* __restrict__ d_rgb, uint32_t* __restrict__ s_dkey,
                                              const uint32_t* __restrict__ vidx) {
  // Block b covers 256 consecutive voxels of view b % views, so the blocks of
  // all views of one voxel range run side by side: a voxel's SH row comes
  // from HBM once and from L2 for its other views.  Items are view-major
  // (i = view * n + voxel), so each block still writes consecutive slots.
  const int view = (int)(blockIdx.x % (unsigned)vs.n);
  const int64_t vox = (int64_t)(blockIdx.x / (unsigned)vs.n) * 256 + threadIdx.x;
  const int64_t i = (int64_t)view * n + vox;
  const bool in = vox < n;
  // the sort by tile's last pass reduces every tile's [first, end) into ranges
  for (int64_t x = blockIdx.x * 256ll + threadIdx.x; x < tiles; x += (int64_t)gridDim.x * 256)
    ranges[x] = make_uint2(~0u, 0u);
  const uint32_t cn = in ? cnt[i] : 0u;  // nonzero exactly for the visible items
  const unsigned long long total = counters[0];
  // the sort by tile's digit counts (every pass) are counted here, and its first look-back words cleared
  __shared__ uint32_t s_cnt[4 * 256];
  for (int x = threadIdx.x; x < passes * 256; x += 256) s_cnt[x] = 0u;
  if (total <= (unsigned long long)pair_cap) {
    const int64_t words = (int64_t)((total + sc.tile - 1) / sc.tile) * 256;
    for (int64_t x = blockIdx.x * 256ll + threadIdx.x; x < words; x += (int64_t)gridDim.x * 256) sc.look0[x] = 0ull;
  }
  __syncthreads();
  if (total > (unsigned long long)pair_cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) report(status, LV_ERR_CAPACITY);
  } else {
    const int lane = threadIdx.x & 31;
    const uint32_t inm = __ballot_sync(FULL, in);  // a prefix of the lanes
    if (inm) {                                     // warp-uniform
      const int last = 31 - __clz(inm);
      // lanes past the last voxel start after every pair, so the search never picks them
      const unsigned long long po = in ? poff[i] : ~0ull;
      uint32_t rx = 0u, ry = 0u, sl = 0u;
      if (cn) {
        const uint2 rc = rect[i];
        rx = rc.x;
        ry = rc.y;
        sl = slot[i];
      }
      const unsigned long long p_begin = __shfl_sync(FULL, po, 0);
      const unsigned long long p_end = __shfl_sync(FULL, po + cn, last);
      const DevView& c = vs.v[view];
      const uint32_t toff = (uint32_t)c.tile_off, tiles_x = (uint32_t)c.tiles_x;
      for (unsigned long long p0 = p_begin; p0 < p_end; p0 += 32) {  // warp-uniform
        const unsigned long long e = p0 + lane;
        int j = 0;  // the largest lane whose first pair is <= e (lane 0's is <= p0)
#pragma unroll
        for (int step = 16; step; step >>= 1) {
          const unsigned long long x = __shfl_sync(FULL, po, (j + step) & 31);
          if (j + step < 32 && x <= e) j += step;
        }
        const unsigned long long pj = __shfl_sync(FULL, po, j);
        const uint32_t jx = __shfl_sync(FULL, rx, j), jy = __shfl_sync(FULL, ry, j);
        const uint32_t js = __shfl_sync(FULL, sl, j);
        if (e < p_end) {
          const uint32_t q = (uint32_t)(e - pj);
          const uint32_t tx0 = jx & 0xffffu, wx = (jx >> 16) - tx0, ty0 = jy & 0xffffu;
          const uint32_t key = toff + (ty0 + q / wx) * tiles_x + tx0 + q % wx;
          pair_tile[e] = key;
          pair_slot[e] = js;
          for (int p = 0; p < passes; ++p) atomicAdd(&s_cnt[p * 256 + ((key >> (8 * p)) & 255u)], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < passes * 256; x += 256)
    if (s_cnt[x]) atomicAdd(&sc.counts[x], s_cnt[x]);
  if (!cn) return;
  const DevView& c = vs.v[view];
  const uint32_t s = slot[i];
  const float4 g = geom[vox];
  const float rx = g.x - c.o[0], ry = g.y - c.o[1], rz = g.z - c.o[2];
  float dir[3];
  unit_dir(rx, ry, rz, dir);
  float Y[16];
  sh_basis(dir[0], dir[1], dir[2], Y);
  float coef[48];
  load_sh_row(sh + 48 * vox, coef);
  float raw[3];
  sh_raw(coef, 1, sh_nb, Y, raw);
  float d[8];
  if (vidx) {  // shared grid-vertex densities
    const uint4 i0 = *(const uint4*)(vidx + 8 * vox), i1 = *(const uint4*)(vidx + 8 * vox + 4);
    d[0] = to_f32(dens[i0.x]); d[1] = to_f32(dens[i0.y]); d[2] = to_f32(dens[i0.z]); d[3] = to_f32(dens[i0.w]);
    d[4] = to_f32(dens[i1.x]); d[5] = to_f32(dens[i1.y]); d[6] = to_f32(dens[i1.z]); d[7] = to_f32(dens[i1.w]);
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) d[k] = to_f32(dens[8 * vox + k]);
  }
  float4* r = rec + 4 * (int64_t)s;
  r[0] = make_float4(rx, ry, rz, g.w);
  r[1] = make_float4(d[0], d[1], d[2], d[3]);
  r[2] = make_float4(d[4], d[5], d[6], d[7]);
  r[3] = make_float4(fmaxf(raw[0], 0.f), fmaxf(raw[1], 0.f), fmaxf(raw[2], 0.f), __fdiv_rn(0.5f, g.w));
  slot_vox[s] = (uint32_t)vox;
  // colour-gradient scratch: xyz cleared, w = which channels passed the clamp
  // (bit c set when raw_c > 0) as a small exact float, read by the SH backward
  d_rgb[s] = make_float4(0.f, 0.f, 0.f,
                         (float)((raw[0] > 0.f ? 1 : 0) | (raw[1] > 0.f ? 2 : 0) | (raw[2] > 0.f ? 4 : 0)));
  rec_bb[s] = pbox[i];
  s_dkey[s] = dkey[i];
}

// pairs usable by the later stages: all of them, or none after an overflow
__device__ __forceinline__ int64_t usable_pairs(const unsigned long long* d_count, int64_t cap) {
  unsigned long long c = *d_count;
  return c <= (unsigned long long)cap ? (int64_t)c : 0;
}

// ------------------------------------------------------------------ per-tile depth order
// After the stable sort by tile id, each tile's pairs are in item order (voxel
// id within a view), and the sort's last pass has left every tile's range in
// ranges (empty tiles: (0xffffffff, 0)).  Each tile's slots are then sorted by
// order key: an LSD radix sort of 9-bit digits of the key minus the tile's
// smallest key (a tile whose keys span less than 2^27 takes 3 passes).  Each
// pass ranks stably (warp-private digit counts; the lanes holding a digit
// found by bit ballots or by __match_any_sync), so equal keys keep item order,
// and each tile's list ends front to back with ties by voxel id: the order one
// stable sort of (tile, order key) pairs in voxel-id order gives.  The tiles
// are shared out by list length:
//   k_tile_sort_warp  one warp per tile: lists of up to TW_MAX pairs; it also
//                     writes every tile's range in final form (empty: (0, 0))
//                     and lists the longer tiles;
//   k_tile_sort       persistent blocks of 512 threads: lists of up to
//                     TS_CHUNK pairs in place, and longer lists cut into
//                     chunks of TS_CHUNK pairs, each sorted into a scratch
//                     copy of the pair arrays;
//   k_tile_merge      persistent blocks over the long tiles: the sorted chunks
//                     merged stably (equal keys of earlier chunks first).
constexpr int TS_BITS = 9, TS_BINS = 1 << TS_BITS;
constexpr int TS_THREADS = 512, TS_WARPS = TS_THREADS / 32, TS_ITEMS = 8, TS_CHUNK = TS_THREADS * TS_ITEMS;
constexpr int TW_MAX = 256, TW_ITEMS = TW_MAX / 32, TW_WARPS = 16;
static_assert(TS_THREADS == TS_BINS, "a thread for each digit");

struct TileSortSmem {
  uint32_t k[TS_CHUNK];                // keys
  uint32_t v[TS_CHUNK];                // slots
  uint16_t wc[TS_WARPS][TS_BINS + 2];  // warp digit counts -> warp prefixes (bin TS_BINS: padding)
  uint32_t base[TS_BINS];              // start of each digit
  uint32_t w[TS_WARPS];
  uint32_t item, kmin, kmax;
};
struct WarpSortSmem {
  uint32_t k[2][TW_MAX];     // keys, ping-pong
  uint32_t v[2][TW_MAX];     // slots, ping-pong
  uint16_t wc[TS_BINS + 2];  // digit counts (bin TS_BINS: padding)
  uint16_t base[TS_BINS];    // start of each digit
};
struct TileSortWarpSmem {
  WarpSortSmem w[TW_WARPS];
};
struct TileMergeSmem {
  uint32_t k[2][2 * TS_CHUNK];  // two runs side by side, then the first merge's output
  uint32_t v[2][2 * TS_CHUNK];
  uint32_t item;
};

// exclusive scan of one value per thread over a block of WARPS warps
template <int WARPS>
__device__ __forceinline__ uint32_t ts_block_excl(uint32_t c, uint32_t* s_w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  uint32_t pre = 0;
#pragma unroll
  for (int w = 0; w < WARPS; ++w) pre += w < warp ? s_w[w] : 0u;
  return pre + x - c;
}

// Stable ranks of R rounds held warp-striped (round j of a warp holds item
// 32 j + lane of the warp's items).  dr[j] holds the digit (TS_BINS for
// padding) on entry; on exit also the item's rank among the warp's items of
// its digit, from bit 10 up.  The warp's counts per digit accumulate in wc.
template <int ITEMS>
__device__ __forceinline__ void ts_rank(uint32_t (&dr)[ITEMS], int R, uint16_t* wc, bool use_match, int lane) {
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    if (j >= R) break;  // warp-uniform
    const uint32_t d = dr[j];
    uint32_t peers;
    if (use_match) {  // warp-uniform
      peers = __match_any_sync(FULL, d);
    } else {
      const uint32_t valid = __ballot_sync(FULL, d < TS_BINS);
      peers = d < TS_BINS ? valid : ~valid;
#pragma unroll
      for (int b = 0; b < TS_BITS; ++b) {
        const uint32_t m = __ballot_sync(FULL, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? m : ~m;
      }
    }
    const bool leader = (peers & lt_mask) == 0;
    use_match = __popc(__ballot_sync(FULL, leader)) <= 16;
    const uint32_t cur = wc[d];
    dr[j] = d | ((cur + __popc(peers & lt_mask)) << 10);
    __syncwarp();
    if (leader) wc[d] = (uint16_t)(cur + __popc(peers));
    __syncwarp();
  }
}

// smallest and largest of the per-thread values into *kmin / *kmax (set to ~0u / 0 before a barrier)
__device__ __forceinline__ void ts_min_max(uint32_t mn, uint32_t mx, uint32_t* kmin, uint32_t* kmax) {
  mn = __reduce_min_sync(FULL, mn);
  mx = __reduce_max_sync(FULL, mx);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(kmin, mn);
    atomicMax(kmax, mx);
  }
}

// the tile's pair range: from the sort's last pass, or the whole list when no pass ran (one tile)
__device__ __forceinline__ void ts_range(const uint32_t* ranges, uint32_t tile, int64_t n, bool ranges_ready,
                                         uint32_t* lo, uint32_t* hi) {
  *lo = *hi = 0u;
  if (n <= 0) return;
  if (!ranges_ready) {
    *hi = (uint32_t)n;
    return;
  }
  const uint2 r = reinterpret_cast<const uint2*>(ranges)[tile];
  if (r.x < r.y) {
    *lo = r.x;
    *hi = r.y;
  }
}

__device__ __forceinline__ int ts_passes(uint32_t span) {
  return span ? (32 - __clz(span) + TS_BITS - 1) / TS_BITS : 0;
}

// ---- short lists: one warp each, TW_WARPS tiles per block
__global__ void __launch_bounds__(TW_WARPS * 32, 2) k_tile_sort_warp(uint32_t* __restrict__ tvals,
                                                                    const uint32_t* __restrict__ s_dkey,
                                                                    const unsigned long long* __restrict__ d_count,
                                                                    int64_t cap, bool ranges_ready, int64_t tiles,
                                                                    uint32_t* __restrict__ ranges,
                                                                    uint32_t* __restrict__ mid_tiles,
                                                                    unsigned int* __restrict__ n_mid,
                                                                    uint2* __restrict__ chunks,
                                                                    unsigned int* __restrict__ n_chunks,
                                                                    uint32_t* __restrict__ long_tiles,
                                                                    unsigned int* __restrict__ n_long) {
  extern __shared__ __align__(16) unsigned char tw_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpSortSmem& W = reinterpret_cast<TileSortWarpSmem*>(tw_raw)->w[warp];
  const int64_t tile64 = (int64_t)blockIdx.x * TW_WARPS + warp;
  if (tile64 >= tiles) return;  // warp-uniform; no block-wide barrier below
  const uint32_t tile = (uint32_t)tile64;
  uint32_t lo = 0, hi = 0;
  if (lane == 0) {
    ts_range(ranges, tile, usable_pairs(d_count, cap), ranges_ready, &lo, &hi);
    reinterpret_cast<uint2*>(ranges)[tile] = make_uint2(lo, hi);
    const uint32_t L = hi - lo;
    if (L > (uint32_t)TS_CHUNK) {
      const uint32_t nc = (L + TS_CHUNK - 1) / TS_CHUNK;
      const uint32_t at = atomicAdd(n_chunks, nc);
      for (uint32_t c = 0; c < nc; ++c) chunks[at + c] = make_uint2(tile, c);
      long_tiles[atomicAdd(n_long, 1u)] = tile;
    } else if (L > (uint32_t)TW_MAX) {
      mid_tiles[atomicAdd(n_mid, 1u)] = tile;
    }
  }
  lo = __shfl_sync(FULL, lo, 0);
  const int L = (int)(__shfl_sync(FULL, hi, 0) - lo);
  if (L < 2 || L > TW_MAX) return;  // warp-uniform
  const int R = (L + 31) / 32;
  uint32_t mn = ~0u, mx = 0u;
  {
    uint32_t kk[TW_ITEMS], vv[TW_ITEMS];
#pragma unroll
    for (int j = 0; j < TW_ITEMS; ++j) {
      if (j >= R) break;
      vv[j] = j * 32 + lane < L ? tvals[lo + j * 32 + lane] : 0u;
    }
#pragma unroll
    for (int j = 0; j < TW_ITEMS; ++j) {
      if (j >= R) break;
      kk[j] = j * 32 + lane < L ? s_dkey[vv[j]] : 0u;
    }
#pragma unroll
    for (int j = 0; j < TW_ITEMS; ++j) {
      if (j >= R) break;
      const int q = j * 32 + lane;
      if (q < L) {
        W.k[0][q] = kk[j];
        W.v[0][q] = vv[j];
        mn = min(mn, kk[j]);
        mx = max(mx, kk[j]);
      }
    }
  }
  const uint32_t kmin = __reduce_min_sync(FULL, mn);
  const int npass = ts_passes(__reduce_max_sync(FULL, mx) - kmin);
  if (npass == 0) return;  // warp-uniform: all keys equal, item order is the order
  __syncwarp();
  int cur = 0;
  for (int pass = 0; pass < npass; ++pass) {
    const int shift = TS_BITS * pass;
    uint32_t dr[TW_ITEMS];
#pragma unroll
    for (int j = 0; j < TW_ITEMS; ++j) {
      if (j >= R) break;
      const int q = j * 32 + lane;
      dr[j] = q < L ? ((W.k[cur][q] - kmin) >> shift) & (TS_BINS - 1) : (uint32_t)TS_BINS;
    }
    uint32_t* wcw = reinterpret_cast<uint32_t*>(W.wc);
    for (int x = lane; x < (TS_BINS + 2) / 2; x += 32) wcw[x] = 0u;
    __syncwarp();
    ts_rank<TW_ITEMS>(dr, R, W.wc, pass > 0, lane);
    __syncwarp();
    // digit starts: lane l takes digits 16 l .. 16 l + 15 (8 words of two counts), the lanes'
    // totals are scanned, then each lane writes its digits' starts
    const uint32_t* wc2 = reinterpret_cast<const uint32_t*>(W.wc) + 8 * lane;
    uint32_t tot = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t c2 = wc2[i];
      tot += (c2 & 0xffffu) + (c2 >> 16);
    }
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    uint32_t run = x - tot;
    uint32_t* base2 = reinterpret_cast<uint32_t*>(W.base) + 8 * lane;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint32_t c2 = wc2[i];
      const uint32_t b0 = run, b1 = run + (c2 & 0xffffu);
      base2[i] = b0 | (b1 << 16);
      run = b1 + (c2 >> 16);
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < TW_ITEMS; ++j) {
      if (j >= R) break;
      const uint32_t d = dr[j] & 1023u;
      if (d < TS_BINS) {
        const int q = j * 32 + lane;
        const uint32_t pos = W.base[d] + (dr[j] >> 10);
        W.k[cur ^ 1][pos] = W.k[cur][q];
        W.v[cur ^ 1][pos] = W.v[cur][q];
      }
    }
    __syncwarp();
    cur ^= 1;
  }
#pragma unroll
  for (int j = 0; j < TW_ITEMS; ++j) {
    if (j >= R) break;
    const int q = j * 32 + lane;
    if (q < L) tvals[lo + q] = W.v[cur][q];
  }
}

// Sorts m <= TS_CHUNK slots src[0, m) by order key with the whole block; the
// sorted slots go to out_v[0, m) (which may be src) and, when out_k is not
// null, their keys to out_k[0, m).  Returns with the block in step.
__device__ __forceinline__ void ts_sort_chunk(TileSortSmem& S, const uint32_t* src,
                                              const uint32_t* __restrict__ s_dkey, int m, uint32_t* out_k,
                                              uint32_t* out_v) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) {
    S.kmin = ~0u;
    S.kmax = 0u;
  }
  __syncthreads();
  const int R = (m + TS_THREADS - 1) / TS_THREADS;  // items per thread, and rounds per warp
  {
    // every slot load, then every key load, in flight at once
    uint32_t kk[TS_ITEMS], vv[TS_ITEMS];
#pragma unroll
    for (int j = 0; j < TS_ITEMS; ++j) {
      if (j >= R) break;
      const int q = t + j * TS_THREADS;
      vv[j] = q < m ? src[q] : 0u;
    }
#pragma unroll
    for (int j = 0; j < TS_ITEMS; ++j) {
      if (j >= R) break;
      const int q = t + j * TS_THREADS;
      kk[j] = q < m ? s_dkey[vv[j]] : 0u;
    }
    uint32_t mn = ~0u, mx = 0u;
#pragma unroll
    for (int j = 0; j < TS_ITEMS; ++j) {
      if (j >= R) break;
      const int q = t + j * TS_THREADS;
      if (q < m) {
        S.k[q] = kk[j];
        S.v[q] = vv[j];
        mn = min(mn, kk[j]);
        mx = max(mx, kk[j]);
      }
    }
    ts_min_max(mn, mx, &S.kmin, &S.kmax);
  }
  __syncthreads();
  const uint32_t kmin = S.kmin;
  const int npass = ts_passes(S.kmax - kmin);
  for (int pass = 0; pass < npass; ++pass) {
    const int shift = TS_BITS * pass;
    uint32_t kk[TS_ITEMS], vv[TS_ITEMS], dr[TS_ITEMS];
#pragma unroll
    for (int j = 0; j < TS_ITEMS; ++j) {
      if (j >= R) break;
      const int q = warp * 32 * R + j * 32 + lane;
      const bool ok = q < m;
      kk[j] = ok ? S.k[q] : 0u;
      vv[j] = ok ? S.v[q] : 0u;
      dr[j] = ok ? ((kk[j] - kmin) >> shift) & (TS_BINS - 1) : (uint32_t)TS_BINS;
    }
    {
      uint32_t* p = reinterpret_cast<uint32_t*>(&S.wc[0][0]);
      for (int x = t; x < TS_WARPS * (TS_BINS + 2) / 2; x += TS_THREADS) p[x] = 0u;
    }
    __syncthreads();
    ts_rank<TS_ITEMS>(dr, R, S.wc[warp], pass > 0, lane);
    __syncthreads();
    uint32_t c = 0;  // digit t: warp counts -> warp prefixes
#pragma unroll
    for (int w = 0; w < TS_WARPS; ++w) {
      const uint32_t x = S.wc[w][t];
      S.wc[w][t] = (uint16_t)c;
      c += x;
    }
    S.base[t] = ts_block_excl<TS_WARPS>(c, S.w);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TS_ITEMS; ++j) {
      if (j >= R) break;
      const uint32_t d = dr[j] & 1023u;
      if (d < TS_BINS) {
        const uint32_t pos = S.base[d] + S.wc[warp][d] + (dr[j] >> 10);
        S.k[pos] = kk[j];
        S.v[pos] = vv[j];
      }
    }
    __syncthreads();
  }
  for (int q = t; q < m; q += TS_THREADS) {
    out_v[q] = S.v[q];
    if (out_k) out_k[q] = S.k[q];
  }
}

// Persistent blocks over the medium tiles (sorted in place), then over the
// chunks of the long tiles (sorted into the scratch arrays xk, xv at the
// chunk's own positions).
__global__ void __launch_bounds__(TS_THREADS, 2) k_tile_sort(uint32_t* __restrict__ tvals,
                                                            uint32_t* __restrict__ xk, uint32_t* __restrict__ xv,
                                                            const uint32_t* __restrict__ s_dkey,
                                                            const uint32_t* __restrict__ ranges,
                                                            const uint32_t* __restrict__ mid_tiles,
                                                            const unsigned int* __restrict__ n_mid,
                                                            const uint2* __restrict__ chunks,
                                                            const unsigned int* __restrict__ n_chunks,
                                                            unsigned int* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char ts_raw[];
  TileSortSmem& S = *reinterpret_cast<TileSortSmem*>(ts_raw);
  const unsigned int nm = *n_mid, total = nm + *n_chunks;
  while (true) {
    if (threadIdx.x == 0) S.item = atomicAdd(work, 1u);
    __syncthreads();
    const unsigned int item = S.item;
    __syncthreads();  // everyone has read the item before it is overwritten
    if (item >= total) return;  // block-uniform
    uint32_t off, m;
    const bool mid = item < nm;
    if (mid) {
      const uint2 r = reinterpret_cast<const uint2*>(ranges)[mid_tiles[item]];
      off = r.x;
      m = r.y - r.x;
    } else {
      const uint2 ch = chunks[item - nm];
      const uint2 r = reinterpret_cast<const uint2*>(ranges)[ch.x];
      off = r.x + ch.y * (uint32_t)TS_CHUNK;
      m = min((uint32_t)TS_CHUNK, r.y - off);
    }
    ts_sort_chunk(S, tvals + off, s_dkey, (int)m, mid ? nullptr : xk + off, (mid ? tvals : xv) + off);
    __syncthreads();
  }
}

// number of entries of the ascending run[0, n) below k (or, with or_equal, not above k); n <= TS_CHUNK
__device__ __forceinline__ uint32_t ts_count_below(const uint32_t* run, uint32_t n, uint32_t k, bool or_equal) {
  uint32_t base = 0;
#pragma unroll
  for (uint32_t step = TS_CHUNK; step; step >>= 1) {
    if (base + step <= n) {
      const uint32_t x = run[base + step - 1];
      if (or_equal ? x <= k : x < k) base += step;
    }
  }
  return base;
}

// (dk, dv)[0, n) = (sk, sv)[0, n), n <= 2 * TS_CHUNK, with every load of a thread in flight at once
__device__ __forceinline__ void ts_stage(uint32_t* dk, uint32_t* dv, const uint32_t* __restrict__ sk,
                                         const uint32_t* __restrict__ sv, int n) {
  constexpr int U = 2 * TS_CHUNK / TS_THREADS;
  uint32_t k[U], v[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int q = threadIdx.x + j * TS_THREADS;
    k[j] = q < n ? sk[q] : 0u;
    v[j] = q < n ? sv[q] : 0u;
  }
  asm volatile("" ::: "memory");  // all loads before the first store
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int q = threadIdx.x + j * TS_THREADS;
    if (q < n) {
      dk[q] = k[j];
      dv[q] = v[j];
    }
  }
}

// Block-wide stable merge of the ascending runs (ak, av)[0, na) and (bk, bv)[0, nb)
// into (ok, ov)[0, na + nb) (ok may be null): equal keys take the first run's
// entries first.  Each thread finds where its share of the output starts in
// both runs by one binary search along the output's diagonal, then merges its
// share sequentially.
__device__ __forceinline__ void ts_merge2(const uint32_t* ak, const uint32_t* av, int na, const uint32_t* bk,
                                          const uint32_t* bv, int nb, uint32_t* ok, uint32_t* ov) {
  const int n = na + nb, per = (n + TS_THREADS - 1) / TS_THREADS;
  const int i0 = min(n, (int)threadIdx.x * per), i1 = min(n, i0 + per);
  int lo = max(0, i0 - nb), hi = min(i0, na);  // entries of the first run among the first i0 outputs
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ak[mid] <= bk[i0 - mid - 1]) lo = mid + 1;
    else hi = mid;
  }
  int ia = lo, ib = i0 - lo;
  for (int i = i0; i < i1; ++i) {
    const bool take_a = ia < na && (ib >= nb || ak[ia] <= bk[ib]);
    const uint32_t k = take_a ? ak[ia] : bk[ib], v = take_a ? av[ia] : bv[ib];
    if (ok) ok[i] = k;
    ov[i] = v;
    ia += take_a ? 1 : 0;
    ib += take_a ? 0 : 1;
  }
}

// Persistent blocks over the long tiles, whose chunks k_tile_sort has sorted
// into the scratch arrays (xk, xv).  Two or three chunks are merged through
// shared memory (the first two, then that with the third); a tile of more
// chunks places each pair behind the pairs of earlier chunks with keys not
// above its own and of later chunks with keys below it, found by binary
// searches of those chunks.
__global__ void __launch_bounds__(TS_THREADS) k_tile_merge(uint32_t* __restrict__ tvals,
                                                          const uint32_t* __restrict__ xk,
                                                          const uint32_t* __restrict__ xv,
                                                          const uint32_t* __restrict__ ranges,
                                                          const uint32_t* __restrict__ long_tiles,
                                                          const unsigned int* __restrict__ n_long,
                                                          unsigned int* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char tm_raw[];
  TileMergeSmem& S = *reinterpret_cast<TileMergeSmem*>(tm_raw);
  const int t = threadIdx.x;
  const unsigned int total = *n_long;
  while (true) {
    if (t == 0) S.item = atomicAdd(work, 1u);
    __syncthreads();
    const unsigned int item = S.item;
    __syncthreads();
    if (item >= total) return;  // block-uniform
    const uint2 r = reinterpret_cast<const uint2*>(ranges)[long_tiles[item]];
    const int L = (int)(r.y - r.x), nc = (L + TS_CHUNK - 1) / TS_CHUNK;
    const uint32_t* ck = xk + r.x;
    const uint32_t* cv = xv + r.x;
    if (nc <= 3) {
      // chunks 0 and 1 side by side in area 0
      const int n01 = min(L, 2 * TS_CHUNK);
      ts_stage(S.k[0], S.v[0], ck, cv, n01);
      __syncthreads();
      const int n1 = n01 - TS_CHUNK;
      if (nc == 2) {
        ts_merge2(S.k[0], S.v[0], TS_CHUNK, S.k[0] + TS_CHUNK, S.v[0] + TS_CHUNK, n1, nullptr, tvals + r.x);
      } else {
        ts_merge2(S.k[0], S.v[0], TS_CHUNK, S.k[0] + TS_CHUNK, S.v[0] + TS_CHUNK, n1, S.k[1], S.v[1]);
        __syncthreads();  // area 0 is read: chunk 2 goes there
        const int n2 = L - n01;
        ts_stage(S.k[0], S.v[0], ck + n01, cv + n01, n2);
        __syncthreads();
        ts_merge2(S.k[1], S.v[1], n01, S.k[0], S.v[0], n2, nullptr, tvals + r.x);
      }
    } else {
      for (int c = 0; c < nc; ++c) {
        const int own = c * TS_CHUNK, m = min(TS_CHUNK, L - own);
        for (int q = t; q < m; q += TS_THREADS) {
          const uint32_t k = ck[own + q], v = cv[own + q];
          uint32_t pos = (uint32_t)q;
          for (int o = 0; o < nc; ++o) {
            if (o == c) continue;
            const int off = o * TS_CHUNK;
            pos += ts_count_below(ck + off, (uint32_t)min(TS_CHUNK, L - off), k, o < c);
          }
          tvals[r.x + pos] = v;
        }
      }
    }
    __syncthreads();  // shared memory is read before the next tile's loads
  }
}

// ------------------------------------------------------------------ per-pixel ray
struct Ray {
  float dx, dy, dz;     // unit direction
  float ix, iy, iz;     // 1 / direction (1e30 for a zero component)
  float ax, ay, az;     // |1 / direction|
  float tnear;          // ray parameter of the near plane (camera depth z_near)
};

__device__ __forceinline__ Ray make_ray(const DevView& c, int px, int py) {
  float dcx = __fdiv_rn((float)px + 0.5f - c.cx, c.fx);
  float dcy = __fdiv_rn((float)py + 0.5f - c.cy, c.fy);
  float wx = c.R[0] * dcx + c.R[3] * dcy + c.R[6];
  float wy = c.R[1] * dcx + c.R[4] * dcy + c.R[7];
  float wz = c.R[2] * dcx + c.R[5] * dcy + c.R[8];
  float inv = rsqrtf(wx * wx + wy * wy + wz * wz);
  Ray r;
  r.dx = wx * inv; r.dy = wy * inv; r.dz = wz * inv;
  r.ix = r.dx != 0.f ? __frcp_rn(r.dx) : 1e30f;
  r.iy = r.dy != 0.f ? __frcp_rn(r.dy) : 1e30f;
  r.iz = r.dz != 0.f ? __frcp_rn(r.dz) : 1e30f;
  r.ax = fabsf(r.ix); r.ay = fabsf(r.iy); r.az = fabsf(r.iz);
  r.tnear = c.z_near * (wx * wx + wy * wy + wz * wz) * inv;  // z_near * |(dcx, dcy, 1)|
  return r;
}

__device__ __forceinline__ float max3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float min3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Chord of the ray (origin at the camera) through the box centred at rc
// (relative to the camera) with half-size h, clipped to start at the near
// plane: slab a enters at (rc_a - h sign) / d_a and leaves at (rc_a + h sign) / d_a.
// Identical code in the forward and backward kernels, so both take the same
// hit decisions.
__device__ __forceinline__ bool chord(const Ray& r, float4 g, float& t_in, float& t_out) {
  const float qx = g.x * r.ix, qy = g.y * r.iy, qz = g.z * r.iz;
  t_in = fmaxf(max3(fmaf(-g.w, r.ax, qx), fmaf(-g.w, r.ay, qy), fmaf(-g.w, r.az, qz)), r.tnear);
  t_out = min3(fmaf(g.w, r.ax, qx), fmaf(g.w, r.ay, qy), fmaf(g.w, r.az, qz));
  return t_out > t_in;
}

// local coordinates u = (p - (c - h)) / (2h) = (t d - rc) / (2h) + 1/2 of the
// ray point at t, clamped to [0,1]^3, and the trilinear density there
__device__ __forceinline__ float trilin(const Ray& r, float4 g, float4 d0, float4 d1, float i2h, float t, float* u) {
  u[0] = __saturatef(fmaf(fmaf(t, r.dx, -g.x), i2h, 0.5f));
  u[1] = __saturatef(fmaf(fmaf(t, r.dy, -g.y), i2h, 0.5f));
  u[2] = __saturatef(fmaf(fmaf(t, r.dz, -g.z), i2h, 0.5f));
  float c00 = fmaf(u[0], d0.y - d0.x, d0.x);
  float c10 = fmaf(u[0], d0.w - d0.z, d0.z);
  float c01 = fmaf(u[0], d1.y - d1.x, d1.x);
  float c11 = fmaf(u[0], d1.w - d1.z, d1.z);
  float c0 = fmaf(u[1], c10 - c00, c00);
  float c1 = fmaf(u[1], c11 - c01, c01);
  return fmaf(u[2], c1 - c0, c0);
}

// Raw density of a sample: the trilinear field at the chord midpoint (u[0..2]),
// or, for the exact-segment variant (SEG), its mean over the chord: along a
// line the field is a cubic in t, so Simpson's rule (f_in + 4 f_mid + f_out) / 6
// is exact (u[3..5] at t_in, u[6..8] at t_out).
template <bool SEG>
__device__ __forceinline__ float sample_density(const Ray& r, float4 g, float4 d0, float4 d1, float i2h, float t_in,
                                                float tm, float t_out, float* u) {
  const float fm = trilin(r, g, d0, d1, i2h, tm, u);
  if constexpr (!SEG) {
    return fm;
  } else {
    const float fa = trilin(r, g, d0, d1, i2h, t_in, u + 3);
    const float fb = trilin(r, g, d0, d1, i2h, t_out, u + 6);
    return (fa + 4.f * fm + fb) * (1.f / 6.f);
  }
}

// v[c] = s * (trilinear weight of corner c at u), or += with ADD
template <bool ADD>
__device__ __forceinline__ void corner_weights(float* v, float s, const float* u) {
  const float ux = u[0], uy = u[1], uz = u[2];
  const float mx = 1.f - ux, my = 1.f - uy, mz = 1.f - uz;
  const float a00 = s * my * mz, a10 = s * uy * mz, a01 = s * my * uz, a11 = s * uy * uz;
  const float w[8] = {mx * a00, ux * a00, mx * a10, ux * a10, mx * a01, ux * a01, mx * a11, ux * a11};
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = ADD ? v[c] + w[c] : w[c];
}

// 1 - exp(-x) given e = exp(-x): a 5-term series below 1/8 (relative error
// < 5e-8 there), 1 - e above; branch-free
__device__ __forceinline__ float one_minus_exp(float x, float e) {
  float p = fmaf(x, -1.f / 120.f, 1.f / 24.f);
  p = fmaf(x, p, -1.f / 6.f);
  p = fmaf(x, p, 0.5f);
  p = fmaf(x, -p, 1.f);
  p *= x;
  return x < 0.125f ? p : 1.f - e;
}

__device__ __forceinline__ int find_view(const ViewSet& vs, int gtile) {
  int v = 0;
  while (v + 1 < vs.n && gtile >= vs.v[v + 1].tile_off) ++v;
  return v;
}

// The pixels of a warp form a 4 x 8 block of its tile (rows x columns; the
// warps of a TS x TS tile are laid out TS/8 across and TS/4 down, lanes
// row-major inside the block, so pixel ids grow with the lane).  Compared with
// a 2 x 16 strip, a small voxel's footprint meets fewer warps and more lanes
// of each.  A record whose conservative pixel box misses the block cannot be
// hit by any lane, so the whole warp skips it (a warp-uniform branch); the hit
// decisions are exactly those of the per-lane chord test.
template <int TS>
struct Strip {
  uint32_t x0, x1, y0, y1;  // [x0, x1) x [y0, y1) in image pixels
  __device__ __forceinline__ Strip(int tile_x, int tile_y, int warp) {
    x0 = (uint32_t)(tile_x * TS + (warp % (TS / 8)) * 8);
    x1 = x0 + 8;
    y0 = (uint32_t)(tile_y * TS + (warp / (TS / 8)) * 4);
    y1 = y0 + 4;
  }
  __device__ __forceinline__ int px(int lane) const { return (int)x0 + (lane & 7); }
  __device__ __forceinline__ int py(int lane) const { return (int)y0 + (lane >> 3); }
  // box: (bx0 | bx1 << 16, by0 | by1 << 16)
  __device__ __forceinline__ bool misses(uint2 box) const {
    return (box.x >> 16) <= x0 || (box.x & 0xffffu) >= x1 || (box.y >> 16) <= y0 || (box.y & 0xffffu) >= y1;
  }
};

// Work items are (tile, warp strip) pairs, item = tile * (TS*TS/32) + strip.
// Without PERSIST every warp takes the item of its own block and warp index;
// with PERSIST a grid sized to the resident warps loops, each warp taking the
// next item from a global counter (one atomicAdd per item, no waiting), so a
// warp that finishes a cheap strip moves on without waiting for its block.
__device__ __forceinline__ uint32_t next_item(unsigned int* work, int lane) {
  uint32_t it = 0;
  if (lane == 0) it = atomicAdd(work, 1u);
  return __shfl_sync(FULL, it, 0);
}

// A persistent grid limited to sm_cut of the n_sms SMs (0: all) is launched at
// full size; a block that lands on an SM outside the first sm_cut (by SM id,
// scaled to the id range) returns at once, so the kept SMs hold their full
// share of blocks and the others stay free for concurrent streams.  The work
// counter hands every item to the blocks that stay.
__device__ __forceinline__ bool sm_excluded(int sm_cut, int n_sms) {
  if (sm_cut <= 0) return false;
  uint32_t smid, nsmid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsmid));
  return (unsigned long long)smid * (unsigned)n_sms >= (unsigned long long)sm_cut * nsmid;
}

// Whether this block of a grid cut to sm_cut SMs leaves at once.  Some block must
// stay, or the work counter's items would be taken by nobody (every block could
// land on an excluded SM while streams of higher priority hold the kept ones), so
// each block counts its arrival in *arrivals (zero before the launch; a block on
// a kept SM adds 1 << 16 as well), and the grid's last block to arrive stays,
// wherever it runs, when no block before it stayed.  Called by every thread of
// the block (block barrier); grids of up to 65535 blocks.
__device__ __forceinline__ bool sm_leave(int sm_cut, int n_sms, unsigned int* arrivals) {
  if (sm_cut <= 0) return false;  // grid-uniform
  __shared__ int s_leave;
  if (threadIdx.x == 0) {
    const bool excl = sm_excluded(sm_cut, n_sms);
    const unsigned int old = atomicAdd(arrivals, excl ? 1u : 0x10001u);
    const bool last_alone = (old & 0xffffu) == gridDim.x - 1 && (old >> 16) == 0;
    s_leave = excl && !last_alone;
  }
  __syncthreads();
  return s_leave != 0;
}

// ------------------------------------------------------------------ forward composite
// Each warp walks its strip's tile list on its own: CH list entries at a time
// (the batch: 32, 64 or 128, CH / 32 per lane, all loads of a batch issued
// before any is used), the entries whose pixel box meets the strip are
// compacted with ballots and their 64-byte records staged in the warp's slice
// of shared memory, then every lane marches its pixel through them front to
// back.  No block-wide barrier: a warp stops as soon as all its pixels have
// stopped.
// per-warp staging slice: CH records (64 B) + voxel id + list entry (+ slot id in the backward)
__host__ __device__ constexpr size_t fwd_slice(int ch) { return (size_t)ch * 64 + (size_t)ch * 4 * 2; }
__host__ __device__ constexpr size_t bwd_slice(int ch) { return (size_t)ch * 64 + (size_t)ch * 4 * 3; }

// Stage the entries [base, base + CH) below `end` whose pixel box meets the
// strip: records in list order at positions 0 .. m - 1 of the warp's slice
// (voxel id, list entry and, with slot_out, the slot id beside them); returns m.
template <int TS, int CH>
__device__ __forceinline__ int stage_batch(uint32_t base, uint32_t end, int lane, const Strip<TS>& strip,
                                           const uint32_t* __restrict__ svals, const float4* __restrict__ rec,
                                           const uint2* __restrict__ rec_bb, const uint32_t* __restrict__ slot_vox,
                                           float4* wr, uint32_t* w_vox, uint32_t* w_ent, uint32_t* w_slot) {
  constexpr int K = CH / 32;
  uint32_t sl[K];
  bool ov[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t e = base + 32 * k + lane;
    sl[k] = e < end ? svals[e] : 0u;
  }
#pragma unroll
  for (int k = 0; k < K; ++k) ov[k] = base + 32 * k + lane < end && !strip.misses(rec_bb[sl[k]]);
  int m = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t mask = __ballot_sync(FULL, ov[k]);
    if (ov[k]) {
      const int pos = m + __popc(mask & ((1u << lane) - 1u));
      const float4* src = rec + 4 * (size_t)sl[k];
      wr[4 * pos + 0] = src[0];
      wr[4 * pos + 1] = src[1];
      wr[4 * pos + 2] = src[2];
      wr[4 * pos + 3] = src[3];
      w_vox[pos] = slot_vox[sl[k]];
      w_ent[pos] = base + 32 * k + lane;
      if (w_slot) w_slot[pos] = sl[k];
    }
    m += __popc(mask);
  }
  return m;
}
// The LF-weighted loss fused into the backward composite (Sec. IV-B, Eq. 8 and
// 18): per pixel dL/drgb = 2 / (3 |P_v|) * (w / <w>) * (rgb - gt), in the
// operation order lv_lf_loss_from_weights uses, and the view's summed
// weighted squared error (FP32 per warp item, FP64 per warp in shared memory,
// summed per block, one global FP64 atomic per block and view).  w == nullptr:
// not fused.
struct LfFuse {
  const float* rgb;    // [P][3] the forward's image
  const float* gt;     // [P][3]
  const float* w;      // [P] unnormalised weights (lv_lf_weights)
  const double* wsum;  // [views] their sums
  double* lsum;        // [views] loss sums
  float* dL;           // [P][3] dL/drgb, also written out (nullable)
};

template <int TS>
constexpr int min_blocks() { return TS == 16 ? 5 : (TS == 8 ? 16 : 1); }

template <int TS, bool SEG, bool PERSIST, int CH>
__global__ void __launch_bounds__(TS* TS, min_blocks<TS>()) k_fwd(const __grid_constant__ ViewSet vs, const uint32_t* __restrict__ ranges,
                                                const uint32_t* __restrict__ svals, const float4* __restrict__ rec,
                                                const uint2* __restrict__ rec_bb,
                                                const uint32_t* __restrict__ slot_vox, float t_stop,
                                                float* __restrict__ rgb, float* __restrict__ depth,
                                                float* __restrict__ T_out, uint32_t* __restrict__ n_contrib,
                                                uint32_t* __restrict__ n_samples, float* __restrict__ tau_out,
                                                unsigned long long* __restrict__ wmax, unsigned int* work,
                                                uint32_t n_items, int sm_cut, int n_sms, unsigned int* arrivals) {
  constexpr int NW = TS * TS / 32;
  extern __shared__ float4 smem_f4[];
  if (PERSIST && sm_leave(sm_cut, n_sms, arrivals)) return;  // block-uniform
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4* wr = (float4*)((char*)smem_f4 + fwd_slice(CH) * warp);
  uint32_t* w_vox = (uint32_t*)(wr + 4 * CH);
  uint32_t* w_ent = w_vox + CH;
  for (uint32_t item = PERSIST ? next_item(work, lane) : blockIdx.x * NW + warp; item < n_items;
       item = PERSIST ? next_item(work, lane) : n_items) {  // warp-uniform
    const int gtile = (int)(item / NW);
    const int view = find_view(vs, gtile);
    const DevView& c = vs.v[view];
    const int lt = gtile - c.tile_off;
    const int tile_x = lt % c.tiles_x, tile_y = lt / c.tiles_x;
    const Strip<TS> strip(tile_x, tile_y, (int)(item % NW));
    const int px = strip.px(lane), py = strip.py(lane);
    const bool inside = px < c.W && py < c.H;
    const Ray r = make_ray(c, px, py);
    const uint32_t start = ranges[2 * gtile], end = ranges[2 * gtile + 1];
    const unsigned long long gid = (unsigned long long)(c.pix_off + (long long)py * c.W + px);
    const unsigned long long gid_key = 0xffffffffull - ((gid + (unsigned long long)vs.id_base) & 0xffffffffull);
    float T = 1.f, tau = 0.f, cr = 0.f, cg = 0.f, cb = 0.f, dep = 0.f;
    uint32_t last = 0, nsamp = 0;
    bool done = !inside;
    for (uint32_t base = start; base < end && !__all_sync(FULL, done); base += CH) {
      const int m = stage_batch<TS, CH>(base, end, lane, strip, svals, rec, rec_bb, slot_vox, wr, w_vox, w_ent,
                                        nullptr);
      if (!m) continue;
      __syncwarp();
      int last_j = -1;  // the lane's last sample of this batch (its list entry is read once, below)
      for (int j = 0; j < m; ++j) {
        if (CH > 32 && (j & 31) == 31 && __all_sync(FULL, done)) break;  // warp-uniform
        const float4 g = wr[4 * j];
        float t_in, t_out;
        const bool hit = !done && chord(r, g, t_in, t_out);
        float w = 0.f;
        if (hit) {
          const float4 d0 = wr[4 * j + 1], d1 = wr[4 * j + 2], col = wr[4 * j + 3];
          const float l = t_out - t_in, tm = 0.5f * (t_in + t_out);
          float u[SEG ? 9 : 3];
          const float sigma = fmaxf(sample_density<SEG>(r, g, d0, d1, col.w, t_in, tm, t_out, u), 0.f);
          const float x = sigma * l;
          const float ex = __expf(-x);
          const float alpha = one_minus_exp(x, ex);
          w = T * alpha;
          cr = fmaf(w, col.x, cr);
          cg = fmaf(w, col.y, cg);
          cb = fmaf(w, col.z, cb);
          dep = fmaf(w, tm, dep);
          tau += x;
          T *= ex;
          last_j = j;
          ++nsamp;
        }
        if (__any_sync(FULL, hit)) {
          // the warp's largest w (ties to the lowest lane = smallest pixel id), one global atomic
          const uint32_t v = hit ? __float_as_uint(w) + 1u : 0u;
          const uint32_t mx = __reduce_max_sync(FULL, v);
          const uint32_t who = __ballot_sync(FULL, v == mx);
          if (wmax && lane == __ffs(who) - 1)
            atomicMax(&wmax[w_vox[j]], ((unsigned long long)(mx - 1u) << 32) | gid_key);
          if (hit && T < t_stop) done = true;
        }
      }
      if (last_j >= 0) last = w_ent[last_j] - start + 1;
      __syncwarp();
    }
    if (inside) {
      const size_t p = (size_t)gid;
      rgb[3 * p + 0] = cr;
      rgb[3 * p + 1] = cg;
      rgb[3 * p + 2] = cb;
      if (depth) depth[p] = dep;
      T_out[p] = T;
      n_contrib[p] = last;
      if (n_samples) n_samples[p] = nsamp;
      tau_out[p] = tau;
    }
    __syncwarp();  // the slice is reused by the next item
  }
}

// ------------------------------------------------------------------ backward composite
// Transposed butterfly: after 16 shuffles even lane l holds the warp sum of
// value (l >> 1) of the 16 inputs (instead of 16 * 5 shuffles).
__device__ __forceinline__ float warp_reduce16(float* v, int lane) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool up = lane & 16;
    float send = up ? v[i] : v[i + 8];
    float keep = up ? v[i + 8] : v[i];
    v[i] = keep + __shfl_xor_sync(FULL, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool up = lane & 8;
    float send = up ? v[i] : v[i + 4];
    float keep = up ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(FULL, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool up = lane & 4;
    float send = up ? v[i] : v[i + 2];
    float keep = up ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(FULL, send, 4);
  }
  {
    const bool up = lane & 2;
    float send = up ? v[0] : v[1];
    float keep = up ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(FULL, send, 2);
  }
  return v[0] + __shfl_xor_sync(FULL, v[0], 1);
}

// Backward: each warp walks its strip's list back to front from the last entry
// any of its pixels used, in the same 32-entry chunks and with the same
// compaction as the forward; the per-record gradients (8 corners + colour) are
// reduced over the warp and sent with three 16-byte global reductions.
template <int TS, bool SEG, bool PERSIST, int CH>
__global__ void __launch_bounds__(TS* TS, min_blocks<TS>()) k_bwd(const __grid_constant__ ViewSet vs, const uint32_t* __restrict__ ranges,
                                                const uint32_t* __restrict__ svals, const float4* __restrict__ rec,
                                                const uint2* __restrict__ rec_bb,
                                                const uint32_t* __restrict__ slot_vox, const float* __restrict__ T_fwd,
                                                const float* __restrict__ tau_in,
                                                const uint32_t* __restrict__ n_contrib,
                                                const float* __restrict__ dL_drgb, const float* __restrict__ dL_ddepth,
                                                const float* __restrict__ dL_dT, float* __restrict__ d_density,
                                                float4* __restrict__ d_rgb, unsigned int* work, uint32_t n_items,
                                                int sm_cut, int n_sms, unsigned int* arrivals, const LfFuse lf) {
  constexpr int NW = TS * TS / 32;
  extern __shared__ float4 smem_f4[];
  __shared__ double s_lf[NW][LV_MAX_VIEWS];  // each warp's loss sums (fused LF loss; no atomics)
  __shared__ float s_mean[LV_MAX_VIEWS], s_gscale[LV_MAX_VIEWS];  // the fused LF loss's per-view constants
  if (PERSIST && sm_leave(sm_cut, n_sms, arrivals)) return;  // block-uniform
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (lf.w) {  // grid-uniform; a warp clears and then adds to its own row only
    for (int v = lane; v < vs.n; v += 32) s_lf[warp][v] = 0.0;
    // each view's mean weight and gradient scale, rounded from FP64 as the loss kernel rounds them,
    // once per block (FP64 division is slow on this part)
    for (int v = tid; v < vs.n; v += TS * TS) {
      const double np = (double)vs.v[v].W * (double)vs.v[v].H;
      s_mean[v] = (float)(lf.wsum[v] / np);
      s_gscale[v] = (float)(2.0 / (3.0 * np));
    }
    __syncthreads();
  }
  float4* wr = (float4*)((char*)smem_f4 + bwd_slice(CH) * warp);
  uint32_t* w_vox = (uint32_t*)(wr + 4 * CH);
  uint32_t* w_slot = w_vox + CH;
  uint32_t* w_ent = w_slot + CH;
  for (uint32_t item = PERSIST ? next_item(work, lane) : blockIdx.x * NW + warp; item < n_items;
       item = PERSIST ? next_item(work, lane) : n_items) {  // warp-uniform
    const int gtile = (int)(item / NW);
    const int view = find_view(vs, gtile);
    const DevView& c = vs.v[view];
    const int lt = gtile - c.tile_off;
    const int tile_x = lt % c.tiles_x, tile_y = lt / c.tiles_x;
    const Strip<TS> strip(tile_x, tile_y, (int)(item % NW));
    const int px = strip.px(lane), py = strip.py(lane);
    const bool inside = px < c.W && py < c.H;
    const Ray r = make_ray(c, px, py);
    const uint32_t start = ranges[2 * gtile];
    const size_t p = (size_t)(c.pix_off + (long long)py * c.W + px);
    uint32_t nc = 0;
    float tau = 0.f, Tf = 1.f, gr = 0.f, gg = 0.f, gb = 0.f, gD = 0.f, gT = 0.f;
    if (inside) {
      nc = n_contrib[p];
      tau = tau_in[p];
      Tf = T_fwd[p];
      if (!lf.w) {
        gr = dL_drgb[3 * p + 0];
        gg = dL_drgb[3 * p + 1];
        gb = dL_drgb[3 * p + 2];
      }
      if (dL_ddepth) gD = dL_ddepth[p];
      if (dL_dT) gT = dL_dT[p];
    }
    if (lf.w) {  // grid-uniform: dL/drgb of the LF-weighted loss from the forward's image
      const float mean = s_mean[view], gscale = s_gscale[view];
      float part = 0.f;
      if (inside) {
        const float wt = lf.w[p] / mean;
        const float r0 = lf.rgb[3 * p] - lf.gt[3 * p], r1 = lf.rgb[3 * p + 1] - lf.gt[3 * p + 1],
                    r2 = lf.rgb[3 * p + 2] - lf.gt[3 * p + 2];
        part = wt * (r0 * r0 + r1 * r1 + r2 * r2);
        const float cf = gscale * wt;
        gr = cf * r0;
        gg = cf * r1;
        gb = cf * r2;
        if (lf.dL) {
          lf.dL[3 * p + 0] = gr;
          lf.dL[3 * p + 1] = gg;
          lf.dL[3 * p + 2] = gb;
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
      if (lane == 0) s_lf[warp][view] += (double)part;
    }
    const uint32_t my_hi = start + nc;  // entries [start, my_hi) were used by this pixel
    const uint32_t warp_hi = start + __reduce_max_sync(FULL, nc);
    const float tgT = Tf * gT;
    float S = 0.f;
    float Tcur = __expf(-tau);  // T after the last sample, from the stored optical depth
    // batches aligned as in the forward: [start + CH k, start + CH k + CH), walked back to front
    for (uint32_t cb = start + (warp_hi - start + CH - 1) / CH * CH; cb > start; cb -= CH) {
      const uint32_t base = cb - CH;
      const int m = stage_batch<TS, CH>(base, warp_hi, lane, strip, svals, rec, rec_bb, slot_vox, wr, w_vox,
                                        w_ent, w_slot);
      if (!m) continue;
      __syncwarp();
      for (int j = m - 1; j >= 0; --j) {
        const float4 g = wr[4 * j];
        float t_in, t_out;
        const bool hit = w_ent[j] < my_hi && chord(r, g, t_in, t_out);
        const unsigned hb = __ballot_sync(FULL, hit);
        if (!hb) continue;
        float v[16];
  #pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = 0.f;
        if (hit) {
          const float4 d0 = wr[4 * j + 1], d1 = wr[4 * j + 2], col = wr[4 * j + 3];
          const float l = t_out - t_in, tm = 0.5f * (t_in + t_out);
          float u[SEG ? 9 : 3];
          const float sraw = sample_density<SEG>(r, g, d0, d1, col.w, t_in, tm, t_out, u);
          const float sigma = fmaxf(sraw, 0.f);
          const float x = sigma * l;
          const float Tk = Tcur;  // transmittance after this sample: the previous step's T_prev
          const float tau_prev = fmaxf(tau - x, 0.f);
          const float T_prev = __expf(-tau_prev);
          Tcur = T_prev;
          const float alpha = one_minus_exp(x, __expf(-x));
          const float w = T_prev * alpha;
          const float a = fmaf(gr, col.x, fmaf(gg, col.y, fmaf(gb, col.z, gD * tm)));
          const float ds = l * (Tk * a - S - tgT);
          S = fmaf(w, a, S);
          tau = tau_prev;
          const float dr = sraw > 0.f ? ds : 0.f;
          corner_weights<false>(v, SEG ? dr * (4.f / 6.f) : dr, u);
          if constexpr (SEG) {
            corner_weights<true>(v, dr * (1.f / 6.f), u + 3);
            corner_weights<true>(v, dr * (1.f / 6.f), u + 6);
          }
          v[8] = w * gr;
          v[9] = w * gg;
          v[10] = w * gb;
        }
        float* dd = d_density + 8 * (size_t)w_vox[j];
        float* dc = (float*)(d_rgb + w_slot[j]);
        if (__popc(hb) <= 8) {
          // up to eight lanes: each sends its own values, cheaper than the butterfly (measured: 8 lanes
          // 2 % faster than 2; every lane, 12x slower, the reductions to one address serialise)
          if (hit) {
            red_add_v4(dd, v[0], v[1], v[2], v[3]);
            red_add_v4(dd + 4, v[4], v[5], v[6], v[7]);
            red_add_v4(dc, v[8], v[9], v[10], 0.f);
          }
        } else {
          const float sum = warp_reduce16(v, lane);  // value (l >> 1) on even lane l
          // gather four values each into lanes 0 (corners 0-3), 1 (corners 4-7) and 2 (colour)
          const int src0 = lane == 0 ? 0 : (lane == 1 ? 8 : 16);
          const float q0 = __shfl_sync(FULL, sum, src0 + 0);
          const float q1 = __shfl_sync(FULL, sum, src0 + 2);
          const float q2 = __shfl_sync(FULL, sum, src0 + 4);
          const float q3 = __shfl_sync(FULL, sum, src0 + 6);
          if (lane == 0) red_add_v4(dd, q0, q1, q2, q3);
          else if (lane == 1) red_add_v4(dd + 4, q0, q1, q2, q3);
          else if (lane == 2) red_add_v4(dc, q0, q1, q2, 0.f);
        }
      }
      __syncwarp();
    }
  }
  if (lf.w) {
    __syncthreads();
    for (int v = tid; v < vs.n; v += TS * TS) {
      double t = 0.0;
      for (int w = 0; w < NW; ++w) t += s_lf[w][v];
      if (t != 0.0) atomicAdd(&lf.lsum[v], t);
    }
  }
}

// ------------------------------------------------------------------ SH backward
// A warp handles 32 consecutive voxels, one per lane.  d c / d SH_j = Y_j(dir)
// where the clamp c = max(0, SH + 0.5) passed; the forward left that per-channel
// mask in the w component of the slot's colour-gradient scratch, so the SH rows
// themselves are not read again.  Each lane sums its voxel's gradients over the
// views; the 32 rows leave through shared memory as coalesced 16-byte stores
// (row stride 49 floats: conflict-free per lane).  With `accumulate`, warps
// without any visible voxel touch nothing.
__global__ void __launch_bounds__(128) k_sh_bwd(const float4* __restrict__ rec, int sh_nb, int64_t n,
                                                const __grid_constant__ ViewSet vs,
                                                const uint32_t* __restrict__ vis, const uint32_t* __restrict__ slot,
                                                float4* __restrict__ d_rgb, float* __restrict__ d_sh,
                                                int accumulate) {
  constexpr int RS = 49;
  __shared__ float s_rows[4][32 * RS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t v0 = (blockIdx.x * 4 + warp) * (int64_t)32;
  if (v0 >= n) return;  // warp-uniform
  const int nrows = (int)min((int64_t)32, n - v0);
  float* buf = s_rows[warp];
  float acc[48];
#pragma unroll
  for (int k = 0; k < 48; ++k) acc[k] = 0.f;
  bool any_vis = false;
  if (lane < nrows) {
    const int64_t vox = v0 + lane;
    for (int view = 0; view < vs.n; ++view) {
      const int64_t i = (int64_t)view * n + vox;  // view-major items
      if (!vis[i]) continue;
      any_vis = true;
      const uint32_t s = slot[i];
      // the record holds the centre relative to this view's camera, as k_emit computed it, so the
      // voxel arrays are not read (a topology change may rewrite them meanwhile)
      const float4 g = rec[4 * (int64_t)s];
      float dir[3];
      unit_dir(g.x, g.y, g.z, dir);
      float Y[16];
      sh_basis(dir[0], dir[1], dir[2], Y);
      const float4 dc = d_rgb[s];
      const int m = (int)dc.w;
      const float dr = (m & 1) ? dc.x : 0.f;
      const float dg = (m & 2) ? dc.y : 0.f;
      const float db = (m & 4) ? dc.z : 0.f;
      d_rgb[s] = make_float4(0.f, 0.f, 0.f, dc.w);  // cleared for the next backward call; mask kept
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j < sh_nb) {
          acc[3 * j + 0] = fmaf(Y[j], dr, acc[3 * j + 0]);
          acc[3 * j + 1] = fmaf(Y[j], dg, acc[3 * j + 1]);
          acc[3 * j + 2] = fmaf(Y[j], db, acc[3 * j + 2]);
        }
      }
    }
  }
  if (accumulate && !__any_sync(FULL, any_vis)) return;  // nothing to add for these 32 voxels
  if (lane < nrows) {
#pragma unroll
    for (int k = 0; k < 48; ++k) buf[lane * RS + k] = acc[k];
  }
  __syncwarp();
  float4* dst = (float4*)(d_sh + 48 * v0);
  for (int w = lane; w < nrows * 12; w += 32) {
    const float* a = buf + (w / 12) * RS + (w % 12) * 4;
    float4 o = make_float4(a[0], a[1], a[2], a[3]);
    if (accumulate) {
      const float4 p = dst[w];
      o.x += p.x; o.y += p.y; o.z += p.z; o.w += p.w;
    }
    dst[w] = o;
  }
}

__global__ void k_unpack_wmax(const unsigned long long* __restrict__ packed, int64_t n, float* __restrict__ w,
                              int64_t* __restrict__ arg) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long v = packed[i];
  if (v == 0ull) {
    w[i] = 0.f;
    if (arg) arg[i] = -1;
  } else {
    w[i] = __uint_as_float((uint32_t)(v >> 32));
    if (arg) arg[i] = (int64_t)(0xffffffffull - (v & 0xffffffffull));
  }
}

__global__ void k_gather_edge(const int64_t* __restrict__ argmax, int64_t n, const float* __restrict__ edge_map,
                              int64_t n_pix, float* __restrict__ edge) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t a = argmax[i];
  edge[i] = (a >= 0 && a < n_pix) ? edge_map[a] : 0.f;
}

__global__ void k_debug_pairs(const uint32_t* __restrict__ k, const uint32_t* __restrict__ v,
                              const uint32_t* __restrict__ slot_vox, const uint32_t* __restrict__ s_dkey,
                              const unsigned long long* d_count, int64_t cap, uint64_t* ko, uint32_t* vo) {
  const int64_t n = usable_pairs(d_count, cap);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (ko) ko[i] = ((uint64_t)k[i] << 32) | s_dkey[v[i]];
    if (vo) vo[i] = slot_vox[v[i]];
  }
}

// ------------------------------------------------------------------ FP64 re-render (gradient checks)
// One thread per listed pixel: the pixel's tile list (from a forward
// workspace) is walked front to back in FP64 from the original voxel arrays
// (geometry, corner densities and SH converted exactly to double): the FP64
// counterpart of k_fwd, used only to take finite differences of the loss.
__device__ __forceinline__ void sh_basis64(double x, double y, double z, double* Y) {
  const double pi = 3.14159265358979323846;
  Y[0] = 0.5 / sqrt(pi);
  const double c1 = sqrt(3.0 / (4.0 * pi));
  Y[1] = c1 * y; Y[2] = c1 * z; Y[3] = c1 * x;
  const double c2a = sqrt(15.0 / (4.0 * pi)), c2b = sqrt(5.0 / (16.0 * pi)), c2c = sqrt(15.0 / (16.0 * pi));
  Y[4] = c2a * x * y; Y[5] = c2a * y * z; Y[6] = c2b * (3.0 * z * z - 1.0); Y[7] = c2a * x * z;
  Y[8] = c2c * (x * x - y * y);
  const double c3a = sqrt(35.0 / (32.0 * pi)), c3b = sqrt(105.0 / (4.0 * pi)), c3c = sqrt(21.0 / (32.0 * pi));
  const double c3d = sqrt(7.0 / (16.0 * pi)), c3e = sqrt(105.0 / (16.0 * pi));
  Y[9] = c3a * y * (3.0 * x * x - y * y); Y[10] = c3b * x * y * z; Y[11] = c3c * y * (5.0 * z * z - 1.0);
  Y[12] = c3d * z * (5.0 * z * z - 3.0); Y[13] = c3c * x * (5.0 * z * z - 1.0); Y[14] = c3e * z * (x * x - y * y);
  Y[15] = c3a * x * (x * x - 3.0 * y * y);
}

template <typename DT, typename ST>
__global__ void k_render_f64(const __grid_constant__ ViewSet vs, const uint32_t* __restrict__ ranges,
                             const uint32_t* __restrict__ svals, const uint32_t* __restrict__ slot_vox,
                             const float4* __restrict__ geom, const DT* __restrict__ dens, const ST* __restrict__ sh,
                             int sh_nb, const int64_t* __restrict__ pixels, int64_t n_px, double t_stop,
                             int segment, const uint32_t* __restrict__ vidx, double* __restrict__ rgb_out,
                             double* __restrict__ T_out) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n_px) return;
  const long long gp = pixels[q];
  int view = 0;
  while (view + 1 < vs.n && gp >= vs.v[view + 1].pix_off) ++view;
  const DevView& c = vs.v[view];
  const long long loc = gp - c.pix_off;
  const int px = (int)(loc % c.W), py = (int)(loc / c.W);
  const int ts = vs.ts;
  const int gtile = c.tile_off + (py / ts) * c.tiles_x + px / ts;
  double o[3], d[3];
  for (int k = 0; k < 3; ++k)
    o[k] = -((double)c.R[k] * c.t[0] + (double)c.R[3 + k] * c.t[1] + (double)c.R[6 + k] * c.t[2]);
  const double dcx = ((double)px + 0.5 - (double)c.cx) / (double)c.fx;
  const double dcy = ((double)py + 0.5 - (double)c.cy) / (double)c.fy;
  double nn = 0.0;
  for (int k = 0; k < 3; ++k) {
    d[k] = (double)c.R[k] * dcx + (double)c.R[3 + k] * dcy + (double)c.R[6 + k];
    nn += d[k] * d[k];
  }
  nn = sqrt(nn);
  for (int k = 0; k < 3; ++k) d[k] /= nn;
  const double t_near = (double)c.z_near * nn;  // camera depth z_near along this ray
  double T = 1.0, cr = 0.0, cg = 0.0, cb = 0.0;
  const uint32_t start = ranges[2 * gtile], end = ranges[2 * gtile + 1];
  for (uint32_t e = start; e < end; ++e) {
    const uint32_t vox = slot_vox[svals[e]];
    const float4 g = geom[vox];
    const double h = (double)g.w, cc[3] = {(double)g.x, (double)g.y, (double)g.z};
    double lo_t = t_near, hi_t = 1e300;
    bool miss = false;
    for (int a = 0; a < 3; ++a) {
      const double lo = cc[a] - h, hi = cc[a] + h;
      if (d[a] == 0.0) {
        if (o[a] < lo || o[a] > hi) miss = true;
        continue;
      }
      const double t1 = (lo - o[a]) / d[a], t2 = (hi - o[a]) / d[a];
      lo_t = fmax(lo_t, fmin(t1, t2));
      hi_t = fmin(hi_t, fmax(t1, t2));
    }
    if (miss || !(hi_t - lo_t > 0.0)) continue;
    const double l = hi_t - lo_t, tm = 0.5 * (lo_t + hi_t);
    // the trilinear field at the midpoint, or its mean over the chord (Simpson, exact for the cubic)
    const double ts3[3] = {tm, lo_t, hi_t}, ws3[3] = {segment ? 4.0 / 6.0 : 1.0, 1.0 / 6.0, 1.0 / 6.0};
    double sr = 0.0;
    for (int q3 = 0; q3 < (segment ? 3 : 1); ++q3) {
      double u[3];
      for (int a = 0; a < 3; ++a)
        u[a] = fmin(fmax((o[a] + ts3[q3] * d[a] - (cc[a] - h)) / (2.0 * h), 0.0), 1.0);
      for (int i = 0; i < 8; ++i) {
        const double w =
            ((i & 1) ? u[0] : 1.0 - u[0]) * ((i & 2) ? u[1] : 1.0 - u[1]) * ((i & 4) ? u[2] : 1.0 - u[2]);
        const size_t di = vidx ? (size_t)vidx[8 * (size_t)vox + i] : 8 * (size_t)vox + i;
        sr += ws3[q3] * w * (double)to_f32(dens[di]);
      }
    }
    const double sigma = fmax(sr, 0.0);
    const double alpha = -expm1(-sigma * l);
    double dir[3] = {cc[0] - o[0], cc[1] - o[1], cc[2] - o[2]};
    const double dn = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (int k = 0; k < 3; ++k) dir[k] = dn > 0.0 ? dir[k] / dn : (k == 2 ? 1.0 : 0.0);
    double Y[16];
    sh_basis64(dir[0], dir[1], dir[2], Y);
    double col[3] = {0.5, 0.5, 0.5};
    for (int j = 0; j < sh_nb; ++j)
      for (int ch = 0; ch < 3; ++ch) col[ch] += (double)to_f32(sh[48 * (size_t)vox + 3 * j + ch]) * Y[j];
    const double w = T * alpha;
    cr += w * fmax(col[0], 0.0);
    cg += w * fmax(col[1], 0.0);
    cb += w * fmax(col[2], 0.0);
    T *= exp(-sigma * l);
    if (T < t_stop) break;
  }
  rgb_out[3 * q + 0] = cr;
  rgb_out[3 * q + 1] = cg;
  rgb_out[3 * q + 2] = cb;
  if (T_out) T_out[q] = T;
}

// ------------------------------------------------------------------ host side
static lv_status check_common(const lv_voxels* vox, const lv_camera* cams, int nv, const lv_raster_opts* o) {
  if (!vox || !cams || !o) { set_error("null argument"); return LV_ERR_INVALID_ARG; }
  if (nv < 1 || nv > LV_MAX_VIEWS) { set_error("n_views %d outside [1, %d]", nv, LV_MAX_VIEWS); return LV_ERR_INVALID_ARG; }
  if (vox->n < 0 || vox->n > 0x7fffffffLL) { set_error("voxel count %lld out of range", (long long)vox->n); return LV_ERR_INVALID_ARG; }
  if (vox->n > 0 && (!vox->geom || !vox->density || !vox->sh)) { set_error("null voxel array"); return LV_ERR_INVALID_ARG; }
  if (vox->density_dtype != LV_F32 && vox->density_dtype != LV_F16) { set_error("density dtype must be F32 or F16"); return LV_ERR_INVALID_ARG; }
  if (vox->sh_dtype != LV_F32 && vox->sh_dtype != LV_BF16) { set_error("sh dtype must be F32 or BF16"); return LV_ERR_INVALID_ARG; }
  if (vox->sh_degree < 0 || vox->sh_degree > 3) { set_error("sh_degree must be 0..3"); return LV_ERR_INVALID_ARG; }
  if (vox->vidx && ((uintptr_t)vox->vidx & 15)) { set_error("vidx must be 16-byte aligned"); return LV_ERR_INVALID_ARG; }
  if (o->tile != 8 && o->tile != 16 && o->tile != 32) { set_error("tile must be 8, 16 or 32"); return LV_ERR_INVALID_ARG; }
  if (o->batch != 32 && o->batch != 64 && o->batch != 128) { set_error("batch must be 32, 64 or 128"); return LV_ERR_INVALID_ARG; }
  if (o->tile == 32 && o->batch == 128) {
    set_error("batch 128 with 32x32 tiles needs more than 227 KB of shared memory per block");
    return LV_ERR_UNSUPPORTED;
  }
  if (!(o->t_stop >= 0.f && o->t_stop < 1.f)) { set_error("t_stop must be in [0, 1)"); return LV_ERR_INVALID_ARG; }
  if (o->persistent_sms < 0) { set_error("persistent_sms must be >= 0"); return LV_ERR_INVALID_ARG; }
  int64_t tiles = 0, pixels = 0;
  for (int i = 0; i < nv; ++i) {
    const lv_camera& c = cams[i];
    if (c.width < 1 || c.height < 1 || c.width > 32768 || c.height > 32768) { set_error("view %d: bad size", i); return LV_ERR_INVALID_ARG; }
    if (!(c.fx > 0.f && c.fy > 0.f && c.z_near > 0.f)) { set_error("view %d: fx, fy, z_near must be > 0", i); return LV_ERR_INVALID_ARG; }
    tiles += (int64_t)((c.width + o->tile - 1) / o->tile) * ((c.height + o->tile - 1) / o->tile);
    pixels += (int64_t)c.width * c.height;
  }
  if (tiles > 0x7fffffffLL || pixels > 0xfffffffeLL) { set_error("too many tiles or pixels"); return LV_ERR_INVALID_ARG; }
  if (o->pixel_id_base < 0 || o->pixel_id_base + pixels > 0xfffffffeLL) {
    set_error("pixel_id_base %lld: the pixel ids must stay in [0, 2^32 - 1)", (long long)o->pixel_id_base);
    return LV_ERR_INVALID_ARG;
  }
  if (vox->n * nv > 0x7fffffffLL) { set_error("voxels x views exceeds 2^31"); return LV_ERR_INVALID_ARG; }
  return LV_OK;
}

static lv_status finish(lv_status st, uint32_t flags, int32_t* d_status, cudaStream_t s, const char* what) {
  if (st != LV_OK) return st;
  lv_status e = cuda_check(cudaGetLastError(), what);
  if (e != LV_OK) return e;
  if (flags & LV_FLAG_SYNC_CHECK) {
    e = cuda_check(cudaStreamSynchronize(s), what);
    if (e != LV_OK) return e;
    int32_t h = 0;
    e = cuda_check(cudaMemcpy(&h, d_status, sizeof(h), cudaMemcpyDeviceToHost), "status readback");
    if (e != LV_OK) return e;
    if (h != 0) { set_error("%s: device reported status %d", what, h); return (lv_status)h; }
  }
  return LV_OK;
}

// resident blocks of a persistent composite (once per kernel)
template <typename K>
static int persistent_blocks(K kernel, int threads, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  return (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
}

// a persistent grid of pb blocks over all SMs, cut to sm_limit SMs (0: all)
// the SM count, and the cut for a persistent grid limited to sm_limit SMs (0: no limit)
static void sm_limits(int sm_limit, int dev, int* sms, int* sm_cut) {
  cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  *sm_cut = (sm_limit > 0 && *sms > 0 && sm_limit < *sms) ? sm_limit : 0;
}

template <int TS, bool SEG, bool PERSIST, int CH>
static void launch_fwd_t(int64_t tiles, cudaStream_t s, const ViewSet& vs, const FwdWs& w, const uint32_t* sv,
                         float t_stop, const lv_fwd_out* out, int sm_limit) {
  const size_t smem = fwd_slice(CH) * (TS * TS / 32);
  static int pblocks[64];  // per device
  static std::atomic<unsigned long long> done{0};
  const int dev = current_device();
  once_per_device(done, [&] {
    cudaFuncSetAttribute(k_fwd<TS, SEG, PERSIST, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (PERSIST && dev < 64) pblocks[dev] = persistent_blocks(k_fwd<TS, SEG, PERSIST, CH>, TS * TS, smem);
  });
  const int pb = dev < 64 ? pblocks[dev] : persistent_blocks(k_fwd<TS, SEG, PERSIST, CH>, TS * TS, smem);
  int sms = 0, sm_cut = 0;
  sm_limits(sm_limit, dev, &sms, &sm_cut);
  const uint32_t n_items = (uint32_t)tiles * (TS * TS / 32);
  unsigned grid = (unsigned)tiles;
  if (PERSIST) grid = (unsigned)(tiles < pb ? tiles : pb);  // work[0] was cleared at the start of the forward
  k_fwd<TS, SEG, PERSIST, CH><<<grid, TS * TS, smem, s>>>(vs, w.ranges, sv, w.rec, w.rec_bb, w.slot_vox, t_stop,
                                                       out->rgb, out->depth, out->T, out->n_contrib,
                                                       out->n_samples, w.tau, out->wmax_packed, w.work, n_items,
                                                       sm_cut, sms, w.work + 8);
}

template <int TS, bool SEG, bool PERSIST, int CH>
static void launch_bwd_t(int64_t tiles, cudaStream_t s, const ViewSet& vs, const FwdWs& w, const uint32_t* sv,
                         const lv_fwd_out* fwd, const float* gC, const float* gD, const float* gT, float* dd,
                         int sm_limit, const LfFuse& lf) {
  const size_t smem = bwd_slice(CH) * (TS * TS / 32);
  static int pblocks[64];  // per device
  static std::atomic<unsigned long long> done{0};
  const int dev = current_device();
  once_per_device(done, [&] {
    cudaFuncSetAttribute(k_bwd<TS, SEG, PERSIST, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (PERSIST && dev < 64) pblocks[dev] = persistent_blocks(k_bwd<TS, SEG, PERSIST, CH>, TS * TS, smem);
  });
  const int pb = dev < 64 ? pblocks[dev] : persistent_blocks(k_bwd<TS, SEG, PERSIST, CH>, TS * TS, smem);
  int sms = 0, sm_cut = 0;
  sm_limits(sm_limit, dev, &sms, &sm_cut);
  const uint32_t n_items = (uint32_t)tiles * (TS * TS / 32);
  unsigned grid = (unsigned)tiles;
  if (PERSIST) {
    zero_async(s, w.work + 1, sizeof(unsigned int), w.work + 9, sizeof(unsigned int));
    grid = (unsigned)(tiles < pb ? tiles : pb);
  }
  k_bwd<TS, SEG, PERSIST, CH><<<grid, TS * TS, smem, s>>>(vs, w.ranges, sv, w.rec, w.rec_bb, w.slot_vox, fwd->T,
                                                       w.tau, fwd->n_contrib, gC, gD, gT, dd, w.d_rgb, w.work + 1,
                                                       n_items, sm_cut, sms, w.work + 9, lf);
}

// tile size, batch, density model (midpoint, or the exact-segment variant) and scheduling
// (one block per tile, or persistent warps on a work counter) from the options; a batch of
// 128 needs more than the 227 KB of shared memory of a block for 32 x 32 tiles (refused by
// check_common)
// The tile-sorted pairs are in (k0, v0) after an even number of digit passes,
// else in (k1, v1); the other pair of arrays is scratch.  One warp per tile
// first (short lists, ranges, the lists of longer tiles), then persistent
// blocks over the medium tiles and the long tiles' chunks, then the merge.
static void launch_tile_sort(const FwdWs& w, int64_t tiles, int64_t pair_cap, cudaStream_t s) {
  static std::atomic<unsigned long long> attr_done{0};
  static int sort_blocks[64], merge_blocks[64];
  int dev = 0;
  cudaGetDevice(&dev);
  once_per_device(attr_done, [dev] {
    cudaFuncSetAttribute(k_tile_sort_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileSortWarpSmem));
    cudaFuncSetAttribute(k_tile_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileSortSmem));
    cudaFuncSetAttribute(k_tile_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileMergeSmem));
    if (dev < 64) {
      sort_blocks[dev] = persistent_blocks(k_tile_sort, TS_THREADS, sizeof(TileSortSmem));
      merge_blocks[dev] = persistent_blocks(k_tile_merge, TS_THREADS, sizeof(TileMergeSmem));
    }
  });
  const int ns = dev < 64 ? sort_blocks[dev] : persistent_blocks(k_tile_sort, TS_THREADS, sizeof(TileSortSmem));
  const int nmg = dev < 64 ? merge_blocks[dev] : persistent_blocks(k_tile_merge, TS_THREADS, sizeof(TileMergeSmem));
  const int passes = sort_passes(tile_bits(tiles));
  const bool odd = passes & 1, ready = passes > 0;
  uint32_t* sv = odd ? w.v1 : w.v0;
  uint32_t* xk = odd ? w.k0 : w.k1;
  uint32_t* xv = odd ? w.v0 : w.v1;
  const unsigned wblocks = (unsigned)((tiles + TW_WARPS - 1) / TW_WARPS);
  k_tile_sort_warp<<<wblocks, TW_WARPS * 32, sizeof(TileSortWarpSmem), s>>>(sv, w.s_dkey, w.counters, pair_cap, ready,
                                                                          tiles, w.ranges, w.mid_tiles, w.work + 4,
                                                                          w.chunks, w.work + 2, w.long_tiles,
                                                                          w.work + 6);
  k_tile_sort<<<(unsigned)ns, TS_THREADS, sizeof(TileSortSmem), s>>>(sv, xk, xv, w.s_dkey, w.ranges, w.mid_tiles,
                                                                     w.work + 4, w.chunks, w.work + 2, w.work + 5);
  k_tile_merge<<<(unsigned)nmg, TS_THREADS, sizeof(TileMergeSmem), s>>>(sv, xk, xv, w.ranges, w.long_tiles,
                                                                        w.work + 6, w.work + 3);
  count_launch(3);
}

static void launch_fwd(const lv_raster_opts* o, int64_t tiles, cudaStream_t s, const ViewSet& vs, const FwdWs& w,
                       const uint32_t* sv, const lv_fwd_out* out) {
  const bool seg = (o->flags & LV_FLAG_EXACT_SEGMENT) != 0, per = (o->flags & LV_FLAG_PERSISTENT) != 0;
  const int sml = per ? o->persistent_sms : 0;
#define LV_FWD_CH(TS, CH)                                                                           \
  if (seg && per) launch_fwd_t<TS, true, true, CH>(tiles, s, vs, w, sv, o->t_stop, out, sml);   \
  else if (seg) launch_fwd_t<TS, true, false, CH>(tiles, s, vs, w, sv, o->t_stop, out, 0);      \
  else if (per) launch_fwd_t<TS, false, true, CH>(tiles, s, vs, w, sv, o->t_stop, out, sml);    \
  else launch_fwd_t<TS, false, false, CH>(tiles, s, vs, w, sv, o->t_stop, out, 0)
#define LV_FWD(TS)                                   \
  if (o->batch == 64) { LV_FWD_CH(TS, 64); }         \
  else if (o->batch == 128) { LV_FWD_CH(TS, 128); }  \
  else { LV_FWD_CH(TS, 32); }
  if (o->tile == 8) { LV_FWD(8) }
  else if (o->tile == 16) { LV_FWD(16) }
  else if (o->batch == 64) { LV_FWD_CH(32, 64); }
  else { LV_FWD_CH(32, 32); }
#undef LV_FWD
#undef LV_FWD_CH
}

static void launch_bwd(const lv_raster_opts* o, int64_t tiles, cudaStream_t s, const ViewSet& vs, const FwdWs& w,
                       const uint32_t* sv, const lv_fwd_out* fwd, const float* gC, const float* gD, const float* gT,
                       float* dd, const LfFuse& lf) {
  const bool seg = (o->flags & LV_FLAG_EXACT_SEGMENT) != 0, per = (o->flags & LV_FLAG_PERSISTENT) != 0;
  const int sml = per ? o->persistent_sms : 0;
#define LV_BWD_CH(TS, CH)                                                                                 \
  if (seg && per) launch_bwd_t<TS, true, true, CH>(tiles, s, vs, w, sv, fwd, gC, gD, gT, dd, sml, lf);    \
  else if (seg) launch_bwd_t<TS, true, false, CH>(tiles, s, vs, w, sv, fwd, gC, gD, gT, dd, 0, lf);       \
  else if (per) launch_bwd_t<TS, false, true, CH>(tiles, s, vs, w, sv, fwd, gC, gD, gT, dd, sml, lf);     \
  else launch_bwd_t<TS, false, false, CH>(tiles, s, vs, w, sv, fwd, gC, gD, gT, dd, 0, lf)
#define LV_BWD(TS)                                   \
  if (o->batch == 64) { LV_BWD_CH(TS, 64); }         \
  else if (o->batch == 128) { LV_BWD_CH(TS, 128); }  \
  else { LV_BWD_CH(TS, 32); }
  if (o->tile == 8) { LV_BWD(8) }
  else if (o->tile == 16) { LV_BWD(16) }
  else if (o->batch == 64) { LV_BWD_CH(32, 64); }
  else { LV_BWD_CH(32, 32); }
#undef LV_BWD
#undef LV_BWD_CH
}

}  // namespace lv

using namespace lv;

extern "C" size_t lv_forward_workspace_size(int64_t n, const lv_camera* cams, int n_views, const lv_raster_opts* opts,
                                            int64_t pair_capacity) {
  if (!cams || !opts || n_views < 1 || n_views > LV_MAX_VIEWS || n < 0 || pair_capacity < 0 ||
      pair_capacity > 0xffffffffLL)
    return 0;
  if (opts->tile != 8 && opts->tile != 16 && opts->tile != 32) return 0;
  ViewSet vs;
  int64_t tiles, pixels;
  make_views(cams, n_views, opts->tile, &vs, &tiles, &pixels);
  return carve_fwd(nullptr, n, n_views, tiles, pixels, pair_capacity).bytes;
}

extern "C" lv_status lv_rasterize_forward(const lv_voxels* vox, const lv_camera* cams, int n_views,
                                          const lv_raster_opts* opts, const lv_fwd_out* out, void* workspace,
                                          size_t ws_bytes, int64_t pair_capacity, int32_t* d_status, void* stream) {
  lv_status st = check_common(vox, cams, n_views, opts);
  if (st != LV_OK) return st;
  if (!out || !out->rgb || !out->T || !out->n_contrib) { set_error("rgb, T and n_contrib outputs are required"); return LV_ERR_INVALID_ARG; }
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  if (pair_capacity < 0 || pair_capacity > 0xffffffffLL) { set_error("pair_capacity out of range"); return LV_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  ViewSet vs;
  int64_t tiles, pixels;
  make_views(cams, n_views, opts->tile, &vs, &tiles, &pixels);
  vs.id_base = opts->pixel_id_base;
  FwdWs w = carve_fwd(workspace, vox->n, n_views, tiles, pixels, pair_capacity);
  if (ws_bytes < w.bytes) { set_error("workspace %zu bytes < required %zu", ws_bytes, w.bytes); return LV_ERR_WORKSPACE; }
  if (!d_status) d_status = w.status;
  const int64_t n = vox->n, items = n * n_views;
  // counters, the fallback status word, the work counters of the persistent kernels and the
  // sort by tile's digit counts, which k_emit accumulates (k_tile_sort_warp writes every tile's range)
  const SortCountTargets sc = sort_count_targets(w.sort_tmp, pair_capacity);
  const int passes = std::min(sort_passes(tile_bits(tiles)), 4);
  zero_async(s, w.counters, 8 * sizeof(unsigned long long), d_status == w.status ? w.status : nullptr,
             sizeof(int32_t), w.work, 16 * sizeof(unsigned int), sc.counts, sc.zero_bytes);
  if (items > 0) {
    int blocks = (int)((items + 255) / 256);
    const unsigned emit_blocks = (unsigned)(((n + 255) / 256) * n_views);  // (voxel range, view) blocks
    k_bin<<<blocks, 256, 0, s>>>((const float4*)vox->geom, n, vs, w.cnt, w.vis, w.rect, w.pbox, w.dkey, out->z_min,
                                 out->delta_min, out->seen);
    if (out->stats_event) cudaEventRecord((cudaEvent_t)out->stats_event, s);  // statistics final
    scan2(w.cnt, w.vis, items, w.poff, w.slot, w.counters, w.scan_tmp, s);
    const int nb = (vox->sh_degree + 1) * (vox->sh_degree + 1);
#define LV_EMIT(DT, ST)                                                                                             \
  k_emit<DT, ST><<<emit_blocks, 256, 0, s>>>((const float4*)vox->geom, (const DT*)vox->density, (const ST*)vox->sh, \
                                             nb, n, vs, w.cnt, w.rect, w.pbox, w.rec_bb, w.slot_vox, w.dkey,          \
                                             w.slot, w.poff, w.counters, pair_capacity, w.k0, w.v0, d_status,         \
                                             (uint2*)w.ranges, tiles, sc, passes, w.rec, w.d_rgb, w.s_dkey,   \
                                             vox->vidx)
    if (vox->density_dtype == LV_F32 && vox->sh_dtype == LV_F32) LV_EMIT(float, float);
    else if (vox->density_dtype == LV_F16 && vox->sh_dtype == LV_F32) LV_EMIT(__half, float);
    else if (vox->density_dtype == LV_F32 && vox->sh_dtype == LV_BF16) LV_EMIT(float, __nv_bfloat16);
    else LV_EMIT(__half, __nv_bfloat16);
#undef LV_EMIT
    count_launch(2);
  } else if (out->stats_event) {
    cudaEventRecord((cudaEvent_t)out->stats_event, s);  // no voxel: nothing to bin
  }
  // stable sort by tile: each tile's list stays in item order; the last pass notes every tile's range
  radix_sort_pairs(w.k0, w.v0, w.k0, w.v0, w.k1, w.v1, w.sort_tmp, w.counters, pair_capacity, tile_bits(tiles),
                   d_status, s, w.ranges, items > 0);
  // each tile's range, and its list front to back
  launch_tile_sort(w, tiles, pair_capacity, s);
  const uint32_t* sv = sorted_pair_slots(w, tiles);
  if (out->composite_event) {
    // a timing mark: inside a stream capture it becomes an event record node of the graph
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags((cudaEvent_t)out->composite_event, s, cudaEventRecordExternal);
    else
      cudaEventRecord((cudaEvent_t)out->composite_event, s);
  }
  launch_fwd(opts, tiles, s, vs, w, sv, out);
  count_launch(2);
  return finish(LV_OK, opts->flags, d_status, s, "lv_rasterize_forward");
}

namespace lv {
namespace {
// four voxels per thread: one 32-byte store of w_max, 16-byte stores of the
// depths, one 4-byte store of seen (scalar at a ragged end or misaligned arrays)
__global__ void k_reset_stats(int64_t n, unsigned long long* wmax, float* z_min, float* delta_min, uint8_t* seen) {
  const float inf = __int_as_float(0x7f800000);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
  const bool vec = (((uintptr_t)wmax | (uintptr_t)z_min | (uintptr_t)delta_min) & 15) == 0 &&
                   ((uintptr_t)seen & 3) == 0;
  for (int64_t i0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 4; i0 < n; i0 += stride) {
    if (vec && i0 + 3 < n) {
      if (wmax) {
        ((uint4*)(wmax + i0))[0] = make_uint4(0u, 0u, 0u, 0u);
        ((uint4*)(wmax + i0))[1] = make_uint4(0u, 0u, 0u, 0u);
      }
      if (z_min) *(float4*)(z_min + i0) = make_float4(inf, inf, inf, inf);
      if (delta_min) *(float4*)(delta_min + i0) = make_float4(inf, inf, inf, inf);
      if (seen) *(uint32_t*)(seen + i0) = 0u;
    } else {
      for (int64_t i = i0; i < n && i < i0 + 4; ++i) {
        if (wmax) wmax[i] = 0ull;
        if (z_min) z_min[i] = inf;
        if (delta_min) delta_min[i] = inf;
        if (seen) seen[i] = 0;
      }
    }
  }
}
}  // namespace
}  // namespace lv

extern "C" lv_status lv_reset_stats(int64_t n, unsigned long long* wmax_packed, float* z_min, float* delta_min,
                                    uint8_t* seen, void* stream) {
  if (n < 0) { set_error("bad voxel count"); return LV_ERR_INVALID_ARG; }
  if (n == 0) return LV_OK;
  int64_t blocks = (n / 4 + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 4 * 1216) blocks = 4 * 1216;
  k_reset_stats<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, wmax_packed, z_min, delta_min, seen);
  count_launch(1);
  return cuda_check(cudaGetLastError(), "lv_reset_stats");
}

extern "C" lv_status lv_workspace_counters(const void* workspace, size_t ws_bytes, int64_t* out2, void* stream) {
  if (!workspace || !out2 || ws_bytes < 64) { set_error("bad arguments"); return LV_ERR_INVALID_ARG; }
  unsigned long long h[2];
  cudaStream_t s = (cudaStream_t)stream;
  lv_status e = cuda_check(cudaMemcpyAsync(h, workspace, sizeof(h), cudaMemcpyDeviceToHost, s), "counters");
  if (e != LV_OK) return e;
  e = cuda_check(cudaStreamSynchronize(s), "counters");
  if (e != LV_OK) return e;
  out2[0] = (int64_t)h[0];
  out2[1] = (int64_t)h[1];
  return LV_OK;
}

static lv_status launch_sh_bwd(const lv_voxels* vox, const ViewSet& vs, const FwdWs& w, float* d_sh, int accumulate,
                               cudaStream_t s) {
  const int64_t n = vox->n;
  if (n == 0) return LV_OK;
  const int nb = (vox->sh_degree + 1) * (vox->sh_degree + 1);
  const int blocks = (int)((n + 127) / 128);  // 4 warps x 32 voxels
  k_sh_bwd<<<blocks, 128, 0, s>>>(w.rec, nb, n, vs, w.vis, w.slot, w.d_rgb, d_sh, accumulate);
  count_launch(1);
  return LV_OK;
}

extern "C" lv_status lv_rasterize_backward(const lv_voxels* vox, const lv_camera* cams, int n_views,
                                           const lv_raster_opts* opts, const lv_fwd_out* fwd, void* workspace,
                                           size_t ws_bytes, int64_t pair_capacity, const float* dL_drgb,
                                           const float* dL_ddepth, const float* dL_dT, float* d_density, float* d_sh,
                                           int accumulate, int32_t* d_status, void* stream) {
  lv_status st = check_common(vox, cams, n_views, opts);
  if (st != LV_OK) return st;
  if (!fwd || !fwd->T || !fwd->n_contrib || !d_density || (!dL_drgb && !fwd->lf_workspace)) { set_error("null argument"); return LV_ERR_INVALID_ARG; }
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  if (pair_capacity < 0 || pair_capacity > 0xffffffffLL) { set_error("pair_capacity out of range"); return LV_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  ViewSet vs;
  int64_t tiles, pixels;
  make_views(cams, n_views, opts->tile, &vs, &tiles, &pixels);
  FwdWs w = carve_fwd(workspace, vox->n, n_views, tiles, pixels, pair_capacity);
  if (ws_bytes < w.bytes) { set_error("workspace %zu bytes < required %zu", ws_bytes, w.bytes); return LV_ERR_WORKSPACE; }
  if (!d_status) d_status = w.status;
  // the LF-weighted loss fused in: dL/drgb from the forward's image, the ground truth and the weights
  LfFuse lf = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (!dL_drgb) {
    if (!fwd->lf_gt || !fwd->rgb) { set_error("the fused LF loss needs lf_gt and the forward's rgb"); return LV_ERR_INVALID_ARG; }
    int32_t wd[LV_MAX_VIEWS], ht[LV_MAX_VIEWS];
    for (int v = 0; v < n_views; ++v) {
      wd[v] = cams[v].width;
      ht[v] = cams[v].height;
    }
    lv_status e = lf_fused_buffers(wd, ht, n_views, fwd->lf_workspace, fwd->lf_ws_bytes, &lf.w, &lf.wsum, &lf.lsum);
    if (e != LV_OK) return e;
    lf.rgb = fwd->rgb;
    lf.gt = fwd->lf_gt;
    lf.dL = fwd->lf_dL;
    if (fwd->lf_wait_event) cudaStreamWaitEvent(s, (cudaEvent_t)fwd->lf_wait_event, 0);  // the weights
  }
  const int64_t n = vox->n;
  const uint32_t* sv = sorted_pair_slots(w, tiles);
  if (!accumulate && n > 0) cudaMemsetAsync(d_density, 0, sizeof(float) * 8 * n, s);
  launch_bwd(opts, tiles, s, vs, w, sv, fwd, dL_drgb, dL_ddepth, dL_dT, d_density, lf);
  count_launch(1);
  if (d_sh) launch_sh_bwd(vox, vs, w, d_sh, accumulate, s);
  return finish(LV_OK, opts->flags, d_status, s, "lv_rasterize_backward");
}

extern "C" lv_status lv_sh_backward(const lv_voxels* vox, const lv_camera* cams, int n_views,
                                    const lv_raster_opts* opts, void* workspace, size_t ws_bytes,
                                    int64_t pair_capacity, float* d_sh, int accumulate, void* stream) {
  lv_status st = check_common(vox, cams, n_views, opts);
  if (st != LV_OK) return st;
  if (!d_sh || !workspace || ((uintptr_t)workspace & 255)) { set_error("bad arguments"); return LV_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  ViewSet vs;
  int64_t tiles, pixels;
  make_views(cams, n_views, opts->tile, &vs, &tiles, &pixels);
  FwdWs w = carve_fwd(workspace, vox->n, n_views, tiles, pixels, pair_capacity);
  if (ws_bytes < w.bytes) { set_error("workspace %zu bytes < required %zu", ws_bytes, w.bytes); return LV_ERR_WORKSPACE; }
  launch_sh_bwd(vox, vs, w, d_sh, accumulate, s);
  return cuda_check(cudaGetLastError(), "lv_sh_backward");
}

extern "C" lv_status lv_unpack_wmax(const unsigned long long* packed, int64_t n, float* w_max, int64_t* argmax,
                                    void* stream) {
  if (n < 0 || (n > 0 && (!packed || !w_max))) { set_error("bad arguments"); return LV_ERR_INVALID_ARG; }
  if (n == 0) return LV_OK;
  k_unpack_wmax<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(packed, n, w_max, argmax);
  count_launch(1);
  return cuda_check(cudaGetLastError(), "lv_unpack_wmax");
}

extern "C" lv_status lv_gather_edge(const int64_t* argmax, int64_t n, const float* edge_map, int64_t n_pix,
                                    float* edge, void* stream) {
  if (n < 0 || n_pix < 0 || (n > 0 && (!argmax || !edge || (n_pix > 0 && !edge_map)))) {
    set_error("bad arguments");
    return LV_ERR_INVALID_ARG;
  }
  if (n == 0) return LV_OK;
  k_gather_edge<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(argmax, n, edge_map, n_pix, edge);
  count_launch(1);
  return cuda_check(cudaGetLastError(), "lv_gather_edge");
}

extern "C" lv_status lv_debug_pairs(int64_t n, const lv_camera* cams, int n_views, const lv_raster_opts* opts,
                                    const void* workspace, size_t ws_bytes, int64_t pair_capacity, uint64_t* keys,
                                    uint32_t* voxel, uint32_t* ranges, void* stream) {
  if (!cams || !opts || !workspace || n_views < 1 || n_views > LV_MAX_VIEWS || n < 0) { set_error("bad arguments"); return LV_ERR_INVALID_ARG; }
  if (opts->tile != 8 && opts->tile != 16 && opts->tile != 32) { set_error("bad tile"); return LV_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  ViewSet vs;
  int64_t tiles, pixels;
  make_views(cams, n_views, opts->tile, &vs, &tiles, &pixels);
  FwdWs w = carve_fwd((void*)workspace, n, n_views, tiles, pixels, pair_capacity);
  if (ws_bytes < w.bytes) { set_error("workspace too small"); return LV_ERR_WORKSPACE; }
  if (keys || voxel) {
    k_debug_pairs<<<608, 256, 0, s>>>(sorted_pair_tiles(w, tiles), sorted_pair_slots(w, tiles), w.slot_vox, w.s_dkey,
                                       w.counters, pair_capacity, keys, voxel);
    count_launch(1);
  }
  if (ranges) cudaMemcpyAsync(ranges, w.ranges, sizeof(uint32_t) * 2 * tiles, cudaMemcpyDeviceToDevice, s);
  return cuda_check(cudaGetLastError(), "lv_debug_pairs");
}

extern "C" lv_status lv_render_pixels_f64(const lv_voxels* vox, const lv_camera* cams, int n_views,
                                          const lv_raster_opts* opts, const void* workspace, size_t ws_bytes,
                                          int64_t pair_capacity, const int64_t* pixels, int64_t n_px, double* rgb,
                                          double* T, void* stream) {
  lv_status st = check_common(vox, cams, n_views, opts);
  if (st != LV_OK) return st;
  if (n_px < 0 || (n_px > 0 && (!pixels || !rgb)) || !workspace) { set_error("bad arguments"); return LV_ERR_INVALID_ARG; }
  if (n_px == 0) return LV_OK;
  cudaStream_t s = (cudaStream_t)stream;
  ViewSet vs;
  int64_t tiles, npix;
  make_views(cams, n_views, opts->tile, &vs, &tiles, &npix);
  FwdWs w = carve_fwd((void*)workspace, vox->n, n_views, tiles, npix, pair_capacity);
  if (ws_bytes < w.bytes) { set_error("workspace too small"); return LV_ERR_WORKSPACE; }
  const uint32_t* sv = sorted_pair_slots(w, tiles);
  const int nb = (vox->sh_degree + 1) * (vox->sh_degree + 1);
  const unsigned grid = (unsigned)((n_px + 127) / 128);
#define LV_F64(DT, ST)                                                                                            \
  k_render_f64<DT, ST><<<grid, 128, 0, s>>>(vs, w.ranges, sv, w.slot_vox, (const float4*)vox->geom,              \
                                            (const DT*)vox->density, (const ST*)vox->sh, nb, pixels, n_px,       \
                                            (double)opts->t_stop, (opts->flags & LV_FLAG_EXACT_SEGMENT) ? 1 : 0,  \
                                            vox->vidx, rgb, T)
  if (vox->density_dtype == LV_F32 && vox->sh_dtype == LV_F32) LV_F64(float, float);
  else if (vox->density_dtype == LV_F16 && vox->sh_dtype == LV_F32) LV_F64(__half, float);
  else if (vox->density_dtype == LV_F32 && vox->sh_dtype == LV_BF16) LV_F64(float, __nv_bfloat16);
  else LV_F64(__half, __nv_bfloat16);
#undef LV_F64
  count_launch(1);
  return cuda_check(cudaGetLastError(), "lv_render_pixels_f64");
}

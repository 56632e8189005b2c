/*
 * lv_oracle.c -- plain, slow CPU oracle for the LiteVoxel rasterizer hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library; both sides are written independently from the paper.
 *
 * What each part follows (LiteVoxel, arXiv 2511.02510):
 *   ora_render / ora_render_backward : Sec. III, Eq. 1 (rays), Eq. 2-4 (front-to-back
 *       alpha compositing), Eq. 5 (w_max), delta_v "local inter-ray spacing".
 *       FP64, one ray per pixel, every voxel the ray crosses, ordered by the
 *       depth key.  The backward pass is plain reverse-mode of Eq. 2-4 over
 *       stored per-sample values.
 *   ora_pairs   : the (tile, depth-key) pair list and the per-voxel depth
 *       statistics, FP32 with a fixed operation order (the binning step of the
 *       "differentiable tile rasterizer", Sec. II-A / Fig. 1).
 *   ora_prune   : Sec. IV-C, Eq. 11-12 (per-bin empirical-CDF quantile) with
 *       guard i (EMA + hysteresis), guard ii (keep-halo) and guard iii
 *       (per-step cap); the annealed, near/far-relaxed q_b; Eq. 14 depth
 *       normalisation for the bins, optionally with running percentiles.
 *       FP32, fixed operation order.
 *   ora_subdivide : Sec. IV-D, Eq. 13 (footprint eligibility), Eq. 14-16
 *       (depth-normalised far bias on the usefulness score), budgeted top-k
 *       and optimizer-state re-initialisation.  FP32, fixed operation order.
 *   ora_lf_loss : Sec. IV-B, Eq. 7-10 and Eq. 18 (inverse-Sobel weight, mean
 *       normalisation, gamma ramp).  FP64.
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *   - exact segment integration (the variant, segment = 1): sigma = max(0,
 *     mean of the trilinear field over the chord), Simpson's rule being exact
 *     for the cubic profile of a trilinear field along a line;
 *   - opacity: 8 corner densities per voxel, sigma = max(0, trilinear at the
 *     segment midpoint), alpha = 1 - exp(-sigma * l), l = ray-box chord length
 *     with t >= 0;
 *   - order along the ray: camera-space z of the voxel centre (FP32 bits),
 *     ties by voxel id;
 *   - a pixel stops after the first sample whose T falls below t_stop;
 *   - depth = sum_k w_k * t_mid_k;
 *   - colour: real SH of degree <= 3 evaluated towards the voxel centre,
 *     c = max(0, sum + 0.5);
 *   - near-plane clipping: a ray's chord starts where its camera depth
 *     reaches z_near (Eq. 1's t >= 0 becomes z_cam >= z_near), so a voxel all
 *     of whose corners have camera z < z_near is culled, and one that crosses
 *     the plane covers the tiles of its part beyond it;
 *   - w_max ties go to the smallest global pixel id;
 *   - delta_v = max(z_v, z_near) / f_x, z_v the camera depth of the centre,
 *     both as minima over views.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared.
 * -ffp-contract=off is required: the FP32 parts must round every operation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int32_t width, height;
  float fx, fy, cx, cy;
  float w2c[12]; /* row-major 3x4 [R | t]: x_cam = R x_world + t */
  float z_near;
} ora_cam;

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static int ora_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int ora_num_threads(void) { return ora_threads(); }

static int ora_tid(void) {
#ifdef _OPENMP
  return omp_get_thread_num();
#else
  return 0;
#endif
}

/* ceil(a * b / 1e6) for non-negative integers */
static int64_t ppm_ceil(int64_t ppm, int64_t n) { return (ppm * n + 999999) / 1000000; }
static int64_t ppm_floor(int64_t ppm, int64_t n) { return (ppm * n) / 1000000; }

/* order-preserving map from float bits to unsigned (negative floats first) */
static uint32_t f32_order_key(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

static uint32_t f32_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

/* ------------------------------------------------------------------ */
/* real spherical harmonics up to degree 3 (orthonormal on the sphere) */
/* ------------------------------------------------------------------ */

/*
 * Y_l^m for the real basis, written from the associated Legendre functions:
 *   l=0: 1/(2 sqrt(pi))
 *   l=1: sqrt(3/(4pi)) * {y, z, x}
 *   l=2: sqrt(15/(4pi)) {xy, yz, xz}, sqrt(5/(16pi)) (3z^2-1), sqrt(15/(16pi)) (x^2-y^2)
 *   l=3: sqrt(35/(32pi)) y(3x^2-y^2), sqrt(105/(4pi)) xyz, sqrt(21/(32pi)) y(5z^2-1),
 *        sqrt(7/(16pi)) z(5z^2-3), sqrt(21/(32pi)) x(5z^2-1), sqrt(105/(16pi)) z(x^2-y^2),
 *        sqrt(35/(32pi)) x(x^2-3y^2)
 */
void ora_sh_basis(const double* dir, double* Y) {
  const double pi = 3.14159265358979323846;
  double x = dir[0], y = dir[1], z = dir[2];
  Y[0] = 0.5 / sqrt(pi);
  double c1 = sqrt(3.0 / (4.0 * pi));
  Y[1] = c1 * y;
  Y[2] = c1 * z;
  Y[3] = c1 * x;
  double c2a = sqrt(15.0 / (4.0 * pi));
  double c2b = sqrt(5.0 / (16.0 * pi));
  double c2c = sqrt(15.0 / (16.0 * pi));
  Y[4] = c2a * x * y;
  Y[5] = c2a * y * z;
  Y[6] = c2b * (3.0 * z * z - 1.0);
  Y[7] = c2a * x * z;
  Y[8] = c2c * (x * x - y * y);
  double c3a = sqrt(35.0 / (32.0 * pi));
  double c3b = sqrt(105.0 / (4.0 * pi));
  double c3c = sqrt(21.0 / (32.0 * pi));
  double c3d = sqrt(7.0 / (16.0 * pi));
  double c3e = sqrt(105.0 / (16.0 * pi));
  Y[9] = c3a * y * (3.0 * x * x - y * y);
  Y[10] = c3b * x * y * z;
  Y[11] = c3c * y * (5.0 * z * z - 1.0);
  Y[12] = c3d * z * (5.0 * z * z - 3.0);
  Y[13] = c3c * x * (5.0 * z * z - 1.0);
  Y[14] = c3e * z * (x * x - y * y);
  Y[15] = c3a * x * (x * x - 3.0 * y * y);
}

static int sh_count(int degree) { return (degree + 1) * (degree + 1); }

/* colour of voxel v seen along unit direction dir; raw[] receives the pre-clamp values */
static void sh_color(const float* sh, int degree, const double* dir, double* rgb, double* raw) {
  double Y[16];
  ora_sh_basis(dir, Y);
  int nb = sh_count(degree);
  for (int c = 0; c < 3; ++c) {
    double s = 0.0;
    for (int j = 0; j < nb; ++j) s += (double)sh[j * 3 + c] * Y[j];
    raw[c] = s + 0.5;
    rgb[c] = raw[c] > 0.0 ? raw[c] : 0.0;
  }
}

/* ------------------------------------------------------------------ */
/* camera                                                              */
/* ------------------------------------------------------------------ */

typedef struct {
  double R[9], t[3], o[3];
  double fx, fy, cx, cy, z_near;
  int W, H;
} cam64;

static void cam_derive(const ora_cam* c, cam64* d) {
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) d->R[r * 3 + k] = (double)c->w2c[r * 4 + k];
    d->t[r] = (double)c->w2c[r * 4 + 3];
  }
  /* camera centre o = -R^T t */
  for (int k = 0; k < 3; ++k)
    d->o[k] = -(d->R[0 * 3 + k] * d->t[0] + d->R[1 * 3 + k] * d->t[1] + d->R[2 * 3 + k] * d->t[2]);
  d->fx = c->fx; d->fy = c->fy; d->cx = c->cx; d->cy = c->cy; d->z_near = c->z_near;
  d->W = c->width; d->H = c->height;
}

/* world-space unit direction of the ray through the centre of pixel (x, y) (Eq. 1); returns
 * t_near, the ray parameter at which the camera depth reaches z_near (near-plane clipping) */
static double cam_ray(const cam64* c, int x, int y, double* d) {
  double dc[3] = {((double)x + 0.5 - c->cx) / c->fx, ((double)y + 0.5 - c->cy) / c->fy, 1.0};
  double n = 0.0;
  for (int k = 0; k < 3; ++k) {
    d[k] = c->R[0 * 3 + k] * dc[0] + c->R[1 * 3 + k] * dc[1] + c->R[2 * 3 + k] * dc[2];
    n += d[k] * d[k];
  }
  n = sqrt(n);
  for (int k = 0; k < 3; ++k) d[k] /= n;
  double dz = c->R[6] * d[0] + c->R[7] * d[1] + c->R[8] * d[2];
  return c->z_near / dz;
}

static void cam_point64(const cam64* c, const double* p, double* q) {
  for (int r = 0; r < 3; ++r)
    q[r] = c->R[r * 3 + 0] * p[0] + c->R[r * 3 + 1] * p[1] + c->R[r * 3 + 2] * p[2] + c->t[r];
}

/* FP32 camera transform with every product and sum rounded, left to right */
static void cam_point32(const ora_cam* c, float X, float Y, float Z, float* q) {
  for (int r = 0; r < 3; ++r) {
    float a = c->w2c[r * 4 + 0] * X;
    float b = c->w2c[r * 4 + 1] * Y;
    float e = c->w2c[r * 4 + 2] * Z;
    float s = a + b;
    s = s + e;
    q[r] = s + c->w2c[r * 4 + 3];
  }
}

/* ------------------------------------------------------------------ */
/* FP32 binning rule: cull test, tile rectangle, depth key             */
/* ------------------------------------------------------------------ */

typedef struct {
  int culled;       /* all 8 corners in front of the near plane */
  int tx0, tx1, ty0, ty1;
  int64_t count;    /* tiles covered */
  float zc;         /* camera z of the centre */
} bin32;

static void bin_voxel32(const float* g, const ora_cam* c, int ts, bin32* b) {
  int tiles_x = (c->width + ts - 1) / ts, tiles_y = (c->height + ts - 1) / ts;
  float cx = g[0], cy = g[1], cz = g[2], h = g[3];
  float q[3];
  cam_point32(c, cx, cy, cz, q);
  b->zc = q[2];
  int n_front = 0;
  float umin = 0, umax = 0, vmin = 0, vmax = 0;
  int have = 0;
  float px[8], py[8], pz[8];
  for (int i = 0; i < 8; ++i) {
    float X = (i & 1) ? cx + h : cx - h;
    float Y = (i & 2) ? cy + h : cy - h;
    float Z = (i & 4) ? cz + h : cz - h;
    float p[3];
    cam_point32(c, X, Y, Z, p);
    px[i] = p[0]; py[i] = p[1]; pz[i] = p[2];
    if (p[2] >= c->z_near) {
      ++n_front;
      float iz = 1.0f / p[2]; /* one correctly rounded reciprocal per corner */
      float rx = p[0] * iz;
      float ry = p[1] * iz;
      float u = c->fx * rx;
      float v = c->fy * ry;
      u = u + c->cx;
      v = v + c->cy;
      if (!have) { umin = umax = u; vmin = vmax = v; have = 1; }
      else { umin = fminf(umin, u); umax = fmaxf(umax, u); vmin = fminf(vmin, v); vmax = fmaxf(vmax, v); }
    }
  }
  b->culled = (n_front == 0);
  if (b->culled) {
    b->tx0 = b->tx1 = b->ty0 = b->ty1 = 0;
    b->count = 0;
    return;
  }
  if (n_front < 8) {
    /* near-plane clipping: the box edges that cross z = z_near add their
       crossing points (edge (i, i|bit), lower index first) */
    for (int i = 0; i < 8; ++i)
      for (int bit = 1; bit < 8; bit <<= 1) {
        if (i & bit) continue;
        int j = i | bit;
        int fi = pz[i] >= c->z_near, fj = pz[j] >= c->z_near;
        if (fi == fj) continue;
        float dz = pz[j] - pz[i];
        float f = (c->z_near - pz[i]) / dz;
        float dx = px[j] - px[i];
        float dy = py[j] - py[i];
        float mx = f * dx;
        float my = f * dy;
        float x = px[i] + mx;
        float y = py[i] + my;
        float rx = x / c->z_near;
        float ry = y / c->z_near;
        float u = c->fx * rx;
        float v = c->fy * ry;
        u = u + c->cx;
        v = v + c->cy;
        umin = fminf(umin, u); umax = fmaxf(umax, u); vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
      }
  }
  float fts = (float)ts;
  float a0 = floorf((umin - 1.0f) / fts), a1 = ceilf((umax + 1.0f) / fts);
  float b0 = floorf((vmin - 1.0f) / fts), b1 = ceilf((vmax + 1.0f) / fts);
  b->tx0 = (int)fminf(fmaxf(a0, 0.0f), (float)tiles_x);
  b->tx1 = (int)fminf(fmaxf(a1, 0.0f), (float)tiles_x);
  b->ty0 = (int)fminf(fmaxf(b0, 0.0f), (float)tiles_y);
  b->ty1 = (int)fminf(fmaxf(b1, 0.0f), (float)tiles_y);
  int64_t wx = b->tx1 - b->tx0, wy = b->ty1 - b->ty0;
  b->count = (wx > 0 && wy > 0) ? wx * wy : 0;
}

typedef struct { uint64_t key; uint32_t val; } kv;

static int kv_cmp(const void* a, const void* b) {
  const kv* x = (const kv*)a;
  const kv* y = (const kv*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->val != y->val) return x->val < y->val ? -1 : 1;
  return 0;
}

/*
 * Sorted (tile, depth-key) pairs for all views, plus per-voxel statistics.
 *   keys[p] = (global_tile << 32) | order_key(z_center); vals[p] = voxel id
 *   global_tile = tile_off[view] + ty * tiles_x + tx
 *   ranges[2*g .. 2*g+1] = [start, end) of global tile g in the sorted list
 *   z_min / delta_min: minimum over views where the voxel covers >= 1 tile of
 *     max(z_center, z_near) and max(z_center, z_near) / fx  (caller sets +inf)
 *   seen: 1 if the voxel covers >= 1 tile in some view (caller zeroes)
 * Returns 0, or -1 when more than `cap` pairs would be produced (n_pairs then
 * holds the required count and nothing else is written).
 */
int ora_pairs(int64_t n, const float* geom, int n_views, const ora_cam* cams, int ts, int64_t cap,
              uint64_t* keys, uint32_t* vals, int64_t* n_pairs, uint32_t* ranges,
              float* z_min, float* delta_min, uint8_t* seen) {
  int64_t total = 0;
  int64_t tiles_total = 0;
  for (int v = 0; v < n_views; ++v) {
    for (int64_t i = 0; i < n; ++i) {
      bin32 b;
      bin_voxel32(geom + 4 * i, &cams[v], ts, &b);
      total += b.count;
    }
    tiles_total += (int64_t)((cams[v].width + ts - 1) / ts) * ((cams[v].height + ts - 1) / ts);
  }
  *n_pairs = total;
  if (total > cap) return -1;
  kv* list = (kv*)malloc(sizeof(kv) * (size_t)(total > 0 ? total : 1));
  int64_t p = 0, tile_off = 0;
  for (int v = 0; v < n_views; ++v) {
    const ora_cam* c = &cams[v];
    int tiles_x = (c->width + ts - 1) / ts, tiles_y = (c->height + ts - 1) / ts;
    for (int64_t i = 0; i < n; ++i) {
      bin32 b;
      bin_voxel32(geom + 4 * i, c, ts, &b);
      if (b.count == 0) continue;
      float zs = fmaxf(b.zc, c->z_near);
      float dl = zs / c->fx;
      if (zs < z_min[i]) z_min[i] = zs;
      if (dl < delta_min[i]) delta_min[i] = dl;
      seen[i] = 1;
      uint32_t dk = f32_order_key(b.zc);
      for (int ty = b.ty0; ty < b.ty1; ++ty)
        for (int tx = b.tx0; tx < b.tx1; ++tx) {
          uint64_t g = (uint64_t)(tile_off + (int64_t)ty * tiles_x + tx);
          list[p].key = (g << 32) | dk;
          list[p].val = (uint32_t)i;
          ++p;
        }
    }
    tile_off += (int64_t)tiles_x * tiles_y;
  }
  qsort(list, (size_t)total, sizeof(kv), kv_cmp);
  for (int64_t g = 0; g < 2 * tiles_total; ++g) ranges[g] = 0;
  for (int64_t q = 0; q < total; ++q) {
    keys[q] = list[q].key;
    vals[q] = list[q].val;
    uint64_t g = list[q].key >> 32;
    if (q == 0 || (list[q - 1].key >> 32) != g) ranges[2 * g] = (uint32_t)q;
    if (q == total - 1 || (list[q + 1].key >> 32) != g) ranges[2 * g + 1] = (uint32_t)(q + 1);
  }
  free(list);
  return 0;
}

/* ------------------------------------------------------------------ */
/* FP64 ray marching                                                   */
/* ------------------------------------------------------------------ */

/* ray-box chord: returns 1 and the entry/exit parameters when l = t_out - t_in > 0, the chord
 * starting at the near plane (t >= t_near, where the ray's camera depth reaches z_near).
 * d_in / d_out receive |d| along the axis whose slab sets the entry / exit
 * (d_in = 0 when the entry is clamped at t = 0); t_in / t_out are written even
 * for a miss, as long as every axis admits the ray. */
static int slab64x(const double* o, const double* d, double t_near, const float* g, double* t_in, double* t_out,
                   double* d_in, double* d_out) {
  double lo_t = -INFINITY, hi_t = INFINITY, din = 0.0, dout = 1.0;
  for (int a = 0; a < 3; ++a) {
    double lo = (double)g[a] - (double)g[3], hi = (double)g[a] + (double)g[3];
    if (d[a] == 0.0) {
      if (o[a] < lo || o[a] > hi) { *t_in = 1.0; *t_out = -1.0; *d_in = 0.0; *d_out = 1.0; return 0; }
      continue;
    }
    double t1 = (lo - o[a]) / d[a], t2 = (hi - o[a]) / d[a];
    double tn = t1 < t2 ? t1 : t2, tf = t1 < t2 ? t2 : t1;
    if (tn > lo_t) { lo_t = tn; din = fabs(d[a]); }
    if (tf < hi_t) { hi_t = tf; dout = fabs(d[a]); }
  }
  if (lo_t < t_near) { lo_t = t_near; din = 0.0; }
  *t_in = lo_t;
  *t_out = hi_t;
  *d_in = din;
  *d_out = dout;
  return hi_t - lo_t > 0.0;
}

/*
 * FP32 shifts of one chord (test tolerances only), for a slab test evaluated
 * in FP32 from a rounded camera-relative centre and a rounded ray direction:
 * with u = 2^-24, each direction component within (7u / |d_a| + 5u) relative
 * (camera transform, normalisation, reciprocal), each centre coordinate within
 * u (|g_a - o_a| + 2 |o_a|), each crossing rounded at its own magnitude, a
 * near-plane entry within 4u.  Entry and exit through the same pair of slab
 * planes share the rounded centre, which cancels from the chord.
 *   dl: how far the chord may move; dp: how far the midpoint sample position
 *   may move; res: the largest t_in - t_out at which an FP32 test may still
 *   report a hit.
 */
#define ORA_U32 (1.0 / 16777216.0)
static void chord_shifts(const double* o, const double* d, double t_near, const float* g, double t_in, double t_out,
                         double* dl, double* dp, double* res) {
  const double u = ORA_U32;
  int ain = -1, aout = -1;
  double tn_best = -INFINITY, tf_best = INFINITY, q[3] = {0, 0, 0}, eta[3] = {0, 0, 0}, gam[3], ad[3];
  double gmax = 0.0, gn = 0.0;
  for (int a = 0; a < 3; ++a) {
    double ga = (double)g[a] - o[a];
    gam[a] = u * (fabs(ga) + 2.0 * fabs(o[a]));
    gmax = gam[a] > gmax ? gam[a] : gmax;
    gn += ga * ga;
    ad[a] = fabs(d[a]);
    if (d[a] == 0.0) continue;
    q[a] = fabs(ga / d[a]);
    eta[a] = 7.0 * u / ad[a] + 5.0 * u;
    double t1 = (ga - (double)g[3]) / d[a], t2 = (ga + (double)g[3]) / d[a];
    double tn = t1 < t2 ? t1 : t2, tf = t1 < t2 ? t2 : t1;
    if (tn > tn_best) { tn_best = tn; ain = a; }
    if (tf < tf_best) { tf_best = tf; aout = a; }
  }
  int clamped = !(tn_best >= t_near);
  double e_in = clamped || ain < 0 ? 4.0 * u * fabs(t_in)
                                   : fabs(t_in) * eta[ain] + gam[ain] / ad[ain] + u * (q[ain] + fabs(t_in));
  double e_out = aout < 0 ? 0.0 : fabs(t_out) * eta[aout] + gam[aout] / ad[aout] + u * (q[aout] + fabs(t_out));
  double l = fabs(t_out - t_in);
  if (!clamped && ain >= 0 && ain == aout)
    *dl = l * eta[ain] + u * (fabs(t_in) + fabs(t_out) + l);
  else
    *dl = e_in + e_out + u * l;
  double tm = 0.5 * fabs(t_in + t_out);
  *dp = 0.5 * (e_in + e_out) + 13.0 * u * tm + gmax + 2.0 * u * (tm + sqrt(gn));
  *res = e_in + e_out;
}

/* FP32 shifts of a sample (test tolerances only): chord (dl), midpoint (dp) and optical depth x = sigma l
 * (dx): the chord shift times sigma plus the chord times the largest density gradient of the trilinear
 * field, sqrt(3) (max - min corner) / (2h), times the midpoint shift */
static void sample_shift(const double* o, const double* d, double t_near, const float* g, const float* d8,
                         double sigma, double l, double t_in, double t_out, double* dl, double* dp, double* dx) {
  double res, cmin = d8[0], cmx = d8[0];
  chord_shifts(o, d, t_near, g, t_in, t_out, dl, dp, &res);
  for (int i = 1; i < 8; ++i) {
    cmin = d8[i] < cmin ? d8[i] : cmin;
    cmx = d8[i] > cmx ? d8[i] : cmx;
  }
  *dx = sigma * *dl + l * 1.7320508075688772 * ((double)cmx - (double)cmin) / (2.0 * (double)g[3]) * *dp;
}

/* trilinear weights of the 8 corners at local coordinates u in [0,1]^3 */
static void trilinear_weights(const double* u, double* w) {
  for (int i = 0; i < 8; ++i) {
    double wx = (i & 1) ? u[0] : 1.0 - u[0];
    double wy = (i & 2) ? u[1] : 1.0 - u[1];
    double wz = (i & 4) ? u[2] : 1.0 - u[2];
    w[i] = wx * wy * wz;
  }
}

typedef struct {
  uint32_t key;
  uint32_t id;
} cand;

static int cand_cmp(const void* a, const void* b) {
  const cand* x = (const cand*)a;
  const cand* y = (const cand*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->id != y->id) return x->id < y->id ? -1 : 1;
  return 0;
}

/* per-view candidate lists: voxels whose conservative FP64 footprint covers the pixel */
typedef struct {
  int64_t* start; /* W*H+1 */
  cand* items;
} pixlists;

static void build_lists(int64_t n, const float* geom, const ora_cam* c, const cam64* cd, int brute,
                        const int* crop, pixlists* L) {
  int W = cd->W, H = cd->H;
  int x0 = crop ? crop[0] : 0, y0 = crop ? crop[1] : 0;
  int x1 = crop ? crop[2] : W, y1 = crop ? crop[3] : H;
  int64_t npx = (int64_t)W * H;
  int* rect = (int*)malloc(sizeof(int) * 4 * (size_t)(n > 0 ? n : 1));
  uint32_t* dkey = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    const float* g = geom + 4 * i;
    bin32 b;
    bin_voxel32(g, c, 16, &b);
    dkey[i] = f32_order_key(b.zc);
    int* r = rect + 4 * i;
    if (b.culled) { r[0] = r[1] = r[2] = r[3] = 0; continue; }
    if (brute) { r[0] = x0; r[1] = y0; r[2] = x1; r[3] = y1; continue; }
    /* FP64 projection of the part of the box beyond the near plane (in-front
       corners and edge crossings of z = z_near), 2-pixel margin */
    double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    double pc[8][3];
    for (int k = 0; k < 8; ++k) {
      double p[3] = {(double)g[0] + ((k & 1) ? 1.0 : -1.0) * (double)g[3],
                     (double)g[1] + ((k & 2) ? 1.0 : -1.0) * (double)g[3],
                     (double)g[2] + ((k & 4) ? 1.0 : -1.0) * (double)g[3]};
      cam_point64(cd, p, pc[k]);
    }
    for (int k = 0; k < 8; ++k) {
      double pts[4][3];
      int np = 0;
      if (pc[k][2] >= cd->z_near) { pts[np][0] = pc[k][0]; pts[np][1] = pc[k][1]; pts[np][2] = pc[k][2]; ++np; }
      for (int bit = 1; bit < 8; bit <<= 1) {
        if (k & bit) continue;
        int j = k | bit;
        if ((pc[k][2] >= cd->z_near) == (pc[j][2] >= cd->z_near)) continue;
        double f = (cd->z_near - pc[k][2]) / (pc[j][2] - pc[k][2]);
        pts[np][0] = pc[k][0] + f * (pc[j][0] - pc[k][0]);
        pts[np][1] = pc[k][1] + f * (pc[j][1] - pc[k][1]);
        pts[np][2] = cd->z_near;
        ++np;
      }
      for (int q = 0; q < np; ++q) {
        double u = cd->fx * pts[q][0] / pts[q][2] + cd->cx, v = cd->fy * pts[q][1] / pts[q][2] + cd->cy;
        if (u < umin) umin = u;
        if (u > umax) umax = u;
        if (v < vmin) vmin = v;
        if (v > vmax) vmax = v;
      }
    }
    double a0 = floor(umin - 2.0), a1 = ceil(umax + 2.0), b0 = floor(vmin - 2.0), b1 = ceil(vmax + 2.0);
    r[0] = (int)fmax(a0, (double)x0); r[1] = (int)fmax(b0, (double)y0);
    r[2] = (int)fmin(a1, (double)x1); r[3] = (int)fmin(b1, (double)y1);
    if (r[2] < r[0]) r[2] = r[0];
    if (r[3] < r[1]) r[3] = r[1];
  }
  L->start = (int64_t*)calloc((size_t)npx + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) {
    int* r = rect + 4 * i;
    for (int y = r[1]; y < r[3]; ++y)
      for (int x = r[0]; x < r[2]; ++x) L->start[(int64_t)y * W + x + 1] += 1;
  }
  for (int64_t p = 0; p < npx; ++p) L->start[p + 1] += L->start[p];
  int64_t tot = L->start[npx];
  L->items = (cand*)malloc(sizeof(cand) * (size_t)(tot > 0 ? tot : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(npx > 0 ? npx : 1));
  memcpy(fill, L->start, sizeof(int64_t) * (size_t)npx);
  for (int64_t i = 0; i < n; ++i) {
    int* r = rect + 4 * i;
    for (int y = r[1]; y < r[3]; ++y)
      for (int x = r[0]; x < r[2]; ++x) {
        int64_t p = (int64_t)y * W + x;
        L->items[fill[p]].key = dkey[i];
        L->items[fill[p]].id = (uint32_t)i;
        fill[p]++;
      }
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t p = 0; p < npx; ++p)
    qsort(L->items + L->start[p], (size_t)(L->start[p + 1] - L->start[p]), sizeof(cand), cand_cmp);
  free(fill);
  free(rect);
  free(dkey);
}

static void free_lists(pixlists* L) {
  free(L->start);
  free(L->items);
}

typedef struct {
  uint32_t id;
  double l, t_mid, sigma_raw, alpha, T_before;
  double w8[8]; /* d sigma_raw / d corner_i */
  /* Test tolerances only (no result depends on them): how far an FP32
   * evaluation may move the chord (dl), the midpoint (dp) and the optical depth
   * sigma*l (dx; sample_shift); the largest |corner density| (dmax) and the voxel's
   * half size (h).  ghost = 1 marks a near miss, a voxel the FP64 ray misses by
   * less than an FP32 chord test can resolve (l = 0, alpha = 0, dl = the
   * resolution): such entries are recorded only on request and never enter a
   * result. */
  double dl, dp, dx, dmax, dabs, h; /* dabs: sum_i w8_i |corner_i|, the scale of the trilinear rounding */
  int ghost;
} sample;

/* local coordinates (clamped to [0,1]^3) of the point o + t d in the voxel g */
static void local_coords(const double* o, const double* d, double t, const float* g, double* u) {
  for (int a = 0; a < 3; ++a) {
    double pa = o[a] + t * d[a];
    double lo = (double)g[a] - (double)g[3];
    double v = (pa - lo) / (2.0 * (double)g[3]);
    u[a] = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
  }
}

/*
 * Weights of the 8 corners in the sample's raw density.
 *   segment == 0 (the default reading): the trilinear field at the chord
 *   midpoint.
 *   segment == 1 (the "exact segment integration" variant): the mean of the
 *   trilinear field over the chord.  Along a line the trilinear field is a
 *   cubic polynomial in t, so Simpson's rule is exact:
 *   (1/l) int f dt = (f(t_in) + 4 f(t_mid) + f(t_out)) / 6.
 */
static void sample_weights(const double* o, const double* d, double t_in, double t_out, const float* g, int segment,
                           double* w8) {
  double u[3];
  local_coords(o, d, 0.5 * (t_in + t_out), g, u);
  trilinear_weights(u, w8);
  if (!segment) return;
  double wa[8], wb[8];
  local_coords(o, d, t_in, g, u);
  trilinear_weights(u, wa);
  local_coords(o, d, t_out, g, u);
  trilinear_weights(u, wb);
  for (int i = 0; i < 8; ++i) w8[i] = (wa[i] + 4.0 * w8[i] + wb[i]) / 6.0;
}

/* march one pixel (Eq. 2-4); returns the number of samples processed, fills s[] if non-null.
 * bnd (nullable) receives the FP32 sensitivity bound of rgb, depth and T
 * (see chord_shifts and sample_shift); cmax is the largest colour channel of the view. */
static int64_t march(const double* o, const double* d, double t_near, const cand* items, int64_t cnt,
                     const float* geom, int segment,
                     const float* dens, const double* colors, double t_stop, sample* s, double* rgb,
                     double* depth, double* T_out, int* near_stop, double* wmax, int64_t* warg, int64_t gid,
                     double cmax, double* bnd, int ghosts, int64_t* n_entries) {
  double T = 1.0;
  int64_t k = 0, ks = 0; /* samples processed; entries written to s (samples and, with ghosts, near misses) */
  double A = 0.0, X = 0.0, tmax = 0.0, cpix = 0.0;
  rgb[0] = rgb[1] = rgb[2] = 0.0;
  *depth = 0.0;
  *near_stop = 0;
  for (int64_t j = 0; j < cnt; ++j) {
    uint32_t id = items[j].id;
    const float* g = geom + 4 * (int64_t)id;
    const float* d8 = dens + 8 * (int64_t)id;
    double t_in, t_out, din, dout;
    if (!slab64x(o, d, t_near, g, &t_in, &t_out, &din, &dout)) {
      /* a near miss that FP32 could count as a hit (chord_shifts' resolution) */
      double gl, gq, res;
      if ((bnd || (s && ghosts)) && t_out > 0.0) chord_shifts(o, d, t_near, g, t_in, t_out, &gl, &gq, &res);
      if ((bnd || (s && ghosts)) && t_out > 0.0 && t_in - t_out < res) {
        double dm = 0.0;
        for (int i = 0; i < 8; ++i) dm = d8[i] > dm ? d8[i] : dm;
        if (bnd) {
          const double* cg = colors + 3 * (int64_t)id;
          A += T * dm * (res - (t_in - t_out));
          X += dm * (res - (t_in - t_out));
          if (t_out > tmax) tmax = t_out;
          for (int ch = 0; ch < 3; ++ch) cpix = cg[ch] > cpix ? cg[ch] : cpix;
        }
        if (s && ghosts) {
          sample* q = &s[ks++];
          memset(q, 0, sizeof(sample));
          q->id = id; q->T_before = T; q->t_mid = 0.5 * (t_in + t_out);
          q->dl = res - (t_in - t_out); /* the longest chord an FP32 test could find */
          q->dp = gq; q->dx = dm * q->dl; q->dmax = dm; q->h = (double)g[3]; q->ghost = 1;
        }
      }
      continue;
    }
    double l = t_out - t_in;
    double tm = 0.5 * (t_in + t_out);
    double w8[8];
    sample_weights(o, d, t_in, t_out, g, segment, w8);
    double sr = 0.0;
    for (int i = 0; i < 8; ++i) sr += w8[i] * (double)d8[i];
    double sigma = sr > 0.0 ? sr : 0.0;
    double alpha = -expm1(-sigma * l);
    double w = T * alpha;
    if (wmax) {
      if (w > wmax[id] || (w == wmax[id] && (warg[id] < 0 || gid < warg[id]))) {
        wmax[id] = w;
        warg[id] = gid;
      }
    }
    const double* c = colors + 3 * (int64_t)id;
    rgb[0] += w * c[0];
    rgb[1] += w * c[1];
    rgb[2] += w * c[2];
    *depth += w * tm;
    if (s) {
      sample* q = &s[ks++];
      q->id = id; q->l = l; q->t_mid = tm; q->sigma_raw = sr; q->alpha = alpha; q->T_before = T;
      for (int i = 0; i < 8; ++i) q->w8[i] = w8[i];
      double dm = 0.0;
      sample_shift(o, d, t_near, g, d8, sigma, l, t_in, t_out, &q->dl, &q->dp, &q->dx);
      for (int i = 0; i < 8; ++i) dm = fabs((double)d8[i]) > dm ? fabs((double)d8[i]) : dm;
      double da = 0.0;
      for (int i = 0; i < 8; ++i) da += w8[i] * fabs((double)d8[i]);
      q->dmax = dm; q->dabs = da; q->h = (double)g[3]; q->ghost = 0;
    }
    double sdx = 0.0;
    if (bnd) {
      double sdl, sdp;
      sample_shift(o, d, t_near, g, d8, sigma, l, t_in, t_out, &sdl, &sdp, &sdx);
      X += sdx;
      if (t_out > tmax) tmax = t_out;
      for (int ch = 0; ch < 3; ++ch) cpix = c[ch] > cpix ? c[ch] : cpix;
    }
    T = T * exp(-sigma * l);
    /* d rgb / d x_k = T_k c_k - sum_{j>k} w_j c_j: at most 2 max(c) T_k, T_k the transmittance after the sample */
    A += T * sdx;
    ++k;
    if (fabs(log(T / t_stop)) <= 1e-4 + X) *near_stop = 1;
    if (T < t_stop) break;
  }
  *T_out = T;
  if (n_entries) *n_entries = ks;
  if (bnd) {
    bnd[0] = 2.0 * (cpix < cmax ? cpix : cmax) * A;
    bnd[1] = 2.0 * tmax * A;
    bnd[2] = T * X;
  }
  return k;
}

static void view_colors(int64_t n, const float* geom, const float* sh, int degree, const cam64* cd,
                        double* colors, double* raw, double* dirs) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double d[3] = {(double)geom[4 * i] - cd->o[0], (double)geom[4 * i + 1] - cd->o[1],
                   (double)geom[4 * i + 2] - cd->o[2]};
    double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (nn > 0) { d[0] /= nn; d[1] /= nn; d[2] /= nn; } else { d[0] = 0; d[1] = 0; d[2] = 1; }
    double r[3];
    sh_color(sh + 48 * i, degree, d, colors + 3 * i, raw ? raw + 3 * i : r);
    if (dirs) { dirs[3 * i] = d[0]; dirs[3 * i + 1] = d[1]; dirs[3 * i + 2] = d[2]; }
  }
}

/*
 * Forward render of n_views views (Eq. 1-5), FP64.
 *   rgb[3*P], depth[P], T[P], n_hit[P], near_stop[P] over all views' pixels
 *   (P = sum W*H, view-major, row-major), only pixels inside `crop`
 *   (x0,y0,x1,y1 per view, or NULL for all) are written;
 *   w_max[n] / w_arg[n]: maximum of T_{k-1} alpha over every processed sample
 *   and the smallest global pixel id attaining it (-1 if never hit); the
 *   caller initialises w_max to 0 and w_arg to -1 and they accumulate.
 *   brute != 0: every non-culled voxel is a candidate of every pixel.
 *   bound[3*P] (nullable): per pixel, how far an FP32 evaluation of the same
 *   pixel may legitimately differ in rgb (max channel), depth and T, from the
 *   sensitivity of each sample to FP32 geometry rounding (sample_shift); near_stop
 *   marks pixels where such a perturbation can change the stop decision.
 */
int ora_render(int64_t n, const float* geom, const float* dens, const float* sh, int sh_degree, int n_views,
               const ora_cam* cams, double t_stop, int brute, const int* crop, double* rgb, double* depth,
               double* T, int32_t* n_hit, uint8_t* near_stop, double* w_max, int64_t* w_arg, double* bound,
               int segment) {
  int nt = ora_threads();
  double* colors = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  double* twm = NULL;
  int64_t* twa = NULL;
  if (w_max) {
    twm = (double*)malloc(sizeof(double) * (size_t)nt * (size_t)(n > 0 ? n : 1));
    twa = (int64_t*)malloc(sizeof(int64_t) * (size_t)nt * (size_t)(n > 0 ? n : 1));
    for (int64_t q = 0; q < (int64_t)nt * n; ++q) { twm[q] = 0.0; twa[q] = -1; }
  }
  int64_t pix_off = 0;
  for (int v = 0; v < n_views; ++v) {
    cam64 cd;
    cam_derive(&cams[v], &cd);
    view_colors(n, geom, sh, sh_degree, &cd, colors, NULL, NULL);
    double cmax = 0.0;
    for (int64_t q = 0; q < 3 * n; ++q) cmax = colors[q] > cmax ? colors[q] : cmax;
    const int* cr = crop ? crop + 4 * v : NULL;
    pixlists L;
    build_lists(n, geom, &cams[v], &cd, brute, cr, &L);
    int x0 = cr ? cr[0] : 0, y0 = cr ? cr[1] : 0, x1 = cr ? cr[2] : cd.W, y1 = cr ? cr[3] : cd.H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = y0; y < y1; ++y) {
      int tid = ora_tid();
      for (int x = x0; x < x1; ++x) {
        int64_t p = (int64_t)y * cd.W + x;
        int64_t gp = pix_off + p;
        double d[3];
        double tn = cam_ray(&cd, x, y, d);
        int ns;
        double Tp;
        int64_t k = march(cd.o, d, tn, L.items + L.start[p], L.start[p + 1] - L.start[p], geom, segment, dens, colors,
                          t_stop, NULL, rgb + 3 * gp, depth + gp, &Tp, &ns, twm ? twm + (int64_t)tid * n : NULL,
                          twa ? twa + (int64_t)tid * n : NULL, gp, cmax, bound ? bound + 3 * gp : NULL, 0, NULL);
        T[gp] = Tp;
        if (n_hit) n_hit[gp] = (int32_t)k;
        if (near_stop) near_stop[gp] = (uint8_t)ns;
      }
    }
    free_lists(&L);
    pix_off += (int64_t)cd.W * cd.H;
  }
  if (w_max) {
    for (int t = 0; t < nt; ++t)
      for (int64_t i = 0; i < n; ++i) {
        double w = twm[(int64_t)t * n + i];
        int64_t a = twa[(int64_t)t * n + i];
        if (a < 0) continue;
        if (w_arg[i] < 0 || w > w_max[i] || (w == w_max[i] && a < w_arg[i])) {
          w_max[i] = w;
          w_arg[i] = a;
        }
      }
    free(twm);
    free(twa);
  }
  free(colors);
  return 0;
}

static void atomic_add(double* p, double v) {
#pragma omp atomic
  *p += v;
}

/*
 * Reverse-mode of ora_render for the loss gradients dL/drgb (3 per pixel),
 * dL/ddepth and dL/dT (nullable); crop (x0,y0,x1,y1 per view, nullable)
 * restricts the pixels that contribute.  Writes (accumulates into, caller zeroes)
 * d_density[8n] and d_sh[48n].  The per-pixel samples of the forward pass are
 * stored and walked back to front:
 *   dL/dsigma_k = l_k * ( T_k * a_k - sum_{j>k} w_j a_j - T_final * g_T ),
 *   a_k = g_C . c_k + g_D * t_mid_k,
 * then through sigma = max(0, trilinear) to the corners and through
 * c = max(0, SH + 0.5) to the SH coefficients.
 */
int ora_render_backward(int64_t n, const float* geom, const float* dens, const float* sh, int sh_degree,
                        int n_views, const ora_cam* cams, double t_stop, const int* crop, const double* dL_drgb,
                        const double* dL_ddepth, const double* dL_dT, double* d_density, double* d_sh, int segment) {
  double* colors = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  double* raw = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  double* dirs = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  double* dcol = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  int64_t pix_off = 0;
  for (int v = 0; v < n_views; ++v) {
    cam64 cd;
    cam_derive(&cams[v], &cd);
    view_colors(n, geom, sh, sh_degree, &cd, colors, raw, dirs);
    for (int64_t i = 0; i < 3 * n; ++i) dcol[i] = 0.0;
    const int* cr = crop ? crop + 4 * v : NULL;
    int x0 = cr ? cr[0] : 0, y0 = cr ? cr[1] : 0, x1 = cr ? cr[2] : cd.W, y1 = cr ? cr[3] : cd.H;
    pixlists L;
    build_lists(n, geom, &cams[v], &cd, 0, cr, &L);
#pragma omp parallel
    {
      int64_t cap = 64;
      sample* s = (sample*)malloc(sizeof(sample) * (size_t)cap);
#pragma omp for schedule(dynamic, 1)
      for (int y = y0; y < y1; ++y) {
        for (int x = x0; x < x1; ++x) {
          int64_t p = (int64_t)y * cd.W + x;
          int64_t gp = pix_off + p;
          int64_t cnt = L.start[p + 1] - L.start[p];
          if (cnt > cap) {
            cap = cnt;
            s = (sample*)realloc(s, sizeof(sample) * (size_t)cap);
          }
          double d[3], rgbp[3], dp, Tf;
          int ns;
          double tn = cam_ray(&cd, x, y, d);
          int64_t K = march(cd.o, d, tn, L.items + L.start[p], cnt, geom, segment, dens, colors, t_stop, s, rgbp, &dp,
                            &Tf, &ns, NULL, NULL, gp, 0.0, NULL, 0, NULL);
          const double* gC = dL_drgb + 3 * gp;
          double gD = dL_ddepth ? dL_ddepth[gp] : 0.0;
          double gT = dL_dT ? dL_dT[gp] : 0.0;
          double S = 0.0;
          for (int64_t k = K - 1; k >= 0; --k) {
            const sample* q = &s[k];
            const double* c = colors + 3 * (int64_t)q->id;
            double a = gC[0] * c[0] + gC[1] * c[1] + gC[2] * c[2] + gD * q->t_mid;
            double w = q->T_before * q->alpha;
            double Tk = q->T_before * (1.0 - q->alpha);
            double ds = q->l * (Tk * a - S - Tf * gT);
            S += w * a;
            for (int ch = 0; ch < 3; ++ch) atomic_add(&dcol[3 * (int64_t)q->id + ch], w * gC[ch]);
            if (q->sigma_raw > 0.0)
              for (int i = 0; i < 8; ++i) atomic_add(&d_density[8 * (int64_t)q->id + i], ds * q->w8[i]);
          }
        }
      }
      free(s);
    }
    free_lists(&L);
    int nb = sh_count(sh_degree);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double Y[16];
      ora_sh_basis(dirs + 3 * i, Y);
      for (int ch = 0; ch < 3; ++ch) {
        if (!(raw[3 * i + ch] > 0.0)) continue;
        double g = dcol[3 * i + ch];
        for (int j = 0; j < nb; ++j) d_sh[48 * i + 3 * j + ch] += Y[j] * g;
      }
    }
    pix_off += (int64_t)cd.W * cd.H;
  }
  free(colors);
  free(raw);
  free(dirs);
  free(dcol);
  return 0;
}

/* one pixel's samples, for invariant checks (T after each sample, and w) */
int ora_trace_pixel(int64_t n, const float* geom, const float* dens, const float* sh, int sh_degree,
                    const ora_cam* cam, double t_stop, int x, int y, int64_t max_out, uint32_t* ids,
                    double* w_out, double* T_after, double* l_out, int64_t* n_out, int segment) {
  cam64 cd;
  cam_derive(cam, &cd);
  double* colors = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
  view_colors(n, geom, sh, sh_degree, &cd, colors, NULL, NULL);
  int crop[4] = {x, y, x + 1, y + 1};
  pixlists L;
  build_lists(n, geom, cam, &cd, 0, crop, &L);
  int64_t p = (int64_t)y * cd.W + x;
  int64_t cnt = L.start[p + 1] - L.start[p];
  sample* s = (sample*)malloc(sizeof(sample) * (size_t)(cnt > 0 ? cnt : 1));
  double d[3], rgbp[3], dp, Tf;
  int ns;
  double tn = cam_ray(&cd, x, y, d);
  int64_t K = march(cd.o, d, tn, L.items + L.start[p], cnt, geom, segment, dens, colors, t_stop, s, rgbp, &dp, &Tf,
                    &ns, NULL, NULL, 0, 0.0, NULL, 0, NULL);
  int64_t m = K < max_out ? K : max_out;
  for (int64_t k = 0; k < m; ++k) {
    ids[k] = s[k].id;
    w_out[k] = s[k].T_before * s[k].alpha;
    T_after[k] = s[k].T_before * (1.0 - s[k].alpha);
    l_out[k] = s[k].l;
  }
  *n_out = K;
  free(s);
  free_lists(&L);
  free(colors);
  return 0;
}

/* ------------------------------------------------------------------ */
/* FP32 error bounds and kink margins for the parity tests             */
/* ------------------------------------------------------------------ */
/*
 * None of these functions changes a result of the method: they compute how far
 * an FP32 evaluation of the same quantities may legitimately land from the FP64
 * values above, and where a finite difference would straddle a kink.  The error
 * model (first order, each term bounded in magnitude):
 *   - geometry: the chord and midpoint shifts of chord_shifts (dl, dp), the
 *     optical-depth shift they cause (dx), and near misses ("ghosts") that an
 *     FP32 chord test may count;
 *   - arithmetic, with u = 2^-24: the trilinear density within 8u sum_i w_i |corner_i|,
 *     each product and sum within u, exp(-x) within (2 + 1.2 x) units of 2u
 *     (the fast exponential), 1 - exp(-x) within 8u relative below x = 1/8 and
 *     within the error of exp(-x) above it;
 *   - transmittance: the relative errors of its factors add up along the ray;
 *     recomputed from an FP32 optical depth, as a backward pass does, it gains
 *     2u K tau + 2u (2 + 1.2 tau) for K samples of total optical depth tau;
 *   - sums in arbitrary order (atomics): n terms within (n + 1) u sum |term|
 *     (the classical bound for recursive summation in any order).
 * Weights take a factor 2 on their first-order bound for the neglected
 * higher-order terms.
 */
/* one sample's optical depth x = sigma l, the FP32 bound of its error dxk
 * (geometry, trilinear rounding, product) and the bound of the error of alpha */
static void entry_terms(const sample* q, double* x, double* dxk, double* ea) {
  *x = q->l * (q->sigma_raw > 0.0 ? q->sigma_raw : 0.0);
  *dxk = q->dx + q->l * 8.0 * ORA_U32 * q->dabs + 2.0 * ORA_U32 * *x;
  double e = exp(-*x);
  *ea = e * *dxk + 8.0 * ORA_U32 * q->alpha + (*x >= 0.125 ? 2.0 * ORA_U32 * (2.0 + 1.2 * *x) * e : 0.0);
}

/* FP32 bound of each entry's weight w = T_before alpha (ew), front to back, for
 * a transmittance formed as the product of the factors exp(-x) (a forward
 * pass); returns the relative error bound of the final transmittance */
static double weight_bounds(const sample* s, int64_t ne, double* ew) {
  double ET = 0.0;
  for (int64_t k = 0; k < ne; ++k) {
    const sample* q = &s[k];
    if (q->ghost) {
      ew[k] = 2.0 * q->T_before * q->dmax * q->dl; /* the largest weight an FP32 hit could carry */
      ET += q->dx;
      continue;
    }
    double x, dxk, ea;
    entry_terms(q, &x, &dxk, &ea);
    double w = q->T_before * q->alpha;
    ew[k] = 2.0 * (w * ET + q->T_before * ea + ORA_U32 * w);
    ET += dxk + 2.0 * ORA_U32 * (3.0 + 1.2 * x);
  }
  return ET;
}

void ora_free(void* p) { free(p); }

typedef struct {
  int64_t v, pix;
  double w, e;
} set_entry;

typedef struct {
  set_entry* a;
  int64_t n, cap;
} set_buf;

static void set_push(set_buf* b, int64_t v, int64_t pix, double w, double e) {
  if (b->n == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 1024;
    b->a = (set_entry*)realloc(b->a, sizeof(set_entry) * (size_t)b->cap);
  }
  b->a[b->n].v = v; b->a[b->n].pix = pix; b->a[b->n].w = w; b->a[b->n].e = e;
  b->n++;
}

/* top-2 of (w, pixel) with the w_max tie rule (equal weights: the smaller pixel id is the larger) */
typedef struct {
  double w1, e1, w2, e2;
  int64_t a1;
} top2;

static void top2_add(top2* t, double w, int64_t pix, double e) {
  if (t->a1 < 0 || w > t->w1 || (w == t->w1 && pix < t->a1)) {
    if (t->a1 >= 0 && (t->w2 < 0.0 || t->w1 > t->w2)) { t->w2 = t->w1; t->e2 = t->e1; }
    t->w1 = w; t->e1 = e; t->a1 = pix;
  } else if (t->w2 < 0.0 || w > t->w2) {
    t->w2 = w; t->e2 = e;
  }
}

/*
 * w_max (Eq. 5) with its FP32 ambiguity, for the argmax parity test.  Per voxel:
 *   w1, a1, e1: the FP64 maximum weight, its pixel (global id, -1 if never hit)
 *     and the FP32 bound of that weight;
 *   w2, e2: the largest weight on any other ray (-1 if none) and its bound;
 *   n_certain: samples whose chord exceeds twice its FP32 shift, on rays whose
 *     stop decision FP32 rounding cannot change (an FP32 pass must hit these).
 * The near-max set: every (voxel, pixel) entry, sample or near miss, whose weight
 * can reach the maximum's lower bound (w + e >= w1 - e1), in arrays allocated
 * here (release with ora_free).  Two passes over all views' pixels.
 */
int ora_wmax_sets(int64_t n, const float* geom, const float* dens, const float* sh, int sh_degree, int n_views,
                  const ora_cam* cams, double t_stop, int segment, double* w1, int64_t* a1, double* e1, double* w2,
                  double* e2, int32_t* n_certain, int64_t* n_set, int64_t** set_v, int64_t** set_pix,
                  double** set_w, double** set_e) {
  int nt = ora_threads();
  int64_t nn = n > 0 ? n : 1;
  top2* tt = (top2*)malloc(sizeof(top2) * (size_t)nt * (size_t)nn);
  int32_t* tc = (int32_t*)calloc((size_t)nt * (size_t)nn, sizeof(int32_t));
  for (int64_t q = 0; q < (int64_t)nt * nn; ++q) { tt[q].w1 = 0.0; tt[q].e1 = 0.0; tt[q].w2 = -1.0; tt[q].e2 = 0.0; tt[q].a1 = -1; }
  set_buf* bufs = (set_buf*)calloc((size_t)nt, sizeof(set_buf));
  double* colors = (double*)malloc(sizeof(double) * 3 * (size_t)nn);
  for (int pass = 0; pass < 2; ++pass) {
    int64_t pix_off = 0;
    for (int v = 0; v < n_views; ++v) {
      cam64 cd;
      cam_derive(&cams[v], &cd);
      view_colors(n, geom, sh, sh_degree, &cd, colors, NULL, NULL);
      pixlists L;
      build_lists(n, geom, &cams[v], &cd, 0, NULL, &L);
#pragma omp parallel
      {
        int tid = ora_tid();
        int64_t cap = 64;
        sample* s = (sample*)malloc(sizeof(sample) * (size_t)cap);
        double* ew = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 1)
        for (int y = 0; y < cd.H; ++y) {
          for (int x = 0; x < cd.W; ++x) {
            int64_t p = (int64_t)y * cd.W + x;
            int64_t gp = pix_off + p;
            int64_t cnt = L.start[p + 1] - L.start[p];
            if (cnt > cap) {
              cap = cnt;
              s = (sample*)realloc(s, sizeof(sample) * (size_t)cap);
              ew = (double*)realloc(ew, sizeof(double) * (size_t)cap);
            }
            double d[3], rgbp[3], dep, Tf;
            int ns;
            int64_t ne = 0;
            double tn = cam_ray(&cd, x, y, d);
            march(cd.o, d, tn, L.items + L.start[p], cnt, geom, segment, dens, colors, t_stop, s, rgbp, &dep, &Tf,
                  &ns, NULL, NULL, gp, 0.0, NULL, 1, &ne);
            weight_bounds(s, ne, ew);
            for (int64_t k = 0; k < ne; ++k) {
              const sample* q = &s[k];
              double w = q->T_before * q->alpha;
              if (pass == 0) {
                if (q->ghost) continue;
                top2_add(&tt[(int64_t)tid * nn + q->id], w, gp, ew[k]);
                if (!ns && q->l > 2.0 * q->dl) tc[(int64_t)tid * nn + q->id] += 1;
              } else if (w + ew[k] >= w1[q->id] - e1[q->id]) {
                set_push(&bufs[tid], (int64_t)q->id, gp, q->ghost ? 0.0 : w, ew[k]);
              }
            }
          }
        }
        free(s);
        free(ew);
      }
      free_lists(&L);
      pix_off += (int64_t)cd.W * cd.H;
    }
    if (pass == 0) {
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) {
        top2 m = tt[i];
        int32_t c = tc[i];
        for (int t = 1; t < nt; ++t) {
          const top2* o = &tt[(int64_t)t * nn + i];
          c += tc[(int64_t)t * nn + i];
          if (o->a1 < 0) continue;
          /* merge: the better first wins, the rest compete for second */
          top2 r = m;
          top2_add(&r, o->w1, o->a1, o->e1);
          if (o->w2 >= 0.0 && (r.w2 < 0.0 || o->w2 > r.w2)) { r.w2 = o->w2; r.e2 = o->e2; }
          m = r;
        }
        w1[i] = m.w1; a1[i] = m.a1; e1[i] = m.e1; w2[i] = m.w2; e2[i] = m.e2;
        n_certain[i] = c;
      }
    }
  }
  int64_t tot = 0;
  for (int t = 0; t < nt; ++t) tot += bufs[t].n;
  int64_t m = tot > 0 ? tot : 1;
  *set_v = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
  *set_pix = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
  *set_w = (double*)malloc(sizeof(double) * (size_t)m);
  *set_e = (double*)malloc(sizeof(double) * (size_t)m);
  int64_t o = 0;
  for (int t = 0; t < nt; ++t) {
    for (int64_t k = 0; k < bufs[t].n; ++k, ++o) {
      (*set_v)[o] = bufs[t].a[k].v; (*set_pix)[o] = bufs[t].a[k].pix;
      (*set_w)[o] = bufs[t].a[k].w; (*set_e)[o] = bufs[t].a[k].e;
    }
    free(bufs[t].a);
  }
  *n_set = tot;
  free(bufs);
  free(tt);
  free(tc);
  free(colors);
  return 0;
}

/* per voxel and channel: 0.5 + sum_j |SH_j Y_j|, the scale of the FP32 rounding of the colour sum (cabs);
 * per voxel the FP32 shift of the viewing direction, from the rounded centre and camera origin (the
 * centre within u (|c - o| + 2 |o|), as in chord_shifts) and the normalisation (3u), times 4, a bound of
 * the gradient of each real SH function of degree <= 3 on the sphere (dY); per voxel and channel the
 * colour shift that direction shift can cause, sum_j |SH_j| dY (cgeo) */
static void color_scales(int64_t n, const float* geom, const float* sh, int degree, const cam64* cd, double* cabs,
                         double* dY, double* cgeo) {
  int nb = sh_count(degree);
  double on = sqrt(cd->o[0] * cd->o[0] + cd->o[1] * cd->o[1] + cd->o[2] * cd->o[2]);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double d[3] = {(double)geom[4 * i] - cd->o[0], (double)geom[4 * i + 1] - cd->o[1], (double)geom[4 * i + 2] - cd->o[2]};
    double nr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (nr > 0) { d[0] /= nr; d[1] /= nr; d[2] /= nr; } else { d[0] = 0; d[1] = 0; d[2] = 1; }
    double Y[16];
    ora_sh_basis(d, Y);
    double ddir = nr > 0 ? ORA_U32 * (nr + 2.0 * on) * 1.7320508075688772 / nr + 3.0 * ORA_U32 : 1.0;
    dY[i] = 4.0 * ddir;
    for (int c = 0; c < 3; ++c) {
      double a = 0.5, b = 0.0;
      for (int j = 0; j < nb; ++j) {
        a += fabs((double)sh[48 * i + j * 3 + c] * Y[j]);
        b += fabs((double)sh[48 * i + j * 3 + c]);
      }
      cabs[3 * i + c] = a;
      cgeo[3 * i + c] = b * dY[i];
    }
  }
}

/*
 * Absolute FP32 error floors of the gradients of ora_render_backward (same
 * arguments), accumulated into e_density[8n] and e_sh[48n] (caller zeroes):
 * the per-sample errors of the reverse pass (chord, midpoint, transmittance
 * recomputed from the stored optical depth, the suffix sums, the colour),
 * near misses an FP32 pass may count, density and colour clamps within their
 * rounding, and the order of the atomic sums, (n + 1) u sum |term| for n terms.
 * A gradient g of the FP64 value ref is within |g - ref| <= e of any FP32
 * evaluation that follows the model above.  arith_only != 0 leaves out every
 * geometric term (exact chords, midpoints and hit decisions): what remains is
 * the rounding of the arithmetic and of the summation order.
 */
int ora_backward_bounds(int64_t n, const float* geom, const float* dens, const float* sh, int sh_degree,
                        int n_views, const ora_cam* cams, double t_stop, const int* crop, const double* dL_drgb,
                        const double* dL_ddepth, const double* dL_dT, double* e_density, double* e_sh, int segment,
                        int arith_only) {
  const double u = ORA_U32;
  int64_t nn = n > 0 ? n : 1;
  double* colors = (double*)malloc(sizeof(double) * 3 * (size_t)nn);
  double* raw = (double*)malloc(sizeof(double) * 3 * (size_t)nn);
  double* dirs = (double*)malloc(sizeof(double) * 3 * (size_t)nn);
  double* cabs = (double*)malloc(sizeof(double) * 3 * (size_t)nn);
  double* cgeo = (double*)malloc(sizeof(double) * 3 * (size_t)nn);
  double* dY = (double*)malloc(sizeof(double) * (size_t)nn);
  double* dcol = (double*)malloc(sizeof(double) * 3 * (size_t)nn);     /* colour gradient (FP64) */
  double* dcol_abs = (double*)malloc(sizeof(double) * 3 * (size_t)nn); /* sum of |terms| */
  double* dcol_err = (double*)malloc(sizeof(double) * 3 * (size_t)nn); /* per-term error bounds */
  double* dd_abs = (double*)calloc(8 * (size_t)nn, sizeof(double));
  int64_t* terms = (int64_t*)calloc((size_t)nn, sizeof(int64_t));
  int64_t* cterms = (int64_t*)malloc(sizeof(int64_t) * (size_t)nn);
  int64_t* views_seen = (int64_t*)calloc((size_t)nn, sizeof(int64_t));
  int64_t pix_off = 0;
  for (int v = 0; v < n_views; ++v) {
    cam64 cd;
    cam_derive(&cams[v], &cd);
    view_colors(n, geom, sh, sh_degree, &cd, colors, raw, dirs);
    color_scales(n, geom, sh, sh_degree, &cd, cabs, dY, cgeo);
    if (arith_only)
      for (int64_t i = 0; i < n; ++i) { dY[i] = 0.0; cgeo[3 * i] = cgeo[3 * i + 1] = cgeo[3 * i + 2] = 0.0; }
    for (int64_t i = 0; i < 3 * n; ++i) { dcol[i] = 0.0; dcol_abs[i] = 0.0; dcol_err[i] = 0.0; }
    for (int64_t i = 0; i < n; ++i) cterms[i] = 0;
    const int* cr = crop ? crop + 4 * v : NULL;
    int x0 = cr ? cr[0] : 0, y0 = cr ? cr[1] : 0, x1 = cr ? cr[2] : cd.W, y1 = cr ? cr[3] : cd.H;
    pixlists L;
    build_lists(n, geom, &cams[v], &cd, 0, cr, &L);
#pragma omp parallel
    {
      int64_t cap = 64;
      sample* s = (sample*)malloc(sizeof(sample) * (size_t)cap);
      double* ew = (double*)malloc(sizeof(double) * (size_t)cap);
      double* ETb = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 1)
      for (int y = y0; y < y1; ++y) {
        for (int x = x0; x < x1; ++x) {
          int64_t p = (int64_t)y * cd.W + x;
          int64_t gp = pix_off + p;
          int64_t cnt = L.start[p + 1] - L.start[p];
          if (cnt > cap) {
            cap = cnt;
            s = (sample*)realloc(s, sizeof(sample) * (size_t)cap);
            ew = (double*)realloc(ew, sizeof(double) * (size_t)cap);
            ETb = (double*)realloc(ETb, sizeof(double) * (size_t)cap);
          }
          double d[3], rgbp[3], dep, Tf;
          int ns;
          int64_t ne = 0;
          double tn = cam_ray(&cd, x, y, d);
          int64_t K = march(cd.o, d, tn, L.items + L.start[p], cnt, geom, segment, dens, colors, t_stop, s, rgbp,
                            &dep, &Tf, &ns, NULL, NULL, gp, 0.0, NULL, !arith_only, &ne);
          if (arith_only)
            for (int64_t k = 0; k < ne; ++k) { s[k].dl = 0.0; s[k].dp = 0.0; s[k].dx = 0.0; }
          /* the final transmittance comes from the forward pass (a product of factors); every other one is
           * recomputed from the stored optical depth: its relative error is the optical-depth error of the
           * samples before it (Xg) plus the rounding of the FP32 optical-depth sums, forward and back
           * (EBsum), plus that of the exponential */
          double ETf = weight_bounds(s, ne, ew);
          double tau = 0.0, tsum = 0.0, Xg = 0.0;
          for (int64_t k = 0; k < ne; ++k) {
            if (s[k].ghost) continue;
            tau += s[k].l * (s[k].sigma_raw > 0.0 ? s[k].sigma_raw : 0.0);
            tsum += tau;
          }
          double EBsum = 2.0 * u * tsum;
          tau = 0.0;
          for (int64_t k = 0; k < ne; ++k) {
            const sample* q = &s[k];
            if (q->ghost) {
              ETb[k] = Xg; /* unused for ghosts */
              Xg += q->dx;
              continue;
            }
            double x, dxk, ea;
            entry_terms(q, &x, &dxk, &ea);
            double ETbefore = Xg + EBsum + 2.0 * u * (2.0 + 1.2 * tau);
            double w = q->T_before * q->alpha;
            ew[k] = 2.0 * (w * ETbefore + q->T_before * ea + u * w);
            Xg += dxk;
            tau += x;
            ETb[k] = Xg + EBsum + 2.0 * u * (2.0 + 1.2 * tau); /* of the transmittance after the sample */
          }
          const double* gC = dL_drgb + 3 * gp;
          double gD = dL_ddepth ? dL_ddepth[gp] : 0.0;
          double gT = dL_dT ? dL_dT[gp] : 0.0;
          double S = 0.0, S_abs = 0.0, S_err = 0.0;
          for (int64_t k = ne - 1; k >= 0; --k) {
            const sample* q = &s[k];
            const double* c = colors + 3 * (int64_t)q->id;
            const double* ca = cabs + 3 * (int64_t)q->id;
            double a_k = gC[0] * c[0] + gC[1] * c[1] + gC[2] * c[2] + q->t_mid * gD;
            double a_abs = fabs(gC[0] * c[0]) + fabs(gC[1] * c[1]) + fabs(gC[2] * c[2]) + fabs(q->t_mid * gD);
            const double* cgq = cgeo + 3 * (int64_t)q->id;
            double da = fabs(gC[0]) * (64.0 * u * ca[0] + cgq[0]) + fabs(gC[1]) * (64.0 * u * ca[1] + cgq[1]) +
                        fabs(gC[2]) * (64.0 * u * ca[2] + cgq[2]) + fabs(gD) * q->dp;
            double* ed = e_density + 8 * (int64_t)q->id;
            double* dda = dd_abs + 8 * (int64_t)q->id;
            double Tb = q->T_before;
            if (q->ghost) {
              /* an FP32 pass may count this near miss: a chord of at most dl */
              double gterm = q->dl * (Tb * a_abs + S_abs + Tf * fabs(gT));
#pragma omp atomic
              terms[q->id] += 1;
              for (int i = 0; i < 8; ++i) {
#pragma omp atomic
                ed[i] += gterm;
              }
              for (int ch = 0; ch < 3; ++ch) {
#pragma omp atomic
                dcol_err[3 * (int64_t)q->id + ch] += ew[k] * fabs(gC[ch]);
              }
#pragma omp atomic
              cterms[q->id] += 1;
              S_err += a_abs * ew[k];
              continue;
            }
            double w = Tb * q->alpha;
            double T_k = Tb * (1.0 - q->alpha);
            double ETa = ETb[k];
            double inner = T_k * a_k - S - Tf * gT;
            double ds_k = q->l * inner;
            double M = T_k * a_abs + S_abs + Tf * fabs(gT);
            double d_inner = T_k * (fabs(a_k) * ETa + da) + S_err + fabs(gT) * Tf * ETf +
                             u * ((double)K + 8.0) * M;
            double d_ds = q->dl * fabs(inner) + q->l * d_inner + u * fabs(ds_k);
            double dsig = 1.7320508075688772 * q->dmax / q->h * q->dp + 8.0 * u * q->dabs;
            int clamp_amb = fabs(q->sigma_raw) <= dsig;
            double dw8 = 3.0 * q->dp / (2.0 * q->h) + 4.0 * u;
#pragma omp atomic
            terms[q->id] += 1;
            for (int i = 0; i < 8; ++i) {
              double t_i = ds_k * q->w8[i];
              double e_i;
              if (q->sigma_raw > 0.0) {
                e_i = d_ds * q->w8[i] + fabs(ds_k) * dw8 + (clamp_amb ? fabs(t_i) : 0.0);
#pragma omp atomic
                dda[i] += fabs(t_i);
              } else {
                e_i = clamp_amb ? (fabs(ds_k) + d_ds) * q->w8[i] : 0.0;
              }
#pragma omp atomic
              ed[i] += e_i;
            }
            for (int ch = 0; ch < 3; ++ch) {
              double tc = w * gC[ch];
#pragma omp atomic
              dcol[3 * (int64_t)q->id + ch] += tc;
#pragma omp atomic
              dcol_abs[3 * (int64_t)q->id + ch] += fabs(tc);
#pragma omp atomic
              dcol_err[3 * (int64_t)q->id + ch] += ew[k] * fabs(gC[ch]) + u * fabs(tc);
            }
#pragma omp atomic
            cterms[q->id] += 1;
            S += w * a_k;
            S_abs += w * a_abs;
            S_err += fabs(a_k) * ew[k] + w * da;
          }
        }
      }
      free(s);
      free(ew);
      free(ETb);
    }
    free_lists(&L);
    int nb = sh_count(sh_degree);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      if (cterms[i] == 0) continue;
      views_seen[i] += 1;
      double Y[16];
      ora_sh_basis(dirs + 3 * i, Y);
      for (int ch = 0; ch < 3; ++ch) {
        double g = dcol[3 * i + ch];
        double eg = dcol_err[3 * i + ch] + u * (double)(cterms[i] + 1) * dcol_abs[3 * i + ch];
        int amb = fabs(raw[3 * i + ch]) <= 64.0 * u * cabs[3 * i + ch] + cgeo[3 * i + ch];
        if (!(raw[3 * i + ch] > 0.0) && !amb) continue;
        for (int j = 0; j < nb; ++j) {
          double e = fabs(Y[j]) * (eg + 32.0 * u * fabs(g)) + (32.0 * u + dY[i]) * fabs(g) +
                     (amb ? fabs(Y[j] * g) : 0.0);
          e_sh[48 * i + 3 * j + ch] += e;
        }
      }
    }
    pix_off += (int64_t)cd.W * cd.H;
  }
  /* the order of the atomic sums: over the samples of each voxel, then over views for the SH rows */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < 8; ++k) e_density[8 * i + k] += u * (double)(terms[i] + 1) * dd_abs[8 * i + k];
    if (views_seen[i] > 1)
      for (int k = 0; k < 48; ++k) e_sh[48 * i + k] *= 1.0 + u * (double)(views_seen[i] + 1);
  }
  free(colors); free(raw); free(dirs); free(cabs); free(cgeo); free(dY); free(dcol); free(dcol_abs); free(dcol_err);
  free(dd_abs); free(terms); free(cterms); free(views_seen);
  return 0;
}

/*
 * Kink margins for finite differences of the render.  Per voxel:
 *   m_sigma: the smallest |sigma_raw| over its samples (a corner step of size
 *     h moves sigma_raw by at most h, so |sigma_raw| > h keeps the clamp
 *     max(0, .) on one side);
 *   m_stop: the smallest corner step that can move the stop decision of a ray
 *     through it, min over its samples k_v of min_{k >= k_v} |tau_k - ln(1/t_stop)| / l_v
 *     (the optical depth after sample k shifts by at most l_v h);
 *   m_color[3]: the smallest |pre-clamp colour| over the views that sample it
 *     (an SH step of size h moves it by at most |Y_j| h <= 1.2 h).
 * +inf where the voxel is never sampled.
 */
int ora_fd_margins(int64_t n, const float* geom, const float* dens, const float* sh, int sh_degree, int n_views,
                   const ora_cam* cams, double t_stop, int segment, double* m_sigma, double* m_stop, double* m_color) {
  int64_t nn = n > 0 ? n : 1;
  double* colors = (double*)malloc(sizeof(double) * 3 * (size_t)nn);
  double* raw = (double*)malloc(sizeof(double) * 3 * (size_t)nn);
  uint8_t* hit = (uint8_t*)malloc((size_t)nn);
  for (int64_t i = 0; i < n; ++i) { m_sigma[i] = INFINITY; m_stop[i] = INFINITY; }
  for (int64_t i = 0; i < 3 * n; ++i) m_color[i] = INFINITY;
  double Ls = log(1.0 / t_stop);
  for (int v = 0; v < n_views; ++v) {
    cam64 cd;
    cam_derive(&cams[v], &cd);
    view_colors(n, geom, sh, sh_degree, &cd, colors, raw, NULL);
    memset(hit, 0, (size_t)nn);
    pixlists L;
    build_lists(n, geom, &cams[v], &cd, 0, NULL, &L);
#pragma omp parallel
    {
      int64_t cap = 64;
      sample* s = (sample*)malloc(sizeof(sample) * (size_t)cap);
      double* tail = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 1)
      for (int y = 0; y < cd.H; ++y) {
        for (int x = 0; x < cd.W; ++x) {
          int64_t p = (int64_t)y * cd.W + x;
          int64_t cnt = L.start[p + 1] - L.start[p];
          if (cnt > cap) {
            cap = cnt;
            s = (sample*)realloc(s, sizeof(sample) * (size_t)cap);
            tail = (double*)realloc(tail, sizeof(double) * (size_t)cap);
          }
          double d[3], rgbp[3], dep, Tf;
          int ns;
          double tn = cam_ray(&cd, x, y, d);
          int64_t K = march(cd.o, d, tn, L.items + L.start[p], cnt, geom, segment, dens, colors, t_stop, s, rgbp,
                            &dep, &Tf, &ns, NULL, NULL, 0, 0.0, NULL, 0, NULL);
          /* tail[k] = min_{j >= k} |tau_j - ln(1/t_stop)|, tau_j the optical depth after sample j */
          double tau = 0.0;
          for (int64_t k = 0; k < K; ++k) {
            tau += s[k].l * (s[k].sigma_raw > 0.0 ? s[k].sigma_raw : 0.0);
            tail[k] = fabs(tau - Ls);
          }
          for (int64_t k = K - 2; k >= 0; --k) tail[k] = tail[k] < tail[k + 1] ? tail[k] : tail[k + 1];
          for (int64_t k = 0; k < K; ++k) {
            uint32_t id = s[k].id;
            double ms = fabs(s[k].sigma_raw);
            double mt = s[k].l > 0.0 ? tail[k] / s[k].l : INFINITY;
            hit[id] = 1;
#pragma omp critical(ora_fd_margins_min)
            {
              if (ms < m_sigma[id]) m_sigma[id] = ms;
              if (mt < m_stop[id]) m_stop[id] = mt;
            }
          }
        }
      }
      free(s);
      free(tail);
    }
    free_lists(&L);
    for (int64_t i = 0; i < n; ++i) {
      if (!hit[i]) continue;
      for (int c = 0; c < 3; ++c) {
        double r = fabs(raw[3 * i + c]);
        if (r < m_color[3 * i + c]) m_color[3 * i + c] = r;
      }
    }
  }
  free(colors);
  free(raw);
  free(hit);
  return 0;
}

/* ------------------------------------------------------------------ */
/* selection helpers                                                   */
/* ------------------------------------------------------------------ */

static int f32_cmp(const void* a, const void* b) {
  float x = *(const float*)a, y = *(const float*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* k-th smallest (1-based) of m floats */
static float kth_smallest(float* buf, int64_t m, int64_t k) {
  qsort(buf, (size_t)m, sizeof(float), f32_cmp);
  return buf[k - 1];
}

/* nearest-rank percentiles (ppm) of z over the flagged voxels; returns count */
static int64_t percentiles(int64_t n, const float* z, const uint8_t* flag, int64_t lo_ppm, int64_t hi_ppm,
                           float* p_lo, float* p_hi) {
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) m += flag[i] ? 1 : 0;
  *p_lo = 0.0f;
  *p_hi = 0.0f;
  if (m == 0) return 0;
  float* buf = (float*)malloc(sizeof(float) * (size_t)m);
  int64_t q = 0;
  for (int64_t i = 0; i < n; ++i)
    if (flag[i]) buf[q++] = z[i];
  qsort(buf, (size_t)m, sizeof(float), f32_cmp);
  int64_t k_lo = ppm_ceil(lo_ppm, m), k_hi = ppm_ceil(hi_ppm, m);
  if (k_lo < 1) k_lo = 1;
  if (k_hi < 1) k_hi = 1;
  if (k_lo > m) k_lo = m;
  if (k_hi > m) k_hi = m;
  *p_lo = buf[k_lo - 1];
  *p_hi = buf[k_hi - 1];
  free(buf);
  return m;
}

/* Eq. 14 in FP32: clip((z - p5) / (p95 - p5), 0, 1); 0 when p95 <= p5 */
static float depth_norm32(float z, float p_lo, float p_hi) {
  float den = p_hi - p_lo;
  if (!(den > 0.0f)) return 0.0f;
  float num = z - p_lo;
  float r = num / den;
  return fminf(fmaxf(r, 0.0f), 1.0f);
}

/*
 * Running depth percentiles (Eq. 14: "running" 5th / 95th percentiles): an
 * EMA over adaptation steps, p <- (1 - r) p + r p_step in FP32 with the two
 * products rounded separately; a state holding NaN (never updated) takes the
 * step's value.  r == 0 or no state: the step's percentiles are used as they
 * are.
 */
static void running_pct(float* p_lo, float* p_hi, float r, float one_minus_r, float* state) {
  if (!(r > 0.0f) || !state) return;
  if (isnan(state[0]) || isnan(state[1])) {
    state[0] = *p_lo;
    state[1] = *p_hi;
    return;
  }
  float a0 = one_minus_r * state[0], b0 = r * *p_lo;
  float a1 = one_minus_r * state[1], b1 = r * *p_hi;
  state[0] = a0 + b0;
  state[1] = a1 + b1;
  *p_lo = state[0];
  *p_hi = state[1];
}

/*
 * Per-bin quantile q_b in ppm (Sec. IV-C: q_b "annealed over training with a
 * mild near/far relaxation"), in integers so both sides agree exactly:
 *   q_b = q * a * (1 - relax * |2 c_b - 1|),  c_b = (b + 1/2) / n_bins,
 * with a (the schedule value) and relax in ppm: qa = floor(q a / 1e6), then
 * q_b = floor(qa (1e6 n_bins - relax |2b + 1 - n_bins|) / (1e6 n_bins)).
 * The relaxation lowers the quantile towards the nearest and farthest bins.
 */
int64_t ora_prune_q_bin(int64_t q_ppm, int64_t anneal_ppm, int64_t relax_ppm, int b, int n_bins) {
  int64_t qa = q_ppm * anneal_ppm / 1000000;
  int64_t dist = 2 * (int64_t)b + 1 - n_bins;
  if (dist < 0) dist = -dist;
  int64_t den = 1000000 * (int64_t)n_bins;
  return qa * (den - relax_ppm * dist) / den;
}

/*
 * Depth-quantile pruning (Eq. 11-12, guards i-iii), FP32 decisions.
 *   Over the seen voxels: z~ from nearest-rank p_lo/p_hi of z (Eq. 14, or
 *   their running EMA), bin b = min(nb-1, floor(nb * z~)); per bin the
 *   quantile q_b (q, or the annealed/relaxed q_b); tau_b = k-th smallest w_max
 *   in bin b, k = max(1, ceil(q_b * |V_b|)) (Eq. 12 as nearest rank on the
 *   empirical CDF of Eq. 11); q_b = 0 sets no threshold (every voxel of the
 *   bin votes in).  Inside score x = [w_max > tau_b]; m <- (1-alpha) m +
 *   alpha x; s <- out if m < m_low, in if m > m_high, else unchanged (guard
 *   i).  Keep-halo (guard ii): a voxel is protected this step when it is small
 *   against the ray footprint (h < halo_small * delta, halo_small > 0 and
 *   h/delta given) or carries a high weight near an image edge (w_max >=
 *   halo_w and edge >= halo_edge, edge given).  Candidates: seen, s == out,
 *   not protected; at most floor(cap * n) of them, those with the smallest
 *   (w_max, id), are pruned (guard iii).
 *   s: 1 = in, 0 = out.  Unseen voxels keep m and s and are never pruned.
 *   one_minus_alpha / one_minus_pct_ema are rounded to FP32 by the caller.
 */
int ora_prune(int64_t n, const float* w_max, const uint8_t* seen, const float* z, float* m, uint8_t* s,
              int n_bins, int64_t q_ppm, float alpha, float one_minus_alpha, float m_low, float m_high,
              int64_t cap_ppm, int64_t lo_ppm, int64_t hi_ppm, uint8_t* prune_mask, int64_t* n_pruned,
              float* tau_out, float* pct_out, int anneal, int64_t anneal_ppm, int64_t relax_ppm,
              const float* h, const float* delta, float halo_small, const float* edge, float halo_w,
              float halo_edge, float pct_ema, float one_minus_pct_ema, float* pct_state) {
  for (int64_t i = 0; i < n; ++i) prune_mask[i] = 0;
  *n_pruned = 0;
  float p_lo, p_hi;
  int64_t ns = percentiles(n, z, seen, lo_ppm, hi_ppm, &p_lo, &p_hi);
  if (ns == 0) {
    if (pct_out) { pct_out[0] = p_lo; pct_out[1] = p_hi; }
    return 0;
  }
  running_pct(&p_lo, &p_hi, pct_ema, one_minus_pct_ema, pct_state);
  if (pct_out) { pct_out[0] = p_lo; pct_out[1] = p_hi; }
  int* bin = (int*)malloc(sizeof(int) * (size_t)n);
  int64_t* cnt = (int64_t*)calloc((size_t)n_bins, sizeof(int64_t));
  float nbf = (float)n_bins;
  for (int64_t i = 0; i < n; ++i) {
    bin[i] = -1;
    if (!seen[i]) continue;
    float zt = depth_norm32(z[i], p_lo, p_hi);
    float sc = nbf * zt;
    int b = (int)floorf(sc);
    if (b > n_bins - 1) b = n_bins - 1;
    bin[i] = b;
    cnt[b]++;
  }
  float* tau = (float*)malloc(sizeof(float) * (size_t)n_bins);
  int* has_tau = (int*)calloc((size_t)n_bins, sizeof(int));
  float* buf = (float*)malloc(sizeof(float) * (size_t)ns);
  for (int b = 0; b < n_bins; ++b) {
    tau[b] = 0.0f;
    if (cnt[b] == 0) continue;
    int64_t qb = anneal ? ora_prune_q_bin(q_ppm, anneal_ppm, relax_ppm, b, n_bins) : q_ppm;
    if (qb <= 0) continue; /* no threshold: every voxel of the bin votes in */
    int64_t q = 0;
    for (int64_t i = 0; i < n; ++i)
      if (bin[i] == b) buf[q++] = w_max[i];
    int64_t k = ppm_ceil(qb, cnt[b]);
    if (k < 1) k = 1;
    tau[b] = kth_smallest(buf, q, k);
    has_tau[b] = 1;
  }
  if (tau_out)
    for (int b = 0; b < n_bins; ++b) tau_out[b] = tau[b];
  int64_t n_cand = 0;
  uint8_t* cand = (uint8_t*)calloc((size_t)n, 1);
  for (int64_t i = 0; i < n; ++i) {
    if (bin[i] < 0) continue;
    float x = (!has_tau[bin[i]] || w_max[i] > tau[bin[i]]) ? 1.0f : 0.0f;
    float a = one_minus_alpha * m[i];
    float c = alpha * x;
    float mm = a + c;
    m[i] = mm;
    if (mm < m_low) s[i] = 0;
    else if (mm > m_high) s[i] = 1;
    int prot = 0;
    if (halo_small > 0.0f && h && delta) {
      float lim = halo_small * delta[i];
      prot |= h[4 * i + 3] < lim;
    }
    if (edge) prot |= (w_max[i] >= halo_w && edge[i] >= halo_edge);
    if (s[i] == 0 && !prot) {
      cand[i] = 1;
      n_cand++;
    }
  }
  int64_t cap = ppm_floor(cap_ppm, n);
  if (n_cand <= cap) {
    for (int64_t i = 0; i < n; ++i)
      if (cand[i]) prune_mask[i] = 1;
    *n_pruned = n_cand;
  } else if (cap > 0) {
    kv* list = (kv*)malloc(sizeof(kv) * (size_t)n_cand);
    int64_t q = 0;
    for (int64_t i = 0; i < n; ++i)
      if (cand[i]) {
        list[q].key = f32_bits(w_max[i]); /* w_max >= 0: bits order = value order */
        list[q].val = (uint32_t)i;
        ++q;
      }
    qsort(list, (size_t)n_cand, sizeof(kv), kv_cmp);
    for (int64_t r = 0; r < cap; ++r) prune_mask[list[r].val] = 1;
    *n_pruned = cap;
    free(list);
  }
  free(cand);
  free(bin);
  free(cnt);
  free(tau);
  free(has_tau);
  free(buf);
  return 0;
}

/* lerp with the product/sum rounding fixed: a * (1 - t) + b * t */
static float lerp32(float a, float b, float t) {
  float omt = 1.0f - t;
  float x = a * omt;
  float y = b * t;
  return x + y;
}

/* parent trilinear field at parent-local coordinates q in {0, 1/2, 1}^3: x, then y, then z */
static float trilerp32(const float* d, const float* q) {
  float cx[4];
  for (int yz = 0; yz < 4; ++yz) cx[yz] = lerp32(d[yz * 2 + 0], d[yz * 2 + 1], q[0]);
  float cy0 = lerp32(cx[0], cx[1], q[1]);
  float cy1 = lerp32(cx[2], cx[3], q[1]);
  return lerp32(cy0, cy1, q[2]);
}

typedef struct { float key; uint32_t id; } pk;

static int pk_cmp_desc(const void* a, const void* b) {
  const pk* x = (const pk*)a;
  const pk* y = (const pk*)b;
  if (x->key != y->key) return x->key > y->key ? -1 : 1;
  return x->id < y->id ? -1 : (x->id > y->id ? 1 : 0);
}

/*
 * Priority-driven subdivision (Eq. 13-16 and the budgeted selection), FP32.
 *   alive = !prune_mask (prune_mask nullable);
 *   z~ from nearest-rank p_lo / p_hi of z over alive & seen voxels (Eq. 14);
 *   eligible = alive & seen & level < l_max & h > kappa * delta (Eq. 13);
 *   p = u * (1 + beta * z~) (Eq. 15-16);
 *   k = min(floor(top * n_alive), floor((budget - n_alive) / 7) (0 if budget <= n_alive), #eligible);
 *   the k eligible voxels with the largest (p, then smallest id) are split.
 * Output (capacity >= n_alive + 7k): survivors (alive, not split) in id
 * order, then 8 children per split parent in parent-id order, child i at
 * centre + (h/2) * (+-1 per bit: bit0 x, bit1 y, bit2 z), half-size h/2,
 * level + 1, corners = parent trilinear field at parent-local (bit_i + bit_j) / 2,
 * SH copied.  Auxiliary per-voxel arrays (aux_in[a] -> aux_out[a], aux_width[a]
 * elements of aux_bytes[a] bytes each) are copied for survivors and filled with
 * the fill pattern aux_fill[a] (bit pattern of one element) for children.
 */
int ora_subdivide(int64_t n, const float* geom, const uint8_t* level, const float* dens, const float* sh,
                  const float* delta, const float* z, const float* u, const uint8_t* seen,
                  const uint8_t* prune_mask, float kappa, float beta, int64_t top_ppm, int64_t budget, int l_max,
                  int64_t lo_ppm, int64_t hi_ppm, int64_t capacity, float* out_geom, uint8_t* out_level,
                  float* out_dens, float* out_sh, uint8_t* selected, int64_t* n_new, int64_t* k_out,
                  int n_aux, void* const* aux_in, void* const* aux_out, const int32_t* aux_width,
                  const int32_t* aux_bytes, const uint32_t* aux_fill, float pct_ema, float one_minus_pct_ema,
                  float* pct_state) {
  uint8_t* flag = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  int64_t n_alive = 0;
  for (int64_t i = 0; i < n; ++i) {
    int alive = prune_mask ? !prune_mask[i] : 1;
    n_alive += alive;
    flag[i] = (uint8_t)(alive && seen[i]);
    selected[i] = 0;
  }
  float p_lo, p_hi;
  if (percentiles(n, z, flag, lo_ppm, hi_ppm, &p_lo, &p_hi) > 0)
    running_pct(&p_lo, &p_hi, pct_ema, one_minus_pct_ema, pct_state);
  pk* list = (pk*)malloc(sizeof(pk) * (size_t)(n > 0 ? n : 1));
  int64_t n_el = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!flag[i]) continue;
    if (!((int)level[i] < l_max)) continue;
    float thr = kappa * delta[i];
    if (!(geom[4 * i + 3] > thr)) continue;
    float zt = depth_norm32(z[i], p_lo, p_hi);
    float bz = beta * zt;
    float b = 1.0f + bz;
    list[n_el].key = u[i] * b;
    list[n_el].id = (uint32_t)i;
    ++n_el;
  }
  int64_t k = ppm_floor(top_ppm, n_alive);
  int64_t kb = budget > n_alive ? (budget - n_alive) / 7 : 0;
  if (kb < k) k = kb;
  if (n_el < k) k = n_el;
  *k_out = k;
  if (n_alive + 7 * k > capacity) {
    free(flag);
    free(list);
    *n_new = n_alive + 7 * k;
    return -1;
  }
  qsort(list, (size_t)n_el, sizeof(pk), pk_cmp_desc);
  for (int64_t r = 0; r < k; ++r) selected[list[r].id] = 1;
  int64_t o = 0;
  for (int64_t i = 0; i < n; ++i) {
    int alive = prune_mask ? !prune_mask[i] : 1;
    if (!alive || selected[i]) continue;
    memcpy(out_geom + 4 * o, geom + 4 * i, 16);
    out_level[o] = level[i];
    memcpy(out_dens + 8 * o, dens + 8 * i, 32);
    memcpy(out_sh + 48 * o, sh + 48 * i, 192);
    for (int a = 0; a < n_aux; ++a) {
      size_t eb = (size_t)aux_bytes[a] * (size_t)aux_width[a];
      memcpy((char*)aux_out[a] + eb * (size_t)o, (const char*)aux_in[a] + eb * (size_t)i, eb);
    }
    ++o;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (!selected[i]) continue;
    const float* g = geom + 4 * i;
    float hc = g[3] * 0.5f;
    for (int c = 0; c < 8; ++c) {
      float* og = out_geom + 4 * o;
      og[0] = g[0] + ((c & 1) ? hc : -hc);
      og[1] = g[1] + ((c & 2) ? hc : -hc);
      og[2] = g[2] + ((c & 4) ? hc : -hc);
      og[3] = hc;
      out_level[o] = (uint8_t)(level[i] + 1);
      for (int j = 0; j < 8; ++j) {
        float q[3];
        q[0] = (float)(((c >> 0) & 1) + ((j >> 0) & 1)) * 0.5f;
        q[1] = (float)(((c >> 1) & 1) + ((j >> 1) & 1)) * 0.5f;
        q[2] = (float)(((c >> 2) & 1) + ((j >> 2) & 1)) * 0.5f;
        out_dens[8 * o + j] = trilerp32(dens + 8 * i, q);
      }
      memcpy(out_sh + 48 * o, sh + 48 * i, 192);
      for (int a = 0; a < n_aux; ++a) {
        size_t w = (size_t)aux_width[a];
        for (size_t e = 0; e < w; ++e) {
          char* dst = (char*)aux_out[a] + (size_t)aux_bytes[a] * (w * (size_t)o + e);
          if (aux_bytes[a] == 4) memcpy(dst, &aux_fill[a], 4);
          else if (aux_bytes[a] == 2) { uint16_t f = (uint16_t)aux_fill[a]; memcpy(dst, &f, 2); }
          else { uint8_t f = (uint8_t)aux_fill[a]; memcpy(dst, &f, 1); }
        }
      }
      ++o;
    }
  }
  *n_new = o;
  free(flag);
  free(list);
  return 0;
}

/* ------------------------------------------------------------------ */
/* LF-weighted photometric loss (Eq. 7-10, 18), FP64                    */
/* ------------------------------------------------------------------ */

/* Eq. 9 */
double ora_lf_gamma(double t, double t0, double t1, double gamma_max) {
  if (t < t0) return 0.0;
  if (t < t1) return gamma_max * (t - t0) / (t1 - t0);
  return gamma_max;
}

static int d_cmp(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/*
 * Per view v (pixels P_v):
 *   Y = (R + G + B) / 3 of the ground truth; 3x3 Sobel with replicated border;
 *   s = clip(|grad Y| / P_pctl(|grad Y|), 0, 1) (0 where the percentile is 0),
 *   nearest rank k = max(1, ceil(pctl * |P_v|));
 *   w = (eps + 1 - s)^gamma, w~ = w / mean(w) (Eq. 7-8);
 *   loss[v] = 1/|P_v| sum w~ * rho(r), rho(r) = mean over channels of r^2 (Eq. 18);
 *   dL/drgb = 2 / (3 |P_v|) * w~ * r.
 * sobel_s (nullable) receives s, weights (nullable) receives w~.
 */
int ora_lf_loss(int n_views, const int32_t* widths, const int32_t* heights, const double* rgb, const double* gt,
                double gamma, double eps, int64_t pctl_ppm, double* loss, double* dL_drgb, double* sobel_s,
                double* weights) {
  int64_t off = 0;
  for (int v = 0; v < n_views; ++v) {
    int W = widths[v], H = heights[v];
    int64_t np = (int64_t)W * H;
    const double* G = gt + 3 * off;
    const double* R = rgb + 3 * off;
    double* Y = (double*)malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
    double* mag = (double*)malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
    double* srt = (double*)malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
    for (int64_t p = 0; p < np; ++p) Y[p] = (G[3 * p] + G[3 * p + 1] + G[3 * p + 2]) / 3.0;
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        int xm = x > 0 ? x - 1 : 0, xp = x < W - 1 ? x + 1 : W - 1;
        int ym = y > 0 ? y - 1 : 0, yp = y < H - 1 ? y + 1 : H - 1;
#define YY(a, b) Y[(int64_t)(b) * W + (a)]
        double gx = (YY(xp, ym) + 2.0 * YY(xp, y) + YY(xp, yp)) - (YY(xm, ym) + 2.0 * YY(xm, y) + YY(xm, yp));
        double gy = (YY(xm, yp) + 2.0 * YY(x, yp) + YY(xp, yp)) - (YY(xm, ym) + 2.0 * YY(x, ym) + YY(xp, ym));
#undef YY
        mag[(int64_t)y * W + x] = sqrt(gx * gx + gy * gy);
      }
    memcpy(srt, mag, sizeof(double) * (size_t)np);
    qsort(srt, (size_t)np, sizeof(double), d_cmp);
    int64_t k = ppm_ceil(pctl_ppm, np);
    if (k < 1) k = 1;
    if (k > np) k = np;
    double P = np > 0 ? srt[k - 1] : 0.0;
    double sw = 0.0;
    for (int64_t p = 0; p < np; ++p) {
      double s = 0.0;
      if (P > 0.0) {
        s = mag[p] / P;
        s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
      }
      if (sobel_s) sobel_s[off + p] = s;
      w[p] = pow(eps + 1.0 - s, gamma);
      sw += w[p];
    }
    double mean = np > 0 ? sw / (double)np : 1.0;
    double L = 0.0;
    for (int64_t p = 0; p < np; ++p) {
      double wt = w[p] / mean;
      if (weights) weights[off + p] = wt;
      double rho = 0.0;
      for (int c = 0; c < 3; ++c) {
        double r = R[3 * p + c] - G[3 * p + c];
        rho += r * r;
        if (dL_drgb) dL_drgb[3 * (off + p) + c] = 2.0 / (3.0 * (double)np) * wt * r;
      }
      L += wt * rho / 3.0;
    }
    loss[v] = np > 0 ? L / (double)np : 0.0;
    free(Y);
    free(mag);
    free(srt);
    free(w);
    off += np;
  }
  return 0;
}

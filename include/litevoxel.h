/*
 * litevoxel.h -- C ABI of the GB300 (sm_103a) sparse-voxel tile rasterizer.
 *
 * The library implements the data-parallel hot path of LiteVoxel's training
 * loop (arXiv 2511.02510): forward and backward passes of the differentiable
 * tile rasterizer for sparse octree voxels (Sec. III, Eq. 1-5), depth-quantile
 * pruning (Sec. IV-C, Eq. 11-12 with guards i-iii), priority-driven
 * subdivision (Sec. IV-D, Eq. 13-16) and the low-frequency-weighted
 * photometric loss (Sec. IV-B, Eq. 7-10 and Eq. 18).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All pointers named d_* or documented as "device" point to CUDA device
 *    memory on the current device.  The caller owns every buffer; the library
 *    never allocates device memory.  Calls that need scratch space take a
 *    caller-allocated workspace whose size comes from the matching
 *    *_workspace_size() query (bytes; 256-byte aligned base required).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is
 *    asynchronous on that stream unless `LV_FLAG_SYNC_CHECK` is set in the
 *    options, in which case the call synchronises the stream and returns the
 *    device-side status.
 *  - Host-detectable argument errors return LV_ERR_INVALID_ARG (a workspace
 *    smaller than its size query: LV_ERR_WORKSPACE; an option that is not
 *    built in: LV_ERR_UNSUPPORTED) and nothing is launched; `lv_last_error()`
 *    describes the most recent failure of the calling thread.  Errors found on the device (pair or voxel capacity
 *    overflow, a bounded inter-block wait of the radix sort that gave up)
 *    are written to `d_status` (int32 device word, first error wins, the
 *    caller zeroes it; lv_check_status reads it) and the affected outputs
 *    are left unspecified.  A launch failure returns LV_ERR_CUDA.
 *  - Pixels of all views are concatenated view-major, each view row-major:
 *    pixel (view v, x, y) has global id pix_off[v] + y * width_v + x.
 *  - Voxel arrays are structure-of-arrays, one row per voxel:
 *      geom     float32 [n][4]  centre x, y, z and half-size h
 *      level    uint8   [n]     octree depth (edge = root_edge / 2^level)
 *      density  [n][8]          corner densities, corner i at
 *                               centre + h * (+-1, +-1, +-1) with bit0 = x,
 *                               bit1 = y, bit2 = z set meaning "+"
 *      sh       [n][48]         real SH coefficients [coef 0..15][r, g, b]
 */
#ifndef LITEVOXEL_H
#define LITEVOXEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LV_VERSION_MAJOR 0
#define LV_VERSION_MINOR 1
#define LV_MAX_VIEWS 64

typedef enum {
  LV_OK = 0,
  LV_ERR_INVALID_ARG = 1,  /* bad pointer, size, dtype or option (host check) */
  LV_ERR_WORKSPACE = 2,    /* workspace smaller than the size query returned */
  LV_ERR_CAPACITY = 3,     /* pair / slot / output-voxel capacity exceeded (device) */
  LV_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed */
  LV_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
  LV_ERR_UNSUPPORTED = 6   /* option combination not built in */
} lv_status;

typedef enum { LV_F32 = 0, LV_F16 = 1, LV_BF16 = 2 } lv_dtype;

#define LV_FLAG_SYNC_CHECK 1u  /* synchronise and return the device status */
/* Density-model variant: a sample's density is the mean of the voxel's
 * trilinear corner field over the chord instead of its value at the chord
 * midpoint (the exact integral of the cubic profile, by Simpson's rule over
 * the chord ends and midpoint), sigma = max(0, mean), alpha = 1 - exp(-sigma l)
 * (Eq. 2-4).  Forward and backward of one step must use the same flags. */
#define LV_FLAG_EXACT_SEGMENT 2u
/* Scheduling of the composite kernels: persistent warps, as many as are
 * resident, each taking the next (tile, 4x8-pixel strip) from a global
 * counter (atomicAdd, no waiting), instead of one block per tile.  Results
 * are identical either way (per pixel the same arithmetic in the same order;
 * gradient sums differ only in FP32 atomic order). */
#define LV_FLAG_PERSISTENT 4u

/* Voxel set (all device pointers). density_dtype: LV_F32 or LV_F16; sh_dtype: LV_F32 or LV_BF16.
 * density is [n][8] corner densities (corner c = x + 2y + 4z), or, when vidx
 * is given, the shared grid-vertex variant: density is a vertex array and
 * corner c of voxel v reads density[vidx[8 v + c]] (see lv_build_vertex_index;
 * the rasterizer's d_density output stays per voxel corner [n][8], turned into
 * the vertex gradient by lv_vertex_scatter_add).  Subdivision needs per-voxel
 * corners (vidx NULL). */
typedef struct {
  int64_t n;
  const float* geom;
  const uint8_t* level; /* only read by lv_subdivide_priority */
  const void* density;
  int32_t density_dtype;
  const void* sh;
  int32_t sh_dtype;
  int32_t sh_degree; /* 0..3; coefficients beyond (degree+1)^2 are ignored */
  const uint32_t* vidx; /* NULL, or [n][8] vertex ids (16-byte aligned) */
} lv_voxels;

/* Pinhole camera (host struct, passed by value to the kernels).
 * x_cam = R x_world + t with w2c = [R | t] row-major 3x4; OpenCV axes
 * (x right, y down, z forward).  Pixel (x, y) is sampled at its centre
 * (x + 0.5, y + 0.5); u = fx * x_cam / z_cam + cx (Eq. 1). */
typedef struct {
  int32_t width, height;
  float fx, fy, cx, cy;
  float w2c[12];
  float z_near; /* near plane: chords start at camera depth z_near; voxels whose 8 corners all
                   have z_cam < z_near are culled, voxels crossing it are clipped */
} lv_camera;

typedef struct {
  int32_t tile;           /* tile edge in pixels: 8, 16 or 32 */
  int32_t batch;          /* list entries a warp stages per round (32, 64 or 128; 128 not with tile 32):
                             their records are loaded together into the warp's shared-memory slice
                             (64 B each) before its pixels march through them; changes no result */
  float t_stop;           /* a ray stops after the sample that takes T below t_stop (1e-4) */
  uint32_t flags;         /* LV_FLAG_* */
  int32_t persistent_sms; /* with LV_FLAG_PERSISTENT: run the composite on this many SMs (0 = all): the
                             full resident grid is launched and the blocks that land on other SMs (by SM
                             id) return at once, so those SMs stay free for kernels of other streams that
                             run beside the composite; it changes no result and may differ between the
                             forward and backward calls */
  int64_t pixel_id_base;  /* global id of this call's first pixel (0): the pixel ids packed into w_max
                             (Eq. 5's argmax and its tie rule) are pixel_id_base + the view-major index;
                             calls or ranks that render disjoint views with disjoint bases accumulate one
                             w_max exactly as one call over all the views; base + pixels must stay
                             below 2^32 - 1 */
} lv_raster_opts;

/* Forward outputs (device).  P = total pixels of all views. */
typedef struct {
  float* rgb;                        /* [P][3] composited colour, Eq. 4 */
  float* depth;                      /* [P] sum_k w_k t_mid_k (nullable) */
  float* T;                          /* [P] final transmittance, Eq. 3 */
  uint32_t* n_contrib;               /* [P] tile-list entries up to the last sample used (backward needs it) */
  unsigned long long* wmax_packed;   /* [n] max-accumulated (f32 bits(w_max) << 32) | (0xffffffff - pixel id),
                                        Eq. 5; caller zeroes; nullable */
  float* z_min;                      /* [n] min over views of max(z_centre, z_near); caller sets +inf; nullable */
  float* delta_min;                  /* [n] min over views of max(z_centre, z_near) / fx, the inter-ray
                                        spacing at the voxel (Sec. III); caller sets +inf; nullable */
  uint8_t* seen;                     /* [n] set to 1 when the voxel covers >= 1 tile of some view; nullable */
  uint32_t* n_samples;               /* [P] samples composited per pixel (hits of Eq. 2-4); nullable */
  void* stats_event;                 /* cudaEvent_t (nullable): recorded on the stream as soon as z_min,
                                        delta_min and seen are final (after binning, before sorting and
                                        compositing), so another stream can start on them early */
  void* composite_event;             /* cudaEvent_t (nullable): recorded on the stream right before the
                                        front-to-back composite is launched (the last launch of the
                                        call), so that an event recorded after the call times the
                                        composite alone; inside a stream capture it is recorded as an
                                        external event node (cudaEventRecordExternal), a timing mark
                                        of every replay rather than a dependency */
  /* Optional LF-weighted loss fused into the backward composite (Sec. IV-B,
   * Eq. 8 and 18), for a caller that ran lv_lf_weights for these views
   * (their widths and heights in camera order).  The forward ignores these
   * fields.  When lf_workspace is not NULL and lv_rasterize_backward gets
   * dL_drgb = NULL, the backward computes every pixel's dL/drgb from rgb,
   * lf_gt and the weights -- bit for bit what lv_lf_loss_from_weights writes
   * -- uses it, writes it into lf_dL when that is not NULL, and adds the
   * views' loss sums into the workspace (FP64, one atomic per block and view);
   * lv_lf_loss_finish then writes the per-view losses.  A wrong workspace size
   * returns LV_ERR_WORKSPACE, mismatched views LV_ERR_INVALID_ARG. */
  const float* lf_gt;                /* [P][3] ground truth, as given to lv_lf_weights */
  void* lf_workspace;                /* lv_lf_weights' workspace (256-byte aligned), or NULL */
  size_t lf_ws_bytes;
  float* lf_dL;                      /* [P][3] dL/drgb output (nullable) */
  void* lf_wait_event;               /* cudaEvent_t (nullable): the backward's stream waits for it before
                                        the composite, so lv_lf_weights can run on another stream
                                        (inside a stream capture: a dependency) */
} lv_fwd_out;

/* ------------------------------------------------------------------ */
/* rasterizer (Sec. III, Eq. 1-5)                                       */
/* ------------------------------------------------------------------ */

/* Bytes of forward/backward workspace for n voxels, the given views and at
 * most pair_capacity (tile, voxel) pairs.  The same workspace must be passed
 * unchanged from lv_rasterize_forward to lv_rasterize_backward.  Returns 0
 * for a configuration the forward pass would refuse on its size arguments
 * (no view or more than LV_MAX_VIEWS, n < 0, a tile edge other than 8 / 16 /
 * 32, pair_capacity outside [0, 2^32 - 1]). */
size_t lv_forward_workspace_size(int64_t n, const lv_camera* cams, int n_views, const lv_raster_opts* opts,
                                 int64_t pair_capacity);

/* Forward pass: per voxel and view, cull / project / bin to tiles (FP32 with
 * a fixed operation order), emit (tile << 32 | depth key, voxel) pairs,
 * radix-sort them, find tile ranges and alpha-composite every pixel front to
 * back (Eq. 2-4): slab-test chord l (starting at the near plane), sigma = max(0, trilinear corner density
 * at the chord midpoint), alpha = 1 - exp(-sigma l), colour from SH towards
 * the voxel centre c = max(0, SH + 0.5).  w_max (Eq. 5) is fused in.
 * Sorted pairs, tile ranges and the per-pixel optical depth stay in the
 * workspace for the backward pass.  More than pair_capacity pairs sets
 * LV_ERR_CAPACITY in d_status (see lv_workspace_counters for the count). */
lv_status lv_rasterize_forward(const lv_voxels* vox, const lv_camera* cams, int n_views, const lv_raster_opts* opts,
                               const lv_fwd_out* out, void* workspace, size_t ws_bytes, int64_t pair_capacity,
                               int32_t* d_status, void* stream);

/* Start a new accumulation window of the per-voxel statistics in one
 * launch: wmax_packed[i] = 0, z_min[i] = delta_min[i] = +inf, seen[i] = 0
 * for i < n (device arrays as in lv_fwd_out; any may be NULL). */
lv_status lv_reset_stats(int64_t n, unsigned long long* wmax_packed, float* z_min, float* delta_min, uint8_t* seen,
                         void* stream);

/* Synchronously read the forward counters from a workspace: out2[0] = pairs
 * the last forward emitted (may exceed its capacity), out2[1] = visible
 * (voxel, view) slots. */
lv_status lv_workspace_counters(const void* workspace, size_t ws_bytes, int64_t* out2, void* stream);

/* Backward pass (reverse-mode of Eq. 2-4), walking each pixel's samples
 * back to front from n_contrib and recomputing transmittance from the stored
 * final optical depth (no per-sample storage):
 *   dL/dsigma_k = l_k (T_k a_k - sum_{j>k} w_j a_j - T_final g_T),
 *   a_k = g_C . c_k + g_D t_mid_k,
 * then to the 8 corners through the trilinear weights (zero where the raw
 * density is negative) and to the SH through c = max(0, SH + 0.5).
 * dL_ddepth and dL_dT may be NULL; dL_drgb too when fwd->lf_workspace fuses the
 * LF loss (see lv_fwd_out).  d_density [n][8] and d_sh [n][48] are
 * FP32; with accumulate = 0 they are overwritten, else added to.  vox, cams,
 * n_views, opts, workspace and pair_capacity must be those of the forward
 * call (the workspace's colour-gradient scratch is reused).  With d_sh = NULL
 * the per-(voxel, view) colour gradients stay in the workspace and
 * lv_sh_backward finishes the SH part later (same arguments). */
lv_status lv_rasterize_backward(const lv_voxels* vox, const lv_camera* cams, int n_views,
                                const lv_raster_opts* opts, const lv_fwd_out* fwd, void* workspace, size_t ws_bytes,
                                int64_t pair_capacity, const float* dL_drgb, const float* dL_ddepth,
                                const float* dL_dT, float* d_density, float* d_sh, int accumulate,
                                int32_t* d_status, void* stream);

/* SH part of the backward pass: d_sh [n][48] (FP32) from the colour
 * gradients a preceding lv_rasterize_backward(d_sh = NULL) left in the
 * workspace, through c = max(0, SH(dir) + 0.5) with dir the unit vector from
 * the camera centre to the voxel centre; sums over views.  Clears the
 * workspace's colour gradients.  accumulate as in lv_rasterize_backward.
 * Reads only the workspace (the camera-relative centres the forward stored),
 * not the voxel arrays, so it may run beside a topology change that rewrites
 * them in place (lv_subdivide_apply_inplace); vox gives n and the SH degree. */
lv_status lv_sh_backward(const lv_voxels* vox, const lv_camera* cams, int n_views, const lv_raster_opts* opts,
                         void* workspace, size_t ws_bytes, int64_t pair_capacity, float* d_sh, int accumulate,
                         void* stream);

/* Autotuner of the composite schedule (batched views in one launch: tile
 * size, batch and scheduling chosen per scene and view set).  Each candidate
 * -- tile edge 8, 16, 32 x one block per tile or persistent warps
 * (LV_FLAG_PERSISTENT) x batch 32, 64, 128 (not 128 with tile 32) -- runs one
 * warm-up forward + backward and then `reps` (1 .. 1000) timed ones on the
 * caller's scene and views, timed with CUDA events on `stream`; the call
 * synchronises the stream.  *best receives *base with the fastest tile,
 * batch and LV_FLAG_PERSISTENT choice.  ms_out (host float[18], nullable)
 * receives each candidate's mean forward + backward time in ms at index
 * (6 t + 3 p + b) for tile t (0: 8, 1: 16, 2: 32), schedule p (0: block per
 * tile, 1: persistent) and batch b (0: 32, 1: 64, 2: 128); -1 for a candidate
 * that is refused or needs more than pair_capacity pairs (skipped), and -1
 * everywhere on a cache hit.  cache_path (nullable) is a text file of
 * "key tile persistent batch" lines keyed by device name, voxel count, view
 * sizes and the other flags (a line without the batch means 32): a hit
 * returns at once, a tuned result is appended.  workspace:
 * lv_autotune_workspace_size(n, cams, n_views, base, pair_capacity) bytes
 * (forward workspace for the largest need, outputs and gradients).
 * LV_ERR_CAPACITY when no candidate fits the pair capacity. */
size_t lv_autotune_workspace_size(int64_t n, const lv_camera* cams, int n_views, const lv_raster_opts* base,
                                  int64_t pair_capacity);
lv_status lv_autotune(const lv_voxels* vox, const lv_camera* cams, int n_views, const lv_raster_opts* base,
                      int64_t pair_capacity, int reps, lv_raster_opts* best, float* ms_out, const char* cache_path,
                      void* workspace, size_t ws_bytes, void* stream);

/* Unpack lv_fwd_out.wmax_packed: w_max[i] (0 if never hit) and the smallest
 * global pixel id attaining it (-1 if never hit).  argmax is nullable. */
lv_status lv_unpack_wmax(const unsigned long long* packed, int64_t n, float* w_max, int64_t* argmax, void* stream);

/* Per-voxel edge score for the keep-halo guard: edge[i] = edge_map[argmax[i]]
 * (the normalised Sobel magnitude of Eq. 7 at the pixel where the voxel's
 * w_max was attained, see lv_lf_params.edge_out), 0 when argmax[i] < 0 or
 * >= n_pix.  argmax: device [n] int64 (lv_unpack_wmax); edge_map: device
 * [n_pix]; edge: device [n]. */
lv_status lv_gather_edge(const int64_t* argmax, int64_t n, const float* edge_map, int64_t n_pix, float* edge,
                         void* stream);

/* Copy the sorted pair list of a forward workspace to device buffers:
 * keys[i] = (global tile << 32) | order-preserving f32 bits of z_centre,
 * voxel[i] = voxel id; ranges [tiles][2] = [start, end) per global tile.
 * keys / voxel hold at least min(pairs, pair_capacity) entries.  Any of the
 * outputs may be NULL.  n, cams, n_views, opts and pair_capacity are those
 * of the forward call.  For tests and debugging. */
lv_status lv_debug_pairs(int64_t n, const lv_camera* cams, int n_views, const lv_raster_opts* opts,
                         const void* workspace, size_t ws_bytes, int64_t pair_capacity, uint64_t* keys,
                         uint32_t* voxel, uint32_t* ranges, void* stream);

/* Check of the radix sort's bounded wait.  The pair sort's pass kernel
 * finds each tile's global offsets by waiting for the digit counts that
 * earlier tiles publish (a decoupled look-back).  This call runs one pass
 * over two 4096-item tiles with only the second tile's block launched, so
 * its wait for the first tile can never end.  The wait gives up after
 * spin_limit polls (1 .. 1048576, the limit the sort uses; 32 ns sleep
 * between polls), writes LV_ERR_TIMEOUT into *d_status (device int32,
 * cleared by the call first) and returns; the stream stays usable.
 * workspace: lv_debug_sort_timeout_workspace_size() bytes, 256-byte
 * aligned.  For tests. */
size_t lv_debug_sort_timeout_workspace_size(void);
lv_status lv_debug_sort_timeout(int32_t spin_limit, void* workspace, size_t ws_bytes, int32_t* d_status,
                                void* stream);

/* FP64 re-render of chosen pixels for finite-difference gradient checks (the
 * only FP64 arithmetic of the library): pixels [n_px] are global pixel ids
 * (device int64); for each, the tile list of a forward workspace is walked
 * front to back (Eq. 2-4) in FP64 from the voxel arrays, with the same chord,
 * near-plane, ordering, colour and stop rules as the forward.  The lists
 * depend on geometry only, so corner densities and SH may be changed between
 * the forward and this call.  rgb [n_px][3] and T [n_px] (nullable) are FP64
 * device outputs. */
lv_status lv_render_pixels_f64(const lv_voxels* vox, const lv_camera* cams, int n_views, const lv_raster_opts* opts,
                               const void* workspace, size_t ws_bytes, int64_t pair_capacity, const int64_t* pixels,
                               int64_t n_px, double* rgb, double* T, void* stream);

/* ------------------------------------------------------------------ */
/* depth-quantile pruning (Sec. IV-C, Eq. 11-12, guards i-iii)          */
/* ------------------------------------------------------------------ */

typedef struct {
  int32_t n_bins;   /* depth bins V_b (16) */
  int32_t q_ppm;    /* quantile q_b in parts per million (50000 = 5 %) */
  float ema_alpha;  /* EMA rate alpha (0.1 for a decay of 0.9) */
  float m_low;      /* hysteresis: state -> out when m < m_low */
  float m_high;     /*             state -> in  when m > m_high */
  int32_t cap_ppm;  /* per-step cap on pruned voxels, ppm of n (10000 = 1 %) */
  int32_t lo_ppm;   /* depth normalisation percentiles (Eq. 14): 50000 */
  int32_t hi_ppm;   /*                                            950000 */
  /* --- optional guards; all-zero fields leave them off ----------------- */
  /* q_b schedule (Sec. IV-C: q_b annealed over training with a mild
   * near/far relaxation).  anneal != 0: q_b = q a (1 - relax |2 c_b - 1|),
   * c_b = (b + 1/2) / n_bins, evaluated in integers (ppm):
   * qa = floor(q anneal_ppm / 1e6), q_b = floor(qa (1e6 nb - relax_ppm
   * |2b + 1 - nb|) / (1e6 nb)).  anneal_ppm = a(t), see lv_prune_anneal_ppm.
   * A bin whose q_b is 0 has no threshold (its voxels all vote in). */
  int32_t anneal;
  int32_t anneal_ppm;
  int32_t relax_ppm;   /* 0..1e6 */
  /* keep-halo (guard ii): a voxel is protected this step (its EMA and state
   * still update) when halo_small > 0 and h_v < halo_small * delta_v (small
   * against the ray footprint; needs geom and delta), or when edge is given
   * and w_max_v >= halo_w and edge_v >= halo_edge (a strong weight on an
   * image edge).  FP32 comparisons. */
  float halo_small;
  float halo_w;
  float halo_edge;
  const float* geom;   /* device N x 4 (cx, cy, cz, h), nullable */
  const float* delta;  /* device N, footprint delta_v (lv_fwd_out.delta_min), nullable */
  const float* edge;   /* device N, edge score in [0, 1] (lv_gather_edge), nullable */
  /* running depth percentiles (Eq. 14 "running"): pct_ema > 0 and pct_state
   * given: p <- (1 - r) p + r p_step (FP32, products rounded separately) over
   * calls; a state holding NaN takes the step's value.  pct_state is a device
   * float[2] (p_lo, p_hi) that the caller initialises to NaN once. */
  float pct_ema;
  float* pct_state;
} lv_prune_params;

/* a(t) = clip((t - t0) / (t1 - t0), 0, 1) in ppm (floor, computed in double);
 * 1000000 when t1 <= t0.  Host only. */
int32_t lv_prune_anneal_ppm(double t, double t0, double t1);

size_t lv_prune_workspace_size(int64_t n, const lv_prune_params* p);

/* Over seen voxels: z~ = clip((z - p_lo) / (p_hi - p_lo), 0, 1) with
 * nearest-rank percentiles of z (Eq. 14; or their running EMA), bin =
 * min(nb - 1, floor(nb z~)), tau_b = nearest-rank q_b-quantile of w_max in
 * the bin (Eq. 11-12; q_b = q unless annealed), inside score x = [w_max >
 * tau_b] (x = 1 in a bin without threshold), m <- (1 - alpha) m + alpha x,
 * hysteresis state s (1 = in, 0 = out) (guard i); candidates are seen voxels
 * with s = out that the keep-halo guard does not protect (guard ii), and at
 * most floor(cap n) of them, the smallest (w_max, id), are pruned (guard
 * iii).  Decisions are FP32 with a fixed operation order.  ema_m and state
 * are updated in place; prune_mask [n] u8 is written; d_n_pruned (int64
 * device) receives the count.  Unseen voxels are unchanged and never pruned.
 * With no seen voxel nothing changes (pct_state included). */
/* The two halves of lv_prune_depth_quantile, for callers that want to start
 * on the depth statistics before w_max exists (see lv_fwd_out.stats_event).
 * lv_prune_bins takes the percentiles of z over the seen voxels (Eq. 14,
 * with the running update when pct_state is set) and bins the seen voxels
 * into n_bins depth bins; lv_prune_finish takes the per-bin quantiles of
 * w_max (Eq. 11-12) and applies guards i-iii.  Same arguments, same
 * workspace, bins first; lv_prune_depth_quantile is bins + finish on one
 * stream, and the split calls give the same bits. */
lv_status lv_prune_bins(int64_t n, const uint8_t* seen, const float* z, const lv_prune_params* p, void* workspace,
                        size_t ws_bytes, void* stream);
lv_status lv_prune_finish(int64_t n, const float* w_max, const uint8_t* seen, const float* z, float* ema_m,
                          uint8_t* state, const lv_prune_params* p, uint8_t* prune_mask, int64_t* d_n_pruned,
                          void* workspace, size_t ws_bytes, int32_t* d_status, void* stream);

lv_status lv_prune_depth_quantile(int64_t n, const float* w_max, const uint8_t* seen, const float* z,
                                  float* ema_m, uint8_t* state, const lv_prune_params* p, uint8_t* prune_mask,
                                  int64_t* d_n_pruned, void* workspace, size_t ws_bytes, int32_t* d_status,
                                  void* stream);

/* ------------------------------------------------------------------ */
/* priority-driven subdivision (Sec. IV-D, Eq. 13-16)                   */
/* ------------------------------------------------------------------ */

typedef struct {
  float kappa;      /* eligibility h > kappa * delta (Eq. 13), ~1 */
  float beta;       /* far bias b(z) = 1 + beta z~ (Eq. 15), 0.1-0.3 */
  int32_t top_ppm;  /* at most floor(top * n_alive) splits per step (50000 = 5 %) */
  int32_t l_max;    /* finest level: voxels at l_max are not split */
  int64_t budget;   /* global growth cap on the voxel count; each split adds 7 */
  int32_t lo_ppm;   /* depth percentiles for Eq. 14 (50000 / 950000) */
  int32_t hi_ppm;
  /* running depth percentiles, as in lv_prune_params (0 / NULL: off) */
  float pct_ema;
  float* pct_state;  /* device float[2], NaN = uninitialised */
} lv_subdiv_params;

/* One per-voxel auxiliary array carried through topology changes (Adam
 * moments, EMA state...): survivors copy their row, children get `fill`
 * (bit pattern of one element) in every element. */
typedef struct {
  const void* in;      /* device [n][width] */
  void* out;           /* device [capacity][width] */
  int32_t width;       /* elements per voxel */
  int32_t elem_bytes;  /* 1, 2 or 4 */
  uint32_t fill;       /* child fill bit pattern (0 for optimizer moments) */
} lv_aux_array;

#define LV_MAX_AUX 16

size_t lv_subdivide_workspace_size(int64_t n, const lv_subdiv_params* p);

/* alive = !prune_mask (prune_mask nullable); z~ from the nearest-rank
 * percentiles of z over alive & seen voxels; eligible = alive & seen &
 * level < l_max & h > kappa * delta; priority p = u (1 + beta z~) (Eq. 15-16);
 * k = min(floor(top n_alive), floor((budget - n_alive) / 7), #eligible);
 * the k eligible voxels with the largest (p, then smallest id) are split.
 * Output (capacity out->n >= n_alive + 7 k, else LV_ERR_CAPACITY in
 * d_status): survivors in id order, then 8 children per split parent in
 * parent order, child c at centre + (h/2)(+-1 by bits of c), half-size h/2,
 * level + 1, corners = the parent's trilinear field at the child corners
 * (FP32, lerp a(1-t)+bt along x, then y, then z), SH copied (in the input
 * dtypes).  Auxiliary arrays follow the same order.  selected [n] u8 marks
 * split parents; d_n_new (int64 device) receives the new count.  `out` must
 * use the same dtypes as `in`; out->geom / level / density / sh are written
 * through the (const-qualified) pointers of `out`.  n_aux <= LV_MAX_AUX.
 * FP16 corner densities are interpolated in FP32 and rounded back to FP16. */
lv_status lv_subdivide_priority(const lv_voxels* in, const float* delta, const float* z, const float* u,
                                const uint8_t* seen, const uint8_t* prune_mask, const lv_subdiv_params* p,
                                const lv_aux_array* aux, int n_aux, const lv_voxels* out, uint8_t* selected,
                                int64_t* d_n_new, void* workspace, size_t ws_bytes, int32_t* d_status,
                                void* stream);

/* Stable compaction without a split, e.g. to drop pruned voxels on steps
 * that do not subdivide.  Rows i with keep[i] != 0 (device [n] u8) are
 * written in id order to out (geom, level, corner densities, SH, in the
 * input dtypes) and to every auxiliary array (lv_aux_array.fill unused);
 * d_n_new (device int64, nullable) receives the number kept.  out->n is the
 * output capacity: fewer rows than kept sets LV_ERR_CAPACITY in d_status
 * and writes nothing.  The same as lv_subdivide_priority with no voxel
 * selected and prune_mask = !keep.  Shared-vertex scenes (in->vidx) are not
 * supported here (LV_ERR_UNSUPPORTED): pass the per-voxel index rows as an
 * auxiliary array instead.  workspace: lv_compact_workspace_size(n). */
size_t lv_compact_workspace_size(int64_t n);
lv_status lv_compact(const lv_voxels* in, const uint8_t* keep, const lv_aux_array* aux, int n_aux,
                     const lv_voxels* out, int64_t* d_n_new, void* workspace, size_t ws_bytes, int32_t* d_status,
                     void* stream);

/* The two halves of lv_subdivide_priority, for callers that want to look at
 * the selection (selected, d_n_new) before the arrays are written, or to time
 * the halves separately.  lv_subdivide_select takes the selection and
 * checks that out_capacity >= n_alive + 7 k (else LV_ERR_CAPACITY in d_status
 * and the apply step writes nothing); lv_subdivide_apply writes the survivors
 * and children into `out` (one kernel).  Both take the same `in`, `p` and
 * workspace, select first; the workspace carries the selection between them. */
lv_status lv_subdivide_select(const lv_voxels* in, const float* delta, const float* z, const float* u,
                              const uint8_t* seen, const uint8_t* prune_mask, const lv_subdiv_params* p,
                              int64_t out_capacity, uint8_t* selected, int64_t* d_n_new, void* workspace,
                              size_t ws_bytes, int32_t* d_status, void* stream);
lv_status lv_subdivide_apply(const lv_voxels* in, const lv_subdiv_params* p, const lv_aux_array* aux, int n_aux,
                             const lv_voxels* out, void* workspace, size_t ws_bytes, void* stream);

/* The topology change of the step (Sec. IV-D, Eq. 13-16 with the optimizer
 * refresh, and the removal of the voxels pruned by Sec. IV-C) written in
 * place: only the rows that change are read or written, instead of every
 * survivor being copied to new arrays.  Call after lv_subdivide_select on
 * the same workspace and stream, with out_capacity = capacity and the same
 * prune mask.  vox: the n = vox->n current rows, in arrays that hold
 * `capacity` rows (geom, level, density, sh); the result holds n' = n - h +
 * 7k rows (h pruned, k split; d_n_new of the select step), the same rows as
 * lv_subdivide_apply writes, placed as follows:
 *   - a split parent's row becomes its child 0;
 *   - children 1..7 of the r-th split parent (id order) take slots 7r .. 7r+6
 *     of [the pruned rows in increasing index, then rows n, n + 1, ...];
 *   - if 7k < h, the occupied rows at index >= n' then move, in increasing
 *     index, into the rows below n' still empty, in increasing index;
 *   - every other row keeps its index and its bytes.
 * Child values and auxiliary fills are those of lv_subdivide_apply.  aux[a].out
 * is updated in place (aux[a].in must be NULL or equal to out); every array
 * must hold `capacity` rows.  If capacity < n' the select step has set
 * LV_ERR_CAPACITY and nothing is written.  Host errors: LV_ERR_INVALID_ARG
 * (null or inconsistent arrays, capacity < n), LV_ERR_WORKSPACE. */
lv_status lv_subdivide_apply_inplace(const lv_voxels* vox, int64_t capacity, const lv_subdiv_params* p,
                                     const lv_aux_array* aux, int n_aux, void* workspace, size_t ws_bytes,
                                     void* stream);

/* Row scatter of up to LV_MAX_AUX arrays in one launch: for each array,
 * dst[idx[j]] = src[j] for j < m (rows of row_bytes bytes), or, with idx =
 * NULL, dst[j] = src[j] (a plain copy of m rows).  The paper has no
 * counterpart: it undoes an in-place topology change from rows the caller
 * saved before it (the rows of the split parents and of the pruned voxels),
 * for a rollback, and lets a benchmark return to the same scene after every
 * step.  Rows move as 16-byte words when row_bytes and both pointers allow
 * it (a plain copy: when the whole range does), byte by byte otherwise.
 * idx: device int64 [m], values distinct within an array and below the
 * destination's rows.  Device pointers; src and dst must not overlap. */
typedef struct {
  void* dst;
  const void* src;
  int64_t row_bytes;
  const int64_t* idx; /* device [m], or NULL */
  int64_t m;
} lv_rows;
lv_status lv_rows_scatter(const lv_rows* arrays, int n_arrays, void* stream);

/* ------------------------------------------------------------------ */
/* LF-weighted photometric loss (Sec. IV-B, Eq. 7-10, 18)               */
/* ------------------------------------------------------------------ */

typedef struct {
  float eps;        /* Eq. 7 epsilon (1e-3) */
  float gamma_max;  /* Eq. 9 */
  float t0, t1;     /* Eq. 9 ramp start / end (iterations) */
  int32_t pctl_ppm; /* Sobel magnitude normalisation percentile (990000 = P99) */
  float* edge_out;  /* optional device [P] FP32: the normalised edge magnitude s
                     * of every pixel (Eq. 7), e.g. for the keep-halo guard */
} lv_lf_params;

/* gamma(t) of Eq. 9 (host scalar). */
float lv_lf_gamma(float t, const lv_lf_params* p);

size_t lv_lf_workspace_size(const int32_t* widths, const int32_t* heights, int n_views);

/* Per view: Y = (R + G + B) / 3 of gt, 3x3 Sobel with replicated border,
 * s = clip(|grad| / P_pctl(|grad|), 0, 1) (0 if the percentile is 0,
 * nearest rank), w = (eps + 1 - s)^gamma(t), w~ = w / mean(w) (Eq. 7-8),
 * loss[v] = mean over pixels of w~ * mean_c (rgb - gt)^2 (Eq. 10, 18) and
 * dL_drgb = 2 / (3 |P_v|) w~ (rgb - gt).  rgb, gt, dL_drgb: [P][3] FP32;
 * loss: [n_views] FP32 device; dL_drgb nullable. */
lv_status lv_lf_weighted_loss(const float* rgb, const float* gt, const int32_t* widths, const int32_t* heights,
                              int n_views, float t, const lv_lf_params* p, float* loss, float* dL_drgb,
                              void* workspace, size_t ws_bytes, void* stream);

/* The two halves of lv_lf_weighted_loss.  The weight map w (Eq. 7-9) and its
 * per-view sum depend on the ground truth and gamma(t) only, so a caller can
 * compute them on a second stream while the forward pass renders rgb.
 * lv_lf_weights writes them into `workspace`; lv_lf_loss_from_weights then
 * reads them from the same workspace (same widths / heights) and writes loss
 * and dL_drgb exactly as lv_lf_weighted_loss does (bit-identical results).
 * lv_lf_weighted_loss is lv_lf_weights followed by lv_lf_loss_from_weights
 * on one stream.  The caller orders the two calls (an event when they run on
 * different streams) and keeps the workspace for the pair. */
lv_status lv_lf_weights(const float* gt, const int32_t* widths, const int32_t* heights, int n_views, float t,
                        const lv_lf_params* p, void* workspace, size_t ws_bytes, void* stream);
lv_status lv_lf_loss_from_weights(const float* rgb, const float* gt, const int32_t* widths, const int32_t* heights,
                                  int n_views, float* loss, float* dL_drgb, void* workspace, size_t ws_bytes,
                                  void* stream);

/* The per-view losses of a backward that fused the LF loss (lv_fwd_out.lf_*):
 * loss[v] = (the view's summed weighted squared error) / (3 |P_v|), the value
 * lv_lf_loss_from_weights writes up to the order of the FP64 sums.  Reads
 * and then clears the sums in `workspace` (lv_lf_weights clears them too), so
 * call it once per fused backward, after the backward on the stream.  loss:
 * device float[n_views]. */
lv_status lv_lf_loss_finish(const int32_t* widths, const int32_t* heights, int n_views, float* loss,
                            void* workspace, size_t ws_bytes, void* stream);

/* Allocation-free variant of lv_lf_weighted_loss.  The paper has no
 * counterpart: it exists for callers that cannot allocate device memory
 * themselves -- for instance code running as a plugin inside a host
 * application that owns every device allocation, or a latency-critical loop
 * that must not call cudaMalloc, which can synchronise the whole device.
 * The caller still passes the inputs and outputs; the scratch space lives in
 * one fixed device array of LV_LF_NOALLOC_SCRATCH_BYTES inside the library,
 * which every GPU that loads the library holds until the process exits.
 *  - Limit: the call needs lv_lf_workspace_size(widths, heights, n_views)
 *    <= LV_LF_NOALLOC_SCRATCH_BYTES (about 1.6 million pixels over all
 *    views); larger requests return LV_ERR_INVALID_ARG without launching.
 *  - The first call on each device looks up the array's device address once
 *    (with that device current); make that first call before any stream
 *    capture.  The address is kept for the life of the process: after a
 *    cudaDeviceReset (or any destruction of the device's primary context) the
 *    library's device array may be loaded elsewhere, so do not call this entry
 *    point again on that device until the library is reloaded.
 *  - All calls share the one array: calls that overlap on the GPU (for
 *    example on two streams at once) race and give wrong results.  Each call
 *    clears the parts of the array that must start at zero.
 * Arguments and results are those of lv_lf_weighted_loss. */
#define LV_LF_NOALLOC_SCRATCH_BYTES (16u << 20)
lv_status lv_lf_weighted_loss_noalloc(const float* rgb, const float* gt, const int32_t* widths,
                                      const int32_t* heights, int n_views, float t, const lv_lf_params* p,
                                      float* loss, float* dL_drgb, void* stream);

/* ------------------------------------------------------------------ */
/* rest of the training step (Eq. 17 auxiliaries, Adam; Sec. IV-D)     */
/* ------------------------------------------------------------------ */

/* Workspace for lv_transmittance_loss and lv_adam_voxels (a few bytes of
 * reduction scratch; one buffer may serve both calls on one stream). */
size_t lv_train_workspace_size(void);

/* Transmittance concentration of Eq. 17 (final T near 0 or 1), read as
 * L_Tc = weight / n_pix * sum_p T_p (1 - T_p).  loss: device float (written);
 * dL_dT: device [n_pix] FP32, nullable, weight (1 - 2 T_p) / n_pix written or,
 * with accumulate != 0, added -- it feeds lv_rasterize_backward's dL_dT. */
lv_status lv_transmittance_loss(const float* T, int64_t n_pix, float weight, float* loss, float* dL_dT,
                                int accumulate, void* workspace, size_t ws_bytes, void* stream);

typedef struct {
  float lr_density;  /* learning rates */
  float lr_sh;
  float beta1;       /* Adam moment decays, in [0, 1) */
  float beta2;
  float eps;
  int64_t step;      /* global step t >= 1 for the bias corrections 1 / (1 - beta^t) */
  float tv_weight;   /* lambda of the density total variation of Eq. 17 (0: none) */
} lv_adam_params;

/* One Adam step on the voxel parameters, in place.  The density gradient is
 * d_density plus the gradient of L_tv = tv_weight / n * sum_v sum over the
 * 12 edges (i, j) of the voxel's corner cube (corner c = x + 2y + 4z) of
 * (d_i - d_j)^2 -- Eq. 17's total variation of the density field, read on the
 * 8 corner densities -- then for every parameter: m <- b1 m + (1 - b1) g,
 * v <- b2 v + (1 - b2) g^2, p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 -
 * b2^t)) + eps).  FP32 arithmetic; FP16 / BF16 parameter storage is rounded
 * to nearest after the update.  density: device [n][8] (F32 or F16); sh:
 * device [n][48] (F32 or BF16), updated only when d_sh is given; gradients
 * and moments: device FP32 arrays of the same shapes, 16-byte aligned.
 * tv_loss: nullable device float receiving L_tv of the densities before the
 * update.  Children of a subdivision start from zero moments (the optimizer
 * refresh of Sec. IV-D: lv_subdivide_apply fills them). */
lv_status lv_adam_voxels(int64_t n, void* density, lv_dtype density_dtype, void* sh, lv_dtype sh_dtype,
                         const float* d_density, const float* d_sh, float* m_density, float* v_density,
                         float* m_sh, float* v_sh, const lv_adam_params* p, float* tv_loss, void* workspace,
                         size_t ws_bytes, void* stream);

/* One Adam step (as lv_adam_voxels, learning rate lr; p->lr_* and
 * p->tv_weight unused) on a flat parameter array of `count` elements, in
 * place: e.g. the vertex densities of the shared grid-vertex variant.
 * param: device F32 / F16 / BF16; grad, m, v: device FP32, 16-byte aligned. */
lv_status lv_adam_array(int64_t count, void* param, lv_dtype dtype, const float* grad, float* m, float* v, float lr,
                        const lv_adam_params* p, void* stream);

/* ------------------------------------------------------------------ */
/* shared grid-vertex densities (density-model variant)                */
/* ------------------------------------------------------------------ */

size_t lv_vertex_index_workspace_size(int64_t n);

/* Corner -> vertex numbering.  Corner c of voxel v lies at centre +- h; its
 * coordinates in units of `unit` (the finest half-size, e.g. root edge /
 * 2^(l_max + 1)) must be integers in [-2^20, 2^20), else the status word gets
 * LV_ERR_INVALID_ARG.  Corners at the same point share a vertex; vertex ids
 * are the ranks of the distinct points in (z, y, x) key order, so they do not
 * depend on scheduling.  vidx: device [n][8] u32 (written); d_n_vert: device
 * int64 (the vertex count). */
lv_status lv_build_vertex_index(const float* geom, int64_t n, double unit, uint32_t* vidx, int64_t* d_n_vert,
                                void* workspace, size_t ws_bytes, int32_t* d_status, void* stream);

/* corners[8 v + c] = vertex_values[vidx[8 v + c]] as FP32 (dtype LV_F32 or LV_F16). */
lv_status lv_vertex_gather(const uint32_t* vidx, int64_t n, const void* vertex_values, lv_dtype dtype,
                           float* corners, void* stream);

/* vertex_sum[vidx[8 v + c]] += corners[8 v + c] (atomics across the voxels
 * that share a vertex), and vertex_count[...] += 1 when vertex_count is given
 * (for averaging per-voxel corners into vertices).  Both device FP32 arrays
 * of the vertex count, accumulated (the caller zeroes them). */
lv_status lv_vertex_scatter_add(const uint32_t* vidx, int64_t n, const float* corners, float* vertex_sum,
                                float* vertex_count, void* stream);

/* ------------------------------------------------------------------ */
/* misc                                                                 */
/* ------------------------------------------------------------------ */

/* Human-readable description of the calling thread's last error ("" if none). */
const char* lv_last_error(void);

/* Synchronise `stream` and return the status word a call left on the device
 * (*d_status, an lv_status code; LV_OK when no kernel reported anything).
 * LV_ERR_CUDA when the copy or the synchronisation fails, or when the word
 * holds no lv_status code.  The word is not cleared. */
lv_status lv_check_status(const int32_t* d_status, void* stream);

/* (major << 16) | minor */
int32_t lv_version(void);

/* Kernels launched by this library since load (all threads), for reporting. */
int64_t lv_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* LITEVOXEL_H */

// lv_tune.cu -- autotuner of the composite schedule (host code).  Every
// candidate (tile edge 8 / 16 / 32, one block per tile or persistent warps
// on a work counter, batch of 32 / 64 / 128 list entries staged per warp
// round) runs the caller's forward + backward on the caller's
// scene and views; the fastest one, timed with CUDA events on the caller's
// stream, is returned and optionally remembered in a text cache file.
#include <stdio.h>
#include <string.h>

#include <string>

#include "lv_common.cuh"

namespace lv {
namespace {

constexpr int N_TILES = 3;
constexpr int TILES[N_TILES] = {8, 16, 32};
constexpr int N_BATCH = 3;
constexpr int BATCHES[N_BATCH] = {32, 64, 128};

struct TuneWs {
  float* rgb;
  float* T;
  uint32_t* n_contrib;
  float* dL;
  float* d_density;
  float* d_sh;
  unsigned long long* wmax;
  float* z_min;
  float* delta_min;
  uint8_t* seen;
  int32_t* status;
  void* fwd;
  size_t fwd_bytes;
  size_t bytes;
};

int64_t total_pixels(const lv_camera* cams, int n_views) {
  int64_t p = 0;
  for (int v = 0; v < n_views; ++v) p += (int64_t)cams[v].width * cams[v].height;
  return p;
}

TuneWs carve_tune(void* base, int64_t n, const lv_camera* cams, int n_views, const lv_raster_opts* opts,
                  int64_t pair_capacity) {
  TuneWs w;
  Carve c(base);
  const int64_t P = total_pixels(cams, n_views);
  w.rgb = c.take<float>(3 * P);
  w.T = c.take<float>(P);
  w.n_contrib = c.take<uint32_t>(P);
  w.dL = c.take<float>(3 * P);
  w.d_density = c.take<float>(8 * n);
  w.d_sh = c.take<float>(48 * n);
  w.wmax = c.take<unsigned long long>(n);
  w.z_min = c.take<float>(n);
  w.delta_min = c.take<float>(n);
  w.seen = c.take<uint8_t>(n);
  w.status = c.take<int32_t>(4);
  w.fwd_bytes = 0;
  for (int t = 0; t < N_TILES; ++t) {
    lv_raster_opts o = *opts;
    o.tile = TILES[t];
    const size_t b = lv_forward_workspace_size(n, cams, n_views, &o, pair_capacity);
    if (b > w.fwd_bytes) w.fwd_bytes = b;
  }
  w.fwd = c.take<char>(w.fwd_bytes);
  w.bytes = c.off + 256;
  return w;
}

// device name | voxels | view sizes | flags other than the schedule
std::string cache_key(int64_t n, const lv_camera* cams, int n_views, const lv_raster_opts* base) {
  cudaDeviceProp prop;
  int dev = 0;
  std::string key = "gpu";
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) key = prop.name;
  for (char& ch : key)
    if (ch == ' ' || ch == '\t') ch = '_';
  key += "|" + std::to_string(n);
  for (int v = 0; v < n_views; ++v) key += "|" + std::to_string(cams[v].width) + "x" + std::to_string(cams[v].height);
  key += "|f" + std::to_string(base->flags & ~(uint32_t)LV_FLAG_PERSISTENT);
  return key;
}

bool cache_lookup(const char* path, const std::string& key, int* tile, int* persistent, int* batch) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[2048];
  bool hit = false;
  while (fgets(line, sizeof(line), f)) {
    char k[1800];
    int t = 0, p = 0, b = 32;
    const int got = sscanf(line, "%1799s %d %d %d", k, &t, &p, &b);
    if (got >= 3 && key == k && (t == 8 || t == 16 || t == 32) && (b == 32 || b == 64 || (b == 128 && t < 32))) {
      *tile = t;
      *persistent = p ? 1 : 0;
      *batch = got == 4 ? b : 32;
      hit = true;  // the last matching line wins
    }
  }
  fclose(f);
  return hit;
}

void cache_store(const char* path, const std::string& key, int tile, int persistent, int batch) {
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d\n", key.c_str(), tile, persistent, batch);
  fclose(f);
}

}  // namespace
}  // namespace lv

using namespace lv;

extern "C" size_t lv_autotune_workspace_size(int64_t n, const lv_camera* cams, int n_views,
                                             const lv_raster_opts* base, int64_t pair_capacity) {
  if (n < 0 || !cams || n_views < 1 || n_views > LV_MAX_VIEWS || !base || pair_capacity < 0) return 0;
  return carve_tune(nullptr, n, cams, n_views, base, pair_capacity).bytes;
}

extern "C" lv_status lv_autotune(const lv_voxels* vox, const lv_camera* cams, int n_views,
                                 const lv_raster_opts* base, int64_t pair_capacity, int reps, lv_raster_opts* best,
                                 float* ms_out, const char* cache_path, void* workspace, size_t ws_bytes,
                                 void* stream) {
  if (!vox || !cams || !base || !best || n_views < 1 || n_views > LV_MAX_VIEWS || reps < 1 || reps > 1000) {
    set_error("lv_autotune: bad arguments");
    return LV_ERR_INVALID_ARG;
  }
  if (ms_out)
    for (int i = 0; i < 2 * N_TILES * N_BATCH; ++i) ms_out[i] = -1.f;
  const std::string key = cache_key(vox->n, cams, n_views, base);
  int tile = 0, persistent = 0, batch = 32;
  if (cache_path && cache_lookup(cache_path, key, &tile, &persistent, &batch)) {
    *best = *base;
    best->tile = tile;
    best->batch = batch;
    best->flags = (base->flags & ~(uint32_t)LV_FLAG_PERSISTENT) | (persistent ? LV_FLAG_PERSISTENT : 0u);
    return LV_OK;
  }
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  TuneWs w = carve_tune(workspace, vox->n, cams, n_views, base, pair_capacity);
  if (ws_bytes < w.bytes) { set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return LV_ERR_WORKSPACE; }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t P = total_pixels(cams, n_views);
  cudaMemsetAsync(w.dL, 0, sizeof(float) * 3 * P, s);
  lv_fwd_out out;
  memset(&out, 0, sizeof(out));
  out.rgb = w.rgb;
  out.T = w.T;
  out.n_contrib = w.n_contrib;
  out.wmax_packed = w.wmax;
  out.z_min = w.z_min;
  out.delta_min = w.delta_min;
  out.seen = w.seen;
  cudaEvent_t e0, e1;
  if (cuda_check(cudaEventCreate(&e0), "lv_autotune") != LV_OK) return LV_ERR_CUDA;
  if (cuda_check(cudaEventCreate(&e1), "lv_autotune") != LV_OK) { cudaEventDestroy(e0); return LV_ERR_CUDA; }
  float best_ms = -1.f;
  lv_status result = LV_OK;
  for (int c = 0; c < 2 * N_TILES * N_BATCH && result == LV_OK; ++c) {
    const int t = c / (2 * N_BATCH), p = (c / N_BATCH) % 2, b = c % N_BATCH;
    if (TILES[t] == 32 && BATCHES[b] == 128) continue;  // more shared memory than a block has
    {
      lv_raster_opts o = *base;
      o.tile = TILES[t];
      o.batch = BATCHES[b];
      o.flags = (base->flags & ~(uint32_t)(LV_FLAG_PERSISTENT | LV_FLAG_SYNC_CHECK)) | (p ? LV_FLAG_PERSISTENT : 0u);
      auto step = [&]() -> lv_status {
        lv_status e = lv_rasterize_forward(vox, cams, n_views, &o, &out, w.fwd, w.fwd_bytes, pair_capacity,
                                           w.status, stream);
        if (e != LV_OK) return e;
        return lv_rasterize_backward(vox, cams, n_views, &o, &out, w.fwd, w.fwd_bytes, pair_capacity, w.dL, nullptr,
                                     nullptr, w.d_density, w.d_sh, 0, w.status, stream);
      };
      cudaMemsetAsync(w.status, 0, sizeof(int32_t), s);
      lv_status e = step();  // warm-up; also finds out whether the pairs fit
      if (e == LV_OK) e = lv_check_status(w.status, stream);
      if (e == LV_ERR_CAPACITY) continue;  // this tile size needs more pairs than the capacity: skipped
      if (e != LV_OK) { result = e; break; }
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && e == LV_OK; ++r) e = step();
      cudaEventRecord(e1, s);
      if (e == LV_OK) e = cuda_check(cudaEventSynchronize(e1), "lv_autotune");
      if (e != LV_OK) { result = e; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= (float)reps;
      if (ms_out) ms_out[c] = ms;
      if (best_ms < 0.f || ms < best_ms) {
        best_ms = ms;
        tile = TILES[t];
        persistent = p;
        batch = BATCHES[b];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != LV_OK) return result;
  if (best_ms < 0.f) {
    set_error("lv_autotune: no tile size fits the pair capacity");
    return LV_ERR_CAPACITY;
  }
  *best = *base;
  best->tile = tile;
  best->batch = batch;
  best->flags = (base->flags & ~(uint32_t)LV_FLAG_PERSISTENT) | (persistent ? LV_FLAG_PERSISTENT : 0u);
  if (cache_path) cache_store(cache_path, key, tile, persistent, batch);
  return LV_OK;
}

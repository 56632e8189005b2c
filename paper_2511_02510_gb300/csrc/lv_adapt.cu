// lv_adapt.cu -- depth-quantile pruning (LiteVoxel Sec. IV-C, Eq. 11-12 with
// guards i-iii) and priority-driven subdivision (Sec. IV-D, Eq. 13-16)
// for sm_103a.  Every selection (percentiles, per-bin quantiles, the cap, the
// top-k) is an exact radix select on order-preserving 32-bit keys, so the
// integer outputs do not depend on thread scheduling; all FP32 decisions use
// a fixed operation order (__fmul_rn / __fadd_rn / __fdiv_rn).
#include <algorithm>

#include "lv_prims.cuh"

namespace lv {

namespace {

constexpr int TPB = 256;

inline int blocks_for(int64_t n) {
  int64_t b = (n + TPB - 1) / TPB;
  return (int)(b < 1 ? 1 : b);
}

// The per-voxel kernels give each thread IPT consecutive voxels (block b owns
// voxels [b EB, (b + 1) EB)), issue all the thread's loads before its stores,
// and combine counts once per block.  Thread order then equals id order
// inside a block, which the tie ranks rely on.
constexpr int IPT = 4;
constexpr int EB = TPB * IPT;
inline int eblocks(int64_t n) {
  int64_t b = (n + EB - 1) / EB;
  return (int)(b < 1 ? 1 : b);
}
__device__ __forceinline__ int64_t first_item() { return blockIdx.x * (int64_t)EB + (int64_t)threadIdx.x * IPT; }

// A thread's IPT (= 4) consecutive elements in one 4-, 8- or 16-byte access
// when they are all in range and the array is aligned for it, else one by one
// (out-of-range elements read as `fill`, are not written).
template <typename T> struct Vec4T;
template <> struct Vec4T<uint8_t> { using V = uchar4; };
template <> struct Vec4T<uint16_t> { using V = ushort4; };
template <> struct Vec4T<uint32_t> { using V = uint4; };
template <> struct Vec4T<float> { using V = float4; };
static_assert(IPT == 4, "the vector accesses move four elements");

template <typename T>
__device__ __forceinline__ void load4(const T* __restrict__ p, int64_t i0, int64_t n, T* v, T fill) {
  using V = typename Vec4T<T>::V;
  if (i0 + 3 < n && ((uintptr_t)p & (sizeof(V) - 1)) == 0) {
    const V q = *(const V*)(p + i0);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = i0 + u < n ? p[i0 + u] : fill;
  }
}

template <typename T>
__device__ __forceinline__ void store4(T* __restrict__ p, int64_t i0, int64_t n, const T* v) {
  using V = typename Vec4T<T>::V;
  if (i0 + 3 < n && ((uintptr_t)p & (sizeof(V) - 1)) == 0) {
    V q;
    q.x = v[0]; q.y = v[1]; q.z = v[2]; q.w = v[3];
    *(V*)(p + i0) = q;
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u < n) p[i0 + u] = v[u];
  }
}

// sum of one count per thread over the block (every thread calls; all get it)
__device__ __forceinline__ uint32_t block_total(uint32_t c) {
  __shared__ uint32_t s_part[TPB / 32];
  c = __reduce_add_sync(FULL, c);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = c;
  __syncthreads();
  uint32_t t = 0;
#pragma unroll
  for (int w = 0; w < TPB / 32; ++w) t += s_part[w];
  __syncthreads();  // s_part is reused by the next call
  return t;
}

// sum of the per-block counts of all earlier blocks (every thread calls): the
// block's offset among the flagged items, read straight from the counts
__device__ __forceinline__ uint32_t block_offset(const uint32_t* __restrict__ blk) {
  uint32_t c = 0;
  for (unsigned k = threadIdx.x; k < blockIdx.x; k += TPB) c += blk[k];
  return block_total(c);
}

// exclusive prefix of one count per thread, in thread order (every thread calls)
__device__ __forceinline__ uint32_t block_excl_count(uint32_t c) {
  __shared__ uint32_t s_part[TPB / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_part[warp] = x;
  __syncthreads();
  uint32_t pre = 0;
#pragma unroll
  for (int w = 0; w < TPB / 32; ++w) pre += w < warp ? s_part[w] : 0u;
  __syncthreads();
  return pre + x - c;
}

// A select's first digit counted by the kernel that produces its keys
// (select_kth_first): each block counts into shared memory, then adds its
// nonzero counts to h0.  h0 == nullptr: nothing is counted.
constexpr int FH_WORDS = 4096;  // rows * bins of one block's counts
struct FirstHist {
  uint32_t* h0;
  int rows, shift, bins, radix;
};
inline FirstHist first_hist(uint32_t* h0, int n_queries, int rows) {
  FirstHist f;
  f.shift = select_first_shift(n_queries);
  f.bins = 1 << (32 - f.shift);
  f.radix = select_radix(n_queries);
  f.rows = rows;
  f.h0 = rows * f.bins <= FH_WORDS ? h0 : nullptr;
  return f;
}
// every thread of the block calls (barriers inside)
__device__ __forceinline__ void fh_clear(const FirstHist& f, uint32_t* sh) {
  if (f.h0)
    for (int i = threadIdx.x; i < f.rows * f.bins; i += TPB) sh[i] = 0u;
  __syncthreads();
}
__device__ __forceinline__ void fh_count(const FirstHist& f, uint32_t* sh, int row, uint32_t key) {
  if (f.h0 && row >= 0 && row < f.rows) atomicAdd(&sh[row * f.bins + (int)(key >> f.shift)], 1u);
}
__device__ __forceinline__ void fh_flush(const FirstHist& f, const uint32_t* sh) {
  __syncthreads();
  if (f.h0)
    for (int i = threadIdx.x; i < f.rows * f.bins; i += TPB) {
      const uint32_t c = sh[i];
      if (c) atomicAdd(&f.h0[(i / f.bins) * f.radix + (i % f.bins)], c);
    }
}

__device__ __forceinline__ float key_to_float(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

// nearest rank: max(1, ceil(ppm * m / 1e6)), 0 when m == 0
__device__ __forceinline__ uint32_t rank_ppm(uint32_t ppm, uint32_t m) {
  if (m == 0) return 0;
  unsigned long long k = ((unsigned long long)ppm * m + 999999ull) / 1000000ull;
  if (k < 1) k = 1;
  if (k > m) k = m;
  return (uint32_t)k;
}

// Eq. 14 in FP32: clip((z - p_lo) / (p_hi - p_lo), 0, 1); 0 when p_hi <= p_lo
__device__ __forceinline__ float depth_norm(float z, float p_lo, float p_hi) {
  float den = __fsub_rn(p_hi, p_lo);
  if (!(den > 0.f)) return 0.f;
  float r = __fdiv_rn(__fsub_rn(z, p_lo), den);
  return fminf(fmaxf(r, 0.f), 1.f);
}

// ------------------------------------------------------------------ pruning
struct PruneState {
  uint32_t ns;            // seen voxels
  uint32_t n_cand;        // out-state candidates after the update
  uint32_t c_lt;          // candidates strictly below the cap threshold
  uint32_t all;           // 1 when every candidate is pruned (n_cand <= cap)
  float p_lo, p_hi;       // depth normalisation of this step (Eq. 14, running or not)
  uint32_t bin_cnt[SELECT_MAX_QUERIES];
};

struct PruneWs {
  PruneState* st;
  SelectQuery* q;
  void* sel_tmp;
  uint16_t* grp;
  uint32_t* zkey;
  uint32_t* wkey;
  uint32_t* blk;  // per-block tie counts -> offsets
  uint32_t* h0_tau;  // first-digit counts of the per-bin selection (k_pr_wkey)
  uint32_t* h0_cap;  // first-digit counts of the cap's selection (k_pr_update)
  size_t bytes;
};

PruneWs carve_prune(void* base, int64_t n) {
  PruneWs w;
  Carve c(base);
  w.st = c.take<PruneState>(1);
  w.q = c.take<SelectQuery>(SELECT_MAX_QUERIES);
  w.sel_tmp = c.take<char>(select_tmp_bytes(SELECT_MAX_QUERIES));
  w.grp = c.take<uint16_t>(n);
  w.zkey = c.take<uint32_t>(n);
  w.wkey = c.take<uint32_t>(n);
  w.blk = c.take<uint32_t>(n / TPB + 1);
  w.h0_tau = c.take<uint32_t>(2 * FH_WORDS);  // covers select_radix(nq) * nq whenever counted
  w.h0_cap = c.take<uint32_t>(select_radix(1));
  w.bytes = c.off + 256;
  return w;
}

__global__ void k_pr_seen(int64_t n, const uint8_t* __restrict__ seen, const float* __restrict__ z, uint16_t* grp,
                          uint32_t* zkey, PruneState* st) {
  const int64_t i0 = first_item();
  uint8_t sv[IPT];
  float zv[IPT];
  load4(seen, i0, n, sv, (uint8_t)0);
  load4(z, i0, n, zv, 0.f);
  uint16_t gv[IPT];
  uint32_t zk[IPT];
  uint32_t c = 0;
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    gv[u] = sv[u] ? 0 : GROUP_NONE;
    zk[u] = order_key(zv[u]);
    c += sv[u] ? 1u : 0u;  // padding reads 0
  }
  store4(grp, i0, n, gv);
  store4(zkey, i0, n, zk);
  // one atomic per block (a same-address atomic per warp serialises at the L2)
  const uint32_t b = block_total(c);
  if (threadIdx.x == 0 && b) atomicAdd(&st->ns, b);
}

// order keys of w_max for the per-bin quantiles and the cap
// order keys of w_max; the per-bin selection's first digit is counted here (row = depth bin)
__global__ void k_pr_wkey(int64_t n, const float* __restrict__ w_max, const uint16_t* __restrict__ grp,
                          uint32_t* __restrict__ wkey, const FirstHist fh) {
  __shared__ uint32_t sh[FH_WORDS];
  fh_clear(fh, sh);
  const int64_t i0 = first_item();
  float wv[IPT];
  uint16_t gv[IPT];
  load4(w_max, i0, n, wv, 0.f);
  load4(grp, i0, n, gv, GROUP_NONE);
  uint32_t wk[IPT];
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    wk[u] = order_key(wv[u]);
    if (gv[u] != GROUP_NONE) fh_count(fh, sh, gv[u], wk[u]);  // padding reads GROUP_NONE
  }
  store4(wkey, i0, n, wk);
  fh_flush(fh, sh);
}

__global__ void k_pr_pct_queries(SelectQuery* q, const PruneState* st, uint32_t lo_ppm, uint32_t hi_ppm,
                                 void* sel_tmp) {
  select_prepare(q, 2, sel_tmp);
  if (threadIdx.x == 0) {
    q[0].group = 0; q[0].k = rank_ppm(lo_ppm, st->ns);
    q[1].group = 0; q[1].k = rank_ppm(hi_ppm, st->ns);
  }
}

// Running percentiles (Eq. 14 "running"): p <- (1 - r) p + r p_step over
// calls, FP32 with the products rounded separately; a NaN state takes the
// step's value.  Leaves this step's (p_lo, p_hi) in *lo_hi.
__device__ __forceinline__ void running_pct(const SelectQuery* pct, float* state, float r, float omr, float* lo_hi) {
  float p_lo = key_to_float(pct[0].result), p_hi = key_to_float(pct[1].result);
  if (state && r > 0.f) {
    if (isnan(state[0]) || isnan(state[1])) {
      state[0] = p_lo;
      state[1] = p_hi;
    } else {
      state[0] = __fadd_rn(__fmul_rn(omr, state[0]), __fmul_rn(r, p_lo));
      state[1] = __fadd_rn(__fmul_rn(omr, state[1]), __fmul_rn(r, p_hi));
      p_lo = state[0];
      p_hi = state[1];
    }
  }
  lo_hi[0] = p_lo;
  lo_hi[1] = p_hi;
}

__global__ void k_pr_pct_apply(const SelectQuery* pct, PruneState* st, float* state, float r, float omr) {
  if (threadIdx.x == 0 && st->ns > 0) running_pct(pct, state, r, omr, &st->p_lo);
}

// bin counts go through a block-local histogram (one global add per bin and block)
__global__ void k_pr_bin(int64_t n, const uint8_t* __restrict__ seen, const float* __restrict__ z, int nb,
                         uint16_t* grp, PruneState* st) {
  __shared__ uint32_t sh[SELECT_MAX_QUERIES];
  if (threadIdx.x < SELECT_MAX_QUERIES) sh[threadIdx.x] = 0;
  __syncthreads();
  const float p_lo = st->p_lo, p_hi = st->p_hi;
  const int64_t i0 = first_item();
  uint8_t sv[IPT];
  float zv[IPT];
  load4(seen, i0, n, sv, (uint8_t)0);
  load4(z, i0, n, zv, 0.f);
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    if (!sv[u]) continue;  // padding reads 0
    const float zt = depth_norm(zv[u], p_lo, p_hi);
    int b = (int)floorf(__fmul_rn((float)nb, zt));
    if (b > nb - 1) b = nb - 1;
    grp[i0 + u] = (uint16_t)b;
    atomicAdd(&sh[b], 1u);
  }
  __syncthreads();
  if (threadIdx.x < nb && sh[threadIdx.x]) atomicAdd(&st->bin_cnt[threadIdx.x], sh[threadIdx.x]);
}

// q_b in ppm: q, or the annealed quantile with its near/far relaxation
// (integers: qa = floor(q a / 1e6), q_b = floor(qa (1e6 nb - relax |2b+1-nb|) / (1e6 nb)))
__device__ __forceinline__ long long q_bin(long long q_ppm, long long anneal_ppm, long long relax_ppm, int b, int nb) {
  const long long qa = q_ppm * anneal_ppm / 1000000ll;
  long long dist = 2ll * b + 1 - nb;
  if (dist < 0) dist = -dist;
  const long long den = 1000000ll * nb;
  return qa * (den - relax_ppm * dist) / den;
}

// a bin with q_b = 0 gets k = 0: no threshold (result stays 0xffffffff)
__global__ void k_pr_tau_queries(SelectQuery* q, const PruneState* st, int nb, uint32_t q_ppm, int anneal,
                                 uint32_t anneal_ppm, uint32_t relax_ppm, void* sel_tmp) {
  select_prepare(q, nb, sel_tmp);
  int b = threadIdx.x;
  if (b < nb) {
    const long long qb = anneal ? q_bin(q_ppm, anneal_ppm, relax_ppm, b, nb) : (long long)q_ppm;
    q[b].group = b;
    q[b].k = qb > 0 ? rank_ppm((uint32_t)qb, st->bin_cnt[b]) : 0u;
  }
}

// guard i: EMA of the inside score and hysteresis; guard ii: keep-halo
// protection; the candidates (out state, not protected) are flagged in mask
// and grouped in cand_grp
struct Halo {
  float small, w, edge;
  const float4* geom;
  const float* delta;
  const float* edge_score;
  const float* w_max;
};

__global__ void k_pr_update(int64_t n, const uint16_t* __restrict__ grp, const uint32_t* __restrict__ wkey,
                            const SelectQuery* tau, float alpha, float oma, float m_low, float m_high, float* ema_m,
                            uint8_t* state, const Halo halo, uint8_t* mask, uint16_t* cand_grp, PruneState* st,
                            const FirstHist fh) {
  __shared__ uint32_t sh[FH_WORDS];
  fh_clear(fh, sh);
  const int64_t i0 = first_item();
  uint16_t gv[IPT];
  uint32_t kv[IPT];
  float mv[IPT];
  uint8_t stv[IPT];
  load4(grp, i0, n, gv, GROUP_NONE);
  load4(wkey, i0, n, kv, 0u);
  load4((const float*)ema_m, i0, n, mv, 0.f);
  load4((const uint8_t*)state, i0, n, stv, (uint8_t)0);
  uint16_t cg[IPT];
  uint8_t mk[IPT];
  uint32_t c = 0;
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    const int64_t i = i0 + u;
    bool cand = false;
    const uint16_t b = gv[u];  // padding reads GROUP_NONE
    if (b != GROUP_NONE) {
      const uint32_t t = tau[b].result;
      const float x = (t == 0xffffffffu || kv[u] > t) ? 1.f : 0.f;  // no threshold: votes in
      const float m = __fadd_rn(__fmul_rn(oma, mv[u]), __fmul_rn(alpha, x));
      mv[u] = m;
      uint8_t s = stv[u];
      if (m < m_low) s = 0;
      else if (m > m_high) s = 1;
      stv[u] = s;
      bool prot = false;
      if (halo.small > 0.f && halo.geom && halo.delta) prot = halo.geom[i].w < __fmul_rn(halo.small, halo.delta[i]);
      if (halo.edge_score) prot = prot || (halo.w_max[i] >= halo.w && halo.edge_score[i] >= halo.edge);
      cand = s == 0 && !prot;
    }
    cg[u] = cand ? 0 : GROUP_NONE;
    mk[u] = cand ? 1 : 0;
    c += cand ? 1u : 0u;
    if (cand) fh_count(fh, sh, 0, kv[u]);  // the cap's selection among the candidates
  }
  // unseen voxels keep their EMA and state: the stores write their loaded values back
  store4(ema_m, i0, n, mv);
  store4(state, i0, n, stv);
  store4(cand_grp, i0, n, cg);
  store4(mask, i0, n, mk);
  // one atomic per block (a same-address atomic per warp serialises at the L2)
  const uint32_t bl = block_total(c);
  if (threadIdx.x == 0 && bl) atomicAdd(&st->n_cand, bl);
  fh_flush(fh, sh);
}

__global__ void k_pr_cap_query(SelectQuery* q, PruneState* st, uint32_t cap, void* sel_tmp) {
  select_prepare(q, 1, sel_tmp);
  if (threadIdx.x == 0) {
    st->all = st->n_cand <= cap ? 1u : 0u;
    q[0].group = 0;
    q[0].k = st->all ? 0u : cap;  // cap-th smallest w_max among the candidates
  }
}

// candidates strictly below the threshold, and per block the candidates at it
// (the ties compete by id: the need = cap - c_lt smallest ids among them go)
__global__ void k_pr_ties(int64_t n, const uint32_t* __restrict__ wkey, const SelectQuery* thr,
                          const uint8_t* __restrict__ cand, uint32_t* blk, PruneState* st) {
  const int64_t i0 = first_item();
  uint32_t clt = 0, ceq = 0;
  if (thr[0].k != 0) {
    const uint32_t v = thr[0].result;
    uint8_t cv[IPT];
    uint32_t kv[IPT];
    load4(cand, i0, n, cv, (uint8_t)0);
    load4(wkey, i0, n, kv, 0u);
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      if (!cv[u]) continue;  // padding reads 0
      const uint32_t k = kv[u];
      clt += k < v ? 1u : 0u;
      ceq += k == v ? 1u : 0u;
    }
  }
  // one atomic per block (a same-address atomic per warp serialises at the L2)
  const uint32_t bl = block_total(clt);
  const uint32_t be = block_total(ceq);
  if (threadIdx.x == 0) {
    if (bl) atomicAdd(&st->c_lt, bl);
    blk[blockIdx.x] = be;
  }
}

// mask holds the candidate flags on entry and the pruning decision on exit;
// a tie's rank among the ties (in id order) is its block's offset plus its
// rank inside the block
__global__ void k_pr_mask(int64_t n, const uint32_t* __restrict__ wkey, const SelectQuery* thr,
                          const uint32_t* __restrict__ blk, const PruneState* st, uint8_t* mask,
                          int64_t* n_pruned, uint32_t cap) {
  const int64_t i0 = first_item();
  const bool all = st->all != 0;
  const bool thr_ok = thr[0].k != 0;
  const uint32_t v = thr[0].result;
  bool lt[IPT], eq[IPT];
  uint8_t c[IPT];
  uint32_t kv[IPT];
  uint32_t ceq = 0;
  load4((const uint8_t*)mask, i0, n, c, (uint8_t)0);
  load4(wkey, i0, n, kv, 0u);
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    lt[u] = eq[u] = false;
    if (c[u] && !all && thr_ok) {  // padding reads 0
      lt[u] = kv[u] < v;
      eq[u] = kv[u] == v;
    }
    ceq += eq[u] ? 1u : 0u;
  }
  uint32_t r = block_excl_count(ceq) + block_offset(blk);  // every thread of the block takes part
  const uint32_t need = cap > st->c_lt ? cap - st->c_lt : 0u;
  uint8_t out[IPT];
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    const bool p = c[u] && (all || lt[u] || (eq[u] && r < need));
    r += eq[u] ? 1u : 0u;
    out[u] = p ? 1 : 0;
  }
  store4(mask, i0, n, out);
  if (i0 == 0 && n_pruned) *n_pruned = all ? (int64_t)st->n_cand : (int64_t)cap;
}

// ------------------------------------------------------------------ subdivision
struct SubState {
  uint32_t n_alive;
  uint32_t n_el;
  uint32_t k;
  uint32_t c_gt;      // eligible voxels with a strictly higher priority than the k-th
  uint32_t fits;      // output capacity suffices
  float p_lo, p_hi;   // depth normalisation of this step (Eq. 14, running or not)
};

struct SubWs {
  SubState* st;
  SelectQuery* q;   // [0..1] percentiles, [2] k-th priority, [3] tie id
  void* sel_tmp;
  uint16_t* grp;
  uint32_t* zkey;
  uint32_t* pkey;
  uint32_t* surv;
  uint32_t* sel;
  unsigned long long* surv_pos;
  uint32_t* sel_list;  // [k] selected parent ids in id order
  uint32_t* blk;       // per-block tie counts -> offsets
  uint32_t* blk_surv;  // per-block survivor counts (k_sd_select)
  uint32_t* blk_sel;   // per-block parent counts (k_sd_select)
  uint32_t* h0_pct;    // first-digit counts of the percentiles' selection (k_sd_flags)
  uint32_t* h0_top;    // first-digit counts of the top-k selection (k_sd_priority)
  unsigned long long* totals;
  void* scan_tmp;
  size_t bytes;
};

SubWs carve_sub(void* base, int64_t n) {
  SubWs w;
  Carve c(base);
  w.st = c.take<SubState>(1);
  w.q = c.take<SelectQuery>(8);
  w.sel_tmp = c.take<char>(select_tmp_bytes(SELECT_MAX_QUERIES));
  w.grp = c.take<uint16_t>(n);
  w.zkey = c.take<uint32_t>(n);
  w.pkey = c.take<uint32_t>(n);
  w.surv = c.take<uint32_t>(n);
  w.sel = c.take<uint32_t>(n);
  w.surv_pos = c.take<unsigned long long>(n);
  w.sel_list = c.take<uint32_t>(n);
  w.blk = c.take<uint32_t>(n / TPB + 1);
  w.blk_surv = c.take<uint32_t>(n / EB + 1);
  w.blk_sel = c.take<uint32_t>(n / EB + 1);
  w.h0_pct = c.take<uint32_t>(2 * select_radix(2));
  w.h0_top = c.take<uint32_t>(select_radix(1));
  w.totals = c.take<unsigned long long>(4);
  w.scan_tmp = c.take<char>(scan2_tmp_bytes());
  w.bytes = c.off + 256;
  return w;
}

__global__ void k_sd_flags(int64_t n, const uint8_t* __restrict__ seen, const uint8_t* __restrict__ pm,
                           const float* __restrict__ z, uint16_t* grp, uint32_t* zkey, SubState* st,
                           const FirstHist fh) {
  __shared__ uint32_t sh[FH_WORDS];
  fh_clear(fh, sh);
  const int64_t i0 = first_item();
  uint8_t pv[IPT] = {0, 0, 0, 0}, sv[IPT];
  float zv[IPT];
  if (pm) load4(pm, i0, n, pv, (uint8_t)0);
  load4(seen, i0, n, sv, (uint8_t)0);
  load4(z, i0, n, zv, 0.f);
  uint16_t gv[IPT];
  uint32_t zk[IPT];
  uint32_t c = 0, c0 = 0;
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    const bool alive = pv[u] == 0;
    gv[u] = (alive && sv[u]) ? 0 : GROUP_NONE;  // padding reads seen = 0
    zk[u] = order_key(zv[u]);
    c += (alive && i0 + u < n) ? 1u : 0u;
    c0 += gv[u] == 0 ? 1u : 0u;
    if (gv[u] == 0) fh_count(fh, sh, 0, zk[u]);  // the depth percentiles' selection
  }
  store4(grp, i0, n, gv);
  store4(zkey, i0, n, zk);
  // one atomic per block and count (a same-address atomic per warp serialises at the L2); n_el
  // counts the alive and seen voxels until the percentiles are applied
  const uint32_t b = block_total(c), b0 = block_total(c0);
  if (threadIdx.x == 0 && b) atomicAdd(&st->n_alive, b);
  if (threadIdx.x == 0 && b0) atomicAdd(&st->n_el, b0);
  fh_flush(fh, sh);
}

// both percentiles are queries of group 0: the flags kernel counted the first digit into row 0 of h0
// (when h0 is not null), and row 1 gets a copy
__global__ void k_sd_pct_queries(SelectQuery* q, uint32_t lo_ppm, uint32_t hi_ppm, const uint32_t* counter,
                                 void* sel_tmp, uint32_t* h0) {
  select_prepare(q, 2, sel_tmp);
  if (h0)
    for (int i = threadIdx.x; i < select_radix(2); i += blockDim.x) h0[select_radix(2) + i] = h0[i];
  if (threadIdx.x == 0) {
    uint32_t m = *counter;
    q[0].group = 0; q[0].k = rank_ppm(lo_ppm, m);
    q[1].group = 0; q[1].k = rank_ppm(hi_ppm, m);
  }
}

// also clears n_el (the alive and seen count until now) for the eligible count
__global__ void k_sd_pct_apply(const SelectQuery* pct, SubState* st, float* state, float r, float omr) {
  if (threadIdx.x == 0) {
    if (st->n_el > 0) running_pct(pct, state, r, omr, &st->p_lo);
    st->n_el = 0u;
  }
}

// Eq. 13 eligibility and Eq. 15-16 priority; pkey orders by descending priority
__global__ void k_sd_priority(int64_t n, const float4* __restrict__ geom, const uint8_t* __restrict__ level,
                              const float* __restrict__ delta, const float* __restrict__ z,
                              const float* __restrict__ u, float kappa, float beta, int l_max, uint16_t* grp,
                              uint32_t* pkey, SubState* st, const FirstHist fh) {
  __shared__ uint32_t sh[FH_WORDS];
  fh_clear(fh, sh);
  const int64_t i0 = first_item();
  const float p_lo = st->p_lo, p_hi = st->p_hi;
  uint16_t gv[IPT];
  uint8_t lv[IPT];
  float dv[IPT], zv[IPT], uv[IPT];
  load4((const uint16_t*)grp, i0, n, gv, GROUP_NONE);
  load4(level, i0, n, lv, (uint8_t)0);
  load4(delta, i0, n, dv, 0.f);
  load4(z, i0, n, zv, 0.f);
  load4(u, i0, n, uv, 0.f);
  uint32_t pk[IPT];
  uint32_t c = 0;
#pragma unroll
  for (int k = 0; k < IPT; ++k) {
    const int64_t i = i0 + k;
    bool el = false;
    pk[k] = 0xffffffffu;  // read only for eligible voxels
    if (gv[k] == 0 && (int)lv[k] < l_max) {  // padding reads GROUP_NONE
      const float thr = __fmul_rn(kappa, dv[k]);
      if (geom[i].w > thr) {
        el = true;
        const float zt = depth_norm(zv[k], p_lo, p_hi);
        const float b = __fadd_rn(1.0f, __fmul_rn(beta, zt));
        const float p = __fmul_rn(uv[k], b);
        pk[k] = ~order_key(p);
      }
    }
    gv[k] = el ? 0 : GROUP_NONE;
    c += el ? 1u : 0u;
    if (el) fh_count(fh, sh, 0, pk[k]);  // the top-k selection
  }
  store4(pkey, i0, n, pk);
  store4(grp, i0, n, gv);
  // one atomic per block (a same-address atomic per warp serialises at the L2)
  const uint32_t b = block_total(c);
  if (threadIdx.x == 0 && b) atomicAdd(&st->n_el, b);
  fh_flush(fh, sh);
}

__global__ void k_sd_k(SelectQuery* q, SubState* st, uint32_t top_ppm, long long budget, void* sel_tmp) {
  select_prepare(q + 2, 1, sel_tmp);
  if (threadIdx.x == 0) {
    const unsigned long long na = st->n_alive;
    unsigned long long k = (unsigned long long)top_ppm * na / 1000000ull;
    const unsigned long long kb = budget > (long long)na ? (unsigned long long)(budget - (long long)na) / 7ull : 0ull;
    if (kb < k) k = kb;
    if (st->n_el < k) k = st->n_el;
    st->k = (uint32_t)k;
    q[2].group = 0;
    q[2].k = (uint32_t)k;
  }
}

// eligible voxels above the k-th priority, and per block those tied with it
// (the ties compete by id: the need = k - c_gt smallest ids among them split)
__global__ void k_sd_ties(int64_t n, const uint32_t* __restrict__ pkey, const SelectQuery* thr,
                          const uint16_t* __restrict__ grp, uint32_t* blk, SubState* st) {
  const int64_t i0 = first_item();
  uint32_t cgt = 0, ceq = 0;
  if (thr->k != 0) {
    const uint32_t v = thr->result;
    uint16_t gv[IPT];
    uint32_t kv[IPT];
    load4(grp, i0, n, gv, GROUP_NONE);
    load4(pkey, i0, n, kv, 0u);
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      if (gv[u] != 0) continue;  // padding reads GROUP_NONE
      const uint32_t k = kv[u];
      cgt += k < v ? 1u : 0u;
      ceq += k == v ? 1u : 0u;
    }
  }
  // one atomic per block (a same-address atomic per warp serialises at the L2)
  const uint32_t bg = block_total(cgt);
  const uint32_t be = block_total(ceq);
  if (threadIdx.x == 0) {
    if (bg) atomicAdd(&st->c_gt, bg);
    blk[blockIdx.x] = be;
  }
}

// grp == 0 marks the eligible voxels (set by the priority kernel); a tie's
// rank among the ties is its block's offset plus its rank inside the block
__global__ void k_sd_select(int64_t n, const uint8_t* __restrict__ pm, const uint16_t* __restrict__ grp,
                            const uint32_t* __restrict__ pkey, const SelectQuery* q,
                            const uint32_t* __restrict__ blk, const SubState* st, uint8_t* selected,
                            uint32_t* surv, uint32_t* sel, uint32_t* blk_surv, uint32_t* blk_sel) {
  const int64_t i0 = first_item();
  const bool any_k = q[2].k != 0;
  const uint32_t v = q[2].result;
  bool gt[IPT], eq[IPT];
  uint8_t pv[IPT] = {0, 0, 0, 0};
  uint16_t gv[IPT];
  uint32_t kv[IPT];
  uint32_t ceq = 0;
  if (pm) load4(pm, i0, n, pv, (uint8_t)0);
  load4(grp, i0, n, gv, GROUP_NONE);
  load4(pkey, i0, n, kv, 0u);
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    gt[u] = eq[u] = false;
    if (any_k && gv[u] == 0) {  // padding reads GROUP_NONE
      gt[u] = kv[u] < v;
      eq[u] = kv[u] == v;
    }
    ceq += eq[u] ? 1u : 0u;
  }
  uint32_t r = block_excl_count(ceq) + block_offset(blk);  // every thread of the block takes part
  const uint32_t need = st->k > st->c_gt ? st->k - st->c_gt : 0u;
  uint8_t so[IPT];
  uint32_t sl[IPT], sv[IPT], cs = 0, cl = 0;
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    const bool s = gt[u] || (eq[u] && r < need);
    r += eq[u] ? 1u : 0u;
    so[u] = s ? 1 : 0;
    sl[u] = s ? 1u : 0u;
    sv[u] = (pv[u] == 0 && !s && i0 + u < n) ? 1u : 0u;
    cs += sv[u];
    cl += sl[u];
  }
  store4(selected, i0, n, so);
  store4(sel, i0, n, sl);
  store4(surv, i0, n, sv);
  // per-block survivor and parent counts: k_sd_list takes its offsets from them
  const uint32_t bs = block_total(cs), bl = block_total(cl);
  if (threadIdx.x == 0) {
    blk_surv[blockIdx.x] = bs;
    blk_sel[blockIdx.x] = bl;
  }
}

__global__ void k_sd_check(const unsigned long long* totals, SubState* st, int64_t capacity, int64_t* n_new,
                           int32_t* status) {
  if (threadIdx.x == 0) {
    const long long nn = (long long)totals[0] + 8ll * (long long)totals[1];
    st->fits = nn <= capacity ? 1u : 0u;
    if (!st->fits) report(status, LV_ERR_CAPACITY);
    if (n_new) *n_new = nn;
  }
}

struct AuxSet {
  int n;
  lv_aux_array a[LV_MAX_AUX];
};

__device__ __forceinline__ void aux_fill(const lv_aux_array& a, int64_t dst) {
  const size_t row = (size_t)a.width * a.elem_bytes;
  char* d = (char*)a.out + row * (size_t)dst;
  if (a.elem_bytes == 4 && (row & 15) == 0 && ((uintptr_t)d & 15) == 0) {
    const uint4 f = make_uint4(a.fill, a.fill, a.fill, a.fill);
    for (size_t k = 0; k < row / 16; ++k) ((uint4*)d)[k] = f;
    return;
  }
  for (int e = 0; e < a.width; ++e) {
    if (a.elem_bytes == 4) ((uint32_t*)d)[e] = a.fill;
    else if (a.elem_bytes == 2) ((uint16_t*)d)[e] = (uint16_t)a.fill;
    else ((uint8_t*)d)[e] = (uint8_t)a.fill;
  }
}

// Copy the surviving rows of 32 consecutive voxels (one warp) of an array
// whose rows are `row` bytes: the survivors of the group land on consecutive
// output rows starting at `base`, so lanes stride over the group's bytes in
// 16-, 4- or 1-byte words and both reads and writes coalesce.
__device__ __forceinline__ void warp_copy_rows(const char* __restrict__ in, char* __restrict__ out, size_t row,
                                               int64_t i0, int nrows, uint32_t keep, int64_t base, int lane) {
  if (row % 16 == 0 && ((((uintptr_t)in) | ((uintptr_t)out)) & 15) == 0) {
    const int wpr = (int)(row / 16);
    const uint4* s = (const uint4*)in + (size_t)i0 * wpr;
    uint4* d = (uint4*)out;
    for (int w = lane; w < nrows * wpr; w += 32) {
      const int r = w / wpr, cw = w - r * wpr;
      if ((keep >> r) & 1u) d[(size_t)(base + __popc(keep & ((1u << r) - 1u))) * wpr + cw] = s[w];
    }
  } else if (row % 4 == 0 && ((((uintptr_t)in) | ((uintptr_t)out)) & 3) == 0) {
    const int wpr = (int)(row / 4);
    const uint32_t* s = (const uint32_t*)in + (size_t)i0 * wpr;
    uint32_t* d = (uint32_t*)out;
    for (int w = lane; w < nrows * wpr; w += 32) {
      const int r = w / wpr, cw = w - r * wpr;
      if ((keep >> r) & 1u) d[(size_t)(base + __popc(keep & ((1u << r) - 1u))) * wpr + cw] = s[w];
    }
  } else {
    const int wpr = (int)row;
    const char* s = in + (size_t)i0 * wpr;
    for (int w = lane; w < nrows * wpr; w += 32) {
      const int r = w / wpr, cw = w - r * wpr;
      if ((keep >> r) & 1u) out[(size_t)(base + __popc(keep & ((1u << r) - 1u))) * wpr + cw] = s[w];
    }
  }
}

template <typename DT, typename ST>
__device__ __forceinline__ void write_survivors(int64_t i0, int64_t n, const uint32_t* __restrict__ surv,
                                                const unsigned long long* __restrict__ pos,
                                                const float4* __restrict__ geom, const uint8_t* __restrict__ level,
                                                const DT* __restrict__ dens, const ST* __restrict__ sh, float4* ogeom,
                                                uint8_t* olevel, DT* odens, ST* osh, const AuxSet& aux) {
  const int lane = threadIdx.x & 31;
  const int64_t i = i0 + lane;
  const uint32_t keep = __ballot_sync(FULL, i < n && surv[i] != 0);
  if (!keep) return;
  const int nrows = (int)min((int64_t)32, n - i0);
  const int64_t base = (int64_t)pos[i0];
  warp_copy_rows((const char*)geom, (char*)ogeom, 16, i0, nrows, keep, base, lane);
  warp_copy_rows((const char*)level, (char*)olevel, 1, i0, nrows, keep, base, lane);
  warp_copy_rows((const char*)dens, (char*)odens, 8 * sizeof(DT), i0, nrows, keep, base, lane);
  warp_copy_rows((const char*)sh, (char*)osh, 48 * sizeof(ST), i0, nrows, keep, base, lane);
  for (int a = 0; a < aux.n; ++a)
    warp_copy_rows((const char*)aux.a[a].in, (char*)aux.a[a].out, (size_t)aux.a[a].width * aux.a[a].elem_bytes, i0,
                   nrows, keep, base, lane);
}

template <typename DT>
__device__ __forceinline__ DT from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }

// a (1 - t) + b t with every product and the sum rounded
__device__ __forceinline__ float lerp_rn(float a, float b, float t) {
  return __fadd_rn(__fmul_rn(a, __fsub_rn(1.0f, t)), __fmul_rn(b, t));
}

__global__ void k_cp_flags(int64_t n, const uint8_t* __restrict__ keep, uint32_t* __restrict__ surv) {
  const int64_t i = blockIdx.x * (int64_t)TPB + threadIdx.x;
  if (i < n) surv[i] = keep[i] ? 1u : 0u;
}

// The split parents in id order (list), the pruned rows -- neither survivor
// nor parent -- in id order (holes, for the in-place topology change) and
// every voxel's survivor position (for the out-of-place one).  Blocks cover
// the voxels as in k_sd_select and take their offsets from its per-block
// counts; the number of pruned rows before i is i - (survivors before i) -
// (parents before i).  The last block also totals the survivors and the
// parents and checks the grown count against the output capacity.  It runs
// with the selection (on the caller's side stream in a training step) so that
// the in-place write does not read these arrays again.
__global__ void k_sd_list(int64_t n, const uint32_t* __restrict__ sel, const uint32_t* __restrict__ surv,
                          const uint32_t* __restrict__ blk_surv, const uint32_t* __restrict__ blk_sel,
                          unsigned long long* __restrict__ surv_pos, uint32_t* __restrict__ list,
                          uint32_t* __restrict__ holes, unsigned long long* totals, SubState* st, int64_t capacity,
                          int64_t* n_new, int32_t* status) {
  const int64_t i0 = first_item();
  uint32_t sl[IPT], sv[IPT], cs = 0, cl = 0;
  load4(sel, i0, n, sl, 0u);
  load4(surv, i0, n, sv, 0u);
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    cs += sv[u];
    cl += sl[u];
  }
  const uint32_t os = block_offset(blk_surv), ol = block_offset(blk_sel);
  uint32_t rs = os + block_excl_count(cs), rl = ol + block_excl_count(cl);
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    const int64_t i = i0 + u;
    if (i >= n) break;
    surv_pos[i] = rs;
    if (sl[u]) list[rl] = (uint32_t)i;
    else if (!sv[u]) holes[i - (int64_t)rs - (int64_t)rl] = (uint32_t)i;
    rs += sv[u];
    rl += sl[u];
  }
  if (blockIdx.x == gridDim.x - 1) {  // block-uniform
    const uint32_t ts = block_total(cs), tl = block_total(cl);
    if (threadIdx.x == 0) {
      totals[0] = (unsigned long long)os + ts;
      totals[1] = (unsigned long long)ol + tl;
      const long long nn = (long long)(os + ts) + 8ll * (long long)(ol + tl);
      st->fits = nn <= capacity ? 1u : 0u;
      if (!st->fits) report(status, LV_ERR_CAPACITY);
      if (n_new) *n_new = nn;
    }
  }
}

// A warp writes 32 consecutive children (output rows o0 .. o0 + 31): one lane
// per child for the geometry, level and interpolated corners; the SH rows and
// the auxiliary rows are written cooperatively in 16-byte words so that the
// stores coalesce (the 8 children of a parent read the same parent row).
template <typename DT, typename ST>
__device__ __forceinline__ void write_children(int64_t t0, const uint32_t* __restrict__ list,
                                               const unsigned long long* totals, const float4* __restrict__ geom,
                                               const uint8_t* __restrict__ level, const DT* __restrict__ dens,
                                               const ST* __restrict__ sh, float4* ogeom, uint8_t* olevel, DT* odens,
                                               ST* osh, const AuxSet& aux) {
  const int lane = threadIdx.x & 31;
  const int64_t nchild = 8 * (int64_t)totals[1];
  if (t0 >= nchild) return;
  const int nrows = (int)min((int64_t)32, nchild - t0);
  const int64_t o0 = (int64_t)totals[0] + t0;
  if (lane < nrows) {
    const int64_t t = t0 + lane;
    const int64_t i = list[t >> 3];
    const int c = (int)(t & 7);
    const int64_t o = o0 + lane;
    const float4 g = geom[i];
    const float hc = __fmul_rn(g.w, 0.5f);
    ogeom[o] = make_float4(__fadd_rn(g.x, (c & 1) ? hc : -hc), __fadd_rn(g.y, (c & 2) ? hc : -hc),
                           __fadd_rn(g.z, (c & 4) ? hc : -hc), hc);
    olevel[o] = (uint8_t)(level[i] + 1);
    float d[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) d[q] = to_f32(dens[8 * i + q]);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float qx = (float)(((c >> 0) & 1) + ((j >> 0) & 1)) * 0.5f;
      const float qy = (float)(((c >> 1) & 1) + ((j >> 1) & 1)) * 0.5f;
      const float qz = (float)(((c >> 2) & 1) + ((j >> 2) & 1)) * 0.5f;
      const float x0 = lerp_rn(d[0], d[1], qx), x1 = lerp_rn(d[2], d[3], qx);
      const float x2 = lerp_rn(d[4], d[5], qx), x3 = lerp_rn(d[6], d[7], qx);
      const float y0 = lerp_rn(x0, x1, qy), y1 = lerp_rn(x2, x3, qy);
      odens[8 * o + j] = from_f32<DT>(lerp_rn(y0, y1, qz));
    }
  }
  // SH rows: copied from the parent
  constexpr int WPR = (int)(48 * sizeof(ST) / 16);
  const uint4* ssrc = (const uint4*)sh;
  uint4* sdst = (uint4*)osh + (size_t)o0 * WPR;
  for (int w = lane; w < nrows * WPR; w += 32) {
    const int r = w / WPR, k = w - r * WPR;
    sdst[w] = __ldg(ssrc + (size_t)list[(t0 + r) >> 3] * WPR + k);
  }
  // auxiliary rows: the child fill pattern
  for (int a = 0; a < aux.n; ++a) {
    const lv_aux_array& A = aux.a[a];
    const size_t row = (size_t)A.width * A.elem_bytes;
    char* base = (char*)A.out + row * (size_t)o0;
    if (A.elem_bytes == 4 && (row & 15) == 0 && ((uintptr_t)base & 15) == 0) {
      const uint4 f = make_uint4(A.fill, A.fill, A.fill, A.fill);
      const int words = (int)(row / 16) * nrows;
      for (int w = lane; w < words; w += 32) ((uint4*)base)[w] = f;
    } else {
      for (int r = lane; r < nrows; r += 32) aux_fill(A, o0 + r);
    }
  }
}

// All the writes of a topology change in one launch: warps [0, sw) copy the
// survivors of 32 consecutive voxels each, warps [sw, ...) write 32 children each.
template <typename DT, typename ST>
__global__ void k_sd_write(int64_t n, int64_t max_children, const uint32_t* __restrict__ surv,
                           const unsigned long long* __restrict__ pos, const uint32_t* __restrict__ list,
                           const unsigned long long* totals, const SubState* st, const float4* __restrict__ geom,
                           const uint8_t* __restrict__ level, const DT* __restrict__ dens, const ST* __restrict__ sh,
                           float4* ogeom, uint8_t* olevel, DT* odens, ST* osh, const __grid_constant__ AuxSet aux) {
  if (!st->fits) return;
  const int64_t gw = (blockIdx.x * (int64_t)TPB + threadIdx.x) >> 5;  // global warp
  const int64_t sw = (n + 31) / 32;
  if (gw < sw) {
    write_survivors<DT, ST>(gw * 32, n, surv, pos, geom, level, dens, sh, ogeom, olevel, odens, osh, aux);
  } else {
    const int64_t t0 = (gw - sw) * 32;
    if (t0 < max_children)
      write_children<DT, ST>(t0, list, totals, geom, level, dens, sh, ogeom, olevel, odens, osh, aux);
  }
}

// ------------------------------------------------------------------ in-place topology change
// The rows a subdivision changes, rewritten where they are (Sec. IV-D): a
// split parent's row becomes its child 0; children 1..7 of the r-th parent (id
// order) take slots 7r .. 7r + 6 of [the pruned rows in index order, then rows
// n, n + 1, ...]; with fewer children than pruned rows, the occupied rows at
// index >= n' then move into the empty rows below n', both in index order.
// Rows the step does not change are neither read nor written.

// a voxel's 8 corners: 16-byte stores where the row is 16-byte aligned (it is in
// a 16-byte aligned array), element stores otherwise
template <typename DT>
__device__ __forceinline__ void store_corners(DT* row, const float* v);
template <>
__device__ __forceinline__ void store_corners<float>(float* row, const float* v) {
  if (((uintptr_t)row & 15) == 0) {
    ((float4*)row)[0] = make_float4(v[0], v[1], v[2], v[3]);
    ((float4*)row)[1] = make_float4(v[4], v[5], v[6], v[7]);
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) row[j] = v[j];
  }
}
template <>
__device__ __forceinline__ void store_corners<__half>(__half* row, const float* v) {
  __half2 h[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) h[q] = __halves2half2(__float2half_rn(v[2 * q]), __float2half_rn(v[2 * q + 1]));
  if (((uintptr_t)row & 15) == 0) {
    uint4 u;
    u.x = *(const uint32_t*)&h[0]; u.y = *(const uint32_t*)&h[1];
    u.z = *(const uint32_t*)&h[2]; u.w = *(const uint32_t*)&h[3];
    *(uint4*)row = u;
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) row[j] = __float2half_rn(v[j]);
  }
}

// row of child c of the parent of rank r (at row `parent`)
__device__ __forceinline__ int64_t ip_child_row(int64_t r, int c, int64_t parent, const uint32_t* __restrict__ holes,
                                                int64_t h, int64_t n) {
  if (c == 0) return parent;
  const int64_t s = 7 * r + (c - 1);
  return s < h ? (int64_t)holes[s] : n + (s - h);
}

// A warp writes the 8 children of 4 consecutive parents (children t0 .. t0 + 31,
// one lane each for the geometry, level and interpolated corners).  Every lane
// reads its parent's geometry, level and corners, and the warp stages its
// parents' SH rows in shared memory, before any child is written: child 0
// overwrites the parent's own row.  The SH and auxiliary rows then go out in
// 16-byte words spread over the lanes.
template <typename DT, typename ST>
__global__ void __launch_bounds__(TPB) k_ip_children(int64_t n, const uint32_t* __restrict__ list,
                                                     const uint32_t* __restrict__ holes,
                                                     const unsigned long long* totals, const SubState* st,
                                                     float4* geom, uint8_t* level, DT* dens, ST* sh,
                                                     const __grid_constant__ AuxSet aux) {
  constexpr int WPR = (int)(48 * sizeof(ST) / 16);  // 16-byte words per SH row
  __shared__ uint4 s_sh[TPB / 32][4 * WPR];
  __shared__ int64_t s_dst[TPB / 32][32];
  if (!st->fits) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t0 = ((blockIdx.x * (int64_t)TPB + threadIdx.x) >> 5) * 32;
  const int64_t k = (int64_t)totals[1];
  const int64_t nchild = 8 * k;
  if (t0 >= nchild) return;  // warp-uniform
  const int64_t h = n - (int64_t)totals[0] - k;
  const int nrows = (int)min((int64_t)32, nchild - t0);
  const bool act = lane < nrows;
  const int64_t t = t0 + lane;
  const int64_t r = t >> 3;
  const int c = (int)(t & 7);
  float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
  uint8_t lvl = 0;
  float d[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) d[q] = 0.f;
  int64_t dst = 0;
  if (act) {
    const int64_t parent = list[r];
    dst = ip_child_row(r, c, parent, holes, h, n);
    g = geom[parent];
    lvl = level[parent];
#pragma unroll
    for (int q = 0; q < 8; ++q) d[q] = to_f32(dens[8 * parent + q]);
  }
  s_dst[warp][lane] = dst;
  const int np = (nrows + 7) >> 3;
  const uint4* ssrc = (const uint4*)sh;
  for (int w = lane; w < np * WPR; w += 32) {
    const int pr = w / WPR, kk = w - pr * WPR;
    s_sh[warp][w] = ssrc[(size_t)list[(t0 >> 3) + pr] * WPR + kk];
  }
  __syncwarp();
  if (act) {
    const float hc = __fmul_rn(g.w, 0.5f);
    geom[dst] = make_float4(__fadd_rn(g.x, (c & 1) ? hc : -hc), __fadd_rn(g.y, (c & 2) ? hc : -hc),
                            __fadd_rn(g.z, (c & 4) ? hc : -hc), hc);
    level[dst] = (uint8_t)(lvl + 1);
    float cd[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float qx = (float)(((c >> 0) & 1) + ((j >> 0) & 1)) * 0.5f;
      const float qy = (float)(((c >> 1) & 1) + ((j >> 1) & 1)) * 0.5f;
      const float qz = (float)(((c >> 2) & 1) + ((j >> 2) & 1)) * 0.5f;
      const float x0 = lerp_rn(d[0], d[1], qx), x1 = lerp_rn(d[2], d[3], qx);
      const float x2 = lerp_rn(d[4], d[5], qx), x3 = lerp_rn(d[6], d[7], qx);
      const float y0 = lerp_rn(x0, x1, qy), y1 = lerp_rn(x2, x3, qy);
      cd[j] = lerp_rn(y0, y1, qz);
    }
    store_corners<DT>(dens + 8 * dst, cd);
  }
  uint4* sdst = (uint4*)sh;
  for (int w = lane; w < nrows * WPR; w += 32) {
    const int rr = w / WPR, kk = w - rr * WPR;
    sdst[(size_t)s_dst[warp][rr] * WPR + kk] = s_sh[warp][(rr >> 3) * WPR + kk];
  }
  // auxiliary rows: the child fill pattern
  for (int a = 0; a < aux.n; ++a) {
    const lv_aux_array& A = aux.a[a];
    const size_t row = (size_t)A.width * A.elem_bytes;
    if (A.elem_bytes == 4 && (row & 15) == 0 && ((uintptr_t)A.out & 15) == 0) {
      const uint4 f = make_uint4(A.fill, A.fill, A.fill, A.fill);
      const int wpr = (int)(row / 16);
      for (int w = lane; w < nrows * wpr; w += 32) {
        const int rr = w / wpr, kk = w - rr * wpr;
        ((uint4*)A.out)[(size_t)s_dst[warp][rr] * wpr + kk] = f;
      }
    } else if (act) {
      aux_fill(A, dst);
    }
  }
}

// first index in [lo, hi) of the sorted holes[] whose value is >= v
__device__ __forceinline__ int64_t ip_lower_bound(const uint32_t* __restrict__ holes, int64_t lo, int64_t hi,
                                                  int64_t v) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)holes[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// one array row moved by a warp, in 4-byte words where aligned
__device__ __forceinline__ void ip_move_row(char* base, size_t row, int64_t src, int64_t dst, int lane) {
  char* s = base + row * (size_t)src;
  char* d = base + row * (size_t)dst;
  if ((row & 3) == 0 && ((uintptr_t)base & 3) == 0) {
    for (size_t w = lane; w < row / 4; w += 32) ((uint32_t*)d)[w] = ((const uint32_t*)s)[w];
  } else {
    for (size_t w = lane; w < row; w += 32) d[w] = s[w];
  }
}

// Shrinking step (7k < h): the occupied rows at index >= n' move into the empty
// rows below n'.  The empty rows are the unfilled holes holes[7k .. h); the
// first m of them lie below n'.  An occupied row i in [n', n) has rank
// (i - n') - (unfilled holes in [n', i)) and moves to holes[7k + rank].  One
// warp per row, grid-stride over [n', n); it runs after the children are
// written, since a moved row may be one of them.
template <typename DT, typename ST>
__global__ void __launch_bounds__(TPB) k_ip_tail(int64_t n, const uint32_t* __restrict__ holes,
                                                 const unsigned long long* totals, const SubState* st, float4* geom,
                                                 uint8_t* level, DT* dens, ST* sh, const __grid_constant__ AuxSet aux) {
  if (!st->fits) return;
  const int64_t k = (int64_t)totals[1];
  const int64_t h = n - (int64_t)totals[0] - k;
  if (7 * k >= h) return;
  const int64_t nn = n - h + 7 * k;
  const int64_t f0 = 7 * k;
  const int64_t fm = ip_lower_bound(holes, f0, h, nn);  // f0 + m
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)TPB + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * TPB) >> 5;
  for (int64_t i = nn + gw; i < n; i += nw) {
    const int64_t pos = ip_lower_bound(holes, fm, h, i);
    if (pos < h && (int64_t)holes[pos] == i) continue;  // an empty row: nothing moves
    const int64_t dst = holes[f0 + (i - nn) - (pos - fm)];
    ip_move_row((char*)geom, 16, i, dst, lane);
    ip_move_row((char*)level, 1, i, dst, lane);
    ip_move_row((char*)dens, 8 * sizeof(DT), i, dst, lane);
    ip_move_row((char*)sh, 48 * sizeof(ST), i, dst, lane);
    for (int a = 0; a < aux.n; ++a)
      ip_move_row((char*)aux.a[a].out, (size_t)aux.a[a].width * aux.a[a].elem_bytes, i, dst, lane);
  }
}

}  // namespace

}  // namespace lv

using namespace lv;

extern "C" int32_t lv_prune_anneal_ppm(double t, double t0, double t1) {
  if (!(t1 > t0)) return 1000000;
  double x = (t - t0) / (t1 - t0);
  x = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
  return (int32_t)floor(1e6 * x);
}

extern "C" size_t lv_prune_workspace_size(int64_t n, const lv_prune_params* p) {
  if (n < 0 || !p) return 0;
  return carve_prune(nullptr, n).bytes;
}

static lv_status check_prune(int64_t n, const lv_prune_params* p, void* workspace, size_t ws_bytes) {
  if (!p || n < 0 || n > 0x7fffffffLL) { set_error("bad arguments"); return LV_ERR_INVALID_ARG; }
  if (p->n_bins < 1 || p->n_bins > SELECT_MAX_QUERIES) { set_error("n_bins must be 1..%d", SELECT_MAX_QUERIES); return LV_ERR_INVALID_ARG; }
  if (p->q_ppm < 0 || p->q_ppm > 1000000 || p->cap_ppm < 0 || p->cap_ppm > 1000000 || p->lo_ppm < 0 ||
      p->lo_ppm > 1000000 || p->hi_ppm < 0 || p->hi_ppm > 1000000) { set_error("ppm parameters must be in [0, 1e6]"); return LV_ERR_INVALID_ARG; }
  if (!(p->ema_alpha >= 0.f && p->ema_alpha <= 1.f)) { set_error("ema_alpha must be in [0, 1]"); return LV_ERR_INVALID_ARG; }
  if (p->anneal && (p->anneal_ppm < 0 || p->anneal_ppm > 1000000 || p->relax_ppm < 0 || p->relax_ppm > 1000000)) {
    set_error("anneal_ppm and relax_ppm must be in [0, 1e6]"); return LV_ERR_INVALID_ARG;
  }
  if (!(p->pct_ema >= 0.f && p->pct_ema <= 1.f)) { set_error("pct_ema must be in [0, 1]"); return LV_ERR_INVALID_ARG; }
  if (!(p->halo_small >= 0.f) || isnan(p->halo_w) || isnan(p->halo_edge)) { set_error("bad keep-halo parameters"); return LV_ERR_INVALID_ARG; }
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  if (ws_bytes < carve_prune(nullptr, n).bytes) {
    set_error("workspace %zu < %zu bytes", ws_bytes, carve_prune(nullptr, n).bytes);
    return LV_ERR_WORKSPACE;
  }
  return LV_OK;
}

extern "C" lv_status lv_prune_bins(int64_t n, const uint8_t* seen, const float* z, const lv_prune_params* p,
                                   void* workspace, size_t ws_bytes, void* stream) {
  lv_status e = check_prune(n, p, workspace, ws_bytes);
  if (e != LV_OK) return e;
  if (n > 0 && (!seen || !z)) { set_error("null array"); return LV_ERR_INVALID_ARG; }
  if (n == 0) return LV_OK;
  PruneWs w = carve_prune(workspace, n);
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = eblocks(n);  // IPT voxels per thread
  zero_async(s, w.st, sizeof(PruneState));
  k_pr_seen<<<blocks, TPB, 0, s>>>(n, seen, z, w.grp, w.zkey, w.st);
  k_pr_pct_queries<<<1, 256, 0, s>>>(w.q, w.st, (uint32_t)p->lo_ppm, (uint32_t)p->hi_ppm, w.sel_tmp);
  select_kth_prepared(w.zkey, w.grp, n, w.q, 2, w.sel_tmp, s);
  const float r = p->pct_ema, omr = 1.0f - r;  // rounded to FP32 once, as the oracle does
  k_pr_pct_apply<<<1, 32, 0, s>>>(w.q, w.st, p->pct_state, r, omr);
  k_pr_bin<<<blocks, TPB, 0, s>>>(n, seen, z, p->n_bins, w.grp, w.st);
  count_launch(4);
  return cuda_check(cudaGetLastError(), "lv_prune_bins");
}

extern "C" lv_status lv_prune_finish(int64_t n, const float* w_max, const uint8_t* seen, const float* z,
                                     float* ema_m, uint8_t* state, const lv_prune_params* p, uint8_t* prune_mask,
                                     int64_t* d_n_pruned, void* workspace, size_t ws_bytes, int32_t* d_status,
                                     void* stream) {
  (void)d_status;
  (void)seen;
  (void)z;
  lv_status e = check_prune(n, p, workspace, ws_bytes);
  if (e != LV_OK) return e;
  if (n > 0 && (!w_max || !ema_m || !state || !prune_mask)) { set_error("null array"); return LV_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    if (d_n_pruned) cudaMemsetAsync(d_n_pruned, 0, sizeof(int64_t), s);
    return cuda_check(cudaGetLastError(), "lv_prune_finish");
  }
  PruneWs w = carve_prune(workspace, n);
  const int nb = p->n_bins;
  const uint32_t cap = (uint32_t)(((unsigned long long)p->cap_ppm * (unsigned long long)n) / 1000000ull);
  const float alpha = p->ema_alpha;
  const float oma = 1.0f - alpha;  // rounded to FP32 once, as the oracle does
  const int blocks = eblocks(n);  // IPT voxels per thread
  // the two selections' first digits are counted by the kernels that write their keys
  const FirstHist fh_tau = first_hist(w.h0_tau, nb, nb), fh_cap = first_hist(w.h0_cap, 1, 1);
  zero_async(s, w.h0_tau, sizeof(uint32_t) * 2 * FH_WORDS, w.h0_cap, sizeof(uint32_t) * select_radix(1));
  k_pr_wkey<<<blocks, TPB, 0, s>>>(n, w_max, w.grp, w.wkey, fh_tau);
  // the percentiles in q[0..1] are consumed: q is reused per bin
  k_pr_tau_queries<<<1, 256, 0, s>>>(w.q, w.st, nb, (uint32_t)p->q_ppm, p->anneal, (uint32_t)p->anneal_ppm,
                                     (uint32_t)p->relax_ppm, w.sel_tmp);
  if (fh_tau.h0) select_kth_first(w.wkey, w.grp, n, w.q, nb, w.h0_tau, w.sel_tmp, s);
  else select_kth_prepared(w.wkey, w.grp, n, w.q, nb, w.sel_tmp, s);
  // candidates get their own group array (zkey is free now: reuse it as u16 storage)
  uint16_t* cand = (uint16_t*)w.zkey;
  Halo halo;
  halo.small = p->halo_small;
  halo.w = p->halo_w;
  halo.edge = p->halo_edge;
  halo.geom = (const float4*)p->geom;
  halo.delta = p->delta;
  halo.edge_score = p->edge;
  halo.w_max = w_max;
  k_pr_update<<<blocks, TPB, 0, s>>>(n, w.grp, w.wkey, w.q, alpha, oma, p->m_low, p->m_high, ema_m, state, halo,
                                      prune_mask, cand, w.st, fh_cap);
  SelectQuery* qc = w.q + SELECT_MAX_QUERIES - 2;  // cap threshold
  k_pr_cap_query<<<1, 256, 0, s>>>(qc, w.st, cap, w.sel_tmp);
  select_kth_first(w.wkey, cand, n, qc, 1, w.h0_cap, w.sel_tmp, s);
  k_pr_ties<<<blocks, TPB, 0, s>>>(n, w.wkey, qc, prune_mask, w.blk, w.st);
  k_pr_mask<<<blocks, TPB, 0, s>>>(n, w.wkey, qc, w.blk, w.st, prune_mask, d_n_pruned, cap);
  count_launch(7);
  return cuda_check(cudaGetLastError(), "lv_prune_finish");
}

extern "C" lv_status lv_prune_depth_quantile(int64_t n, const float* w_max, const uint8_t* seen, const float* z,
                                             float* ema_m, uint8_t* state, const lv_prune_params* p,
                                             uint8_t* prune_mask, int64_t* d_n_pruned, void* workspace,
                                             size_t ws_bytes, int32_t* d_status, void* stream) {
  if (n > 0 && (!w_max || !seen || !z || !ema_m || !state || !prune_mask)) { set_error("null array"); return LV_ERR_INVALID_ARG; }
  lv_status e = lv_prune_bins(n, seen, z, p, workspace, ws_bytes, stream);
  if (e != LV_OK) return e;
  return lv_prune_finish(n, w_max, seen, z, ema_m, state, p, prune_mask, d_n_pruned, workspace, ws_bytes, d_status,
                         stream);
}

extern "C" size_t lv_subdivide_workspace_size(int64_t n, const lv_subdiv_params* p) {
  if (n < 0 || !p) return 0;
  return carve_sub(nullptr, n).bytes;
}

static lv_status check_arrays(const lv_voxels* in, int n_aux, const lv_aux_array* aux, const lv_voxels* out);

static lv_status check_sub(const lv_voxels* in, const lv_subdiv_params* p, int n_aux, const lv_aux_array* aux,
                           const lv_voxels* out) {
  if (!in || !p) { set_error("null argument"); return LV_ERR_INVALID_ARG; }
  if (p->top_ppm < 0 || p->top_ppm > 1000000 || p->lo_ppm < 0 || p->lo_ppm > 1000000 || p->hi_ppm < 0 ||
      p->hi_ppm > 1000000) { set_error("ppm parameters must be in [0, 1e6]"); return LV_ERR_INVALID_ARG; }
  if (!(p->pct_ema >= 0.f && p->pct_ema <= 1.f)) { set_error("pct_ema must be in [0, 1]"); return LV_ERR_INVALID_ARG; }
  return check_arrays(in, n_aux, aux, out);
}

// the voxel, output and auxiliary arrays of a topology change
static lv_status check_arrays(const lv_voxels* in, int n_aux, const lv_aux_array* aux, const lv_voxels* out) {
  if (!in) { set_error("null argument"); return LV_ERR_INVALID_ARG; }
  const int64_t n = in->n;
  if (n < 0 || n > 0x7fffffffLL) { set_error("bad voxel count"); return LV_ERR_INVALID_ARG; }
  if (n > 0 && (!in->geom || !in->level || !in->density || !in->sh)) { set_error("null voxel array"); return LV_ERR_INVALID_ARG; }
  if (in->vidx) { set_error("subdivision needs per-voxel corner densities (vidx must be NULL)"); return LV_ERR_UNSUPPORTED; }
  if (in->density_dtype != LV_F32 && in->density_dtype != LV_F16) { set_error("density dtype must be F32 or F16"); return LV_ERR_INVALID_ARG; }
  if (in->sh_dtype != LV_F32 && in->sh_dtype != LV_BF16) { set_error("sh dtype must be F32 or BF16"); return LV_ERR_INVALID_ARG; }
  if (out) {
    if (out->n < 0) { set_error("bad output capacity"); return LV_ERR_INVALID_ARG; }
    if (out->n > 0 && (!out->geom || !out->level || !out->density || !out->sh)) { set_error("null output array"); return LV_ERR_INVALID_ARG; }
    if (in->density_dtype != out->density_dtype || in->sh_dtype != out->sh_dtype) { set_error("output dtypes must match the input"); return LV_ERR_INVALID_ARG; }
  }
  if (n_aux < 0 || n_aux > LV_MAX_AUX || (n_aux > 0 && !aux)) { set_error("n_aux must be 0..%d", LV_MAX_AUX); return LV_ERR_INVALID_ARG; }
  for (int a = 0; a < n_aux; ++a) {
    const int eb = aux[a].elem_bytes;
    if ((eb != 1 && eb != 2 && eb != 4) || aux[a].width < 1 || (n > 0 && (!aux[a].in || !aux[a].out))) {
      set_error("aux array %d: bad description", a); return LV_ERR_INVALID_ARG;
    }
  }
  return LV_OK;
}

extern "C" lv_status lv_subdivide_select(const lv_voxels* in, const float* delta, const float* z, const float* u,
                                         const uint8_t* seen, const uint8_t* prune_mask, const lv_subdiv_params* p,
                                         int64_t out_capacity, uint8_t* selected, int64_t* d_n_new, void* workspace,
                                         size_t ws_bytes, int32_t* d_status, void* stream) {
  lv_status e = check_sub(in, p, 0, nullptr, nullptr);
  if (e != LV_OK) return e;
  const int64_t n = in->n;
  if (n > 0 && (!delta || !z || !u || !seen || !selected)) { set_error("null array"); return LV_ERR_INVALID_ARG; }
  if (out_capacity < 0) { set_error("bad output capacity"); return LV_ERR_INVALID_ARG; }
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  SubWs w = carve_sub(workspace, n);
  if (ws_bytes < w.bytes) { set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return LV_ERR_WORKSPACE; }
  cudaStream_t s = (cudaStream_t)stream;
  // the state, and the first-digit counts of the two selections (counted by the kernels that
  // write their keys)
  zero_async(s, w.st, sizeof(SubState), w.h0_pct, sizeof(uint32_t) * 2 * select_radix(2), w.h0_top,
             sizeof(uint32_t) * select_radix(1));
  if (n == 0) {
    cudaMemsetAsync(w.totals, 0, 4 * sizeof(unsigned long long), s);
    if (d_n_new) cudaMemsetAsync(d_n_new, 0, sizeof(int64_t), s);
    return cuda_check(cudaGetLastError(), "lv_subdivide_select");
  }
  const int blocks = eblocks(n);  // IPT voxels per thread
  k_sd_flags<<<blocks, TPB, 0, s>>>(n, seen, prune_mask, z, w.grp, w.zkey, w.st, first_hist(w.h0_pct, 2, 1));
  k_sd_pct_queries<<<1, 256, 0, s>>>(w.q, (uint32_t)p->lo_ppm, (uint32_t)p->hi_ppm, &w.st->n_el, w.sel_tmp,
                                     w.h0_pct);
  select_kth_first(w.zkey, w.grp, n, w.q, 2, w.h0_pct, w.sel_tmp, s);
  k_sd_pct_apply<<<1, 32, 0, s>>>(w.q, w.st, p->pct_state, p->pct_ema, 1.0f - p->pct_ema);
  k_sd_priority<<<blocks, TPB, 0, s>>>(n, (const float4*)in->geom, in->level, delta, z, u, p->kappa, p->beta,
                                        p->l_max, w.grp, w.pkey, w.st, first_hist(w.h0_top, 1, 1));
  k_sd_k<<<1, 256, 0, s>>>(w.q, w.st, (uint32_t)p->top_ppm, (long long)p->budget, w.sel_tmp);
  select_kth_first(w.pkey, w.grp, n, w.q + 2, 1, w.h0_top, w.sel_tmp, s);
  k_sd_ties<<<blocks, TPB, 0, s>>>(n, w.pkey, w.q + 2, w.grp, w.blk, w.st);
  k_sd_select<<<blocks, TPB, 0, s>>>(n, prune_mask, w.grp, w.pkey, w.q, w.blk, w.st, selected, w.surv, w.sel,
                                      w.blk_surv, w.blk_sel);
  k_sd_list<<<blocks, TPB, 0, s>>>(n, w.sel, w.surv, w.blk_surv, w.blk_sel, w.surv_pos, w.sel_list, w.zkey,
                                   w.totals, w.st, out_capacity, d_n_new, d_status);
  count_launch(9);
  return cuda_check(cudaGetLastError(), "lv_subdivide_select");
}

extern "C" lv_status lv_subdivide_apply(const lv_voxels* in, const lv_subdiv_params* p, const lv_aux_array* aux,
                                        int n_aux, const lv_voxels* out, void* workspace, size_t ws_bytes,
                                        void* stream) {
  lv_status e = check_sub(in, p, n_aux, aux, out);
  if (e != LV_OK) return e;
  if (!out) { set_error("null output"); return LV_ERR_INVALID_ARG; }
  const int64_t n = in->n;
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  SubWs w = carve_sub(workspace, n);
  if (ws_bytes < w.bytes) { set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return LV_ERR_WORKSPACE; }
  if (n == 0) return LV_OK;
  AuxSet as;
  as.n = n_aux;
  for (int a = 0; a < n_aux; ++a) as.a[a] = aux[a];
  cudaStream_t s = (cudaStream_t)stream;
  // children: at most floor(top * n) splits
  const int64_t max_children = 8 * (int64_t)(((unsigned long long)p->top_ppm * (unsigned long long)n) / 1000000ull);
  const int64_t warps = (n + 31) / 32 + (max_children + 31) / 32;
  const unsigned grid = (unsigned)((warps * 32 + TPB - 1) / TPB);
#define LV_SUB(DT, ST)                                                                                                 \
  k_sd_write<DT, ST><<<grid, TPB, 0, s>>>(n, max_children, w.surv, w.surv_pos, w.sel_list, w.totals, w.st,           \
                                          (const float4*)in->geom, in->level, (const DT*)in->density,                \
                                          (const ST*)in->sh, (float4*)out->geom, (uint8_t*)out->level,               \
                                          (DT*)out->density, (ST*)out->sh, as)
  if (in->density_dtype == LV_F32 && in->sh_dtype == LV_F32) LV_SUB(float, float);
  else if (in->density_dtype == LV_F16 && in->sh_dtype == LV_F32) LV_SUB(__half, float);
  else if (in->density_dtype == LV_F32 && in->sh_dtype == LV_BF16) LV_SUB(float, __nv_bfloat16);
  else LV_SUB(__half, __nv_bfloat16);
#undef LV_SUB
  count_launch(1);
  return cuda_check(cudaGetLastError(), "lv_subdivide_apply");
}

extern "C" lv_status lv_subdivide_priority(const lv_voxels* in, const float* delta, const float* z, const float* u,
                                           const uint8_t* seen, const uint8_t* prune_mask, const lv_subdiv_params* p,
                                           const lv_aux_array* aux, int n_aux, const lv_voxels* out,
                                           uint8_t* selected, int64_t* d_n_new, void* workspace, size_t ws_bytes,
                                           int32_t* d_status, void* stream) {
  lv_status e = check_sub(in, p, n_aux, aux, out);
  if (e != LV_OK) return e;
  if (!out) { set_error("null output"); return LV_ERR_INVALID_ARG; }
  e = lv_subdivide_select(in, delta, z, u, seen, prune_mask, p, out->n, selected, d_n_new, workspace, ws_bytes,
                          d_status, stream);
  if (e != LV_OK) return e;
  return lv_subdivide_apply(in, p, aux, n_aux, out, workspace, ws_bytes, stream);
}

extern "C" lv_status lv_subdivide_apply_inplace(const lv_voxels* vox, int64_t capacity, const lv_subdiv_params* p,
                                                const lv_aux_array* aux, int n_aux, void* workspace, size_t ws_bytes,
                                                void* stream) {
  lv_status e = check_sub(vox, p, n_aux, aux, nullptr);
  if (e != LV_OK) return e;
  const int64_t n = vox->n;
  if (capacity < n) { set_error("capacity %lld < voxel count %lld", (long long)capacity, (long long)n); return LV_ERR_INVALID_ARG; }
  for (int a = 0; a < n_aux; ++a)
    if (aux[a].in && aux[a].in != aux[a].out) { set_error("aux array %d: in place, in must be NULL or equal out", a); return LV_ERR_INVALID_ARG; }
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  SubWs w = carve_sub(workspace, n);
  if (ws_bytes < w.bytes) { set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return LV_ERR_WORKSPACE; }
  if (n == 0) return LV_OK;
  AuxSet as;
  as.n = n_aux;
  for (int a = 0; a < n_aux; ++a) as.a[a] = aux[a];
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t* holes = w.zkey;  // the pruned rows in id order, from the selection (k_sd_list)
  const int64_t max_children = 8 * (int64_t)(((unsigned long long)p->top_ppm * (unsigned long long)n) / 1000000ull);
  const unsigned grid = (unsigned)((max_children + TPB - 1) / TPB);  // one warp per 32 children
  const unsigned tail_grid = (unsigned)std::min<int64_t>((n + TPB / 32 - 1) / (TPB / 32), 1216);
#define LV_IP(DT, ST)                                                                                                  \
  do {                                                                                                                \
    if (grid > 0)                                                                                                     \
      k_ip_children<DT, ST><<<grid, TPB, 0, s>>>(n, w.sel_list, holes, w.totals, w.st, (float4*)vox->geom,            \
                                                 (uint8_t*)vox->level, (DT*)vox->density, (ST*)vox->sh, as);          \
    k_ip_tail<DT, ST><<<tail_grid, TPB, 0, s>>>(n, holes, w.totals, w.st, (float4*)vox->geom, (uint8_t*)vox->level,   \
                                                (DT*)vox->density, (ST*)vox->sh, as);                                 \
  } while (0)
  if (vox->density_dtype == LV_F32 && vox->sh_dtype == LV_F32) LV_IP(float, float);
  else if (vox->density_dtype == LV_F16 && vox->sh_dtype == LV_F32) LV_IP(__half, float);
  else if (vox->density_dtype == LV_F32 && vox->sh_dtype == LV_BF16) LV_IP(float, __nv_bfloat16);
  else LV_IP(__half, __nv_bfloat16);
#undef LV_IP
  count_launch(grid > 0 ? 2 : 1);
  return cuda_check(cudaGetLastError(), "lv_subdivide_apply_inplace");
}

extern "C" size_t lv_compact_workspace_size(int64_t n) {
  if (n < 0) return 0;
  return carve_sub(nullptr, n).bytes;
}

extern "C" lv_status lv_compact(const lv_voxels* in, const uint8_t* keep, const lv_aux_array* aux, int n_aux,
                                const lv_voxels* out, int64_t* d_n_new, void* workspace, size_t ws_bytes,
                                int32_t* d_status, void* stream) {
  lv_status e = check_arrays(in, n_aux, aux, out);
  if (e != LV_OK) return e;
  if (!out) { set_error("null output"); return LV_ERR_INVALID_ARG; }
  const int64_t n = in->n;
  if (n > 0 && !keep) { set_error("null keep mask"); return LV_ERR_INVALID_ARG; }
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  SubWs w = carve_sub(workspace, n);
  if (ws_bytes < w.bytes) { set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return LV_ERR_WORKSPACE; }
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    if (d_n_new) cudaMemsetAsync(d_n_new, 0, sizeof(int64_t), s);
    return cuda_check(cudaGetLastError(), "lv_compact");
  }
  AuxSet as;
  as.n = n_aux;
  for (int a = 0; a < n_aux; ++a) as.a[a] = aux[a];
  cudaMemsetAsync(w.st, 0, sizeof(SubState), s);
  const int blocks = blocks_for(n);
  k_cp_flags<<<blocks, TPB, 0, s>>>(n, keep, w.surv);
  scan2(w.surv, nullptr, n, w.surv_pos, nullptr, w.totals, w.scan_tmp, s);  // totals[1] = 0: no children
  k_sd_check<<<1, 32, 0, s>>>(w.totals, w.st, out->n, d_n_new, d_status);
  const unsigned grid = (unsigned)((((n + 31) / 32) * 32 + TPB - 1) / TPB);  // one warp per 32 voxels
#define LV_CP(DT, ST)                                                                                         \
  k_sd_write<DT, ST><<<grid, TPB, 0, s>>>(n, 0, w.surv, w.surv_pos, w.sel_list, w.totals, w.st,            \
                                          (const float4*)in->geom, in->level, (const DT*)in->density,       \
                                          (const ST*)in->sh, (float4*)out->geom, (uint8_t*)out->level,      \
                                          (DT*)out->density, (ST*)out->sh, as)
  if (in->density_dtype == LV_F32 && in->sh_dtype == LV_F32) LV_CP(float, float);
  else if (in->density_dtype == LV_F16 && in->sh_dtype == LV_F32) LV_CP(__half, float);
  else if (in->density_dtype == LV_F32 && in->sh_dtype == LV_BF16) LV_CP(float, __nv_bfloat16);
  else LV_CP(__half, __nv_bfloat16);
#undef LV_CP
  count_launch(3);
  return cuda_check(cudaGetLastError(), "lv_compact");
}

// lv_prims.cu -- scan, radix sort and radix select kernels (sm_103a).
#include "lv_prims.cuh"

namespace lv {

// ============================================================ two-channel scan
namespace {

constexpr int SCAN_THREADS = 256;

__device__ __forceinline__ void block_exclusive_scan2(unsigned long long& a, uint32_t& b, unsigned long long* sa,
                                                      uint32_t* sb, unsigned long long& tot_a, uint32_t& tot_b) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long ia = a;
  uint32_t ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long ta = __shfl_up_sync(FULL, ia, o);
    uint32_t tb = __shfl_up_sync(FULL, ib, o);
    if (lane >= o) { ia += ta; ib += tb; }
  }
  if (lane == 31) { sa[warp] = ia; sb[warp] = ib; }
  __syncthreads();
  if (warp == 0) {
    unsigned long long wa = lane < SCAN_THREADS / 32 ? sa[lane] : 0ull;
    uint32_t wb = lane < SCAN_THREADS / 32 ? sb[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned long long ta = __shfl_up_sync(FULL, wa, o);
      uint32_t tb = __shfl_up_sync(FULL, wb, o);
      if (lane >= o) { wa += ta; wb += tb; }
    }
    if (lane < SCAN_THREADS / 32) { sa[lane] = wa; sb[lane] = wb; }
  }
  __syncthreads();
  tot_a = sa[SCAN_THREADS / 32 - 1];
  tot_b = sb[SCAN_THREADS / 32 - 1];
  unsigned long long pa = warp ? sa[warp - 1] : 0ull;
  uint32_t pb = warp ? sb[warp - 1] : 0u;
  a = pa + ia - a;
  b = pb + ib - b;
  __syncthreads();
}

__global__ void k_scan2_reduce(const uint32_t* a, const uint32_t* b, int64_t n, int64_t chunk,
                               unsigned long long* bsa, uint32_t* bsb) {
  __shared__ unsigned long long sa[32];
  __shared__ uint32_t sb[32];
  int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  unsigned long long ta = 0;
  uint32_t tb = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += SCAN_THREADS) {
    ta += a[i];
    if (b) tb += b[i];
  }
  unsigned long long xa = ta, tot_a;
  uint32_t xb = tb, tot_b;
  block_exclusive_scan2(xa, xb, sa, sb, tot_a, tot_b);
  if (threadIdx.x == 0) { bsa[blockIdx.x] = tot_a; bsb[blockIdx.x] = tot_b; }
}

__global__ void k_scan2_blocks(unsigned long long* bsa, uint32_t* bsb, int nb, unsigned long long* totals) {
  __shared__ unsigned long long sa[32];
  __shared__ uint32_t sb[32];
  // nb <= SCAN_BLOCKS = 2 * SCAN_THREADS: two items per thread
  int i0 = threadIdx.x * 2;
  unsigned long long a0 = i0 < nb ? bsa[i0] : 0, a1 = i0 + 1 < nb ? bsa[i0 + 1] : 0;
  uint32_t b0 = i0 < nb ? bsb[i0] : 0, b1 = i0 + 1 < nb ? bsb[i0 + 1] : 0;
  unsigned long long xa = a0 + a1, ta;
  uint32_t xb = b0 + b1, tb;
  block_exclusive_scan2(xa, xb, sa, sb, ta, tb);
  if (i0 < nb) { bsa[i0] = xa; bsb[i0] = xb; }
  if (i0 + 1 < nb) { bsa[i0 + 1] = xa + a0; bsb[i0 + 1] = xb + b0; }
  if (threadIdx.x == 0) { totals[0] = ta; totals[1] = tb; }
}

// Each block scans its chunk in tiles of SCAN_THREADS x SCAN_ITEMS items.  A
// tile is loaded coalesced into shared memory, each thread then scans
// SCAN_ITEMS consecutive items serially, one block scan of the per-thread
// totals places them, and the results leave through shared memory as
// coalesced stores.
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
__global__ void __launch_bounds__(SCAN_THREADS) k_scan2_apply(const uint32_t* a, const uint32_t* b, int64_t n,
                                                             int64_t chunk, const unsigned long long* bsa,
                                                             const uint32_t* bsb, unsigned long long* out_a,
                                                             uint32_t* out_b) {
  __shared__ unsigned long long sa[32];
  __shared__ uint32_t sb[32];
  // one pad word per 8 items: a thread's 8 consecutive items then sit in
  // distinct banks across the warp
  __shared__ unsigned long long ta_s[SCAN_TILE + SCAN_TILE / 8];  // a in, then out_a
  __shared__ uint32_t tb_s[SCAN_TILE + SCAN_TILE / 8];            // b in, then out_b
  int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  unsigned long long carry_a = bsa[blockIdx.x];
  uint32_t carry_b = bsb[blockIdx.x];
  for (int64_t base = lo; base < hi; base += SCAN_TILE) {
    const int m = (int)min((int64_t)SCAN_TILE, hi - base);
    for (int q = threadIdx.x; q < SCAN_TILE; q += SCAN_THREADS) {
      ta_s[q + (q >> 3)] = q < m ? a[base + q] : 0ull;
      tb_s[q + (q >> 3)] = (b && q < m) ? b[base + q] : 0u;
    }
    __syncthreads();
    const int q0 = threadIdx.x * (SCAN_ITEMS + 1);  // padded index of item threadIdx.x * 8
    unsigned long long va[SCAN_ITEMS];
    uint32_t vb[SCAN_ITEMS];
    unsigned long long ta = 0;
    uint32_t tb = 0;
#pragma unroll
    for (int u = 0; u < SCAN_ITEMS; ++u) {
      va[u] = ta_s[q0 + u];
      vb[u] = tb_s[q0 + u];
      ta += va[u];
      tb += vb[u];
    }
    unsigned long long xa = ta, tot_a;
    uint32_t xb = tb, tot_b;
    block_exclusive_scan2(xa, xb, sa, sb, tot_a, tot_b);  // ends with a barrier
    unsigned long long ra = carry_a + xa;
    uint32_t rb = carry_b + xb;
#pragma unroll
    for (int u = 0; u < SCAN_ITEMS; ++u) {
      ta_s[q0 + u] = ra;
      tb_s[q0 + u] = rb;
      ra += va[u];
      rb += vb[u];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < m; q += SCAN_THREADS) {
      if (out_a) out_a[base + q] = ta_s[q + (q >> 3)];
      if (out_b) out_b[base + q] = tb_s[q + (q >> 3)];
    }
    __syncthreads();
    carry_a += tot_a;
    carry_b += tot_b;
  }
}

}  // namespace

size_t scan2_tmp_bytes() { return SCAN_BLOCKS * (sizeof(unsigned long long) + sizeof(uint32_t)) + 256; }

void scan2(const uint32_t* a, const uint32_t* b, int64_t n, unsigned long long* out_a, uint32_t* out_b,
           unsigned long long* totals, void* tmp, cudaStream_t s) {
  unsigned long long* bsa = (unsigned long long*)tmp;
  uint32_t* bsb = (uint32_t*)(bsa + SCAN_BLOCKS);
  int64_t chunk = (n + SCAN_BLOCKS - 1) / SCAN_BLOCKS;
  if (chunk < 1) chunk = 1;
  k_scan2_reduce<<<SCAN_BLOCKS, SCAN_THREADS, 0, s>>>(a, b, n, chunk, bsa, bsb);
  k_scan2_blocks<<<1, SCAN_THREADS, 0, s>>>(bsa, bsb, SCAN_BLOCKS, totals);
  k_scan2_apply<<<SCAN_BLOCKS, SCAN_THREADS, 0, s>>>(a, b, n, chunk, bsa, bsb, out_a, out_b);
  count_launch(3);
}

// ============================================================ radix sort
// LSD radix sort with 8-bit digits and one kernel per digit pass (a
// "one-sweep" schedule).  One histogram kernel first counts every pass's
// digits over all items.  Each pass kernel then takes tiles of Os<K>::TILE items
// in ticket order (an atomic counter, so a tile's predecessors are already
// running or done), ranks its items by digit in shared memory (a warp-private
// histogram per warp; the lanes of a digit found by bit ballots or by
// __match_any_sync, whichever suits the keys), publishes its per-digit counts, and
// finds the number of items with each digit in all earlier tiles by looking
// back through their published words (decoupled look-back: a tile that has
// published its inclusive prefix ends the walk).  A published word packs a
// 2-bit flag (0 not yet, 1 tile count, 2 inclusive prefix) and a 62-bit
// count, so one 64-bit load reads both.  Every wait is bounded: a walk that
// gives up reports LV_ERR_TIMEOUT and counts the missing word as zero.
namespace {

constexpr int OS_ITEMS = 8;                      // per lane
constexpr int RADIX = 256;
constexpr int OS_MAX_PASSES = 8;
constexpr int OS_HIST_BLOCKS = 2 * 152;
constexpr unsigned long long OS_FLAG_AGG = 1ull << 62;
constexpr unsigned long long OS_FLAG_INC = 2ull << 62;
constexpr unsigned long long OS_VALUE = (1ull << 62) - 1;
constexpr unsigned OS_SPIN_LIMIT = 1u << 20;     // polls per look-back walk before giving up
constexpr int OS_LOOK_WINDOW = 8;                // earlier tiles' words loaded together
constexpr float OS_MATCH_BELOW = 6.f;            // expected distinct digits per warp below which match_any ranks
constexpr int OS_MATCH_MAX_GROUPS = 16;          // distinct digits in a warp's round up to which match_any ranks next
constexpr int OS_HIST_THREADS = 256;

// Tile shape of the pass kernel: 512 threads (4096 items, about 52 KB of
// static shared memory) for 32-bit keys, 256 threads (2048 items, about 36 KB)
// for 64-bit keys, whose staged keys are twice as large; 64 registers a thread
// either way, so 2048 threads fit on an SM.  Threads d < RADIX look after
// digit d.
template <typename K>
struct Os {
  static constexpr int THREADS = sizeof(K) == 4 ? 512 : 256;
  static constexpr int WARPS = THREADS / 32;
  static constexpr int TILE = THREADS * OS_ITEMS;
  static constexpr int MIN_BLOCKS = 1024 / THREADS;
  static_assert(THREADS >= RADIX && THREADS % 32 == 0, "one thread per digit");
};
constexpr int OS_MIN_TILE = 256 * OS_ITEMS;  // the look-back words are sized for the smaller tile

// On overflow (more pairs than capacity) the list is treated as empty: the
// emit step then left holes in the buffers, and the caller's status word
// carries LV_ERR_CAPACITY.
__device__ __forceinline__ int64_t rs_count(const unsigned long long* d_count, int64_t cap) {
  unsigned long long c = *d_count;
  return c <= (unsigned long long)cap ? (int64_t)c : 0;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

struct SortTmp {
  uint32_t* ghist;               // [OS_MAX_PASSES][RADIX] digit counts of every pass
  uint32_t* ticket;              // [2] tile tickets (pass p uses p & 1)
  unsigned long long* look[2];   // [tiles][RADIX] published words (pass p uses p & 1)
  size_t bytes;
};

SortTmp carve_sort(void* base, int64_t cap) {
  SortTmp t;
  Carve c(base);
  const int64_t tiles = (cap + OS_MIN_TILE - 1) / OS_MIN_TILE;
  t.ghist = c.take<uint32_t>(OS_MAX_PASSES * RADIX + 64);  // the tickets follow the counts
  t.ticket = t.ghist ? t.ghist + OS_MAX_PASSES * RADIX : nullptr;
  t.look[0] = c.take<unsigned long long>(tiles * RADIX);
  t.look[1] = c.take<unsigned long long>(tiles * RADIX);
  t.bytes = c.off;
  return t;
}

// Digit counts of all passes (block-private shared histograms, one global
// atomic per nonzero bin), and clears the look-back words of the first pass.
template <typename K>
__global__ void __launch_bounds__(OS_HIST_THREADS) k_os_hist(const K* __restrict__ keys, const unsigned long long* d_count,
                                                       int64_t cap, int passes, uint32_t* __restrict__ ghist,
                                                       unsigned long long* __restrict__ look0) {
  __shared__ uint32_t sh[OS_MAX_PASSES * RADIX];
  for (int i = threadIdx.x; i < passes * RADIX; i += OS_HIST_THREADS) sh[i] = 0;
  __syncthreads();
  const int64_t n = rs_count(d_count, cap);
  const int64_t ntiles = (n + Os<K>::TILE - 1) / Os<K>::TILE;
  const int64_t stride = (int64_t)gridDim.x * OS_HIST_THREADS;
  for (int64_t i = blockIdx.x * (int64_t)OS_HIST_THREADS + threadIdx.x; i < ntiles * RADIX; i += stride) look0[i] = 0ull;
  int64_t i = blockIdx.x * (int64_t)OS_HIST_THREADS + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    K k[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) k[u] = keys[i + u * stride];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      for (int p = 0; p < passes; ++p) atomicAdd(&sh[p * RADIX + ((uint32_t)(k[u] >> (8 * p)) & (RADIX - 1))], 1u);
  }
  for (; i < n; i += stride) {
    const K k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p * RADIX + ((uint32_t)(k >> (8 * p)) & (RADIX - 1))], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < passes * RADIX; b += OS_HIST_THREADS)
    if (sh[b]) atomicAdd(&ghist[b], sh[b]);
}

// exclusive scan of one value per thread over the block of WARPS warps
template <int WARPS>
__device__ __forceinline__ uint32_t os_block_excl(uint32_t c, uint32_t* s_w) {
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

template <typename K>
__global__ void __launch_bounds__(Os<K>::THREADS, Os<K>::MIN_BLOCKS) k_os_pass(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                         K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                         const unsigned long long* d_count, int64_t cap, int pass,
                                                         const uint32_t* __restrict__ ghist, uint32_t* ticket,
                                                         unsigned long long* look, unsigned long long* look_next,
                                                         int32_t* status, unsigned spin_limit,
                                                         uint32_t* __restrict__ key_ranges) {
  constexpr int OS_THREADS = Os<K>::THREADS, OS_WARPS = Os<K>::WARPS, OS_TILE = Os<K>::TILE;
  __shared__ uint32_t s_wh[OS_WARPS][RADIX + 1];  // warp digit counts -> warp prefixes (bin RADIX: padding items)
  __shared__ uint32_t s_start[RADIX];             // tile-local start of each digit
  __shared__ long long s_off[RADIX];              // global position of the digit's first item minus s_start
  __shared__ uint32_t s_w[2][OS_WARPS];
  __shared__ K s_k[OS_TILE];
  __shared__ uint32_t s_v[OS_TILE];
  __shared__ uint32_t s_tile;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int shift = 8 * pass;
  if (t == 0) s_tile = atomicAdd(&ticket[pass & 1], 1u);
  for (int i = t; i < OS_WARPS * (RADIX + 1); i += OS_THREADS) (&s_wh[0][0])[i] = 0u;
  __syncthreads();
  const int64_t n = rs_count(d_count, cap);
  const int64_t ntiles = (n + OS_TILE - 1) / OS_TILE;
  const int64_t tile = s_tile;
  if (tile >= ntiles) return;  // block-uniform
  if (tile == 0 && t == 0) ticket[(pass + 1) & 1] = 0u;  // the next pass's counter (last used two passes ago)
  if (t < RADIX) look_next[tile * RADIX + t] = 0ull;      // and its look-back words

  const uint32_t gcount = t < RADIX ? ghist[pass * RADIX + t] : 0u;  // read early: its latency overlaps the loads
  // ---- load (warp-striped: lane l of warp w holds items w*256 + j*32 + l)
  const int64_t base = tile * OS_TILE;
  const int m = (int)min((int64_t)OS_TILE, n - base);
  K k[OS_ITEMS];
  uint32_t v[OS_ITEMS], dr[OS_ITEMS];  // digit (RADIX for padding) in bits 0-8, then the warp rank
  const int wofs = warp * (32 * OS_ITEMS) + lane;
  if (m == OS_TILE) {
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
      const int64_t i = base + wofs + j * 32;
      k[j] = kin[i];
      v[j] = vin ? vin[i] : (uint32_t)i;  // no values: the item's position
    }
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) dr[j] = (uint32_t)(k[j] >> shift) & (RADIX - 1);
  } else {
#pragma unroll
    for (int j = 0; j < OS_ITEMS; ++j) {
      const int q = wofs + j * 32;
      const int64_t i = base + q;
      const bool ok = q < m;
      k[j] = ok ? kin[i] : (K)0;
      v[j] = ok ? (vin ? vin[i] : (uint32_t)i) : 0u;
      dr[j] = ok ? ((uint32_t)(k[j] >> shift) & (RADIX - 1)) : (uint32_t)RADIX;
    }
  }
  // ---- digit base of this pass: exclusive scan of the global counts
  const uint32_t gbase = os_block_excl<OS_WARPS>(gcount, s_w[0]);
  // Expected number of distinct digits among 32 items of this pass, from the
  // global counts: sum over digits of 1 - (1 - p_d)^32.  __match_any_sync
  // finds the lanes of a digit fastest when a warp holds few distinct digits
  // (clustered keys such as the high bytes of depths); eight bit ballots cost
  // the same for any keys and win when they are spread.
  bool use_match;
  {
    __shared__ float s_e[OS_WARPS];
    float q = t < RADIX ? 1.f - (float)gcount / (float)n : 1.f;
#pragma unroll
    for (int k = 0; k < 5; ++k) q *= q;  // (1 - p)^32
    float e = 1.f - q;
#pragma unroll
    for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(FULL, e, o);
    if (lane == 0) s_e[warp] = e;
    __syncthreads();
    float tot = 0.f;
#pragma unroll
    for (int w = 0; w < OS_WARPS; ++w) tot += s_e[w];
    use_match = tot < OS_MATCH_BELOW;  // block-uniform
  }

  // ---- stable rank inside each warp (items in j-major, lane-minor order)
  // The histogram's guess starts each warp off; after every round the warp
  // switches by the number of distinct digits that round held, since
  // neighbouring items are often alike (pairs of one voxel, depths of nearby
  // voxels) in ways the global counts do not show.
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < OS_ITEMS; ++j) {
    const uint32_t d = dr[j];
    uint32_t peers;
    if (use_match) {  // warp-uniform
      peers = __match_any_sync(FULL, d);
    } else {
      // lanes holding the same digit: eight bit ballots intersected
      const uint32_t valid = __ballot_sync(FULL, d < RADIX);
      peers = d < RADIX ? valid : ~valid;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const uint32_t m = __ballot_sync(FULL, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? m : ~m;
      }
    }
    const bool leader = (peers & lt_mask) == 0;
    use_match = __popc(__ballot_sync(FULL, leader)) <= OS_MATCH_MAX_GROUPS;
    const uint32_t cur = s_wh[warp][d];
    dr[j] = d | ((cur + __popc(peers & lt_mask)) << 9);
    __syncwarp();
    if (leader) s_wh[warp][d] = cur + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // ---- per digit: warp prefixes and the tile count, published at once
  uint32_t cnt = 0;
  if (t < RADIX) {
#pragma unroll
    for (int w = 0; w < OS_WARPS; ++w) {
      const uint32_t c = s_wh[w][t];
      s_wh[w][t] = cnt;
      cnt += c;
    }
    st_relaxed(&look[tile * RADIX + t], (tile == 0 ? OS_FLAG_INC : OS_FLAG_AGG) | cnt);
  }
  const uint32_t start = os_block_excl<OS_WARPS>(cnt, s_w[1]);
  if (t < RADIX) s_start[t] = start;
  __syncthreads();
  // ---- scatter into shared memory in (digit, rank) order
#pragma unroll
  for (int j = 0; j < OS_ITEMS; ++j) {
    const uint32_t d = dr[j] & 511u;
    if (d < RADIX) {
      const uint32_t pos = s_start[d] + s_wh[warp][d] + (dr[j] >> 9);
      s_k[pos] = k[j];
      s_v[pos] = v[j];
    }
  }
  // ---- look back: items of digit t in all earlier tiles, OS_LOOK_WINDOW words per round trip
  unsigned long long excl = 0;
  if (tile > 0 && t < RADIX) {
    int64_t j = tile - 1;  // nearest word not summed yet
    unsigned spins = 0;    // polls of unpublished words over the whole walk
    bool done = false;
    while (!done) {
      unsigned long long wv[OS_LOOK_WINDOW];
#pragma unroll
      for (int u = 0; u < OS_LOOK_WINDOW; ++u)  // before tile 0: an inclusive zero
        wv[u] = j - u >= 0 ? ld_relaxed(&look[(j - u) * RADIX + t]) : OS_FLAG_INC;
      int u = 0;
#pragma unroll
      for (; u < OS_LOOK_WINDOW; ++u) {
        if ((wv[u] >> 62) == 0ull) break;
        excl += wv[u] & OS_VALUE;
        if (wv[u] & OS_FLAG_INC) { done = true; break; }
      }
      if (done) break;
      j -= u;
      if (u < OS_LOOK_WINDOW) {
        // word j is not published yet: wait for it alone
        while (true) {
          if (spins >= spin_limit) {
            // out of patience: report once, count this and any further unpublished word as zero
            if (spins++ == spin_limit) report(status, LV_ERR_TIMEOUT);
            --j;
            break;
          }
          ++spins;
          __nanosleep(32);
          if ((ld_relaxed(&look[j * RADIX + t]) >> 62) != 0ull) break;
        }
      }
    }
    st_relaxed(&look[tile * RADIX + t], OS_FLAG_INC | (excl + cnt));
  }
  if (t < RADIX) s_off[t] = (long long)gbase + (long long)excl - (long long)start;
  __syncthreads();
  // ---- write out: consecutive threads take consecutive sorted items
#pragma unroll
  for (int j = 0; j < OS_ITEMS; ++j) {
    const int q = j * OS_THREADS + t;
    if (q < m) {
      const K kk = s_k[q];
      const int64_t g = s_off[(uint32_t)(kk >> shift) & (RADIX - 1)] + q;
      kout[g] = kk;
      vout[g] = s_v[q];
      if constexpr (sizeof(K) == 4) if (key_ranges) {
        // items of one digit are consecutive here and in the output, so a key's first and last
        // item in this tile bound its positions; the extremes over all tiles are its range
        if (q == 0 || s_k[q - 1] != kk) atomicMin(&key_ranges[2 * (uint64_t)kk], (uint32_t)g);
        if (q == m - 1 || s_k[q + 1] != kk) atomicMax(&key_ranges[2 * (uint64_t)kk + 1], (uint32_t)(g + 1));
      }
    }
  }
}

}  // namespace

size_t sort_tmp_bytes(int64_t cap) { return carve_sort(nullptr, cap > 0 ? cap : 1).bytes; }
int sort_passes(int end_bit) { return (end_bit + 7) / 8; }

template <typename K>
static int radix_sort_t(const K* kin, const uint32_t* vin, K* k0, uint32_t* v0, K* k1, uint32_t* v1, void* tmp,
                        const unsigned long long* d_count, int64_t cap, int end_bit, int32_t* status,
                        cudaStream_t s, uint32_t* key_ranges, bool counted) {
  int passes = sort_passes(end_bit);
  if (passes > (int)sizeof(K)) passes = (int)sizeof(K);
  if (passes == 0 || cap <= 0) return 0;
  SortTmp st = carve_sort(tmp, cap);
  K* kb[2] = {k0, k1};
  uint32_t* vb[2] = {v0, v1};
  const int64_t tiles = (cap + Os<K>::TILE - 1) / Os<K>::TILE;
  if (!counted) {
    zero_async(s, st.ghist, sizeof(uint32_t) * (OS_MAX_PASSES * RADIX + 2));  // counts and tickets
    const int hb = (int)min((int64_t)OS_HIST_BLOCKS, tiles);
    k_os_hist<K><<<hb, OS_HIST_THREADS, 0, s>>>(kin, d_count, cap, passes, st.ghist, st.look[0]);
  }
  for (int p = 0; p < passes; ++p) {
    // pass 0 reads the input (kept intact unless it is k0 / v0), pass p writes buffer (p + 1) & 1
    const K* ks = p == 0 ? kin : kb[p & 1];
    const uint32_t* vs = p == 0 ? vin : vb[p & 1];
    const int dst = (p + 1) & 1;
    k_os_pass<K><<<(unsigned)tiles, Os<K>::THREADS, 0, s>>>(ks, vs, kb[dst], vb[dst], d_count, cap, p, st.ghist,
                                                       st.ticket, st.look[p & 1], st.look[(p + 1) & 1], status,
                                                       OS_SPIN_LIMIT, p == passes - 1 ? key_ranges : nullptr);
  }
  count_launch((counted ? 0 : 1) + passes);
  return passes & 1;
}

int radix_sort_pairs(const uint32_t* kin, const uint32_t* vin, uint32_t* k0, uint32_t* v0, uint32_t* k1,
                     uint32_t* v1, void* tmp, const unsigned long long* d_count, int64_t cap, int end_bit,
                     int32_t* status, cudaStream_t s, uint32_t* key_ranges, bool counted) {
  return radix_sort_t<uint32_t>(kin, vin, k0, v0, k1, v1, tmp, d_count, cap, end_bit, status, s, key_ranges,
                                counted);
}

SortCountTargets sort_count_targets(void* tmp, int64_t cap) {
  const SortTmp st = carve_sort(tmp, cap);
  SortCountTargets t;
  t.counts = st.ghist;
  t.look0 = st.look[0];
  t.tile = Os<uint32_t>::TILE;
  t.zero_bytes = sizeof(uint32_t) * (OS_MAX_PASSES * RADIX + 2);
  return t;
}

int radix_sort_pairs(const uint64_t* kin, const uint32_t* vin, uint64_t* k0, uint32_t* v0, uint64_t* k1,
                     uint32_t* v1, void* tmp, const unsigned long long* d_count, int64_t cap, int end_bit,
                     int32_t* status, cudaStream_t s) {
  return radix_sort_t<uint64_t>(kin, vin, k0, v0, k1, v1, tmp, d_count, cap, end_bit, status, s, nullptr, false);
}

// ---- bounded-wait check: one pass over two tiles where only the second tile's
// block runs (its ticket counter starts at 1), so the first tile's counts are
// never published and the look-back must give up.
namespace {
constexpr int64_t DBG_ITEMS = 2 * Os<uint32_t>::TILE;

struct DbgWs {
  uint32_t *k0, *k1, *v1;
  unsigned long long* count;
  void* tmp;
  size_t bytes;
};
DbgWs carve_dbg(void* base) {
  DbgWs w;
  Carve c(base);
  w.k0 = c.take<uint32_t>(DBG_ITEMS);
  w.k1 = c.take<uint32_t>(DBG_ITEMS);
  w.v1 = c.take<uint32_t>(DBG_ITEMS);
  w.count = c.take<unsigned long long>(1);
  w.tmp = c.take<char>(sort_tmp_bytes(DBG_ITEMS));
  w.bytes = c.off;
  return w;
}
__global__ void k_dbg_setup(unsigned long long* count, uint32_t* ticket) {
  if (threadIdx.x == 0) {
    *count = (unsigned long long)DBG_ITEMS;
    ticket[0] = 1u;  // the one block launched takes tile 1
  }
}
}  // namespace

}  // namespace lv

extern "C" size_t lv_debug_sort_timeout_workspace_size(void) { return lv::carve_dbg(nullptr).bytes; }

extern "C" lv_status lv_debug_sort_timeout(int32_t spin_limit, void* workspace, size_t ws_bytes, int32_t* d_status,
                                           void* stream) {
  using namespace lv;
  if (spin_limit < 1 || spin_limit > (int32_t)OS_SPIN_LIMIT || !d_status) { set_error("bad arguments"); return LV_ERR_INVALID_ARG; }
  if (!workspace || ((uintptr_t)workspace & 255)) { set_error("workspace must be non-null and 256-byte aligned"); return LV_ERR_INVALID_ARG; }
  DbgWs w = carve_dbg(workspace);
  if (ws_bytes < w.bytes) { set_error("workspace %zu < %zu bytes", ws_bytes, w.bytes); return LV_ERR_WORKSPACE; }
  cudaStream_t s = (cudaStream_t)stream;
  SortTmp st = carve_sort(w.tmp, DBG_ITEMS);
  cudaMemsetAsync(workspace, 0, w.bytes, s);  // keys, counts, tickets and look-back words
  cudaMemsetAsync(d_status, 0, sizeof(int32_t), s);
  k_dbg_setup<<<1, 32, 0, s>>>(w.count, st.ticket);
  k_os_pass<uint32_t><<<1, Os<uint32_t>::THREADS, 0, s>>>(w.k0, nullptr, w.k1, w.v1, w.count, DBG_ITEMS, 0, st.ghist,
                                                          st.ticket, st.look[0], st.look[1], d_status,
                                                          (unsigned)spin_limit, nullptr);
  count_launch(2);
  return cuda_check(cudaGetLastError(), "lv_debug_sort_timeout");
}

namespace lv {

// ============================================================ grouped select
namespace {

constexpr int SEL_THREADS = 256;
constexpr int SEL_BLOCKS = 304;
constexpr int SEL_MAX_Q_PER_GROUP = 2;
constexpr int SEL_ITEMS = 16;       // items per thread per iteration, loads issued together

// One warp per query: find the digit holding the k-th item (warp scan over
// RADIX / 32 digits per lane) and extend the prefix; returns the updated query.
template <int RADIX>
__device__ __forceinline__ SelectQuery warp_pick(const uint32_t* __restrict__ row, SelectQuery s, int shift,
                                                 int lane) {
  constexpr int PER = RADIX / 32;  // 8 or 64 digits per lane, contiguous
  const uint4* hrow = (const uint4*)(row + lane * PER);
  uint32_t lsum = 0;
#pragma unroll 4
  for (int i = 0; i < PER / 4; ++i) {
    const uint4 c = hrow[i];
    lsum += c.x + c.y + c.z + c.w;
  }
  uint32_t incl = lsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  const uint32_t excl = incl - lsum;
  const uint32_t ball = __ballot_sync(FULL, s.k != 0 && incl >= s.k);
  int digit = -1;
  uint32_t newk = 0;
  if (ball) {
    // lane L's PER digits hold the k-th item: the warp loads them together (PER / 32 each),
    // scans them and finds the digit by ballot
    const int L = __ffs(ball) - 1;
    const uint32_t base = __shfl_sync(FULL, excl, L);
    const uint32_t* h = row + L * PER;
    constexpr int EPL = PER / 32 > 0 ? PER / 32 : 1;  // digits per lane: 2 (RADIX 2048) or 1 (256: lanes 0-7)
    uint32_t c[EPL];
    uint32_t my = 0;
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const int idx = lane * EPL + e;
      c[e] = idx < PER ? h[idx] : 0u;
      my += c[e];
    }
    uint32_t inc = my;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += y;
    }
    const uint32_t b2 = __ballot_sync(FULL, base + inc >= s.k);  // nonzero: the chunk holds the k-th item
    const int L2 = __ffs(b2) - 1;
    if (lane == L2) {
      uint32_t cum = base + inc - my;
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        if (digit < 0 && cum + c[e] >= s.k) { digit = L * PER + lane * EPL + e; newk = s.k - cum; }
        cum += c[e];
      }
    }
    digit = __shfl_sync(FULL, digit, L2);
    newk = __shfl_sync(FULL, newk, L2);
  }
  if (s.k == 0 || digit < 0) {
    s.k = 0;
    s.result = 0xffffffffu;
  } else {
    s.k = newk;
    s.prefix |= (uint32_t)digit << shift;
    if (shift == 0) s.result = s.prefix;
  }
  return s;
}

// The last digit's pick: one warp per query, q_in -> q (the two may be the same), and the
// histogram row cleared.
template <int RADIX>
__global__ void k_sel_pick(const SelectQuery* q_in, SelectQuery* q, int nq, int shift, uint32_t* hist) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= nq) return;  // warp-uniform
  const SelectQuery s = warp_pick<RADIX>(hist + (size_t)j * RADIX, q_in[j], shift, lane);
  uint4* hrow = (uint4*)(hist + (size_t)j * RADIX + lane * (RADIX / 32));
#pragma unroll 4
  for (int i = 0; i < RADIX / 128; ++i) hrow[i] = make_uint4(0u, 0u, 0u, 0u);
  if (lane == 0) q[j] = s;
}

// Histogram of the current digit (bits [shift, shift + width)) of every item
// whose bits above the digit match its query's prefix, by shared-memory
// atomics (combining the lanes of a bin first with __match_any_sync measured
// slower: the match costs more than the serialised atomics it saves).  When
// every query is in group 0 (at most two queries) a lean per-item path runs;
// otherwise queries of a group are contiguous, at most two per group.
// With hist_prev, every block first takes the previous digit's pick step from
// q_in and hist_prev itself, one warp per query (one launch less per digit than
// a separate pick kernel), and block 0 stores the picked queries in q_out.  clear (nullable)
// is zeroed by the grid for a later pass: nothing reads or writes it here.
template <int RADIX>
__global__ void __launch_bounds__(SEL_THREADS) k_sel_hist(const uint32_t* keys, const uint16_t* grp, int64_t n,
                                                         const SelectQuery* q, int nq, int shift, int width,
                                                         uint32_t* hist, const uint32_t* hist_prev, int prev_shift,
                                                         SelectQuery* q_out, uint32_t* clear, int clear_words) {
  extern __shared__ uint4 sh4[];  // nq * RADIX counters
  uint32_t* sh = (uint32_t*)sh4;
  __shared__ SelectQuery sq[SELECT_MAX_QUERIES];
  __shared__ uint8_t qfirst[SELECT_MAX_QUERIES], qcount[SELECT_MAX_QUERIES];
  if (clear)
    for (int64_t i = blockIdx.x * (int64_t)SEL_THREADS + threadIdx.x; i < clear_words;
         i += (int64_t)gridDim.x * SEL_THREADS)
      clear[i] = 0u;
  for (int i = threadIdx.x; i < nq; i += SEL_THREADS) sq[i] = q[i];
  __syncthreads();
  if (hist_prev) {
    // one warp per query, the block's warps in parallel
    const int lane = threadIdx.x & 31;
    for (int j = threadIdx.x >> 5; j < nq; j += SEL_THREADS / 32) {
      const SelectQuery r = warp_pick<RADIX>(hist_prev + (size_t)j * RADIX, sq[j], prev_shift, lane);
      if (lane == 0) sq[j] = r;
    }
    __syncthreads();
    if (blockIdx.x == 0)
      for (int i = threadIdx.x; i < nq; i += SEL_THREADS) q_out[i] = sq[i];
  }
  // nothing to do when every query is finished (k == 0): skip the rest of the pass
  int active = 0, all0 = nq <= SEL_MAX_Q_PER_GROUP;
  for (int j = 0; j < nq; ++j) {
    active |= sq[j].k != 0;
    all0 &= sq[j].group == 0;
  }
  if (!active) return;  // uniform over the grid
  for (int i = threadIdx.x; i < nq * RADIX / 4; i += SEL_THREADS) sh4[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = threadIdx.x; i < SELECT_MAX_QUERIES; i += SEL_THREADS) qcount[i] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = nq - 1; j >= 0; --j) {
      const uint32_t g = sq[j].group;
      if (g < SELECT_MAX_QUERIES) { qfirst[g] = (uint8_t)j; qcount[g]++; }
    }
  }
  __syncthreads();
  const int top = shift + width;
  const uint32_t hi_mask = top >= 32 ? 0u : (0xffffffffu << top);
  const uint32_t dmask = (1u << width) - 1u;
  const int64_t stride = (int64_t)gridDim.x * SEL_THREADS * SEL_ITEMS;
  if (all0) {
    // lean path: one group, queries 0 (and 1) in registers
    const uint32_t k0 = sq[0].k, p0 = sq[0].prefix;
    const uint32_t k1 = nq > 1 ? sq[1].k : 0u, p1 = nq > 1 ? sq[1].prefix : 0u;
    for (int64_t base = blockIdx.x * (int64_t)SEL_THREADS * SEL_ITEMS; base < n; base += stride) {  // warp-uniform
      uint32_t gv[SEL_ITEMS], kv[SEL_ITEMS];
#pragma unroll
      for (int u = 0; u < SEL_ITEMS; ++u) {  // issue all loads first
        const int64_t i = base + u * SEL_THREADS + threadIdx.x;
        gv[u] = i < n ? grp[i] : GROUP_NONE;
        kv[u] = i < n ? (keys ? keys[i] : (uint32_t)i) : 0u;
      }
#pragma unroll
      for (int u = 0; u < SEL_ITEMS; ++u) {
        const bool in = gv[u] == 0;
        const uint32_t key = kv[u], hk = key & hi_mask, d = (key >> shift) & dmask;
        int h = (in && k0 != 0 && hk == p0) ? (int)d : -1;
        if (h >= 0) atomicAdd(&sh[h], 1u);
        h = (in && k1 != 0 && hk == p1) ? RADIX + (int)d : -1;
        if (h >= 0) atomicAdd(&sh[h], 1u);
      }
    }
  } else {
    for (int64_t base = blockIdx.x * (int64_t)SEL_THREADS * SEL_ITEMS; base < n; base += stride) {  // warp-uniform
      uint32_t gv[SEL_ITEMS], kv[SEL_ITEMS];
#pragma unroll
      for (int u = 0; u < SEL_ITEMS; ++u) {  // issue all loads first
        const int64_t i = base + u * SEL_THREADS + threadIdx.x;
        gv[u] = i < n ? grp[i] : GROUP_NONE;
        kv[u] = i < n ? (keys ? keys[i] : (uint32_t)i) : 0u;
      }
#pragma unroll
      for (int u = 0; u < SEL_ITEMS; ++u) {
        const uint32_t g = gv[u], key = kv[u];
        const int cnt = g < SELECT_MAX_QUERIES ? qcount[g] : 0;
        const uint32_t d = (key >> shift) & dmask;
#pragma unroll
        for (int a = 0; a < SEL_MAX_Q_PER_GROUP; ++a) {
          int h = -1;
          if (a < cnt) {
            const int j = qfirst[g] + a;
            if (sq[j].k != 0 && (key & hi_mask) == sq[j].prefix) h = j * RADIX + (int)d;
          }
          if (h >= 0) atomicAdd(&sh[h], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nq * RADIX / 4; i += SEL_THREADS) {
    const uint4 c = sh4[i];
    if (c.x) atomicAdd(&hist[4 * i], c.x);
    if (c.y) atomicAdd(&hist[4 * i + 1], c.y);
    if (c.z) atomicAdd(&hist[4 * i + 2], c.z);
    if (c.w) atomicAdd(&hist[4 * i + 3], c.w);
  }
}

__global__ void k_sel_init(SelectQuery* q, int nq, uint32_t* hist, int hist_words) {
  int j = threadIdx.x;
  if (j < nq) { q[j].prefix = 0; q[j].result = 0xffffffffu; }
  for (int i = threadIdx.x; i < hist_words; i += blockDim.x) hist[i] = 0;
}

template <int RADIX>
void select_passes(const uint32_t* keys, const uint16_t* grp, int64_t n, SelectQuery* d_queries, int nq,
                   uint32_t* hist, SelectQuery* qs, int key_bits, int width, cudaStream_t s, uint32_t* h0) {
  // enough blocks to keep many loads in flight; fewer when every block must
  // clear and flush a large histogram (wide digits or many queries)
  const int64_t want = (n + SEL_THREADS * SEL_ITEMS - 1) / (SEL_THREADS * SEL_ITEMS);
  const int64_t cap_blocks = nq * RADIX <= 512 ? 2048 : SEL_BLOCKS;
  int blocks = (int)(want < cap_blocks ? want : cap_blocks);
  if (blocks < 1) blocks = 1;
  const size_t smem = sizeof(uint32_t) * RADIX * nq;
  static std::atomic<unsigned long long> done{0};
  once_per_device(done, [] {
    cudaFuncSetAttribute(k_sel_hist<RADIX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(uint32_t) * 256 * SELECT_MAX_QUERIES));
  });
  // three histogram buffers: pass p writes H[p % 3], reads H[(p - 1) % 3] for its pick step and
  // clears H[(p + 1) % 3] for pass p + 1 (k_sel_init cleared H[0]); the queries after p picks
  // are A[p]: A[0] = d_queries, then the two scratch copies in turn; the last pick writes d_queries.
  // With h0, the key producer has counted the first digit into H[0] = h0 and the query kernel
  // cleared H[1]; the passes and the last pick leave h0 cleared.
  const int words = nq * RADIX;
  uint32_t* H[3] = {hist, hist + words, hist + 2 * words};
  if (h0) {
    H[0] = h0;
    H[1] = hist;
    H[2] = hist + words;
  }
  auto A = [&](int p) { return p == 0 ? d_queries : qs + ((p - 1) % 2) * nq; };
  // digits from the top: the first one takes the remainder bits, the rest `width` each
  const int npass = (key_bits + width - 1) / width;
  int shift = key_bits, prev_shift = 0;
  for (int p = 0; p < npass; ++p) {
    const int wbits = p == 0 ? key_bits - width * (npass - 1) : width;
    shift -= wbits;
    if (p > 0 || !h0)
      k_sel_hist<RADIX><<<blocks, SEL_THREADS, smem, s>>>(keys, grp, n, A(p > 0 ? p - 1 : 0), nq, shift, wbits,
                                                          H[p % 3], p > 0 ? H[(p - 1) % 3] : nullptr, prev_shift,
                                                          p > 0 ? A(p) : nullptr, H[(p + 1) % 3], words);
    prev_shift = shift;
  }
  k_sel_pick<RADIX><<<(nq + 7) / 8, 256, 0, s>>>(A(npass - 1), d_queries, nq, 0, H[(npass - 1) % 3]);
  count_launch(npass + (h0 ? 0 : 1));
}

}  // namespace

size_t select_tmp_bytes(int n_queries) {
  const size_t narrow = 256 * (size_t)n_queries;
  const size_t wide = 2048 * (size_t)(n_queries < SEL_WIDE_MAX_Q ? n_queries : SEL_WIDE_MAX_Q);
  // three histogram buffers, then two copies of the queries
  return 3 * sizeof(uint32_t) * (narrow > wide ? narrow : wide) + 2 * sizeof(SelectQuery) * (size_t)n_queries + 512;
}

// the digit passes and the last pick, after the queries and the first histogram buffer are set up
static void select_run(const uint32_t* keys, const uint16_t* grp, int64_t n, SelectQuery* d_queries, int n_queries,
                       void* tmp, cudaStream_t s, uint32_t* h0) {
  const bool wide = n_queries <= SEL_WIDE_MAX_Q;
  const int words = select_hist_words(n_queries);
  uint32_t* hist = (uint32_t*)tmp;
  SelectQuery* qs = (SelectQuery*)(hist + 3 * (size_t)words);
  // ranking by index needs only the bits of n - 1 (at least one)
  int key_bits = 32;
  if (!keys) {
    key_bits = 1;
    while (key_bits < 32 && ((int64_t)1 << key_bits) < n) ++key_bits;
  }
  if (wide) select_passes<2048>(keys, grp, n, d_queries, n_queries, hist, qs, key_bits, 11, s, h0);
  else select_passes<256>(keys, grp, n, d_queries, n_queries, hist, qs, key_bits, 8, s, h0);
}

void select_kth(const uint32_t* keys, const uint16_t* grp, int64_t n, SelectQuery* d_queries, int n_queries,
                void* tmp, cudaStream_t s) {
  k_sel_init<<<1, 256, 0, s>>>(d_queries, n_queries, (uint32_t*)tmp, select_hist_words(n_queries));
  count_launch(1);
  select_run(keys, grp, n, d_queries, n_queries, tmp, s, nullptr);
}

void select_kth_prepared(const uint32_t* keys, const uint16_t* grp, int64_t n, SelectQuery* d_queries,
                         int n_queries, void* tmp, cudaStream_t s) {
  select_run(keys, grp, n, d_queries, n_queries, tmp, s, nullptr);
}

void select_kth_first(const uint32_t* keys, const uint16_t* grp, int64_t n, SelectQuery* d_queries, int n_queries,
                      uint32_t* h0, void* tmp, cudaStream_t s) {
  select_run(keys, grp, n, d_queries, n_queries, tmp, s, h0);
}

}  // namespace lv

// lv_prims.cuh -- device primitives: two-channel exclusive scan, LSD radix sort
// of (key, u32 value) pairs, grouped radix select.  No CUB: every kernel here
// is written for this library.  The scan and the select are reduce-then-scan
// with no inter-block waits; the sort's look-back waits are bounded.
#pragma once

#include "lv_common.cuh"

namespace lv {

// ---------------------------------------------------------------- scan
// out_a[i] = sum_{j<i} a[j] (64-bit), out_b[i] = sum_{j<i} b[j] (32-bit);
// totals[0] = sum a, totals[1] = sum b.  n is known on the host.  b == nullptr
// counts as all zeros; a null out_a or out_b is not written.
constexpr int SCAN_BLOCKS = 512;
size_t scan2_tmp_bytes();
void scan2(const uint32_t* a, const uint32_t* b, int64_t n, unsigned long long* out_a, uint32_t* out_b,
           unsigned long long* totals, void* tmp, cudaStream_t s);

// ---------------------------------------------------------------- radix sort
// Stable LSD sort of the first *d_count (key, value) pairs, 32- or 64-bit
// keys, on bits [0, end_bit) with 8-bit digits; nothing is sorted when
// *d_count > cap (an overflowed emit leaves holes).  The first pass reads
// (kin, vin), which may be (k0, v0); vin == nullptr stands for the values 0,
// 1, 2, ... (the items' positions).  Returns 0 when the result is in (k0, v0)
// and 1 when it is in (k1, v1).  With end_bit == 0 nothing runs and 0 is
// returned, so a caller that may sort no bits passes kin == k0 and vin == v0.
// tmp: sort_tmp_bytes(cap) bytes, 256-byte aligned, no initial contents.
// A bounded inter-block wait that gives up reports LV_ERR_TIMEOUT in *status
// (nullable).  key_ranges (32-bit keys, nullable): the last pass also writes
// the [first, end) positions of every key k it places into key_ranges[2k] by
// atomicMin and key_ranges[2k + 1] by atomicMax, so the caller sets them to
// (0xffffffff, 0) beforehand and keys absent from the list keep those values.
// counted (32-bit keys): the kernel that wrote the keys has already counted
// every pass's digits -- see sort_count_targets -- so no counting kernel runs.
size_t sort_tmp_bytes(int64_t cap);
int sort_passes(int end_bit);
int radix_sort_pairs(const uint32_t* kin, const uint32_t* vin, uint32_t* k0, uint32_t* v0, uint32_t* k1,
                     uint32_t* v1, void* tmp, const unsigned long long* d_count, int64_t cap, int end_bit,
                     int32_t* status, cudaStream_t s, uint32_t* key_ranges = nullptr, bool counted = false);

// What a kernel that writes the 32-bit keys does for radix_sort_pairs(counted
// = true) on the same tmp: the first `zero_bytes` of tmp are zero before it
// runs; it adds 1 at counts[p * 256 + ((key >> 8 p) & 255)] for every key and
// pass p < sort_passes(end_bit), and zeroes look0[0, ceil(items / tile) * 256)
// for the items the sort will see.
struct SortCountTargets {
  uint32_t* counts;
  unsigned long long* look0;
  int tile;
  size_t zero_bytes;
};
SortCountTargets sort_count_targets(void* tmp, int64_t cap);
int radix_sort_pairs(const uint64_t* kin, const uint32_t* vin, uint64_t* k0, uint32_t* v0, uint64_t* k1,
                     uint32_t* v1, void* tmp, const unsigned long long* d_count, int64_t cap, int end_bit,
                     int32_t* status, cudaStream_t s);

// ---------------------------------------------------------------- grouped select
// For each query q (group g_q, 1-based rank k_q), find the k-th smallest
// 32-bit key among the items i with grp[i] == g_q (0xffff = excluded).
// Queries live in device memory so that k can be computed on the device.
// After select_kth, queries[q].result holds the key, or 0xffffffff when
// k == 0 or the group has fewer than k items (queries[q].k is then 0).
// keys == nullptr ranks the items by their index (key = i).  Queries of one
// group must be contiguous, at most two per group, groups < 64.
constexpr int SELECT_MAX_QUERIES = 64;
constexpr uint16_t GROUP_NONE = 0xffff;
struct SelectQuery {
  uint32_t group;
  uint32_t k;
  uint32_t prefix;
  uint32_t result;
};
size_t select_tmp_bytes(int n_queries);
void select_kth(const uint32_t* keys, const uint16_t* grp, int64_t n, SelectQuery* d_queries, int n_queries,
                void* tmp, cudaStream_t s);

// select_kth without its set-up launch: the kernel that writes the queries
// also calls select_prepare (all threads of one block) for the same queries
// and scratch, so a select costs one launch less on the caller's stream.
constexpr int SEL_WIDE_MAX_Q = 4;  // up to this many queries use 11-bit digits
__host__ __device__ constexpr int select_hist_words(int n_queries) {
  return (n_queries <= SEL_WIDE_MAX_Q ? 2048 : 256) * n_queries;
}
__device__ __forceinline__ void select_prepare(SelectQuery* q, int n_queries, void* tmp) {
  for (int j = threadIdx.x; j < n_queries; j += blockDim.x) {
    q[j].prefix = 0u;
    q[j].result = 0xffffffffu;
  }
  uint32_t* hist = (uint32_t*)tmp;
  for (int i = threadIdx.x; i < select_hist_words(n_queries); i += blockDim.x) hist[i] = 0u;
}
void select_kth_prepared(const uint32_t* keys, const uint16_t* grp, int64_t n, SelectQuery* d_queries,
                         int n_queries, void* tmp, cudaStream_t s);

// select_kth_prepared whose first digit's histogram the kernel producing the
// keys has already counted into h0 (select_radix(n) words per query row, row q
// counting the items of query q's group at digit key >> select_first_shift(n)),
// so the select runs one histogram pass less.  h0 must be zero before that
// producer runs; the select leaves it zero again.  32-bit keys only.
__host__ __device__ constexpr int select_radix(int n_queries) { return n_queries <= SEL_WIDE_MAX_Q ? 2048 : 256; }
__host__ __device__ constexpr int select_first_shift(int n_queries) { return n_queries <= SEL_WIDE_MAX_Q ? 22 : 24; }
void select_kth_first(const uint32_t* keys, const uint16_t* grp, int64_t n, SelectQuery* d_queries, int n_queries,
                      uint32_t* h0, void* tmp, cudaStream_t s);

}  // namespace lv

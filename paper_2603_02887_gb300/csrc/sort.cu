// Device radix sort (stable LSD, 8-bit digits), exclusive scan of tile counts, and tile ranges.
//
// The sort works on `nseg` equal segments of seg_len items at once, each sorted on its own (the depth sort
// of a batch sorts every view's Gaussians in one launch per kernel). Each pass runs three kernels:
//   upsweep   per block of 1024 (or 4096) items of a segment: digit histogram -> hist[segment][digit][block]
//   scan      one block per (segment, digit): exclusive scan of that row in place, total -> totals
//   downsweep per block: stable rank of every item within the block (warp multi-split: the lanes with
//             the same digit from one ballot per digit bit; warps in order), reorder in shared memory so
//             that items of one digit are contiguous, then a coalesced scatter to
//             segment start + base(digit) + hist[segment][digit][block] + rank, base = exclusive scan of
//             the segment's digit totals.
// Stability (equal digits keep their input order) makes the LSD passes a correct sort, and it is what
// orders equal depths by Gaussian index (the pairs are emitted in index order within one depth).
// A count known only on the device (the number of pairs, inside a captured graph) is read by every
// kernel: blocks past it contribute empty histograms and move nothing.
#include "ngs_internal.cuh"

namespace ngs {
namespace {

// Exclusive prefix sum over a block (warp shuffles, then one warp scans the warp totals).
// `s_warp` needs THREADS/32 entries; all threads must call it. Returns the exclusive prefix of `v`;
// *total receives the block's sum.
template <int THREADS, typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* s_warp, T* total) {
  constexpr int NW = THREADS / 32;
  static_assert(NW <= 32, "block too large");
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < NW ? s_warp[lane] : (T)0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NW) s_warp[lane] = w;
  }
  __syncthreads();
  T prefix = warp > 0 ? s_warp[warp - 1] : (T)0;
  *total = s_warp[NW - 1];
  __syncthreads();
  return prefix + x - v;
}

constexpr int kThreads = 256;
// Items per thread: 4 (1024 per CTA) up to kSmallSort items per segment, where the passes are latency-bound
// and more CTAs hide more latency (a sweep of 4..16 on GB300 at 0.5-3.3 M items); 16 above it, where the
// per-digit scans over the CTAs' counts would otherwise grow long.
constexpr int kSmallSort = 1 << 23;
template <int ITEMS>
struct SortTile {
  static constexpr int kTile = kThreads * ITEMS;
};
__host__ __device__ constexpr int tile_items(uint32_t seg_len) { return seg_len <= (uint32_t)kSmallSort ? 1024 : 4096; }
constexpr int kWarps = kThreads / 32;
constexpr int kDigits = 256;

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift) {
  return (uint32_t)(key >> shift) & 0xFFu;
}

__device__ __forceinline__ uint32_t segment_count(uint32_t seg_len, const uint32_t* n_dev) {
  return n_dev ? min(*n_dev, seg_len) : seg_len;
}

template <typename K, int ITEMS>
__global__ void __launch_bounds__(kThreads) upsweep_kernel(const K* __restrict__ keys, uint32_t seg_len,
                                                           const uint32_t* __restrict__ n_dev, int shift,
                                                           uint32_t* __restrict__ hist, uint32_t nblocks) {
  pdl_wait();
  __shared__ uint32_t s_hist[kWarps][kDigits];
  int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t seg = blockIdx.x / nblocks, blk = blockIdx.x - seg * nblocks;
  const uint32_t n = segment_count(seg_len, n_dev);
  keys += (size_t)seg * seg_len;
  hist += (size_t)seg * kDigits * nblocks;
  for (int i = tid; i < kWarps * kDigits; i += kThreads) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  constexpr int kTile = SortTile<ITEMS>::kTile;
  uint32_t base = blk * (uint32_t)kTile;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    uint32_t idx = base + j * kThreads + tid;
    // a plain shared-memory atomic per item (measured on GB300: faster than aggregating the warp's equal
    // digits with __match_any_sync first, by 11 % on the depth sort and 18 % on the tile sort)
    if (idx < n) atomicAdd(&s_hist[warp][digit_of(keys[idx], shift)], 1u);
  }
  __syncthreads();
  for (int d = tid; d < kDigits; d += kThreads) {
    uint32_t sum = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) sum += s_hist[w][d];
    hist[(size_t)d * nblocks + blk] = sum;
  }
}

// One block per (segment, digit): exclusive scan of that digit's per-block counts; the digit's total goes
// to totals[segment][digit] (stored after the histograms).
__global__ void __launch_bounds__(1024) scan_digit_kernel(uint32_t* hist, uint32_t nblocks, uint32_t* totals) {
  pdl_wait();
  __shared__ uint32_t s_warp[32];
  uint32_t* row = hist + (size_t)blockIdx.x * nblocks;
  uint32_t carry = 0;
  for (uint32_t base = 0; base < nblocks; base += 1024) {
    uint32_t i = base + threadIdx.x;
    uint32_t v = i < nblocks ? row[i] : 0u, agg;
    uint32_t ex = block_exclusive_sum<1024>(v, s_warp, &agg);
    if (i < nblocks) row[i] = ex + carry;
    carry += agg;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

template <typename K, int ITEMS>
__global__ void __launch_bounds__(kThreads) downsweep_kernel(const K* __restrict__ keys_in,
                                                             const uint32_t* __restrict__ vals_in,
                                                             K* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                             uint32_t seg_len, const uint32_t* __restrict__ n_dev,
                                                             int shift, const uint32_t* __restrict__ hist,
                                                             const uint32_t* __restrict__ totals, uint32_t nblocks) {
  pdl_wait();
  constexpr int kTile = SortTile<ITEMS>::kTile, kItems = ITEMS;
  const uint32_t seg = blockIdx.x / nblocks, blk = blockIdx.x - seg * nblocks;
  const uint32_t n = segment_count(seg_len, n_dev);
  if (blk * (uint32_t)kTile >= n) return;  // the whole block is past the segment's items
  {
    const size_t off = (size_t)seg * seg_len;
    keys_in += off;
    vals_in += off;
    keys_out += off;
    vals_out += off;
    hist += (size_t)seg * kDigits * nblocks;
    totals += (size_t)seg * kDigits;
  }
  extern __shared__ __align__(16) unsigned char smem[];
  K* s_keys = reinterpret_cast<K*>(smem);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(smem + sizeof(K) * kTile);
  __shared__ uint32_t s_cnt[kWarps][kDigits];  // per-warp digit counters, then per-warp offsets
  __shared__ uint32_t s_local[kDigits];         // block-local start of each digit
  __shared__ uint32_t s_global[kDigits];        // global start of this block's run of each digit
  __shared__ uint32_t s_warp[kWarps];

  int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < kWarps * kDigits; i += kThreads) (&s_cnt[0][0])[i] = 0;
  __syncthreads();

  uint32_t base = blk * (uint32_t)kTile + warp * (kTile / kWarps);
  K key[kItems];
  uint32_t val[kItems], rank[kItems], dig[kItems];
  uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    uint32_t idx = base + r * 32 + lane;
    bool valid = idx < n;
    key[r] = valid ? keys_in[idx] : (K)0;
    val[r] = valid ? vals_in[idx] : 0u;
    uint32_t d = valid ? digit_of(key[r], shift) : (uint32_t)kDigits;  // kDigits = "no item"
    dig[r] = d;
    // lanes holding the same digit (0..255, or 256 for "no item"): one ballot per bit of d (measured on
    // GB300: 2-4 % faster sorts than __match_any_sync)
    uint32_t peers = 0xFFFFFFFFu;
#pragma unroll
    for (int bit = 0; bit < 9; ++bit) {
      const bool one = (d >> bit) & 1u;
      const uint32_t bal = __ballot_sync(0xFFFFFFFFu, one);
      peers &= one ? bal : ~bal;
    }
    uint32_t before = valid ? s_cnt[warp][d] : 0u;
    rank[r] = before + __popc(peers & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) s_cnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive offsets over warps, block total, block-local digit start, global start
  uint32_t total = 0;
  {
    int d = tid;  // kThreads == kDigits
    for (int w = 0; w < kWarps; ++w) {
      uint32_t c = s_cnt[w][d];
      s_cnt[w][d] = total;
      total += c;
    }
    uint32_t agg;
    s_local[d] = block_exclusive_sum<kThreads>(total, s_warp, &agg);
  }
  {
    // global digit base = exclusive scan of the digit totals; this block's run starts hist[d][b] into it
    uint32_t agg;
    uint32_t ex = block_exclusive_sum<kThreads>(totals[tid], s_warp, &agg);
    s_global[tid] = ex + hist[(size_t)tid * nblocks + blk];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    if (dig[r] < (uint32_t)kDigits) {
      uint32_t pos = s_local[dig[r]] + s_cnt[warp][dig[r]] + rank[r];
      s_keys[pos] = key[r];
      s_vals[pos] = val[r];
    }
  }
  __syncthreads();
  uint32_t count = min((uint32_t)kTile, n - blk * (uint32_t)kTile);
  for (uint32_t i = tid; i < count; i += kThreads) {
    K k = s_keys[i];
    uint32_t d = digit_of(k, shift);
    uint32_t g = s_global[d] + (i - s_local[d]);
    keys_out[g] = k;
    vals_out[g] = s_vals[i];
  }
}

template <typename K, int ITEMS>
int radix_sort(K* keys[2], uint32_t* vals[2], uint32_t seg_len, uint32_t nseg, const uint32_t* n_dev, int begin_bit,
               int end_bit, uint32_t* hist, cudaStream_t s, int* launches) {
  constexpr int kTile = SortTile<ITEMS>::kTile;
  int cur = 0;
  if (seg_len <= 1 || nseg == 0 || begin_bit >= end_bit) return cur;
  uint32_t nblocks = (seg_len + kTile - 1) / kTile;
  uint32_t grid = nblocks * nseg;
  uint32_t* totals = hist + (size_t)kDigits * nblocks * nseg;
  // at most 24 KB of dynamic shared memory (for 64-bit keys), within the default limit without an opt-in
  size_t smem = (sizeof(K) + sizeof(uint32_t)) * kTile;
  for (int shift = begin_bit; shift < end_bit; shift += 8) {
    launch_pdl(upsweep_kernel<K, ITEMS>, grid, kThreads, 0, s, keys[cur], seg_len, n_dev, shift, hist, nblocks);
    launch_pdl(scan_digit_kernel, kDigits * nseg, 1024, 0, s, hist, nblocks, totals);
    launch_pdl(downsweep_kernel<K, ITEMS>, grid, kThreads, smem, s, keys[cur], vals[cur], keys[cur ^ 1],
               vals[cur ^ 1], seg_len, n_dev, shift, hist, totals, nblocks);
    cur ^= 1;
    *launches += 3;
  }
  return cur;
}

// ---- exclusive scan of tile counts taken in depth order ---------------------------------------------

constexpr int kScanThreads = 512;
// Items per thread: 2 up to kScanSmall items, where the scan is a few hundred CTAs of gathers and more
// CTAs hide their latency; 8 above, which keeps the per-CTA sums that one CTA scans short.
constexpr uint32_t kScanSmall = 1u << 21;
constexpr int scan_items(uint32_t n) { return n <= kScanSmall ? 2 : 8; }

template <int kScanItems>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t* __restrict__ count,
                                                                   const uint32_t* __restrict__ order, uint32_t n,
                                                                   uint64_t* __restrict__ block_sums) {
  pdl_wait();
  __shared__ uint64_t s_warp[kScanThreads / 32];
  constexpr int kScanTile = kScanThreads * kScanItems;
  uint64_t sum = 0;
  uint32_t base = blockIdx.x * (uint32_t)kScanTile;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    uint32_t i = base + j * kScanThreads + threadIdx.x;
    if (i < n) sum += count[order[i]];
  }
  uint64_t agg;
  block_exclusive_sum<kScanThreads>(sum, s_warp, &agg);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = agg;
}

__global__ void __launch_bounds__(1024) scan_block_sums_kernel(uint64_t* block_sums, uint32_t nblocks, uint64_t* total) {
  pdl_wait();
  __shared__ uint64_t s_warp[32];
  uint64_t carry = 0;
  for (uint32_t base = 0; base < nblocks; base += 1024) {
    uint32_t i = base + threadIdx.x;
    uint64_t v = i < nblocks ? block_sums[i] : 0, agg;
    uint64_t ex = block_exclusive_sum<1024>(v, s_warp, &agg);
    if (i < nblocks) block_sums[i] = ex + carry;
    carry += agg;
  }
  if (threadIdx.x == 0) *total = carry;
}

template <int kScanItems>
__global__ void __launch_bounds__(kScanThreads) scan_final_kernel(const uint32_t* __restrict__ count,
                                                                  const uint32_t* __restrict__ order, uint32_t n,
                                                                  const uint64_t* __restrict__ block_offsets,
                                                                  uint32_t* __restrict__ offsets) {
  pdl_wait();
  constexpr int kScanTile = kScanThreads * kScanItems;
  __shared__ uint32_t s_warp[kScanThreads / 32];
  uint32_t base = blockIdx.x * (uint32_t)kScanTile + threadIdx.x * kScanItems;  // blocked arrangement
  uint32_t v[kScanItems], local = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    uint32_t i = base + j;
    v[j] = i < n ? count[order[i]] : 0u;
    local += v[j];
  }
  uint32_t agg;
  uint32_t run = (uint32_t)block_offsets[blockIdx.x] + block_exclusive_sum<kScanThreads>(local, s_warp, &agg);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    uint32_t i = base + j;
    if (i < n) offsets[i] = run;
    run += v[j];
    if (i == n - 1) offsets[n] = run;
  }
}

// Global tile of pair i: the view's first tile plus the view-local tile it was sorted by.
__device__ __forceinline__ uint32_t global_tile(const uint32_t* __restrict__ tiles, const uint32_t* __restrict__ vals,
                                                const ViewParams* __restrict__ views, uint32_t n_per_view,
                                                uint32_t n_views, uint32_t i) {
  return n_views == 1 ? tiles[i] : __ldg(&views[vals[i] / n_per_view].tile_base) + tiles[i];
}

__global__ void tile_ranges_kernel(const uint32_t* __restrict__ tiles, const uint32_t* __restrict__ vals,
                                   const ViewParams* __restrict__ views, uint32_t n_per_view, uint32_t n_views,
                                   uint32_t npairs_cap, const uint32_t* __restrict__ npairs_dev, uint32_t ntiles,
                                   uint2* __restrict__ ranges, uint32_t* check) {
  pdl_wait();
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t npairs = npairs_dev ? min(*npairs_dev, npairs_cap) : npairs_cap;
  if (i >= npairs) return;
  if (n_views == 1) {
    const uint32_t t = tiles[i];
    if (t >= ntiles) {  // never from a correct sort: skipped and reported
      atomicOr(check, kCheckTile);
      return;
    }
    if (i == 0 || tiles[i - 1] != t) ranges[t].x = i;
    if (i == npairs - 1 || tiles[i + 1] != t) ranges[t].y = i + 1;
    return;
  }
  // a batch: a run is a (view-local tile, view) pair, compared without the view table; only the first and
  // last pair of a run look up the view's first tile
  const uint32_t n_records = n_per_view * n_views;
  const uint32_t v = vals[i];
  if (v >= n_records) {  // never from a correct sort: skipped and reported (the compositing checks it too)
    atomicOr(check, kCheckIndex);
    return;
  }
  const uint32_t loc = tiles[i], view = v / n_per_view;
  auto same = [&](uint32_t j) { return tiles[j] == loc && vals[j] / n_per_view == view; };
  const bool first = i == 0 || !same(i - 1), last = i == npairs - 1 || !same(i + 1);
  if (!(first || last)) return;
  const uint32_t t = __ldg(&views[view].tile_base) + loc;
  if (t >= ntiles) {
    atomicOr(check, kCheckTile);
    return;
  }
  if (first) ranges[t].x = i;
  if (last) ranges[t].y = i + 1;
}

__global__ void compose_keys_kernel(const uint32_t* __restrict__ tiles, const uint32_t* __restrict__ vals,
                                    const float4* __restrict__ rec, const ViewParams* __restrict__ views,
                                    uint32_t n_per_view, uint32_t n_views, uint32_t npairs,
                                    uint64_t* __restrict__ keys) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npairs) return;
  const float z = rec[3 * (size_t)vals[i] + 2].y;
  const uint32_t t = global_tile(tiles, vals, views, n_per_view, n_views, i);
  keys[i] = ((uint64_t)t << 32) | (uint64_t)__float_as_uint(z);
}

// ---- tile work order for the persistent composite: descending pair count ---------------------------

__device__ __forceinline__ uint32_t cost_bucket(uint2 r) {
  const uint32_t c = r.y - r.x;
  return (uint32_t)(kCostBuckets - 1) - (c ? 32u - (uint32_t)__clz(c) : 0u);  // 0 = most pairs
}

__global__ void __launch_bounds__(256) tile_bucket_count_kernel(const uint2* __restrict__ ranges, uint32_t ntiles,
                                                                uint32_t* __restrict__ counts) {
  pdl_wait();
  __shared__ uint32_t s_cnt[kCostBuckets];
  if (threadIdx.x < kCostBuckets) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ntiles) atomicAdd(&s_cnt[cost_bucket(ranges[t])], 1u);
  __syncthreads();
  if (threadIdx.x < kCostBuckets && s_cnt[threadIdx.x]) atomicAdd(&counts[threadIdx.x], s_cnt[threadIdx.x]);
}

__global__ void __launch_bounds__(256) tile_bucket_scatter_kernel(const uint2* __restrict__ ranges, uint32_t ntiles,
                                                                  const uint32_t* __restrict__ counts,
                                                                  uint32_t* __restrict__ cursors,
                                                                  uint32_t* __restrict__ work) {
  pdl_wait();
  __shared__ uint32_t s_start[kCostBuckets];
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int b = 0; b < kCostBuckets; ++b) {
      s_start[b] = run;
      run += counts[b];
    }
  }
  __syncthreads();
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t b = t < ntiles ? cost_bucket(ranges[t]) : (uint32_t)kCostBuckets;
  const uint32_t peers = __match_any_sync(0xFFFFFFFFu, b);
  const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (b < (uint32_t)kCostBuckets && lane == leader) base = atomicAdd(&cursors[b], (uint32_t)__popc(peers));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (b < (uint32_t)kCostBuckets) work[s_start[b] + base + __popc(peers & ((1u << lane) - 1u))] = t;
}

}  // namespace

void launch_tile_order(const uint2* ranges, uint32_t ntiles, uint32_t* sched, uint32_t* work, cudaStream_t s,
                       int* launches) {
  if (ntiles == 0) return;
  const unsigned blocks = (ntiles + 255) / 256;
  launch_pdl(tile_bucket_count_kernel, blocks, 256, 0, s, ranges, ntiles, sched + 2);
  launch_pdl(tile_bucket_scatter_kernel, blocks, 256, 0, s, ranges, ntiles, sched + 2, sched + 2 + kCostBuckets, work);
  *launches += 2;
}

size_t radix_hist_words(uint32_t seg_len, uint32_t nseg) {
  const uint32_t tile = (uint32_t)tile_items(seg_len);
  uint32_t nblocks = (seg_len + tile - 1) / tile;
  return (size_t)kDigits * (nblocks + 1) * nseg;
}

int radix_sort_u32(uint32_t* keys[2], uint32_t* vals[2], uint32_t seg_len, uint32_t nseg, const uint32_t* n_dev,
                   int begin_bit, int end_bit, uint32_t* hist, cudaStream_t s, int* launches) {
  if (tile_items(seg_len) == SortTile<4>::kTile)
    return radix_sort<uint32_t, 4>(keys, vals, seg_len, nseg, n_dev, begin_bit, end_bit, hist, s, launches);
  return radix_sort<uint32_t, 16>(keys, vals, seg_len, nseg, n_dev, begin_bit, end_bit, hist, s, launches);
}



size_t scan_tmp_words(uint32_t n) {
  const uint32_t tile = (uint32_t)(kScanThreads * scan_items(n));
  return (size_t)(n + tile - 1) / tile + 1;
}

cudaError_t launch_scan_counts(const uint32_t* tile_count, const uint32_t* order, uint32_t n, uint32_t* offsets,
                               uint64_t* block_sums, uint64_t* total, cudaStream_t s, int* launches) {
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(offsets, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
    return e;
  }
  const int items = scan_items(n);
  const uint32_t tile = (uint32_t)(kScanThreads * items);
  const uint32_t nblocks = (n + tile - 1) / tile;
  if (items == 2) launch_pdl(scan_reduce_kernel<2>, nblocks, kScanThreads, 0, s, tile_count, order, n, block_sums);
  else launch_pdl(scan_reduce_kernel<8>, nblocks, kScanThreads, 0, s, tile_count, order, n, block_sums);
  launch_pdl(scan_block_sums_kernel, 1, 1024, 0, s, block_sums, nblocks, total);
  if (items == 2)
    launch_pdl(scan_final_kernel<2>, nblocks, kScanThreads, 0, s, tile_count, order, n, block_sums, offsets);
  else
    launch_pdl(scan_final_kernel<8>, nblocks, kScanThreads, 0, s, tile_count, order, n, block_sums, offsets);
  *launches += 3;
  return cudaSuccess;
}

void launch_tile_ranges(const uint32_t* tiles, const uint32_t* vals, const ViewParams* views, uint32_t n_per_view,
                        uint32_t n_views, uint32_t npairs_cap, const uint32_t* npairs_dev, uint32_t ntiles,
                        uint2* ranges, uint32_t* check, cudaStream_t s) {
  if (npairs_cap == 0) return;
  launch_pdl(tile_ranges_kernel, (npairs_cap + 255) / 256, 256, 0, s, tiles, vals, views, n_per_view, n_views,
             npairs_cap, npairs_dev, ntiles, ranges, check);
}

void launch_compose_keys(const uint32_t* tiles, const uint32_t* vals, const float4* rec, const ViewParams* views,
                         uint32_t n_per_view, uint32_t n_views, uint32_t npairs, uint64_t* keys, cudaStream_t s) {
  if (npairs == 0) return;
  compose_keys_kernel<<<(npairs + 255) / 256, 256, 0, s>>>(tiles, vals, rec, views, n_per_view, n_views, npairs,
                                                           keys);
}

}  // namespace ngs

// Tile keys and depth sort: per image tile, the list of intersecting splats
// in (depth, index) order, with CUB-free onesweep radix passes.
//
// Paper: arXiv 2606.11390 §4 (each camera's Gaussians are depth-sorted before
// rasterisation; the multi-GPU merge sort of §4 is not needed on one GPU) and
// §3.2 (the paper sorts with CUB's radix sort, Merrill & Grimshaw 2011). The
// digit passes follow the onesweep scheme (Adinets & Merrill 2022): digit
// histograms of all passes are gathered up front, and each pass reads and
// writes the data once, every tile of 4096 items finding its global digit
// offsets by decoupled look-back over its predecessors. Tiles take their
// order from an atomic ticket, so a tile only waits on tiles that are already
// running, and every wait is bounded (GS_STATUS_TIMEOUT).
//
// The sorted order is that of the stable sort of the 64-bit keys
// (tile << 32) | bits(depth) emitted in (view, Gaussian, row-major tile)
// order. It is reached in three steps:
//   1. compact the visible records and sort them by depth bits (4 passes over
//      32-bit keys; stability keeps equal depths in record-index order);
//   2. bin the records, in depth order, into super-tiles of 8 x 8 tiles (one
//      entry per super-tile a rectangle meets, about 1.3 per record) and sort
//      the entries stably by super-tile id (1-2 passes);
//   3. per chunk of 256 records of a super-tile's list, place each record in
//      the lists of the tiles it covers: a 64-bit coverage mask per record,
//      one warp ballot per tile for the ranks, per-chunk tile counts scanned
//      over the super-tile's chunks and over all tiles; every intersection is
//      written once, at its final position.
// Within a tile the entries then run in (depth, record) order, exactly the
// order of the 64-bit key sort, while the large list (one entry per tile
// intersection) is written once, 4 bytes per entry, instead of going through
// 64-bit key passes.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagIncl = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;
constexpr int kRadix = 256;
constexpr int kDepthPasses = 4;
// Wait bound used with GS_FLAG_TEST_STALL_LOOKBACK (milliseconds, not seconds).
constexpr uint32_t kTestSpinLimit = 1u << 12;

__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Decoupled look-back for scan tile `t` (t >= 1), run by one full warp;
// returns the exclusive prefix of the tile.
__device__ uint64_t lookback_warp(const uint64_t* tiles, uint32_t t, int32_t* status) {
  const int lane = threadIdx.x & 31;
  uint64_t prefix = 0;
  int64_t base = static_cast<int64_t>(t) - 1;
  uint32_t spins = 0;
  while (base >= 0) {
    const int64_t j = base - lane;
    uint64_t s = j >= 0 ? ld_relaxed_u64(tiles + j) : kFlagIncl;
    while (__any_sync(0xffffffffu, (s >> 62) == 0)) {
      if (++spins > kSpinLimit) {
        set_status(status, GS_STATUS_TIMEOUT);
        return prefix;
      }
      if ((s >> 62) == 0) s = ld_relaxed_u64(tiles + j);
    }
    const uint32_t incl = __ballot_sync(0xffffffffu, (s >> 62) == 2);
    const int stop = incl ? (__ffs(incl) - 1) : 31;
    uint64_t v = lane <= stop ? (s & kValMask) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    prefix += v;
    if (incl) break;
    base -= 32;
  }
  return prefix;
}

// Block-wide exclusive scan (256 threads) of one u64 per thread; also
// publishes the block total through decoupled look-back and returns the
// block's global exclusive prefix in *block_prefix.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

struct ScanState {
  uint64_t* tiles;   // [n_scan_tiles] flag | value
  uint32_t* ticket;  // [1]
};

__device__ __forceinline__ uint64_t block_scan_lookback(uint64_t local, uint32_t t, const ScanState& st,
                                                        uint64_t* s_warp, uint64_t* s_prefix, int32_t* status) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t incl = warp_incl_scan_u64(local);
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
    w = warp_incl_scan_u64(w);
    if (lane < kScanThreads / 32) s_warp[lane] = w;
  }
  __syncthreads();
  const uint64_t block_total = s_warp[kScanThreads / 32 - 1];
  const uint64_t excl_thread = incl - local + (warp > 0 ? s_warp[warp - 1] : 0);
  if (warp == 0) {
    if (t == 0) {
      if (lane == 0) {
        st_relaxed_u64(st.tiles, kFlagIncl | block_total);
        *s_prefix = 0;
      }
    } else {
      if (lane == 0) st_relaxed_u64(st.tiles + t, kFlagAgg | block_total);
      const uint64_t p = lookback_warp(st.tiles, t, status);
      if (lane == 0) {
        st_relaxed_u64(st.tiles + t, kFlagIncl | (p + block_total));
        *s_prefix = p;
      }
    }
  }
  __syncthreads();
  return *s_prefix + excl_thread;
}

// ---------------------------------------------------------------------------
// 1a. Compaction of visible records: (depth bits, record) pairs in record
//     order, plus the digit histograms of the four depth passes.
// ---------------------------------------------------------------------------
// With depth_keys (float bits of each record's depth, 0 for a culled record,
// as gs_project writes them) the kernel reads 4 coalesced bytes per record;
// without, the tile counts and a gather of the depth from each 48-byte
// projected record. Items are striped (item i of thread (warp, lane) is
// record i * 256 + warp * 32 + lane of the tile), so a warp reads 32
// consecutive records and writes its visible ones to consecutive positions:
// the position is the tile's prefix, plus the visible counts of the (item,
// warp) groups before it in record order, plus the lane's rank in its
// group's ballot. The two high depth digits take few distinct values (the
// exponent byte of a positive float is nearly constant over a scene), so
// their histogram updates are aggregated per warp (one atomic per distinct
// digit); the two low digits are spread and take one atomic per record.
__global__ void __launch_bounds__(kScanThreads) compact_visible_kernel(
    const uint32_t* __restrict__ counts, const float* __restrict__ projected, const uint32_t* __restrict__ depth_keys,
    int64_t n, uint32_t index_base, ScanState st, uint32_t* __restrict__ dkeys, uint32_t* __restrict__ dvals,
    uint32_t* __restrict__ hist, int64_t* n_visible, int32_t* status) {
  constexpr int kWarps = kScanThreads / 32;
  static_assert(kScanItems <= 32 && (kScanItems * kWarps) % 32 == 0, "item bits in one word; offsets split over a warp");
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_warp[kWarps];
  __shared__ uint64_t s_prefix;
  __shared__ uint32_t s_off[kScanItems * kWarps];  // visible count, then exclusive offset, of each (item, warp)
  __shared__ uint32_t s_total;
  __shared__ uint32_t s_hist[kDepthPasses][kRadix];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < kDepthPasses * kRadix; i += kScanThreads) (&s_hist[0][0])[i] = 0;
  if (tid == 0) s_tile = atomicAdd(st.ticket, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const int64_t base = static_cast<int64_t>(t) * kScanTile + warp * 32 + lane;  // item i: base + i * kScanThreads
  uint32_t vis = 0;  // bit i: item i visible
  uint32_t dkey[kScanItems];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t r = base + static_cast<int64_t>(i) * kScanThreads;
    bool v;
    if (depth_keys) {
      dkey[i] = r < n ? depth_keys[r] : 0u;
      v = dkey[i] != 0u;
    } else {
      dkey[i] = 0u;
      v = r < n && counts[r] > 0;
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, v);
    if (v) vis |= 1u << i;
    if (lane == 0) s_off[i * kWarps + warp] = __popc(bal);
  }
  // the tile's global prefix (in s_prefix; the thread-order offset is unused)
  (void)block_scan_lookback(__popc(vis), t, st, s_warp, &s_prefix, status);
  if (warp == 0) {
    // exclusive scan of the (item, warp) counts in record order
    constexpr int kPer = kScanItems * kWarps / 32;
    uint32_t c[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      c[k] = s_off[lane * kPer + k];
      sum += c[k];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t nb = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += nb;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      s_off[lane * kPer + k] = run;
      run += c[k];
    }
    if (lane == 31) s_total = incl;
  }
  __syncthreads();
  const uint64_t tile_prefix = s_prefix;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint32_t bal = __ballot_sync(0xffffffffu, (vis >> i) & 1u);
    if ((vis >> i) & 1u) {
      const int64_t r = base + static_cast<int64_t>(i) * kScanThreads;
      const uint32_t d = depth_keys ? dkey[i] : __float_as_uint(projected[r * kRecordFloats + 6]);
      const uint64_t pos = tile_prefix + s_off[i * kWarps + warp] + __popc(bal & lt);
      dkeys[pos] = d;
      dvals[pos] = index_base + static_cast<uint32_t>(r);
      atomicAdd(&s_hist[0][d & 0xffu], 1u);
      atomicAdd(&s_hist[1][(d >> 8) & 0xffu], 1u);
#pragma unroll
      for (int p = 2; p < kDepthPasses; ++p) {
        const uint32_t dp = (d >> (8 * p)) & 0xffu;
        const uint32_t peers = __match_any_sync(bal, dp);
        if (lane == __ffs(peers) - 1) atomicAdd(&s_hist[p][dp], static_cast<uint32_t>(__popc(peers)));
      }
    }
  }
  const int64_t tile_start = static_cast<int64_t>(t) * kScanTile;
  if (tid == 0 && n > 0 && tile_start <= n - 1 && n - 1 < tile_start + kScanTile)
    *n_visible = static_cast<int64_t>(tile_prefix + s_total);
  __syncthreads();
  for (int i = tid; i < kDepthPasses * kRadix; i += kScanThreads) {
    const uint32_t c = (&s_hist[0][0])[i];
    if (c) atomicAdd(hist + i, c);
  }
}

// Exclusive scan of each pass's 256 digit counts, in place (one block of 256).
__global__ void hist_scan_kernel(uint32_t* hist, int passes) {
  const int d = threadIdx.x, lane = d & 31, warp = d >> 5;
  __shared__ uint32_t s_w[kRadix / 32];
  for (int p = 0; p < passes; ++p) {
    const uint32_t c = hist[p * kRadix + d];
    uint32_t v = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t nb = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += nb;
    }
    if (lane == 31) s_w[warp] = v;
    __syncthreads();
    uint32_t add = 0;
    for (int w = 0; w < warp; ++w) add += s_w[w];
    hist[p * kRadix + d] = v - c + add;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Onesweep digit pass over (u32 key, u32 value) pairs.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
// Items per thread of a digit pass (tile = 256 x items).
#ifndef GS_SORT_ITEMS
#define GS_SORT_ITEMS 16
#endif
constexpr int kSortItems = GS_SORT_ITEMS;
// CTAs per SM the digit pass is compiled for (caps registers at 65536 / (256 x this)).
#ifndef GS_SORT_MIN_BLOCKS
#define GS_SORT_MIN_BLOCKS 4
#endif
constexpr int kSortTile = kSortThreads * kSortItems;
static_assert(32 * kSortItems <= 1024, "a within-warp rank must fit the 10 bits it is packed in");

struct PassArgs {
  const uint32_t* keys_in;
  const uint32_t* vals_in;
  uint32_t* keys_out;  // may be null: the keys are not written
  uint32_t* vals_out;
  uint2* ranges;             // last pass: per-key (~first, last + 1) bounds, else null
  uint32_t n_keys;           // ranges has n_keys entries
  uint32_t key_mask;         // the bits of a key that name its range (others ride along unsorted)
  const int64_t* n_total;   // items = min(*n_total, cap)
  int64_t cap;
  int shift;
  const uint32_t* digit_offsets;  // [256]: exclusive offsets, or the digit counts when scan_digits
  int scan_digits;                // 1: each CTA scans the counts into offsets itself
  uint32_t* ticket;
  uint64_t* lookback;  // [sort tiles][256]
  int32_t stall_tile;   // test hook: this tile never publishes (-1: none)
  uint32_t spin_limit;  // bound on each look-back wait
};

struct __align__(16) SortSmem {
  uint32_t keys[kSortTile];                // 16 KB
  uint32_t vals[kSortTile];                // 16 KB
  uint32_t warp_hist[kSortWarps][kRadix];  // 8 KB
  uint32_t local_start[kRadix];
  uint32_t base[kRadix];  // output position of local index 0 of each digit, modulo 2^32
  uint32_t wsum[kSortWarps];
  uint32_t doff[kRadix];  // exclusive output offset of each digit
  uint32_t tile;
};

// BITS: significant bits of this pass's digit (the last tile-id pass may
// need fewer than 8; the higher digit bits are zero for every item there, so
// their ballots would change nothing).
template <int BITS>
__global__ void __launch_bounds__(kSortThreads, GS_SORT_MIN_BLOCKS) sort_pass_kernel(PassArgs a, int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem& sm = *reinterpret_cast<SortSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int64_t n = *a.n_total;
  if (n > a.cap) n = a.cap;
  {
    // the pass's digit offsets: given, or the exclusive scan of the digit
    // counts (every CTA scans the 256 counts itself: no separate launch)
    uint32_t c = a.digit_offsets[tid];  // kSortThreads == kRadix
    if (a.scan_digits) {
      uint32_t v = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t nb = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += nb;
      }
      if (lane == 31) sm.wsum[warp] = v;
      __syncthreads();
      uint32_t add = 0;
      for (int w = 0; w < warp; ++w) add += sm.wsum[w];
      c = v - c + add;
    }
    sm.doff[tid] = c;  // read after the loop's first barrier
  }
  // Persistent CTA: take tiles in ticket order until the data is exhausted.
  // A tile only waits on tiles with smaller tickets, all held by running CTAs.
  for (;;) {
  if (tid == 0) sm.tile = atomicAdd(a.ticket, 1u);
  for (int i = tid; i < kSortWarps * kRadix; i += kSortThreads) (&sm.warp_hist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t t = sm.tile;
  const int64_t tile_start = static_cast<int64_t>(t) * kSortTile;
  if (tile_start >= n) return;  // past the data: publishes nothing, awaited by nobody
  const int n_valid = static_cast<int>(n - tile_start < kSortTile ? n - tile_start : kSortTile);
  if (tid == 0) {
    // the tile one grid ahead (taken by some CTA about one round later): into L2 now
    const int64_t pf_start = tile_start + static_cast<int64_t>(gridDim.x) * kSortTile;
    if (pf_start < n) {
      const int64_t items = n - pf_start < kSortTile ? n - pf_start : kSortTile;
      const uint32_t bytes = static_cast<uint32_t>(items * 4) & ~15u;
      const uint32_t* kp = a.keys_in + pf_start;
      const uint32_t* vp = a.vals_in + pf_start;
      if (bytes && !(reinterpret_cast<uintptr_t>(kp) & 15u) && !(reinterpret_cast<uintptr_t>(vp) & 15u)) {
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(kp), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(vp), "r"(bytes) : "memory");
      }
    }
  }

  // 1. load everything first (warp-striped), so the loads overlap
  uint32_t key[kSortItems], val[kSortItems];
  const int warp_base = warp * 32 * kSortItems;
  const uint32_t* kin = a.keys_in + tile_start + warp_base + lane;
  const uint32_t* vin = a.vals_in + tile_start + warp_base + lane;
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const bool ok = warp_base + i * 32 + lane < n_valid;
    key[i] = ok ? kin[i * 32] : 0u;
    val[i] = ok ? vin[i * 32] : 0u;
  }
  // 2. stable rank within the warp, item by item: the lanes holding the same
  //    digit are found with one ballot per digit bit (cheaper than match_any)
  uint32_t rpk[(kSortItems + 2) / 3];  // ranks (< 32 x items <= 1024), 10 bits each, 3 per register
#pragma unroll
  for (int i = 0; i < (kSortItems + 2) / 3; ++i) rpk[i] = 0u;
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int li = warp_base + i * 32 + lane;
    const bool valid = li < n_valid;
    const uint32_t d = (key[i] >> a.shift) & 0xffu;
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int bit = 0; bit < BITS; ++bit) {
      const uint32_t bal = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
      peers &= bal ^ (((d >> bit) & 1u) - 1u);  // bal where the bit is set, ~bal where not
    }
    // Every lane of a digit group reads the group's running count (a
    // broadcast) and writes the same new value: no leader, no divergence.
    const uint32_t before = sm.warp_hist[warp][d];
    rpk[i / 3] |= (before + __popc(peers & lt_mask)) << (10 * (i % 3));
    __syncwarp();
    if (valid) sm.warp_hist[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // 3. per digit: warp offsets, tile total, publish, local start, look-back
  const int d = tid;  // kSortThreads == kRadix
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const uint32_t c = sm.warp_hist[w][d];
    sm.warp_hist[w][d] = total;
    total += c;
  }
  uint64_t* lb = a.lookback;
  const bool publish = static_cast<int32_t>(t) != a.stall_tile;
  if (publish) st_relaxed_u64(lb + static_cast<int64_t>(t) * kRadix + d, (t == 0 ? kFlagIncl : kFlagAgg) | total);
  {
    uint32_t v = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t nb = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += nb;
    }
    if (lane == 31) sm.wsum[warp] = v;
    __syncthreads();
    uint32_t add = 0;
    for (int w = 0; w < warp; ++w) add += sm.wsum[w];
    sm.local_start[d] = v - total + add;
  }
  uint64_t prefix = 0;
  if (t > 0) {
    int64_t j = static_cast<int64_t>(t) - 1;
    uint32_t spins = 0;
    while (j >= 0) {
      const uint64_t s = ld_relaxed_u64(lb + j * kRadix + d);
      const uint64_t f = s >> 62;
      if (f == 0) {
        if (++spins > a.spin_limit) {
          set_status(status, GS_STATUS_TIMEOUT);
          break;
        }
        continue;
      }
      prefix += s & kValMask;
      if (f == 2) break;
      --j;
    }
    if (publish) st_relaxed_u64(lb + static_cast<int64_t>(t) * kRadix + d, kFlagIncl | (prefix + total));
  }
  sm.base[d] = sm.doff[d] + static_cast<uint32_t>(prefix) - sm.local_start[d];
  __syncthreads();

  // 4. scatter into shared memory in local sorted order
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int li = warp_base + i * 32 + lane;
    if (li < n_valid) {
      const uint32_t dd = (key[i] >> a.shift) & 0xffu;
      const uint32_t p = sm.local_start[dd] + sm.warp_hist[warp][dd] + ((rpk[i / 3] >> (10 * (i % 3))) & 0x3ffu);
      sm.keys[p] = key[i];
      sm.vals[p] = val[i];
    }
  }
  __syncthreads();

  // 5. write out: runs of equal digits land contiguously
  // (positions are below n < 2^32 - 1, so 32-bit wrapping arithmetic is exact)
  const uint32_t n32 = static_cast<uint32_t>(n);
  for (int idx = tid; idx < n_valid; idx += kSortThreads) {
    const uint32_t k = sm.keys[idx];
    const uint32_t p = sm.base[(k >> a.shift) & 0xffu] + static_cast<uint32_t>(idx);
    if (p < n32) {
      if (a.keys_out) a.keys_out[p] = k;
      a.vals_out[p] = sm.vals[idx];
      if (a.ranges) {
        // Last pass: the input is sorted by the lower digits, so a key's
        // items are contiguous in this tile's local order, and the key's
        // runs from successive tiles are adjacent in the output. The run's
        // first and last items bound the key's range: the start kept as
        // ~position under atomicMax (zero-initialised), the end as
        // position + 1.
        const uint32_t kk = k & a.key_mask;
        if (kk < a.n_keys) {
          if (idx == 0 || (sm.keys[idx - 1] & a.key_mask) != kk) atomicMax(&a.ranges[kk].x, ~p);
          if (idx == n_valid - 1 || (sm.keys[idx + 1] & a.key_mask) != kk) atomicMax(&a.ranges[kk].y, p + 1);
        } else {
          set_status(status, GS_STATUS_BOUNDS);
        }
      }
    } else {
      set_status(status, GS_STATUS_BOUNDS);
    }
  }
  __syncthreads();  // shared memory is reused by the next tile
  }
}

// ---------------------------------------------------------------------------
// Tile scheduling order: tile ids by decreasing list length, counting-sorted
// into half-octave buckets (one CTA; order within a bucket is arbitrary).
// ---------------------------------------------------------------------------
constexpr int kOrderThreads = 1024;
constexpr int kOrderBuckets = 64;

__device__ __forceinline__ int order_bucket(uint32_t len) {
  if (len == 0) return kOrderBuckets - 1;  // empty tiles last
  const int lg2 = 31 - __clz(len);                            // floor(log2 len)
  const int half = (len >> (lg2 > 0 ? lg2 - 1 : 0)) & 1;     // upper half of the octave
  const int b = 2 * lg2 + (lg2 > 0 ? half : 0);              // 0 .. 63, increasing with len
  return kOrderBuckets - 2 - (b < kOrderBuckets - 2 ? b : kOrderBuckets - 2);
}

__global__ void __launch_bounds__(kOrderThreads) tile_order_kernel(const uint2* __restrict__ ranges, int64_t n_tiles,
                                                                   uint32_t* __restrict__ order) {
  __shared__ uint32_t s_cnt[kOrderBuckets];
  const int tid = threadIdx.x;
  if (tid < kOrderBuckets) s_cnt[tid] = 0;
  __syncthreads();
  for (int64_t t = tid; t < n_tiles; t += kOrderThreads) {
    const uint2 r = ranges[t];
    atomicAdd(&s_cnt[order_bucket(r.y - r.x)], 1u);
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t run = 0;
    for (int b = 0; b < kOrderBuckets; ++b) {
      const uint32_t c = s_cnt[b];
      s_cnt[b] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int64_t t = tid; t < n_tiles; t += kOrderThreads) {
    const uint2 r = ranges[t];
    order[atomicAdd(&s_cnt[order_bucket(r.y - r.x)], 1u)] = static_cast<uint32_t>(t);
  }
}

// ---------------------------------------------------------------------------
// Merge of sorted partitions (the emulated multi-partition depth sort).
//
// The paper (§4) sorts a camera's Gaussians across devices by sorting each
// device's shard locally and combining the sorted shards in a log2(P)-level
// merge tree, every pair of partitions locating the split of each output
// range with a merge-path binary search (Green et al. 2012), so no partition
// has to gather all the data. Here the P partitions are record ranges of one
// GPU: each is compacted and depth-sorted on its own (4 digit passes), then
// every merge level is one launch in which each CTA owns 2048 consecutive
// outputs of one pair of runs, finds where its output range starts and ends
// in the two inputs by binary search, stages both input pieces in shared
// memory and merges them, each thread producing 8 outputs from its own
// merge-path split. Ties take the left run first, and runs hold increasing
// record ranges, so the result equals the stable depth sort of all records.
// ---------------------------------------------------------------------------
constexpr int kMergeThreads = 256;
constexpr int kMergeItems = 8;
constexpr int kMergeTile = kMergeThreads * kMergeItems;

struct MergeArgs {
  const uint32_t* keys_in;
  const uint32_t* vals_in;
  uint32_t* keys_out;
  uint32_t* vals_out;
  const int64_t* part_n;    // [P] sorted items per partition
  int64_t stride;           // partition p's items start at p * stride
  int level;                // inputs are runs of 2^level partitions
  int64_t ctas_per_pair;
  int64_t* n_total;         // written by the last level (one pair)
};

// Number of elements of a taken among the first d outputs (a first on ties).
__device__ __forceinline__ int64_t merge_path_split(const uint32_t* a, int64_t na, const uint32_t* b, int64_t nb,
                                                    int64_t d) {
  int64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] <= b[d - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kMergeThreads) merge_runs_kernel(MergeArgs m) {
  __shared__ uint32_t s_keys[kMergeTile];
  __shared__ uint32_t s_vals[kMergeTile];
  __shared__ int64_t s_split[2];
  const int tid = threadIdx.x;
  const int64_t pair = blockIdx.x / m.ctas_per_pair;
  const int64_t c = blockIdx.x - pair * m.ctas_per_pair;
  const int span = 1 << m.level;
  const int pa = static_cast<int>(2 * pair) * span, pb = pa + span;
  int64_t na = 0, nb = 0;
  for (int q = 0; q < span; ++q) {
    na += m.part_n[pa + q];
    nb += m.part_n[pb + q];
  }
  const int64_t n = na + nb;
  if (c == 0 && tid == 0 && m.n_total) *m.n_total = n;
  const int64_t d0 = c * kMergeTile;
  if (d0 >= n) return;
  const int64_t d1 = d0 + kMergeTile < n ? d0 + kMergeTile : n;
  const uint32_t* ak = m.keys_in + pa * m.stride;
  const uint32_t* bk = m.keys_in + pb * m.stride;
  const uint32_t* av = m.vals_in + pa * m.stride;
  const uint32_t* bv = m.vals_in + pb * m.stride;
  if (tid < 2) s_split[tid] = merge_path_split(ak, na, bk, nb, tid == 0 ? d0 : d1);
  __syncthreads();
  const int64_t a0 = s_split[0], a1 = s_split[1];
  const int64_t b0 = d0 - a0, b1 = d1 - a1;
  const int la = static_cast<int>(a1 - a0), lb = static_cast<int>(b1 - b0);
  for (int i = tid; i < la; i += kMergeThreads) {
    s_keys[i] = ak[a0 + i];
    s_vals[i] = av[a0 + i];
  }
  for (int i = tid; i < lb; i += kMergeThreads) {
    s_keys[la + i] = bk[b0 + i];
    s_vals[la + i] = bv[b0 + i];
  }
  __syncthreads();
  // this thread's 8 outputs
  const int len = la + lb;
  const int dl = tid * kMergeItems;
  uint32_t ok[kMergeItems], ov[kMergeItems];
  int cnt = 0;
  if (dl < len) {
    int lo = dl > lb ? dl - lb : 0, hi = dl < la ? dl : la;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (s_keys[mid] <= s_keys[la + dl - 1 - mid]) lo = mid + 1;
      else hi = mid;
    }
    int ai = lo, bi = dl - lo;
#pragma unroll
    for (int i = 0; i < kMergeItems; ++i) {
      if (dl + i < len) {
        const bool take_a = ai < la && (bi >= lb || s_keys[ai] <= s_keys[la + bi]);
        const int src = take_a ? ai : la + bi;
        ok[i] = s_keys[src];
        ov[i] = s_vals[src];
        ai += take_a ? 1 : 0;
        bi += take_a ? 0 : 1;
        ++cnt;
      }
    }
  }
  __syncthreads();  // all reads of the staged inputs are done
#pragma unroll
  for (int i = 0; i < kMergeItems; ++i) {
    if (i < cnt) {
      s_keys[dl + i] = ok[i];
      s_vals[dl + i] = ov[i];
    }
  }
  __syncthreads();
  uint32_t* ok_g = m.keys_out + pa * m.stride + d0;
  uint32_t* ov_g = m.vals_out + pa * m.stride + d0;
  for (int i = tid; i < len; i += kMergeThreads) {
    ok_g[i] = s_keys[i];
    ov_g[i] = s_vals[i];
  }
}

// ---------------------------------------------------------------------------
// 2. Tile lists through super-tiles.
//    The visible records are in depth order (1a, 1b). Each is binned into the
//    super-tiles (blocks of 8 x 8 tiles of its view) that its rectangle
//    meets: emission in depth order and 1-2 stable digit passes by super-tile
//    id, over about 1.3 entries per record instead of one per tile. A
//    super-tile's list is then cut into chunks of 256 records. Within a
//    chunk, each record's coverage of the super-tile's 64 tiles is a 64-bit
//    mask, and the rank of a record in one tile's list is the population
//    count of one warp ballot per tile, below the lane. Counting per (chunk,
//    tile), a scan over each super-tile's chunks, a scan over all tiles in
//    tile-id order (the tile ranges) and a scatter then write every tile
//    entry once, 4 bytes, at its final position; the order within a tile is
//    the record order of the super-tile's list, i.e. (depth, record).
// ---------------------------------------------------------------------------
constexpr int kSuperLog = 3;
constexpr int kSuperDim = 1 << kSuperLog;           // tiles per super-tile side
constexpr int kSuperTiles = kSuperDim * kSuperDim;  // 64: one bit each in a record's mask
constexpr int kChunk = 256;                         // records per chunk
constexpr int kChunkThreads = kChunk;               // one record per thread
constexpr int kChunkWarps = kChunkThreads / 32;
constexpr int kMaxSuperPasses = 4;

// Super-tile grid of a call: view v has stx[v] x ceil(nty_v / 8) super-tiles,
// with ids from sbase[v] in row-major order.
struct SuperLayout {
  int32_t n_super;
  int32_t stx[kMaxViews];
  uint32_t sbase[kMaxViews + 1];
};

SuperLayout make_super_layout(const Layout& L) {
  SuperLayout S;
  uint32_t base = 0;
  for (int v = 0; v < kMaxViews; ++v) {
    S.sbase[v] = base;
    S.stx[v] = 0;
    if (v < L.V) {
      S.stx[v] = (L.ntx[v] + kSuperDim - 1) >> kSuperLog;
      base += static_cast<uint32_t>(S.stx[v]) * static_cast<uint32_t>((L.nty[v] + kSuperDim - 1) >> kSuperLog);
    }
  }
  S.sbase[kMaxViews] = base;
  S.n_super = static_cast<int32_t>(base);
  return S;
}

__device__ __forceinline__ int view_of_super(const SuperLayout& S, int V, uint32_t s) {
  int v = 0;
  while (v + 1 < V && s >= S.sbase[v + 1]) ++v;
  return v;
}

// View index of record vg = v * N + g (float quotient and exact fix-up).
__device__ __forceinline__ int view_of_record(uint32_t vg, int64_t N, int V, float invN) {
  if (V == 1) return 0;
  int v = __float2int_rz(static_cast<float>(vg) * invN);
  while (v > 0 && static_cast<int64_t>(v) * N > static_cast<int64_t>(vg)) --v;
  while (static_cast<int64_t>(v + 1) * N <= static_cast<int64_t>(vg)) ++v;
  return v;
}

// 2a. Super-tile emission. Each CTA takes a tile of 1024 depth-sorted
//     records by ticket, scans their super-tile counts (block scan with
//     decoupled look-back, clamped at the capacity), then expands them one
//     warp per 32 records, load-balanced: the warp scans the records' counts
//     and lane l produces entries l, l + 32, ... of the warp's concatenated
//     output. It also adds the records' tile counts into *n_isect (the exact
//     intersection count) and gathers the digit histograms of the super-tile
//     passes. With `packed`, each key also carries, above the 16-bit
//     super-tile id, the record's rectangle clipped to that super-tile in its
//     local tile coordinates (3 bits each for x0, y0, x1 - 1, y1 - 1): the
//     sort passes use only the id's bits as digits and carry the rest, so the
//     chunk kernels read a record's coverage from its sorted key instead of
//     gathering its rectangle.
constexpr int kEmitThreads = 256;
static_assert(kEmitThreads == kScanThreads, "the emission scans its records with the block scan");
constexpr int kEmitItems = 4;                         // records per thread in the count scan
constexpr int kEmitTile = kEmitThreads * kEmitItems;  // records per emission tile
constexpr int kEmitGroups = kEmitTile / 32;           // 32-record groups per tile

__device__ __forceinline__ uint32_t super_count(short4 rc) {
  const int sx0 = rc.x >> kSuperLog, sx1 = ((rc.z - 1) >> kSuperLog) + 1;
  const int sy0 = rc.y >> kSuperLog, sy1 = ((rc.w - 1) >> kSuperLog) + 1;
  return static_cast<uint32_t>((sx1 - sx0) * (sy1 - sy0));
}

__global__ void __launch_bounds__(kEmitThreads) emit_super_kernel(
    const uint32_t* __restrict__ order, const int64_t* n_visible, const short4* __restrict__ rects, int64_t N,
    const Layout L, const SuperLayout S, uint64_t capacity, int passes, int packed, ScanState st,
    uint32_t* __restrict__ skeys, uint32_t* __restrict__ svals, uint32_t* __restrict__ hist,
    int64_t* n_super_total, unsigned long long* __restrict__ n_isect, int32_t* status) {
  __shared__ uint32_t s_hist[kMaxSuperPasses][kRadix];
  __shared__ uint32_t s_vg[kEmitTile], s_cnt[kEmitTile], s_off[kEmitTile];
  __shared__ short4 s_rect[kEmitTile];  // the records' rectangles, gathered once
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_warp[kScanThreads / 32];
  __shared__ uint64_t s_prefix;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) s_tile = atomicAdd(st.ticket, 1u);
  for (int i = tid; i < kMaxSuperPasses * kRadix; i += kEmitThreads) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t t = s_tile;
  const int64_t n = *n_visible;
  const int64_t tile0 = static_cast<int64_t>(t) * kEmitTile;
  if (tile0 >= n) return;  // past the data: publishes nothing, awaited by nobody
  // 1. the records (depth order), their super-tile counts, scanned with
  //    decoupled look-back into output offsets (clamped at the capacity),
  //    and their tile counts, summed into the intersection count
  const int64_t base = tile0 + static_cast<int64_t>(tid) * kEmitItems;
  uint32_t c[kEmitItems];
  uint64_t local = 0;
  uint64_t tiles = 0;
#pragma unroll
  for (int i = 0; i < kEmitItems; ++i) {
    const bool ok = base + i < n;
    const uint32_t vg = ok ? order[base + i] : 0u;
    c[i] = 0u;
    short4 rc = make_short4(0, 0, 1, 1);
    if (ok) {
      rc = rects[vg];
      c[i] = super_count(rc);
      tiles += static_cast<uint64_t>(rc.z - rc.x) * static_cast<uint64_t>(rc.w - rc.y);
    }
    s_rect[tid * kEmitItems + i] = rc;
    s_vg[tid * kEmitItems + i] = vg;
    s_cnt[tid * kEmitItems + i] = c[i];
    local += c[i];
  }
  {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tiles += __shfl_xor_sync(0xffffffffu, tiles, o);
    if (lane == 0 && tiles) atomicAdd(n_isect, static_cast<unsigned long long>(tiles));
  }
  uint64_t run = block_scan_lookback(local, t, st, s_warp, &s_prefix, status);
#pragma unroll
  for (int i = 0; i < kEmitItems; ++i) {
    s_off[tid * kEmitItems + i] = static_cast<uint32_t>(run < capacity ? run : capacity);
    run += c[i];
  }
  if (base <= n - 1 && n - 1 < base + kEmitItems) *n_super_total = static_cast<int64_t>(run);
  __syncthreads();
  // 2. emission of (super-tile id, record) pairs, one warp per 32 records,
  //    load-balanced as in the count scan's order
  const float invN = 1.0f / static_cast<float>(N);
  for (int g = tid >> 5; g < kEmitGroups && capacity > 0; g += kEmitThreads / 32) {
    const int r = g * 32 + lane;
    const int64_t j = tile0 + r;
    uint32_t vg = 0, cnt = 0, sb = 0, xy = 0, wn = 1;
    if (j < n) {
      vg = s_vg[r];
      cnt = s_cnt[r];
      const short4 rc = s_rect[r];
      const int v = view_of_record(vg, N, L.V, invN);
      sb = S.sbase[v];
      const int sx0 = rc.x >> kSuperLog, sx1 = ((rc.z - 1) >> kSuperLog) + 1, sy0 = rc.y >> kSuperLog;
      // packed super-rectangle fields: (x0, y0) and (width, super-tiles per row), 16 bits each
      xy = static_cast<uint32_t>(sx0) | (static_cast<uint32_t>(sy0) << 16);
      wn = static_cast<uint32_t>(sx1 - sx0) | (static_cast<uint32_t>(S.stx[v]) << 16);
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t nb = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += nb;
    }
    const uint32_t excl = incl - cnt;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint64_t out_base = s_off[g * 32];
    const uint32_t le_mask = 0xffffffffu >> (31 - lane);  // bits 0..lane
    uint32_t started = 0;  // records (lanes) whose entries start before this group of 32 entries
    for (uint32_t eb = 0; eb < total; eb += 32) {
      // bit i: a record's first entry is entry eb + i (counts are >= 1, so
      // the starts are distinct); the record of entry eb + lane is the last
      // one started at or before it
      const uint32_t stb = (cnt > 0 && excl >= eb && excl - eb < 32u) ? (1u << (excl - eb)) : 0u;
      const uint32_t starts = __reduce_or_sync(0xffffffffu, stb);
      const int src = static_cast<int>(started + __popc(starts & le_mask)) - 1;
      started += __popc(starts);
      const uint32_t e = eb + lane;
      const uint32_t k = e - __shfl_sync(0xffffffffu, excl, src);
      const uint32_t r_vg = __shfl_sync(0xffffffffu, vg, src);
      const uint32_t r_xy = __shfl_sync(0xffffffffu, xy, src);
      const uint32_t r_wn = __shfl_sync(0xffffffffu, wn, src);
      const uint32_t r_sb = L.V > 1 ? __shfl_sync(0xffffffffu, sb, src) : sb;
      const uint64_t pos = out_base + e;
      if (e < total && pos < capacity) {
        const uint32_t r_w = r_wn & 0xffffu, r_stx = r_wn >> 16;
        const uint32_t row = k / r_w, col = k - row * r_w;
        const uint32_t sxa = (r_xy & 0xffffu) + col, sya = (r_xy >> 16) + row;
        const uint32_t s = r_sb + sya * r_stx + sxa;
        uint32_t key = s;
        if (packed) {
          // the record's rectangle in the super-tile's local tile coordinates
          const short4 rc = s_rect[g * 32 + (src & 31)];
          const int ox = static_cast<int>(sxa) << kSuperLog, oy = static_cast<int>(sya) << kSuperLog;
          const int lx0 = max(rc.x - ox, 0), lx1 = min(rc.z - ox, kSuperDim);
          const int ly0 = max(rc.y - oy, 0), ly1 = min(rc.w - oy, kSuperDim);
          key |= static_cast<uint32_t>(lx0 | (ly0 << 3) | ((lx1 - 1) << 6) | ((ly1 - 1) << 9)) << 16;
        }
        skeys[pos] = key;
        svals[pos] = r_vg;
        for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][(s >> (8 * p)) & 0xffu], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < passes * kRadix; i += kEmitThreads) {
    const uint32_t cc = (&s_hist[0][0])[i];
    if (cc) atomicAdd(hist + i, cc);
  }
}

// 2c. Super-tile ranges and the chunk table (one CTA): restores the starts
//     the last super-tile pass left complemented (with no pass, the one
//     super-tile holds the whole list), turns each super-tile's length into
//     chunks of kChunk records (chunk_base: exclusive offsets, chunk_base
//     [n_super] the total); chunk_info_kernel then describes every chunk
//     (first record, length, super-tile, packed view and grid position).
constexpr int kChunkTableThreads = 1024;

__global__ void __launch_bounds__(kChunkTableThreads) super_chunks_kernel(
    uint2* __restrict__ sranges, int32_t n_super, int passes, const int64_t* n_super_total, int64_t capacity,
    uint32_t* __restrict__ chunk_base) {
  __shared__ uint32_t s_w[kChunkTableThreads / 32];
  __shared__ uint32_t s_run;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_run = 0;
  __syncthreads();
  for (int s0 = 0; s0 < n_super; s0 += kChunkTableThreads) {
    const int s = s0 + tid;
    uint32_t nc = 0;
    if (s < n_super) {
      uint2 r = sranges[s];
      if (passes == 0) {
        const int64_t n = *n_super_total < capacity ? *n_super_total : capacity;
        r = make_uint2(0u, static_cast<uint32_t>(n));
        sranges[s] = r;
      } else if (r.y) {
        r.x = ~r.x;
        sranges[s] = r;
      }
      nc = (r.y - r.x + kChunk - 1) / kChunk;
    }
    uint32_t v = nc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t nb = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += nb;
    }
    if (lane == 31) s_w[warp] = v;
    __syncthreads();
    uint32_t add = s_run;
    for (int w = 0; w < warp; ++w) add += s_w[w];
    if (s < n_super) chunk_base[s] = add + v - nc;
    __syncthreads();
    if (tid == kChunkTableThreads - 1) s_run = add + v;
    __syncthreads();
  }
  if (tid == 0) chunk_base[n_super] = s_run;
}

// The chunk table, one warp per super-tile (many CTAs: the table has a
// 16-byte entry per chunk, 328K on the 16-view workload).
constexpr int kChunkInfoThreads = 256;

__global__ void __launch_bounds__(kChunkInfoThreads) chunk_info_kernel(const uint2* __restrict__ sranges,
                                                                       int32_t n_super,
                                                                       const uint32_t* __restrict__ chunk_base,
                                                                       uint4* __restrict__ chunk_info,
                                                                       const SuperLayout S, int V) {
  const int lane = threadIdx.x & 31;
  constexpr int kWarps = kChunkInfoThreads / 32;
  const int nw = static_cast<int>(gridDim.x) * kWarps;
  for (int s = static_cast<int>(blockIdx.x) * kWarps + (threadIdx.x >> 5); s < n_super; s += nw) {
    const uint2 r = sranges[s];
    const uint32_t c0 = chunk_base[s], nc = chunk_base[s + 1] - c0;
    // the super-tile's view and position in its view's super grid, packed
    // once here for the chunk kernels (view < 64, coordinates < 4096)
    const int v = view_of_super(S, V, static_cast<uint32_t>(s));
    const uint32_t local = static_cast<uint32_t>(s) - S.sbase[v], stx = static_cast<uint32_t>(S.stx[v]);
    const uint32_t sy = local / stx, sx = local - sy * stx;
    const uint32_t pos = static_cast<uint32_t>(v) | (sx << 6) | (sy << 18);
    for (uint32_t j = lane; j < nc; j += 32) {
      const uint32_t first = r.x + j * kChunk;
      chunk_info[c0 + j] = make_uint4(first, min(static_cast<uint32_t>(kChunk), r.y - first), static_cast<uint32_t>(s), pos);
    }
  }
}

// A chunk of a super-tile's list as a CTA sees it: its records, one per
// thread, and each record's coverage of the super-tile's 64 tiles.
struct ChunkArgs {
  const uint32_t* svals;        // super-tile lists (records), depth order within each
  const uint32_t* skeys;        // their keys with the local rectangles (or null: gather the rectangles)
  const uint2* sranges;         // [n_super] [start, end) in svals
  const uint32_t* chunk_base;   // [n_super + 1]
  const uint4* chunk_info;      // [chunks] first record, length, super-tile, packed (view, sx, sy)
  const short4* rects;
  uint32_t* chunk_cnt;          // [chunks][64]: tile counts, then their exclusive prefix within the super-tile
  const uint2* ranges;          // [n_tiles] tile ranges (scatter)
  uint32_t* vals;               // [capacity] output (scatter)
  uint64_t capacity;
};

struct ChunkView {
  uint32_t s, sx, sy;  // super-tile and its position in its view's super grid
  int v;               // view
  uint32_t first, len;  // records [first, first + len) of svals
};

__device__ __forceinline__ ChunkView chunk_view(const ChunkArgs& a, uint32_t c) {
  ChunkView cv;
  const uint4 info = a.chunk_info[c];
  cv.first = info.x;
  cv.len = info.y;
  cv.s = info.z;
  cv.v = static_cast<int>(info.w & 63u);
  cv.sx = (info.w >> 6) & 0xfffu;
  cv.sy = info.w >> 18;
  return cv;
}

// Bit ly * 8 + lx: the record's rectangle covers local tile (lx, ly).
__device__ __forceinline__ uint64_t coverage_mask(short4 rc, const ChunkView& cv) {
  const int ox = static_cast<int>(cv.sx) << kSuperLog, oy = static_cast<int>(cv.sy) << kSuperLog;
  const int lx0 = max(rc.x - ox, 0), lx1 = min(rc.z - ox, kSuperDim);
  const int ly0 = max(rc.y - oy, 0), ly1 = min(rc.w - oy, kSuperDim);
  if (lx0 >= lx1 || ly0 >= ly1) return 0ull;
  const uint64_t row = ((1ull << (lx1 - lx0)) - 1ull) << lx0;  // < 256
  // one byte per covered row: the multiplication places copies without carries
  const uint64_t rows = (0x0101010101010101ull >> (8 * (kSuperDim - (ly1 - ly0)))) << (8 * ly0);
  return row * rows;
}

// The same mask from a record's rectangle in the super-tile's local
// coordinates, packed as the emission stores it above the key's id.
__device__ __forceinline__ uint64_t packed_mask(uint32_t pack) {
  const int lx0 = pack & 7, ly0 = (pack >> 3) & 7, lx1 = ((pack >> 6) & 7) + 1, ly1 = ((pack >> 9) & 7) + 1;
  const uint64_t row = ((1ull << (lx1 - lx0)) - 1ull) << lx0;
  const uint64_t rows = (0x0101010101010101ull >> (8 * (kSuperDim - (ly1 - ly0)))) << (8 * ly0);
  return row * rows;
}

// Coverage mask of the chunk's record `e` (a position in the super-tile lists).
__device__ __forceinline__ uint64_t record_mask(const ChunkArgs& a, const ChunkView& cv, uint32_t e, uint32_t vg) {
  return a.skeys ? packed_mask(a.skeys[e] >> 16) : coverage_mask(a.rects[vg], cv);
}

// Global tile id of local tile t of the chunk's super-tile, or -1 if it lies
// beyond the view's tile grid (a partial super-tile at the right or bottom).
__device__ __forceinline__ int64_t tile_of(const Layout& L, const ChunkView& cv, int t) {
  const int tx = (static_cast<int>(cv.sx) << kSuperLog) + (t & (kSuperDim - 1));
  const int ty = (static_cast<int>(cv.sy) << kSuperLog) + (t >> kSuperLog);
  if (tx >= L.ntx[cv.v] || ty >= L.nty[cv.v]) return -1;
  return static_cast<int64_t>(L.tile_base[cv.v]) + static_cast<int64_t>(ty) * L.ntx[cv.v] + tx;
}

// 32 x 32 bit transpose across a warp: on entry lane l holds row l, on exit
// lane l holds column l (bit i of the result = bit l of lane i's row). Stage
// j swaps bit j of the row index (the lane) with bit j of the column index
// (the bit position); the five swaps together exchange the two indices.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x) {
  const int lane = threadIdx.x & 31;
  const uint32_t masks[5] = {0x55555555u, 0x33333333u, 0x0f0f0f0fu, 0x00ff00ffu, 0x0000ffffu};
#pragma unroll
  for (int k = 4; k >= 0; --k) {
    const int j = 1 << k;
    const uint32_t m = masks[k];  // bit positions whose bit j is 0
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & ~m) | ((y & ~m) >> j)) : ((x & m) | ((y & m) << j));
  }
  return x;
}

// For the warp's 32 coverage masks: in lane l, the lanes covering tile l
// (lo) and tile l + 32 (hi), as 32-bit lane sets.
__device__ __forceinline__ void warp_tile_lanes(uint64_t m, uint32_t& lo, uint32_t& hi) {
  lo = warp_transpose32(static_cast<uint32_t>(m));
  hi = warp_transpose32(static_cast<uint32_t>(m >> 32));
}

// 2d. Tile counts per chunk.
__global__ void __launch_bounds__(kChunkThreads) chunk_count_kernel(const ChunkArgs a, const Layout L,
                                                                     const SuperLayout S) {
  __shared__ uint32_t s_cnt[kChunkWarps][kSuperTiles];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t n_chunks = a.chunk_base[S.n_super];
  for (uint32_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    const ChunkView cv = chunk_view(a, c);
    uint64_t m = 0;
    if (static_cast<uint32_t>(tid) < cv.len) {
      const uint32_t e = cv.first + tid;
      m = record_mask(a, cv, e, a.skeys ? 0u : a.svals[e]);
    }
    uint32_t lo, hi;
    warp_tile_lanes(m, lo, hi);
    s_cnt[warp][lane] = __popc(lo);
    s_cnt[warp][lane + 32] = __popc(hi);
    __syncthreads();
    if (tid < kSuperTiles) {
      uint32_t sum = 0;
#pragma unroll
      for (int w = 0; w < kChunkWarps; ++w) sum += s_cnt[w][tid];
      a.chunk_cnt[static_cast<size_t>(c) * kSuperTiles + tid] = sum;
    }
    __syncthreads();
  }
}

// 2e. Per super-tile (one CTA each): the exclusive prefix of every tile's
//     counts over the super-tile's chunks (in place) and the tile totals.
// 16 groups of 64 threads, each walking a 16th of the super-tile's chunks
// with 4 loads in flight: the largest super-tiles (about a thousand chunks at
// the centre of a 4K view) set the kernel's time.
constexpr int kSuperScanThreads = 1024;
constexpr int kSuperScanGroups = kSuperScanThreads / kSuperTiles;

__global__ void __launch_bounds__(kSuperScanThreads) super_scan_kernel(uint32_t* __restrict__ chunk_cnt,
                                                                       const uint32_t* __restrict__ chunk_base,
                                                                       const Layout L, const SuperLayout S,
                                                                       uint32_t* __restrict__ tile_cnt) {
  __shared__ uint32_t s_part[kSuperScanGroups][kSuperTiles];
  const uint32_t s = blockIdx.x;
  const int t = threadIdx.x % kSuperTiles, g = threadIdx.x / kSuperTiles;
  const uint32_t c0 = chunk_base[s], nc = chunk_base[s + 1] - c0;
  const uint32_t per = (nc + kSuperScanGroups - 1) / kSuperScanGroups;
  const uint32_t j0 = min(nc, g * per), j1 = min(nc, j0 + per);
  uint32_t* col = chunk_cnt + static_cast<size_t>(c0) * kSuperTiles + t;
  uint32_t sum = 0;
#pragma unroll 4
  for (uint32_t j = j0; j < j1; ++j) sum += col[static_cast<size_t>(j) * kSuperTiles];
  s_part[g][t] = sum;
  __syncthreads();
  uint32_t run = 0, total = 0;
#pragma unroll
  for (int h = 0; h < kSuperScanGroups; ++h) {
    const uint32_t p = s_part[h][t];
    if (h < g) run += p;
    total += p;
  }
  uint32_t j = j0;
  for (; j + 4 <= j1; j += 4) {
    uint32_t x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = col[static_cast<size_t>(j + k) * kSuperTiles];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      col[static_cast<size_t>(j + k) * kSuperTiles] = run;
      run += x[k];
    }
  }
  for (; j < j1; ++j) {
    const uint32_t x = col[static_cast<size_t>(j) * kSuperTiles];
    col[static_cast<size_t>(j) * kSuperTiles] = run;
    run += x;
  }
  if (g == 0) {
    ChunkView cv;
    cv.s = s;
    cv.v = view_of_super(S, L.V, s);
    const uint32_t local = s - S.sbase[cv.v], stx = static_cast<uint32_t>(S.stx[cv.v]);
    cv.sy = local / stx;
    cv.sx = local - cv.sy * stx;
    const int64_t tile = tile_of(L, cv, t);
    if (tile >= 0) tile_cnt[tile] = total;
  }
}

// 2f. Tile ranges: exclusive scan of the tile counts in tile-id order (block
//     scan with decoupled look-back); flags a capacity overflow. The ranges
//     are clamped at the capacity, so that even after an overflow (flagged,
//     results unusable) a rasteriser reading them stays inside `vals`.
__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(const uint32_t* __restrict__ tile_cnt,
                                                                 int64_t n_tiles, ScanState st,
                                                                 uint2* __restrict__ ranges,
                                                                 const int64_t* n_isect, int64_t capacity,
                                                                 int32_t* status) {
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_warp[kScanThreads / 32];
  __shared__ uint64_t s_prefix;
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(st.ticket, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  if (t == 0 && tid == 0 && *n_isect > capacity) set_status(status, GS_STATUS_CAPACITY);
  const int64_t base = static_cast<int64_t>(t) * kScanTile + static_cast<int64_t>(tid) * kScanItems;
  uint32_t cnt[kScanItems];
  uint64_t local = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    cnt[i] = base + i < n_tiles ? tile_cnt[base + i] : 0u;
    local += cnt[i];
  }
  uint64_t run = block_scan_lookback(local, t, st, s_warp, &s_prefix, status);
  const uint64_t cap = static_cast<uint64_t>(capacity);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n_tiles) {
      const uint64_t end = run + cnt[i];
      ranges[base + i] = make_uint2(static_cast<uint32_t>(run < cap ? run : cap), static_cast<uint32_t>(end < cap ? end : cap));
    }
    run += cnt[i];
  }
}

// 2g. Scatter. A record's entry in covered tile t goes to (tile start + the
//     chunk's prefix for t + the warps before it + the lanes below it that
//     cover t). After the transpose, lane l of a warp holds the lanes that
//     cover tiles l and l + 32, so it produces those two tiles' entries in
//     lane order: the work per lane is the entries of two neighbouring tiles,
//     which vary much less than the tiles per record. Each entry is staged
//     in shared memory as 16 bits (tile, record within the chunk), tile by
//     tile (the chunk's runs in tile order), and the CTA then writes the runs
//     with consecutive threads on consecutive positions. A chunk with more
//     entries than the staging holds (at 4K the largest has 5963) writes them
//     directly.
constexpr int kStage = 8192;

__global__ void __launch_bounds__(kChunkThreads) scatter_kernel(const ChunkArgs a, const Layout L,
                                                                 const SuperLayout S) {
  __shared__ uint32_t s_vg[kChunkThreads];              // record of each thread
  __shared__ uint32_t s_pre[kChunkWarps][kSuperTiles];  // counts, then the chunk-local prefix per tile
  __shared__ uint32_t s_gbase[kSuperTiles];             // global position of the chunk's first entry in t
  __shared__ uint32_t s_tloc[kSuperTiles + 1];          // start of tile t's run in the staging
  __shared__ uint16_t s_stage[kStage];                  // tile << 8 | record within the chunk
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t n_chunks = a.chunk_base[S.n_super];
  for (uint32_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    const ChunkView cv = chunk_view(a, c);
    // the tile bases do not depend on the records: their loads go out first
    // (warp 0, tiles lane and lane + 32)
    uint32_t gb[2] = {0u, 0u};
    if (warp == 0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t tile = tile_of(L, cv, lane + 32 * h);
        if (tile >= 0) gb[h] = a.ranges[tile].x + a.chunk_cnt[static_cast<size_t>(c) * kSuperTiles + lane + 32 * h];
      }
    }
    uint64_t m = 0;
    uint32_t vg = 0;
    if (static_cast<uint32_t>(tid) < cv.len) {
      const uint32_t e = cv.first + tid;
      vg = a.svals[e];
      m = record_mask(a, cv, e, vg);
    }
    uint32_t lo, hi;
    warp_tile_lanes(m, lo, hi);
    s_vg[tid] = vg;
    s_pre[warp][lane] = __popc(lo);
    s_pre[warp][lane + 32] = __popc(hi);
    __syncthreads();
    if (warp == 0) {
      // per tile (lane, lane + 32): the warps' exclusive prefix and the total,
      // then the staging layout, an exclusive scan of the 64 totals
      uint32_t tot[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int t = lane + 32 * h;
        s_gbase[t] = gb[h];
        tot[h] = 0;
#pragma unroll
        for (int w = 0; w < kChunkWarps; ++w) {
          const uint32_t x = s_pre[w][t];
          s_pre[w][t] = tot[h];
          tot[h] += x;
        }
      }
      uint32_t v0 = tot[0], v1 = tot[1];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t n0 = __shfl_up_sync(0xffffffffu, v0, o), n1 = __shfl_up_sync(0xffffffffu, v1, o);
        if (lane >= o) {
          v0 += n0;
          v1 += n1;
        }
      }
      const uint32_t first_half = __shfl_sync(0xffffffffu, v0, 31);
      s_tloc[lane + 1] = v0;
      s_tloc[lane + 33] = v1 + first_half;
      if (lane == 0) s_tloc[0] = 0;
    }
    __syncthreads();
    const uint32_t total = s_tloc[kSuperTiles];
    const bool staged = total <= static_cast<uint32_t>(kStage);
    const uint32_t wbase = static_cast<uint32_t>(warp) * 32u;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int t = lane + 32 * h;
      uint32_t set = h ? hi : lo;
      const uint32_t k0 = s_pre[warp][t];
      if (staged) {
        uint32_t i = s_tloc[t] + k0;
        const uint32_t tag = static_cast<uint32_t>(t) << 8;
        while (set) {
          const uint32_t r = static_cast<uint32_t>(__ffs(set) - 1);
          set &= set - 1;
          s_stage[i++] = static_cast<uint16_t>(tag | (wbase + r));
        }
      } else {
        const uint32_t g = s_gbase[t] + k0;
        for (uint32_t k = 0; set; ++k) {
          const uint32_t r = static_cast<uint32_t>(__ffs(set) - 1);
          set &= set - 1;
          if (static_cast<uint64_t>(g) + k < a.capacity) a.vals[g + k] = s_vg[wbase + r];
        }
      }
    }
    __syncthreads();
    if (staged) {
      for (uint32_t i = tid; i < total; i += kChunkThreads) {
        const uint32_t e = s_stage[i];
        const uint32_t t = e >> 8;
        const uint64_t pos = static_cast<uint64_t>(s_gbase[t]) + (i - s_tloc[t]);
        if (pos < a.capacity) a.vals[pos] = s_vg[e & 0xffu];
      }
    }
    __syncthreads();
  }
}

// Optional 64-bit keys (tile << 32) | bits(depth) of the sorted list.
__global__ void keys64_kernel(const uint2* __restrict__ ranges, int64_t n_tiles, const uint32_t* __restrict__ vals,
                              const float* __restrict__ projected, const uint32_t* __restrict__ depth_keys,
                              int64_t capacity, uint64_t* __restrict__ keys) {
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const uint2 r = ranges[t];
    for (int64_t p = static_cast<int64_t>(r.x) + threadIdx.x; p < r.y && p < capacity; p += blockDim.x) {
      const uint32_t vg = vals[p];
      const uint32_t d =
          depth_keys ? depth_keys[vg] : __float_as_uint(projected[static_cast<int64_t>(vg) * kRecordFloats + 6]);
      keys[p] = (static_cast<uint64_t>(t) << 32) | d;
    }
  }
}

// ---------------------------------------------------------------------------
// Workspace layout.
// ---------------------------------------------------------------------------
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Digit passes (8 bits each) that sort keys below n_keys.
int passes_for(int64_t n_keys) {
  int bits = 0;
  while ((int64_t(1) << bits) < n_keys) ++bits;
  return (bits + 7) / 8;
}

// Super-tile ids never exceed the tile count (a super-tile holds at least one
// tile), so the super-tile buffers are sized from n_tiles.
struct WsLayout {
  size_t dkeys0, dvals0, dkeys1, dvals1, skeys0, skeys1, svals0, svals1;
  size_t chunk_cnt, chunk_info, chunk_base, tile_cnt;
  size_t zero_begin, scan1, scan_s, scan_t, hist_d, hist_s, tickets, n_visible, n_super_total, sranges, lb_depth,
      lb_super;
  size_t part_scan, part_hist, part_tickets, part_n, part_lb, zero_end, total;
  int64_t n_scan_tiles, n_emit_tiles, n_depth_tiles, n_super_sort_tiles, n_tile_scan_tiles, max_chunks;
  int64_t part_stride, part_scan_tiles, part_sort_tiles;
  int super_passes;
};

constexpr int kPartTickets = 8;  // per partition: compaction + 4 depth passes

// P > 1: the depth sort runs as P partitions of the records, merged after.
WsLayout ws_layout(int64_t N, int32_t V, int64_t capacity, int64_t n_tiles, int P = 1) {
  WsLayout w;
  const int64_t VN = N * V;
  w.part_stride = P > 1 ? (VN + P - 1) / P : VN;
  const int64_t depth_slots = P > 1 ? w.part_stride * P : VN;
  const size_t cap = static_cast<size_t>(capacity > 0 ? capacity : 1);
  const size_t ds = static_cast<size_t>(depth_slots > 0 ? depth_slots : 1);
  const size_t nt = static_cast<size_t>(n_tiles > 0 ? n_tiles : 1);
  w.super_passes = passes_for(n_tiles);
  w.n_scan_tiles = (VN + kScanTile - 1) / kScanTile;
  w.n_emit_tiles = (VN + kEmitTile - 1) / kEmitTile;
  w.n_depth_tiles = (VN + kSortTile - 1) / kSortTile;
  w.n_super_sort_tiles = (capacity + kSortTile - 1) / kSortTile;
  w.n_tile_scan_tiles = (n_tiles + kScanTile - 1) / kScanTile;
  w.max_chunks = static_cast<int64_t>((cap + kChunk - 1) / kChunk + nt);
  w.part_scan_tiles = (w.part_stride + kScanTile - 1) / kScanTile;
  w.part_sort_tiles = (w.part_stride + kSortTile - 1) / kSortTile;
  const size_t mc = static_cast<size_t>(w.max_chunks);
  size_t o = 0;
  w.dkeys0 = o; o = align256(o + 4 * ds);
  w.dvals0 = o; o = align256(o + 4 * ds);
  w.dkeys1 = o; o = align256(o + 4 * ds);
  w.dvals1 = o; o = align256(o + 4 * ds);
  w.skeys0 = o; o = align256(o + 4 * cap);
  w.skeys1 = o; o = align256(o + 4 * cap);
  w.svals0 = o; o = align256(o + 4 * cap);
  w.svals1 = o; o = align256(o + 4 * cap);
  w.chunk_cnt = o; o = align256(o + 4 * kSuperTiles * mc);
  w.chunk_info = o; o = align256(o + 16 * mc);
  w.chunk_base = o; o = align256(o + 4 * (nt + 1));
  w.tile_cnt = o; o = align256(o + 4 * nt);
  w.zero_begin = o;
  w.scan1 = o; o = align256(o + 8 * static_cast<size_t>(w.n_scan_tiles + 1));
  w.scan_s = o; o = align256(o + 8 * static_cast<size_t>(w.n_emit_tiles + 1));
  w.scan_t = o; o = align256(o + 8 * static_cast<size_t>(w.n_tile_scan_tiles + 1));
  w.hist_d = o; o = align256(o + 4 * kDepthPasses * kRadix);
  w.hist_s = o; o = align256(o + 4 * kMaxSuperPasses * kRadix);
  w.tickets = o; o = align256(o + 4 * 16);
  w.n_visible = o; o = align256(o + 8);
  w.n_super_total = o; o = align256(o + 8);
  w.sranges = o; o = align256(o + 8 * nt);
  w.lb_depth = o; o = align256(o + 8 * kRadix * kDepthPasses * static_cast<size_t>(w.n_depth_tiles + 1));
  w.lb_super = o;
  o = align256(o + 8 * kRadix * static_cast<size_t>(w.super_passes) * static_cast<size_t>(w.n_super_sort_tiles + 1));
  const size_t np = static_cast<size_t>(P > 1 ? P : 0);
  w.part_scan = o; o = align256(o + 8 * np * static_cast<size_t>(w.part_scan_tiles + 1));
  w.part_hist = o; o = align256(o + 4 * np * kDepthPasses * kRadix);
  w.part_tickets = o; o = align256(o + 4 * np * kPartTickets);
  w.part_n = o; o = align256(o + 8 * np);
  w.part_lb = o; o = align256(o + 8 * np * kRadix * kDepthPasses * static_cast<size_t>(w.part_sort_tiles + 1));
  w.zero_end = o;
  w.total = o;
  return w;
}

// Per-device launch facts, filled on the first call made on each device
// (with that device current) under one lock, so that threads making their
// first calls at once, or on different devices, see complete entries.
struct DeviceFacts {
  std::mutex m;
  int sms[kMaxDevices] = {};
  int sort_ctas_per_sm[kMaxDevices] = {};  // 0: the digit pass's attributes are not set yet
};
DeviceFacts& device_facts() {
  static DeviceFacts f;
  return f;
}

int query_sm_count(int dev) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 148;
}

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (dev < 0 || dev >= kMaxDevices) return query_sm_count(dev);
  DeviceFacts& f = device_facts();
  std::lock_guard<std::mutex> lock(f.m);
  if (!f.sms[dev]) f.sms[dev] = query_sm_count(dev);
  return f.sms[dev];
}

// Sets the digit pass's shared-memory attributes on the current device and
// returns its resident CTAs per SM (0 on a CUDA error).
int setup_sort_pass() {
  {
    const void* fns[8] = {reinterpret_cast<const void*>(sort_pass_kernel<1>), reinterpret_cast<const void*>(sort_pass_kernel<2>),
                          reinterpret_cast<const void*>(sort_pass_kernel<3>), reinterpret_cast<const void*>(sort_pass_kernel<4>),
                          reinterpret_cast<const void*>(sort_pass_kernel<5>), reinterpret_cast<const void*>(sort_pass_kernel<6>),
                          reinterpret_cast<const void*>(sort_pass_kernel<7>), reinterpret_cast<const void*>(sort_pass_kernel<8>)};
    for (const void* f : fns)
      if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sizeof(SortSmem))) !=
              cudaSuccess ||
          cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
              cudaSuccess)
        return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sort_pass_kernel<8>, kSortThreads, sizeof(SortSmem)) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm;
}

}  // namespace

// Occupancy-derived persistent grid for the digit passes; sets the kernel's
// shared-memory attributes on the first call made on each device.
int sort_grid_cap(int64_t* cap) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
  int per_sm = 0;
  if (dev < 0 || dev >= kMaxDevices) {
    per_sm = setup_sort_pass();
  } else {
    DeviceFacts& f = device_facts();
    std::lock_guard<std::mutex> lock(f.m);
    if (!f.sort_ctas_per_sm[dev]) f.sort_ctas_per_sm[dev] = setup_sort_pass();
    per_sm = f.sort_ctas_per_sm[dev];
  }
  if (per_sm < 1) return GS_ERR_CUDA;
  *cap = static_cast<int64_t>(sm_count()) * per_sm;
  return GS_OK;
}

int64_t sort_tiles_for(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

void launch_hist_scan(uint32_t* hist, int passes, cudaStream_t stream) {
  hist_scan_kernel<<<1, kRadix, 0, stream>>>(hist, passes);
}

int run_u32_sort_passes(uint32_t* const keys[2], uint32_t* const vals[2], const int64_t* n_dev, int64_t cap,
                        int passes, const uint32_t* hist, uint32_t* tickets, uint64_t* lookback, int32_t* status,
                        cudaStream_t stream) {
  int64_t grid_cap = 0;
  const int rc = sort_grid_cap(&grid_cap);
  if (rc != GS_OK) return rc;
  const int64_t tiles = sort_tiles_for(cap);
  const unsigned grid = static_cast<unsigned>(tiles < grid_cap ? (tiles > 0 ? tiles : 1) : grid_cap);
  for (int p = 0; p < passes; ++p) {
    PassArgs a;
    a.keys_in = keys[p & 1]; a.vals_in = vals[p & 1]; a.keys_out = keys[(p + 1) & 1]; a.vals_out = vals[(p + 1) & 1];
    a.n_total = n_dev; a.cap = cap; a.shift = 8 * p; a.digit_offsets = hist + p * kRadix; a.scan_digits = 0;
    a.ticket = tickets + p;
    a.ranges = nullptr; a.n_keys = 0; a.key_mask = 0xffffffffu;
    a.stall_tile = -1;
    a.spin_limit = kSpinLimit;
    a.lookback = lookback + static_cast<size_t>(p) * (tiles + 1) * kRadix;
    sort_pass_kernel<8><<<grid, kSortThreads, sizeof(SortSmem), stream>>>(a, status);
  }
  return cuda_status(cudaGetLastError());
}

}  // namespace gs

namespace gs {
namespace {

bool valid_partitions(int P) { return P >= 1 && P <= 64 && (P & (P - 1)) == 0; }

int bin_sort_impl(const float* projected, const int16_t* rects, const uint32_t* counts, const uint32_t* depth_keys,
                  int64_t N,
                  const int32_t* sizes, int32_t V, const gs_config* cfg, uint64_t* keys, uint32_t* vals,
                  int64_t capacity, uint32_t* tile_ranges, int64_t* n_isect_dev, void* workspace,
                  size_t workspace_bytes, int32_t* status_dev, cudaStream_t stream, int P) {
  Layout L;
  int rc = build_layout(sizes, V, cfg, &L, nullptr);
  if (rc != GS_OK) return rc;
  if (N < 0 || capacity < 0 || capacity >= (int64_t(1) << 32) - 1) return GS_ERR_ARG;
  if (N * static_cast<int64_t>(V) >= (int64_t(1) << 32) - 1) return GS_ERR_ARG;
  if (!tile_ranges || !n_isect_dev || !workspace) return GS_ERR_ARG;
  if (N > 0 && (!projected || !rects || !counts)) return GS_ERR_ARG;
  if (capacity > 0 && !vals) return GS_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) || (reinterpret_cast<uintptr_t>(rects) & 7u)) return GS_ERR_ARG;
  if (!valid_partitions(P)) return GS_ERR_ARG;
  const WsLayout w = ws_layout(N, V, capacity, L.n_tiles, P);
  if (workspace_bytes < w.total) return GS_ERR_ARG;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  auto u32 = [&](size_t off) { return reinterpret_cast<uint32_t*>(ws + off); };
  uint32_t* tickets = u32(w.tickets);
  int64_t* n_visible = reinterpret_cast<int64_t*>(ws + w.n_visible);

  cudaError_t e = cudaMemsetAsync(ws + w.zero_begin, 0, w.zero_end - w.zero_begin, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * static_cast<size_t>(L.n_tiles), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n_isect_dev, 0, sizeof(int64_t), stream);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  const int64_t VN = N * V;
  if (VN == 0) {
    if (cfg->flags & GS_FLAG_TILE_ORDER)
      tile_order_kernel<<<1, kOrderThreads, 0, stream>>>(reinterpret_cast<const uint2*>(tile_ranges), L.n_tiles,
                                                         tile_ranges + 2 * L.n_tiles);
    return cuda_status(cudaGetLastError());
  }
  int64_t sort_grid_cap = 0;
  rc = gs::sort_grid_cap(&sort_grid_cap);
  if (rc != GS_OK) return rc;
  auto sort_grid = [&](int64_t tiles) {
    return static_cast<unsigned>(tiles < sort_grid_cap ? (tiles > 0 ? tiles : 1) : sort_grid_cap);
  };
  const unsigned scan_grid = static_cast<unsigned>(w.n_scan_tiles);

  // 1a. visible records -> (depth bits, record), depth digit histograms
  uint32_t* dk[2] = {u32(w.dkeys0), u32(w.dkeys1)};
  uint32_t* dv[2] = {u32(w.dvals0), u32(w.dvals1)};
  const uint32_t* order = dv[0];
  if (P == 1) {
    ScanState st1{reinterpret_cast<uint64_t*>(ws + w.scan1), tickets + 0};
    uint32_t* hist_d = u32(w.hist_d);
    compact_visible_kernel<<<scan_grid, kScanThreads, 0, stream>>>(counts, projected, depth_keys, VN, 0u, st1, dk[0],
                                                                     dv[0], hist_d, n_visible, status_dev);
    // 1b. four depth passes (even count: the result is back in dk[0], dv[0])
    for (int p = 0; p < kDepthPasses; ++p) {
      PassArgs a;
      a.keys_in = dk[p & 1]; a.vals_in = dv[p & 1]; a.keys_out = dk[(p + 1) & 1]; a.vals_out = dv[(p + 1) & 1];
      a.n_total = n_visible; a.cap = VN; a.shift = 8 * p; a.digit_offsets = hist_d + p * kRadix;
      a.scan_digits = 1;  // the counts gathered by the compaction
      a.ticket = tickets + 2 + p;
      a.ranges = nullptr; a.n_keys = 0; a.key_mask = 0xffffffffu;
      a.stall_tile = (p == 0 && (cfg->flags & GS_FLAG_TEST_STALL_LOOKBACK)) ? 0 : -1;
      a.spin_limit = (cfg->flags & GS_FLAG_TEST_STALL_LOOKBACK) ? kTestSpinLimit : kSpinLimit;
      a.lookback = reinterpret_cast<uint64_t*>(ws + w.lb_depth) + static_cast<size_t>(p) * (w.n_depth_tiles + 1) * kRadix;
      sort_pass_kernel<8><<<sort_grid(w.n_depth_tiles), kSortThreads, sizeof(SortSmem), stream>>>(a, status_dev);
    }
  } else {
    // 1a'/1b'. P partitions of the records, each compacted and depth-sorted
    //          on its own into its slot of part_stride entries ...
    const int64_t S = w.part_stride;
    uint64_t* part_scan = reinterpret_cast<uint64_t*>(ws + w.part_scan);
    uint32_t* part_hist = u32(w.part_hist);
    uint32_t* part_tickets = u32(w.part_tickets);
    int64_t* part_n = reinterpret_cast<int64_t*>(ws + w.part_n);
    uint64_t* part_lb = reinterpret_cast<uint64_t*>(ws + w.part_lb);
    for (int p = 0; p < P; ++p) {
      const int64_t lo = p * S, cnt = VN - lo < S ? VN - lo : S;
      if (cnt <= 0) continue;  // an empty partition keeps part_n = 0
      ScanState stp{part_scan + static_cast<size_t>(p) * (w.part_scan_tiles + 1), part_tickets + p * kPartTickets};
      compact_visible_kernel<<<static_cast<unsigned>((cnt + kScanTile - 1) / kScanTile), kScanThreads, 0, stream>>>(
          counts + lo, projected + lo * kRecordFloats, depth_keys ? depth_keys + lo : nullptr, cnt,
          static_cast<uint32_t>(lo), stp, dk[0] + lo, dv[0] + lo,
          part_hist + p * kDepthPasses * kRadix, part_n + p, status_dev);
    }
    hist_scan_kernel<<<1, kRadix, 0, stream>>>(part_hist, kDepthPasses * P);
    for (int p = 0; p < P; ++p) {
      const int64_t lo = p * S;
      if (VN - lo <= 0) continue;
      uint32_t* const pk[2] = {dk[0] + lo, dk[1] + lo};
      uint32_t* const pv[2] = {dv[0] + lo, dv[1] + lo};
      rc = run_u32_sort_passes(pk, pv, part_n + p, S, kDepthPasses, part_hist + p * kDepthPasses * kRadix,
                               part_tickets + p * kPartTickets + 1,
                               part_lb + static_cast<size_t>(p) * kDepthPasses * (w.part_sort_tiles + 1) * kRadix,
                               status_dev, stream);
      if (rc != GS_OK) return rc;
    }
    // ... then merged pairwise, log2(P) levels, into one run at offset 0
    int src = 0;
    int levels = 0;
    while ((1 << levels) < P) ++levels;
    for (int level = 0; level < levels; ++level) {
      MergeArgs m;
      m.keys_in = dk[src]; m.vals_in = dv[src]; m.keys_out = dk[1 - src]; m.vals_out = dv[1 - src];
      m.part_n = part_n;
      m.stride = S;
      m.level = level;
      m.ctas_per_pair = ((S << (level + 1)) + kMergeTile - 1) / kMergeTile;
      m.n_total = level == levels - 1 ? n_visible : nullptr;
      const int64_t grid = static_cast<int64_t>(P >> (level + 1)) * m.ctas_per_pair;
      merge_runs_kernel<<<static_cast<unsigned>(grid), kMergeThreads, 0, stream>>>(m);
      src = 1 - src;
    }
    order = dv[src];
  }
  // 2a. super-tile emission in depth order (and the exact intersection count)
  const SuperLayout S = make_super_layout(L);
  const int SP = passes_for(S.n_super);
  // super-tile ids of at most 16 bits leave the key's high half for the local rectangles
  const bool packed = S.n_super <= (1 << 16);
  uint32_t* sk[2] = {u32(w.skeys0), u32(w.skeys1)};
  uint32_t* sv[2] = {u32(w.svals0), u32(w.svals1)};
  uint32_t* hist_s = u32(w.hist_s);
  int64_t* n_super_total = reinterpret_cast<int64_t*>(ws + w.n_super_total);
  uint2* sranges = reinterpret_cast<uint2*>(ws + w.sranges);
  uint2* ranges = reinterpret_cast<uint2*>(tile_ranges);
  ScanState st2{reinterpret_cast<uint64_t*>(ws + w.scan_s), tickets + 1};
  emit_super_kernel<<<static_cast<unsigned>(w.n_emit_tiles), kEmitThreads, 0, stream>>>(
      order, n_visible, reinterpret_cast<const short4*>(rects), N, L, S, static_cast<uint64_t>(capacity), SP,
      packed ? 1 : 0, st2, sk[0], sv[0], hist_s, n_super_total, reinterpret_cast<unsigned long long*>(n_isect_dev),
      status_dev);
  // 2b. stable super-tile passes; the last one bounds the super-tile ranges
  for (int p = 0; p < SP; ++p) {
    PassArgs a;
    a.keys_in = sk[p & 1]; a.vals_in = sv[p & 1]; a.keys_out = sk[(p + 1) & 1]; a.vals_out = sv[(p + 1) & 1];
    a.ranges = nullptr; a.n_keys = 0; a.key_mask = packed ? 0xffffu : 0xffffffffu;
    if (p == SP - 1) {
      // the last pass bounds the super-tile ranges; it writes the keys too
      // when they carry the records' local rectangles
      a.ranges = sranges;
      a.n_keys = static_cast<uint32_t>(S.n_super);
      if (!packed) a.keys_out = nullptr;
    }
    a.n_total = n_super_total; a.cap = capacity; a.shift = 8 * p; a.digit_offsets = hist_s + p * kRadix;
    a.scan_digits = 1;  // the counts gathered by the emission
    a.ticket = tickets + 6 + p;
    a.stall_tile = -1;
    a.spin_limit = kSpinLimit;
    a.lookback = reinterpret_cast<uint64_t*>(ws + w.lb_super) +
                 static_cast<size_t>(p) * (w.n_super_sort_tiles + 1) * kRadix;
    int bits = 8;
    if (p == SP - 1) {
      bits = 0;
      while ((int64_t(1) << bits) < S.n_super) ++bits;
      bits -= 8 * (SP - 1);
    }
    const unsigned grid = sort_grid(w.n_super_sort_tiles);
    switch (bits) {
      case 1: sort_pass_kernel<1><<<grid, kSortThreads, sizeof(SortSmem), stream>>>(a, status_dev); break;
      case 2: sort_pass_kernel<2><<<grid, kSortThreads, sizeof(SortSmem), stream>>>(a, status_dev); break;
      case 3: sort_pass_kernel<3><<<grid, kSortThreads, sizeof(SortSmem), stream>>>(a, status_dev); break;
      case 4: sort_pass_kernel<4><<<grid, kSortThreads, sizeof(SortSmem), stream>>>(a, status_dev); break;
      case 5: sort_pass_kernel<5><<<grid, kSortThreads, sizeof(SortSmem), stream>>>(a, status_dev); break;
      case 6: sort_pass_kernel<6><<<grid, kSortThreads, sizeof(SortSmem), stream>>>(a, status_dev); break;
      case 7: sort_pass_kernel<7><<<grid, kSortThreads, sizeof(SortSmem), stream>>>(a, status_dev); break;
      default: sort_pass_kernel<8><<<grid, kSortThreads, sizeof(SortSmem), stream>>>(a, status_dev); break;
    }
  }
  // 2c-2g. chunk table, tile counts per chunk, per super-tile prefixes, tile
  //        ranges, scatter into `vals`
  uint32_t* chunk_base = u32(w.chunk_base);
  uint4* chunk_info = reinterpret_cast<uint4*>(ws + w.chunk_info);
  super_chunks_kernel<<<1, kChunkTableThreads, 0, stream>>>(sranges, S.n_super, SP, n_super_total, capacity,
                                                           chunk_base);
  {
    const int64_t want = (S.n_super + kChunkInfoThreads / 32 - 1) / (kChunkInfoThreads / 32);
    const unsigned grid = static_cast<unsigned>(want < 4 * static_cast<int64_t>(sm_count()) ? (want > 0 ? want : 1)
                                                                                             : 4 * sm_count());
    chunk_info_kernel<<<grid, kChunkInfoThreads, 0, stream>>>(sranges, S.n_super, chunk_base, chunk_info, S, L.V);
  }
  ChunkArgs ca;
  ca.svals = sv[SP & 1];
  ca.skeys = packed ? sk[SP & 1] : nullptr;
  ca.sranges = sranges;
  ca.chunk_base = chunk_base;
  ca.chunk_info = chunk_info;
  ca.rects = reinterpret_cast<const short4*>(rects);
  ca.chunk_cnt = u32(w.chunk_cnt);
  ca.ranges = ranges;
  ca.vals = vals;
  ca.capacity = static_cast<uint64_t>(capacity);
  const int n_sm = sm_count();
  // persistent grids: every CTA loops over chunks, none waits on another
  const unsigned chunk_grid = static_cast<unsigned>(
      w.max_chunks < 8 * static_cast<int64_t>(n_sm) ? (w.max_chunks > 0 ? w.max_chunks : 1) : 8 * n_sm);
  chunk_count_kernel<<<chunk_grid, kChunkThreads, 0, stream>>>(ca, L, S);
  super_scan_kernel<<<static_cast<unsigned>(S.n_super), kSuperScanThreads, 0, stream>>>(ca.chunk_cnt, chunk_base, L, S,
                                                                                        u32(w.tile_cnt));
  ScanState st3{reinterpret_cast<uint64_t*>(ws + w.scan_t), tickets + 10};
  tile_scan_kernel<<<static_cast<unsigned>(w.n_tile_scan_tiles), kScanThreads, 0, stream>>>(
      u32(w.tile_cnt), L.n_tiles, st3, ranges, n_isect_dev, capacity, status_dev);
  if (capacity > 0) scatter_kernel<<<chunk_grid, kChunkThreads, 0, stream>>>(ca, L, S);
  // 2h. optional 64-bit keys, tile order
  if (keys && capacity > 0)
    keys64_kernel<<<static_cast<unsigned>(4 * n_sm), 256, 0, stream>>>(ranges, L.n_tiles, vals, projected, depth_keys,
                                                                       capacity, keys);
  if (cfg->flags & GS_FLAG_TILE_ORDER)
    tile_order_kernel<<<1, kOrderThreads, 0, stream>>>(ranges, L.n_tiles, tile_ranges + 2 * L.n_tiles);
  return cuda_status(cudaGetLastError());
}

}  // namespace
}  // namespace gs

extern "C" size_t gs_bin_sort_workspace_bytes(int64_t N, int32_t V, int64_t capacity, int64_t n_tiles) {
  if (N < 0 || V < 1 || capacity < 0 || n_tiles < 1) return 0;
  return gs::ws_layout(N, V, capacity, n_tiles).total;
}

extern "C" int gs_bin_sort(const float* projected, const int16_t* rects, const uint32_t* counts,
                           const uint32_t* depth_keys, int64_t N, const int32_t* sizes, int32_t V, const gs_config* cfg,
                           uint64_t* keys, uint32_t* vals, int64_t capacity, uint32_t* tile_ranges,
                           int64_t* n_isect_dev, void* workspace, size_t workspace_bytes, int32_t* status_dev,
                           gs_stream_t stream) {
  return gs::bin_sort_impl(projected, rects, counts, depth_keys, N, sizes, V, cfg, keys, vals, capacity, tile_ranges, n_isect_dev,
                           workspace, workspace_bytes, status_dev, reinterpret_cast<cudaStream_t>(stream), 1);
}

extern "C" size_t gs_bin_sort_partitioned_workspace_bytes(int64_t N, int32_t V, int64_t capacity, int64_t n_tiles,
                                                          int32_t partitions) {
  if (N < 0 || V < 1 || capacity < 0 || n_tiles < 1 || !gs::valid_partitions(partitions)) return 0;
  return gs::ws_layout(N, V, capacity, n_tiles, partitions).total;
}

extern "C" int gs_bin_sort_partitioned(const float* projected, const int16_t* rects, const uint32_t* counts,
                                       const uint32_t* depth_keys, int64_t N, const int32_t* sizes, int32_t V,
                                       const gs_config* cfg, uint64_t* keys, uint32_t* vals, int64_t capacity,
                                       uint32_t* tile_ranges, int64_t* n_isect_dev, int32_t partitions,
                                       void* workspace, size_t workspace_bytes, int32_t* status_dev,
                                       gs_stream_t stream) {
  return gs::bin_sort_impl(projected, rects, counts, depth_keys, N, sizes, V, cfg, keys, vals, capacity, tile_ranges, n_isect_dev,
                           workspace, workspace_bytes, status_dev, reinterpret_cast<cudaStream_t>(stream), partitions);
}

// Tile keys and depth sort: CUB-free onesweep radix sorts producing, per
// image tile, the list of intersecting splats in (depth, index) order.
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
// order. It is reached in two smaller sorts:
//   1. compact the visible records and sort them by depth bits (4 passes over
//      32-bit keys; stability keeps equal depths in record-index order);
//   2. emit one (tile id, record) pair per covered tile, records in depth
//      order, and stably sort the pairs by tile id (ceil(log2 tiles / 8)
//      passes over 32-bit keys).
// Within a tile the entries then run in (depth, record) order, exactly the
// order of the 64-bit key sort, while the large list (one entry per tile
// intersection) goes through 2 passes of 16 bytes per entry instead of 6
// passes of 24 bytes.
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
constexpr int kMaxTilePasses = 4;

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
// projected record.
__global__ void __launch_bounds__(kScanThreads) compact_visible_kernel(
    const uint32_t* __restrict__ counts, const float* __restrict__ projected, const uint32_t* __restrict__ depth_keys,
    int64_t n, uint32_t index_base, ScanState st, uint32_t* __restrict__ dkeys, uint32_t* __restrict__ dvals,
    uint32_t* __restrict__ hist, int64_t* n_visible, int32_t* status) {
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_warp[kScanThreads / 32];
  __shared__ uint64_t s_prefix;
  __shared__ uint32_t s_hist[kDepthPasses][kRadix];
  const int tid = threadIdx.x;
  for (int i = tid; i < kDepthPasses * kRadix; i += kScanThreads) (&s_hist[0][0])[i] = 0;
  if (tid == 0) s_tile = atomicAdd(st.ticket, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const int64_t base = static_cast<int64_t>(t) * kScanTile + static_cast<int64_t>(tid) * kScanItems;
  uint32_t vis = 0;  // bit i: item i visible
  uint32_t dkey[kScanItems];
  if (depth_keys) {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      dkey[i] = base + i < n ? depth_keys[base + i] : 0u;
      if (dkey[i] != 0u) vis |= 1u << i;
    }
  } else {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      dkey[i] = 0u;
      if (base + i < n && counts[base + i] > 0) vis |= 1u << i;
    }
  }
  const uint64_t pos0 = block_scan_lookback(__popc(vis), t, st, s_warp, &s_prefix, status);
  uint64_t pos = pos0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (vis & (1u << i)) {
      const uint32_t d = depth_keys ? dkey[i] : __float_as_uint(projected[(base + i) * kRecordFloats + 6]);
      dkeys[pos] = d;
      dvals[pos] = index_base + static_cast<uint32_t>(base + i);
#pragma unroll
      for (int p = 0; p < kDepthPasses; ++p) atomicAdd(&s_hist[p][(d >> (8 * p)) & 0xffu], 1u);
      ++pos;
    }
  }
  if (n > 0 && base <= n - 1 && n - 1 < base + kScanItems) *n_visible = static_cast<int64_t>(pos);
  __syncthreads();
  for (int i = tid; i < kDepthPasses * kRadix; i += kScanThreads) {
    const uint32_t c = (&s_hist[0][0])[i];
    if (c) atomicAdd(hist + i, c);
  }
}

// ---------------------------------------------------------------------------
// 1c + 2a. Tile-count offsets in depth order and emission in one kernel.
//     Each CTA takes a tile of 1024 depth-sorted records by ticket, scans
//     their tile counts (block scan + decoupled look-back, clamped at the
//     capacity), then expands them one warp per 32 records, load-balanced:
//     the warp scans the records' counts, and lane l produces entries l,
//     l + 32, ... of the warp's concatenated output, finding the record of
//     each entry from the record starts of the round. All lanes stay busy
//     whatever the record sizes, and each warp store writes 32 consecutive
//     positions except at record boundaries. The tile-id digit histograms of
//     the tile passes are gathered on the way with shared atomics.
// ---------------------------------------------------------------------------
constexpr int kEmitThreads = 256;
static_assert(kEmitThreads == kScanThreads, "the emission scans its records with the block scan");
constexpr int kEmitItems = 4;                              // records per thread in the count scan
constexpr int kEmitTile = kEmitThreads * kEmitItems;       // records per emission tile
constexpr int kEmitGroups = kEmitTile / 32;                // 32-record groups per tile

__global__ void __launch_bounds__(kEmitThreads) emit_tiles_kernel(
    const uint32_t* __restrict__ order, const int64_t* n_visible, const uint32_t* __restrict__ counts,
    const short4* __restrict__ rects, int64_t N, const Layout L, uint64_t capacity, int tile_passes, ScanState st,
    uint32_t* __restrict__ tkeys, uint32_t* __restrict__ tvals, uint32_t* __restrict__ hist, int64_t* n_total,
    int32_t* status) {
  __shared__ uint32_t s_hist[kMaxTilePasses][kRadix];
  __shared__ uint32_t s_vg[kEmitTile], s_cnt[kEmitTile], s_off[kEmitTile];
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_warp[kScanThreads / 32];
  __shared__ uint64_t s_prefix;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) s_tile = atomicAdd(st.ticket, 1u);
  for (int i = tid; i < kMaxTilePasses * kRadix; i += kEmitThreads) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t t = s_tile;
  const int64_t n = *n_visible;
  const int64_t tile0 = static_cast<int64_t>(t) * kEmitTile;
  if (tile0 >= n) return;  // past the data: publishes nothing, awaited by nobody
  // 1. the tile's records (depth order) and their tile counts, scanned with
  //    decoupled look-back: output offsets, clamped at the capacity
  const int64_t base = tile0 + static_cast<int64_t>(tid) * kEmitItems;
  uint32_t c[kEmitItems];
  uint64_t local = 0;
#pragma unroll
  for (int i = 0; i < kEmitItems; ++i) {
    const uint32_t vg = base + i < n ? order[base + i] : 0u;
    c[i] = base + i < n ? counts[vg] : 0u;
    s_vg[tid * kEmitItems + i] = vg;
    s_cnt[tid * kEmitItems + i] = c[i];
    local += c[i];
  }
  uint64_t run = block_scan_lookback(local, t, st, s_warp, &s_prefix, status);
#pragma unroll
  for (int i = 0; i < kEmitItems; ++i) {
    s_off[tid * kEmitItems + i] = static_cast<uint32_t>(run < capacity ? run : capacity);
    run += c[i];
  }
  if (base <= n - 1 && n - 1 < base + kEmitItems) {
    *n_total = static_cast<int64_t>(run);
    if (run > capacity) set_status(status, GS_STATUS_CAPACITY);
  }
  __syncthreads();
  // 2. emission, one warp per group of 32 records, load-balanced: the warp
  //    scans the records' counts, and lane l produces entries l, l + 32, ...
  //    of the group's concatenated output, finding the record of each entry
  //    from the record starts of the round. The tile-id digit histograms of
  //    the tile passes are gathered on the way with shared atomics.
  const float invN = 1.0f / static_cast<float>(N);
  for (int g = tid >> 5; g < kEmitGroups && capacity > 0; g += kEmitThreads / 32) {
    const int r = g * 32 + lane;
    const int64_t j = tile0 + r;
    uint32_t vg = 0, cnt = 0, tb = 0, xy = 0, wn = 1;
    if (j < n) {
      vg = s_vg[r];
      cnt = s_cnt[r];
      const short4 rc = rects[vg];
      // view index v = vg / N by float quotient and exact fix-up (one view: 0)
      int v = 0;
      if (L.V > 1) {
        v = __float2int_rz(static_cast<float>(vg) * invN);
        while (v > 0 && static_cast<int64_t>(v) * N > static_cast<int64_t>(vg)) --v;
        while (static_cast<int64_t>(v + 1) * N <= static_cast<int64_t>(vg)) ++v;
      }
      tb = L.tile_base[v];
      // packed record fields: (x0, y0) and (width, tiles per row), 16 bits each
      xy = static_cast<uint32_t>(static_cast<uint16_t>(rc.x)) | (static_cast<uint32_t>(static_cast<uint16_t>(rc.y)) << 16);
      wn = static_cast<uint32_t>(rc.z - rc.x) | (static_cast<uint32_t>(L.ntx[v]) << 16);
    }
    // exclusive prefix of the counts within the group; the group's entries are
    // contiguous in the output from its first record's offset
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
    uint32_t started = 0;  // records (lanes) whose entries start before this round
    for (uint32_t eb = 0; eb < total; eb += 32) {
      // bit i: a record's first entry is entry eb + i (records have count >= 1,
      // so the starts are distinct); the record of entry eb + lane is the
      // last one started at or before it
      const uint32_t stb = (cnt > 0 && excl >= eb && excl - eb < 32u) ? (1u << (excl - eb)) : 0u;
      const uint32_t starts = __reduce_or_sync(0xffffffffu, stb);
      const int src = static_cast<int>(started + __popc(starts & le_mask)) - 1;
      started += __popc(starts);
      const uint32_t e = eb + lane;
      const uint32_t k = e - __shfl_sync(0xffffffffu, excl, src);
      const uint32_t r_vg = __shfl_sync(0xffffffffu, vg, src);
      const uint32_t r_xy = __shfl_sync(0xffffffffu, xy, src);
      const uint32_t r_wn = __shfl_sync(0xffffffffu, wn, src);
      const uint32_t r_tb = L.V > 1 ? __shfl_sync(0xffffffffu, tb, src) : tb;
      const uint64_t pos = out_base + e;
      if (e < total && pos < capacity) {
        const int r_w = static_cast<int>(r_wn & 0xffffu);
        const uint32_t r_ntx = r_wn >> 16;
        const int r_x0 = static_cast<int16_t>(r_xy & 0xffffu), r_y0 = static_cast<int16_t>(r_xy >> 16);
        // k = row * w + col: quotient from the approximate reciprocal, then an
        // exact fix-up (the estimate is off by at most one)
        int row = __float2int_rz(static_cast<float>(k) * rcp_approx(static_cast<float>(r_w)));
        int col = static_cast<int>(k) - row * r_w;
        if (col < 0) { --row; col += r_w; }
        if (col >= r_w) { ++row; col -= r_w; }
        const uint32_t tile = r_tb + static_cast<uint32_t>(r_y0 + row) * r_ntx + static_cast<uint32_t>(r_x0 + col);
        tkeys[pos] = tile;
        tvals[pos] = r_vg;
        for (int p = 0; p < tile_passes; ++p) atomicAdd(&s_hist[p][(tile >> (8 * p)) & 0xffu], 1u);
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < tile_passes * kRadix; i += kEmitThreads) {
    const uint32_t cc = (&s_hist[0][0])[i];
    if (cc) atomicAdd(hist + i, cc);
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
  uint2* ranges;             // last tile-id pass: per-key (~first, last + 1) bounds, else null
  uint32_t n_keys;           // ranges has n_keys entries
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
        if (k < a.n_keys) {
          if (idx == 0 || sm.keys[idx - 1] != k) atomicMax(&a.ranges[k].x, ~p);
          if (idx == n_valid - 1 || sm.keys[idx + 1] != k) atomicMax(&a.ranges[k].y, p + 1);
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

// With fixup, the starts of the non-empty tiles come complemented from the
// last tile-id pass and are restored here first (ranges_fixup_kernel's job).
__global__ void __launch_bounds__(kOrderThreads) tile_order_kernel(uint2* __restrict__ ranges, int64_t n_tiles,
                                                                   uint32_t* __restrict__ order, int fixup) {
  __shared__ uint32_t s_cnt[kOrderBuckets];
  const int tid = threadIdx.x;
  if (tid < kOrderBuckets) s_cnt[tid] = 0;
  __syncthreads();
  for (int64_t t = tid; t < n_tiles; t += kOrderThreads) {
    uint2 r = ranges[t];
    if (fixup && r.y) {
      r.x = ~r.x;
      ranges[t].x = r.x;
    }
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

// Tile ranges from the sorted tile ids (ranges zeroed beforehand): four ids
// per thread from one 16-byte load; a range starts where the id differs from
// its predecessor and ends where it differs from its successor.
__global__ void tile_ranges_kernel(const uint32_t* __restrict__ tkeys, const int64_t* n_total, int64_t capacity,
                                   uint32_t n_tiles, uint2* __restrict__ ranges, int32_t* status) {
  int64_t n = *n_total;
  if (n > capacity) n = capacity;
  const int64_t n4 = (n + 3) / 4;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < n4;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i0 = 4 * q;
    uint32_t k[4];
    if (i0 + 3 < n) {
      const uint4 v = reinterpret_cast<const uint4*>(tkeys)[q];
      k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
    } else {
      for (int j = 0; j < 4; ++j) k[j] = i0 + j < n ? tkeys[i0 + j] : 0xffffffffu;
    }
    uint32_t prev = i0 > 0 ? tkeys[i0 - 1] : 0xffffffffu;
    const uint32_t next = i0 + 4 < n ? tkeys[i0 + 4] : 0xffffffffu;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t i = i0 + j;
      if (i >= n) break;
      const uint32_t t = k[j];
      const uint32_t nx = j < 3 ? (i + 1 < n ? k[j + 1] : 0xffffffffu) : next;
      if (t >= n_tiles) {
        set_status(status, GS_STATUS_BOUNDS);
      } else {
        if (t != prev) ranges[t].x = static_cast<uint32_t>(i);
        if (t != nx) ranges[t].y = static_cast<uint32_t>(i + 1);
      }
      prev = t;
    }
  }
}

// Ranges left by the last tile-id pass: a non-empty tile holds (~start, end);
// empty tiles stay (0, 0).
__global__ void ranges_fixup_kernel(uint2* __restrict__ ranges, int64_t n_tiles) {
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < n_tiles;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint2 r = ranges[t];
    if (r.y) ranges[t].x = ~r.x;
  }
}

// Optional 64-bit keys (tile << 32) | bits(depth) of the sorted list.
__global__ void keys64_kernel(const uint32_t* __restrict__ tkeys, const uint32_t* __restrict__ vals,
                              const float* __restrict__ projected, const int64_t* n_total, int64_t capacity,
                              uint64_t* __restrict__ keys) {
  int64_t n = *n_total;
  if (n > capacity) n = capacity;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t d = __float_as_uint(projected[static_cast<int64_t>(vals[i]) * kRecordFloats + 6]);
    keys[i] = (static_cast<uint64_t>(tkeys[i]) << 32) | d;
  }
}

// ---------------------------------------------------------------------------
// Workspace layout.
// ---------------------------------------------------------------------------
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int tile_passes_for(int64_t n_tiles) {
  int bits = 0;
  while ((int64_t(1) << bits) < n_tiles) ++bits;
  return (bits + 7) / 8;
}

struct WsLayout {
  size_t dkeys0, dvals0, dkeys1, dvals1, tkeys0, tkeys1, tvals_alt;
  size_t zero_begin, scan1, scan2, hist_d, hist_t, tickets, n_visible, lb_depth, lb_tile;
  size_t part_scan, part_hist, part_tickets, part_n, part_lb, zero_end, total;
  int64_t n_scan_tiles, n_emit_tiles, n_depth_tiles, n_tile_tiles;
  int64_t part_stride, part_scan_tiles, part_sort_tiles;
  int tile_passes;
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
  w.tile_passes = tile_passes_for(n_tiles);
  w.n_scan_tiles = (VN + kScanTile - 1) / kScanTile;
  w.n_depth_tiles = (VN + kSortTile - 1) / kSortTile;
  w.n_tile_tiles = (capacity + kSortTile - 1) / kSortTile;
  w.part_scan_tiles = (w.part_stride + kScanTile - 1) / kScanTile;
  w.part_sort_tiles = (w.part_stride + kSortTile - 1) / kSortTile;
  size_t o = 0;
  w.dkeys0 = o; o = align256(o + 4 * ds);
  w.dvals0 = o; o = align256(o + 4 * ds);
  w.dkeys1 = o; o = align256(o + 4 * ds);
  w.dvals1 = o; o = align256(o + 4 * ds);
  w.tkeys0 = o; o = align256(o + 4 * cap);
  w.tkeys1 = o; o = align256(o + 4 * cap);
  w.tvals_alt = o; o = align256(o + 4 * cap);
  w.zero_begin = o;
  w.scan1 = o; o = align256(o + 8 * static_cast<size_t>(w.n_scan_tiles + 1));
  w.n_emit_tiles = (VN + kEmitTile - 1) / kEmitTile;
  w.scan2 = o; o = align256(o + 8 * static_cast<size_t>(w.n_emit_tiles + 1));
  w.hist_d = o; o = align256(o + 4 * kDepthPasses * kRadix);
  w.hist_t = o; o = align256(o + 4 * kMaxTilePasses * kRadix);
  w.tickets = o; o = align256(o + 4 * 16);
  w.n_visible = o; o = align256(o + 8);
  w.lb_depth = o; o = align256(o + 8 * kRadix * kDepthPasses * static_cast<size_t>(w.n_depth_tiles + 1));
  w.lb_tile = o; o = align256(o + 8 * kRadix * static_cast<size_t>(w.tile_passes) * static_cast<size_t>(w.n_tile_tiles + 1));
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
    a.ranges = nullptr; a.n_keys = 0;
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
      tile_order_kernel<<<1, kOrderThreads, 0, stream>>>(reinterpret_cast<uint2*>(tile_ranges), L.n_tiles,
                                                         tile_ranges + 2 * L.n_tiles, 0);
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
      a.ranges = nullptr; a.n_keys = 0;
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
  // 1c + 2a. tile-count offsets in depth order and emission, one kernel; the
  //     buffers are chosen so that the last tile pass writes the values into
  //     `vals`
  ScanState st2{reinterpret_cast<uint64_t*>(ws + w.scan2), tickets + 1};
  const int TP = w.tile_passes;
  uint32_t* tk[2] = {u32(w.tkeys0), u32(w.tkeys1)};
  uint32_t* tv[2];
  tv[TP & 1] = vals;
  tv[(TP + 1) & 1] = u32(w.tvals_alt);
  uint32_t* hist_t = u32(w.hist_t);
  const int n_sm = sm_count();
  emit_tiles_kernel<<<static_cast<unsigned>(w.n_emit_tiles), kEmitThreads, 0, stream>>>(
      order, n_visible, counts, reinterpret_cast<const short4*>(rects), N, L, static_cast<uint64_t>(capacity), TP, st2,
      capacity > 0 ? tk[0] : nullptr, capacity > 0 ? tv[0] : nullptr, hist_t, n_isect_dev, status_dev);
  if (capacity == 0) {
    if (cfg->flags & GS_FLAG_TILE_ORDER)
      tile_order_kernel<<<1, kOrderThreads, 0, stream>>>(reinterpret_cast<uint2*>(tile_ranges), L.n_tiles,
                                                         tile_ranges + 2 * L.n_tiles, 0);
    return cuda_status(cudaGetLastError());
  }
  // 2b. stable tile-id passes
  for (int p = 0; p < TP; ++p) {
    PassArgs a;
    a.keys_in = tk[p & 1]; a.vals_in = tv[p & 1]; a.keys_out = tk[(p + 1) & 1]; a.vals_out = tv[(p + 1) & 1];
    a.ranges = nullptr; a.n_keys = 0;
    if (p == TP - 1) {
      // the last pass bounds the tile ranges itself; it writes the ids only
      // when the 64-bit keys are asked for
      a.ranges = reinterpret_cast<uint2*>(tile_ranges);
      a.n_keys = static_cast<uint32_t>(L.n_tiles);
      if (!keys) a.keys_out = nullptr;
    }
    a.n_total = n_isect_dev; a.cap = capacity; a.shift = 8 * p; a.digit_offsets = hist_t + p * kRadix;
    a.scan_digits = 1;  // the counts gathered by the emission
    a.ticket = tickets + 6 + p;
    a.stall_tile = -1;
    a.spin_limit = kSpinLimit;
    a.lookback = reinterpret_cast<uint64_t*>(ws + w.lb_tile) + static_cast<size_t>(p) * (w.n_tile_tiles + 1) * kRadix;
    int bits = 8;
    if (p == TP - 1) {
      bits = 0;
      while ((int64_t(1) << bits) < L.n_tiles) ++bits;
      bits -= 8 * (TP - 1);
    }
    const unsigned grid = sort_grid(w.n_tile_tiles);
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
  const uint32_t* tkeys_final = tk[TP & 1];
  // 2c. tile ranges (from the ids themselves when there is no tile pass),
  //     optional 64-bit keys
  // (with a tile order the order kernel restores the starts itself)
  const bool ordered = (cfg->flags & GS_FLAG_TILE_ORDER) != 0;
  if (TP > 0 && !ordered)
    ranges_fixup_kernel<<<static_cast<unsigned>((L.n_tiles + 255) / 256), 256, 0, stream>>>(
        reinterpret_cast<uint2*>(tile_ranges), L.n_tiles);
  else if (TP == 0)
    tile_ranges_kernel<<<static_cast<unsigned>(4 * n_sm), 256, 0, stream>>>(
        tkeys_final, n_isect_dev, capacity, static_cast<uint32_t>(L.n_tiles), reinterpret_cast<uint2*>(tile_ranges),
        status_dev);
  if (keys)
    keys64_kernel<<<static_cast<unsigned>(4 * n_sm), 256, 0, stream>>>(tkeys_final, vals, projected, n_isect_dev,
                                                                        capacity, keys);
  if (ordered)
    tile_order_kernel<<<1, kOrderThreads, 0, stream>>>(reinterpret_cast<uint2*>(tile_ranges), L.n_tiles,
                                                       tile_ranges + 2 * L.n_tiles, TP > 0 ? 1 : 0);
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

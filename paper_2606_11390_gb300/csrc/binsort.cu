// Tile keys and depth sort: scan of per-record tile counts, key emission,
// CUB-free onesweep LSD radix sort, tile ranges.
//
// Paper: arXiv 2606.11390 §4 (each camera's Gaussians are depth-sorted before
// rasterisation; the multi-GPU merge of §4 is not needed on one GPU) and §3.2
// (the paper's sort is CUB's radix sort, Merrill & Grimshaw 2011). The sort
// here follows the onesweep scheme (Adinets & Merrill 2022): one upfront pass
// builds the digit histograms of all passes, then each 8-bit digit pass is a
// single read and write of the keys in which every tile of 4096 keys finds
// its global digit offsets by decoupled look-back over its predecessors.
// Tiles take their position from an atomic ticket, so a tile only waits on
// tiles that are already running; every wait is bounded (GS_STATUS_TIMEOUT).
//
// Keys: (global tile id << 32) | float bits of depth (depth > 0, so the bits
// order like the values). Emission order is (view, Gaussian, row-major tile),
// and every pass is stable, so equal keys stay in Gaussian-index order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

// ---------------------------------------------------------------------------
// Exclusive scan of counts -> offsets (clamped at capacity), decoupled look-back.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagIncl = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;

struct ScanState {
  uint64_t* tiles;   // [n_tiles] flag | value
  uint32_t* ticket;  // [1]
};

__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Look-back for tile `t` (t >= 1) by one warp; returns the exclusive prefix.
__device__ uint64_t lookback_warp(const uint64_t* tiles, uint32_t t, int32_t* status) {
  const int lane = threadIdx.x & 31;
  uint64_t prefix = 0;
  int64_t base = static_cast<int64_t>(t) - 1;
  uint32_t spins = 0;
  while (base >= 0) {
    const int64_t j = base - lane;
    uint64_t s = j >= 0 ? ld_relaxed_u64(tiles + j) : kFlagIncl;
    // wait until every lane sees a published value
    while (__any_sync(0xffffffffu, (s >> 62) == 0)) {
      if (++spins > kSpinLimit) {
        set_status(status, GS_STATUS_TIMEOUT);
        return prefix;
      }
      if ((s >> 62) == 0) s = ld_relaxed_u64(tiles + j);
    }
    const uint32_t incl = __ballot_sync(0xffffffffu, (s >> 62) == 2);
    // sum values of lanes up to and including the first inclusive one
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

__global__ void __launch_bounds__(kScanThreads) scan_counts_kernel(const uint32_t* __restrict__ counts, int64_t n,
                                                                     uint32_t* __restrict__ offsets, uint64_t capacity,
                                                                     ScanState st, int64_t* n_total, int32_t* status) {
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_warp[kScanThreads / 32];
  __shared__ uint64_t s_prefix;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(st.ticket, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const int64_t base = static_cast<int64_t>(t) * kScanTile + static_cast<int64_t>(tid) * kScanItems;
  uint32_t c[kScanItems];
  uint64_t local = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    c[i] = (base + i < n) ? counts[base + i] : 0u;
    local += c[i];
  }
  // block scan of per-thread sums
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
        s_prefix = 0;
      }
    } else {
      if (lane == 0) st_relaxed_u64(st.tiles + t, kFlagAgg | block_total);
      const uint64_t p = lookback_warp(st.tiles, t, status);
      if (lane == 0) {
        st_relaxed_u64(st.tiles + t, kFlagIncl | (p + block_total));
        s_prefix = p;
      }
    }
  }
  __syncthreads();
  uint64_t run = s_prefix + excl_thread;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) offsets[base + i] = static_cast<uint32_t>(run < capacity ? run : capacity);
    run += c[i];
  }
  // the tile holding the last element reports the total
  if (n > 0 && base <= n - 1 && n - 1 < base + kScanItems) {
    *n_total = static_cast<int64_t>(run);
    if (run > capacity) set_status(status, GS_STATUS_CAPACITY);
  }
}

// ---------------------------------------------------------------------------
// Key emission: one thread per record, keys of its rectangle in row-major order.
// ---------------------------------------------------------------------------
__global__ void emit_keys_kernel(const float4* __restrict__ projected, const short4* __restrict__ rects,
                                 const uint32_t* __restrict__ counts, const uint32_t* __restrict__ offsets, int64_t N,
                                 const Layout L, uint64_t capacity, uint64_t* __restrict__ keys,
                                 uint32_t* __restrict__ vals) {
  const int64_t vg = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t VN = N * L.V;
  if (vg >= VN) return;
  const uint32_t cnt = counts[vg];
  if (cnt == 0) return;
  const int v = static_cast<int>(vg / N);
  const short4 r = rects[vg];
  const uint32_t depth_bits = __float_as_uint(projected[3 * vg + 1].z);
  uint64_t pos = offsets[vg];
  const uint32_t tb = L.tile_base[v];
  const int ntx = L.ntx[v];
  for (int ty = r.y; ty < r.w; ++ty) {
    for (int tx = r.x; tx < r.z; ++tx) {
      if (pos >= capacity) return;
      const uint64_t tile = tb + static_cast<uint32_t>(ty * ntx + tx);
      keys[pos] = (tile << 32) | depth_bits;
      vals[pos] = static_cast<uint32_t>(vg);
      ++pos;
    }
  }
}

// ---------------------------------------------------------------------------
// Onesweep radix sort.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys
constexpr int kRadix = 256;
constexpr int kMaxPasses = 8;

struct SortWork {
  uint32_t* hist;       // [kMaxPasses][256] digit counts
  uint32_t* tickets;    // [kMaxPasses]
  uint64_t* lookback;   // [kMaxPasses][n_tiles][256]
  int64_t n_tiles;      // sort tiles for the capacity
};

__device__ __forceinline__ int64_t clamp_n(const int64_t* n_total, int64_t capacity) {
  const int64_t n = *n_total;
  return n < capacity ? n : capacity;
}

// Histogram of every digit position for all passes in one read of the keys.
__global__ void __launch_bounds__(kSortThreads) sort_histogram_kernel(const uint64_t* __restrict__ keys,
                                                                        const int64_t* n_total, int64_t capacity,
                                                                        int passes, uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_hist[kMaxPasses][kRadix];
  for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const int64_t n = clamp_n(n_total, capacity);
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint64_t k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][(k >> (8 * p)) & 0xff], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    const uint32_t c = (&s_hist[0][0])[i];
    if (c) atomicAdd(hist + i, c);
  }
}

// Exclusive scan of each pass's 256 digit counts, in place (one block).
__global__ void sort_hist_scan_kernel(uint32_t* hist, int passes) {
  __shared__ uint32_t s[kRadix];
  const int d = threadIdx.x;
  for (int p = 0; p < passes; ++p) {
    s[d] = hist[p * kRadix + d];
    __syncthreads();
    // Hillis-Steele inclusive scan over 256 entries
    for (int o = 1; o < kRadix; o <<= 1) {
      const uint32_t v = d >= o ? s[d - o] : 0u;
      __syncthreads();
      s[d] += v;
      __syncthreads();
    }
    hist[p * kRadix + d] = d > 0 ? s[d - 1] : 0u;
    __syncthreads();
  }
}

struct __align__(16) SortSmem {
  uint64_t keys[kSortTile];             // 32 KB
  uint32_t vals[kSortTile];             // 16 KB
  uint32_t warp_hist[kSortWarps][kRadix];  // 8 KB
  uint32_t local_start[kRadix];
  int64_t base[kRadix];                 // global position of this tile's first key of each digit, minus local start
  uint32_t tile;
};

__global__ void __launch_bounds__(kSortThreads) sort_pass_kernel(const uint64_t* __restrict__ keys_in,
                                                                   const uint32_t* __restrict__ vals_in,
                                                                   uint64_t* __restrict__ keys_out,
                                                                   uint32_t* __restrict__ vals_out,
                                                                   const int64_t* n_total, int64_t capacity, int pass,
                                                                   SortWork W, int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem& sm = *reinterpret_cast<SortSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int shift = 8 * pass;
  const int64_t n = clamp_n(n_total, capacity);
  if (tid == 0) sm.tile = atomicAdd(W.tickets + pass, 1u);
  for (int i = tid; i < kSortWarps * kRadix; i += kSortThreads) (&sm.warp_hist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t t = sm.tile;
  const int64_t tile_start = static_cast<int64_t>(t) * kSortTile;
  if (tile_start >= n) return;  // tiles past the data publish nothing and nobody waits on them
  const int n_valid = static_cast<int>(n - tile_start < kSortTile ? n - tile_start : kSortTile);

  // 1. load (warp-striped) and rank within each warp, stably
  uint64_t key[kSortItems];
  uint32_t val[kSortItems];
  uint32_t rank[kSortItems];
  const int warp_base = warp * 32 * kSortItems;
  const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int li = warp_base + i * 32 + lane;
    const bool valid = li < n_valid;
    key[i] = valid ? keys_in[tile_start + li] : 0ull;
    val[i] = valid ? vals_in[tile_start + li] : 0u;
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    rank[i] = 0;
    if (valid) {
      const uint32_t d = static_cast<uint32_t>(key[i] >> shift) & 0xffu;
      const uint32_t peers = __match_any_sync(vmask, d);
      const int leader = __ffs(peers) - 1;
      uint32_t before = 0;
      if (lane == leader) before = sm.warp_hist[warp][d];
      before = __shfl_sync(vmask, before, leader);
      rank[i] = before + __popc(peers & lt_mask);
      if (lane == leader) sm.warp_hist[warp][d] = before + __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();

  // 2. per digit: offsets of each warp, tile total; publish and look back
  const int d = tid;  // kSortThreads == kRadix
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const uint32_t c = sm.warp_hist[w][d];
    sm.warp_hist[w][d] = total;
    total += c;
  }
  uint64_t* lb = W.lookback + (static_cast<int64_t>(pass) * W.n_tiles) * kRadix;
  if (t == 0) st_relaxed_u64(lb + d, kFlagIncl | total);
  else st_relaxed_u64(lb + static_cast<int64_t>(t) * kRadix + d, kFlagAgg | total);
  // local exclusive scan of tile totals over digits (block scan)
  {
    uint32_t v = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t nb = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += nb;
    }
    __shared__ uint32_t s_wsum[kSortWarps];
    if (lane == 31) s_wsum[warp] = v;
    __syncthreads();
    uint32_t add = 0;
    for (int w = 0; w < warp; ++w) add += s_wsum[w];
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
        if (++spins > kSpinLimit) {
          set_status(status, GS_STATUS_TIMEOUT);
          break;
        }
        continue;
      }
      prefix += s & kValMask;
      if (f == 2) break;
      --j;
    }
    st_relaxed_u64(lb + static_cast<int64_t>(t) * kRadix + d, kFlagIncl | (prefix + total));
  }
  const uint32_t digit_offset = W.hist[pass * kRadix + d];
  sm.base[d] = static_cast<int64_t>(digit_offset) + static_cast<int64_t>(prefix) - sm.local_start[d];
  __syncthreads();

  // 3. scatter into shared memory in local sorted order
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int li = warp_base + i * 32 + lane;
    if (li < n_valid) {
      const uint32_t dd = static_cast<uint32_t>(key[i] >> shift) & 0xffu;
      const uint32_t pos = sm.local_start[dd] + sm.warp_hist[warp][dd] + rank[i];
      sm.keys[pos] = key[i];
      sm.vals[pos] = val[i];
    }
  }
  __syncthreads();

  // 4. write out: runs of equal digits land contiguously
  for (int idx = tid; idx < n_valid; idx += kSortThreads) {
    const uint64_t k = sm.keys[idx];
    const uint32_t dd = static_cast<uint32_t>(k >> shift) & 0xffu;
    const int64_t pos = sm.base[dd] + idx;
    if (pos >= 0 && pos < n) {
      keys_out[pos] = k;
      vals_out[pos] = sm.vals[idx];
    } else {
      set_status(status, GS_STATUS_BOUNDS);
    }
  }
}

// Tile ranges from the sorted keys (ranges zeroed beforehand).
__global__ void tile_ranges_kernel(const uint64_t* __restrict__ keys, const int64_t* n_total, int64_t capacity,
                                   uint32_t n_tiles, uint2* __restrict__ ranges, int32_t* status) {
  const int64_t n = clamp_n(n_total, capacity);
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t tile = static_cast<uint32_t>(keys[i] >> 32);
    if (tile >= n_tiles) {
      set_status(status, GS_STATUS_BOUNDS);
      continue;
    }
    if (i == 0 || static_cast<uint32_t>(keys[i - 1] >> 32) != tile) ranges[tile].x = static_cast<uint32_t>(i);
    if (i == n - 1 || static_cast<uint32_t>(keys[i + 1] >> 32) != tile) ranges[tile].y = static_cast<uint32_t>(i + 1);
  }
}

// ---------------------------------------------------------------------------
// Workspace layout.
// ---------------------------------------------------------------------------
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct WsLayout {
  size_t offsets, scan_tiles, alt_keys, alt_vals, hist, tickets, lookback, total;
  size_t zero_begin, zero_end;  // region cleared at the start of every call
  int64_t n_scan_tiles, n_sort_tiles;
};

WsLayout ws_layout(int64_t N, int32_t V, int64_t capacity) {
  WsLayout w;
  const int64_t VN = N * V;
  w.n_scan_tiles = (VN + kScanTile - 1) / kScanTile;
  w.n_sort_tiles = (capacity + kSortTile - 1) / kSortTile;
  size_t o = 0;
  w.offsets = o; o = align256(o + sizeof(uint32_t) * static_cast<size_t>(VN > 0 ? VN : 1));
  w.alt_keys = o; o = align256(o + sizeof(uint64_t) * static_cast<size_t>(capacity > 0 ? capacity : 1));
  w.alt_vals = o; o = align256(o + sizeof(uint32_t) * static_cast<size_t>(capacity > 0 ? capacity : 1));
  w.zero_begin = o;
  w.scan_tiles = o; o = align256(o + sizeof(uint64_t) * static_cast<size_t>(w.n_scan_tiles + 1));
  w.hist = o; o = align256(o + sizeof(uint32_t) * kMaxPasses * kRadix);
  w.tickets = o; o = align256(o + sizeof(uint32_t) * (kMaxPasses + 1));
  w.lookback = o; o = align256(o + sizeof(uint64_t) * kMaxPasses * kRadix * static_cast<size_t>(w.n_sort_tiles + 1));
  w.zero_end = o;
  w.total = o;
  return w;
}

int num_passes(int64_t n_tiles) {
  int bits = 1;
  while ((int64_t(1) << bits) < n_tiles) ++bits;
  return 4 + (bits + 7) / 8;
}

}  // namespace
}  // namespace gs

extern "C" size_t gs_bin_sort_workspace_bytes(int64_t N, int32_t V, int64_t capacity, int64_t n_tiles) {
  (void)n_tiles;
  if (N < 0 || V < 1 || capacity < 0) return 0;
  return gs::ws_layout(N, V, capacity).total;
}

extern "C" int gs_bin_sort(const float* projected, const int16_t* rects, const uint32_t* counts, int64_t N,
                           const int32_t* sizes, int32_t V, const gs_config* cfg, uint64_t* keys, uint32_t* vals,
                           int64_t capacity, uint32_t* tile_ranges, int64_t* n_isect_dev, void* workspace,
                           size_t workspace_bytes, int32_t* status_dev, gs_stream_t stream_) {
  using namespace gs;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  Layout L;
  int rc = build_layout(sizes, V, cfg, &L, nullptr);
  if (rc != GS_OK) return rc;
  if (N < 0 || capacity < 0 || capacity >= (int64_t(1) << 32) - 1) return GS_ERR_ARG;
  if (N * static_cast<int64_t>(V) >= (int64_t(1) << 32)) return GS_ERR_ARG;
  if (!tile_ranges || !n_isect_dev || !workspace) return GS_ERR_ARG;
  if (N > 0 && (!projected || !rects || !counts)) return GS_ERR_ARG;
  if (capacity > 0 && (!keys || !vals)) return GS_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) & 255u) return GS_ERR_ARG;
  const WsLayout w = ws_layout(N, V, capacity);
  if (workspace_bytes < w.total) return GS_ERR_ARG;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  uint32_t* offsets = reinterpret_cast<uint32_t*>(ws + w.offsets);
  uint64_t* alt_keys = reinterpret_cast<uint64_t*>(ws + w.alt_keys);
  uint32_t* alt_vals = reinterpret_cast<uint32_t*>(ws + w.alt_vals);
  ScanState st;
  st.tiles = reinterpret_cast<uint64_t*>(ws + w.scan_tiles);
  SortWork sw;
  sw.hist = reinterpret_cast<uint32_t*>(ws + w.hist);
  sw.tickets = reinterpret_cast<uint32_t*>(ws + w.tickets);
  st.ticket = sw.tickets + kMaxPasses;
  sw.lookback = reinterpret_cast<uint64_t*>(ws + w.lookback);
  sw.n_tiles = w.n_sort_tiles;

  cudaError_t e = cudaMemsetAsync(ws + w.zero_begin, 0, w.zero_end - w.zero_begin, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * static_cast<size_t>(L.n_tiles), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n_isect_dev, 0, sizeof(int64_t), stream);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  const int64_t VN = N * V;
  if (VN == 0) return GS_OK;

  // 1. scan of counts
  scan_counts_kernel<<<static_cast<unsigned>(w.n_scan_tiles), kScanThreads, 0, stream>>>(
      counts, VN, offsets, static_cast<uint64_t>(capacity), st, n_isect_dev, status_dev);
  if (capacity == 0) return cuda_status(cudaGetLastError());
  const int passes = num_passes(L.n_tiles);
  // 2. emission into the buffer that makes the last pass land in keys/vals
  uint64_t* k0 = (passes % 2 == 0) ? keys : alt_keys;
  uint32_t* v0 = (passes % 2 == 0) ? vals : alt_vals;
  uint64_t* k1 = (passes % 2 == 0) ? alt_keys : keys;
  uint32_t* v1 = (passes % 2 == 0) ? alt_vals : vals;
  {
    const int threads = 256;
    const int64_t blocks = (VN + threads - 1) / threads;
    emit_keys_kernel<<<static_cast<unsigned>(blocks), threads, 0, stream>>>(
        reinterpret_cast<const float4*>(projected), reinterpret_cast<const short4*>(rects), counts, offsets, N, L,
        static_cast<uint64_t>(capacity), k0, v0);
  }
  // 3. histograms of all passes
  int n_sm = 148;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  }
  sort_histogram_kernel<<<static_cast<unsigned>(2 * n_sm), kSortThreads, 0, stream>>>(k0, n_isect_dev, capacity, passes,
                                                                                         sw.hist);
  sort_hist_scan_kernel<<<1, kRadix, 0, stream>>>(sw.hist, passes);
  // 4. digit passes
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(sort_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sizeof(SortSmem))) != cudaSuccess)
      return GS_ERR_CUDA;
    attr_set = true;
  }
  for (int p = 0; p < passes; ++p) {
    const uint64_t* kin = (p % 2 == 0) ? k0 : k1;
    const uint32_t* vin = (p % 2 == 0) ? v0 : v1;
    uint64_t* kout = (p % 2 == 0) ? k1 : k0;
    uint32_t* vout = (p % 2 == 0) ? v1 : v0;
    sort_pass_kernel<<<static_cast<unsigned>(w.n_sort_tiles), kSortThreads, sizeof(SortSmem), stream>>>(
        kin, vin, kout, vout, n_isect_dev, capacity, p, sw, status_dev);
  }
  // 5. tile ranges
  tile_ranges_kernel<<<static_cast<unsigned>(4 * n_sm), 256, 0, stream>>>(keys, n_isect_dev, capacity,
                                                                            static_cast<uint32_t>(L.n_tiles),
                                                                            reinterpret_cast<uint2*>(tile_ranges),
                                                                            status_dev);
  return cuda_status(cudaGetLastError());
}

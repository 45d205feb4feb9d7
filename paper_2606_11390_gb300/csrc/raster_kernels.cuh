// Tile rasterisation kernels: front-to-back alpha compositing (forward) and
// its reverse-order backward. Included by raster.cu (entry points and
// dispatch) and by the raster_inst_*.cu units, which instantiate the
// launchers for every tile shape, pixels per thread and splat batch size.
//
// Paper: arXiv 2606.11390 §4 - rasterisation is partitioned per camera (or per
// image tile), and its backward keeps the forward partitioning and sums the
// per-Gaussian gradients with atomics (device scope suffices on one GPU).
// Compositing rule of 3D Gaussian Splatting (Kerbl et al. 2023): per pixel,
// for the tile's depth-sorted entries, alpha = min(cap, o exp(-power)),
// skip alpha < alpha_min, stop before T(1 - alpha) < t_stop, C += c alpha T.
//
// GB300 design. One CTA per (view, tile); each thread owns PPT pixels of one
// column (4 by default: a warp covers a 16x8 block; 2 for 8x8 tiles or on
// request: 8x8 blocks). The tile's splats are staged into shared memory 128 at
// a time; while staging, each splat gets a bitmask of the warps whose block
// meets the ellipse on which its alpha can reach alpha_min (exact
// ellipse-rectangle test with a safety margin), so a warp skips splats that
// cannot touch its pixels. Skipped pairs are pairs the compositing rule would
// skip anyway, so the result is unchanged. The per-pixel step has no
// branches: every lane evaluates the splat and the decisions select, so a
// thread's pixels interleave; the forward steps them two at a time in packed
// f32x2 operations (one issue slot for two pixels' adds, multiplies and
// FMAs). The per-pair arithmetic is written with explicitly rounded
// operations and a fixed ex2.approx so that the backward recomputes
// bit-identical alphas and takes exactly the forward's skip / stop
// decisions. The backward walks the list in reverse, each warp from the
// largest `last` among its pixels, recovers T_k = T_{k+1} / (1 - alpha_k) from
// the stored final T, sums a splat's 9 gradient values over the thread's
// pixels (the geometric ones as dy-moments, the pixels sharing dx), reduces
// them across the warp with a reduce-scatter (two splats' 18 values with 20
// shuffles; a lone splat's 9 with 12, instead of 9 x 5 butterfly
// shuffles), sums the warps of the CTA in shared memory and issues
// one FP32 atomic per value per (tile, splat) to the per-record gradient
// buffer.
//
// Template parameters: tile shape TW x TH, pixels per thread PPT, splats
// staged per shared-memory batch B (any power of two from 32 to 512; a batch
// may hold fewer splats than the CTA has threads), and COUNT, which compiles
// a variant that also counts the pixel-splat pairs it executes, evaluates and
// composites (same arithmetic and results; never used in a timed step).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_common.cuh"
#include "gs_internal.h"
#include "raster_launch.h"

namespace gs {
namespace rast {

constexpr float kLog2e = 1.4426950408889634f;

// Splat data staged in shared memory, with the conic pre-scaled so that
// e = (A' dx + B' dy) dx + C' dy dy = -power * log2(e).
struct SplatS {
  float4 a;  // mean.x, mean.y, A' = -0.5 A log2e, B' = -B log2e
  float4 b;  // C' = -0.5 C log2e, opacity, r, g
  float c;   // b
};

__device__ __forceinline__ void load_splat(const float4* __restrict__ projected, uint32_t vg, float4& a, float4& b,
                                           float& c) {
  const float4 r0 = __ldg(projected + 3 * static_cast<size_t>(vg));
  const float4 r1 = __ldg(projected + 3 * static_cast<size_t>(vg) + 1);
  const float4 r2 = __ldg(projected + 3 * static_cast<size_t>(vg) + 2);
  a = make_float4(r0.x, r0.y, -0.5f * kLog2e * r0.z, -kLog2e * r0.w);
  b = make_float4(-0.5f * kLog2e * r1.x, r1.y, r2.x, r2.y);
  c = r2.z;
}

// e = -power*log2(e) = A' dx^2 + B' dx dy + C' dy^2 for pixel centre
// (px, py), dx = px - mean.x, dy = py - mean.y. A thread's pixels share a
// column, so the dx terms are formed once per splat (SplatCol) and each pixel
// adds dy * (C' dy + B' dx) to A' dx^2: one subtraction and two FMAs. Every
// operation is explicitly rounded so the forward and the backward compute
// the same bits.
struct SplatCol {
  float dx, adx2, bdx;
};

__device__ __forceinline__ SplatCol splat_column(float px, const float4& a) {
  SplatCol c;
  c.dx = __fsub_rn(px, a.x);
  c.adx2 = __fmul_rn(__fmul_rn(a.z, c.dx), c.dx);
  c.bdx = __fmul_rn(a.w, c.dx);
  return c;
}

// Resident warps per SM the 4-pixel backward is compiled for (0: no register
// cap). Uncapped it takes 96 registers at 32x16 tiles (5 CTAs of 128
// threads); capped for 24 warps it takes 80 (6 CTAs, 4-8 bytes of spills)
// and runs 1.322 -> 1.287 ms at 4K. At 2 pixels a thread the same cap
// raises the count the compiler picks (70 -> 77 registers at 16x16 tiles,
// 7 -> 6 CTAs, 10.57 -> 10.73 ms on 16 views), so those stay uncapped: a
// minimum of 0 CTAs leaves the count to the compiler as if none were given
// (a minimum of 1 would let it grow to 87-93 registers there).
#ifndef GS_RBWD_WARPS_4PX
#define GS_RBWD_WARPS_4PX 24
#endif
constexpr int bwd_min_ctas(int threads, int ppt) {
  return ppt == 4 && GS_RBWD_WARPS_4PX > 0 ? GS_RBWD_WARPS_4PX / (threads / 32) : 0;
}

// Thread / pixel geometry. With PPT pixels per thread a warp covers a block
// of WB = 4 PPT columns by 8 rows: lane l owns column l % WB and rows
// l / WB + r * (32 / WB), r < PPT. The warps of a TW x TH tile tile it in
// TW / WB columns and TH / 8 rows of blocks.
template <int TW, int TH, int PPT>
struct Geo {
  static constexpr int WB = 4 * PPT;
  static constexpr int RS = 32 / WB;
  static constexpr int NT = TW * TH / PPT;
  static constexpr int NW = NT / 32;
  static constexpr int WXN = TW / WB;
  static_assert(TW % WB == 0 && TH % 8 == 0 && PPT * RS == 8, "unsupported tile / pixels-per-thread");
  static_assert(NW <= 32, "at most 32 warps");
  __device__ static void pixel_of(int tid, int& x, int& y0) {
    const int w = tid >> 5, l = tid & 31;
    x = WB * (w % WXN) + (l % WB);
    y0 = 8 * (w / WXN) + (l / WB);
  }
};

// Per-entry cull masks handed from the forward to the backward: 16 bits per
// sorted-list entry, the warps whose block the splat can reach (low byte)
// and a tag naming the tile shape and pixels per thread (high byte), so that
// the backward uses a mask only when it was made for the same warp layout
// and computes the cull itself otherwise. Layouts with more than 8 warps
// (32x32 tiles at 2 pixels per thread) do not hand masks over (tag 0).
template <int TW, int TH, int PPT>
constexpr uint32_t cull_tag() {
  return (TW == 8 && TH == 8 && PPT == 2)     ? 0x81u
         : (TW == 16 && TH == 16 && PPT == 2) ? 0x82u
         : (TW == 16 && TH == 16 && PPT == 4) ? 0x83u
         : (TW == 32 && TH == 16 && PPT == 2) ? 0x84u
         : (TW == 32 && TH == 16 && PPT == 4) ? 0x85u
         : (TW == 32 && TH == 32 && PPT == 4) ? 0x86u
                                              : 0u;
}

// Minimum over y in [y0, y1] of q(x, y) = m00 x^2 + 2 m01 x y + m11 y^2 for
// fixed x: the quadratic in y is minimised at y = k x with k = -m01 / m11
// (one division per splat, not per edge), clamped to the edge. A y a rounding
// away from the true minimiser raises q only by m11 dy^2, far inside the
// cull's margins.
__device__ __forceinline__ float edge_min_y(float x, float y0, float y1, float m00, float m01, float m11, float k) {
  const float y = fminf(fmaxf(k * x, y0), y1);
  return (m00 * x + 2.0f * m01 * y) * x + m11 * y * y;
}

// Bitmask of the warps of the tile at (tx0, ty0) whose pixel block can hold a
// pixel with alpha >= alpha_min. With the scaled conic
// M = [[-2A', -B'], [-B', -2C']] (so e = -d^T M d / 2) that set is the
// ellipse d^T M d <= 2 ts, ts = log2(o / alpha_min). A block is kept if its
// rectangle of pixel centres meets the ellipse: the minimum of d^T M d over
// the rectangle is 0 when the centre lies inside, else the smallest of the
// edge minima over the edges that face the centre (from the minimising
// point the direction to the centre lowers the quadratic, so it must leave
// the rectangle there: at most one vertical and one horizontal edge). ts and
// the rectangle are widened (x1.001 + margins), far beyond the rounding of
// the per-pixel evaluation and of the approximate divisions and square roots
// here (a few ulp), so no pixel of a dropped block can pass the alpha test.
template <class G>
__device__ __forceinline__ uint32_t warp_cull_mask(const float4& a, const float4& b, float tx0, float ty0,
                                                    float amin, float log2_amin) {
  constexpr uint32_t kAll = (G::NW >= 32) ? 0xffffffffu : ((1u << G::NW) - 1u);
  const float o = b.y;
  if (!(o > amin)) return 0u;
  const float m00 = -2.0f * a.z, m01 = -a.w, m11 = -2.0f * b.x;
  const float det = m00 * m11 - m01 * m01;
  if (!(det > 0.0f) || !(m00 > 0.0f) || !(m11 > 0.0f)) return kAll;
  const float ts = (__log2f(o) - log2_amin) * 1.001f + 0.01f;
  const float lim = 2.0f * ts;
  const float idet = __fdividef(1.0f, det);
  const float sx = lim * m11 * idet, sy = lim * m00 * idet;
  const float hx = sx * rsqrtf(sx) * 1.001f + 0.05f;
  const float hy = sy * rsqrtf(sy) * 1.001f + 0.05f;
  if (!(hx < 1e30f) || !(hy < 1e30f)) return kAll;
  // minimisers of the quadratic along vertical (y = kx x) and horizontal
  // (x = ky y) edges
  const float kx = __fdividef(-m01, m11), ky = __fdividef(-m01, m00);
  const float lim_kept = lim * 1.001f + 0.01f;
  const float kInf = __int_as_float(0x7f800000);
  uint32_t mask = 0;
#pragma unroll
  for (int w = 0; w < G::NW; ++w) {
    // rectangle of the block's pixel centres relative to the mean, widened
    const float x0 = tx0 + static_cast<float>(G::WB * (w % G::WXN)) + 0.45f - a.x;
    const float x1 = x0 + static_cast<float>(G::WB - 1) + 0.1f;
    const float y0 = ty0 + static_cast<float>(8 * (w / G::WXN)) + 0.45f - a.y;
    const float y1 = y0 + 7.1f;
    if (x1 < -hx || x0 > hx || y1 < -hy || y0 > hy) continue;  // outside the bounding box
    const bool left = x0 > 0.0f, right = x1 < 0.0f, below = y0 > 0.0f, above = y1 < 0.0f;
    if (!left && !right && !below && !above) {
      mask |= 1u << w;  // the centre lies in the block
      continue;
    }
    const float qv = (left || right) ? edge_min_y(left ? x0 : x1, y0, y1, m00, m01, m11, kx) : kInf;
    const float qh = (below || above) ? edge_min_y(below ? y0 : y1, x0, x1, m11, m01, m00, ky) : kInf;
    if (fminf(qv, qh) <= lim_kept) mask |= 1u << w;
  }
  return mask;
}

// One compositing step (forward rule) for two pixels of a thread, rows r and
// r + 1 of its column, in f32x2 operations: the .x lanes carry the first
// pixel, the .y lanes the second. The step has no branches: every lane
// evaluates the splat and the decisions select what changes, so the
// compiler can interleave the independent pixels of a thread (a branch only
// saves issue slots when all 32 lanes agree, which a partly covered block
// rarely does). Adding w = 0 leaves the colour unchanged bit for bit. A pixel
// that has stopped (or lies outside the image) carries an infinite alpha
// threshold, so no later splat passes its test. A packed add, multiply or
// FMA rounds each lane as __fadd_rn / __fmul_rn / __fmaf_rn does, and a
// subtraction x - y is formed as fma(y, -1, x), which rounds the exact
// difference once as __fsub_rn does. The backward (pixel_grad2) forms each
// exponent and alpha with the same packed operations, so it recomputes the
// forward's decisions exactly. The splat's constants
// enter as broadcast pairs (no extra instructions), and a packed operation
// takes one issue slot for two lanes' work.
struct PixelFwd2 {
  float2 T, c0, c1, c2;
  float2 thr;  // alpha threshold: alpha_min while compositing, +inf once stopped or outside the image
  uint32_t last0, last1;
};

__device__ __forceinline__ float2 bc2(float x) { return make_float2(x, x); }

// The splat's exponent and alpha at both pixels (independent of the pixel state).
__device__ __forceinline__ void splat_alpha2(const SplatCol& col, float2 py, const float4& a, const float4& b,
                                             float cap, float2& e, float2& alpha) {
  const float2 dy = __ffma2_rn(bc2(a.y), bc2(-1.0f), py);
  e = __ffma2_rn(dy, __ffma2_rn(bc2(b.x), dy, bc2(col.bdx)), bc2(col.adx2));
  const float2 oG = __fmul2_rn(bc2(b.y), make_float2(ex2_approx(e.x), ex2_approx(e.y)));
  alpha = make_float2(fminf(cap, oG.x), fminf(cap, oG.y));
}

// The compositing decisions and update of both pixels for a splat with
// exponents e and alphas alpha; returns how many of the two took it.
__device__ __forceinline__ int composite_apply2(PixelFwd2& P, float2 e, float2 alpha, const float4& b, float cb,
                                                uint32_t rel, float tstop) {
  const float2 Tn = __fmul2_rn(P.T, __ffma2_rn(alpha, bc2(-1.0f), bc2(1.0f)));
  const float2 w = __fmul2_rn(alpha, P.T);
  const bool ok0 = !(e.x > 0.0f) && !(alpha.x < P.thr.x);
  const bool ok1 = !(e.y > 0.0f) && !(alpha.y < P.thr.y);
  const bool stop0 = ok0 && Tn.x < tstop, stop1 = ok1 && Tn.y < tstop;
  const bool take0 = ok0 && !stop0, take1 = ok1 && !stop1;
  const float2 ws = make_float2(take0 ? w.x : 0.0f, take1 ? w.y : 0.0f);
  P.c0 = __ffma2_rn(bc2(b.z), ws, P.c0);
  P.c1 = __ffma2_rn(bc2(b.w), ws, P.c1);
  P.c2 = __ffma2_rn(bc2(cb), ws, P.c2);
  P.T = make_float2(take0 ? Tn.x : P.T.x, take1 ? Tn.y : P.T.y);
  P.last0 = take0 ? rel + 1 : P.last0;
  P.last1 = take1 ? rel + 1 : P.last1;
  const float kInf = __int_as_float(0x7f800000);
  P.thr = make_float2(stop0 ? kInf : P.thr.x, stop1 ? kInf : P.thr.y);
  return static_cast<int>(take0) + static_cast<int>(take1);
}

// Pair counters of the COUNT variants, per thread, added once per warp to
// counts[0..2]: pixel-splat pairs executed (listed splat x the thread's
// pixels, whether or not a pixel is still compositing or inside the image),
// pairs evaluated (the pixel still compositing in the forward, the entry
// before the pixel's last contributor in the backward) and pairs composited.
struct PairCount {
  uint32_t ex = 0, ev = 0, co = 0;
  __device__ __forceinline__ void flush(unsigned long long* counts) const {
    const uint32_t s0 = __reduce_add_sync(0xffffffffu, ex);
    const uint32_t s1 = __reduce_add_sync(0xffffffffu, ev);
    const uint32_t s2 = __reduce_add_sync(0xffffffffu, co);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(counts, static_cast<unsigned long long>(s0));
      atomicAdd(counts + 1, static_cast<unsigned long long>(s1));
      atomicAdd(counts + 2, static_cast<unsigned long long>(s2));
    }
  }
};


// Resident threads per SM the forward is compiled for. At 4 pixels a thread
// 1024 (8 CTAs of 128 at 32x16 tiles, 64 registers, no spills): 0.5 %
// faster than 7 CTAs at 72 registers; 1280 would leave 48 registers and
// spill 90-116 bytes. At 2 pixels and at most 256 splats a batch 1280: 48
// registers without spills at 16x16 and 32x16 tiles (1024 gives 64 and
// spills 4-8 bytes at 16x16), 4.73 -> 4.63 ms on the 16-view workload. The
// 512-splat batch keeps 1024: at 48 registers it spills 8 bytes at 32x16 and
// the 64M-Gaussian street forward ran 5.02 -> 5.11 ms. A minimum above the
// SM's 32 resident CTAs (32-thread 8x8 tiles) would be ignored, so it is
// clamped there.
constexpr int fwd_min_ctas(int threads, int ppt, int batch) {
  const int per_sm = ppt == 2 && batch <= 256 ? 1280 : 1024;
  return per_sm / threads < 32 ? per_sm / threads : 32;
}

template <int TW, int TH, int PPT, int B, bool COUNT>
__global__ void __launch_bounds__(TW* TH / PPT, fwd_min_ctas(TW* TH / PPT, PPT, B)) raster_fwd_kernel(const float4* __restrict__ projected,
                                                                   const uint32_t* __restrict__ vals,
                                                                   const uint2* __restrict__ ranges,
                                                                   const uint32_t* __restrict__ order, const Layout L,
                                                                   const Consts K, float* __restrict__ image,
                                                                   float* __restrict__ final_T,
                                                                   uint32_t* __restrict__ last, const ImageLoss IL,
                                                                   unsigned long long* __restrict__ counts,
                                                                   uint16_t* __restrict__ cull_out) {
  using G = Geo<TW, TH, PPT>;
  constexpr int NT = G::NT;
  static_assert(B >= 32 && B <= 512 && (B & (B - 1)) == 0, "splats per batch: a power of two in [32, 512]");
  static_assert(fwd_smem_bytes(B, G::NW) <= kStaticSmem, "forward shared memory over 48 KB");
  __shared__ float4 s_a[B];
  __shared__ float4 s_b[B];
  __shared__ float s_c[B];
  __shared__ uint32_t s_m[B];
  __shared__ uint16_t s_list[G::NW][B];  // per warp: the staged splats that can touch its block
  // CTA i takes tile order[i] (longest lists first) when an order is given
  const uint32_t tile = order ? order[blockIdx.x] : blockIdx.x;
  if (tile >= L.n_tiles) return;
  const int v = view_of_tile(L, tile);
  const uint32_t local = tile - L.tile_base[v];
  const int ntx = L.ntx[v];
  const int tx = static_cast<int>(local % ntx), ty = static_cast<int>(local / ntx);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t wbit = 1u << warp;
  int lx, ly;
  G::pixel_of(tid, lx, ly);
  const int W = L.width[v], H = L.height[v];
  const int x = tx * TW + lx, y0 = ty * TH + ly;
  const float px = static_cast<float>(x) + 0.5f, py0 = static_cast<float>(y0) + 0.5f;
  const uint2 range = ranges[tile];
  const int n = static_cast<int>(range.y - range.x);
  const float cap = K.alpha_cap, amin = K.alpha_min, tstop = K.t_stop, log2_amin = __log2f(amin);
  const float tx0 = static_cast<float>(tx * TW), ty0 = static_cast<float>(ty * TH);
  const float kInf = __int_as_float(0x7f800000);
  static_assert(PPT % 2 == 0, "pixels are stepped in pairs");
  constexpr int NP = PPT / 2;
  PixelFwd2 P[NP];
  float2 py2[NP];  // pixel centres of each pair's rows
  PairCount pc;
  bool all_done = true;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const bool in0 = x < W && y0 + 2 * k * G::RS < H, in1 = x < W && y0 + (2 * k + 1) * G::RS < H;
    P[k] = PixelFwd2{bc2(1.0f), bc2(0.0f), bc2(0.0f), bc2(0.0f), make_float2(in0 ? amin : kInf, in1 ? amin : kInf),
                     0u, 0u};
    py2[k] = make_float2(py0 + static_cast<float>(2 * k * G::RS), py0 + static_cast<float>((2 * k + 1) * G::RS));
    all_done = all_done && !in0 && !in1;
  }
  for (int b0 = 0; b0 < n; b0 += B) {
    if (__syncthreads_count(all_done) == NT) break;
    for (int k = tid; k < B && b0 + k < n; k += NT) {
      float4 a, b;
      float c;
      load_splat(projected, vals[range.x + b0 + k], a, b, c);
      s_a[k] = a;
      s_b[k] = b;
      s_c[k] = c;
      const uint32_t mk = warp_cull_mask<G>(a, b, tx0, ty0, amin, log2_amin);
      s_m[k] = mk;
      constexpr uint32_t kTag = cull_tag<TW, TH, PPT>();
      if (kTag && cull_out) cull_out[range.x + b0 + k] = static_cast<uint16_t>(mk | (kTag << 8));
    }
    __syncthreads();
    const int cnt = min(B, n - b0);
    // the warp's list of staged splats that can touch its block
    int nl = 0;
    for (int jb = 0; jb < cnt; jb += 32) {
      const int j = jb + lane;
      const bool keep = j < cnt && (s_m[j] & wbit);
      const uint32_t bal = __ballot_sync(0xffffffffu, keep);
      if (keep) s_list[warp][nl + __popc(bal & ((1u << lane) - 1u))] = static_cast<uint16_t>(j);
      nl += __popc(bal);
    }
    __syncwarp();
    int q = 0;
#ifndef GS_FWD_GROUP
#define GS_FWD_GROUP 4
#endif
    // GS_FWD_GROUP splats per iteration: their exponents / alphas are
    // independent of the pixel state and are issued first; the compositing
    // then applies them in list order
    constexpr int GR = GS_FWD_GROUP;
    for (; q + GR - 1 < nl && !all_done; q += GR) {
      float2 e[GR][NP], al[GR][NP];
      int js[GR];
#pragma unroll
      for (int u = 0; u < GR; ++u) {
        js[u] = s_list[warp][q + u];
        const float4 a = s_a[js[u]], b = s_b[js[u]];
        const SplatCol col = splat_column(px, a);
#pragma unroll
        for (int k = 0; k < NP; ++k) splat_alpha2(col, py2[k], a, b, cap, e[u][k], al[u][k]);
      }
      all_done = true;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
#pragma unroll
        for (int u = 0; u < GR; ++u) {
          const float4 b = s_b[js[u]];
          if constexpr (COUNT) pc.ev += (P[k].thr.x != kInf) + (P[k].thr.y != kInf);
          const int took =
              composite_apply2(P[k], e[u][k], al[u][k], b, s_c[js[u]], static_cast<uint32_t>(b0 + js[u]), tstop);
          if constexpr (COUNT) pc.co += took;
        }
        all_done = all_done && P[k].thr.x == kInf && P[k].thr.y == kInf;
      }
      if constexpr (COUNT) pc.ex += GR * PPT;
    }
    for (; q < nl && !all_done; ++q) {
      const int j = s_list[warp][q];
      const float4 a = s_a[j];
      const float4 b = s_b[j];
      const float cb = s_c[j];
      const uint32_t rel = static_cast<uint32_t>(b0 + j);
      const SplatCol col = splat_column(px, a);
      all_done = true;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        if constexpr (COUNT) pc.ev += (P[k].thr.x != kInf) + (P[k].thr.y != kInf);
        float2 e, al;
        splat_alpha2(col, py2[k], a, b, cap, e, al);
        const int took = composite_apply2(P[k], e, al, b, cb, rel, tstop);
        if constexpr (COUNT) pc.co += took;
        all_done = all_done && P[k].thr.x == kInf && P[k].thr.y == kInf;
      }
      if constexpr (COUNT) pc.ex += PPT;
    }
  }
  if constexpr (COUNT) pc.flush(counts);
  const size_t pb = L.pix_base[v];
  const bool with_loss = IL.target != nullptr;
  float part = 0.0f;
#pragma unroll
  for (int r = 0; r < PPT; ++r) {
    const int yy = y0 + r * G::RS;
    if (x < W && yy < H) {
      const size_t p = pb + static_cast<size_t>(yy) * W + x;
      const PixelFwd2& Q = P[r / 2];
      const bool hi = r & 1;
      const float T = hi ? Q.T.y : Q.T.x;
      const float c[3] = {(hi ? Q.c0.y : Q.c0.x) + T * K.bg[0], (hi ? Q.c1.y : Q.c1.x) + T * K.bg[1],
                          (hi ? Q.c2.y : Q.c2.x) + T * K.bg[2]};
#pragma unroll
      for (int k = 0; k < 3; ++k) image[3 * p + k] = c[k];
      final_T[p] = T;
      last[p] = hi ? Q.last1 : Q.last0;
      if (with_loss) {
        // the L1 + L2 image loss of these values (same arithmetic as gs_image_loss)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float rr = c[k] - IL.target[3 * p + k];
          IL.grad[3 * p + k] = l1l2_grad(rr, IL.w1, IL.w2, IL.inv_n);
          part += IL.w1 * fabsf(rr) + IL.w2 * rr * rr;
        }
      }
    }
  }
  if (with_loss) {
    // CTA sum of the loss terms, one double atomic per CTA
    __shared__ double s_loss[G::NW];
    double acc = part;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) s_loss[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < G::NW; ++w) t += s_loss[w];
      atomicAdd(IL.loss, t * IL.inv_n_d);
    }
  }
}

// Reduce-scatter of 9 values over a warp with 12 shuffles. On return, the
// lane holds the warp-wide sum of value index slot_of_lane(lane) (or 0 where
// that is -1); lanes 2k and 2k+1 hold the same slot.
__device__ __forceinline__ float warp_reduce9(const float v[9], int lane) {
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
  float s[5];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = h4 ? v[i] : v[5 + i];
    s[i] = (h4 ? v[5 + i] : v[i]) + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  {
    const float send = h4 ? v[4] : 0.0f;
    const float r = __shfl_xor_sync(0xffffffffu, send, 16);
    s[4] = h4 ? 0.0f : v[4] + r;
  }
  float t[3];
  t[0] = (h3 ? s[3] : s[0]) + __shfl_xor_sync(0xffffffffu, h3 ? s[0] : s[3], 8);
  t[1] = (h3 ? s[4] : s[1]) + __shfl_xor_sync(0xffffffffu, h3 ? s[1] : s[4], 8);
  t[2] = (h3 ? 0.0f : s[2]) + __shfl_xor_sync(0xffffffffu, h3 ? s[2] : 0.0f, 8);
  float u[2];
  u[0] = (h2 ? t[2] : t[0]) + __shfl_xor_sync(0xffffffffu, h2 ? t[0] : t[2], 4);
  u[1] = (h2 ? 0.0f : t[1]) + __shfl_xor_sync(0xffffffffu, h2 ? t[1] : 0.0f, 4);
  float w = (h1 ? u[1] : u[0]) + __shfl_xor_sync(0xffffffffu, h1 ? u[0] : u[1], 2);
  w += __shfl_xor_sync(0xffffffffu, w, 1);
  return w;
}

__device__ __forceinline__ int slot_of_lane(int lane) {
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
  int s[5];
  for (int i = 0; i < 4; ++i) s[i] = h4 ? 5 + i : i;
  s[4] = h4 ? -1 : 4;
  int t[3] = {h3 ? s[3] : s[0], h3 ? s[4] : s[1], h3 ? -1 : s[2]};
  int u[2] = {h2 ? t[2] : t[0], h2 ? -1 : t[1]};
  return h1 ? u[1] : u[0];
}

// Reduce-scatter of the 18 values of two splats (a[9], then b[9]) over a warp
// with 20 shuffles (instead of 2 x 12): on return, the lane holds the
// warp-wide sum of value index slot18_of_lane(lane) (0..8: a, 9..17: b), or
// 0 where that is -1. Every value lands in exactly one lane.
__device__ __forceinline__ float warp_reduce18(const float a[9], const float b[9], int lane) {
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2, h0 = lane & 1;
  float s[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) s[i] = (h4 ? b[i] : a[i]) + __shfl_xor_sync(0xffffffffu, h4 ? a[i] : b[i], 16);
  float t[5];
#pragma unroll
  for (int i = 0; i < 4; ++i) t[i] = (h3 ? s[5 + i] : s[i]) + __shfl_xor_sync(0xffffffffu, h3 ? s[i] : s[5 + i], 8);
  t[4] = (h3 ? 0.0f : s[4]) + __shfl_xor_sync(0xffffffffu, h3 ? s[4] : 0.0f, 8);
  float u[3];
  u[0] = (h2 ? t[3] : t[0]) + __shfl_xor_sync(0xffffffffu, h2 ? t[0] : t[3], 4);
  u[1] = (h2 ? t[4] : t[1]) + __shfl_xor_sync(0xffffffffu, h2 ? t[1] : t[4], 4);
  u[2] = (h2 ? 0.0f : t[2]) + __shfl_xor_sync(0xffffffffu, h2 ? t[2] : 0.0f, 4);
  float w[2];
  w[0] = (h1 ? u[2] : u[0]) + __shfl_xor_sync(0xffffffffu, h1 ? u[0] : u[2], 2);
  w[1] = (h1 ? 0.0f : u[1]) + __shfl_xor_sync(0xffffffffu, h1 ? u[1] : 0.0f, 2);
  return (h0 ? w[1] : w[0]) + __shfl_xor_sync(0xffffffffu, h0 ? w[0] : w[1], 1);
}

__device__ __forceinline__ int slot18_of_lane(int lane) {
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2, h0 = lane & 1;
  int s[9];
  for (int i = 0; i < 9; ++i) s[i] = (h4 ? 9 : 0) + i;
  int t[5];
  for (int i = 0; i < 4; ++i) t[i] = h3 ? s[5 + i] : s[i];
  t[4] = h3 ? -1 : s[4];
  const int u[3] = {h2 ? t[3] : t[0], h2 ? t[4] : t[1], h2 ? -1 : t[2]};
  const int w[2] = {h1 ? u[2] : u[0], h1 ? -1 : u[1]};
  return h0 ? w[1] : w[0];
}

// Two pixels of a thread (rows r and r + 1 of its column) in the backward,
// stepped together in f32x2 operations as in the forward (.x: the first
// pixel, .y: the second).
struct PixelBwd2 {
  // S = (colour accumulated behind the current entry, normalised) . dL/dC:
  // the alpha gradient needs the accumulated colour only through this dot
  // product, so one scalar replaces the three channels
  float2 T, g0, g1, g2, gbg, S;
  uint32_t last0, last1;
};

// Backward contribution of splat (a, b, cb) at relative position `rel` to one
// pixel, added into gv[9]; returns whether the pixel took part. Constant
// factors are applied once per splat when the sums are flushed:
//   gv[0..1] = sum dalpha*alpha*(2A'dx + B'dy, B'dx + 2C'dy)  -> dmean = -gv/log2e
//   gv[2..4] = sum dalpha*alpha*(dx^2, dx dy, dy^2)          -> dconic = -(gv2/2, gv3, gv4/2)
//   gv[5..7] = sum alpha T dL/dC, gv[8] = sum dalpha G          (as is)
// From the moments m0 = sum dpw, m1 = sum dpw dy, m2 = sum dpw dy^2 of a
// thread's pixels (common dx) to
//   gv[0..1] = sum dpw (2A'dx + B'dy, B'dx + 2C'dy),
//   gv[2..4] = sum dpw (dx^2, dx dy, dy^2).
__device__ __forceinline__ void finish_geometry(float gv[9], const SplatCol& col, const float4& a, const float4& b) {
  const float m0 = gv[0], m1 = gv[1], m2 = gv[2], dx = col.dx;
  gv[0] = fmaf(2.0f * a.z * dx, m0, a.w * m1);
  gv[1] = fmaf(col.bdx, m0, 2.0f * b.x * m1);
  gv[2] = dx * dx * m0;
  gv[3] = dx * m1;
  gv[4] = m2;
}

// The backward step of both pixels of a PixelBwd2 for one splat, adding
// into gv[9] (per pixel, in .x / .y); returns whether either took part.
// Exponent and alpha are the forward's bits (same packed operations), so
// the skip / stop decisions are the forward's.
template <bool BG, bool COUNT>
__device__ __forceinline__ bool pixel_grad2(PixelBwd2& P, const SplatCol& col, float2 py, const float4& a,
                                            const float4& b, float cb, uint32_t rel, float cap, float amin,
                                            float2 gv[9], PairCount& pc) {
  // branch-free, like the forward step: decisions select, zeros add nothing
  const float2 dy = __ffma2_rn(bc2(a.y), bc2(-1.0f), py);
  const float2 e = __ffma2_rn(dy, __ffma2_rn(bc2(b.x), dy, bc2(col.bdx)), bc2(col.adx2));
  const float2 G = make_float2(ex2_approx(e.x), ex2_approx(e.y));
  const float2 oG = __fmul2_rn(bc2(b.y), G);
  const float2 al = make_float2(fminf(cap, oG.x), fminf(cap, oG.y));
  const bool in0 = rel < P.last0, in1 = rel < P.last1;
  const bool ok0 = in0 && !(e.x > 0.0f) && !(al.x < amin);
  const bool ok1 = in1 && !(e.y > 0.0f) && !(al.y < amin);
  if constexpr (COUNT) {
    pc.ev += static_cast<uint32_t>(in0) + static_cast<uint32_t>(in1);
    pc.co += static_cast<uint32_t>(ok0) + static_cast<uint32_t>(ok1);
  }
  const float2 om = __ffma2_rn(al, bc2(-1.0f), bc2(1.0f));
  const float2 inv = make_float2(rcp_approx(om.x), rcp_approx(om.y));
  const float2 Ti = __fmul2_rn(P.T, inv);
  P.T = make_float2(ok0 ? Ti.x : P.T.x, ok1 ? Ti.y : P.T.y);  // transmittance in front of this entry
  const float2 aok = make_float2(ok0 ? al.x : 0.0f, ok1 ? al.y : 0.0f);
  const float2 w = __fmul2_rn(aok, P.T);
  gv[5] = __ffma2_rn(w, P.g0, gv[5]);
  gv[6] = __ffma2_rn(w, P.g1, gv[6]);
  gv[7] = __ffma2_rn(w, P.g2, gv[7]);
  // (c - accumulated) . dL/dC = c . dL/dC - S
  const float2 cd = __ffma2_rn(bc2(cb), P.g2, __ffma2_rn(bc2(b.w), P.g1, __fmul2_rn(bc2(b.z), P.g0)));
  const float2 dcs = __ffma2_rn(P.S, bc2(-1.0f), cd);
  // with a zero background (the default) the background term vanishes
  float2 dal = __fmul2_rn(P.T, dcs);
  if constexpr (BG) dal = __ffma2_rn(__fmul2_rn(P.gbg, bc2(-1.0f)), inv, dal);
  P.S = __ffma2_rn(aok, dcs, P.S);
  const float2 da = make_float2((ok0 && !(oG.x > cap)) ? dal.x : 0.0f, (ok1 && !(oG.y > cap)) ? dal.y : 0.0f);
  gv[8] = __ffma2_rn(da, G, gv[8]);
  // The geometric sums need dpw = dalpha * alpha only through its moments in
  // dy (the thread's pixels share dx): gv[0..2] collect sum dpw, sum dpw dy,
  // sum dpw dy^2 here and finish_geometry turns them into the five sums.
  const float2 dpw = __fmul2_rn(da, al);
  const float2 dpy = __fmul2_rn(dpw, dy);
  gv[0] = __fadd2_rn(gv[0], dpw);
  gv[1] = __fadd2_rn(gv[1], dpy);
  gv[2] = __ffma2_rn(dpy, dy, gv[2]);
  return ok0 || ok1;
}

// The nine gradient sums of one splat over a thread's pixels (NP pairs),
// collapsed to one value each and finished (finish_geometry); returns
// whether any of the pixels took part.
template <bool BG, bool COUNT, int NP>
__device__ __forceinline__ bool splat_grads(PixelBwd2 (&P)[NP], const float2 (&py2)[NP], float px, const float4& a,
                                            const float4& b, float cb, uint32_t rel, float cap, float amin,
                                            float g[9], PairCount& pc) {
  const SplatCol col = splat_column(px, a);
  float2 acc[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) acc[i] = bc2(0.0f);
  bool any = false;
#pragma unroll
  for (int k = 0; k < NP; ++k) any |= pixel_grad2<BG, COUNT>(P[k], col, py2[k], a, b, cb, rel, cap, amin, acc, pc);
#pragma unroll
  for (int i = 0; i < 9; ++i) g[i] = acc[i].x + acc[i].y;
  finish_geometry(g, col, a, b);
  return any;
}

template <int TW, int TH, int PPT, int B, bool BG, bool COUNT>
__global__ void __launch_bounds__(TW* TH / PPT, bwd_min_ctas(TW* TH / PPT, PPT)) raster_bwd_kernel(
    const float4* __restrict__ projected, const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ order, const Layout L, const Consts K, const float* __restrict__ final_T,
    const uint32_t* __restrict__ last, const float* __restrict__ dL_dimage, float* __restrict__ d_proj,
    unsigned long long* __restrict__ counts, const uint16_t* __restrict__ cull_in) {
  using Gm = Geo<TW, TH, PPT>;
  constexpr int NT = Gm::NT, NW = Gm::NW;
  static_assert(B >= 32 && B <= 512 && (B & (B - 1)) == 0, "splats per batch: a power of two in [32, 512]");
  static_assert(bwd_smem_bytes(B, NW) <= kMaxSmem, "backward shared memory over the opt-in limit");
  // the staged batch, its gradient slots, the warps' bounds and lists:
  // static shared memory up to 48 KB, above it dynamic (opted in by
  // launch_bwd). The static size also steers the compiler's register choice
  // (as dynamic memory the 16x16 2-pixel instance took 64 registers and
  // spilled instead of 70).
  constexpr bool kDyn = bwd_smem_bytes(B, NW) > kStaticSmem;
  __shared__ __align__(16) unsigned char bwd_smem_st[kDyn ? 16 : bwd_smem_bytes(B, NW)];
  extern __shared__ __align__(16) unsigned char bwd_smem_dyn[];
  unsigned char* bwd_smem = kDyn ? bwd_smem_dyn : bwd_smem_st;
  float4* s_a = reinterpret_cast<float4*>(bwd_smem);
  float4* s_b = s_a + B;
  float* s_c = reinterpret_cast<float*>(s_b + B);
  uint32_t* s_m = reinterpret_cast<uint32_t*>(s_c + B);
  uint32_t* s_vg = s_m + B;
  float* s_grad = reinterpret_cast<float*>(s_vg + B);
  uint32_t* s_wmax = reinterpret_cast<uint32_t*>(s_grad + 9 * B);
  uint16_t(*s_list)[B] = reinterpret_cast<uint16_t(*)[B]>(s_wmax + NW);  // per warp: the staged splats that can touch its block
  // CTA i takes tile order[i] (longest lists first) when an order is given
  const uint32_t tile = order ? order[blockIdx.x] : blockIdx.x;
  if (tile >= L.n_tiles) return;
  const int v = view_of_tile(L, tile);
  const uint32_t local = tile - L.tile_base[v];
  const int ntx = L.ntx[v];
  const int tx = static_cast<int>(local % ntx), ty = static_cast<int>(local / ntx);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t wbit = 1u << warp;
  int lx, ly;
  Gm::pixel_of(tid, lx, ly);
  const int W = L.width[v], H = L.height[v];
  const int x = tx * TW + lx, y0 = ty * TH + ly;
  const float px = static_cast<float>(x) + 0.5f, py0 = static_cast<float>(y0) + 0.5f;
  const uint2 range = ranges[tile];
  const float cap = K.alpha_cap, amin = K.alpha_min, log2_amin = __log2f(amin);
  const float tx0 = static_cast<float>(tx * TW), ty0 = static_cast<float>(ty * TH);
  static_assert(PPT % 2 == 0, "pixels are stepped in pairs");
  constexpr int NP = PPT / 2;
  PixelBwd2 P[NP];
  float2 py2[NP];  // pixel centres of each pair's rows
  PairCount pc;
  uint32_t lmax = 0;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    float T[2] = {1.0f, 1.0f}, g0[2] = {0.f, 0.f}, g1[2] = {0.f, 0.f}, g2[2] = {0.f, 0.f}, gbg[2] = {0.f, 0.f};
    uint32_t ls[2] = {0u, 0u};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int yy = y0 + (2 * k + h) * Gm::RS;
      if (x < W && yy < H) {
        const size_t p = static_cast<size_t>(L.pix_base[v]) + static_cast<size_t>(yy) * W + x;
        T[h] = final_T[p];
        ls[h] = last[p];
        g0[h] = dL_dimage[3 * p];
        g1[h] = dL_dimage[3 * p + 1];
        g2[h] = dL_dimage[3 * p + 2];
        gbg[h] = T[h] * (g0[h] * K.bg[0] + g1[h] * K.bg[1] + g2[h] * K.bg[2]);
      }
      lmax = max(lmax, ls[h]);
    }
    P[k] = PixelBwd2{make_float2(T[0], T[1]),     make_float2(g0[0], g0[1]), make_float2(g1[0], g1[1]),
                     make_float2(g2[0], g2[1]),   make_float2(gbg[0], gbg[1]), bc2(0.0f), ls[0], ls[1]};
    py2[k] = make_float2(py0 + static_cast<float>(2 * k * Gm::RS), py0 + static_cast<float>((2 * k + 1) * Gm::RS));
  }
  const int my_slot = slot_of_lane(lane);
  // the pair reduction: which splat of the pair and which of its 9 values
  const int slot18 = slot18_of_lane(lane);
  const bool pair_b = slot18 >= 9;
  const int pair_slot = slot18 >= 9 ? slot18 - 9 : slot18;
  const uint32_t wmax = __reduce_max_sync(0xffffffffu, lmax);
  if (lane == 0) s_wmax[warp] = wmax;
  for (int i = tid; i < B * 9; i += NT) s_grad[i] = 0.0f;
  __syncthreads();
  uint32_t max_last = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) max_last = max(max_last, s_wmax[w]);

  // Adds the gradients gathered in slot k (one splat of the batch) to its
  // record with one atomic per non-zero value, and clears the slot.
  auto flush_slot = [&](int k) {
    float* dst = d_proj + static_cast<size_t>(s_vg[k]) * kDRecordFloats;
    constexpr float kScale[9] = {-1.0f / kLog2e, -1.0f / kLog2e, -0.5f, -1.0f, -0.5f, 1.0f, 1.0f, 1.0f, 1.0f};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float gval = s_grad[k * 9 + i];
      if (gval != 0.0f) {
        atomicAdd(dst + i, gval * kScale[i]);
        s_grad[k * 9 + i] = 0.0f;
      }
    }
  };
  int prev_cnt = 0;
  for (int b_end = static_cast<int>(max_last); b_end > 0; b_end -= B) {
    const int cnt = min(B, b_end);
    // each thread flushes the slots it staged for the previous batch, then
    // stages the same slots for this one: no other thread touches them in
    // between, so one barrier covers both
    for (int k = tid; k < B; k += NT) {
      if (k < prev_cnt) flush_slot(k);
      if (k >= cnt) continue;
      const uint32_t vg = vals[range.x + b_end - 1 - k];
      float4 a, b;
      float c;
      load_splat(projected, vg, a, b, c);
      s_a[k] = a;
      s_b[k] = b;
      s_c[k] = c;
      s_vg[k] = vg;
      // the forward's mask for this entry when it made one for this layout
      constexpr uint32_t kTag = cull_tag<TW, TH, PPT>();
      const uint32_t handed = (kTag && cull_in) ? cull_in[range.x + b_end - 1 - k] : 0u;
      s_m[k] = (handed >> 8) == kTag && kTag ? (handed & 0xffu) : warp_cull_mask<Gm>(a, b, tx0, ty0, amin, log2_amin);
    }
    __syncthreads();
    // entries j hold relative position b_end-1-j; this warp needs rel < wmax.
    // The warp first lists the staged splats that can touch its block, then
    // takes them in pairs: the second splat's pixel work is issued before the
    // first one's warp reduction, so the reduction's shuffle latency overlaps
    // independent arithmetic (the pixel state still advances splat by splat).
    const int j0 = max(0, b_end - static_cast<int>(wmax));
    int nl = 0;
    for (int jb = j0; jb < cnt; jb += 32) {
      const int j = jb + lane;
      const bool keep = j < cnt && (s_m[j] & wbit);
      const uint32_t bal = __ballot_sync(0xffffffffu, keep);
      if (keep) s_list[warp][nl + __popc(bal & ((1u << lane) - 1u))] = static_cast<uint16_t>(j);
      nl += __popc(bal);
    }
    __syncwarp();
    int q = 0;
    for (; q + 1 < nl; q += 2) {
      const int jA = s_list[warp][q], jB = s_list[warp][q + 1];
      float gA[9], gB[9];
      splat_grads<BG, COUNT>(P, py2, px, s_a[jA], s_b[jA], s_c[jA], static_cast<uint32_t>(b_end - 1 - jA), cap, amin,
                             gA, pc);
      splat_grads<BG, COUNT>(P, py2, px, s_a[jB], s_b[jB], s_c[jB], static_cast<uint32_t>(b_end - 1 - jB), cap, amin,
                             gB, pc);
      // listed splats nearly always contribute: reduce without a branch, so
      // the two reductions and the pixel work form one block to schedule
      if constexpr (COUNT) pc.ex += 2 * PPT;
      const float red = warp_reduce18(gA, gB, lane);
      if (slot18 >= 0 && red != 0.0f) atomicAdd(&s_grad[(pair_b ? jB : jA) * 9 + pair_slot], red);
    }
    if (q < nl) {
      const int j = s_list[warp][q];
      float gv[9];
      const bool contrib = splat_grads<BG, COUNT>(P, py2, px, s_a[j], s_b[j], s_c[j],
                                                  static_cast<uint32_t>(b_end - 1 - j), cap, amin, gv, pc);
      if constexpr (COUNT) pc.ex += PPT;
      if (__any_sync(0xffffffffu, contrib)) {
        const float red = warp_reduce9(gv, lane);
        if (!(lane & 1) && my_slot >= 0 && red != 0.0f) atomicAdd(&s_grad[j * 9 + my_slot], red);
      }
    }
    __syncthreads();
    prev_cnt = cnt;
  }
  for (int k = tid; k < prev_cnt; k += NT) flush_slot(k);
  if constexpr (COUNT) pc.flush(counts);
}



// One CTA per tile of the call (in the tile order when there is one).
template <int TW, int TH, int PPT, int B, bool COUNT>
int launch_fwd(const FwdArgs& a, cudaStream_t stream) {
  raster_fwd_kernel<TW, TH, PPT, B, COUNT><<<static_cast<unsigned>(a.L.n_tiles), TW * TH / PPT, 0, stream>>>(
      a.projected, a.vals, a.ranges, a.order, a.L, a.K, a.image, a.final_T, a.last, a.IL, a.counts, a.cull);
  return cuda_status(cudaGetLastError());
}

template <int TW, int TH, int PPT, int B, bool BG, bool COUNT>
int launch_bwd(const BwdArgs& a, cudaStream_t stream) {
  // above 48 KB the shared memory is dynamic and the kernel opted in (set
  // on every call: the attribute belongs to the current device)
  constexpr int bytes = bwd_smem_bytes(B, TW * TH / PPT / 32);
  constexpr int dyn = bytes > kStaticSmem ? bytes : 0;
  if (dyn && cudaFuncSetAttribute(raster_bwd_kernel<TW, TH, PPT, B, BG, COUNT>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess)
    return GS_ERR_CUDA;
  raster_bwd_kernel<TW, TH, PPT, B, BG, COUNT><<<static_cast<unsigned>(a.L.n_tiles), TW * TH / PPT, dyn, stream>>>(
      a.projected, a.vals, a.ranges, a.order, a.L, a.K, a.final_T, a.last, a.dL_dimage, a.d_proj, a.counts, a.cull);
  return cuda_status(cudaGetLastError());
}

}  // namespace rast
}  // namespace gs

// Explicit instantiations of the launchers: GS_RASTER_FWD(TW, TH, PPT, B,
// COUNT) and GS_RASTER_BWD(TW, TH, PPT, B, BG, COUNT), one unit per group.
#define GS_RASTER_FWD(TW, TH, PPT, B, COUNT) \
  template int gs::rast::launch_fwd<TW, TH, PPT, B, COUNT>(const gs::rast::FwdArgs&, cudaStream_t);
#define GS_RASTER_BWD(TW, TH, PPT, B, BG, COUNT) \
  template int gs::rast::launch_bwd<TW, TH, PPT, B, BG, COUNT>(const gs::rast::BwdArgs&, cudaStream_t);


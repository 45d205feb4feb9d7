// Fused SSIM image loss, forward and backward in one kernel.
//
// Paper: arXiv 2606.11390 §4 runs a fused SSIM loss operator per camera next to
// the rasteriser (SSIM of Wang et al. 2004, fused as in Taming 3DGS). The loss
// is L = (1 - lam) mean|x - y| + lam (1 - mean SSIM(x, y)) over every pixel and
// channel of every view. SSIM per channel uses an 11x11 Gaussian window of
// standard deviation 1.5 (weights normalised to sum 1), C1 = 0.01^2 and
// C2 = 0.03^2; window sums treat pixels outside the image as zero.
//
// Design. One CTA owns a 32x32 output tile of one view and keeps everything
// on chip: it loads x and y over the tile plus a 10-pixel halo, forms the four
// window sums SSIM needs (mu_x, mu_y, E[xx + yy], E[xy]) on the tile plus a
// 5-pixel halo with two separable 11-tap passes, turns them into SSIM and its
// three partials (d/dmu_x, d/dE[xx + yy], d/dE[xy]) per pixel, and filters the partials
// back with the same window (the adjoint of a symmetric window sum) to get
// dL/dx on the tile. Nothing but x, y (read) and dL/dx (written) touches HBM;
// the halo recomputation replaces the round trip of the partial maps. Each
// filter pass is register-blocked along its direction: a work item produces
// 4-6 consecutive outputs from the 14-16 inputs it holds in registers, so
// shared-memory loads stay well below the FMAs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kWin = 11;
constexpr int kHalf = kWin / 2;            // 5
constexpr int kTX = 32, kTY = 32;          // output tile
constexpr int kR1W = kTX + 2 * kHalf;      // 42: maps / partials region
constexpr int kR1H = kTY + 2 * kHalf;      // 42
constexpr int kR0W = kTX + 4 * kHalf;      // 52: input region
constexpr int kR0H = kTY + 4 * kHalf;      // 52
constexpr int kSsimThreads = 256;
constexpr int kMaxSsimViews = 64;
// register blocking: outputs per work item along the filter direction
// register blocking (measured at 4K: 6 / 6 / 4 0.515 ms, 3 / 3 / 2 0.551 ms)
constexpr int kHR = 6;  // forward horizontal pass: outputs per work item (7 runs per row)
constexpr int kVR = 6;  // forward vertical pass (7 runs per column)
constexpr int kBR = 4;  // backward passes
static_assert(kR1W % kHR == 0 && kR1H % kVR == 0 && kTX % kBR == 0 && kTY % kBR == 0, "run lengths");

struct SsimLayout {
  int32_t V;
  int32_t width[kMaxSsimViews], height[kMaxSsimViews], ntx[kMaxSsimViews];
  int32_t tile_base[kMaxSsimViews + 1];
  int64_t pix_base[kMaxSsimViews + 1];
};

struct SsimArgs {
  float w[kWin];
  float c1, c2;
  float l1_scale;    // (1 - lam) / M
  float ssim_scale;  // lam / M
};

// x/y live until the forward horizontal pass, then their space holds the
// partial maps; the horizontal sums' space later holds the backward
// horizontal pass. 57 KB: three CTAs per SM.
struct SsimSmem {
  union {
    struct {
      float x[kR0H][kR0W];  // one channel of the image over the tile + 10-pixel halo
      float y[kR0H][kR0W];  // the same of the target
    } in;
    float p[3][kR1H][kR1W];  // dS/dmu_x, dS/dE[xx + yy], dS/dE[xy]
  } a;
  union {
    float h[4][kR0H][kR1W];  // horizontal sums of x, y, xx + yy, xy
    float q[3][kR1H][kTX];   // backward horizontal sums of the partials
  } b;
  double red[kSsimThreads / 32];
};

__global__ void __launch_bounds__(kSsimThreads) ssim_loss_kernel(const float* __restrict__ image,
                                                                 const float* __restrict__ target, const SsimLayout L,
                                                                 const SsimArgs A, float* __restrict__ grad,
                                                                 double* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SsimSmem& s = *reinterpret_cast<SsimSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  int v = 0;
  while (v + 1 < L.V && tile >= L.tile_base[v + 1]) ++v;
  const int W = L.width[v], H = L.height[v];
  const int t = tile - L.tile_base[v];
  const int tx = t % L.ntx[v], ty = t / L.ntx[v];
  const int gx0 = tx * kTX - 2 * kHalf, gy0 = ty * kTY - 2 * kHalf;
  const int64_t pb = L.pix_base[v];

  float part = 0.0f;  // this thread's share of the loss
  for (int c = 0; c < 3; ++c) {
    // 1. channel c of x and y over the tile and a 10-pixel halo (zero outside)
    for (int e = tid; e < kR0H * kR0W; e += kSsimThreads) {
      const int r = e / kR0W, j = e - r * kR0W;
      const int gx = gx0 + j, gy = gy0 + r;
      float xa = 0.0f, ya = 0.0f;
      if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
        const int64_t i = 3 * (pb + static_cast<int64_t>(gy) * W + gx) + c;
        xa = image[i];
        ya = target[i];
      }
      s.a.in.x[r][j] = xa;
      s.a.in.y[r][j] = ya;
    }
    __syncthreads();
    // 2. horizontal 11-tap sums of x, y, xx + yy, xy on kR0H x kR1W, kHR
    //    outputs per item from kHR + 10 inputs held in registers. SSIM needs
    //    the two second moments of x and y only through their sum.
    for (int e = tid; e < kR0H * (kR1W / kHR); e += kSsimThreads) {
      const int r = e / (kR1W / kHR), j0 = (e - r * (kR1W / kHR)) * kHR;
      float m[4][kHR];
#pragma unroll
      for (int o = 0; o < kHR; ++o) m[0][o] = m[1][o] = m[2][o] = m[3][o] = 0.0f;
#pragma unroll
      for (int u = 0; u < kHR + kWin - 1; ++u) {
        const float xa = s.a.in.x[r][j0 + u], ya = s.a.in.y[r][j0 + u];
        const float sq = fmaf(xa, xa, ya * ya), xy = xa * ya;
#pragma unroll
        for (int o = 0; o < kHR; ++o) {
          const int k = u - o;
          if (k >= 0 && k < kWin) {
            m[0][o] = fmaf(A.w[k], xa, m[0][o]);
            m[1][o] = fmaf(A.w[k], ya, m[1][o]);
            m[2][o] = fmaf(A.w[k], sq, m[2][o]);
            m[3][o] = fmaf(A.w[k], xy, m[3][o]);
          }
        }
      }
#pragma unroll
      for (int o = 0; o < kHR; ++o) {
#pragma unroll
        for (int n = 0; n < 4; ++n) s.b.h[n][r][j0 + o] = m[n][o];
      }
    }
    __syncthreads();
    // 3. vertical sums -> SSIM and its partials on kR1H x kR1W, kVR rows per item
    for (int e = tid; e < kR1W * (kR1H / kVR); e += kSsimThreads) {
      const int j = e % kR1W, i0 = (e / kR1W) * kVR;
      float m[4][kVR];
#pragma unroll
      for (int o = 0; o < kVR; ++o) m[0][o] = m[1][o] = m[2][o] = m[3][o] = 0.0f;
#pragma unroll
      for (int u = 0; u < kVR + kWin - 1; ++u) {
#pragma unroll
        for (int n = 0; n < 4; ++n) {
          const float hv = s.b.h[n][i0 + u][j];
#pragma unroll
          for (int o = 0; o < kVR; ++o) {
            const int k = u - o;
            if (k >= 0 && k < kWin) m[n][o] = fmaf(A.w[k], hv, m[n][o]);
          }
        }
      }
      const int gx = gx0 + kHalf + j;
#pragma unroll
      for (int o = 0; o < kVR; ++o) {
        const int i = i0 + o;
        const int gy = gy0 + kHalf + i;
        float p0 = 0.f, p1 = 0.f, p2 = 0.f;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
          const float mux = m[0][o], muy = m[1][o];
          const float mm = mux * mux + muy * muy;
          const float a1 = 2.0f * mux * muy + A.c1, a2 = 2.0f * (m[3][o] - mux * muy) + A.c2;
          const float b1 = mm + A.c1, b2 = (m[2][o] - mm) + A.c2;
          const float ib1 = __fdividef(1.0f, b1), ib2 = __fdividef(1.0f, b2);
          const float ib12 = ib1 * ib2;
          const float ssim = a1 * a2 * ib12;
          p0 = 2.0f * muy * (a2 - a1) * ib12 + 2.0f * mux * ssim * (ib2 - ib1);
          p1 = -ssim * ib2;
          p2 = 2.0f * a1 * ib12;
          if (i >= kHalf && i < kHalf + kTY && j >= kHalf && j < kHalf + kTX) part += A.ssim_scale * (1.0f - ssim);
        }
        s.a.p[0][i][j] = p0;
        s.a.p[1][i][j] = p1;
        s.a.p[2][i][j] = p2;
      }
    }
    __syncthreads();
    // 4. backward horizontal sums of the partials on kR1H x kTX
    for (int e = tid; e < kR1H * (kTX / kBR); e += kSsimThreads) {
      const int i = e / (kTX / kBR), j0 = (e - i * (kTX / kBR)) * kBR;
      float r[3][kBR];
#pragma unroll
      for (int o = 0; o < kBR; ++o) r[0][o] = r[1][o] = r[2][o] = 0.0f;
#pragma unroll
      for (int u = 0; u < kBR + kWin - 1; ++u) {
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          const float pv = s.a.p[n][i][j0 + u];
#pragma unroll
          for (int o = 0; o < kBR; ++o) {
            const int k = u - o;
            if (k >= 0 && k < kWin) r[n][o] = fmaf(A.w[k], pv, r[n][o]);
          }
        }
      }
#pragma unroll
      for (int o = 0; o < kBR; ++o) {
        s.b.q[0][i][j0 + o] = r[0][o];
        s.b.q[1][i][j0 + o] = r[1][o];
        s.b.q[2][i][j0 + o] = r[2][o];
      }
    }
    __syncthreads();
    // 5. backward vertical sums -> dL/dx on the tile, kBR rows per item; x and
    //    y of the tile come again from global memory (the copy in shared
    //    memory now holds the partials; these reads hit L2)
    for (int e = tid; e < kTX * (kTY / kBR); e += kSsimThreads) {
      const int j = e % kTX, i0 = (e / kTX) * kBR;
      float r[3][kBR];
#pragma unroll
      for (int o = 0; o < kBR; ++o) r[0][o] = r[1][o] = r[2][o] = 0.0f;
#pragma unroll
      for (int u = 0; u < kBR + kWin - 1; ++u) {
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          const float qv = s.b.q[n][i0 + u][j];
#pragma unroll
          for (int o = 0; o < kBR; ++o) {
            const int k = u - o;
            if (k >= 0 && k < kWin) r[n][o] = fmaf(A.w[k], qv, r[n][o]);
          }
        }
      }
      const int gx = gx0 + 2 * kHalf + j;
#pragma unroll
      for (int o = 0; o < kBR; ++o) {
        const int gy = gy0 + 2 * kHalf + i0 + o;
        if (gx < W && gy < H) {
          const int64_t idx = 3 * (pb + static_cast<int64_t>(gy) * W + gx) + c;
          const float xv = image[idx], yv = target[idx];
          const float rr = xv - yv;
          const float sg = rr > 0.0f ? 1.0f : (rr < 0.0f ? -1.0f : 0.0f);
          const float dssim = r[0][o] + 2.0f * xv * r[1][o] + yv * r[2][o];
          grad[idx] = A.l1_scale * sg - A.ssim_scale * dssim;
          part += A.l1_scale * fabsf(rr);
        }
      }
    }
    __syncthreads();  // shared memory is rewritten for the next channel
  }

  // 6. loss: block sum in double, one atomic per CTA
  double d = part;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((tid & 31) == 0) s.red[tid >> 5] = d;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < kSsimThreads / 32; ++w) tot += s.red[w];
    atomicAdd(loss, tot);
  }
}

}  // namespace
}  // namespace gs

extern "C" int gs_ssim_loss(const float* image, const float* target, const int32_t* sizes, int32_t V, float lambda,
                            float* dL_dimage, double* loss_dev, gs_stream_t stream_) {
  using namespace gs;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!image || !target || !sizes || !dL_dimage || !loss_dev) return GS_ERR_ARG;
  if (V < 1 || V > kMaxSsimViews || !(lambda >= 0.0f && lambda <= 1.0f)) return GS_ERR_ARG;
  SsimLayout L{};
  L.V = V;
  int64_t tiles = 0, pixels = 0;
  for (int v = 0; v < V; ++v) {
    const int32_t w = sizes[2 * v], h = sizes[2 * v + 1];
    if (w < 1 || h < 1 || w > 32768 || h > 32768) return GS_ERR_ARG;
    L.width[v] = w;
    L.height[v] = h;
    L.ntx[v] = (w + kTX - 1) / kTX;
    L.tile_base[v] = static_cast<int32_t>(tiles);
    L.pix_base[v] = pixels;
    tiles += static_cast<int64_t>(L.ntx[v]) * ((h + kTY - 1) / kTY);
    pixels += static_cast<int64_t>(w) * h;
  }
  L.tile_base[V] = static_cast<int32_t>(tiles);
  L.pix_base[V] = pixels;
  if (tiles > 0x7fffffff) return GS_ERR_ARG;

  SsimArgs A;
  {
    double w[kWin], sum = 0.0;
    for (int k = 0; k < kWin; ++k) {
      const double d = k - kHalf;
      w[k] = exp(-d * d / (2.0 * 1.5 * 1.5));
      sum += w[k];
    }
    for (int k = 0; k < kWin; ++k) A.w[k] = static_cast<float>(w[k] / sum);
  }
  A.c1 = 0.01f * 0.01f;
  A.c2 = 0.03f * 0.03f;
  const double M = 3.0 * static_cast<double>(pixels);
  A.l1_scale = static_cast<float>((1.0 - lambda) / M);
  A.ssim_scale = static_cast<float>(lambda / M);

  // set on every call: the attribute belongs to the current device
  if (cudaFuncSetAttribute(ssim_loss_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(sizeof(SsimSmem))) != cudaSuccess)
    return GS_ERR_CUDA;
  if (cudaMemsetAsync(loss_dev, 0, sizeof(double), stream) != cudaSuccess) return GS_ERR_CUDA;
  ssim_loss_kernel<<<static_cast<unsigned>(tiles), kSsimThreads, sizeof(SsimSmem), stream>>>(image, target, L, A,
                                                                                              dL_dimage, loss_dev);
  return cuda_status(cudaGetLastError());
}

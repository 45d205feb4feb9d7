// Launch interface of the tile rasteriser: the argument structs and the
// launcher templates, which raster_kernels.cuh defines and the
// raster_inst_*.cu units instantiate. raster.cu dispatches to them without
// seeing the kernels, so each kernel variant is compiled in one unit only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_common.cuh"

namespace gs {
namespace rast {

// Optional L1 + L2 image loss computed in the forward's epilogue (target
// null: none). grad and loss as gs_image_loss: dL/dimage = (w1 sign(r) +
// 2 w2 r) / n, loss += sum(w1 |r| + w2 r^2) / n, r = image - target.
struct ImageLoss {
  const float* target;
  float* grad;
  double* loss;
  float w1, w2, inv_n;
  double inv_n_d;
};

// Default splats per shared-memory batch: the forward stages
// max(threads, 128) (at 4K 128 is 3 % faster than 256: warps wait less at the
// batch barrier); the backward, which flushes a batch's gradients between
// two barriers, runs best with small batches: one splat per thread, at least
// 64 and at most 256 (at 4K 8 % faster than 256; on the 16-view workload
// with 16x16 tiles 64 beats 128; 64 with 128 threads is 5 % slower at 4K).
// The cap keeps the backward's shared memory under 48 KB with 512 threads.
// Other sizes are a tuning choice (gs_config.raster_batch_fwd / _bwd).
template <int NT>
constexpr int default_batch_fwd() {
  return NT > 128 ? NT : 128;
}
template <int NT>
constexpr int default_batch_bwd() {
  return NT < 64 ? 64 : (NT > 256 ? 256 : NT);
}

// Shared memory of one CTA with B splats per batch and NW warps. The forward
// keeps it within the 48 KB a CTA gets without an opt-in; the backward's is
// static up to that and dynamic above it (512 splats on tiles of more than 4
// warps: 49 KB at 32x32 tiles and 4 pixels a thread), up to kMaxSmem.
constexpr int fwd_smem_bytes(int B, int NW) { return B * (40 + 2 * NW); }
constexpr int bwd_smem_bytes(int B, int NW) { return B * (80 + 2 * NW) + 4 * NW; }
constexpr int kStaticSmem = 48 * 1024;
constexpr int kMaxSmem = 227 * 1024;  // a CTA's opt-in limit

// Arguments of one forward / backward launch (unpacked into the kernels'
// parameters, so the kernels read them from parameter space as before).
struct FwdArgs {
  const float4* projected;
  const uint32_t* vals;
  const uint2* ranges;
  const uint32_t* order;
  Layout L;
  Consts K;
  float* image;
  float* final_T;
  uint32_t* last;
  ImageLoss IL;
  unsigned long long* counts;
  uint16_t* cull;  // optional: per-entry cull masks written for the backward
};

struct BwdArgs {
  const float4* projected;
  const uint32_t* vals;
  const uint2* ranges;
  const uint32_t* order;
  Layout L;
  Consts K;
  const float* final_T;
  const uint32_t* last;
  const float* dL_dimage;
  float* d_proj;
  unsigned long long* counts;
  const uint16_t* cull;  // optional: the forward's per-entry cull masks
};

template <int TW, int TH, int PPT, int B, bool COUNT>
int launch_fwd(const FwdArgs& a, cudaStream_t stream);

template <int TW, int TH, int PPT, int B, bool BG, bool COUNT>
int launch_bwd(const BwdArgs& a, cudaStream_t stream);

}  // namespace rast
}  // namespace gs

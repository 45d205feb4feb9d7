// Device-side helpers shared by the kernels of libgs_gb300 (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

constexpr int kMaxViews = GS_MAX_VIEWS;

// Upper bound on the iterations of any device-side wait (look-back spins and
// mbarrier waits). A wait that runs out records GS_STATUS_TIMEOUT and the
// kernel carries on with whatever it has, so it always terminates.
constexpr uint32_t kSpinLimit = 1u << 24;

// View layout of one call, passed by value as a kernel parameter (about 1.6
// KB, well inside the parameter space). Built on the host from `sizes`.
struct Layout {
  int32_t V, tile_w, tile_h, n_tiles;
  int32_t width[kMaxViews], height[kMaxViews], ntx[kMaxViews], nty[kMaxViews];
  uint32_t tile_base[kMaxViews + 1];
  uint32_t pix_base[kMaxViews + 1];
};

// Rendering constants as the kernels use them.
struct Consts {
  float near_plane, far_plane, eps2d, alpha_cap, alpha_min, t_stop;
  float bg[3];
  int32_t sh_degree, flags;
};

inline Consts make_consts(const gs_config& c) {
  Consts k;
  k.near_plane = c.near_plane; k.far_plane = c.far_plane; k.eps2d = c.eps2d;
  k.alpha_cap = c.alpha_cap; k.alpha_min = c.alpha_min; k.t_stop = c.t_stop;
  k.bg[0] = c.bg[0]; k.bg[1] = c.bg[1]; k.bg[2] = c.bg[2];
  k.sh_degree = c.sh_degree;
  k.flags = c.flags;
  return k;
}

__device__ __forceinline__ void set_status(int32_t* status, int32_t bits) {
  if (status) atomicOr(status, bits);
}

// View of a global tile id (linear search; V <= 64 and the loop is uniform).
__device__ __forceinline__ int view_of_tile(const Layout& L, uint32_t tile) {
  int v = 0;
  while (v + 1 < L.V && tile >= L.tile_base[v + 1]) ++v;
  return v;
}

// ---- 64-bit single-copy-atomic accesses used by the look-back protocols ----
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void nanosleep_ns(uint32_t ns) { asm volatile("nanosleep.u32 %0;" ::"r"(ns)); }

// ---- mbarrier + 1D bulk copy (TMA) into shared memory ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Bulk copy of `bytes` (multiple of 16) from global `src` (16-byte aligned)
// to shared `dst` (16-byte aligned), completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Bounded wait for phase `parity` of `bar`; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t addr = smem_u32(bar);
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (it > 64) nanosleep_ns(64);
  }
  return false;
}

// ---- fast transcendental pieces with fixed rounding (identical wherever used) ----
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// dL/dr of L = (w1 |r| + w2 r^2) / n for one value r, every step a single
// rounded operation, so that the loss kernel and the forward's fused loss
// produce the same bits.
__device__ __forceinline__ float l1l2_grad(float r, float w1, float w2, float inv_n) {
  const float sg = r > 0.0f ? 1.0f : (r < 0.0f ? -1.0f : 0.0f);
  return __fmul_rn(__fadd_rn(__fmul_rn(w1, sg), __fmul_rn(__fmul_rn(2.0f, w2), r)), inv_n);
}

constexpr int kRecordFloats = GS_RECORD_FLOATS;
constexpr int kDRecordFloats = GS_DRECORD_FLOATS;

}  // namespace gs

// Per-Gaussian stages: SH colour + EWA projection (forward) and its backward.
//
// Paper: arXiv 2606.11390 §4 - the spherical-harmonics and projection
// operators are partitioned per Gaussian and produce, for every camera of the
// batch, a colour and the projected geometry; their backward needs no
// cross-partition atomics. Mathematics: 3D Gaussian Splatting (Kerbl et al.
// 2023, cited in §1).
//
// GB300 design: one thread per Gaussian loops over all views, so the 236-byte
// parameter record is read from HBM once per step whatever the number of
// views. A CTA of 128 Gaussians stages its contiguous parameter slices
// (means, log-scales, quaternions, opacities, SH) into shared memory with TMA
// bulk copies (cp.async.bulk + mbarrier), and writes its projected records
// with three 16-byte stores per thread (a warp's stores cover its records'
// contiguous bytes; staging them through shared memory cost two barriers per
// view: 3.35 -> 2.92 ms for 16 views). With its own copies
// it asks L2 to prefetch (cp.async.bulk.prefetch.L2) the slices of the CTA
// one resident wave later, which then stages from L2 instead of DRAM. With
// several views the SH slice is staged chunk-major by TMA tensor copies
// (cp.async.bulk.tensor), so that the per-view re-reads of the coefficients
// are free of bank conflicts, and the backward's SH gradients leave by
// tensor stores.
//
// Bit-exact tile rectangles. Steps 1-8 of the projection (scale activation
// through the tile rectangle) decide integers, so they are evaluated with
// explicitly rounded single operations (__fmul_rn, __fadd_rn, __fdiv_rn,
// __fsqrt_rn: no contraction into FMA) in a fixed order, and the scale
// activation uses a project-written exponential (Cody & Waite range
// reduction, degree-7 Taylor polynomial) instead of expf, whose last bit is
// not specified. Any float implementation that follows the same order gets
// the same rectangles.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kProjBlock = 128;

// ---- SH slices as 2-D tensors for TMA ----
// An [N][48] float array (the SH coefficients, or their gradients) viewed as
// a 2-D tensor with boxes of 4 floats x kProjBlock rows: box (4j, g0) is the
// float4 chunk j of the CTA's Gaussians, which a tensor copy lays down in
// shared memory as kProjBlock consecutive float4. A CTA's slice thus arrives
// chunk-major (float4 j of Gaussian t at j * kProjBlock + t), where each
// thread's 16-byte loads of its own coefficients are conflict-free; in the
// Gaussian-major order of a plain copy (a 192-byte stride per thread) 8
// threads of a phase meet only 2 of the 8 16-byte bank groups.
//
// Host: encodes the map, or returns false where the array is not 16-byte
// aligned or the driver entry point is unavailable (the kernels then take
// plain loads and stores).
bool encode_sh_map(CUtensorMap* m, const float* base, int64_t N) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode || !aligned16(base) || N <= 0) return false;
  const cuuint64_t dims[2] = {48, static_cast<cuuint64_t>(N)};
  const cuuint64_t strides[1] = {48 * sizeof(float)};
  const cuuint32_t box[2] = {4, kProjBlock};
  const cuuint32_t elem[2] = {1, 1};
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, elem,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Box (x, y) of `map` into shared `dst`, completing on `bar` (rows past the
// tensor's end are filled with zeros). x is a multiple of 4 floats.
__device__ __forceinline__ void tma_load_box(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Shared `src` into box (x, y) of `map` (stored, or added to what is there);
// rows past the tensor's end are not written.
__device__ __forceinline__ void tma_store_box(const CUtensorMap* map, int x, int y, const void* src, bool add) {
  if (add)
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
  else
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
                 "r"(y), "r"(smem_u32(src))
                 : "memory");
}
// CTAs per SM the backward is compiled for (register cap 65536 / (128 x this)).
#ifndef GS_PBWD_MIN_BLOCKS
#define GS_PBWD_MIN_BLOCKS 4
#endif


__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
// ((a0*b0 + a1*b1) + a2*b2), each operation rounded
__device__ __forceinline__ float dot3(float a0, float b0, float a1, float b1, float a2, float b2) {
  return fadd(fadd(fmul(a0, b0), fmul(a1, b1)), fmul(a2, b2));
}

// Scale activation exp(x): Cody-Waite reduction x = k ln2 + r (ln2 split into a
// 16-bit head and a tail), Taylor series of e^r to degree 7 by Horner's rule,
// times 2^k assembled from exponent bits. Input clamped to [-87, 88].
__device__ float exp_scale(float x) {
  if (!(x > -87.0f)) x = -87.0f;
  if (x > 88.0f) x = 88.0f;
  const float log2e = 0x1.715476p+0f;   // 1/ln 2
  const float ln2_hi = 0x1.62e4p-1f;    // 45426/65536
  const float ln2_lo = 0x1.7f7d1cp-20f; // ln 2 - ln2_hi
  const float k = rintf(fmul(x, log2e));
  float r = fsub(x, fmul(k, ln2_hi));
  r = fsub(r, fmul(k, ln2_lo));
  float p = 0x1.a01a02p-13f;               // 1/7!
  p = fadd(fmul(p, r), 0x1.6c16c2p-10f);   // 1/6!
  p = fadd(fmul(p, r), 0x1.111112p-7f);    // 1/5!
  p = fadd(fmul(p, r), 0x1.555556p-5f);    // 1/4!
  p = fadd(fmul(p, r), 0x1.555556p-3f);    // 1/3!
  p = fadd(fmul(p, r), 0.5f);              // 1/2!
  p = fadd(fmul(p, r), 1.0f);
  p = fadd(fmul(p, r), 1.0f);
  const int ki = static_cast<int>(k);
  return fmul(p, __int_as_float((ki + 127) << 23));
}

// View-independent part of a Gaussian.
struct GaussLocal {
  float mean[3];
  float s[3];        // exp(log_scale)
  float qn[4];       // normalised (w, x, y, z)
  float Rm[9];       // rotation of qn, row-major
  float M[9];        // Rm diag(s)
  float Sig[6];      // Sigma = M M^T: 00 01 02 11 12 22
  float o;           // sigmoid(opacity logit)
};

__device__ __forceinline__ void gauss_local(const float* mean, const float* ls, float4 q, float ol, GaussLocal& G) {
  G.mean[0] = mean[0]; G.mean[1] = mean[1]; G.mean[2] = mean[2];
  for (int i = 0; i < 3; ++i) G.s[i] = exp_scale(ls[i]);
  const float n2 = fadd(fadd(fadd(fmul(q.x, q.x), fmul(q.y, q.y)), fmul(q.z, q.z)), fmul(q.w, q.w));
  const float nrm = __fsqrt_rn(n2);
  G.qn[0] = fdiv(q.x, nrm); G.qn[1] = fdiv(q.y, nrm); G.qn[2] = fdiv(q.z, nrm); G.qn[3] = fdiv(q.w, nrm);
  const float qw = G.qn[0], qx = G.qn[1], qy = G.qn[2], qz = G.qn[3];
  const float xx = fmul(qx, qx), yy = fmul(qy, qy), zz = fmul(qz, qz);
  const float xy = fmul(qx, qy), xz = fmul(qx, qz), yz = fmul(qy, qz);
  const float wx = fmul(qw, qx), wy = fmul(qw, qy), wz = fmul(qw, qz);
  float* R = G.Rm;
  R[0] = fsub(1.0f, fmul(2.0f, fadd(yy, zz)));
  R[1] = fmul(2.0f, fsub(xy, wz));
  R[2] = fmul(2.0f, fadd(xz, wy));
  R[3] = fmul(2.0f, fadd(xy, wz));
  R[4] = fsub(1.0f, fmul(2.0f, fadd(xx, zz)));
  R[5] = fmul(2.0f, fsub(yz, wx));
  R[6] = fmul(2.0f, fsub(xz, wy));
  R[7] = fmul(2.0f, fadd(yz, wx));
  R[8] = fsub(1.0f, fmul(2.0f, fadd(xx, yy)));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) G.M[3 * i + j] = fmul(R[3 * i + j], G.s[j]);
  const float* M = G.M;
  G.Sig[0] = dot3(M[0], M[0], M[1], M[1], M[2], M[2]);
  G.Sig[1] = dot3(M[0], M[3], M[1], M[4], M[2], M[5]);
  G.Sig[2] = dot3(M[0], M[6], M[1], M[7], M[2], M[8]);
  G.Sig[3] = dot3(M[3], M[3], M[4], M[4], M[5], M[5]);
  G.Sig[4] = dot3(M[3], M[6], M[4], M[7], M[5], M[8]);
  G.Sig[5] = dot3(M[6], M[6], M[7], M[7], M[8], M[8]);
  G.o = 1.0f / (1.0f + __expf(-ol));
}

// Full Sigma entry (i, j) from the 6 unique values.
__device__ __forceinline__ float sig_at(const float* S, int i, int j) {
  const int a = i < j ? i : j, b = i < j ? j : i;
  return a == 0 ? S[b] : (a == 1 ? S[2 + b] : S[5]);
}

// Per-view projection state (forward values and what the backward reuses).
struct ViewProj {
  bool visible, clamp_x, clamp_y;
  float t[3], u, w, uc, wc;
  float J00, J02, J11, J12;
  float T[6];   // J W (2x3)
  float U[6];   // T Sigma (2x3)
  float a, b, c, det, A, B, C, mx, my, radius;
  int x0, y0, x1, y1;
  uint32_t count;
};

// Steps 2-8 for one view, in the fixed operation order.
__device__ __forceinline__ void project_view(const GaussLocal& G, const gs_camera& cam, int W, int H, int tile_w,
                                             int tile_h, int ntx, int nty, const Consts& K, ViewProj& P) {
  const float* vm = cam.viewmat;
  // 2. view transform t = W mean + t_cam
  for (int i = 0; i < 3; ++i)
    P.t[i] = fadd(dot3(vm[4 * i], G.mean[0], vm[4 * i + 1], G.mean[1], vm[4 * i + 2], G.mean[2]), vm[4 * i + 3]);
  const float tz = P.t[2];
  bool visible = (tz > K.near_plane) && (tz < K.far_plane);
  // 4. Jacobian with frustum clamp at 1.3x the field of view
  const float Wf = static_cast<float>(W), Hf = static_cast<float>(H);
  P.u = fdiv(P.t[0], tz);
  P.w = fdiv(P.t[1], tz);
  const float lox = fdiv(fsub(fmul(-0.15f, Wf), cam.cx), cam.fx);
  const float hix = fdiv(fsub(fmul(1.15f, Wf), cam.cx), cam.fx);
  const float loy = fdiv(fsub(fmul(-0.15f, Hf), cam.cy), cam.fy);
  const float hiy = fdiv(fsub(fmul(1.15f, Hf), cam.cy), cam.fy);
  P.uc = P.u < lox ? lox : (P.u > hix ? hix : P.u);
  P.wc = P.w < loy ? loy : (P.w > hiy ? hiy : P.w);
  P.clamp_x = !(P.u > lox && P.u < hix);
  P.clamp_y = !(P.w > loy && P.w < hiy);
  P.J00 = fdiv(cam.fx, tz);
  P.J02 = fdiv(fmul(-cam.fx, P.uc), tz);
  P.J11 = fdiv(cam.fy, tz);
  P.J12 = fdiv(fmul(-cam.fy, P.wc), tz);
  for (int j = 0; j < 3; ++j) {
    P.T[j] = fadd(fmul(P.J00, vm[j]), fmul(P.J02, vm[8 + j]));
    P.T[3 + j] = fadd(fmul(P.J11, vm[4 + j]), fmul(P.J12, vm[8 + j]));
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j)
      P.U[3 * i + j] = dot3(P.T[3 * i], sig_at(G.Sig, 0, j), P.T[3 * i + 1], sig_at(G.Sig, 1, j), P.T[3 * i + 2],
                            sig_at(G.Sig, 2, j));
  P.a = fadd(dot3(P.U[0], P.T[0], P.U[1], P.T[1], P.U[2], P.T[2]), K.eps2d);
  P.b = dot3(P.U[0], P.T[3], P.U[1], P.T[4], P.U[2], P.T[5]);
  P.c = fadd(dot3(P.U[3], P.T[3], P.U[4], P.T[4], P.U[5], P.T[5]), K.eps2d);
  // 5. determinant, conic
  P.det = fsub(fmul(P.a, P.c), fmul(P.b, P.b));
  visible = visible && (P.det > 0.0f);
  P.A = fdiv(P.c, P.det);
  P.B = fdiv(-P.b, P.det);
  P.C = fdiv(P.a, P.det);
  // 6. 2D mean
  P.mx = fadd(fmul(cam.fx, P.u), cam.cx);
  P.my = fadd(fmul(cam.fy, P.w), cam.cy);
  // 7. radius
  const float half = fmul(0.5f, fadd(P.a, P.c));
  const float disc = fsub(fmul(half, half), P.det);
  const float lam = fadd(half, __fsqrt_rn(fmaxf(0.1f, disc)));
  P.radius = ceilf(fmul(3.0f, __fsqrt_rn(lam)));
  // 8. tile rectangle (NaN-safe clamps)
  const float tw = static_cast<float>(tile_w), th = static_cast<float>(tile_h);
  auto tclamp = [](float f, int n) -> int {
    if (f >= 0.0f) return f <= static_cast<float>(n) ? static_cast<int>(f) : n;
    return 0;
  };
  P.x0 = tclamp(floorf(fdiv(fsub(P.mx, P.radius), tw)), ntx);
  P.x1 = tclamp(ceilf(fdiv(fadd(P.mx, P.radius), tw)), ntx);
  P.y0 = tclamp(floorf(fdiv(fsub(P.my, P.radius), th)), nty);
  P.y1 = tclamp(ceilf(fdiv(fadd(P.my, P.radius), th)), nty);
  uint32_t count = 0;
  if (visible && P.x1 > P.x0 && P.y1 > P.y0) count = static_cast<uint32_t>((P.x1 - P.x0) * (P.y1 - P.y0));
  P.visible = visible && count > 0;
  P.count = P.visible ? count : 0u;
}

// Per-view quantities the backward needs (everything but the rectangle),
// with fast reciprocals. Only the frustum-clamp decision must match the
// forward exactly, so u = tx/tz and w = ty/tz are divided with correct
// rounding as there; the rest only needs to be accurate.
__device__ __forceinline__ void project_view_bwd(const GaussLocal& G, const gs_camera& cam, int W, int H,
                                                 const Consts& K, ViewProj& P) {
  const float* vm = cam.viewmat;
  for (int i = 0; i < 3; ++i)
    P.t[i] = fadd(dot3(vm[4 * i], G.mean[0], vm[4 * i + 1], G.mean[1], vm[4 * i + 2], G.mean[2]), vm[4 * i + 3]);
  const float tz = P.t[2];
  const float itz = rcp_approx(tz);
  const float Wf = static_cast<float>(W), Hf = static_cast<float>(H);
  P.u = fdiv(P.t[0], tz);
  P.w = fdiv(P.t[1], tz);
  const float lox = fdiv(fsub(fmul(-0.15f, Wf), cam.cx), cam.fx);
  const float hix = fdiv(fsub(fmul(1.15f, Wf), cam.cx), cam.fx);
  const float loy = fdiv(fsub(fmul(-0.15f, Hf), cam.cy), cam.fy);
  const float hiy = fdiv(fsub(fmul(1.15f, Hf), cam.cy), cam.fy);
  P.uc = P.u < lox ? lox : (P.u > hix ? hix : P.u);
  P.wc = P.w < loy ? loy : (P.w > hiy ? hiy : P.w);
  P.clamp_x = !(P.u > lox && P.u < hix);
  P.clamp_y = !(P.w > loy && P.w < hiy);
  P.J00 = cam.fx * itz;
  P.J02 = -cam.fx * P.uc * itz;
  P.J11 = cam.fy * itz;
  P.J12 = -cam.fy * P.wc * itz;
  for (int j = 0; j < 3; ++j) {
    P.T[j] = P.J00 * vm[j] + P.J02 * vm[8 + j];
    P.T[3 + j] = P.J11 * vm[4 + j] + P.J12 * vm[8 + j];
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j)
      P.U[3 * i + j] = P.T[3 * i] * sig_at(G.Sig, 0, j) + P.T[3 * i + 1] * sig_at(G.Sig, 1, j) +
                       P.T[3 * i + 2] * sig_at(G.Sig, 2, j);
  P.a = P.U[0] * P.T[0] + P.U[1] * P.T[1] + P.U[2] * P.T[2] + K.eps2d;
  P.b = P.U[0] * P.T[3] + P.U[1] * P.T[4] + P.U[2] * P.T[5];
  P.c = P.U[3] * P.T[3] + P.U[4] * P.T[4] + P.U[5] * P.T[5] + K.eps2d;
  P.det = P.a * P.c - P.b * P.b;
}

// Real SH basis (degree <= 3) in 3DGS coefficient order, Cartesian form.
// Constants: sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the factors of the
// associated Legendre polynomials (Condon-Shortley phase included).
constexpr float kSH0 = 0.28209479177387814f;
constexpr float kSH1 = 0.4886025119029199f;
constexpr float kSH2a = 1.0925484305920792f, kSH2b = 0.31539156525252005f, kSH2c = 0.5462742152960396f;
constexpr float kSH3a = 0.5900435899266435f, kSH3b = 2.890611442640554f, kSH3c = 0.4570457994644658f;
constexpr float kSH3d = 0.3731763325901154f, kSH3e = 1.445305721320277f;

template <int DEG>
__device__ __forceinline__ void sh_basis(const float d[3], float Y[16]) {
  const float x = d[0], y = d[1], z = d[2];
  Y[0] = kSH0;
  if (DEG < 1) return;
  Y[1] = -kSH1 * y; Y[2] = kSH1 * z; Y[3] = -kSH1 * x;
  if (DEG < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kSH2a * x * y;
  Y[5] = -kSH2a * y * z;
  Y[6] = kSH2b * (2.0f * zz - xx - yy);
  Y[7] = -kSH2a * x * z;
  Y[8] = kSH2c * (xx - yy);
  if (DEG < 3) return;
  Y[9] = -kSH3a * y * (3.0f * xx - yy);
  Y[10] = kSH3b * x * y * z;
  Y[11] = -kSH3c * y * (4.0f * zz - xx - yy);
  Y[12] = kSH3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
  Y[13] = -kSH3c * x * (4.0f * zz - xx - yy);
  Y[14] = kSH3e * z * (xx - yy);
  Y[15] = -kSH3a * x * (xx - 3.0f * yy);
}

// Adds sum_i coef_i * grad(Y_i)(d) to g.
template <int DEG>
__device__ __forceinline__ void sh_basis_grad_acc(const float d[3], const float coef[16], float g[3]) {
  const float x = d[0], y = d[1], z = d[2];
  if (DEG < 1) return;
  g[0] += -kSH1 * coef[3];
  g[1] += -kSH1 * coef[1];
  g[2] += kSH1 * coef[2];
  if (DEG < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  g[0] += kSH2a * y * coef[4] - kSH2a * z * coef[7] + kSH2b * (-2.0f * x) * coef[6] + kSH2c * 2.0f * x * coef[8];
  g[1] += kSH2a * x * coef[4] - kSH2a * z * coef[5] + kSH2b * (-2.0f * y) * coef[6] - kSH2c * 2.0f * y * coef[8];
  g[2] += -kSH2a * y * coef[5] + kSH2b * 4.0f * z * coef[6] - kSH2a * x * coef[7];
  if (DEG < 3) return;
  g[0] += -kSH3a * 6.0f * x * y * coef[9] + kSH3b * y * z * coef[10] - kSH3c * (-2.0f * x * y) * coef[11] +
          kSH3d * (-6.0f * x * z) * coef[12] - kSH3c * (4.0f * zz - 3.0f * xx - yy) * coef[13] +
          kSH3e * 2.0f * x * z * coef[14] - kSH3a * (3.0f * xx - 3.0f * yy) * coef[15];
  g[1] += -kSH3a * (3.0f * xx - 3.0f * yy) * coef[9] + kSH3b * x * z * coef[10] -
          kSH3c * (4.0f * zz - xx - 3.0f * yy) * coef[11] + kSH3d * (-6.0f * y * z) * coef[12] -
          kSH3c * (-2.0f * x * y) * coef[13] - kSH3e * 2.0f * y * z * coef[14] - kSH3a * (-6.0f * x * y) * coef[15];
  g[2] += kSH3b * x * y * coef[10] - kSH3c * 8.0f * y * z * coef[11] +
          kSH3d * (6.0f * zz - 3.0f * xx - 3.0f * yy) * coef[12] - kSH3c * 8.0f * x * z * coef[13] +
          kSH3e * (xx - yy) * coef[14];
}

// View direction from the camera centre c = -R^T t_cam to the mean.
__device__ __forceinline__ void view_dir(const gs_camera& cam, const float* mean, float dvec[3], float& dnorm) {
  const float* vm = cam.viewmat;
  for (int j = 0; j < 3; ++j) {
    const float cj = -(vm[j] * vm[3] + vm[4 + j] * vm[7] + vm[8 + j] * vm[11]);
    dvec[j] = mean[j] - cj;
  }
  dnorm = sqrtf(dvec[0] * dvec[0] + dvec[1] * dvec[1] + dvec[2] * dvec[2]);
}

// Shared-memory staging of one CTA's parameter slices (128-byte aligned for
// the tensor copies into `sh`).
struct __align__(128) ParamSmem {
  float4 sh[kProjBlock * 12];       // 24 KB: Gaussian-major, or chunk-major (float4 j of Gaussian t at j * kProjBlock + t)
  float4 quats[kProjBlock];         // 2 KB
  float means[kProjBlock * 3];      // 1.5 KB
  float log_scales[kProjBlock * 3]; // 1.5 KB
  float opac[kProjBlock];           // 0.5 KB
  gs_camera cams[kMaxViews];        // 5 KB
  uint64_t bar;
};

// Loads the CTA's slice [g0, g0+n) of all parameter arrays and the cameras.
// Full, aligned slices go through TMA bulk copies; others through plain
// loads. CM: the SH slice chunk-major, by the tensor copies of `tm_sh` (or
// plain loads in that order), for kernels that re-read the coefficients in
// every view. With one view they are read once, and the contiguous 24 KB
// bulk copy of the Gaussian-major slice is the faster staging: the tensor
// boxes' 16-byte rows at a 192-byte stride took the 4K projection 0.216 ->
// 0.261 ms and its backward 0.452 -> 0.514 ms.
// Optional extra bulk copies that join the parameter staging transaction.
struct ExtraCopies {
  int n = 0;
  void* dst[2];
  const void* src[2];
  const void* pf_src[2];  // the same arrays at the prefetched slice
  uint32_t bytes[2];
};

// Asks L2 to fetch [src, src + bytes) (16-byte aligned, a multiple of 16 bytes).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

template <bool CM>
__device__ __forceinline__ void stage_params(ParamSmem& sm, const float* means, const float* log_scales,
                                             const float* quats, const float* opac, const float* sh, int64_t g0, int n,
                                             const gs_camera* cams, int V, bool use_bulk, const CUtensorMap* tm_sh,
                                             int32_t* status, int64_t g_pf, const ExtraCopies& extra = ExtraCopies()) {
  const int tid = threadIdx.x;
  {
    const float* src = reinterpret_cast<const float*>(cams);
    float* dst = reinterpret_cast<float*>(sm.cams);
    for (int i = tid; i < V * 20; i += blockDim.x) dst[i] = src[i];
  }
  const bool bulk = use_bulk && n == kProjBlock;
  if (bulk) {
    if (tid == 0) {
      mbar_init(&sm.bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
      const uint32_t b_means = kProjBlock * 12, b_quat = kProjBlock * 16, b_op = kProjBlock * 4,
                     b_sh = kProjBlock * 192;
      uint32_t b_extra = 0;
      for (int i = 0; i < extra.n; ++i) b_extra += extra.bytes[i];
      mbar_arrive_expect_tx(&sm.bar, 2 * b_means + b_quat + b_op + b_sh + b_extra);
      for (int i = 0; i < extra.n; ++i) bulk_g2s(extra.dst[i], extra.src[i], extra.bytes[i], &sm.bar);
      bulk_g2s(sm.means, means + g0 * 3, b_means, &sm.bar);
      bulk_g2s(sm.log_scales, log_scales + g0 * 3, b_means, &sm.bar);
      bulk_g2s(sm.quats, quats + g0 * 4, b_quat, &sm.bar);
      bulk_g2s(sm.opac, opac + g0, b_op, &sm.bar);
      if constexpr (CM) {
        for (int j = 0; j < 12; ++j) tma_load_box(&sm.sh[j * kProjBlock], tm_sh, 4 * j, static_cast<int>(g0), &sm.bar);
      } else {
        bulk_g2s(sm.sh, sh + g0 * 48, b_sh, &sm.bar);
      }
      // the slice of the CTA that will take this one's place: into L2 now,
      // so that its staging copies find it there
      if (g_pf >= 0) {
        bulk_prefetch_l2(sh + g_pf * 48, b_sh);
        bulk_prefetch_l2(means + g_pf * 3, b_means);
        bulk_prefetch_l2(log_scales + g_pf * 3, b_means);
        bulk_prefetch_l2(quats + g_pf * 4, b_quat);
        bulk_prefetch_l2(opac + g_pf, b_op);
        for (int i = 0; i < extra.n; ++i) bulk_prefetch_l2(extra.pf_src[i], extra.bytes[i]);
      }
    }
    if (!mbar_wait(&sm.bar, 0)) {
      set_status(status, GS_STATUS_TIMEOUT);
      mbar_wait(&sm.bar, 0);  // give copies in flight one more bounded chance to land
    }
  } else {
    for (int i = tid; i < n * 3; i += blockDim.x) {
      sm.means[i] = means[g0 * 3 + i];
      sm.log_scales[i] = log_scales[g0 * 3 + i];
    }
    for (int i = tid; i < n; i += blockDim.x) {
      sm.quats[i] = make_float4(quats[(g0 + i) * 4], quats[(g0 + i) * 4 + 1], quats[(g0 + i) * 4 + 2],
                                quats[(g0 + i) * 4 + 3]);
      sm.opac[i] = opac[g0 + i];
    }
    const float* shs = sh + g0 * 48;
    float* shd = reinterpret_cast<float*>(sm.sh);
    for (int i = tid; i < n * 48; i += blockDim.x) {
      const int g = i / 48, f = i - 48 * g;  // value f of Gaussian g
      shd[CM ? ((f >> 2) * kProjBlock + g) * 4 + (f & 3) : i] = shs[i];
    }
  }
  __syncthreads();
}

// Per-thread pipeline of the backward's per-view inputs where they are not
// staged in bulk (several views, or a partial slice): the count of view
// v + 2 is loaded into a register and the gradient-record fields of view
// v + 1 (F floats from field `first`; records are 36 bytes, so the copies
// are 4-byte cp.async pieces, and only for a view whose count is non-zero)
// go into the thread's own slot of a shared ring while view v is processed,
// so each view's load latency overlaps the previous view's arithmetic. A
// thread reads only its own slots: the waits are per thread
// (cp.async.wait_group) and need no barrier.
constexpr int kRingFields = 5;

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <int F, class Body>
__device__ __forceinline__ void pipelined_views(bool active, int V, int64_t N, int64_t g, const uint32_t* counts,
                                                const float* d_proj, int first,
                                                float (&ring)[2][kRingFields][kProjBlock], Body body) {
  static_assert(F <= kRingFields, "ring slot too small");
  const int tid = threadIdx.x;
  auto count_of = [&](int v) -> uint32_t { return (active && v < V) ? counts[static_cast<int64_t>(v) * N + g] : 0u; };
  auto fetch = [&](int v, int slot) {
    const float* src = d_proj + (static_cast<int64_t>(v) * N + g) * kDRecordFloats + first;
#pragma unroll
    for (int k = 0; k < F; ++k) cp_async4(&ring[slot][k][tid], src + k);
  };
  uint32_t c_cur = count_of(0), c_next = count_of(1);
  if (c_cur) fetch(0, 0);
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int v = 0; v < V; ++v) {
    const uint32_t c_after = count_of(v + 2);
    if (c_next) fetch(v + 1, (v + 1) & 1);  // non-zero only for v + 1 < V
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // all but view v + 1's copies have landed
    if (c_cur) {
      float f[F];
#pragma unroll
      for (int k = 0; k < F; ++k) f[k] = ring[v & 1][k][tid];
      body(v, f);
    }
    c_cur = c_next;
    c_next = c_after;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

struct __align__(128) ProjFwdSmem {
  ParamSmem p;
};

// Compiled for 5 resident CTAs per SM (at most 102 registers): 0.234 -> 0.225
// ms at 4K against the unconstrained 124 registers (4 CTAs).
template <int DEG, bool CM>
__global__ void __launch_bounds__(kProjBlock, 5) project_fwd_kernel(
    const float* __restrict__ means, const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ opac, const float* __restrict__ sh, int64_t N, const gs_camera* __restrict__ cams,
    const Layout L, const Consts K, float4* __restrict__ projected, short4* __restrict__ rects,
    uint32_t* __restrict__ counts, uint32_t* __restrict__ depth_keys, int use_bulk, int64_t ahead, int32_t* status,
    const __grid_constant__ CUtensorMap tm_sh) {
  __shared__ ProjFwdSmem sm;
  const int tid = threadIdx.x;
  const int64_t g0 = static_cast<int64_t>(blockIdx.x) * kProjBlock;
  const int n = static_cast<int>(N - g0 < kProjBlock ? N - g0 : kProjBlock);
  const int64_t g_pf = (static_cast<int64_t>(blockIdx.x) + ahead) * kProjBlock;
  stage_params<CM>(sm.p, means, log_scales, quats, opac, sh, g0, n, cams, L.V, use_bulk != 0, &tm_sh, status,
                   ahead > 0 && g_pf + kProjBlock <= N ? g_pf : -1);
  const bool active = tid < n;
  constexpr int NB = (DEG + 1) * (DEG + 1);
  GaussLocal G;
  float shc[3 * NB];
  if (active) {
    gauss_local(&sm.p.means[3 * tid], &sm.p.log_scales[3 * tid], sm.p.quats[tid], sm.p.opac[tid], G);
    const float* s1 = reinterpret_cast<const float*>(sm.p.sh) + (CM ? 4 : 48) * tid;
#pragma unroll
    for (int i = 0; i < 3 * NB; ++i) shc[i] = s1[CM ? (i >> 2) * (4 * kProjBlock) + (i & 3) : i];
  }
  for (int v = 0; v < L.V; ++v) {
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
    if (active) {
      const gs_camera& cam = sm.p.cams[v];
      ViewProj P;
      project_view(G, cam, L.width[v], L.height[v], L.tile_w, L.tile_h, L.ntx[v], L.nty[v], K, P);
      const int64_t vg = static_cast<int64_t>(v) * N + g0 + tid;
      counts[vg] = P.count;
      rects[vg] = P.visible ? make_short4(P.x0, P.y0, P.x1, P.y1) : make_short4(0, 0, 0, 0);
      if (depth_keys) depth_keys[vg] = P.visible ? __float_as_uint(P.t[2]) : 0u;
      if (P.visible) {
        float dvec[3], dnorm;
        view_dir(cam, G.mean, dvec, dnorm);
        const float inv = 1.0f / dnorm;
        const float d[3] = {dvec[0] * inv, dvec[1] * inv, dvec[2] * inv};
        float Y[16];
        sh_basis<DEG>(d, Y);
        float rgb[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          float acc = 0.0f;
#pragma unroll
          for (int i = 0; i < NB; ++i) acc += Y[i] * shc[3 * i + ch];
          acc += 0.5f;
          rgb[ch] = acc > 0.0f ? acc : 0.0f;
        }
        r0 = make_float4(P.mx, P.my, P.A, P.B);
        r1 = make_float4(P.C, G.o, P.t[2], P.radius);
        r2 = make_float4(rgb[0], rgb[1], rgb[2], 0.0f);
      }
    }
    if (active) {
      // a warp's three stores cover its 32 records' 1536 contiguous bytes
      float4* dst = projected + (static_cast<int64_t>(v) * N + g0 + tid) * 3;
      dst[0] = r0;
      dst[1] = r1;
      dst[2] = r2;
    }
  }
}

// ---------------------------------------------------------------------------
// Backward: one thread per Gaussian, summed over views (no atomics). The SH
// gradient accumulates in registers and leaves through the thread's own slot
// of the shared-memory staging area, then as coalesced stores.
// ---------------------------------------------------------------------------
// MULTI: the instance for several views, whose per-view inputs go through
// the per-thread pipeline; the single-view instance stages them with the
// parameters (full slices) or reads them directly (the last, partial slice),
// and keeps the registers the pipeline would take.
template <int DEG, bool MULTI>
__global__ void __launch_bounds__(kProjBlock, GS_PBWD_MIN_BLOCKS) project_bwd_kernel(
    const float* __restrict__ means, const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ opac, const float* __restrict__ sh, int64_t N, const gs_camera* __restrict__ cams,
    const Layout L, const Consts K, const uint32_t* __restrict__ counts, const float* __restrict__ d_proj,
    float* __restrict__ d_means, float* __restrict__ d_log_scales, float* __restrict__ d_quats,
    float* __restrict__ d_opac, float* __restrict__ d_sh, int use_bulk, int64_t ahead, int32_t* status,
    const __grid_constant__ CUtensorMap tm_sh, const __grid_constant__ CUtensorMap tm_dsh, int store_tma) {
  constexpr int NB = (DEG + 1) * (DEG + 1);
  __shared__ ParamSmem sm_p;
  struct {
    ParamSmem& p;
  } sm{sm_p};
  const int tid = threadIdx.x;
  const int64_t g0 = static_cast<int64_t>(blockIdx.x) * kProjBlock;
  const int n = static_cast<int>(N - g0 < kProjBlock ? N - g0 : kProjBlock);
  // one view: the CTA's gradient records and tile counts join the staging
  __shared__ __align__(16) float s_dp[MULTI ? 4 : kProjBlock * kDRecordFloats];
  __shared__ __align__(16) uint32_t s_cnt[MULTI ? 4 : kProjBlock];
  // several views: the per-thread view pipeline's ring
  __shared__ __align__(16) float s_ring[MULTI ? 2 : 1][kRingFields][MULTI ? kProjBlock : 1];
  const bool staged = !MULTI && use_bulk == 2 && L.V == 1 && n == kProjBlock;
  ExtraCopies ex;
  if (staged) {
    ex.n = 2;
    ex.dst[0] = s_dp;
    ex.src[0] = d_proj + g0 * kDRecordFloats;
    ex.bytes[0] = kProjBlock * kDRecordFloats * 4;
    ex.dst[1] = s_cnt;
    ex.src[1] = counts + g0;
    ex.bytes[1] = kProjBlock * 4;
  }
  const int64_t g_pf = (static_cast<int64_t>(blockIdx.x) + ahead) * kProjBlock;
  const bool pf = ahead > 0 && g_pf + kProjBlock <= N;
  if (staged) {
    ex.pf_src[0] = d_proj + (pf ? g_pf : g0) * kDRecordFloats;
    ex.pf_src[1] = counts + (pf ? g_pf : g0);
  }
  // the SH slice chunk-major with several views, Gaussian-major with one
  stage_params<MULTI>(sm.p, means, log_scales, quats, opac, sh, g0, n, cams, L.V, use_bulk != 0, &tm_sh, status,
                      pf ? g_pf : -1, ex);
  const bool active = tid < n;
  float gm[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, go = 0.f;
  // coefficient f (0..47) of this thread's Gaussian: the colour pass
  // re-reads them in every view that sees the Gaussian, and in the
  // chunk-major slice a warp's 16-byte loads of one chunk cover 512
  // contiguous bytes
  const float* shb = reinterpret_cast<const float*>(sm.p.sh) + (MULTI ? 4 : 48) * tid;
  auto shc = [&](int f) -> float { return shb[MULTI ? (f >> 2) * (4 * kProjBlock) + (f & 3) : f]; };
  // Pass 1: colour -> SH coefficients and view direction, over all views.
  // The coefficients are read from this thread's staging slot when needed
  // rather than held in registers, and the slot then takes the SH gradients;
  // the geometric pass below starts with those registers free.
  {
    float gsh[3 * NB];
#pragma unroll
    for (int i = 0; i < 3 * NB; ++i) gsh[i] = 0.0f;
    const float* mean = &sm.p.means[3 * tid];
    const float o = active ? 1.0f / (1.0f + __expf(-sm.p.opac[tid])) : 0.0f;
    // one view's colour gradients (dL/dc, and dL/dopacity through the
    // record's field 8)
    auto colour_view = [&](int v, float gc0, float gc1, float gc2, float gop) {
      go += gop * o * (1.0f - o);
      const gs_camera& cam = sm.p.cams[v];
      float dvec[3], dnorm;
      view_dir(cam, mean, dvec, dnorm);
      const float inv = 1.0f / dnorm;
      const float d[3] = {dvec[0] * inv, dvec[1] * inv, dvec[2] * inv};
      float Y[16];
      sh_basis<DEG>(d, Y);
      float acc0 = 0.5f, acc1 = 0.5f, acc2 = 0.5f;
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        acc0 += Y[i] * shc(3 * i);
        acc1 += Y[i] * shc(3 * i + 1);
        acc2 += Y[i] * shc(3 * i + 2);
      }
      const float graw[3] = {acc0 > 0.0f ? gc0 : 0.0f, acc1 > 0.0f ? gc1 : 0.0f, acc2 > 0.0f ? gc2 : 0.0f};
      float coef[16];
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        coef[i] = shc(3 * i) * graw[0] + shc(3 * i + 1) * graw[1] + shc(3 * i + 2) * graw[2];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) gsh[3 * i + ch] += Y[i] * graw[ch];
      }
      float gdir[3] = {0.f, 0.f, 0.f};
      sh_basis_grad_acc<DEG>(d, coef, gdir);
      const float dd = d[0] * gdir[0] + d[1] * gdir[1] + d[2] * gdir[2];
      for (int k = 0; k < 3; ++k) gm[k] += (gdir[k] - d[k] * dd) * inv;
    };
    if constexpr (MULTI) {
      pipelined_views<4>(active, L.V, N, g0 + tid, counts, d_proj, 5, s_ring,
                         [&](int v, const float (&f)[4]) { colour_view(v, f[0], f[1], f[2], f[3]); });
    } else {
      for (int v = 0; active && v < L.V; ++v) {
        const int64_t vg = static_cast<int64_t>(v) * N + g0 + tid;
        if ((staged ? s_cnt[tid] : counts[vg]) == 0) continue;
        const float* dp = staged ? &s_dp[kDRecordFloats * tid] : d_proj + vg * kDRecordFloats;
        colour_view(v, dp[5], dp[6], dp[7], dp[8]);
      }
    }
    // SH gradients into the thread's own slots of the slice (coefficients
    // past the degree get 0), which only this thread reads; they leave at
    // the end by tensor stores (or plain ones)
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      float q[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) q[k] = (4 * i + k < 3 * NB) ? gsh[(4 * i + k < 3 * NB) ? 4 * i + k : 0] : 0.0f;
      sm.p.sh[MULTI ? i * kProjBlock + tid : 12 * tid + i] = make_float4(q[0], q[1], q[2], q[3]);
    }
  }
  // Pass 2: geometry (2D mean and conic -> mean, scales, rotation), over all views.
  GaussLocal G;
  if (active) gauss_local(&sm.p.means[3 * tid], &sm.p.log_scales[3 * tid], sm.p.quats[tid], sm.p.opac[tid], G);
  // one view's geometric gradients (dL/dmean2d, dL/dconic: the record's
  // fields 0..4)
  auto geometry_view = [&](int v, const float (&g9)[5]) {
    const gs_camera& cam = sm.p.cams[v];
    ViewProj P;
    project_view_bwd(G, cam, L.width[v], L.height[v], K, P);
    const float* vm = cam.viewmat;
  // conic -> Sigma2 (a, b, c)
    const float idet = 1.0f / P.det;
    const float gA = g9[2], gB = g9[3], gC = g9[4];
    const float gdet = -(gA * P.c - gB * P.b + gC * P.a) * idet * idet;
    const float ga = gC * idet + gdet * P.c;
    const float gc = gA * idet + gdet * P.a;
    const float gb = -gB * idet - 2.0f * P.b * gdet;
    const float Gs00 = ga, Gs01 = 0.5f * gb, Gs11 = gc;
    // Sigma2 = T Sigma T^T: gT = 2 Gs U, gSigma = T^T Gs T
    float gT[6];
    for (int j = 0; j < 3; ++j) {
      gT[j] = 2.0f * (Gs00 * P.U[j] + Gs01 * P.U[3 + j]);
      gT[3 + j] = 2.0f * (Gs01 * P.U[j] + Gs11 * P.U[3 + j]);
    }
    float gSig[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const float t0i = P.T[i], t1i = P.T[3 + i], t0j = P.T[j], t1j = P.T[3 + j];
        gSig[3 * i + j] = t0i * (Gs00 * t0j + Gs01 * t1j) + t1i * (Gs01 * t0j + Gs11 * t1j);
      }
    // T = J W
    float gJ00 = 0.f, gJ02 = 0.f, gJ11 = 0.f, gJ12 = 0.f;
    for (int j = 0; j < 3; ++j) {
      gJ00 += gT[j] * vm[j];
      gJ02 += gT[j] * vm[8 + j];
      gJ11 += gT[3 + j] * vm[4 + j];
      gJ12 += gT[3 + j] * vm[8 + j];
    }
    const float tz = P.t[2], itz = 1.0f / tz, itz2 = itz * itz;
    float gt[3] = {0.f, 0.f, 0.f};
    gt[2] += -(gJ00 * cam.fx + gJ11 * cam.fy) * itz2 + (gJ02 * cam.fx * P.uc + gJ12 * cam.fy * P.wc) * itz2;
    float gu = g9[0] * cam.fx, gw = g9[1] * cam.fy;
    if (!P.clamp_x) gu += -gJ02 * cam.fx * itz;
    if (!P.clamp_y) gw += -gJ12 * cam.fy * itz;
    gt[0] += gu * itz;
    gt[1] += gw * itz;
    gt[2] += -(gu * P.t[0] + gw * P.t[1]) * itz2;
    for (int k = 0; k < 3; ++k) gm[k] += vm[k] * gt[0] + vm[4 + k] * gt[1] + vm[8 + k] * gt[2];
    // Sigma = M M^T -> gM = 2 gSigma M (gSigma symmetric)
    float gR[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const float gMij =
            2.0f * (gSig[3 * i] * G.M[j] + gSig[3 * i + 1] * G.M[3 + j] + gSig[3 * i + 2] * G.M[6 + j]);
        gR[3 * i + j] = gMij * G.s[j];
        gs[j] += gMij * G.Rm[3 * i + j];
      }
    const float w = G.qn[0], x = G.qn[1], y = G.qn[2], z = G.qn[3];
    float gqn[4];
    gqn[0] = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    gqn[1] = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] -
                    2.f * x * gR[8]);
    gqn[2] = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] -
                    2.f * y * gR[8]);
    gqn[3] = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] + y * gR[5] + x * gR[6] +
                    y * gR[7]);
    for (int k = 0; k < 4; ++k) gq[k] += gqn[k];
  };
  if constexpr (MULTI) {
    pipelined_views<5>(active, L.V, N, g0 + tid, counts, d_proj, 0, s_ring, geometry_view);
  } else {
    for (int v = 0; active && v < L.V; ++v) {
      const int64_t vg = static_cast<int64_t>(v) * N + g0 + tid;
      if ((staged ? s_cnt[tid] : counts[vg]) == 0) continue;
      const float* dp = staged ? &s_dp[kDRecordFloats * tid] : d_proj + vg * kDRecordFloats;
      const float g9[5] = {dp[0], dp[1], dp[2], dp[3], dp[4]};
      geometry_view(v, g9);
    }
  }
  const bool acc = (K.flags & GS_FLAG_ACCUMULATE_GRADS) != 0;
  if (active) {
    const int64_t g = g0 + tid;
    for (int k = 0; k < 3; ++k) {
      d_means[3 * g + k] = gm[k] + (acc ? d_means[3 * g + k] : 0.0f);
      d_log_scales[3 * g + k] = gs[k] * G.s[k] + (acc ? d_log_scales[3 * g + k] : 0.0f);
    }
    // q_n = q/|q|: gq = (gqn - qn (qn . gqn)) / |q|
    const float4 q = sm.p.quats[tid];
    const float qnorm = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float dotp = gq[0] * G.qn[0] + gq[1] * G.qn[1] + gq[2] * G.qn[2] + gq[3] * G.qn[3];
    for (int k = 0; k < 4; ++k)
      d_quats[4 * g + k] = (gq[k] - G.qn[k] * dotp) / qnorm + (acc ? d_quats[4 * g + k] : 0.0f);
    d_opac[g] = go + (acc ? d_opac[g] : 0.0f);
  }
  if (MULTI && store_tma) {
    // the slice's 12 boxes by tensor stores (added to the gradients there
    // when accumulating; rows past N are not written), issued once every
    // thread's shared writes are visible to the copy engine; the issuing
    // thread waits until they have been read out before the CTA exits
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      for (int j = 0; j < 12; ++j) tma_store_box(&tm_dsh, 4 * j, static_cast<int>(g0), &sm.p.sh[j * kProjBlock], acc);
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
  } else {
    __syncthreads();
    float* dst = d_sh + g0 * 48;
    const float* src = reinterpret_cast<const float*>(sm.p.sh);
    for (int i = tid; i < n * 48; i += kProjBlock) {
      const int g = i / 48, f = i - 48 * g;  // value f of Gaussian g
      dst[i] = src[MULTI ? ((f >> 2) * kProjBlock + g) * 4 + (f & 3) : i] + (acc ? dst[i] : 0.0f);
    }
  }
}

}  // namespace

// CTAs of `kernel` resident on the whole current GPU at once (queried once
// per kernel and device, under a lock).
template <int Tag, class F>
int64_t resident_ctas(F kernel) {
  static std::mutex m;
  static int64_t cached[kMaxDevices] = {};
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const bool slot = dev >= 0 && dev < kMaxDevices;
  if (slot) {
    std::lock_guard<std::mutex> lock(m);
    if (cached[dev] > 0) return cached[dev];
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kProjBlock, 0) != cudaSuccess)
    return 0;
  const int64_t n = static_cast<int64_t>(sms) * per_sm;
  if (slot) {
    std::lock_guard<std::mutex> lock(m);
    cached[dev] = n;
  }
  return n;
}

int launch_project_bwd(const float* means, const float* log_scales, const float* quats, const float* opacity_logits,
                       const float* sh, int64_t N, const gs_camera* cams, const Layout& L, const Consts& K,
                       const uint32_t* counts, const float* d_projected, float* d_means, float* d_log_scales,
                       float* d_quats, float* d_opacity_logits, float* d_sh, int32_t* status, cudaStream_t stream) {
  if (N == 0) return GS_OK;
  // several views: the SH slice chunk-major, staged and stored by tensor
  // copies where the arrays allow (tensor coordinates are 32-bit)
  const bool cm = L.V > 1, small = N < (int64_t(1) << 31);
  CUtensorMap tm_sh{}, tm_dsh{};
  const bool bulk = aligned16(means) && aligned16(log_scales) && aligned16(quats) && aligned16(opacity_logits) &&
                    aligned16(sh) && (!cm || (small && encode_sh_map(&tm_sh, sh, N)));
  const int store_tma = cm && small && encode_sh_map(&tm_dsh, d_sh, N) ? 1 : 0;
  // 2: the gradient records and counts can join the bulk staging too
  const int bulk_mode = !bulk ? 0 : (aligned16(d_projected) && aligned16(counts) ? 2 : 1);
  const unsigned blocks = static_cast<unsigned>((N + kProjBlock - 1) / kProjBlock);
#define GS_PBWD_M(D, M)                                                                                           \
  project_bwd_kernel<D, M><<<blocks, kProjBlock, 0, stream>>>(                                                     \
      means, log_scales, quats, opacity_logits, sh, N, cams, L, K, counts, d_projected, d_means, d_log_scales,     \
      d_quats, d_opacity_logits, d_sh, bulk_mode, resident_ctas<10 + D + (M ? 4 : 0)>(project_bwd_kernel<D, M>),   \
      status, tm_sh, tm_dsh, store_tma)
#define GS_PBWD(D)          \
  if (L.V > 1)              \
    GS_PBWD_M(D, true);     \
  else                      \
    GS_PBWD_M(D, false)
  switch (K.sh_degree) {
    case 0: GS_PBWD(0); break;
    case 1: GS_PBWD(1); break;
    case 2: GS_PBWD(2); break;
    default: GS_PBWD(3); break;
  }
#undef GS_PBWD
#undef GS_PBWD_M
  return cuda_status(cudaGetLastError());
}

}  // namespace gs

extern "C" int gs_project(const float* means, const float* log_scales, const float* quats,
                          const float* opacity_logits, const float* sh, int64_t N, const gs_camera* cams_dev,
                          const int32_t* sizes, int32_t V, const gs_config* cfg, float* projected, int16_t* rects,
                          uint32_t* counts, uint32_t* depth_keys, int32_t* status_dev, gs_stream_t stream) {
  using namespace gs;
  if (N < 0 || !cfg || cfg->sh_degree < 0 || cfg->sh_degree > 3) return GS_ERR_ARG;
  Layout L;
  int rc = build_layout(sizes, V, cfg, &L, nullptr);
  if (rc != GS_OK) return rc;
  if (N == 0) return GS_OK;
  if (N * static_cast<int64_t>(V) >= (int64_t(1) << 32)) return GS_ERR_ARG;
  if (!means || !log_scales || !quats || !opacity_logits || !sh || !cams_dev || !projected || !rects || !counts)
    return GS_ERR_ARG;
  if (!aligned16(projected) || (reinterpret_cast<uintptr_t>(rects) & 7u)) return GS_ERR_ARG;
  // several views: the SH slice chunk-major, staged by tensor copies where
  // the array allows (tensor coordinates are 32-bit)
  const bool cm = L.V > 1;
  CUtensorMap tm_sh{};
  const bool bulk = aligned16(means) && aligned16(log_scales) && aligned16(quats) && aligned16(opacity_logits) &&
                    aligned16(sh) && (!cm || (N < (int64_t(1) << 31) && encode_sh_map(&tm_sh, sh, N)));
  const unsigned blocks = static_cast<unsigned>((N + kProjBlock - 1) / kProjBlock);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Consts K = make_consts(*cfg);
#define GS_PFWD_C(D, C)                                                                                     \
  project_fwd_kernel<D, C><<<blocks, kProjBlock, 0, st>>>(                                                        \
      means, log_scales, quats, opacity_logits, sh, N, cams_dev, L, K, reinterpret_cast<float4*>(projected),      \
      reinterpret_cast<short4*>(rects), counts, depth_keys, bulk ? 1 : 0,                                         \
      resident_ctas<D + (C ? 4 : 0)>(project_fwd_kernel<D, C>), status_dev, tm_sh)
#define GS_PFWD(D)         \
  if (cm)                  \
    GS_PFWD_C(D, true);    \
  else                     \
    GS_PFWD_C(D, false)
  switch (cfg->sh_degree) {
    case 0: GS_PFWD(0); break;
    case 1: GS_PFWD(1); break;
    case 2: GS_PFWD(2); break;
    default: GS_PFWD(3); break;
  }
#undef GS_PFWD_C
#undef GS_PFWD
  return cuda_status(cudaGetLastError());
}

extern "C" int gs_project_bwd(const float* means, const float* log_scales, const float* quats,
                              const float* opacity_logits, const float* sh, int64_t N, const gs_camera* cams_dev,
                              const int32_t* sizes, int32_t V, const gs_config* cfg, const uint32_t* counts,
                              const float* d_projected, float* d_means, float* d_log_scales, float* d_quats,
                              float* d_opacity_logits, float* d_sh, int32_t* status_dev, gs_stream_t stream) {
  using namespace gs;
  Layout L;
  int rc = build_layout(sizes, V, cfg, &L, nullptr);
  if (rc != GS_OK) return rc;
  if (N < 0 || cfg->sh_degree < 0 || cfg->sh_degree > 3) return GS_ERR_ARG;
  if (N == 0) return GS_OK;
  if (N * static_cast<int64_t>(V) >= (int64_t(1) << 32)) return GS_ERR_ARG;
  if (!means || !log_scales || !quats || !opacity_logits || !sh || !cams_dev || !counts || !d_projected || !d_means ||
      !d_log_scales || !d_quats || !d_opacity_logits || !d_sh)
    return GS_ERR_ARG;
  return launch_project_bwd(means, log_scales, quats, opacity_logits, sh, N, cams_dev, L, make_consts(*cfg), counts,
                            d_projected, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh, status_dev,
                            reinterpret_cast<cudaStream_t>(stream));
}

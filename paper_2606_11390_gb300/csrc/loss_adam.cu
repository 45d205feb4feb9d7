// Image-space loss gradient and fused Adam.
//
// Paper: arXiv 2606.11390 §4 names an image-space loss per camera (the
// paper's is fused SSIM; the workloads here use L1 + w L2) and §3.2 a fused
// Adam whose speed came from vectorised loads and stores and from caching
// transcendental results in shared memory. Adam is the update of Kingma & Ba
// (2015): bias corrections 1 - beta^t are computed once per CTA from the step
// counter in device memory (so a captured CUDA graph always sees the current
// step) and kept in shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs_common.cuh"
#include "gs_internal.h"

namespace gs {
namespace {

constexpr int kLossThreads = 256;

__global__ void __launch_bounds__(kLossThreads) image_loss_kernel(const float* __restrict__ image,
                                                                   const float* __restrict__ target, int64_t n,
                                                                   float w1, float w2, float* __restrict__ grad,
                                                                   double* __restrict__ loss) {
  __shared__ double s_part[kLossThreads / 32];
  const float inv_n = 1.0f / static_cast<float>(n);
  double acc = 0.0;
  const int64_t n4 = n / 4;
  const float4* img4 = reinterpret_cast<const float4*>(image);
  const float4* tgt4 = reinterpret_cast<const float4*>(target);
  float4* g4 = reinterpret_cast<float4*>(grad);
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 a = img4[i], b = tgt4[i];
    const float r[4] = {a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w};
    float g[4];
    float part = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      g[k] = l1l2_grad(r[k], w1, w2, inv_n);
      part += w1 * fabsf(r[k]) + w2 * r[k] * r[k];
    }
    g4[i] = make_float4(g[0], g[1], g[2], g[3]);
    acc += part;
  }
  for (int64_t i = 4 * n4 + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float r = image[i] - target[i];
    grad[i] = l1l2_grad(r, w1, w2, inv_n);
    acc += w1 * fabsf(r) + w2 * r * r;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kLossThreads / 32; ++w) t += s_part[w];
    atomicAdd(loss, t / static_cast<double>(n));
  }
}

constexpr int kAdamThreads = 256;

__global__ void __launch_bounds__(kAdamThreads) adam_kernel(float* __restrict__ param, const float* __restrict__ grad,
                                                            float* __restrict__ m, float* __restrict__ v, int64_t n,
                                                            float lr, float beta1, float beta2, float eps,
                                                            const int32_t* __restrict__ step) {
  __shared__ float s_bc[2];
  if (threadIdx.x == 0) {
    const float t = static_cast<float>(*step);
    s_bc[0] = 1.0f / (1.0f - powf(beta1, t));          // 1 / (1 - beta1^t)
    s_bc[1] = 1.0f / sqrtf(1.0f - powf(beta2, t));     // 1 / sqrt(1 - beta2^t)
  }
  __syncthreads();
  const float ibc1 = s_bc[0], isbc2 = s_bc[1];
  const int64_t n4 = n / 4;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  float4* p4 = reinterpret_cast<float4*>(param);
  const float4* g4 = reinterpret_cast<const float4*>(grad);
  float4* m4 = reinterpret_cast<float4*>(m);
  float4* v4 = reinterpret_cast<float4*>(v);
  auto upd = [&](float& p, float g, float& mm, float& vv) {
    mm = beta1 * mm + (1.0f - beta1) * g;
    vv = beta2 * vv + (1.0f - beta2) * g * g;
    // p -= lr * (m / bc1) / (sqrt(v / bc2) + eps)
    p -= lr * (mm * ibc1) / (sqrtf(vv) * isbc2 + eps);
  };
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
    float4 p = p4[i], mm = m4[i], vv = v4[i];
    const float4 g = g4[i];
    upd(p.x, g.x, mm.x, vv.x);
    upd(p.y, g.y, mm.y, vv.y);
    upd(p.z, g.z, mm.z, vv.z);
    upd(p.w, g.w, mm.w, vv.w);
    p4[i] = p;
    m4[i] = mm;
    v4[i] = vv;
  }
  for (int64_t i = 4 * n4 + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    upd(param[i], grad[i], m[i], v[i]);
}

int grid_for(int64_t work, int threads) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (work + threads - 1) / threads;
  const int64_t cap = static_cast<int64_t>(sms) * 8;
  return static_cast<int>(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace
}  // namespace gs

extern "C" int gs_image_loss(const float* image, const float* target, int64_t n, float w_l1, float w_l2,
                             float* dL_dimage, double* loss_dev, gs_stream_t stream_) {
  using namespace gs;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (n <= 0 || !image || !target || !dL_dimage || !loss_dev) return GS_ERR_ARG;
  if (!aligned16(image) || !aligned16(target) || !aligned16(dL_dimage)) return GS_ERR_ARG;
  if (cudaMemsetAsync(loss_dev, 0, sizeof(double), stream) != cudaSuccess) return GS_ERR_CUDA;
  image_loss_kernel<<<grid_for(n / 4 + 1, kLossThreads), kLossThreads, 0, stream>>>(image, target, n, w_l1, w_l2,
                                                                                     dL_dimage, loss_dev);
  return cuda_status(cudaGetLastError());
}

extern "C" int gs_adam_step(float* param, const float* grad, float* exp_avg, float* exp_avg_sq, int64_t n, float lr,
                            float beta1, float beta2, float eps, const int32_t* step_dev, gs_stream_t stream_) {
  using namespace gs;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (n < 0 || !step_dev) return GS_ERR_ARG;
  if (n == 0) return GS_OK;
  if (!param || !grad || !exp_avg || !exp_avg_sq) return GS_ERR_ARG;
  if (!aligned16(param) || !aligned16(grad) || !aligned16(exp_avg) || !aligned16(exp_avg_sq)) return GS_ERR_ARG;
  adam_kernel<<<grid_for(n / 4 + 1, kAdamThreads), kAdamThreads, 0, stream>>>(param, grad, exp_avg, exp_avg_sq, n, lr,
                                                                               beta1, beta2, eps, step_dev);
  return cuda_status(cudaGetLastError());
}

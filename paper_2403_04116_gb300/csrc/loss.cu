// L1 term of the training objective (Eq. 11): loss = scale * sum |I - I*| and its gradient
// scale * sign(I - I*), in one pass (HBM-bound: 8 bytes read and 4 written per pixel).
#include "xg_internal.cuh"

namespace xg {

__global__ void __launch_bounds__(256) k_loss_l1(const float* __restrict__ image, const float* __restrict__ target,
                                                 int64_t count, float scale, float* __restrict__ grad,
                                                 float* __restrict__ loss) {
  __shared__ float s_warp[8];
  float acc = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool vec = ((((uintptr_t)image | (uintptr_t)target | (uintptr_t)grad) & 15) == 0);
  const int64_t n4 = vec ? count / 4 : 0;
  for (int64_t i = t0; i < n4; i += stride) {
    const float4 a = reinterpret_cast<const float4*>(image)[i];
    const float4 b = reinterpret_cast<const float4*>(target)[i];
    const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
    acc += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
    float4 g;
    g.x = d0 > 0.f ? scale : (d0 < 0.f ? -scale : 0.f);
    g.y = d1 > 0.f ? scale : (d1 < 0.f ? -scale : 0.f);
    g.z = d2 > 0.f ? scale : (d2 < 0.f ? -scale : 0.f);
    g.w = d3 > 0.f ? scale : (d3 < 0.f ? -scale : 0.f);
    reinterpret_cast<float4*>(grad)[i] = g;
  }
  for (int64_t i = 4 * n4 + t0; i < count; i += stride) {
    const float d = image[i] - target[i];
    acc += fabsf(d);
    grad[i] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < 8 ? s_warp[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(loss, v * scale);
  }
}

cudaError_t launch_loss_l1(const float* image, const float* target, int64_t count, float scale, float* grad,
                           float* loss, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (e != cudaSuccess) return e;
  const int64_t want = (count / 4 + 255) / 256;
  const int blocks = (int)(want < 152 * 8 ? (want > 0 ? want : 1) : 152 * 8);
  k_loss_l1<<<blocks, 256, 0, st>>>(image, target, count, scale, grad, loss);
  return cudaGetLastError();
}

// The decision exponential, scalar and packed, for tests: thread i takes x[2i] and x[2i+1]
// (the second lane repeats the first when n is odd).
__global__ void __launch_bounds__(256) k_exp_check(const float* __restrict__ x, float* __restrict__ ys,
                                                   float* __restrict__ yp, int64_t n) {
  const int64_t i = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n) return;
  const bool two = i + 1 < n;
  const float a = x[i], b = two ? x[i + 1] : a;
  const float2 p = xg_exp2v(make_float2(a, b));
  ys[i] = xg_exp(a);
  yp[i] = p.x;
  if (two) {
    ys[i + 1] = xg_exp(b);
    yp[i + 1] = p.y;
  }
}

cudaError_t launch_exp_check(const float* x, float* ys, float* yp, int64_t n, cudaStream_t st) {
  const int64_t pairs = (n + 1) / 2;
  k_exp_check<<<(unsigned)((pairs + 255) / 256), 256, 0, st>>>(x, ys, yp, n);
  return cudaGetLastError();
}

}  // namespace xg

// Peak FP32 arithmetic rate of the device, measured: the denominator of the compositing
// kernels' roofline.  No stage of the rasterizer is a dense contraction, so the binding
// compute roof is the FP32 pipe; this kernel runs nothing but independent fused
// multiply-add chains on every SM at full occupancy, scalar (FFMA) or on packed pairs
// (the two-lane f32x2 FMA of sm_100 and later), so that its rate is the pipe's limit.
#include "xg_internal.cuh"

namespace xg {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSM = 8;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kPeakThreads) k_fma_chains(int iters, float a, float b, float* sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 1234.5f) sink[0] = s;  // keeps the chains live; never true for the inputs used
}

__global__ void __launch_bounds__(kPeakThreads) k_fma2_chains(int iters, float a, float b, float* sink) {
  float2 x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2((float)(threadIdx.x + c), (float)(threadIdx.x - c));
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s == 1234.5f) sink[0] = s;
}

}  // namespace
}  // namespace xg

extern "C" xg_status xg_fp32_peak(int32_t packed, int32_t iters, float* sink, int64_t* lane_ops, void* stream) {
  using namespace xg;
  if (!sink || !lane_ops || iters < 1 || (packed != 0 && packed != 1)) return XG_ERR_INVALID_ARG;
  const int blocks = kPeakCtasPerSM * device_sms();
  // a = 1 - 2^-20 and b = 2^-10 keep every chain finite and away from denormals
  const float a = 0.99999904632568359375f, b = 0.0009765625f;
  if (packed)
    k_fma2_chains<<<blocks, kPeakThreads, 0, (cudaStream_t)stream>>>(iters, a, b, sink);
  else
    k_fma_chains<<<blocks, kPeakThreads, 0, (cudaStream_t)stream>>>(iters, a, b, sink);
  *lane_ops = (int64_t)blocks * kPeakThreads * iters * kChains * (packed ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

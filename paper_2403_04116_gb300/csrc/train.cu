// The rest of a training step around the rasterizer (Sec. 3.1-3.2 and implementation
// details of Sec. 4.1):
//
//   k_activate / k_activate_bwd  scale = exp(s), opacity = sigmoid(o), and the radiation
//                                intensity of the RIRF, i = sigmoid(sum_k lambda_k f_k) (Eq. 3);
//   k_ssim_*                     the training objective (1 - gamma) L1 + gamma (1 - SSIM)
//                                (Eq. 11) and its gradient, SSIM with the 11-tap Gaussian
//                                window of sigma 1.5 and zero padding;
//   k_adam                       Adam with bias correction and an exponentially decaying
//                                learning rate, the step count kept on the device so the whole
//                                step can be replayed from a CUDA graph;
//   k_psnr_*                     peak signal-to-noise ratio per view (peak 1).
//
// All are elementwise or small-stencil passes bound by memory bandwidth.
#include <math.h>

#include "xg_internal.cuh"

namespace xg {

// ------------------------------------------------------------------------------------------
// activations
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float sigmoidf(float x) { return 1.f / (1.f + expf(-x)); }

__global__ void __launch_bounds__(256) k_activate(const float* __restrict__ log_scale,
                                                  const float* __restrict__ opacity_logit,
                                                  const float* __restrict__ features, const float* __restrict__ lambda,
                                                  int nf, int64_t n, float* __restrict__ scale,
                                                  float* __restrict__ opacity, float* __restrict__ intensity) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
#pragma unroll
  for (int k = 0; k < 3; ++k) scale[k * n + g] = expf(log_scale[k * n + g]);
  opacity[g] = sigmoidf(opacity_logit[g]);
  float z = 0.f;
  for (int k = 0; k < nf; ++k) z = fmaf(lambda[k], features[k * n + g], z);
  intensity[g] = sigmoidf(z);
}

__global__ void __launch_bounds__(256) k_activate_bwd(const float* __restrict__ log_scale,
                                                      const float* __restrict__ opacity_logit,
                                                      const float* __restrict__ features,
                                                      const float* __restrict__ lambda, int nf, int64_t n,
                                                      const float* __restrict__ g_scale,
                                                      const float* __restrict__ g_opacity,
                                                      const float* __restrict__ g_intensity,
                                                      float* __restrict__ g_log_scale,
                                                      float* __restrict__ g_opacity_logit,
                                                      float* __restrict__ g_features) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
#pragma unroll
  for (int k = 0; k < 3; ++k) g_log_scale[k * n + g] = g_scale[k * n + g] * expf(log_scale[k * n + g]);
  const float o = sigmoidf(opacity_logit[g]);
  g_opacity_logit[g] = g_opacity[g] * o * (1.f - o);
  float z = 0.f;
  for (int k = 0; k < nf; ++k) z = fmaf(lambda[k], features[k * n + g], z);
  const float i = sigmoidf(z);
  const float gz = g_intensity[g] * i * (1.f - i);
  for (int k = 0; k < nf; ++k) g_features[k * n + g] = gz * lambda[k];
}

// ------------------------------------------------------------------------------------------
// (1 - gamma) L1 + gamma (1 - SSIM)
// ------------------------------------------------------------------------------------------
constexpr int kWin = 11;
constexpr int kHalf = 5;
constexpr float kC1 = 0.01f * 0.01f;  // (0.01 L)^2, dynamic range L = 1
constexpr float kC2 = 0.03f * 0.03f;  // (0.03 L)^2

struct Window {
  float w[kWin];
};

// Horizontal pass of the 5 blurred moments x, y, x^2, y^2, xy (zero padding).
__global__ void __launch_bounds__(256) k_ssim_h5(const float* __restrict__ x, const float* __restrict__ y, int V,
                                                 int H, int W, Window win, float* __restrict__ out) {
  const int64_t P = (int64_t)V * H * W;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const int c = (int)(i % W);
  const int64_t row = i - c;
  float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kWin; ++k) {
    const int cc = c + k - kHalf;
    if (cc < 0 || cc >= W) continue;
    const float a = x[row + cc], b = y[row + cc], wk = win.w[k];
    m[0] = fmaf(wk, a, m[0]);
    m[1] = fmaf(wk, b, m[1]);
    m[2] = fmaf(wk, a * a, m[2]);
    m[3] = fmaf(wk, b * b, m[3]);
    m[4] = fmaf(wk, a * b, m[4]);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) out[q * P + i] = m[q];
}

// Vertical pass, the SSIM map, and the three adjoint fields of the gradient
// A = dS/dmu_x - 2 mu_x dS/dsxx - mu_y dS/dsxy, B = dS/dsxx, Cm = dS/dsxy; sums of S and |x-y|.
__global__ void __launch_bounds__(256) k_ssim_v5(const float* __restrict__ h5, const float* __restrict__ x,
                                                 const float* __restrict__ y, int V, int H, int W, Window win,
                                                 float* __restrict__ adj, float* __restrict__ sums) {
  __shared__ float s_red[2][8];
  const int64_t P = (int64_t)V * H * W;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float s_val = 0.f, l1 = 0.f;
  if (i < P) {
    const int c = (int)(i % W);
    const int r = (int)((i / W) % H);
    const int64_t plane0 = i - (int64_t)r * W - c;  // start of this view
    float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      const int rr = r + k - kHalf;
      if (rr < 0 || rr >= H) continue;
      const int64_t j = plane0 + (int64_t)rr * W + c;
      const float wk = win.w[k];
#pragma unroll
      for (int q = 0; q < 5; ++q) m[q] = fmaf(wk, h5[q * P + j], m[q]);
    }
    const float mx = m[0], my = m[1];
    const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
    const float n1 = 2.f * mx * my + kC1, n2 = 2.f * sxy + kC2;
    const float d1 = mx * mx + my * my + kC1, d2 = sxx + syy + kC2;
    const float S = (n1 * n2) / (d1 * d2);
    const float dS_dmx = 2.f * my * n2 / (d1 * d2) - S * 2.f * mx / d1;
    const float dS_dsxx = -S / d2;
    const float dS_dsxy = 2.f * n1 / (d1 * d2);
    adj[i] = dS_dmx - 2.f * mx * dS_dsxx - my * dS_dsxy;
    adj[P + i] = dS_dsxx;
    adj[2 * P + i] = dS_dsxy;
    s_val = S;
    l1 = fabsf(x[i] - y[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s_val += __shfl_xor_sync(0xffffffffu, s_val, o);
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_red[0][threadIdx.x >> 5] = s_val;
    s_red[1][threadIdx.x >> 5] = l1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f;
    for (int w = 0; w < 8; ++w) {
      a += s_red[0][w];
      b += s_red[1][w];
    }
    atomicAdd(&sums[0], a);
    atomicAdd(&sums[1], b);
  }
}

// Horizontal pass of the three adjoint fields.
__global__ void __launch_bounds__(256) k_ssim_h3(const float* __restrict__ adj, int V, int H, int W, Window win,
                                                 float* __restrict__ out) {
  const int64_t P = (int64_t)V * H * W;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const int c = (int)(i % W);
  const int64_t row = i - c;
  float m[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kWin; ++k) {
    const int cc = c + k - kHalf;
    if (cc < 0 || cc >= W) continue;
    const float wk = win.w[k];
#pragma unroll
    for (int q = 0; q < 3; ++q) m[q] = fmaf(wk, adj[q * P + row + cc], m[q]);
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) out[q * P + i] = m[q];
}

// Vertical pass and the gradient of the loss with respect to the image.
__global__ void __launch_bounds__(256) k_ssim_grad(const float* __restrict__ h3, const float* __restrict__ x,
                                                   const float* __restrict__ y, int V, int H, int W, Window win,
                                                   float gamma, float* __restrict__ grad) {
  const int64_t P = (int64_t)V * H * W;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const int c = (int)(i % W);
  const int r = (int)((i / W) % H);
  const int64_t plane0 = i - (int64_t)r * W - c;
  float m[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kWin; ++k) {
    const int rr = r + k - kHalf;
    if (rr < 0 || rr >= H) continue;
    const int64_t j = plane0 + (int64_t)rr * W + c;
    const float wk = win.w[k];
#pragma unroll
    for (int q = 0; q < 3; ++q) m[q] = fmaf(wk, h3[q * P + j], m[q]);
  }
  const float xi = x[i], yi = y[i];
  const float dmeanS = (m[0] + 2.f * xi * m[1] + yi * m[2]) / (float)P;
  const float d = xi - yi;
  const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
  grad[i] = (1.f - gamma) * sgn / (float)P - gamma * dmeanS;
}

__global__ void k_ssim_finish(const float* __restrict__ sums, int64_t P, float gamma, float* __restrict__ loss) {
  if (threadIdx.x != 0) return;
  const float mean_s = sums[0] / (float)P, mean_l1 = sums[1] / (float)P;
  loss[0] = (1.f - gamma) * mean_l1 + gamma * (1.f - mean_s);
  loss[1] = mean_l1;
  loss[2] = mean_s;
}

// ------------------------------------------------------------------------------------------
// Adam
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adam(AdamGroups groups, const int32_t* __restrict__ step, float beta1,
                                              float beta2, float eps) {
  const int gi = blockIdx.y;
  if (gi >= groups.count) return;
  const xg_adam_group& G = groups.g[gi];
  const float t = (float)(*step + 1);
  const float bc1 = 1.f - powf(beta1, t), bc2 = 1.f - powf(beta2, t);
  float lr = G.lr;
  if (G.decay_steps > 0) {
    const float frac = fminf(t / (float)G.decay_steps, 1.f);
    lr = G.lr * powf(G.lr_final / G.lr, frac);
  }
  const float step_size = lr / bc1;
  const float inv_sqrt_bc2 = rsqrtf(bc2);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < G.count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float g = G.grad[i];
    const float m = fmaf(beta1, G.m[i], (1.f - beta1) * g);
    const float v = fmaf(beta2, G.v[i], (1.f - beta2) * g * g);
    G.m[i] = m;
    G.v[i] = v;
    G.param[i] -= step_size * m / (sqrtf(v) * inv_sqrt_bc2 + eps);
  }
}

__global__ void k_count_step(int32_t* step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

// ------------------------------------------------------------------------------------------
// PSNR per view
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_psnr_sum(const float* __restrict__ x, const float* __restrict__ y,
                                                  int64_t per_view, float* __restrict__ sse) {
  __shared__ float s_red[8];
  const int v = blockIdx.y;
  float acc = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_view; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = x[v * per_view + i] - y[v * per_view + i];
    acc = fmaf(d, d, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f;
    for (int w = 0; w < 8; ++w) a += s_red[w];
    atomicAdd(&sse[v], a);
  }
}

__global__ void k_psnr_finish(float* __restrict__ sse, int V, int64_t per_view) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const float mse = sse[v] / (float)per_view;
  sse[v] = mse > 0.f ? -10.f * log10f(mse) : INFINITY;
}

}  // namespace xg

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
namespace {
unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

bool valid_raw(const xg_raw_gaussians* r) {
  return r && r->n >= 1 && r->log_scale && r->opacity_logit && r->features && r->lambda && r->n_features >= 1 &&
         r->n_features <= 64;
}

xg::Window gaussian_window() {
  xg::Window w;
  double sum = 0.0, v[xg::kWin];
  for (int k = 0; k < xg::kWin; ++k) {
    const double d = k - xg::kHalf;
    v[k] = exp(-d * d / (2.0 * 1.5 * 1.5));
    sum += v[k];
  }
  for (int k = 0; k < xg::kWin; ++k) w.w[k] = (float)(v[k] / sum);
  return w;
}
}  // namespace

extern "C" {

xg_status xg_activate(const xg_raw_gaussians* raw, float* scale, float* opacity, float* intensity, void* stream) {
  if (!valid_raw(raw) || !scale || !opacity || !intensity) return XG_ERR_INVALID_ARG;
  xg::k_activate<<<blocks_for(raw->n), 256, 0, (cudaStream_t)stream>>>(
      raw->log_scale, raw->opacity_logit, raw->features, raw->lambda, raw->n_features, raw->n, scale, opacity,
      intensity);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

xg_status xg_activate_bwd(const xg_raw_gaussians* raw, const float* g_scale, const float* g_opacity,
                          const float* g_intensity, float* g_log_scale, float* g_opacity_logit, float* g_features,
                          void* stream) {
  if (!valid_raw(raw) || !g_scale || !g_opacity || !g_intensity || !g_log_scale || !g_opacity_logit || !g_features)
    return XG_ERR_INVALID_ARG;
  xg::k_activate_bwd<<<blocks_for(raw->n), 256, 0, (cudaStream_t)stream>>>(
      raw->log_scale, raw->opacity_logit, raw->features, raw->lambda, raw->n_features, raw->n, g_scale, g_opacity,
      g_intensity, g_log_scale, g_opacity_logit, g_features);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

size_t xg_loss_workspace_bytes(int32_t n_views, int32_t width, int32_t height) {
  if (n_views < 1 || width < 1 || height < 1) return 0;
  const size_t P = (size_t)n_views * width * height;
  return (8 * P + 64) * sizeof(float);
}

xg_status xg_loss_l1_ssim(const float* image, const float* target, int32_t n_views, int32_t width, int32_t height,
                          float gamma, float* grad, float* loss, void* workspace, size_t workspace_bytes,
                          void* stream) {
  const size_t need = xg_loss_workspace_bytes(n_views, width, height);
  if (!image || !target || !grad || !loss || need == 0 || !(gamma >= 0.f && gamma <= 1.f)) return XG_ERR_INVALID_ARG;
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace % 16) != 0) return XG_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t P = (int64_t)n_views * width * height;
  float* ws = (float*)workspace;
  float* sums = ws;            // 2 floats (padded to 64)
  float* h5 = ws + 64;         // 5 P
  float* adj = h5 + 5 * P;     // 3 P
  float* h3 = h5;              // reuses the first 3 planes of h5 once adj is built
  const xg::Window win = gaussian_window();
  if (cudaMemsetAsync(sums, 0, 2 * sizeof(float), st) != cudaSuccess) return XG_ERR_CUDA;
  xg::k_ssim_h5<<<blocks_for(P), 256, 0, st>>>(image, target, n_views, height, width, win, h5);
  xg::k_ssim_v5<<<blocks_for(P), 256, 0, st>>>(h5, image, target, n_views, height, width, win, adj, sums);
  xg::k_ssim_h3<<<blocks_for(P), 256, 0, st>>>(adj, n_views, height, width, win, h3);
  xg::k_ssim_grad<<<blocks_for(P), 256, 0, st>>>(h3, image, target, n_views, height, width, win, gamma, grad);
  xg::k_ssim_finish<<<1, 32, 0, st>>>(sums, P, gamma, loss);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

xg_status xg_adam_step(const xg_adam_group* groups, int32_t n_groups, int32_t* step, float beta1, float beta2,
                       float eps, void* stream) {
  if (!groups || n_groups < 1 || n_groups > XG_ADAM_MAX_GROUPS || !step) return XG_ERR_INVALID_ARG;
  xg::AdamGroups G;
  G.count = n_groups;
  int64_t most = 0;
  for (int k = 0; k < n_groups; ++k) {
    const xg_adam_group& g = groups[k];
    if (!g.param || !g.grad || !g.m || !g.v || g.count < 0 || !(g.lr >= 0.f) || g.decay_steps < 0 ||
        (g.decay_steps > 0 && !(g.lr > 0.f && g.lr_final > 0.f)))
      return XG_ERR_INVALID_ARG;
    G.g[k] = g;
    most = g.count > most ? g.count : most;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned bx = (unsigned)(most < 256 * 152 * 4 ? (most + 255) / 256 : 152 * 4);
  if (bx > 0) xg::k_adam<<<dim3(bx, (unsigned)n_groups), 256, 0, st>>>(G, step, beta1, beta2, eps);
  xg::k_count_step<<<1, 32, 0, st>>>(step);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

xg_status xg_psnr(const float* image, const float* target, int32_t n_views, int64_t pixels_per_view, float* psnr,
                  void* stream) {
  if (!image || !target || !psnr || n_views < 1 || pixels_per_view < 1) return XG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(psnr, 0, sizeof(float) * (size_t)n_views, st) != cudaSuccess) return XG_ERR_CUDA;
  const unsigned bx = (unsigned)((pixels_per_view + 255) / 256 < 64 ? (pixels_per_view + 255) / 256 : 64);
  xg::k_psnr_sum<<<dim3(bx, (unsigned)n_views), 256, 0, st>>>(image, target, pixels_per_view, psnr);
  xg::k_psnr_finish<<<(n_views + 255) / 256, 256, 0, st>>>(psnr, n_views, pixels_per_view);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

}  // extern "C"

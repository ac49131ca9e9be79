// Adaptive density control (Sec. 3.2: the Gaussians are adjusted by the adaptive control of
// 3D Gaussian splatting, whose published rules are restated here): statistics of the
// projected-centre gradients, the clone / split / prune plan and its application, and the
// opacity reset.
//
// Decisions are taken in FP32 against thresholds given in log / logit space, so no
// transcendental function enters them: densify where accum / denom >= grad_thresh
// (IEEE division), split rather than clone where the largest log-scale exceeds
// size_log_thresh, prune where the opacity logit is below prune_logit or the largest
// log-scale exceeds max_log_size (children tested with their own log-scale).  Outputs are
// ordered by source Gaussian: [itself if kept], [its clone], [child 0, child 1].
#include <math.h>

#include "xg_internal.cuh"

namespace xg {
namespace {

constexpr float kLnSplit = 0.47000362924573558f;  // ln 1.6: children have scales s / 1.6

struct Rules {
  float grad_thresh, size_log_thresh, prune_logit, max_log_size;
};

struct Plan {
  bool keep, clone, child;
};

__device__ __forceinline__ Plan plan_of(const float* __restrict__ log_scale, const float* __restrict__ opacity_logit,
                                        const float* __restrict__ accum, const int32_t* __restrict__ denom,
                                        int64_t n, int64_t g, const Rules& r) {
  const int32_t d = denom[g];
  const float avg = d > 0 ? __fdiv_rn(accum[g], (float)d) : 0.f;
  const bool dens = avg >= r.grad_thresh;
  const float maxls = fmaxf(fmaxf(log_scale[g], log_scale[n + g]), log_scale[2 * n + g]);
  const bool big = maxls > r.size_log_thresh;
  const bool low = opacity_logit[g] < r.prune_logit;
  const bool large = maxls > r.max_log_size;
  const bool child_large = fsub(maxls, kLnSplit) > r.max_log_size;
  Plan p;
  p.keep = !(dens && big) && !low && !large;
  p.clone = dens && !big && !low && !large;
  p.child = dens && big && !low && !child_large;
  return p;
}

__device__ __forceinline__ uint32_t outputs_of(const Plan& p) {
  return (uint32_t)p.keep + (uint32_t)p.clone + 2u * (uint32_t)p.child;
}

__global__ void k_density_stats(const uint32_t* __restrict__ count, const float* __restrict__ g2d, int64_t n,
                                int n_views, float scale, float* __restrict__ accum, int32_t* __restrict__ denom) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    float a = 0.f;
    int32_t c = 0;
    for (int v = 0; v < n_views; ++v) {
      const int64_t e = (int64_t)v * n + g;
      if (count[e] == 0) continue;  // not visible in this view
      const float2 du = *reinterpret_cast<const float2*>(g2d + 8 * e);
      a = fadd(a, fmul(__fsqrt_rn(fadd(fmul(du.x, du.x), fmul(du.y, du.y))), scale));
      ++c;
    }
    if (c) {
      accum[g] = fadd(accum[g], a);
      denom[g] += c;
    }
  }
}

// Exclusive scan of n u32 counts in place (offsets[n] receives the total), in three
// launches over sort_blocks() contiguous chunks.
__global__ void k_plan_count(const float* __restrict__ log_scale, const float* __restrict__ opacity_logit,
                             const float* __restrict__ accum, const int32_t* __restrict__ denom, int64_t n, Rules r,
                             uint32_t* __restrict__ offsets, unsigned long long* __restrict__ part) {
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(n, beg + chunk);
  unsigned long long local = 0;
  for (int64_t g = beg + threadIdx.x; g < end; g += blockDim.x) {
    const uint32_t c = outputs_of(plan_of(log_scale, opacity_logit, accum, denom, n, g, r));
    offsets[g] = c;
    local += c;
  }
  __shared__ unsigned long long s[256];
  s[threadIdx.x] = local;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void k_plan_top(unsigned long long* __restrict__ part, int nparts, uint32_t* __restrict__ offsets, int64_t n) {
  if (threadIdx.x != 0) return;
  unsigned long long run = 0;
  for (int b = 0; b < nparts; ++b) {
    const unsigned long long c = part[b];
    part[b] = run;
    run += c;
  }
  offsets[n] = (uint32_t)run;
}

__global__ void k_plan_down(int64_t n, const unsigned long long* __restrict__ part, uint32_t* __restrict__ offsets) {
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(n, beg + chunk);
  __shared__ uint32_t s_warp[8];
  __shared__ unsigned long long s_base;
  if (threadIdx.x == 0) s_base = part[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t b0 = beg; b0 < end; b0 += blockDim.x) {
    const int64_t g = b0 + threadIdx.x;
    const uint32_t c = g < end ? offsets[g] : 0u;
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t wbase = 0, total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < warp) wbase += s_warp[w];
      total += s_warp[w];
    }
    if (g < end) offsets[g] = (uint32_t)s_base + wbase + x - c;
    __syncthreads();
    if (threadIdx.x == 0) s_base += total;
    __syncthreads();
  }
}

struct Sets {
  xg_param_set in, m, v, out, om, ov;
};

__device__ __forceinline__ void copy_gaussian(const xg_param_set& a, int64_t g, const xg_param_set& b, int64_t o,
                                              bool zero) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    b.mean[k * b.n + o] = zero ? 0.f : a.mean[k * a.n + g];
    b.log_scale[k * b.n + o] = zero ? 0.f : a.log_scale[k * a.n + g];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) b.quat[k * b.n + o] = zero ? 0.f : a.quat[k * a.n + g];
  b.opacity_logit[o] = zero ? 0.f : a.opacity_logit[g];
  for (int k = 0; k < a.n_features; ++k) b.features[k * b.n + o] = zero ? 0.f : a.features[k * a.n + g];
}

__global__ void k_plan_apply(Sets S, const float* __restrict__ accum, const int32_t* __restrict__ denom, Rules r,
                             const uint32_t* __restrict__ offsets, const float* __restrict__ normals) {
  const xg_param_set& P = S.in;
  const int64_t n = P.n;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const Plan pl = plan_of(P.log_scale, P.opacity_logit, accum, denom, n, g, r);
    int64_t o = offsets[g];
    if (pl.keep) {
      copy_gaussian(P, g, S.out, o, false);
      copy_gaussian(S.m, g, S.om, o, false);
      copy_gaussian(S.v, g, S.ov, o, false);
      ++o;
    }
    if (pl.clone) {
      copy_gaussian(P, g, S.out, o, false);
      copy_gaussian(S.m, g, S.om, o, true);
      copy_gaussian(S.v, g, S.ov, o, true);
      ++o;
    }
    if (pl.child) {
      // centres mu + R diag(s) z with R from the normalised quaternion (w, x, y, z)
      float q[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) q[k] = P.quat[k * n + g];
      const float inv = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
      const float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
      const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                             {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                             {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
      float s[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) s[k] = expf(P.log_scale[k * n + g]);
      for (int c = 0; c < 2; ++c) {
        copy_gaussian(P, g, S.out, o, false);
        copy_gaussian(S.m, g, S.om, o, true);
        copy_gaussian(S.v, g, S.ov, o, true);
        float sz[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) sz[k] = s[k] * normals[(c * 3 + k) * n + g];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          S.out.mean[k * S.out.n + o] = P.mean[k * n + g] + (R[k][0] * sz[0] + R[k][1] * sz[1] + R[k][2] * sz[2]);
          S.out.log_scale[k * S.out.n + o] = fsub(P.log_scale[k * n + g], kLnSplit);
        }
        ++o;
      }
    }
  }
}

__global__ void k_opacity_reset(float* __restrict__ opacity_logit, float* __restrict__ adam_m,
                                float* __restrict__ adam_v, int64_t n, float reset_logit) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    opacity_logit[g] = fminf(opacity_logit[g], reset_logit);
    if (adam_m) adam_m[g] = 0.f;
    if (adam_v) adam_v[g] = 0.f;
  }
}

bool valid_set(const xg_param_set* p, int64_t n, int32_t nf) {
  return p && p->mean && p->log_scale && p->quat && p->opacity_logit && p->n == n && p->n_features == nf &&
         (nf == 0 || p->features);
}

bool rules_of(const xg_density_rules* r, Rules* out) {
  if (!r || isnan(r->grad_thresh) || isnan(r->size_log_thresh) || isnan(r->prune_logit) || isnan(r->max_log_size))
    return false;
  *out = Rules{r->grad_thresh, r->size_log_thresh, r->prune_logit, r->max_log_size};
  return true;
}

unsigned blocks_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)device_sms() * 16); }

}  // namespace
}  // namespace xg

extern "C" {

xg_status xg_densify_stats(xg_frame* frame, float scale, float* accum, int32_t* denom, void* stream) {
  if (!frame || !accum || !denom || !isfinite(scale)) return XG_ERR_INVALID_ARG;
  xg::k_density_stats<<<xg::blocks_for(frame->n), 256, 0, (cudaStream_t)stream>>>(
      frame->p.count, frame->p.grad2d, frame->n, frame->n_views, scale, accum, denom);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

size_t xg_densify_workspace_bytes(void) { return sizeof(unsigned long long) * xg::sort_blocks(); }

xg_status xg_densify_plan(const xg_param_set* params, const float* accum, const int32_t* denom,
                          const xg_density_rules* rules, uint32_t* offsets, void* workspace, void* stream) {
  xg::Rules r;
  if (!params || !xg::valid_set(params, params->n, params->n_features) || params->n < 1 ||
      params->n > ((int64_t)1 << 30) || !accum || !denom || !offsets || !workspace || !xg::rules_of(rules, &r))
    return XG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  auto* part = (unsigned long long*)workspace;
  const int blocks = xg::sort_blocks();  // the count xg_densify_workspace_bytes sized `workspace` for
  xg::k_plan_count<<<blocks, 256, 0, st>>>(params->log_scale, params->opacity_logit, accum, denom, params->n, r,
                                           offsets, part);
  xg::k_plan_top<<<1, 32, 0, st>>>(part, blocks, offsets, params->n);
  xg::k_plan_down<<<blocks, 256, 0, st>>>(params->n, part, offsets);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

xg_status xg_densify_apply(const xg_param_set* params, const xg_param_set* adam_m, const xg_param_set* adam_v,
                           const float* accum, const int32_t* denom, const xg_density_rules* rules,
                           const uint32_t* offsets, const float* normals, const xg_param_set* out_params,
                           const xg_param_set* out_m, const xg_param_set* out_v, void* stream) {
  xg::Rules r;
  if (!params || !out_params) return XG_ERR_INVALID_ARG;
  const int64_t n = params->n, m = out_params->n;
  const int32_t nf = params->n_features;
  if (!xg::valid_set(params, n, nf) || !xg::valid_set(adam_m, n, nf) || !xg::valid_set(adam_v, n, nf) || n < 1 ||
      n > ((int64_t)1 << 30) || !accum || !denom || !offsets || !normals || !xg::rules_of(rules, &r))
    return XG_ERR_INVALID_ARG;
  if (!out_m || !out_v || out_m->n != m || out_v->n != m) return XG_ERR_INVALID_ARG;
  if (m == 0) return XG_OK;  // every Gaussian pruned: nothing to write
  if (!xg::valid_set(out_params, m, nf) || !xg::valid_set(out_m, m, nf) || !xg::valid_set(out_v, m, nf))
    return XG_ERR_INVALID_ARG;
  xg::Sets S{*params, *adam_m, *adam_v, *out_params, *out_m, *out_v};
  xg::k_plan_apply<<<xg::blocks_for(n), 256, 0, (cudaStream_t)stream>>>(S, accum, denom, r, offsets, normals);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

xg_status xg_opacity_reset(float* opacity_logit, float* adam_m, float* adam_v, int64_t n, float reset_logit,
                           void* stream) {
  if (!opacity_logit || n < 1 || isnan(reset_logit)) return XG_ERR_INVALID_ARG;
  xg::k_opacity_reset<<<xg::blocks_for(n), 256, 0, (cudaStream_t)stream>>>(opacity_logit, adam_m, adam_v, n,
                                                                           reset_logit);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

}  // extern "C"

// Front-to-back alpha compositing of intensity per detector pixel (Eq. 10) and its
// backward pass.
//
// One CTA per (tile, view), one thread per pixel, each warp an 8x4 block of pixels.  The
// tile's depth-sorted list is staged through shared memory in batches (the record of each
// Gaussian read once per CTA and broadcast to all its pixels); a CTA stops fetching as soon
// as every pixel's transmittance has hit the floor (__syncthreads_count).  Per batch, each
// warp compacts the staged entries whose footprint box meets its 8x4 block (ballot) and
// walks only those.
//
// Most (pixel, list entry) pairs lie outside the Gaussian's footprint.  Each staged record
// carries a conservative exponent threshold ln(1/(255 o)) - 1e-4: below it the opacity
// provably stays under 1/255 (the FP32 exp used for the decision is accurate to 3e-7), so
// the pair is skipped without evaluating exp.  Every other pair goes through the fixed
// FP32 decision sequence, so decisions are exactly those of the full test.
//
// The backward pass walks each pixel's list back to front from its last contributor,
// recovering the transmittance by division instead of storing it.  Per list entry, a warp
// with any contributing pixel reduces its 7 gradient terms with an 8-value reduce-scatter
// butterfly (9 shuffles; lane 4k ends with the sum of term k), adds them to shared memory,
// and after the batch each Gaussian gets two float4 atomics in global memory.
#include "xg_internal.cuh"

namespace xg {


constexpr int kMaxWarps = 16;  // 512-thread tiles

// Stage list entries [first, first + cnt) of a tile: records rescaled for the exponent,
// the exponent threshold, and a conservative pixel box of each footprint.
__device__ __forceinline__ void stage_batch(const uint32_t* __restrict__ value, const float4* __restrict__ rec,
                                            int64_t vn_base, uint32_t first, int cnt, const Camera& cam, float4* s_a,
                                            float4* s_b, float4* s_box, uint32_t* s_g) {
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const uint32_t g = value[first + j];
    const float4 a = rec[2 * (vn_base + g)];
    const float4 b = rec[2 * (vn_base + g) + 1];
    // (u_x, u_y, -a/2, -b) and (-c/2, opacity, intensity): exact rescalings of the conic;
    // w: exponent below which the opacity cannot reach 1/255
    s_a[j] = make_float4(a.x, a.y, -0.5f * a.z, -a.w);
    s_b[j] = make_float4(-0.5f * b.x, b.y, b.z, logf(kAlphaMin / b.y) - 1e-4f);
    // Pixels where the opacity can reach 1/255 satisfy d^T K d <= 2 ln(255 o); their x
    // offsets lie within sqrt(2 ln(255 o) (K^-1)_xx), and likewise for y.  Widened by 0.1 %
    // and 0.01 px, far beyond FP32 rounding, so the box never drops a contributing pixel.
    const float two_l = 2.f * fmaxf(logf(255.f * b.y), 0.f);
    const float det = a.z * b.x - a.w * a.w;
    float ex = INFINITY, ey = INFINITY;
    if (det > 0.f) {
      ex = sqrtf(two_l * b.x / det) * 1.001f + 0.01f;
      ey = sqrtf(two_l * a.z / det) * 1.001f + 0.01f;
    }
    const float cx = a.x + cam.hw, cy = a.y + cam.hh;  // footprint centre in pixel indices
    s_box[j] = make_float4(cx - ex, cx + ex, cy - ey, cy + ey);
    if (s_g) s_g[j] = g;
  }
}

// The staged entries whose box meets this warp's 8x4 pixel block [bx0, bx0+7] x [by0, by0+3],
// in list order; returns their count.
__device__ __forceinline__ int warp_list(const float4* s_box, int cnt, float bx0, float by0, uint16_t* list,
                                         int lane) {
  const uint32_t lt_mask = (1u << lane) - 1u;
  int m = 0;
  for (int j0 = 0; j0 < cnt; j0 += 32) {
    const int j = j0 + lane;
    bool hit = false;
    if (j < cnt) {
      const float4 bx = s_box[j];
      hit = bx.x <= bx0 + 7.f && bx.y >= bx0 && bx.z <= by0 + 3.f && bx.w >= by0;
    }
    const uint32_t mask = __ballot_sync(0xffffffffu, hit);
    if (hit) list[m + __popc(mask & lt_mask)] = (uint16_t)j;
    m += __popc(mask);
  }
  __syncwarp();
  return m;
}

// Work counters: one atomic per warp.
__device__ __forceinline__ void add_counts(uint32_t ev, uint32_t nc, unsigned long long* ev_out,
                                           unsigned long long* nc_out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ev += __shfl_xor_sync(0xffffffffu, ev, o);
    nc += __shfl_xor_sync(0xffffffffu, nc, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (ev) atomicAdd(ev_out, (unsigned long long)ev);
    if (nc) atomicAdd(nc_out, (unsigned long long)nc);
  }
}

// Pixel of thread `tid` inside a tw-wide tile: warps own 8x4 blocks, row-major.
__device__ __forceinline__ void pixel_in_tile(int tid, int tw, int& lx, int& ly) {
  const int lane = tid & 31, warp = tid >> 5, wx = tw >> 3;
  lx = (warp % wx) * 8 + (lane & 7);
  ly = (warp / wx) * 4 + (lane >> 3);
}

// Sum of v[k] over the warp for k = 0..7, scattered: returns the total of term
// ((lane >> 2) & 7) in every lane.  9 shuffles instead of 8 x 5.
__device__ __forceinline__ float warp_reduce_scatter8(const float (&v)[8], int lane) {
  float a[4], c[2];
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float send = b4 ? v[k] : v[k + 4];
    a[k] = (b4 ? v[k + 4] : v[k]) + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = b3 ? a[k] : a[k + 2];
    c[k] = (b3 ? a[k + 2] : a[k]) + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float d = (b2 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, b2 ? c[0] : c[1], 4);
  d += __shfl_xor_sync(0xffffffffu, d, 2);
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  return d;
}

// The exponent -1/2 d^T K d and sigma = min(0.99, o e^p) in the fixed FP32 sequence.
__device__ __forceinline__ float power_of(const float4 a, const float nc, float px, float py, float& dx, float& dy) {
  dx = fsub(a.x, px);
  dy = fsub(a.y, py);
  float p = fmul(a.w, fmul(dx, dy));
  p = ffma(nc, fmul(dy, dy), p);
  p = ffma(a.z, fmul(dx, dx), p);
  return p;
}

template <int kBatch>
__global__ void __launch_bounds__(512) k_render_fwd(const uint2* __restrict__ range, const uint32_t* __restrict__ value,
                                                    const float4* __restrict__ rec, int64_t n, int W, int H,
                                                    int tiles_x, int64_t tiles_per_view, int tw,
                                                    const Camera* __restrict__ cams, DevStatus* __restrict__ st,
                                                    float* __restrict__ image, uint32_t* __restrict__ ncontrib,
                                                    float* __restrict__ tfinal, uint32_t* __restrict__ last) {
  __shared__ float4 s_a[kBatch], s_b[kBatch], s_box[kBatch];
  __shared__ uint16_t s_list[kMaxWarps][kBatch];
  const int tile = blockIdx.x, v = blockIdx.y;
  const int th_ = blockDim.x / tw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int lx, ly;
  pixel_in_tile(threadIdx.x, tw, lx, ly);
  const int tx0 = (tile % tiles_x) * tw, ty0 = (tile / tiles_x) * th_;
  const int x = tx0 + lx, y = ty0 + ly;
  const float bx0 = (float)(tx0 + (lx & ~7)), by0 = (float)(ty0 + (ly & ~3));  // this warp's block
  const bool inside = x < W && y < H;
  const Camera cam = cams[v];
  const float px = fsub((float)x, cam.hw), py = fsub((float)y, cam.hh);
  const uint2 r = st->code == XG_OK ? range[(int64_t)v * tiles_per_view + tile] : make_uint2(0u, 0u);
  const int nlist = (int)(r.y - r.x);
  const int64_t vn_base = (int64_t)v * n;
  uint16_t* my_list = s_list[warp];

  float T = 1.0f, C = 0.0f;
  uint32_t nc = 0, lastp = 0, nev = 0;
  bool done = !inside;
  for (int base = 0; base < nlist; base += kBatch) {
    if (__syncthreads_count(done) == (int)blockDim.x) break;
    const int cnt = min(kBatch, nlist - base);
    stage_batch(value, rec, vn_base, r.x + base, cnt, cam, s_a, s_b, s_box, nullptr);
    __syncthreads();
    if (__all_sync(0xffffffffu, done)) continue;
    const int m = warp_list(s_box, cnt, bx0, by0, my_list, lane);
    if (!done) {
      for (int k = 0; k < m; ++k) {
        const int j = my_list[k];
        const float4 a = s_a[j];
        const float4 b = s_b[j];
        float dx, dy;
        const float p = power_of(a, b.x, px, py, dx, dy);
        ++nev;
        if (p < b.w) continue;  // opacity provably below 1/255
        const float al = fminf(kAlphaMax, fmul(b.y, xg_exp(p)));
        if (al < kAlphaMin) continue;
        const float Tn = fmul(T, fsub(1.0f, al));
        if (Tn < kTMin) {
          done = true;
          break;
        }
        C = ffma(b.z, fmul(al, T), C);
        T = Tn;
        ++nc;
        lastp = (uint32_t)(base + j + 1);
      }
    }
  }
  if (inside) {
    const int64_t pix = ((int64_t)v * H + y) * W + x;
    image[pix] = C;
    tfinal[pix] = T;
    last[pix] = lastp;
    if (ncontrib) ncontrib[pix] = nc;
  }
  add_counts(nev, nc, &st->fwd_evaluated, &st->fwd_contrib);
}

cudaError_t launch_render_fwd(xg_frame* f, float* image, uint32_t* n_contrib, cudaStream_t st) {
  const FramePtrs& p = f->p;
  dim3 grid((unsigned)f->tiles_per_view, (unsigned)f->n_views);
  Timed t(f, kRenderFwd, st);
  const int threads = f->cfg.tile_w * f->cfg.tile_h;
#define XG_FWD(B)                                                                                              \
  k_render_fwd<B><<<grid, threads, 0, st>>>(p.range, p.value[f->sorted_buf], p.rec, f->n, f->width, f->height, \
                                            f->tiles_x, f->tiles_per_view, f->cfg.tile_w, p.cam, p.status,     \
                                            image, n_contrib, p.tfinal, p.last)
  switch (f->cfg.batch) {
    case 64: XG_FWD(64); break;
    case 128: XG_FWD(128); break;
    default: XG_FWD(256); break;
  }
#undef XG_FWD
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// backward
// ------------------------------------------------------------------------------------------
template <int kBatch>
__global__ void __launch_bounds__(512) k_render_bwd(const uint2* __restrict__ range, const uint32_t* __restrict__ value,
                                                    const float4* __restrict__ rec, int64_t n, int n_views, int W,
                                                    int H, int tiles_x, int64_t tiles_per_view, int tw,
                                                    const Camera* __restrict__ cams, DevStatus* __restrict__ st,
                                                    const float* __restrict__ grad_image,
                                                    const float* __restrict__ tfinal, const uint32_t* __restrict__ last,
                                                    float* __restrict__ g2d) {
  __shared__ float4 s_a[kBatch], s_b[kBatch], s_box[kBatch];
  __shared__ uint32_t s_g[kBatch];
  __shared__ __align__(16) float s_acc[kBatch * 8];
  __shared__ uint16_t s_list[kMaxWarps][kBatch];
  __shared__ uint32_t s_maxlast;
  if (st->code != XG_OK) return;
  const int tile = blockIdx.x, v = blockIdx.y;
  const int th_ = blockDim.x / tw;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int lx, ly;
  pixel_in_tile(threadIdx.x, tw, lx, ly);
  const int tx0 = (tile % tiles_x) * tw, ty0 = (tile / tiles_x) * th_;
  const int x = tx0 + lx, y = ty0 + ly;
  const float bx0 = (float)(tx0 + (lx & ~7)), by0 = (float)(ty0 + (ly & ~3));
  const bool inside = x < W && y < H;
  const Camera cam = cams[v];
  const float px = fsub((float)x, cam.hw), py = fsub((float)y, cam.hh);
  const uint2 r = range[(int64_t)v * tiles_per_view + tile];
  const int64_t vn_base = (int64_t)v * n;
  uint16_t* my_list = s_list[warp];

  float G = 0.f, Tc = 1.f;
  uint32_t L = 0;
  if (inside) {
    const int64_t pix = ((int64_t)v * H + y) * W + x;
    G = grad_image[pix];
    Tc = tfinal[pix];
    L = G != 0.f ? last[pix] : 0u;
  }
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  if (L) atomicMax(&s_maxlast, L);
  __syncthreads();
  const int maxl = (int)s_maxlast;
  // the longest prefix any lane of this warp walks
  uint32_t wl = L;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
  float A = 0.f;  // intensity blended behind the current position, per unit transmittance
  uint32_t nev = 0, ncon = 0;

  for (int end_pos = maxl; end_pos > 0; end_pos -= kBatch) {
    const int base = max(0, end_pos - kBatch);
    const int cnt = end_pos - base;
    stage_batch(value, rec, vn_base, r.x + base, cnt, cam, s_a, s_b, s_box, s_g);
    for (int i = threadIdx.x; i < cnt * 8; i += blockDim.x) s_acc[i] = 0.f;
    __syncthreads();
    if ((uint32_t)base < wl) {
      const int m = warp_list(s_box, min(cnt, (int)wl - base), bx0, by0, my_list, lane);
      for (int k = m - 1; k >= 0; --k) {
        const int j = my_list[k];
        float gv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool contrib = false;
        if ((uint32_t)(base + j) < L) {
          ++nev;
          const float4 a = s_a[j];
          const float4 b = s_b[j];
          float dx, dy;
          const float p = power_of(a, b.x, px, py, dx, dy);
          if (p >= b.w) {
            const float e = xg_exp(p);
            const float oe = fmul(b.y, e);
            const float al = fminf(kAlphaMax, oe);
            if (al >= kAlphaMin) {
              contrib = true;
              ++ncon;
              Tc = __fdividef(Tc, 1.f - al);
              const float in = b.z;
              gv[6] = G * al * Tc;                 // dL/d intensity
              const float dL_dal = G * Tc * (in - A);
              A = al * in + (1.f - al) * A;
              if (oe < kAlphaMax) {
                gv[5] = dL_dal * e;                // dL/d opacity
                const float dp = dL_dal * al;      // dL/d power
                gv[0] = dp * (2.f * a.z * dx + a.w * dy);  // dL/du_x = dp * -(a dx + b dy)
                gv[1] = dp * (2.f * b.x * dy + a.w * dx);  // dL/du_y = dp * -(b dx + c dy)
                gv[2] = dp * (-0.5f * dx * dx);            // dL/d conic a
                gv[3] = dp * (-dx * dy);                   // dL/d conic b
                gv[4] = dp * (-0.5f * dy * dy);            // dL/d conic c
              }
            }
          }
        }
        if (__any_sync(0xffffffffu, contrib)) {
          const float sum = warp_reduce_scatter8(gv, lane);
          const int q = (lane >> 2) & 7;
          if ((lane & 3) == 0 && q < 7) atomicAdd(&s_acc[j * 8 + q], sum);
        }
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      const float4 a0 = *reinterpret_cast<const float4*>(&s_acc[j * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&s_acc[j * 8 + 4]);
      if (a0.x != 0.f || a0.y != 0.f || a0.z != 0.f || a0.w != 0.f || a1.x != 0.f || a1.y != 0.f ||
          a1.z != 0.f) {
        float4* dst = reinterpret_cast<float4*>(g2d + 8 * (vn_base + s_g[j]));
        atomicAdd(dst, a0);
        atomicAdd(dst + 1, a1);
      }
    }
    __syncthreads();
  }
  add_counts(nev, ncon, &st->bwd_evaluated, &st->bwd_contrib);
}

cudaError_t launch_render_bwd(xg_frame* f, const float* grad_image, cudaStream_t st) {
  const FramePtrs& p = f->p;
  const int64_t VN = (int64_t)f->n_views * f->n;
  cudaError_t e;
  {
    Timed t(f, kMemset, st);
    e = cudaMemsetAsync(p.grad2d, 0, sizeof(float) * 8 * (size_t)VN, st);
  }
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)f->tiles_per_view, (unsigned)f->n_views);
  Timed t(f, kRenderBwd, st);
  const int threads = f->cfg.tile_w * f->cfg.tile_h;
#define XG_BWD(B)                                                                                                \
  k_render_bwd<B><<<grid, threads, 0, st>>>(p.range, p.value[f->sorted_buf], p.rec, f->n, f->n_views, f->width, \
                                            f->height, f->tiles_x, f->tiles_per_view, f->cfg.tile_w, p.cam,    \
                                            p.status, grad_image, p.tfinal, p.last, p.grad2d)
  switch (f->cfg.batch) {
    case 64: XG_BWD(64); break;
    case 128: XG_BWD(128); break;
    default: XG_BWD(256); break;
  }
#undef XG_BWD
  return cudaGetLastError();
}

}  // namespace xg

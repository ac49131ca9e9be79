// Front-to-back alpha compositing of intensity per detector pixel (Eq. 10) and its
// backward pass.
//
// One CTA per (tile, view).  Each thread owns PPT pixels (1, 2 or 4, 4 rows apart), so
// a warp owns an 8 x 4*PPT block.  The tile's depth-sorted list is staged through shared
// memory in batches (the record of each Gaussian read once per CTA and broadcast to all its
// pixels); a CTA stops fetching as soon as every pixel's transmittance has hit the floor
// (__syncthreads_count).  Per batch, each warp compacts the staged entries whose footprint
// box meets its block (ballot) and walks only those.
//
// Most (pixel, list entry) pairs lie outside the Gaussian's footprint.  Each staged record
// carries a conservative exponent threshold ln(1/(255 o)) - 1e-4: below it the opacity
// provably stays under 1/255 (the FP32 exp used for the decision is accurate to 3e-7), so
// the pair is skipped without evaluating exp.  Every other pair goes through the fixed
// FP32 decision sequence, so decisions are exactly those of the full test.
//
// The backward pass walks each pixel's list back to front from its last contributor,
// recovering the transmittance by division instead of storing it.  Per list entry, a warp
// with contributing pixels sums its 7 per-pixel terms (six moments of dL/dpower and the
// intensity term) with an 8-value reduce-scatter butterfly (9 shuffles; lane 4k ends with
// the sum of term k) into shared memory.  After the batch each Gaussian's sums are turned into dL/du, dL/dconic and
// dL/dopacity and added to global memory with two float4 atomics.
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

// The staged entries whose box meets this warp's pixel block [bx0, bx0+7] x [by0, by1], in
// list order; returns their count.
__device__ __forceinline__ int warp_list(const float4* s_box, int cnt, float bx0, float by0, float by1,
                                         uint16_t* list, int lane) {
  const uint32_t lt_mask = (1u << lane) - 1u;
  int m = 0;
  for (int j0 = 0; j0 < cnt; j0 += 32) {
    const int j = j0 + lane;
    bool hit = false;
    if (j < cnt) {
      const float4 bx = s_box[j];
      hit = bx.x <= bx0 + 7.f && bx.y >= bx0 && bx.z <= by1 && bx.w >= by0;
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

// First pixel of thread `tid` inside a tw-wide tile: warps own 8 x 4*PPT blocks, row-major;
// the thread's other pixels are 4, 8, 12 rows below.
template <int PPT>
__device__ __forceinline__ void pixel_in_tile(int tid, int tw, int& lx, int& ly) {
  const int lane = tid & 31, warp = tid >> 5, wx = tw >> 3;
  lx = (warp % wx) * 8 + (lane & 7);
  ly = (warp / wx) * (4 * PPT) + (lane >> 3);
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

// The exponent -1/2 d^T K d = dx (na dx + nb dy) + (nc dy) dy, with na = -a/2, nb = -b,
// nc = -c/2, in the fixed FP32 sequence.
__device__ __forceinline__ float power_of(const float4 a, const float nc, float px, float py, float& dx, float& dy) {
  dx = fsub(a.x, px);
  dy = fsub(a.y, py);
  const float t = ffma(a.z, dx, fmul(a.w, dy));
  return ffma(dx, t, fmul(fmul(nc, dy), dy));
}

template <int kBatch, int PPT>
__global__ void __launch_bounds__(512) k_render_fwd(const uint2* __restrict__ range, const uint32_t* __restrict__ value,
                                                    const float4* __restrict__ rec, int64_t n, int W, int H,
                                                    int tiles_x, int64_t tiles_per_view, int tw, int th,
                                                    const Camera* __restrict__ cams, DevStatus* __restrict__ st,
                                                    float* __restrict__ image, uint32_t* __restrict__ ncontrib,
                                                    float* __restrict__ tfinal, uint32_t* __restrict__ last) {
  __shared__ float4 s_a[kBatch], s_b[kBatch], s_box[kBatch];
  __shared__ uint16_t s_list[kMaxWarps][kBatch];
  const int tile = blockIdx.x, v = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int lx, ly;
  pixel_in_tile<PPT>(threadIdx.x, tw, lx, ly);
  const int tx0 = (tile % tiles_x) * tw, ty0 = (tile / tiles_x) * th;
  const int x = tx0 + lx;
  const float bx0 = (float)(tx0 + (lx & ~7)), by0 = (float)(ty0 + (ly & ~3));  // this warp's block
  const float by1 = by0 + (float)(4 * PPT - 1);
  const Camera cam = cams[v];
  const float px = fsub((float)x, cam.hw);
  const uint2 r = st->code == XG_OK ? range[(int64_t)v * tiles_per_view + tile] : make_uint2(0u, 0u);
  const int nlist = (int)(r.y - r.x);
  const int64_t vn_base = (int64_t)v * n;
  uint16_t* my_list = s_list[warp];

  float py[PPT], T[PPT], C[PPT];
  uint32_t nc[PPT], lastp[PPT];
  bool done[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int y = ty0 + ly + 4 * q;
    py[q] = fsub((float)y, cam.hh);
    T[q] = 1.0f;
    C[q] = 0.0f;
    nc[q] = lastp[q] = 0;
    done[q] = !(x < W && y < H);
  }
  uint32_t nev = 0;
  auto all_done = [&]() {
    bool d = true;
#pragma unroll
    for (int q = 0; q < PPT; ++q) d = d && done[q];
    return d;
  };
  for (int base = 0; base < nlist; base += kBatch) {
    if (__syncthreads_count(all_done()) == (int)blockDim.x) break;
    const int cnt = min(kBatch, nlist - base);
    stage_batch(value, rec, vn_base, r.x + base, cnt, cam, s_a, s_b, s_box, nullptr);
    __syncthreads();
    if (__all_sync(0xffffffffu, all_done())) continue;
    const int m = warp_list(s_box, cnt, bx0, by0, by1, my_list, lane);
#pragma unroll 2
    for (int k = 0; k < m; ++k) {
      if (all_done()) break;
      const int j = my_list[k];
      const float4 a = s_a[j];
      const float4 b = s_b[j];
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        if (done[q]) continue;
        float dx, dy;
        const float p = power_of(a, b.x, px, py[q], dx, dy);
        ++nev;
        if (p < b.w) continue;  // opacity provably below 1/255
        const float al = fminf(kAlphaMax, fmul(b.y, xg_exp(p)));
        if (al < kAlphaMin) continue;
        const float Tn = fmul(T[q], fsub(1.0f, al));
        if (Tn < kTMin) {
          done[q] = true;
          continue;
        }
        C[q] = ffma(b.z, fmul(al, T[q]), C[q]);
        T[q] = Tn;
        ++nc[q];
        lastp[q] = (uint32_t)(base + j + 1);
      }
    }
  }
  uint32_t nct = 0;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int y = ty0 + ly + 4 * q;
    nct += nc[q];
    if (x < W && y < H) {
      const int64_t pix = ((int64_t)v * H + y) * W + x;
      image[pix] = C[q];
      tfinal[pix] = T[q];
      last[pix] = lastp[q];
      if (ncontrib) ncontrib[pix] = nc[q];
    }
  }
  add_counts(nev, nct, &st->fwd_evaluated, &st->fwd_contrib);
}

cudaError_t launch_render_fwd(xg_frame* f, float* image, uint32_t* n_contrib, cudaStream_t st) {
  const FramePtrs& p = f->p;
  dim3 grid((unsigned)f->tiles_per_view, (unsigned)f->n_views);
  Timed t(f, kRenderFwd, st);
  const int ppt = f->cfg.pixels_per_thread;
  const int threads = f->cfg.tile_w * f->cfg.tile_h / ppt;
#define XG_FWD(B, P)                                                                                       \
  k_render_fwd<B, P><<<grid, threads, 0, st>>>(p.range, p.value[f->sorted_buf], p.rec, f->n, f->width,    \
                                               f->height, f->tiles_x, f->tiles_per_view, f->cfg.tile_w,   \
                                               f->cfg.tile_h, p.cam, p.status, image, n_contrib, p.tfinal, \
                                               p.last)
  switch (ppt * 1000 + f->cfg.batch) {
    case 1064: XG_FWD(64, 1); break;
    case 1128: XG_FWD(128, 1); break;
    case 1256: XG_FWD(256, 1); break;
    case 2064: XG_FWD(64, 2); break;
    case 2128: XG_FWD(128, 2); break;
    case 2256: XG_FWD(256, 2); break;
    case 4064: XG_FWD(64, 4); break;
    case 4128: XG_FWD(128, 4); break;
    default: XG_FWD(256, 4); break;
  }
#undef XG_FWD
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// backward
// ------------------------------------------------------------------------------------------
template <int kBatch, int PPT>
__global__ void __launch_bounds__(512) k_render_bwd(const uint2* __restrict__ range, const uint32_t* __restrict__ value,
                                                    const float4* __restrict__ rec, int64_t n, int n_views, int W,
                                                    int H, int tiles_x, int64_t tiles_per_view, int tw, int th,
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
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int lx, ly;
  pixel_in_tile<PPT>(threadIdx.x, tw, lx, ly);
  const int tx0 = (tile % tiles_x) * tw, ty0 = (tile / tiles_x) * th;
  const int x = tx0 + lx;
  const float bx0 = (float)(tx0 + (lx & ~7)), by0 = (float)(ty0 + (ly & ~3));
  const float by1 = by0 + (float)(4 * PPT - 1);
  const Camera cam = cams[v];
  const float px = fsub((float)x, cam.hw);
  const uint2 r = range[(int64_t)v * tiles_per_view + tile];
  const int64_t vn_base = (int64_t)v * n;
  uint16_t* my_list = s_list[warp];

  float py[PPT], G[PPT], Tc[PPT], A[PPT];
  uint32_t L[PPT];
  uint32_t lmax = 0;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int y = ty0 + ly + 4 * q;
    py[q] = fsub((float)y, cam.hh);
    G[q] = 0.f;
    Tc[q] = 1.f;
    A[q] = 0.f;  // intensity blended behind the current position, per unit transmittance
    L[q] = 0;
    if (x < W && y < H) {
      const int64_t pix = ((int64_t)v * H + y) * W + x;
      G[q] = grad_image[pix];
      Tc[q] = tfinal[pix];
      L[q] = G[q] != 0.f ? last[pix] : 0u;
    }
    lmax = max(lmax, L[q]);
  }
  if (threadIdx.x == 0) s_maxlast = 0;
  __syncthreads();
  if (lmax) atomicMax(&s_maxlast, lmax);
  __syncthreads();
  const int maxl = (int)s_maxlast;
  // the longest prefix any pixel of this warp walks
  uint32_t wl = lmax;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
  uint32_t nev = 0, ncon = 0;

  for (int end_pos = maxl; end_pos > 0; end_pos -= kBatch) {
    const int base = max(0, end_pos - kBatch);
    const int cnt = end_pos - base;
    stage_batch(value, rec, vn_base, r.x + base, cnt, cam, s_a, s_b, s_box, s_g);
    for (int i = threadIdx.x; i < cnt * 8; i += blockDim.x) s_acc[i] = 0.f;
    __syncthreads();
    if ((uint32_t)base < wl) {
      const int m = warp_list(s_box, min(cnt, (int)wl - base), bx0, by0, by1, my_list, lane);
      for (int k = m - 1; k >= 0; --k) {
        const int j = my_list[k];
        const float4 a = s_a[j];
        const float4 b = s_b[j];
        float gv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool contrib = false;
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
          if ((uint32_t)(base + j) >= L[q]) continue;
          ++nev;
          float dx, dy;
          const float p = power_of(a, b.x, px, py[q], dx, dy);
          if (p < b.w) continue;
          const float e = xg_exp(p);
          const float oe = fmul(b.y, e);
          const float al = fminf(kAlphaMax, oe);
          if (al < kAlphaMin) continue;
          contrib = true;
          ++ncon;
          Tc[q] = __fdividef(Tc[q], 1.f - al);
          const float in = b.z;
          gv[6] += G[q] * al * Tc[q];                 // dL/d intensity
          const float dL_dal = G[q] * Tc[q] * (in - A[q]);
          A[q] = al * in + (1.f - al) * A[q];
          if (oe < kAlphaMax) {
            // moments of dp = dL/d power: sum dp (dL/d opacity = sum dp / opacity, as
            // d sigma / d opacity = e^p = sigma / opacity) and sum dp d, dp d d^T; the
            // conic and the opacity enter once per Gaussian at the flush
            const float dp = dL_dal * al;
            const float sx = dp * dx, sy = dp * dy;
            gv[0] += sx;
            gv[1] += sy;
            gv[2] += sx * dx;
            gv[3] += sx * dy;
            gv[4] += sy * dy;
            gv[5] += dp;
          }
        }
        if (__any_sync(0xffffffffu, contrib)) {
          const float sum = warp_reduce_scatter8(gv, lane);
          const int t8 = (lane >> 2) & 7;
          if ((lane & 3) == 0 && t8 < 7) atomicAdd(&s_acc[j * 8 + t8], sum);
        }
      }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
      // sums over the tile's pixels: S_x, S_y, S_xx, S_xy, S_yy, S_1 of dp = dL/dpower times
      // (d, d d^T, 1), and dL/dintensity.  power = -1/2 (a dx^2 + 2 b dx dy + c dy^2), d = u - p:
      // dL/du = -(K (S_x, S_y)), dL/d(a, b, c) = (-S_xx / 2, -S_xy, -S_yy / 2),
      // dL/dopacity = S_1 / opacity.
      const float4 m0 = *reinterpret_cast<const float4*>(&s_acc[j * 8]);
      const float4 m1 = *reinterpret_cast<const float4*>(&s_acc[j * 8 + 4]);
      if (m0.x != 0.f || m0.y != 0.f || m0.z != 0.f || m0.w != 0.f || m1.x != 0.f || m1.y != 0.f ||
          m1.z != 0.f) {
        const float4 a = s_a[j];  // (u_x, u_y, -a/2, -b)
        const float nc = s_b[j].x;  // -c/2
        const float4 q0 = make_float4(2.f * a.z * m0.x + a.w * m0.y, a.w * m0.x + 2.f * nc * m0.y, -0.5f * m0.z,
                                      -m0.w);
        const float4 q1 = make_float4(-0.5f * m1.x, __fdividef(m1.y, s_b[j].y), m1.z, 0.f);
        float4* dst = reinterpret_cast<float4*>(g2d + 8 * (vn_base + s_g[j]));
        atomicAdd(dst, q0);
        atomicAdd(dst + 1, q1);
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
  const int ppt = f->cfg.pixels_per_thread;
  const int threads = f->cfg.tile_w * f->cfg.tile_h / ppt;
#define XG_BWD(B, P)                                                                                            \
  k_render_bwd<B, P><<<grid, threads, 0, st>>>(p.range, p.value[f->sorted_buf], p.rec, f->n, f->n_views,       \
                                               f->width, f->height, f->tiles_x, f->tiles_per_view,             \
                                               f->cfg.tile_w, f->cfg.tile_h, p.cam, p.status, grad_image,      \
                                               p.tfinal, p.last, p.grad2d)
  switch (ppt * 1000 + f->cfg.batch) {
    case 1064: XG_BWD(64, 1); break;
    case 1128: XG_BWD(128, 1); break;
    case 1256: XG_BWD(256, 1); break;
    case 2064: XG_BWD(64, 2); break;
    case 2128: XG_BWD(128, 2); break;
    case 2256: XG_BWD(256, 2); break;
    case 4064: XG_BWD(64, 4); break;
    case 4128: XG_BWD(128, 4); break;
    default: XG_BWD(256, 4); break;
  }
#undef XG_BWD
  return cudaGetLastError();
}

}  // namespace xg

// Front-to-back alpha compositing of intensity per detector pixel (Eq. 10) and its
// backward pass.
//
// One CTA per (tile, view).  Each thread owns PPT pixels (1, 2 or 4, 4 rows apart), so
// a warp owns an 8 x 4*PPT block.  The tile's depth-sorted list is staged through shared
// memory in batches (the record of each Gaussian read once per CTA and broadcast to all its
// pixels); a CTA stops fetching as soon as every pixel's transmittance has hit the floor
// (__syncthreads_count).  Per batch, each warp compacts the staged entries whose footprint
// can reach its block (box test, then the largest exponent over the block) and walks only
// those.
//
// A thread's pixels are processed in pairs with the packed two-lane FP32 instructions of
// sm_100+ (f32x2 add / mul / fma): both pixels of a pair see the same list entry, so the
// exponent, exp, opacity, transmittance and colour (forward) or gradient terms (backward)
// of the two run as one instruction stream.  Each lane rounds as the scalar operation
// would, so results are those of the documented scalar FP32 sequence.
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
// the sum of term k) into shared memory.  After the batch each Gaussian's sums are turned
// into dL/du, dL/dconic and dL/dopacity and added to global memory with two float4 atomics.
#include "xg_internal.cuh"

namespace xg {


constexpr int kMaxWarps = 16;  // 512-thread tiles

// One list entry staged for the pixel-pair kernels: every field duplicated so that one
// broadcast shared load yields both lanes of a packed operand.  q0..q3 = (u_x u_x u_y u_y),
// (na na nb nb), (nc nc o o), (i i thr thr) with na, nb, nc = -a/2, -b, -c/2 and thr the
// exponent threshold; box = conservative pixel box (x0, x1, y0, y1) of the footprint.
struct Staged {
  float4 q0, q1, q2, q3, box;
};

__device__ __forceinline__ Staged stage_record(const float4 a, const float4 b, const Camera& cam) {
  Staged e;
  const float na = -0.5f * a.z, nb = -a.w, nc = -0.5f * b.x;
  // ln(255 o) with the fast hardware log (absolute error below 1e-5 here): the threshold
  // keeps a 1e-4 margin and the box 0.1 % + 0.01 px, so both stay conservative
  const float l255o = __logf(255.f * b.y);
  const float thr = -l255o - 1e-4f;
  e.q0 = make_float4(a.x, a.x, a.y, a.y);
  e.q1 = make_float4(na, na, nb, nb);
  e.q2 = make_float4(nc, nc, b.y, b.y);
  e.q3 = make_float4(b.z, b.z, thr, thr);
  const float two_l = 2.f * fmaxf(l255o, 0.f);
  const float det = a.z * b.x - a.w * a.w;
  float ex = INFINITY, ey = INFINITY;
  if (det > 0.f) {
    const float sdet = __fdividef(two_l, det);
    ex = __fsqrt_rn(sdet * b.x) * 1.001f + 0.01f;
    ey = __fsqrt_rn(sdet * a.z) * 1.001f + 0.01f;
  }
  const float cx = a.x + cam.hw, cy = a.y + cam.hh;
  e.box = make_float4(cx - ex, cx + ex, cy - ey, cy + ey);
  return e;
}

// Stages list entries [first, first + cnt) of a tile into shared memory for the whole CTA.
template <int kBatch>
__device__ __forceinline__ void stage_batch_pairs(const uint32_t* __restrict__ value, const float4* __restrict__ rec,
                                                  int64_t vn_base, uint32_t first, int cnt, const Camera& cam,
                                                  float4 (*s_q)[kBatch], float4* s_box, uint32_t* s_g) {
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const uint32_t g = value[first + j];
    const Staged e = stage_record(rec[2 * (vn_base + g)], rec[2 * (vn_base + g) + 1], cam);
    s_q[0][j] = e.q0;
    s_q[1][j] = e.q1;
    s_q[2][j] = e.q2;
    s_q[3][j] = e.q3;
    s_box[j] = e.box;
    if (s_g) s_g[j] = g;
  }
}

// Largest exponent na dx^2 + nb dx dy + nc dy^2 (na, nc < 0) over the offsets
// d in [dx0, dx1] x [dy0, dy1]: 0 if the rectangle holds the centre, else the best point on
// one of its edges (the concave quadratic restricted to an edge peaks at the clamped
// stationary point).
__device__ __forceinline__ float max_power_over_rect(float na, float nb, float nc, float dx0, float dx1, float dy0,
                                                     float dy1) {
  if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) return 0.f;
  const float ky = __fdividef(-nb, 2.f * nc), kx = __fdividef(-nb, 2.f * na);
  float best = -INFINITY;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float X = e ? dx1 : dx0;
    const float dy = fminf(fmaxf(ky * X, dy0), dy1);
    best = fmaxf(best, X * (na * X + nb * dy) + nc * dy * dy);
    const float Y = e ? dy1 : dy0;
    const float dx = fminf(fmaxf(kx * Y, dx0), dx1);
    best = fmaxf(best, dx * (na * dx + nb * Y) + nc * Y * Y);
  }
  return best;
}

// Whether a footprint can reach the warp's pixel block [bx0, bx0+7] x [by0, by1] (pixel
// indices): its box meets the block and the largest exponent over the block's pixel centres
// is within a margin (1e-2 + 1e-3 |thr|, far above FP32 rounding of these sums) of the
// threshold below which no pixel can reach opacity 1/255.  Only entries that no pixel of the
// block could take fail, so decisions are unchanged.
__device__ __forceinline__ bool reaches_block(const float4 box, float ux, float uy, float na, float nb, float nc,
                                              float thr, float bx0, float by0, float by1, const Camera& cam) {
  if (!(box.x <= bx0 + 7.f && box.y >= bx0 && box.z <= by1 && box.w >= by0)) return false;
  const float cx = ux + cam.hw, cy = uy + cam.hh;
  const float best = max_power_over_rect(na, nb, nc, cx - (bx0 + 7.f), cx - bx0, cy - by1, cy - by0);
  return best >= thr - (1e-2f + 1e-3f * fabsf(thr));
}

// The staged entries that can reach this warp's block (reaches_block), in list order;
// returns their count.
template <int kBatch>
__device__ __forceinline__ int warp_list(const float4 (*s_q)[kBatch], const float4* s_box, int cnt, float bx0,
                                         float by0, float by1, const Camera& cam, uint16_t* list, int lane) {
  const uint32_t lt_mask = (1u << lane) - 1u;
  int m = 0;
  for (int j0 = 0; j0 < cnt; j0 += 32) {
    const int j = j0 + lane;
    const bool hit = j < cnt && reaches_block(s_box[j], s_q[0][j].x, s_q[0][j].z, s_q[1][j].x, s_q[1][j].z,
                                              s_q[2][j].x, s_q[3][j].z, bx0, by0, by1, cam);
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

// One list entry for a thread's pixel pairs: exponent, exp, opacity, transmittance and
// colour of both pixels of each pair with packed instructions, decisions per pixel.
template <int NP>
__device__ __forceinline__ void fwd_entry(const float4 q0, const float4 q1, const float4 q2, const float4 q3,
                                          uint32_t pos, float2 npx, const float2 (&npy)[NP], float2 (&T)[NP],
                                          float2 (&C)[NP], uint32_t (&nc)[NP][2], uint32_t (&lastp)[NP][2],
                                          bool (&done)[NP][2], uint32_t& nev) {
  const float2 dx = fadd2(make_float2(q0.x, q0.y), npx);
#pragma unroll
  for (int pr = 0; pr < NP; ++pr) {
    if (done[pr][0] && done[pr][1]) continue;
    // the exponent dx (na dx + nb dy) + (nc dy) dy of both pixels
    const float2 dy = fadd2(make_float2(q0.z, q0.w), npy[pr]);
    const float2 t = ffma2(make_float2(q1.x, q1.y), dx, fmul2(make_float2(q1.z, q1.w), dy));
    const float2 p = ffma2(dx, t, fmul2(fmul2(make_float2(q2.x, q2.y), dy), dy));
    nev += (uint32_t)!done[pr][0] + (uint32_t)!done[pr][1];
    const bool in0 = !done[pr][0] && !(p.x < q3.z), in1 = !done[pr][1] && !(p.y < q3.z);
    if (!(in0 || in1)) continue;  // opacity provably below 1/255 for both
    const float2 oe = fmul2(make_float2(q2.z, q2.w), xg_exp2v(p));
    const float2 al = make_float2(fminf(kAlphaMax, oe.x), fminf(kAlphaMax, oe.y));
    const float2 Tn = fmul2(T[pr], ffma2(al, f2(-1.0f), f2(1.0f)));
    const float2 Cn = ffma2(make_float2(q3.x, q3.y), fmul2(al, T[pr]), C[pr]);
    if (in0 && !(al.x < kAlphaMin)) {
      if (Tn.x < kTMin) {
        done[pr][0] = true;
      } else {
        C[pr].x = Cn.x;
        T[pr].x = Tn.x;
        ++nc[pr][0];
        lastp[pr][0] = pos;
      }
    }
    if (in1 && !(al.y < kAlphaMin)) {
      if (Tn.y < kTMin) {
        done[pr][1] = true;
      } else {
        C[pr].y = Cn.y;
        T[pr].y = Tn.y;
        ++nc[pr][1];
        lastp[pr][1] = pos;
      }
    }
  }
}

// Forward.  A thread's pixels are taken in pairs (4 rows apart; for one pixel per thread
// the second of the pair is idle), and the exponent, exp, opacity, transmittance and colour
// of both are computed with packed two-lane instructions; the decisions stay per pixel.
template <int kBatch, int PPT>
__global__ void __launch_bounds__(512) k_render_fwd(const uint2* __restrict__ range, const uint32_t* __restrict__ order,
                                                    int tiles_per_view, const uint32_t* __restrict__ value,
                                                    const float4* __restrict__ rec, int64_t n, int W, int H,
                                                    int tiles_x, int64_t range_stride, int tw, int th,
                                                    const Camera* __restrict__ cams, DevStatus* __restrict__ st,
                                                    float* __restrict__ image, uint32_t* __restrict__ ncontrib,
                                                    float* __restrict__ tfinal, uint32_t* __restrict__ last) {
  constexpr int NP = PPT > 1 ? PPT / 2 : 1;  // pixel pairs per thread
  const uint32_t work = order[blockIdx.x];  // (view, tile) items, longest tile lists first
  if (work >= gridDim.x) return;            // only an order that no xg_bin_sort wrote
  const int v = (int)(work / (uint32_t)tiles_per_view), tile = (int)(work % (uint32_t)tiles_per_view);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int lx, ly;
  pixel_in_tile<PPT>(threadIdx.x, tw, lx, ly);
  const int tx0 = (tile % tiles_x) * tw, ty0 = (tile / tiles_x) * th;
  const int x = tx0 + lx;
  const float bx0 = (float)(tx0 + (lx & ~7)), by0 = (float)(ty0 + (ly & ~3));  // this warp's block
  const float by1 = by0 + (float)(4 * PPT - 1);
  const Camera cam = cams[v];
  const float2 npx = f2(-fsub((float)x, cam.hw));
  const uint2 r = st->code == XG_OK ? range[(int64_t)v * range_stride + tile] : make_uint2(0u, 0u);
  const int nlist = (int)(r.y - r.x);
  const int64_t vn_base = (int64_t)v * n;

  float2 npy[NP], T[NP], C[NP];
  uint32_t nc[NP][2], lastp[NP][2];
  bool done[NP][2];
#pragma unroll
  for (int pr = 0; pr < NP; ++pr) {
    float ny[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int y = ty0 + ly + 4 * (2 * pr + h);
      ny[h] = -fsub((float)y, cam.hh);
      nc[pr][h] = lastp[pr][h] = 0;
      done[pr][h] = !((PPT > 1 || h == 0) && x < W && y < H);
    }
    npy[pr] = make_float2(ny[0], ny[1]);
    T[pr] = f2(1.0f);
    C[pr] = f2(0.0f);
  }
  uint32_t nev = 0;
  auto all_done = [&]() {
    bool d = true;
#pragma unroll
    for (int pr = 0; pr < NP; ++pr) d = d && done[pr][0] && done[pr][1];
    return d;
  };
  __shared__ float4 s_q[4][kBatch];
  __shared__ float4 s_box[kBatch];
  __shared__ uint16_t s_list[kMaxWarps][kBatch];
  uint16_t* my_list = s_list[warp];
  for (int base = 0; base < nlist; base += kBatch) {
    if (__syncthreads_count(all_done()) == (int)blockDim.x) break;
    const int cnt = min(kBatch, nlist - base);
    stage_batch_pairs<kBatch>(value, rec, vn_base, r.x + base, cnt, cam, s_q, s_box, nullptr);
    __syncthreads();
    if (__all_sync(0xffffffffu, all_done())) continue;
    const int m = warp_list<kBatch>(s_q, s_box, cnt, bx0, by0, by1, cam, my_list, lane);
#pragma unroll 2
    for (int k = 0; k < m; ++k) {
      if (all_done()) break;
      const int j = my_list[k];
      fwd_entry<NP>(s_q[0][j], s_q[1][j], s_q[2][j], s_q[3][j], (uint32_t)(base + j + 1), npx, npy, T, C, nc,
                    lastp, done, nev);
    }
  }
  uint32_t nct = 0;
#pragma unroll
  for (int pr = 0; pr < NP; ++pr) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (PPT == 1 && h == 1) continue;
      const int y = ty0 + ly + 4 * (2 * pr + h);
      nct += nc[pr][h];
      if (x < W && y < H) {
        const int64_t pix = ((int64_t)v * H + y) * W + x;
        image[pix] = h ? C[pr].y : C[pr].x;
        tfinal[pix] = h ? T[pr].y : T[pr].x;
        last[pix] = lastp[pr][h];
        if (ncontrib) ncontrib[pix] = nc[pr][h];
      }
    }
  }
  add_counts(nev, nct, &st->fwd_evaluated, &st->fwd_contrib);
}

cudaError_t launch_render_fwd(xg_frame* f, float* image, uint32_t* n_contrib, cudaStream_t st) {
  const FramePtrs& p = f->p;
  const dim3 grid((unsigned)(f->tiles_per_view * f->n_views));
  Timed t(f, kRenderFwd, st);
  const int ppt = f->cfg.pixels_per_thread;
  const int threads = f->cfg.tile_w * f->cfg.tile_h / ppt;
#define XG_FWD(B, P)                                                                                       \
  k_render_fwd<B, P><<<grid, threads, 0, st>>>(p.range, p.order, (int)f->tiles_per_view,                  \
                                               p.value, p.rec, f->n, f->width,            \
                                               f->height, f->tiles_x, (int64_t)1 << f->tile_bits, f->cfg.tile_w,   \
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
// Backward.  Pixels are taken in pairs as in the forward kernel.  A pixel of the pair that
// does not contribute to an entry takes alpha = 0 there, which leaves its transmittance,
// its blended-behind intensity and every gradient term unchanged, so the pair's update is
// one packed, branch-free sequence.
template <int kBatch, int PPT>
__global__ void __launch_bounds__(512) k_render_bwd(const uint2* __restrict__ range, const uint32_t* __restrict__ order,
                                                    int tiles_per_view, const uint32_t* __restrict__ value,
                                                    const float4* __restrict__ rec, int64_t n, int n_views, int W,
                                                    int H, int tiles_x, int64_t range_stride, int tw, int th,
                                                    const Camera* __restrict__ cams, DevStatus* __restrict__ st,
                                                    const float* __restrict__ grad_image,
                                                    const float* __restrict__ tfinal, const uint32_t* __restrict__ last,
                                                    float* __restrict__ g2d) {
  constexpr int NP = PPT > 1 ? PPT / 2 : 1;
  __shared__ float4 s_q[4][kBatch];
  __shared__ float4 s_box[kBatch];
  __shared__ uint32_t s_g[kBatch];
  __shared__ __align__(16) float s_acc[kBatch * 8];
  __shared__ uint16_t s_list[kMaxWarps][kBatch];
  __shared__ uint32_t s_maxlast;
  if (st->code != XG_OK) return;
  const uint32_t work = order[blockIdx.x];  // (view, tile) items, longest tile lists first
  if (work >= gridDim.x) return;            // only an order that no xg_bin_sort wrote
  const int v = (int)(work / (uint32_t)tiles_per_view), tile = (int)(work % (uint32_t)tiles_per_view);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int lx, ly;
  pixel_in_tile<PPT>(threadIdx.x, tw, lx, ly);
  const int tx0 = (tile % tiles_x) * tw, ty0 = (tile / tiles_x) * th;
  const int x = tx0 + lx;
  const float bx0 = (float)(tx0 + (lx & ~7)), by0 = (float)(ty0 + (ly & ~3));
  const float by1 = by0 + (float)(4 * PPT - 1);
  const Camera cam = cams[v];
  const float2 npx = f2(-fsub((float)x, cam.hw));
  const uint2 r = range[(int64_t)v * range_stride + tile];
  const int64_t vn_base = (int64_t)v * n;
  uint16_t* my_list = s_list[warp];

  float2 npy[NP], G[NP], Tc[NP], A[NP];
  uint32_t L[NP][2];
  uint32_t lmax = 0;
#pragma unroll
  for (int pr = 0; pr < NP; ++pr) {
    float ny[2], g[2], tc[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int y = ty0 + ly + 4 * (2 * pr + h);
      ny[h] = -fsub((float)y, cam.hh);
      g[h] = 0.f;
      tc[h] = 1.f;
      L[pr][h] = 0;
      if ((PPT > 1 || h == 0) && x < W && y < H) {
        const int64_t pix = ((int64_t)v * H + y) * W + x;
        g[h] = grad_image[pix];
        tc[h] = tfinal[pix];
        L[pr][h] = g[h] != 0.f ? last[pix] : 0u;
      }
      lmax = max(lmax, L[pr][h]);
    }
    npy[pr] = make_float2(ny[0], ny[1]);
    G[pr] = make_float2(g[0], g[1]);
    Tc[pr] = make_float2(tc[0], tc[1]);
    A[pr] = f2(0.f);  // intensity blended behind the current position, per unit transmittance
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
    stage_batch_pairs<kBatch>(value, rec, vn_base, r.x + base, cnt, cam, s_q, s_box, s_g);
    for (int i = threadIdx.x; i < cnt * 8; i += blockDim.x) s_acc[i] = 0.f;
    __syncthreads();
    if ((uint32_t)base < wl) {
      const int m = warp_list<kBatch>(s_q, s_box, min(cnt, (int)wl - base), bx0, by0, by1, cam, my_list, lane);
      for (int k = m - 1; k >= 0; --k) {
        const int j = my_list[k];
        const float4 q0 = s_q[0][j], q1 = s_q[1][j], q2 = s_q[2][j], q3 = s_q[3][j];
        const float2 dx = fadd2(make_float2(q0.x, q0.y), npx);
        const uint32_t pos = (uint32_t)(base + j);
        // packed sums over the thread's pixels: six moments of dp = dL/dpower (dp, dp d,
        // dp d d^T) and dL/dintensity
        float2 gm[7];  // set by the thread's first contributing pair, then accumulated
        bool contrib = false;
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
          const bool act0 = pos < L[pr][0], act1 = pos < L[pr][1];
          if (!(act0 || act1)) continue;
          nev += (uint32_t)act0 + (uint32_t)act1;
          const float2 dy = fadd2(make_float2(q0.z, q0.w), npy[pr]);
          const float2 t = ffma2(make_float2(q1.x, q1.y), dx, fmul2(make_float2(q1.z, q1.w), dy));
          const float2 p = ffma2(dx, t, fmul2(fmul2(make_float2(q2.x, q2.y), dy), dy));
          const bool in0 = act0 && !(p.x < q3.z), in1 = act1 && !(p.y < q3.z);
          if (!(in0 || in1)) continue;
          const float2 oe = fmul2(make_float2(q2.z, q2.w), xg_exp2v(p));
          const float2 al = make_float2(fminf(kAlphaMax, oe.x), fminf(kAlphaMax, oe.y));
          const bool ok0 = in0 && !(al.x < kAlphaMin), ok1 = in1 && !(al.y < kAlphaMin);
          if (!(ok0 || ok1)) continue;
          ncon += (uint32_t)ok0 + (uint32_t)ok1;
          // alpha of the pixels that contribute, 0 for the other one
          const float2 alm = make_float2(ok0 ? al.x : 0.f, ok1 ? al.y : 0.f);
          const float2 omal = ffma2(alm, f2(-1.0f), f2(1.0f));
          Tc[pr] = make_float2(__fdividef(Tc[pr].x, omal.x), __fdividef(Tc[pr].y, omal.y));
          const float2 gw = fmul2(G[pr], Tc[pr]);  // dL/dC T; gw alm is the dL/d intensity term
          const float2 dl_dal = fmul2(gw, ffma2(A[pr], f2(-1.0f), make_float2(q3.x, q3.y)));
          A[pr] = ffma2(alm, make_float2(q3.x, q3.y), fmul2(omal, A[pr]));
          // dp = dL/dalpha alpha where the opacity is not clamped (the clamp has zero slope)
          const float2 aln = make_float2(oe.x < kAlphaMax ? alm.x : 0.f, oe.y < kAlphaMax ? alm.y : 0.f);
          const float2 dp = fmul2(dl_dal, aln);
          const float2 sx = fmul2(dp, dx), sy = fmul2(dp, dy);
          if (!contrib) {
            gm[0] = sx;
            gm[1] = sy;
            gm[2] = fmul2(sx, dx);
            gm[3] = fmul2(sx, dy);
            gm[4] = fmul2(sy, dy);
            gm[5] = dp;
            gm[6] = fmul2(gw, alm);
            contrib = true;
          } else {
            gm[0] = fadd2(gm[0], sx);
            gm[1] = fadd2(gm[1], sy);
            gm[2] = ffma2(sx, dx, gm[2]);
            gm[3] = ffma2(sx, dy, gm[3]);
            gm[4] = ffma2(sy, dy, gm[4]);
            gm[5] = fadd2(gm[5], dp);
            gm[6] = ffma2(gw, alm, gm[6]);
          }
        }
        if (__any_sync(0xffffffffu, contrib)) {
          float gv[8];
#pragma unroll
          for (int t = 0; t < 7; ++t) gv[t] = contrib ? gm[t].x + gm[t].y : 0.f;
          gv[7] = 0.f;
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
        const float na = s_q[1][j].x, nb = s_q[1][j].z;  // -a/2, -b
        const float nc = s_q[2][j].x, o = s_q[2][j].z;   // -c/2, opacity
        const float4 q0 = make_float4(2.f * na * m0.x + nb * m0.y, nb * m0.x + 2.f * nc * m0.y, -0.5f * m0.z,
                                      -m0.w);
        const float4 q1 = make_float4(-0.5f * m1.x, __fdividef(m1.y, o), m1.z, 0.f);
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
  const dim3 grid((unsigned)(f->tiles_per_view * f->n_views));
  Timed t(f, kRenderBwd, st);
  const int ppt = f->cfg.pixels_per_thread;
  const int threads = f->cfg.tile_w * f->cfg.tile_h / ppt;
#define XG_BWD(B, P)                                                                                            \
  k_render_bwd<B, P><<<grid, threads, 0, st>>>(p.range, p.order, (int)f->tiles_per_view,                       \
                                               p.value, p.rec, f->n, f->n_views,               \
                                               f->width, f->height, f->tiles_x, (int64_t)1 << f->tile_bits,             \
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

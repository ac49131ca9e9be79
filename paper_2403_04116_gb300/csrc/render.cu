// Front-to-back alpha compositing of intensity per detector pixel (Eq. 10) and its
// backward pass.
//
// Work item: one warp's pixel block, 8 columns by 4*PPT rows of one (view, tile).  A thread
// owns PPT pixels (1, 2 or 4, four rows apart) and takes them in pairs with the packed
// two-lane FP32 instructions of sm_100 and later (f32x2 add / mul / fma): both pixels of a
// pair see the same list entry, and each lane is rounded as the scalar operation would be,
// so results are those of the documented scalar FP32 sequence.
//
// The warps of a tile never wait for one another: each walks the tile's depth-sorted list
// on its own, so no warp idles at a block-wide barrier while another finishes a longer
// walk.  A warp fetches the list 32 entries a round, one per lane: the Gaussian index, then
// its 32-byte record copied asynchronously (cp.async) into the warp's ring of RING
// shared-memory slots, RING - 1 rounds ahead of the round being processed (the frame's
// "batch" = 32 (RING - 1) records in flight per warp).  Each lane tests its own record --
// can the footprint reach the warp's block?  (the largest exponent of the footprint over
// the block's pixel centres, against the record's threshold) -- and the warp walks the
// entries that can, in list order.
//
// Most (pixel, entry) pairs of a walked entry still lie outside the footprint.  The record
// carries the exponent threshold ln(1/(255 o)) - 1e-4, below which the opacity provably
// stays under 1/255 (the FP32 exp used for the decision is accurate to 3e-7): such a pair
// skips exp.  Every other pair goes through the fixed FP32 decision sequence, so decisions
// are exactly those of the full test.
//
// The backward pass walks each pixel's list back to front from its last contributor and
// recovers the transmittance by division instead of storing it: T_j = T_{j+1} / (1 -
// alpha_j), with 1 - alpha_j in [0.01, 1], as a hardware reciprocal refined by one Newton
// step and one residual correction of the quotient (Markstein's scheme for correctly
// rounded division, here without the special cases that cannot occur).  The round's
// entries that reach the block are first written in a duplicated form (one broadcast load
// gives both lanes of a packed operand).  Per walked entry every lane runs the same
// branch-free sequence: a pixel that does not take the entry gets alpha = 0, which leaves
// its state and terms exactly unchanged.  A warp with contributing pixels then sums its 7
// per-pixel terms -- six moments of dL/dpower (S_1, S_x, S_y, S_xx, S_xy, S_yy
// over the pixel offsets d = u - p) and the intensity term -- by a transpose through the
// current ring slot (each lane writes its 7 values, four lanes per term add 8 each, two
// shuffles combine them; lane k ends with the sum of term k), and lanes 0-6
// add them to the (view, Gaussian)'s sums in global memory in one atomic instruction.  The
// projection's backward pass turns the sums into dL/du, dL/dconic and dL/dopacity.
//
// Launch forms: one block per (view, tile), its warps the tile's blocks; or persistent
// blocks (as many as fit on the device at once) whose warps take work items from a counter
// in the status word, in longest-tile-list-first order.
#include <algorithm>

#include "xg_internal.cuh"


namespace xg {

// Shared memory per warp: RING rounds of 32 records of 32 bytes, the rounds' Gaussian indices
// (32 words each), then the current round's entries in the duplicated form (32 x 64 bytes).
template <int RING>
__host__ __device__ constexpr int ring_bytes() { return RING * 32 * (32 + 4) + 32 * 64; }
// the same, for a ring depth known at run time (the launch's dynamic shared memory per warp);
// the forward kernel keeps only the record slots (no indices, no duplicated form)
inline int ring_bytes_rt(int ring, bool bwd) { return bwd ? ring * 32 * (32 + 4) + 32 * 64 : ring * 32 * 32; }
static_assert(ring_bytes<3>() == 3 * 32 * 36 + 2048, "ring layout");

struct RenderArgs {
  const uint2* range;
  const uint32_t* order;
  const uint32_t* value;
  const float4* rec;
  const Camera* cams;
  DevStatus* st;
  uint32_t* counter;  // persistent form: next work item
  int64_t n;
  int64_t range_stride;
  int tiles_per_view, tiles_x, W, H, tw, th;
  int wpt;            // warps (pixel blocks) per tile
  uint32_t items;     // work items: views * tiles * wpt
  // forward
  float* image;
  uint32_t* ncontrib;
  float* tfinal;
  uint32_t* last;
  // backward
  const float* grad_image;
  const float* tfinal_in;
  const uint32_t* last_in;
  float* g2d;
};

// The warp's ring of record slots: slot (round % RING), one 32-byte record per lane.
template <int RING>
__device__ __forceinline__ float4* warp_ring(int warp_in_cta) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  return reinterpret_cast<float4*>(s_dyn + (size_t)warp_in_cta * ring_bytes<RING>());
}
// the forward kernel's ring: RING slots of 32 records, nothing else
template <int RING>
__device__ __forceinline__ float4* warp_ring_fwd(int warp_in_cta) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  return reinterpret_cast<float4*>(s_dyn + (size_t)warp_in_cta * RING * 32 * 32);
}
// Per warp, after the ring: the round's entries in the duplicated form, one per lane:
// (u_x u_x u_y u_y), (na na nb nb), (nc nc o o), (i i thr thr) as [4][32] float4.
template <int RING>
__device__ __forceinline__ float4* warp_stage(int warp_in_cta) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  return reinterpret_cast<float4*>(s_dyn + (size_t)warp_in_cta * ring_bytes<RING>() + RING * 32 * 36);
}
template <int RING>
__device__ __forceinline__ uint32_t* ring_index(int warp_in_cta) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  return reinterpret_cast<uint32_t*>(s_dyn + (size_t)warp_in_cta * ring_bytes<RING>() + RING * 32 * 32);
}

// Asynchronous 16-byte global -> shared copies (cp.async, cached in L1: the warps of a tile
// read the same records), one commit group per round.
__device__ __forceinline__ void copy16(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
// waits until at most N of this thread's commit groups are still pending
template <int N>
__device__ __forceinline__ void copy_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Issues the copy of the record of Gaussian g into this lane's place of ring slot `slot`
// (nothing for a lane past the list), then commits the round's group.
template <int RING>
__device__ __forceinline__ void fetch_round(float4* ring, int slot, int lane, bool valid, const float4* rec,
                                            int64_t vn_base, uint32_t g) {
  if (valid) {
    float4* dst = ring + (slot * 32 + lane) * 2;
    const float4* src = rec + 2 * (vn_base + g);
    copy16(dst, src);
    copy16(dst + 1, src + 1);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
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

// Whether a record's footprint can reach the block [bx0, bx0 + 7] x [by0, by1] (pixel
// indices): the largest exponent over the block's pixel centres is within a margin
// (1e-2 + 1e-3 |thr|, far above FP32 rounding of these sums) of the threshold below which
// no pixel can reach opacity 1/255.  Only entries that no pixel of the block could take
// fail, so decisions are unchanged.  Records of culled Gaussians are all zero and fail.
__device__ __forceinline__ bool reaches_block(const float4 a, const float4 b, float bx0, float by0, float by1,
                                              const Camera& cam) {
  if (!(b.y > 0.f)) return false;
  const float na = a.z, nb = a.w, nc = b.x, thr = b.w;
  const float cx = a.x + cam.hw, cy = a.y + cam.hh;
  const float best = max_power_over_rect(na, nb, nc, cx - (bx0 + 7.f), cx - bx0, cy - by1, cy - by0);
  return best >= thr - (1e-2f + 1e-3f * fabsf(thr));
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

// Sums over the warp of the 7 per-lane values v[0..6] through shared memory, with no
// lane-dependent register selection: lane j writes v[t] to row t (a row of 36 words: 32 lanes
// and 4 of padding), then lane l adds the 8 values of row (l & 7) written by lanes
// 8 (l >> 3) .. 8 (l >> 3) + 7 (two 16-byte loads; rows 36 words apart put the 8 lanes of
// each quarter-warp load on distinct banks) and two shuffles combine the four lanes of the
// same row.  Lanes 0..6 return the sums of terms 0..6; lanes with (l & 7) == 7 re-read row 6
// and return a value that is not used.  `buf` holds 7 x 36 words; the warp must be
// converged.
__device__ __forceinline__ float warp_sum7_transposed(const float (&v)[7], float* buf, int lane) {
  __syncwarp();  // the previous call's loads are done before the rows are rewritten
#pragma unroll
  for (int t = 0; t < 7; ++t) buf[t * 36 + lane] = v[t];
  __syncwarp();
  const int row = min(lane & 7, 6);
  const float4* src = reinterpret_cast<const float4*>(buf + row * 36 + 8 * (lane >> 3));
  const float4 a = src[0], b = src[1];
  // the 8 values as four packed pairs: three packed adds and one scalar add
  const float2 h = fadd2(fadd2(make_float2(a.x, a.y), make_float2(a.z, a.w)),
                         fadd2(make_float2(b.x, b.y), make_float2(b.z, b.w)));
  float s = fadd(h.x, h.y);
  s = fadd(s, __shfl_xor_sync(0xffffffffu, s, 8));
  return fadd(s, __shfl_xor_sync(0xffffffffu, s, 16));
}

// T / om for om = 1 - alpha in [0.01, 1] and T in (0, 1], lane by lane, given nom = -om =
// alpha - 1 (exact, as is 1 - alpha): the hardware reciprocal r0 of om (relative error
// below 2^-22), one Newton step r = r0 + r0 (1 - om r0), the quotient q = T r and one
// residual correction q + r (T - q om) with the residual formed exactly by an FMA
// (Markstein).  Every product with om is written as one with nom, so no operand needs a
// negation.  No operand is zero, infinite, NaN or subnormal here, so none of the special
// cases of a general division arise.
__device__ __forceinline__ float2 div_recover(float2 T, float2 nom) {
  float rx, ry;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rx) : "f"(-nom.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ry) : "f"(-nom.y));
  float2 r = make_float2(rx, ry);
  const float2 e = ffma2(nom, r, f2(1.0f));  // 1 - om r
  r = ffma2(r, e, r);
  const float2 q = fmul2(T, r);
  const float2 res = ffma2(q, nom, T);  // T - q om
  return ffma2(res, r, q);
}

// The block of work item `item`: its (view, tile) and the warp's block inside the tile.
struct Item {
  int v, tile, tx0, ty0, bx, by;  // bx, by: the block's first pixel column and row
  bool ok;
};

template <int PPT>
__device__ __forceinline__ Item item_of(const RenderArgs& A, uint32_t item) {
  Item it;
  const uint32_t tile_item = item / (uint32_t)A.wpt, sub = item - tile_item * (uint32_t)A.wpt;
  const uint32_t work = A.order[tile_item];
  const uint32_t tiles = (uint32_t)A.tiles_per_view;
  it.ok = item < A.items && work < A.items / (uint32_t)A.wpt;  // an order that no xg_bin_sort wrote fails
  it.v = (int)(work / tiles);
  it.tile = (int)(work - (uint32_t)it.v * tiles);
  it.tx0 = (it.tile % A.tiles_x) * A.tw;
  it.ty0 = (it.tile / A.tiles_x) * A.th;
  const int wx = A.tw >> 3;
  it.bx = it.tx0 + (int)(sub % (uint32_t)wx) * 8;
  it.by = it.ty0 + (int)(sub / (uint32_t)wx) * (4 * PPT);
  return it;
}

// Next work item of this warp: the persistent form takes one from the counter, the other
// form has exactly one, blockIdx.x * wpt + warp.
template <bool PERSIST>
__device__ __forceinline__ uint32_t next_item(const RenderArgs& A, int lane, int warp, bool first) {
  if (!PERSIST) return first ? blockIdx.x * (uint32_t)A.wpt + (uint32_t)warp : 0xffffffffu;
  uint32_t it = 0;
  if (lane == 0) it = atomicAdd(A.counter, 1u);
  return __shfl_sync(0xffffffffu, it, 0);
}

// ------------------------------------------------------------------------------------------
// forward
// ------------------------------------------------------------------------------------------

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
    const float2 dy = fadd2(make_float2(q0.z, q0.w), npy[pr]);
    const float2 t = ffma2(make_float2(q1.x, q1.y), dx, fmul2(make_float2(q1.z, q1.w), dy));
    const float2 p = ffma2(dx, t, fmul2(fmul2(make_float2(q2.x, q2.y), dy), dy));
    nev += (uint32_t)!done[pr][0] + (uint32_t)!done[pr][1];
    const bool in0 = !done[pr][0] && !(p.x < q3.z), in1 = !done[pr][1] && !(p.y < q3.z);
    if (!(in0 || in1)) continue;  // opacity provably below 1/255 for both
    const float2 oe = fmul2(make_float2(q2.z, q2.w), xg_exp2v_core(p));
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

template <int PPT, int RING, bool PERSIST>
__global__ void __launch_bounds__(512) k_render_fwd(const RenderArgs A) {
  constexpr int NP = PPT > 1 ? PPT / 2 : 1;  // pixel pairs per thread
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4* const ring = warp_ring_fwd<RING>(warp);
  const bool status_ok = A.st->code == XG_OK;
  uint32_t nev = 0, nct = 0;
  for (uint32_t item = next_item<PERSIST>(A, lane, warp, true);; item = next_item<PERSIST>(A, lane, warp, false)) {
    if (item >= A.items) break;
    const Item it = item_of<PPT>(A, item);
    if (!it.ok) break;
    const Camera cam = A.cams[it.v];
    const int x = it.bx + (lane & 7);
    const float bx0 = (float)it.bx, by0 = (float)it.by, by1 = by0 + (float)(4 * PPT - 1);
    const float2 npx = f2(-fsub((float)x, cam.hw));
    const uint2 r = status_ok ? A.range[(int64_t)it.v * A.range_stride + it.tile] : make_uint2(0u, 0u);
    const int nlist = (int)(r.y - r.x);
    const int64_t vn_base = (int64_t)it.v * A.n;

    float2 npy[NP], T[NP], C[NP];
    uint32_t nc[NP][2], lastp[NP][2];
    bool done[NP][2];
#pragma unroll
    for (int pr = 0; pr < NP; ++pr) {
      float ny[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int y = it.by + (lane >> 3) + 4 * (2 * pr + h);
        ny[h] = -fsub((float)y, cam.hh);
        nc[pr][h] = lastp[pr][h] = 0;
        done[pr][h] = !((PPT > 1 || h == 0) && x < A.W && y < A.H);
      }
      npy[pr] = make_float2(ny[0], ny[1]);
      T[pr] = f2(1.0f);
      C[pr] = f2(0.0f);
    }
    auto all_done = [&]() {
      bool d = true;
#pragma unroll
      for (int pr = 0; pr < NP; ++pr) d = d && done[pr][0] && done[pr][1];
      return d;
    };
    // round q: list positions [32 q, 32 q + 32), lane l at 32 q + l; the records of the next
    // RING - 1 rounds are in flight while round q is walked
    const int rounds = (nlist + 31) / 32;
#pragma unroll
    for (int q = 0; q < RING - 1; ++q) {
      const int e = 32 * q + lane;
      const uint32_t g = e < nlist ? A.value[r.x + e] : 0u;
      fetch_round<RING>(ring, q, lane, e < nlist, A.rec, vn_base, g);
    }
    uint32_t g_next = 32 * (RING - 1) + lane < nlist ? A.value[r.x + 32 * (RING - 1) + lane] : 0u;
    for (int q = 0; q < rounds; ++q) {
      if (__all_sync(0xffffffffu, all_done())) break;
      {
        const int e = 32 * (q + RING - 1) + lane;
        fetch_round<RING>(ring, (q + RING - 1) % RING, lane, e < nlist, A.rec, vn_base, g_next);
        g_next = e + 32 < nlist ? A.value[r.x + e + 32] : 0u;
      }
      copy_wait<RING - 1>();  // round q's records have landed
      __syncwarp();
      const float4* slot = ring + (q % RING) * 64;
      const bool hit = 32 * q + lane < nlist && reaches_block(slot[2 * lane], slot[2 * lane + 1], bx0, by0, by1, cam);
      uint32_t mask = __ballot_sync(0xffffffffu, hit);
      // (a thread whose pixels have stopped skips the remaining entries inside fwd_entry; the
      // round-level vote above ends the walk once every pixel of the warp has stopped)
      while (mask) {
        const int k = __ffs(mask) - 1;
        mask &= mask - 1;
        const float4 a = slot[2 * k], b = slot[2 * k + 1];
        const float na = a.z, nb = a.w, nc2 = b.x;
        fwd_entry<NP>(make_float4(a.x, a.x, a.y, a.y), make_float4(na, na, nb, nb), make_float4(nc2, nc2, b.y, b.y),
                      make_float4(b.z, b.z, b.w, b.w), (uint32_t)(32 * q + k + 1), npx, npy, T, C, nc, lastp, done,
                      nev);
      }
      __syncwarp();  // the slot is refilled next round
    }
    copy_wait<0>();  // no copy may land after the ring is reused or the block exits
    __syncwarp();
#pragma unroll
    for (int pr = 0; pr < NP; ++pr) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (PPT == 1 && h == 1) continue;
        const int y = it.by + (lane >> 3) + 4 * (2 * pr + h);
        nct += nc[pr][h];
        if (x < A.W && y < A.H) {
          const int64_t pix = ((int64_t)it.v * A.H + y) * A.W + x;
          A.image[pix] = h ? C[pr].y : C[pr].x;
          A.tfinal[pix] = h ? T[pr].y : T[pr].x;
          A.last[pix] = lastp[pr][h];
          if (A.ncontrib) A.ncontrib[pix] = nc[pr][h];
        }
      }
    }
  }
  add_counts(nev, nct, &A.st->fwd_evaluated, &A.st->fwd_contrib);
}

// ------------------------------------------------------------------------------------------
// backward
// ------------------------------------------------------------------------------------------
// Pixels are taken in pairs as in the forward kernel.  A pixel of a pair that does not
// contribute to an entry takes alpha = 0 there, which leaves its transmittance, its
// blended-behind intensity and every gradient term unchanged, so the pair's update is one
// packed, branch-free sequence.
template <int PPT, int RING, bool PERSIST>
__global__ void __launch_bounds__(512) k_render_bwd(const RenderArgs A) {
  constexpr int NP = PPT > 1 ? PPT / 2 : 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4* const ring = warp_ring<RING>(warp);
  uint32_t* const ring_g = ring_index<RING>(warp);
  float4* const stage = warp_stage<RING>(warp);
  if (A.st->code != XG_OK) return;
  uint32_t nev = 0, ncon = 0;
  for (uint32_t item = next_item<PERSIST>(A, lane, warp, true);; item = next_item<PERSIST>(A, lane, warp, false)) {
    if (item >= A.items) break;
    const Item it = item_of<PPT>(A, item);
    if (!it.ok) break;
    const Camera cam = A.cams[it.v];
    const int x = it.bx + (lane & 7);
    const float bx0 = (float)it.bx, by0 = (float)it.by, by1 = by0 + (float)(4 * PPT - 1);
    const float2 npx = f2(-fsub((float)x, cam.hw));
    const uint2 r = A.range[(int64_t)it.v * A.range_stride + it.tile];
    const int64_t vn_base = (int64_t)it.v * A.n;

    float2 npy[NP], G[NP], Tc[NP], Ab[NP];
    uint32_t Lp[NP][2];
    uint32_t lmax = 0;
#pragma unroll
    for (int pr = 0; pr < NP; ++pr) {
      float ny[2], g[2], tc[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int y = it.by + (lane >> 3) + 4 * (2 * pr + h);
        ny[h] = -fsub((float)y, cam.hh);
        g[h] = 0.f;
        tc[h] = 1.f;
        Lp[pr][h] = 0;
        if ((PPT > 1 || h == 0) && x < A.W && y < A.H) {
          const int64_t pix = ((int64_t)it.v * A.H + y) * A.W + x;
          g[h] = A.grad_image[pix];
          tc[h] = A.tfinal_in[pix];
          Lp[pr][h] = g[h] != 0.f ? A.last_in[pix] : 0u;
        }
        lmax = max(lmax, Lp[pr][h]);
      }
      npy[pr] = make_float2(ny[0], ny[1]);
      G[pr] = make_float2(g[0], g[1]);
      Tc[pr] = make_float2(tc[0], tc[1]);
      Ab[pr] = f2(0.f);  // intensity blended behind the current position, per unit transmittance
    }
    // the longest prefix any pixel of this warp walks: positions [0, wl), walked downwards;
    // round q holds positions wl - 1 - 32 q - l for lanes l (lane 0 the highest)
    int wl = (int)lmax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
    const int rounds = (wl + 31) / 32;
#pragma unroll
    for (int q = 0; q < RING - 1; ++q) {
      const int e = wl - 1 - 32 * q - lane;
      const uint32_t g = e >= 0 ? A.value[r.x + e] : 0u;
      ring_g[q * 32 + lane] = g;
      fetch_round<RING>(ring, q, lane, e >= 0, A.rec, vn_base, g);
    }
    int e_next = wl - 1 - 32 * (RING - 1) - lane;
    uint32_t g_next = e_next >= 0 ? A.value[r.x + e_next] : 0u;
    for (int q = 0; q < rounds; ++q) {
      {
        const int slot = (q + RING - 1) % RING;
        ring_g[slot * 32 + lane] = g_next;
        fetch_round<RING>(ring, slot, lane, e_next >= 0, A.rec, vn_base, g_next);
        e_next -= 32;
        g_next = e_next >= 0 ? A.value[r.x + e_next] : 0u;
      }
      copy_wait<RING - 1>();  // round q's records have landed
      __syncwarp();
      const int sq = q % RING;
      const float4* slot = ring + sq * 64;
      const int top = wl - 1 - 32 * q;  // position of lane 0's entry
      bool hit = false;
      if (top - lane >= 0) {
        const float4 a = slot[2 * lane], b = slot[2 * lane + 1];
        hit = reaches_block(a, b, bx0, by0, by1, cam);
        if (hit) {
          const float na = a.z, nb = a.w, nc = b.x;
          stage[lane] = make_float4(a.x, a.x, a.y, a.y);
          stage[32 + lane] = make_float4(na, na, nb, nb);
          stage[64 + lane] = make_float4(nc, nc, b.y, b.y);
          stage[96 + lane] = make_float4(b.z, b.z, b.w, b.w);
        }
      }
      uint32_t mask = __ballot_sync(0xffffffffu, hit);
      // the round's evaluated pairs, counted once per round: a pixel re-evaluates walked entry
      // k (position top - k) when its last contributor lies beyond it, k >= top - L + 1
#pragma unroll
      for (int pr = 0; pr < NP; ++pr)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int sh = top - (int)Lp[pr][h] + 1;
          const uint32_t ge = sh <= 0 ? 0xffffffffu : (sh >= 32 ? 0u : 0xffffffffu << sh);
          nev += (uint32_t)__popc(mask & ge);
        }
      __syncwarp();
      while (mask) {
        const int k = __ffs(mask) - 1;
        mask &= mask - 1;
        const float4 q0 = stage[k], q1 = stage[32 + k], q2 = stage[64 + k], q3 = stage[96 + k];
        const uint32_t gk = ring_g[sq * 32 + k];
        const uint32_t pos = (uint32_t)(top - k);
        const float2 dx = fadd2(make_float2(q0.x, q0.y), npx);
        // the exponent of every pixel pair; a pixel that is not walking this entry, whose
        // exponent is below the threshold, or whose opacity stays under 1/255 takes
        // alpha = 0 below, which leaves its transmittance, blended-behind intensity and
        // every term unchanged (exactly: division by 1, products with 0)
        float2 p[NP], dyv[NP];
        bool in[NP][2];
        bool any_in = false;
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
          const bool act0 = pos < Lp[pr][0], act1 = pos < Lp[pr][1];
          dyv[pr] = fadd2(make_float2(q0.z, q0.w), npy[pr]);
          const float2 t = ffma2(make_float2(q1.x, q1.y), dx, fmul2(make_float2(q1.z, q1.w), dyv[pr]));
          p[pr] = ffma2(dx, t, fmul2(fmul2(make_float2(q2.x, q2.y), dyv[pr]), dyv[pr]));
          in[pr][0] = act0 && !(p[pr].x < q3.z);
          in[pr][1] = act1 && !(p[pr].y < q3.z);
          any_in |= in[pr][0] || in[pr][1];
        }
        if (!__any_sync(0xffffffffu, any_in)) continue;  // no pixel of the warp can reach 1/255
        // sums over the thread's pixels of the six moments of dp = dL/dpower (dp, dp d,
        // dp d d^T) and of dL/dintensity.  The pixels of a pair share their column, so
        // dx is the same for both: S_x = S_1 dx, S_xx = S_x dx and S_xy = S_y dx.
        float gv[7];  // S_x, S_y, S_xx, S_xy, S_yy, S_1, dL/di
        bool any_ok = false;
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
          const float2 oe = fmul2(make_float2(q2.z, q2.w), xg_exp2v_core(p[pr]));
          const float2 al = make_float2(fminf(kAlphaMax, oe.x), fminf(kAlphaMax, oe.y));
          const bool ok0 = in[pr][0] && !(al.x < kAlphaMin), ok1 = in[pr][1] && !(al.y < kAlphaMin);
          any_ok |= ok0 || ok1;
          ncon += (uint32_t)ok0 + (uint32_t)ok1;
          const float2 alm = make_float2(ok0 ? al.x : 0.f, ok1 ? al.y : 0.f);
          Tc[pr] = div_recover(Tc[pr], fadd2(alm, f2(-1.0f)));  // T / (1 - alpha)
          const float2 gw = fmul2(G[pr], Tc[pr]);  // dL/dC T; gw alm is the dL/d intensity term
          const float2 ib = ffma2(Ab[pr], f2(-1.0f), make_float2(q3.x, q3.y));  // i - Ab
          const float2 dl_dal = fmul2(gw, ib);
          Ab[pr] = ffma2(alm, ib, Ab[pr]);  // Ab + alpha (i - Ab): the blend behind the previous entry
          // dp = dL/dalpha alpha where the opacity is not clamped (the clamp has zero slope)
          const float2 aln = make_float2(oe.x < kAlphaMax ? alm.x : 0.f, oe.y < kAlphaMax ? alm.y : 0.f);
          const float2 dp = fmul2(dl_dal, aln);
          const float2 sy = fmul2(dp, dyv[pr]);
          const float2 di = fmul2(gw, alm);
          const float s1 = fadd(dp.x, dp.y), sy1 = fadd(sy.x, sy.y), si = fadd(di.x, di.y);
          const float syy = ffma(sy.x, dyv[pr].x, fmul(sy.y, dyv[pr].y));
          if (pr == 0) {
            gv[5] = s1, gv[1] = sy1, gv[4] = syy, gv[6] = si;
          } else {
            gv[5] = fadd(gv[5], s1), gv[1] = fadd(gv[1], sy1), gv[4] = fadd(gv[4], syy), gv[6] = fadd(gv[6], si);
          }
        }
        if (__any_sync(0xffffffffu, any_ok)) {
          gv[0] = fmul(gv[5], dx.x);
          gv[2] = fmul(gv[0], dx.x);
          gv[3] = fmul(gv[1], dx.x);
          // sums over the block's pixels: S_x, S_y, S_xx, S_xy, S_yy, S_1 of dp = dL/dpower
          // times (d, d d^T, 1), and dL/dintensity; lane k (k < 7) ends with the sum of term
          // k, added to the Gaussian's sums.  The rows are the current ring slot's record
          // area: its records were staged above and the slot is refilled only next round.
          const float sum = warp_sum7_transposed(gv, reinterpret_cast<float*>(ring + sq * 64), lane);
          if (lane < 7) atomicAdd(A.g2d + 8 * (vn_base + gk) + lane, sum);
        }
      }
      __syncwarp();  // the slot is refilled next round
    }
    copy_wait<0>();
    __syncwarp();
  }
  add_counts(nev, ncon, &A.st->bwd_evaluated, &A.st->bwd_contrib);
}

// ------------------------------------------------------------------------------------------
// launches
// ------------------------------------------------------------------------------------------
namespace {

template <int PPT, int RING, bool PERSIST>
void* fn_of(bool bwd) { return bwd ? (void*)k_render_bwd<PPT, RING, PERSIST> : (void*)k_render_fwd<PPT, RING, PERSIST>; }

template <int RING>
void* kernel_ring(bool bwd, int ppt, bool persist) {
#define XG_PICK(P) \
  if (ppt == P) return persist ? fn_of<P, RING, true>(bwd) : fn_of<P, RING, false>(bwd);
  XG_PICK(1) XG_PICK(2) XG_PICK(4)
#undef XG_PICK
  return nullptr;
}

// batch = records in flight per warp = 32 (RING - 1)
void* kernel_of(bool bwd, int ppt, bool persist, int batch, int* ring) {
  switch (batch) {
    case 64: *ring = 3; return kernel_ring<3>(bwd, ppt, persist);
    case 128: *ring = 5; return kernel_ring<5>(bwd, ppt, persist);
    case 256: *ring = 9; return kernel_ring<9>(bwd, ppt, persist);
    default: *ring = 17; return kernel_ring<17>(bwd, ppt, persist);
  }
}

constexpr int kPersistWarps = 4;

RenderArgs args_of(const xg_frame* f) {
  const FramePtrs& p = f->p;
  RenderArgs A{};
  A.range = p.range;
  A.order = p.order;
  A.value = p.value;
  A.rec = p.rec;
  A.cams = p.cam;
  A.st = p.status;
  A.counter = &p.status->next_item;
  A.n = f->n;
  A.range_stride = (int64_t)1 << f->tile_bits;
  A.tiles_per_view = (int)f->tiles_per_view;
  A.tiles_x = f->tiles_x;
  A.W = f->width;
  A.H = f->height;
  A.tw = f->cfg.tile_w;
  A.th = f->cfg.tile_h;
  const int ppt = f->cfg.pixels_per_thread;
  A.wpt = (A.tw / 8) * (A.th / (4 * ppt));
  A.items = (uint32_t)(f->tiles_per_view * f->n_views * A.wpt);
  return A;
}

int ring_of(int batch) { return batch / 32 + 1; }

// Dynamic shared memory of a compositing block of this configuration.
size_t block_smem(const xg_config* cfg, bool bwd = true) {
  const int ppt = cfg->pixels_per_thread == 0 ? 2 : cfg->pixels_per_thread;
  const int batch = cfg->batch == 0 ? 64 : cfg->batch;
  const int warps = cfg->persistent ? kPersistWarps : (cfg->tile_w / 8) * (cfg->tile_h / (4 * ppt));
  return (size_t)warps * (size_t)ring_bytes_rt(ring_of(batch), bwd);
}

cudaError_t launch(xg_frame* f, bool bwd, const RenderArgs& A, cudaStream_t st) {
  const bool persist = f->cfg.persistent != 0;
  int ring = 0;
  void* fn = kernel_of(bwd, f->cfg.pixels_per_thread, persist, f->cfg.batch, &ring);
  const int warps = persist ? kPersistWarps : A.wpt;
  unsigned grid = (unsigned)(f->tiles_per_view * f->n_views);
  if (persist) {
    const unsigned need = (A.items + kPersistWarps - 1) / kPersistWarps;
    grid = std::min(need, (unsigned)f->render_blocks[bwd ? 1 : 0]);
    const cudaError_t e = cudaMemsetAsync(A.counter, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
  }
  void* params[] = {(void*)&A};
  return cudaLaunchKernel(fn, dim3(grid), dim3(warps * 32), params, block_smem(&f->cfg, bwd), st);
}

}  // namespace

size_t render_smem_bytes(const xg_config* cfg) { return block_smem(cfg); }

// The compositing kernels' shared-memory limit and, for the persistent form, the blocks
// that fit on the device at once.  Called at frame creation (outside any stream capture).
cudaError_t render_prepare(xg_frame* f) {
  const bool persist = f->cfg.persistent != 0;
  const int warps = persist ? kPersistWarps : (f->cfg.tile_w / 8) * (f->cfg.tile_h / (4 * f->cfg.pixels_per_thread));
  for (int bwd = 0; bwd < 2; ++bwd) {
    int ring = 0;
    void* fn = kernel_of(bwd != 0, f->cfg.pixels_per_thread, persist, f->cfg.batch, &ring);
    const size_t smem = block_smem(&f->cfg, bwd != 0);
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, fn);
    if (e != cudaSuccess) return e;
    if ((size_t)attr.maxDynamicSharedSizeBytes < smem) {
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    f->render_blocks[bwd] = 0;
    if (persist) {
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem);
      if (e != cudaSuccess) return e;
      f->render_blocks[bwd] = std::max(1, per_sm) * device_sms();
    }
  }
  return cudaSuccess;
}

cudaError_t launch_render_fwd(xg_frame* f, float* image, uint32_t* n_contrib, cudaStream_t st) {
  RenderArgs A = args_of(f);
  A.image = image;
  A.ncontrib = n_contrib;
  A.tfinal = f->p.tfinal;
  A.last = f->p.last;
  Timed t(f, kRenderFwd, st);
  return launch(f, false, A, st);
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
  RenderArgs A = args_of(f);
  A.grad_image = grad_image;
  A.tfinal_in = p.tfinal;
  A.last_in = p.last;
  A.g2d = p.grad2d;
  Timed t(f, kRenderBwd, st);
  return launch(f, true, A, st);
}

}  // namespace xg

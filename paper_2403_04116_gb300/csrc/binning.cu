// Tile binning and the depth-keyed radix sort (Sec. 3.2: Gaussians are assigned to the
// tiles their projection touches and sorted by depth).
//
// The (view, tile, depth) order of the pairs is built in two stable LSD radix sorts, so
// that the many pairs (one per touched tile) are moved only by their tile index:
//
//   1. the V*n (view, Gaussian) entries, keyed (view, bits of t_z) -- 4 depth passes and
//      ceil(log2(V)/8) view passes over V*n entries (k_project writes the keys);
//   2. the tile counts, gathered in that order, are prefix-summed and every entry emits one
//      (view << B | tile, Gaussian) pair per touched tile at its offset (B = ceil(log2 T)),
//      so the emitted list is ordered by (view, depth, index);
//   3. the pairs are sorted stably by the B tile bits alone (ceil(B/8) passes): the list
//      ends up ordered by (tile, view, depth, index), every (view, tile) list contiguous and
//      in (depth, index) order;
//   4. ranges: [start, end) per (view, tile), indexed by the pair key view << B | tile.
//
// Each (view, tile) list equals a stable sort of that tile's pairs by the bits of t_z, at
// well under half of the memory traffic of sorting all pairs by a 64-bit key.
//
// Every kernel here runs on a fixed grid of kSortBlocks CTAs that split the work into
// contiguous chunks computed on the device from the item count, so the host never needs to
// know the pair count and the whole sequence can be captured in a CUDA graph.  There is no
// inter-CTA waiting: every scan is reduce / scan-of-partials / down-sweep in three launches.
#include <stdlib.h>

#include "xg_internal.cuh"

namespace xg {

constexpr int kWarps = kSortThreads / 32;

__device__ __forceinline__ int64_t chunk_of(int64_t total) {
  // per-CTA chunk: ceil(total / kSortBlocks) rounded up to whole radix tiles
  const int64_t c = (total + kSortBlocks - 1) / kSortBlocks;
  return (c + kSortTile - 1) / kSortTile * kSortTile;
}

// Item count of a sort: `fixed` if it is >= 0, else the pairs recorded in the status word.
__device__ __forceinline__ int64_t items_of(const DevStatus* st, int64_t fixed) {
  if (fixed >= 0) return fixed;
  return st->code == XG_OK ? st->pairs : 0;
}

// exclusive scan of one value per thread across a block of NT threads; returns the total
template <int NT, typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* s_warp, T& total) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < NW ? s_warp[lane] : T(0);
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NW) s_warp[lane] = w;
  }
  __syncthreads();
  const T before = warp > 0 ? s_warp[warp - 1] : T(0);
  total = s_warp[NW - 1];
  __syncthreads();
  return before + x - v;
}

// ------------------------------------------------------------------------------------------
// scan of the tile counts, read in the (view, depth) order of stage 1
// ------------------------------------------------------------------------------------------
// Tile count of sorted entry i; an entry outside [0, V) x [0, n) (which a correct stage 1
// never produces) counts 0 and records XG_ERR_CHECK.
__device__ __forceinline__ uint32_t count_at(const uint32_t* __restrict__ count, const uint32_t* __restrict__ view,
                                             const uint32_t* __restrict__ gid, int64_t n, int64_t total, int64_t i,
                                             DevStatus* __restrict__ st) {
  const int64_t e = (int64_t)view[i] * n + gid[i];
  if (gid[i] >= n || e >= total) {
    st->code = XG_ERR_CHECK;
    return 0u;
  }
  return count[e];
}

__global__ void __launch_bounds__(kSortThreads) k_scan_reduce(const uint32_t* __restrict__ count,
                                                              const uint32_t* __restrict__ view,
                                                              const uint32_t* __restrict__ gid, int64_t n,
                                                              int64_t total, DevStatus* __restrict__ st,
                                                              unsigned long long* __restrict__ part) {
  __shared__ unsigned long long s_warp[kWarps];
  if (st->code != XG_OK) {  // stage 1 failed a check: its entries are not to be read
    if (threadIdx.x == 0) part[blockIdx.x] = 0ull;
    return;
  }
  const int64_t chunk = chunk_of(total);
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(total, beg + chunk);
  unsigned long long acc = 0;
  for (int64_t i = beg + threadIdx.x; i < end; i += kSortThreads) acc += count_at(count, view, gid, n, total, i, st);
  unsigned long long tot;
  block_exclusive_scan<kSortThreads>(acc, s_warp, tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(unsigned long long* __restrict__ part, int64_t capacity,
                                                  DevStatus* __restrict__ st) {
  static_assert(kSortBlocks <= 1024, "one partial per thread");
  __shared__ unsigned long long s_warp[32];
  const int b = threadIdx.x;
  const unsigned long long c = b < kSortBlocks ? part[b] : 0ull;
  unsigned long long run;
  const unsigned long long ex = block_exclusive_scan<1024>(c, s_warp, run);
  if (b < kSortBlocks) part[b] = ex;
  if (b == 0) {
    const bool failed = st->code != XG_OK;  // a check failed in stage 1: keep its code
    st->scan_total = failed ? 0ull : run;
    st->pairs = failed ? 0ll : (long long)run;
    st->fwd_evaluated = st->fwd_contrib = st->bwd_evaluated = st->bwd_contrib = 0ull;
    if (!failed) st->code = run > (unsigned long long)capacity ? XG_ERR_CAPACITY : XG_OK;
  }
}

__global__ void __launch_bounds__(kSortThreads) k_scan_down(const uint32_t* __restrict__ count,
                                                            const uint32_t* __restrict__ view,
                                                            const uint32_t* __restrict__ gid, int64_t n,
                                                            int64_t total, DevStatus* __restrict__ st,
                                                            const unsigned long long* __restrict__ part,
                                                            uint32_t* __restrict__ offset) {
  __shared__ unsigned long long s_warp[kWarps];
  if (st->code == XG_ERR_CHECK) return;
  const int64_t chunk = chunk_of(total);
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(total, beg + chunk);
  unsigned long long run = part[blockIdx.x];
  for (int64_t base = beg; base < end; base += kSortThreads) {
    const int64_t i = base + threadIdx.x;
    const unsigned long long c = i < end ? count_at(count, view, gid, n, total, i, st) : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_scan<kSortThreads>(c, s_warp, tot);
    if (i < end) offset[i] = (uint32_t)(run + ex);
    run += tot;
  }
}

// ------------------------------------------------------------------------------------------
// emit one (tile key, Gaussian) pair per touched tile, in (view, depth) order
// ------------------------------------------------------------------------------------------
// A warp takes 32 consecutive entries, whose pairs are contiguous in the output; lane l
// writes pairs l, l+32, ... of the warp, finding its entry by a binary search over the
// warp's prefix of counts, so every store instruction writes consecutive addresses.
__global__ void __launch_bounds__(256) k_emit(const uint32_t* __restrict__ count, const uint32_t* __restrict__ offset,
                                              const ushort4* __restrict__ rect, const uint32_t* __restrict__ view,
                                              const uint32_t* __restrict__ gid, int64_t n, int64_t total,
                                              int tiles_x, int tile_bits, int64_t capacity,
                                              DevStatus* __restrict__ st, uint32_t* __restrict__ key_tile,
                                              uint32_t* __restrict__ value) {
  if (st->code != XG_OK) return;
  const int64_t warp_first = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~(int64_t)31;
  if (warp_first >= total) return;
  const int lane = threadIdx.x & 31;
  const int64_t i = warp_first + lane;
  uint32_t v = 0, g = 0, cnt = 0, o = 0, xy0 = 0, xy1 = 0;
  if (i < total) {
    v = view[i];
    g = gid[i];
    const int64_t vg = (int64_t)v * n + g;
    cnt = count[vg];
    o = offset[i];
    if (cnt) {
      const ushort4 r = rect[vg];
      xy0 = (uint32_t)r.x | ((uint32_t)r.y << 16);
      xy1 = (uint32_t)r.z | ((uint32_t)r.w << 16);
    }
  }
  // exclusive prefix of the counts over the warp
  uint32_t incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  const uint32_t pre = incl - cnt;
  const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
  const uint32_t base = __shfl_sync(0xffffffffu, o, 0);
  if ((int64_t)base + tot > capacity) {  // cannot happen when the scan is right
    if (lane == 0) st->code = XG_ERR_CHECK;
    return;
  }
  for (uint32_t p0 = 0; p0 < tot; p0 += 32) {
    const uint32_t p = p0 + lane;
    // the last entry whose prefix is <= p (entries without pairs share the next prefix)
    int e = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int cand = min(e + step, 31);
      const uint32_t pc = __shfl_sync(0xffffffffu, pre, cand);
      if (e + step <= 31 && pc <= p) e = cand;
    }
    const uint32_t e_pre = __shfl_sync(0xffffffffu, pre, e);
    const uint32_t e_xy0 = __shfl_sync(0xffffffffu, xy0, e);
    const uint32_t e_xy1 = __shfl_sync(0xffffffffu, xy1, e);
    const uint32_t e_v = __shfl_sync(0xffffffffu, v, e);
    const uint32_t e_g = __shfl_sync(0xffffffffu, g, e);
    if (p < tot) {
      const uint32_t k = p - e_pre;
      const uint32_t x0 = e_xy0 & 0xffffu, y0 = e_xy0 >> 16, x1 = e_xy1 & 0xffffu;
      const uint32_t wdt = x1 - x0 + 1u;
      const uint32_t ty = y0 + k / wdt, tx = x0 + k % wdt;
      key_tile[base + p] = (e_v << tile_bits) | (ty * (uint32_t)tiles_x + tx);
      value[base + p] = e_g;
    }
  }
}

// ------------------------------------------------------------------------------------------
// LSD radix sort, one 8-bit digit per pass, of WORDS parallel u32 arrays; the digit comes
// from array `digit_word`.  Histograms are block-major: hist[block][256], then the 256
// digit totals.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ word, int shift, uint32_t mask,
                                                             const DevStatus* __restrict__ st, int64_t fixed_count,
                                                             uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_h[kWarps][256];
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&s_h[0][0])[i] = 0;
  __syncthreads();
  const int64_t total = items_of(st, fixed_count);
  const int64_t chunk = chunk_of(total);
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(total, beg + chunk);
  for (int64_t i = beg + threadIdx.x; i < end; i += kSortThreads) atomicAdd(&s_h[warp][(word[i] >> shift) & mask], 1u);
  __syncthreads();
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) c += s_h[w][threadIdx.x];
  hist[blockIdx.x * 256 + threadIdx.x] = c;
}

// Per digit, the exclusive prefix over blocks of hist[block][digit], in place, and the
// digit's total in hist[kSortBlocks][digit].  One CTA per digit; the scatter turns the totals
// into digit bases itself.
__global__ void __launch_bounds__(256) k_radix_colscan(uint32_t* __restrict__ hist) {
  constexpr int kPer = (kSortBlocks + 255) / 256;
  __shared__ uint32_t s_warp[kWarps];
  const int d = blockIdx.x;
  const int b0 = threadIdx.x * kPer;
  uint32_t c[kPer];
  uint32_t local = 0;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    c[k] = b0 + k < kSortBlocks ? hist[(b0 + k) * 256 + d] : 0u;
    local += c[k];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan<256>(local, s_warp, total);
#pragma unroll
  for (int k = 0; k < kPer; ++k)
    if (b0 + k < kSortBlocks) {
      hist[(b0 + k) * 256 + d] = run;
      run += c[k];
    }
  if (threadIdx.x == 0) hist[kSortBlocks * 256 + d] = total;
}

// ---- bulk asynchronous copies into shared memory, completed on an mbarrier ----------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t arrivals) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(arrivals) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for the phase with this parity; false if `limit` tries ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t spin = 0; spin < limit; ++spin)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// orders this thread's earlier generic-proxy shared-memory accesses before later bulk copies
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Stable scatter of one digit.  Each CTA walks its chunk in tiles of kSortTile items; in a
// tile, warp w owns items [w*256, w*256+256) in 8 rounds of 32 and ranks them with
// match_any against per-warp digit counts; the tile is reordered by digit in shared memory
// and written out in digit runs.
// Two tile buffers alternate: while tile j is ranked and reordered in one, a bulk
// asynchronous copy brings tile j+1 into the other, so every CTA keeps a tile of loads in
// flight through its whole chunk.  Full tiles of 16-byte aligned arrays take that path;
// the rest (a chunk's ragged last tile, unaligned caller arrays) are loaded directly.
template <int WORDS, int DW>
__global__ void __launch_bounds__(kSortThreads, kSortCtasPerSM) k_radix_scatter(SortArrays<WORDS> arr, int shift,
                                                                                uint32_t mask, uint32_t spin,
                                                                DevStatus* __restrict__ st, int64_t fixed_count,
                                                                const uint32_t* __restrict__ hist) {
  extern __shared__ __align__(128) uint32_t s_dyn[];  // [2][WORDS][kSortTile]
  // per warp and digit: the tile's count, then the digit's first slot in the reordered tile
  // (16 bits each, two digits per word so that one 32-bit shared atomic adds to a count)
  __shared__ uint32_t s_wcnt[kWarps][128];
  __shared__ uint32_t s_delta[256];  // output position minus tile slot, per digit
  __shared__ uint32_t s_warp[kWarps];
  __shared__ __align__(8) uint64_t s_bar;
  uint16_t* const s_wc16 = reinterpret_cast<uint16_t*>(&s_wcnt[0][0]);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t total = items_of(st, fixed_count);
  const int64_t chunk = chunk_of(total);
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(total, beg + chunk);
  if (beg >= end) return;
  bool aligned = true;
#pragma unroll
  for (int w = 0; w < WORDS; ++w) aligned &= ((uintptr_t)arr.in[w] & 15u) == 0;
#define BULK_TILE(b) (aligned && end - (b) >= kSortTile)
#define BUF(j, w) (s_dyn + (((j) & 1) * WORDS + (w)) * kSortTile)
  constexpr uint32_t kTileBytes = (uint32_t)(WORDS * kSortTile * sizeof(uint32_t));
  // thread `tid` owns digit `tid`: its next output position for this CTA
  uint32_t bofs;
  {
    uint32_t all;
    const uint32_t digit_base = block_exclusive_scan<kSortThreads>(hist[kSortBlocks * 256 + tid], s_warp, all);
    bofs = digit_base + hist[blockIdx.x * 256 + tid];
  }
  for (int i = tid; i < kWarps * 128; i += kSortThreads) (&s_wcnt[0][0])[i] = 0;
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    if (BULK_TILE(beg)) {
      mbar_expect_tx(&s_bar, kTileBytes);
#pragma unroll
      for (int w = 0; w < WORDS; ++w) bulk_load(BUF(0, w), arr.in[w] + beg, kSortTile * 4u, &s_bar);
    }
  }
  __syncthreads();

  int j = 0;
  for (int64_t base = beg; base < end; base += kSortTile, ++j) {
    uint32_t item[kSortItems][WORDS], dig[kSortItems], rank[kSortItems];
    if (BULK_TILE(base)) {
      // every tile before j was a full bulk tile, so tile j completes phase j
      const bool ok = mbar_wait_bounded(&s_bar, (uint32_t)(j & 1), spin);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) st->code = XG_ERR_CHECK;
        mbar_wait_bounded(&s_bar, (uint32_t)(j & 1), kSpinLimit);  // let the copy in flight land first
        return;
      }
#pragma unroll
      for (int k = 0; k < kSortItems; ++k)
#pragma unroll
        for (int w = 0; w < WORDS; ++w) item[k][w] = BUF(j, w)[warp * (32 * kSortItems) + k * 32 + lane];
    } else {
#pragma unroll
      for (int k = 0; k < kSortItems; ++k) {
        const int64_t i = base + warp * (32 * kSortItems) + k * 32 + lane;
#pragma unroll
        for (int w = 0; w < WORDS; ++w) item[k][w] = i < end ? __ldg(arr.in[w] + i) : 0u;
      }
    }
    __syncthreads();  // tile j is in registers: its buffer becomes the reorder buffer
    if (tid == 0 && BULK_TILE(base + kSortTile)) {
      mbar_expect_tx(&s_bar, kTileBytes);
#pragma unroll
      for (int w = 0; w < WORDS; ++w) bulk_load(BUF(j + 1, w), arr.in[w] + base + kSortTile, kSortTile * 4u, &s_bar);
    }
    // rank within the warp: the leader of each digit group adds the group to the warp's
    // count and hands the previous count to the group
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      const int64_t i = base + warp * (32 * kSortItems) + k * 32 + lane;
      const bool valid = i < end;
      dig[k] = valid ? ((item[k][DW] >> shift) & mask) : 256u;
      const uint32_t peers = __match_any_sync(0xffffffffu, dig[k]);
      const int leader = __ffs(peers) - 1;
      if constexpr (WORDS == 2) {
        const uint32_t half = (dig[k] & 1u) * 16u;
        uint32_t old = 0;
        if (valid && lane == leader) old = atomicAdd(&s_wcnt[warp][dig[k] >> 1], (uint32_t)__popc(peers) << half);
        old = __shfl_sync(0xffffffffu, old, leader);
        rank[k] = ((old >> half) & 0xffffu) + __popc(peers & lt_mask);
      } else {  // fewer live registers: read the count, then the leader writes it back
        rank[k] = valid ? s_wc16[warp * 256 + dig[k]] + __popc(peers & lt_mask) : 0u;
        __syncwarp();
        if (valid && lane == leader) s_wc16[warp * 256 + dig[k]] += (uint16_t)__popc(peers);
        __syncwarp();
      }
    }
    __syncthreads();
    // digit `tid`: the tile's count, its first slot, and each warp's first slot
    uint32_t tile_count = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) tile_count += s_wc16[w * 256 + tid];
    uint32_t tile_total;
    uint32_t slot = block_exclusive_scan<kSortThreads>(tile_count, s_warp, tile_total);
    s_delta[tid] = bofs - slot;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = s_wc16[w * 256 + tid];
      s_wc16[w * 256 + tid] = (uint16_t)slot;
      slot += c;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      if (dig[k] < 256u) {
        const uint32_t loc = s_wc16[warp * 256 + dig[k]] + rank[k];
#pragma unroll
        for (int w = 0; w < WORDS; ++w) BUF(j, w)[loc] = item[k][w];
      }
    }
    __syncthreads();
    const int n_tile = (int)min((int64_t)kSortTile, end - base);
    for (int i = tid; i < n_tile; i += kSortThreads) {
      const uint32_t d = (BUF(j, DW)[i] >> shift) & mask;
      const uint32_t pos = s_delta[d] + (uint32_t)i;
      if ((int64_t)pos >= total) {  // cannot happen when the histograms are right
        st->code = XG_ERR_CHECK;
        continue;
      }
#pragma unroll
      for (int w = 0; w < WORDS; ++w) arr.out[w][pos] = BUF(j, w)[i];
    }
    fence_proxy_async_smem();  // this buffer receives tile j+2 by bulk copy
    bofs += tile_count;
    for (int i = tid; i < kWarps * 128; i += kSortThreads) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
  }
#undef BULK_TILE
#undef BUF
}


// ------------------------------------------------------------------------------------------
// tile ranges in the sorted pairs
// ------------------------------------------------------------------------------------------
// One thread per 4 consecutive sorted pairs (one 16-byte load); the keys just outside its
// four come from the neighbouring loads through L1.  The key array is 16-byte aligned and
// padded to a multiple of 16 bytes, so the last load stays inside it.
__global__ void __launch_bounds__(256) k_ranges(const uint32_t* __restrict__ key_tile, int64_t n_keys,
                                                DevStatus* __restrict__ st, uint2* __restrict__ range) {
  const int64_t total = items_of(st, -1);
  const int64_t quads = (total + 3) / 4;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < quads; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = 4 * q;
    const uint4 k4 = __ldg(reinterpret_cast<const uint4*>(key_tile) + q);
    const uint32_t k[6] = {i0 > 0 ? __ldg(key_tile + i0 - 1) : 0xffffffffu, k4.x, k4.y, k4.z, k4.w,
                           i0 + 4 < total ? __ldg(key_tile + i0 + 4) : 0xffffffffu};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int64_t i = i0 + e;
      if (i >= total) break;
      const uint32_t t = k[e + 1];
      if ((int64_t)t >= n_keys) {  // cannot happen when emit and sort are right
        st->code = XG_ERR_CHECK;
        continue;
      }
      if (i == 0 || k[e] != t) range[t].x = (uint32_t)i;
      if (i == total - 1 || k[e + 2] != t) range[t].y = (uint32_t)(i + 1);
    }
  }
}

// The compositing kernels take the (view, tile) work items in this order: by descending
// bucket of list length (four buckets per octave), so the long lists start in the first
// waves and the short ones fill the tail.  One CTA: a histogram, its scan, a scatter.
constexpr int kOrderBuckets = 129;

__device__ __forceinline__ int length_bucket(uint32_t len) {
  if (len == 0) return 0;
  const int lead = 31 - __clz(len);                                    // floor(log2 len)
  const int frac = lead >= 2 ? (int)((len >> (lead - 2)) & 3u) : (int)((len << (2 - lead)) & 3u);
  return 1 + 4 * lead + frac;                                          // 1 .. 128
}

__global__ void __launch_bounds__(1024) k_work_order(const uint2* __restrict__ range, int n_views, int tiles_per_view,
                                                     int tile_bits, const DevStatus* __restrict__ st,
                                                     uint32_t* __restrict__ order) {
  __shared__ uint32_t s_cnt[kOrderBuckets], s_base[kOrderBuckets];
  const int items = n_views * tiles_per_view;
  const bool ok = st->code == XG_OK;
  for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) s_cnt[b] = 0;
  __syncthreads();
  auto bucket_of = [&](int w) {
    const int v = w / tiles_per_view, t = w - v * tiles_per_view;
    const uint2 r = ok ? range[((int64_t)v << tile_bits) + t] : make_uint2(0u, 0u);
    return length_bucket(r.y - r.x);
  };
  for (int w = threadIdx.x; w < items; w += blockDim.x) atomicAdd(&s_cnt[bucket_of(w)], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int b = kOrderBuckets - 1; b >= 0; --b) {  // longest first
      s_base[b] = run;
      run += s_cnt[b];
    }
  }
  __syncthreads();
  for (int w = threadIdx.x; w < items; w += blockDim.x) order[atomicAdd(&s_base[bucket_of(w)], 1u)] = (uint32_t)w;
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
uint32_t spin_limit() {
  static const uint32_t limit = [] {
    const char* e = getenv("XG_SPIN_LIMIT");
    if (!e || !*e) return kSpinLimit;
    const unsigned long v = strtoul(e, nullptr, 10);
    return v < kSpinLimit ? (uint32_t)v : kSpinLimit;
  }();
  return limit;
}

template <int WORDS>
constexpr size_t scatter_smem() {
  return 2 * WORDS * kSortTile * sizeof(uint32_t);
}

template <int WORDS, int DW>
cudaError_t scatter_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_radix_scatter<WORDS, DW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)scatter_smem<WORDS>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_radix_scatter<WORDS, DW>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  return e;
}

// Dynamic shared memory of the scatter kernels, set once per process (the first call must
// not be inside a stream capture; frame creation makes it).
cudaError_t radix_prepare() {
  static cudaError_t once = [] {
    cudaError_t e = scatter_attrs<2, 0>();
    if (e == cudaSuccess) e = scatter_attrs<2, 1>();
    if (e == cudaSuccess) e = scatter_attrs<3, 0>();
    if (e == cudaSuccess) e = scatter_attrs<3, 1>();
    return e;
  }();
  return once;
}

template <int WORDS>
cudaError_t radix_pass(xg_frame* f, const SortArrays<WORDS>& arr, int digit_word, int shift, uint32_t mask,
                       int64_t fixed_count,
                       DevStatus* status, uint32_t* hist, cudaStream_t st) {
  const cudaError_t prep = radix_prepare();
  if (prep != cudaSuccess) return prep;
  {
    Timed t(f, kRadixHist, st);
    k_radix_hist<<<kSortBlocks, kSortThreads, 0, st>>>(arr.in[digit_word], shift, mask, status, fixed_count, hist);
  }
  {
    Timed t(f, kRadixScan, st);
    k_radix_colscan<<<256, 256, 0, st>>>(hist);
  }
  {
    Timed t(f, kRadixScatter, st);
    constexpr size_t smem = scatter_smem<WORDS>();
    if (digit_word == 0)
      k_radix_scatter<WORDS, 0><<<kSortBlocks, kSortThreads, smem, st>>>(arr, shift, mask, spin_limit(), status,
                                                                          fixed_count, hist);
    else
      k_radix_scatter<WORDS, 1><<<kSortBlocks, kSortThreads, smem, st>>>(arr, shift, mask, spin_limit(), status,
                                                                          fixed_count, hist);
  }
  return cudaGetLastError();
}

template cudaError_t radix_pass<2>(xg_frame*, const SortArrays<2>&, int, int, uint32_t, int64_t, DevStatus*, uint32_t*,
                                    cudaStream_t);
template cudaError_t radix_pass<3>(xg_frame*, const SortArrays<3>&, int, int, uint32_t, int64_t, DevStatus*, uint32_t*,
                                    cudaStream_t);

cudaError_t launch_bin_sort(xg_frame* f, cudaStream_t st) {
  const FramePtrs& p = f->p;
  const int64_t VN = (int64_t)f->n_views * f->n;
  // every binning starts from a clean code (a failed check of an earlier call does not stick)
  {
    Timed t(f, kMemset, st);
    const cudaError_t e = cudaMemsetAsync(&p.status->code, 0, sizeof(p.status->code), st);
    if (e != cudaSuccess) return e;
  }
  // stage 1: (view, depth) order of the V*n entries; words: view, depth bits, Gaussian
  int cur = 0;
  for (int pass = 0; pass < f->entry_passes; ++pass) {
    const int digit_word = pass < 4 ? 1 : 0;
    const int shift = pass < 4 ? 8 * pass : 8 * (pass - 4);
    SortArrays<3> arr;
    arr.in[0] = p.ent_view[cur], arr.in[1] = p.ent_depth[cur], arr.in[2] = p.ent_gid[cur];
    arr.out[0] = p.ent_view[cur ^ 1], arr.out[1] = p.ent_depth[cur ^ 1], arr.out[2] = p.ent_gid[cur ^ 1];
    const cudaError_t e = radix_pass<3>(f, arr, digit_word, shift, 255u, VN, p.status, p.hist, st);
    if (e != cudaSuccess) return e;
    cur ^= 1;
  }
  const uint32_t* ent_view = p.ent_view[cur];
  const uint32_t* ent_gid = p.ent_gid[cur];
  // stage 2: offsets of each entry's pairs in that order, then the pairs
  {
    Timed t(f, kScanReduce, st);
    k_scan_reduce<<<kSortBlocks, kSortThreads, 0, st>>>(p.count, ent_view, ent_gid, f->n, VN, p.status, p.scan_part);
  }
  {
    Timed t(f, kScanTop, st);
    k_scan_top<<<1, 1024, 0, st>>>(p.scan_part, f->cfg.pair_capacity, p.status);
  }
  {
    Timed t(f, kScanDown, st);
    k_scan_down<<<kSortBlocks, kSortThreads, 0, st>>>(p.count, ent_view, ent_gid, f->n, VN, p.status, p.scan_part,
                                                      p.offset);
  }
  {
    Timed t(f, kEmit, st);
    k_emit<<<(unsigned)((VN + 255) / 256), 256, 0, st>>>(p.count, p.offset, p.rect, ent_view, ent_gid, f->n, VN,
                                                         f->tiles_x, f->tile_bits, f->cfg.pair_capacity,
                                                         p.status, p.key_tile[0], p.value[0]);
  }
  // stage 3: stable sort of the pairs by tile key
  int pc = 0;
  for (int pass = 0; pass < f->tile_passes; ++pass) {
    SortArrays<2> arr;
    arr.in[0] = p.key_tile[pc], arr.in[1] = p.value[pc];
    arr.out[0] = p.key_tile[pc ^ 1], arr.out[1] = p.value[pc ^ 1];
    // the last pass takes only the tile bits left: the view bits above them must not move pairs
    const int left = f->tile_bits - 8 * pass;
    const uint32_t mask = left >= 8 ? 255u : (1u << left) - 1u;
    const cudaError_t e = radix_pass<2>(f, arr, 0, 8 * pass, mask, -1, p.status, p.hist, st);
    if (e != cudaSuccess) return e;
    pc ^= 1;
  }
  // stage 4: ranges
  cudaError_t e;
  {
    Timed t(f, kMemset, st);
    e = cudaMemsetAsync(p.range, 0, sizeof(uint2) * (size_t)f->range_keys, st);
  }
  if (e != cudaSuccess) return e;
  {
    Timed t(f, kRanges, st);
    k_ranges<<<kSortBlocks * 4, 256, 0, st>>>(p.key_tile[pc], f->range_keys, p.status,
                                               p.range);
  }
  {
    Timed t(f, kRanges, st);
    k_work_order<<<1, 1024, 0, st>>>(p.range, f->n_views, (int)f->tiles_per_view, f->tile_bits, p.status, p.order);
  }
  return cudaGetLastError();
}

}  // namespace xg

// Tile binning and the depth order of every tile's list (Sec. 3.2: Gaussians are assigned
// to the tiles their projection touches and sorted by depth).
//
// The (tile, view, depth) order of the pairs is built without sorting the pairs:
//
//   1. the V*n (view, Gaussian) entries, written by k_project at v*n + Gaussian, are sorted
//      within each view by the bits of t_z with a stable LSD radix sort (4 passes of 8 bits
//      over the (depth key, Gaussian) words, every view a segment of its own), so view v's
//      entries [v*n, (v+1)*n) come out in (depth, index) order;
//   2. each view's sorted entries are cut into units of E; per unit, the pairs falling on
//      every tile are counted from the entries' tile rectangles with a 2-D difference array;
//   3. a prefix over the units of each (view, tile) and a scan of the (view, tile) totals in
//      (tile, view) order give every (unit, tile) its first output position, and the
//      ranges [start, end) per (view, tile), indexed by view << B | tile (B = ceil(log2 T));
//   4. each unit's entries are walked in order again and every pair's Gaussian index is
//      written at its tile's next position.  Warp w of a CTA owns the tile rows congruent
//      to w modulo 8, so each tile is advanced by one warp only, in entry order: the list
//      of every (view, tile) comes out in (depth, index) order, contiguous, with no key
//      array and no pass over the pairs other than the one that writes them.
//
// The radix passes run on about 4 CTAs per SM (the frame's sort_blocks), each view's
// segment split among ceil(sort_blocks / V) of them; these grids and the binning grids depend only on the
// frame's sizes.  The host never needs to know the pair count, so the whole
// sequence can be captured in a CUDA graph, and no CTA waits on another.
#include <stdlib.h>

#include "xg_internal.cuh"

namespace xg {

constexpr int kWarps = kSortThreads / 32;
constexpr int kLocalPrefixBlocks = 64;  // segments of at most this many blocks: no column scan

// Items [beg, end) of this CTA in a segmented radix pass: segment s = blockIdx.x / per_seg
// holds items [s * seg_len, (s + 1) * seg_len) and is split among its per_seg CTAs in chunks
// of whole radix tiles.
__device__ __forceinline__ void sort_range(const SortGeom& g, int& seg, int64_t& beg, int64_t& end) {
  seg = (int)(blockIdx.x / (unsigned)g.per_seg);
  const int64_t j = blockIdx.x - (int64_t)seg * g.per_seg;
  int64_t c = (g.seg_len + g.per_seg - 1) / g.per_seg;
  c = (c + kSortTile - 1) / kSortTile * kSortTile;
  const int64_t s0 = (int64_t)seg * g.seg_len, s1 = s0 + g.seg_len;
  beg = min(s1, s0 + j * c);
  end = min(s1, beg + c);
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
// LSD radix sort, one 8-bit digit per pass, of WORDS parallel u32 arrays; the digit comes
// from array `digit_word`.  Histograms are block-major: hist[block][256].  Where a segment
// has at most kLocalPrefixBlocks blocks, each scatter CTA sums its segment's rows for its
// positions; otherwise a column scan over all blocks runs first.
// ------------------------------------------------------------------------------------------
// Whether the digits at `shift` and above are the same for every nonzero key of the span
// (the keys lying between the smallest and the largest share every bit above the highest
// bit in which those two differ); false when no key was nonzero.
__device__ __forceinline__ bool digits_constant(const uint32_t* span, int shift) {
  const uint32_t mx = span[0], mn = ~span[1];
  return mx >= mn && ((mx ^ mn) >> shift) == 0u;
}

// The entry sort's two ping-pong plane sets and its key span.  The passes that run write set
// 1, 0, 1, ... in turn; the passes that the span shows constant are the last ones and leave
// the planes where they are, so the sorted entries are in set (passes run) mod 2, and the
// other set is free.
struct SortedPlanes {
  uint32_t *depth0, *depth1, *gid0, *gid1;
  const uint32_t* span;
  int passes;
};
__device__ __forceinline__ int sorted_set(const SortedPlanes& sp) {
  int run = 1;
  for (int q = 1; q < sp.passes; ++q) run += digits_constant(sp.span, 8 * q) ? 0 : 1;
  return run & 1;
}

// With `span`: at shift 0 the histogram pass also records the range of the nonzero keys
// (largest key and largest complement, by atomic maxima); at a later shift it does nothing
// when that pass's digits are constant.
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ word, int shift, uint32_t mask,
                                                             SortGeom geom, uint32_t* __restrict__ hist,
                                                             uint32_t* __restrict__ span) {
  __shared__ uint32_t s_h[kWarps][256];
  if (span && shift > 0 && digits_constant(span, shift)) return;
  const bool record = span && shift == 0;
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&s_h[0][0])[i] = 0;
  __syncthreads();
  int seg;
  int64_t beg, end;
  sort_range(geom, seg, beg, end);
  uint32_t mx = 0u, mxn = 0u;
  for (int64_t i = beg + threadIdx.x; i < end; i += kSortThreads) {
    const uint32_t k = word[i];
    atomicAdd(&s_h[warp][(k >> shift) & mask], 1u);
    if (record && k != 0u) {
      mx = max(mx, k);
      mxn = max(mxn, ~k);
    }
  }
  __shared__ uint32_t s_span[2];
  if (record) {  // one pair of atomics per block: the two words are the same for every block
    if (threadIdx.x == 0) s_span[0] = s_span[1] = 0u;
    __syncthreads();
    mx = __reduce_max_sync(0xffffffffu, mx);
    mxn = __reduce_max_sync(0xffffffffu, mxn);
    if ((threadIdx.x & 31) == 0) {
      atomicMax(&s_span[0], mx);
      atomicMax(&s_span[1], mxn);
    }
  }
  __syncthreads();
  if (record && threadIdx.x == 0 && s_span[0] != 0u) {
    atomicMax(&span[0], s_span[0]);
    atomicMax(&span[1], s_span[1]);
  }
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) c += s_h[w][threadIdx.x];
  hist[blockIdx.x * 256 + threadIdx.x] = c;
}

// Segments of many blocks (more than kLocalPrefixBlocks): per digit, the exclusive prefix
// over all blocks of hist[block][digit], in place, and the digit's total in
// hist[blocks][digit] (counts wrap modulo 2^32; the scatter only takes differences inside one
// segment).  One CTA per digit; the scatter turns the prefixes into positions inside its
// segment itself.
__global__ void __launch_bounds__(256) k_radix_colscan(uint32_t* __restrict__ hist, int blocks,
                                                       const uint32_t* __restrict__ span, int shift) {
  __shared__ uint32_t s_warp[kWarps];
  if (span && shift > 0 && digits_constant(span, shift)) return;
  const int d = blockIdx.x;
  const int per = (blocks + 255) / 256;
  const int b0 = min(blocks, (int)threadIdx.x * per), b1 = min(blocks, b0 + per);
  uint32_t local = 0;
  for (int b = b0; b < b1; ++b) local += hist[b * 256 + d];
  uint32_t total;
  uint32_t run = block_exclusive_scan<256>(local, s_warp, total);
  for (int b = b0; b < b1; ++b) {
    const uint32_t c = hist[b * 256 + d];
    hist[b * 256 + d] = run;
    run += c;
  }
  if (threadIdx.x == 0) hist[blocks * 256 + d] = total;
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
// IOTA1: word 1 is not read but generated, the item's index within its segment (the first
// pass over the entries, whose Gaussian index is that position).
template <int WORDS, int DW, bool IOTA1>
__global__ void __launch_bounds__(kSortThreads, kSortCtasPerSM) k_radix_scatter(SortArrays<WORDS> arr, int shift,
                                                                                uint32_t mask, uint32_t spin,
                                                                DevStatus* __restrict__ st, SortGeom geom,
                                                                const uint32_t* __restrict__ hist,
                                                                const uint32_t* __restrict__ span) {
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
  int seg;
  int64_t beg, end;
  sort_range(geom, seg, beg, end);
  if (beg >= end) return;
  // every nonzero key has the same digit here: the stable pass would move none of them, so
  // the planes stay where they are (the consumers find them through sorted_buffer)
  if (!IOTA1 && span && shift > 0 && digits_constant(span, shift)) return;
  const int64_t seg_base = (int64_t)seg * geom.seg_len;
  constexpr int LOADED = IOTA1 ? 1 : WORDS;  // words read from memory (the first LOADED)
  bool aligned = true;  // every tile of the chunk starts 16-byte aligned in every array read
#pragma unroll
  for (int w = 0; w < LOADED; ++w) aligned &= ((uintptr_t)(arr.in[w] + beg) & 15u) == 0;
#define BULK_TILE(b) (aligned && end - (b) >= kSortTile)
#define BUF(j, w) (s_dyn + (((j) & 1) * WORDS + (w)) * kSortTile)
  constexpr uint32_t kTileBytes = (uint32_t)(LOADED * kSortTile * sizeof(uint32_t));
  // thread `tid` owns digit `tid`: its next output position for this CTA, counted from the
  // start of the segment (prefix differences taken modulo 2^32 are exact: a segment holds
  // fewer than 2^32 items)
  uint32_t bofs;
  {
    // the digit's count in this segment and in the segment's blocks before this one: summed
    // from the blocks' rows (at most kLocalPrefixBlocks independent loads per thread), or
    // taken from the column scan's prefixes
    const int b0 = seg * geom.per_seg, b1 = b0 + geom.per_seg, me = (int)blockIdx.x;
    uint32_t in_seg = 0u, before = 0u;
    if (geom.per_seg <= kLocalPrefixBlocks) {
#pragma unroll 4
      for (int b = b0; b < b1; ++b) {
        const uint32_t c = hist[b * 256 + tid];
        in_seg += c;
        before += b < me ? c : 0u;
      }
    } else {
      const uint32_t first = hist[b0 * 256 + tid];
      in_seg = hist[b1 * 256 + tid] - first;
      before = hist[me * 256 + tid] - first;
    }
    uint32_t all;
    const uint32_t digit_base = block_exclusive_scan<kSortThreads>(in_seg, s_warp, all);
    bofs = digit_base + before;
  }
  for (int i = tid; i < kWarps * 128; i += kSortThreads) (&s_wcnt[0][0])[i] = 0;
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    if (BULK_TILE(beg)) {
      mbar_expect_tx(&s_bar, kTileBytes);
#pragma unroll
      for (int w = 0; w < LOADED; ++w) bulk_load(BUF(0, w), arr.in[w] + beg, kSortTile * 4u, &s_bar);
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
        for (int w = 0; w < LOADED; ++w) item[k][w] = BUF(j, w)[warp * (32 * kSortItems) + k * 32 + lane];
    } else {
#pragma unroll
      for (int k = 0; k < kSortItems; ++k) {
        const int64_t i = base + warp * (32 * kSortItems) + k * 32 + lane;
#pragma unroll
        for (int w = 0; w < LOADED; ++w) item[k][w] = i < end ? __ldg(arr.in[w] + i) : 0u;
      }
    }
    if constexpr (IOTA1) {
#pragma unroll
      for (int k = 0; k < kSortItems; ++k)
        item[k][1] = (uint32_t)(base + warp * (32 * kSortItems) + k * 32 + lane - seg_base);
    }
    __syncthreads();  // tile j is in registers: its buffer becomes the reorder buffer
    if (tid == 0 && BULK_TILE(base + kSortTile)) {
      mbar_expect_tx(&s_bar, kTileBytes);
#pragma unroll
      for (int w = 0; w < LOADED; ++w) bulk_load(BUF(j + 1, w), arr.in[w] + base + kSortTile, kSortTile * 4u, &s_bar);
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
      if ((int64_t)pos >= geom.seg_len) {  // cannot happen when the histograms are right
        st->code = XG_ERR_CHECK;
        continue;
      }
#pragma unroll
      for (int w = 0; w < WORDS; ++w) arr.out[w][seg_base + pos] = BUF(j, w)[i];
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
// stages 2-4: the pairs, written straight into (tile, view, depth, index) order
// ------------------------------------------------------------------------------------------
struct BinGeom {
  int64_t n;      // Gaussians: view v's sorted entries are [v*n, (v+1)*n)
  int64_t tiles;  // T, tiles per view
  int32_t n_views;
  int32_t tiles_x, tiles_y, tile_bits;
  int32_t unit, units, rows, groups;  // E entries per unit, J units per view, R rows per group, G groups
};

// The CTA's unit u = v*J + j of sorted entries [beg, end) and its group of tile rows
// [r0, r0 + rows): blockIdx.x = u*G + group.
struct BinWork {
  int64_t u, beg, end;
  int v, r0, rows;
};

__device__ __forceinline__ BinWork bin_work(const BinGeom& g) {
  BinWork w;
  const int grp = (int)(blockIdx.x % (unsigned)g.groups);
  w.u = blockIdx.x / (unsigned)g.groups;
  w.v = (int)(w.u / g.units);
  const int64_t j = w.u - (int64_t)w.v * g.units;
  w.beg = (int64_t)w.v * g.n + j * g.unit;
  w.end = min((int64_t)(w.v + 1) * g.n, w.beg + g.unit);
  w.r0 = grp * g.rows;
  w.rows = min(g.rows, g.tiles_y - w.r0);
  return w;
}

// Sorted entry i's Gaussian and its whole tile rectangle (rows not clipped); false if the
// Gaussian touches no tile, or (recording XG_ERR_CHECK) if its index or rectangle is out of
// range.
__device__ __forceinline__ bool entry_full_rect(const BinGeom& g, const BinWork& w, int64_t i,
                                                const uint32_t* __restrict__ ent_gid,
                                                const uint32_t* __restrict__ count, const ushort4* __restrict__ rect,
                                                DevStatus* __restrict__ st, uint32_t& gid, int& x0, int& x1, int& y0,
                                                int& y1) {
  gid = ent_gid[i];
  if (gid >= g.n) {
    st->code = XG_ERR_CHECK;
    return false;
  }
  const int64_t vg = (int64_t)w.v * g.n + gid;
  if (count[vg] == 0) return false;
  const ushort4 r = rect[vg];
  if (r.x > r.z || r.y > r.w || r.z >= g.tiles_x || r.w >= g.tiles_y) {
    st->code = XG_ERR_CHECK;
    return false;
  }
  x0 = r.x;
  x1 = r.z;
  y0 = r.y;
  y1 = r.w;
  return true;
}

// (R + 1) x (tiles_x + 1) words, R * tiles_x <= max(kBinGroupTiles, tiles_x), R and tiles_x <= 512
constexpr int kBinDiffWords = kBinGroupTiles + 2 * 512 + 1;
constexpr int kCountBatch = 4;  // sorted entries a counting thread loads at a time

// Stage 2: pairs per tile of one unit (and group of rows).  Every entry adds its rectangle
// to a 2-D difference array in four shared atomics; prefix sums along the rows and then
// down the columns turn it into the count of every tile.
//
// The CTAs of the first group also write every sorted entry's tile rectangle in entry order
// (columns x0 | x1 << 16 in ent_x, rows y0 | y1 << 16 in ent_y; ent_y = 1 (y0 > y1) for an
// entry with no tile), so that the pair scatter reads them sequentially instead of
// gathering them by Gaussian index again.
__global__ void __launch_bounds__(kBinThreads) k_bin_count(BinGeom g, SortedPlanes sp,
                                                           const uint32_t* __restrict__ count,
                                                           const ushort4* __restrict__ rect,
                                                           DevStatus* __restrict__ st,
                                                           uint32_t* __restrict__ bin_hist) {
  __shared__ int32_t s_d[kBinDiffWords];
  if (st->code != XG_OK) return;  // stage 1 failed a check: its entries are not to be read
  // the sorted entries, and the free planes of the other set for the rectangles
  const bool set1 = sorted_set(sp) == 1;
  const uint32_t* __restrict__ ent_gid = set1 ? sp.gid1 : sp.gid0;
  uint32_t* __restrict__ ent_x = set1 ? sp.depth0 : sp.depth1;
  uint32_t* __restrict__ ent_y = set1 ? sp.gid0 : sp.gid1;
  const BinWork w = bin_work(g);
  const int cols = g.tiles_x + 1;
  const int cells = (w.rows + 1) * cols;
  for (int k = threadIdx.x; k < cells; k += kBinThreads) s_d[k] = 0;
  __syncthreads();
  const bool writer = w.r0 == 0;  // the first group writes the sorted rectangles
  // kCountBatch entries per thread at a time: every load of the batch is issued before any
  // of its results is used (the Gaussian index, then its count and rectangle together)
  for (int64_t i0 = w.beg + threadIdx.x; i0 < w.end; i0 += kCountBatch * kBinThreads) {
    uint32_t gid[kCountBatch], cnt[kCountBatch];
    ushort4 rc[kCountBatch];
#pragma unroll
    for (int u = 0; u < kCountBatch; ++u) {
      const int64_t i = i0 + (int64_t)u * kBinThreads;
      gid[u] = i < w.end ? ent_gid[i] : 0xffffffffu;
    }
#pragma unroll
    for (int u = 0; u < kCountBatch; ++u) {
      const bool ok = gid[u] < (uint64_t)g.n;
      const int64_t vg = (int64_t)w.v * g.n + (ok ? gid[u] : 0u);
      cnt[u] = ok ? count[vg] : 0u;
      rc[u] = ok ? rect[vg] : make_ushort4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < kCountBatch; ++u) {
      const int64_t i = i0 + (int64_t)u * kBinThreads;
      if (i >= w.end) break;
      bool any = false;
      int x0 = 0, x1 = 0, ya = 0, yb = 0;
      if (gid[u] >= (uint64_t)g.n) {
        st->code = XG_ERR_CHECK;
      } else if (cnt[u] != 0u) {
        const ushort4 r = rc[u];
        if (r.x > r.z || r.y > r.w || r.z >= g.tiles_x || r.w >= g.tiles_y) {
          st->code = XG_ERR_CHECK;
        } else {
          any = true;
          x0 = r.x, x1 = r.z, ya = r.y, yb = r.w;
        }
      }
      if (writer) {
        ent_x[i] = any ? (uint32_t)x0 | (uint32_t)x1 << 16 : 0u;
        ent_y[i] = any ? (uint32_t)ya | (uint32_t)yb << 16 : 1u;
      }
      if (!any) continue;
      ya = max(ya, w.r0);
      yb = min(yb, w.r0 + w.rows - 1);
      if (ya > yb) continue;
      const int a = (ya - w.r0) * cols, b = (yb - w.r0 + 1) * cols;
      atomicAdd(&s_d[a + x0], 1);
      atomicAdd(&s_d[a + x1 + 1], -1);
      atomicAdd(&s_d[b + x0], -1);
      atomicAdd(&s_d[b + x1 + 1], 1);
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int y = warp; y < w.rows; y += kBinThreads / 32) {  // along each row: a warp per row
    int carry = 0;
    for (int xb = 0; xb < g.tiles_x; xb += 32) {
      const int x = xb + lane;
      int v = x < g.tiles_x ? s_d[y * cols + x] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      v += carry;
      if (x < g.tiles_x) s_d[y * cols + x] = v;
      carry = __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < g.tiles_x; x += kBinThreads) {  // down each column
    int run = 0;
    for (int y = 0; y < w.rows; ++y) {
      run += s_d[y * cols + x];
      s_d[y * cols + x] = run;
    }
  }
  __syncthreads();
  uint32_t* out = bin_hist + w.u * g.tiles + (int64_t)w.r0 * g.tiles_x;
  const int nt = w.rows * g.tiles_x;
  for (int k = threadIdx.x; k < nt; k += kBinThreads) {
    const int y = k / g.tiles_x;
    out[k] = (uint32_t)s_d[y * cols + (k - y * g.tiles_x)];
  }
}

// Stage 3a: per (view, tile), the exclusive prefix over the view's units of bin_hist, in
// place, and the total in bin_total[tile * V + view].  A CTA takes 32 tiles of one view
// (blockIdx.x = view * ceil(T / 32) + tile block); its 8 warps split the units in slices.
__global__ void __launch_bounds__(256) k_bin_colscan(BinGeom g, const DevStatus* __restrict__ st,
                                                     uint32_t* __restrict__ bin_hist, uint32_t* __restrict__ bin_total) {
  __shared__ uint32_t s_part[8][32];
  if (st->code != XG_OK) return;
  const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
  const int64_t blocks = (g.tiles + 31) / 32;
  const int v = (int)(blockIdx.x / blocks);
  const int64_t t = (blockIdx.x - (int64_t)v * blocks) * 32 + lane;
  const int per = (g.units + 7) / 8;
  const int j0 = min(g.units, slice * per), j1 = min(g.units, j0 + per);
  uint32_t* col = bin_hist + (int64_t)v * g.units * g.tiles + t;
  uint32_t sum = 0;
  if (t < g.tiles)
    for (int j = j0; j < j1; ++j) sum += col[(int64_t)j * g.tiles];
  s_part[slice][lane] = sum;
  __syncthreads();
  if (slice == 0) {
    uint32_t run = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint32_t c = s_part[k][lane];
      s_part[k][lane] = run;
      run += c;
    }
    if (t < g.tiles) bin_total[t * g.n_views + v] = run;
  }
  __syncthreads();
  if (t < g.tiles) {
    uint32_t run = s_part[slice][lane];
    for (int j = j0; j < j1; ++j) {
      const uint32_t c = col[(int64_t)j * g.tiles];
      col[(int64_t)j * g.tiles] = run;
      run += c;
    }
  }
}

// The compositing kernels take the (view, tile) work items in order of descending list
// length bucket (four buckets per octave), so the long lists start in the first waves and
// the short ones fill the tail.  k_bin_base counts the items of every bucket as it writes
// the ranges and leaves each bucket's first position in order_base; k_work_order, a grid
// of CTAs, then places its items: one shared atomic per run of lanes with the same bucket
// (neighbouring tiles mostly share a bucket), one global atomic per bucket and CTA.
constexpr int kOrderThreads = 512;

__device__ __forceinline__ int length_bucket(uint32_t len) {
  if (len == 0) return 0;
  const int lead = 31 - __clz(len);                                    // floor(log2 len)
  const int frac = lead >= 2 ? (int)((len >> (lead - 2)) & 3u) : (int)((len << (2 - lead)) & 3u);
  return 1 + 4 * lead + frac;                                          // 1 .. 128
}

// Stage 3b: the exclusive prefix of bin_total in (tile, view) order gives every (view,
// tile) list its place; written as range[view << B | tile] = [start, end), with [0, 0) for
// empty lists and the keys past the last tile.  The pair count and the capacity check go to the status word
// (on a failed stage 1 or capacity overflow every range is empty).  The items of each list
// length bucket are counted on the way, and order_base[b] receives the first work-order
// position of bucket b (longest first).  One CTA.
__global__ void __launch_bounds__(1024) k_bin_base(BinGeom g, int64_t capacity, const uint32_t* __restrict__ bin_total,
                                                   DevStatus* __restrict__ st, uint2* __restrict__ range,
                                                   uint32_t* __restrict__ order_base) {
  __shared__ unsigned long long s_warp[32];
  __shared__ uint32_t s_bucket[kOrderBuckets];
  for (int b = threadIdx.x; b < kOrderBuckets; b += 1024) s_bucket[b] = 0u;
  const bool failed = st->code != XG_OK;
  const int64_t nb = g.tiles * g.n_views;
  const int64_t per = (nb + 1023) / 1024;
  const int64_t q0 = min(nb, (int64_t)threadIdx.x * per), q1 = min(nb, q0 + per);
  unsigned long long sum = 0;
  if (!failed)
    for (int64_t q = q0; q < q1; ++q) sum += bin_total[q];
  unsigned long long total;
  unsigned long long run = block_exclusive_scan<1024>(sum, s_warp, total);
  const bool ok = !failed && total <= (unsigned long long)capacity;
  int64_t t = q0 / g.n_views, v = q0 - t * g.n_views;  // q = t * V + v, advanced in step with q
  for (int64_t q = q0; q < q1; ++q) {
    const uint32_t c = ok ? bin_total[q] : 0u;
    range[(v << g.tile_bits) + t] = c ? make_uint2((uint32_t)run, (uint32_t)(run + c)) : make_uint2(0u, 0u);
    atomicAdd(&s_bucket[length_bucket(c)], 1u);
    run += c;
    if (++v == g.n_views) {
      v = 0;
      ++t;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // descending exclusive scan of the bucket counts: lane l takes buckets 128 - 5l .. 124 - 5l
    const int lane = threadIdx.x;
    uint32_t own = 0u;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const int b = kOrderBuckets - 1 - (5 * lane + j);
      if (b >= 0) own += s_bucket[b];
    }
    uint32_t incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t at = incl - own;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const int b = kOrderBuckets - 1 - (5 * lane + j);
      if (b >= 0) {
        order_base[b] = at;
        at += s_bucket[b];
      }
    }
  }
  const int64_t pad = ((int64_t)1 << g.tile_bits) - g.tiles;
  for (int64_t k = threadIdx.x; k < pad * g.n_views; k += 1024) {
    const int64_t v = k / pad;
    range[(v << g.tile_bits) + g.tiles + (k - v * pad)] = make_uint2(0u, 0u);
  }
  if (threadIdx.x == 0) {
    st->scan_total = failed ? 0ull : total;
    st->pairs = failed ? 0ll : (long long)total;
    st->fwd_evaluated = st->fwd_contrib = st->bwd_evaluated = st->bwd_contrib = 0ull;
    if (!failed) st->code = ok ? XG_OK : XG_ERR_CAPACITY;
  }
}

// One staged entry: (x0 | x1 << 16, ya | yb << 16) with the rows clipped to the CTA's group,
// or ya > yb when it has no tile here; read in entry order from the rectangles the counting
// pass wrote (already checked there).
__device__ __forceinline__ uint2 stage_entry(const BinWork& w, int64_t i, const uint32_t* __restrict__ ent_gid,
                                             const uint32_t* __restrict__ ent_x, const uint32_t* __restrict__ ent_y,
                                             uint32_t& gid) {
  if (i < w.end) {
    const uint32_t ey = ent_y[i];
    const int ya = max((int)(ey & 0xffffu), w.r0), yb = min((int)(ey >> 16), w.r0 + w.rows - 1);
    if (ya <= yb) {
      gid = ent_gid[i];
      return make_uint2(ent_x[i], (uint32_t)ya | (uint32_t)yb << 16);
    }
  }
  gid = 0u;
  return make_uint2(0u, 1u);
}

// Stage 4: the unit's pairs at their places.  The CTA's tiles keep their next output
// position in shared memory (range start + the unit's prefix).  Blocks of kBinStage entries
// are staged in shared memory (the next block's loads are in flight while one is processed);
// warp w walks every entry of the block in order, but only over the tile rows r0 + w,
// r0 + w + 8, ... of its rectangle, 32 pairs at a time.  A pass of the warp takes K
// consecutive entries per lane (32 K of the block): a warp scan of the lanes' pair counts
// places them, the entries with pairs are compacted in order, and a round finds each lane's
// entry by an OR-reduction over the round's entry starts.  Two pairs of one round on the
// same tile come from different entries and are ranked in lane (= entry) order, by a
// per-tile lane mask built with shared atomics (kMaskRank; cheaper on large dense groups,
// whose full rounds hold 32 distinct tiles) or by match_any (cheaper on small groups).
//
// Stores are combined per kSlots values (16 bytes) of the output: a tile's values wait in a
// kSlots-entry shared buffer (slot = position mod kSlots) until the run of kSlots is
// complete, and then leave in one 16-byte store; a run filled within one round is stored by
// its lanes directly.  Only the runs a unit shares with its neighbours at the ends of a
// tile's list are written value by value (the slots before the list hold kNoValue).
constexpr uint32_t kNoValue = 0xffffffffu;
constexpr uint32_t kSlots = 4;
constexpr int kBinStage = 256;  // sorted entries staged per block (one per thread)
constexpr int kBinMaskRankTiles = 1024;  // groups above this many tiles rank by lane mask
// entries per lane in a warp's pass over the staged block: more entries give fuller rounds
// and fewer passes (the measured best: 2 on the large mask-ranked groups, 4 on the others)
constexpr int kMaskRankLaneEntries = 2;
constexpr int kMatchLaneEntries = 4;
static_assert(kBinStage % (32 * kMaskRankLaneEntries) == 0 && kBinStage % (32 * kMatchLaneEntries) == 0,
              "a staged block holds whole passes");

// K consecutive words from shared memory in one vector load (the address is K-word aligned).
template <int K>
__device__ __forceinline__ void load_words(const uint32_t* src, uint32_t (&out)[K]) {
  if constexpr (K == 4) {
    const uint4 v = *reinterpret_cast<const uint4*>(src);
    out[0] = v.x, out[1] = v.y, out[2] = v.z, out[3] = v.w;
  } else if constexpr (K == 2) {
    const uint2 v = *reinterpret_cast<const uint2*>(src);
    out[0] = v.x, out[1] = v.y;
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = src[k];
  }
}

// Words of a per-tile shared array of `tiles` tiles padded by one word every 32 tiles.
__host__ __device__ __forceinline__ int bin_padded(int tiles) { return tiles + (tiles >> 5) + 1; }

template <bool kMaskRank, int K>
__global__ void __launch_bounds__(kBinThreads) k_bin_scatter(BinGeom g, SortedPlanes sp,
                                                             const uint32_t* __restrict__ bin_hist,
                                                             const uint2* __restrict__ range,
                                                             DevStatus* __restrict__ st, uint32_t* __restrict__ value) {
  constexpr int kW = kBinThreads / 32;  // warps; warp w owns the rows congruent to w mod kW
  // per tile: next position, lane mask, then [slot][tile] buffers; tile t sits at
  // t + t / 32 so that tiles a multiple of 32 apart (a warp's rows) use different banks
  extern __shared__ uint32_t s_dyn[];
  const int ntg = g.rows * g.tiles_x;  // tiles of a full group
  const int npad = bin_padded(ntg);
  uint32_t* const s_pos = s_dyn;
  uint32_t* const s_mask = s_dyn + npad;
  uint32_t* const s_buf = s_dyn + 2 * npad;
  // staged entries, one plane per word (a lane's K consecutive entries are one vector load)
  __shared__ __align__(16) uint32_t s_ex[2][kBinStage];
  __shared__ __align__(16) uint32_t s_ey[2][kBinStage];
  __shared__ __align__(16) uint32_t s_gid[2][kBinStage];
  __shared__ uint4 s_cmp[kW][32 * K];  // per warp: its entries with pairs, compacted (prefix, packed, 1/width, Gaussian)
  if (st->code != XG_OK) return;
  const bool set1 = sorted_set(sp) == 1;  // the sorted entries, and the rectangles in the other set
  const uint32_t* __restrict__ ent_gid = set1 ? sp.gid1 : sp.gid0;
  const uint32_t* __restrict__ ent_x = set1 ? sp.depth0 : sp.depth1;
  const uint32_t* __restrict__ ent_y = set1 ? sp.gid0 : sp.gid1;
  const int64_t pairs = st->pairs;
  const BinWork w = bin_work(g);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t t0 = (int64_t)w.r0 * g.tiles_x;
  const int nt = w.rows * g.tiles_x;
  {
    const uint2* rng = range + ((int64_t)w.v << g.tile_bits) + t0;
    const uint32_t* hst = bin_hist + w.u * g.tiles + t0;
    for (int k = threadIdx.x; k < nt; k += kBinThreads) {
      const uint32_t p = rng[k].x + hst[k];
      const int kp = k + (k >> 5);
      s_pos[kp] = p;
      s_mask[kp] = 0u;
      for (uint32_t q = 0; q < (p & (kSlots - 1)); ++q) s_buf[q * npad + kp] = kNoValue;
    }
  }
  bool bad = false;  // a position past the pair count (cannot happen when the counts are right)
  const bool stager = threadIdx.x < kBinStage;
  uint32_t gid_next = 0u;
  uint2 ent_next = make_uint2(0u, 1u);
  if (stager) {
    ent_next = stage_entry(w, w.beg + threadIdx.x, ent_gid, ent_x, ent_y, gid_next);
    s_ex[0][threadIdx.x] = ent_next.x;
    s_ey[0][threadIdx.x] = ent_next.y;
    s_gid[0][threadIdx.x] = gid_next;
  }
  __syncthreads();
  int buf = 0;
  for (int64_t blk = w.beg; blk < w.end; blk += kBinStage, buf ^= 1) {
    const bool more = blk + kBinStage < w.end;
    if (more && stager)
      ent_next = stage_entry(w, blk + kBinStage + threadIdx.x, ent_gid, ent_x, ent_y, gid_next);
    for (int sub = 0; sub < kBinStage / (32 * K); ++sub) {
      // lane l takes the staged entries sub*32K + l*K + k, k < K (consecutive: the prefix
      // over the warp's pairs is a warp scan of the lanes' sums)
      uint32_t cnt[K], pre[K], pk[K], rcp[K], gk[K], ex[K], ey[K];
      uint32_t lsum = 0u, nh = 0u;
      const int ix0 = sub * 32 * K + lane * K;
      load_words<K>(&s_ex[buf][ix0], ex);
      load_words<K>(&s_ey[buf][ix0], ey);
      load_words<K>(&s_gid[buf][ix0], gk);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int x0 = (int)(ex[k] & 0xffffu), x1 = (int)(ex[k] >> 16), ya = (int)(ey[k] & 0xffffu),
                  yb = (int)(ey[k] >> 16);
        const int yf = ya + ((warp - (ya - w.r0)) & (kW - 1));  // this warp's first row at or after ya
        const uint32_t wdt = (uint32_t)(x1 - x0 + 1);
        cnt[k] = yf <= yb ? ((uint32_t)(yb - yf) / kW + 1u) * wdt : 0u;
        pre[k] = lsum;
        lsum += cnt[k];
        nh += cnt[k] > 0u ? 1u : 0u;
        pk[k] = (uint32_t)(yf - w.r0) | (uint32_t)x0 << 10 | (wdt - 1u) << 20;
        rcp[k] = __float_as_uint(__frcp_rn((float)wdt));
      }
      uint32_t incl = lsum, hincl = nh;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        const uint32_t yh = __shfl_up_sync(0xffffffffu, hincl, d);
        if (lane >= d) {
          incl += y;
          hincl += yh;
        }
      }
      const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      if (tot == 0u) continue;
      // the entries with pairs, compacted in order: entry c's pairs are [pre_c, pre_c + cnt_c)
      {
        uint32_t hb = hincl - nh;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          pre[k] += incl - lsum;
          if (cnt[k] > 0u) s_cmp[warp][hb++] = make_uint4(pre[k], pk[k], rcp[k], gk[k]);
        }
        __syncwarp();
      }
      int last = -1;  // compacted entry holding the position before the round
      for (uint32_t p0 = 0; p0 < tot; p0 += 32) {
        const uint32_t p = p0 + lane;
        // the round's entry starts as a bit mask over its positions; a lane's entry is the
        // previous round's last one plus the starts at or before its position
        uint32_t bits = 0u;
#pragma unroll
        for (int k = 0; k < K; ++k) bits |= cnt[k] > 0u && pre[k] - p0 < 32u ? 1u << (pre[k] - p0) : 0u;
        const uint32_t starts = __reduce_or_sync(0xffffffffu, bits);
        const int ei = last + __popc(starts & (0xffffffffu >> (31 - lane)));
        last = __shfl_sync(0xffffffffu, ei, 31);
        const uint4 ce = s_cmp[warp][ei];
        const uint32_t e_pre = ce.x, e_pk = ce.y, e_gid = ce.w;
        const float e_rcp = __uint_as_float(ce.z);
        const uint32_t k = p - e_pre, ew = (e_pk >> 20) + 1u;
        // k / ew: the quotient is below 64 and (k + 1/2) / ew is at least 1/(2 ew) >= 2^-10
        // away from an integer, far above the 2^-23 relative error of the two roundings
        const uint32_t row = __float2uint_rz(__fmul_rn(__uint2float_rn(k) + 0.5f, e_rcp));
        const uint32_t col = k - row * ew;
        const uint32_t tl0 = ((e_pk & 1023u) + row * kW) * (uint32_t)g.tiles_x + ((e_pk >> 10) & 1023u) + col;
        const uint32_t tl = tl0 + (tl0 >> 5);  // padded index of the tile
        bool valid = p < tot;
        // the lanes of this round on the same tile, as a bit mask: earlier lanes hold earlier
        // entries, so a lane's rank among them is the count of lower bits
        uint32_t peers;
        if constexpr (kMaskRank) {
          if (valid) atomicOr(&s_mask[tl], 1u << lane);
          __syncwarp();
          peers = valid ? s_mask[tl] : 0u;
        } else {
          peers = __match_any_sync(0xffffffffu, valid ? tl : 0xffffffffu);
        }
        const uint32_t old = valid ? s_pos[tl] : 0u;
        const uint32_t pos = old + (uint32_t)__popc(peers & lt_mask);
        const uint32_t end = old + (uint32_t)__popc(peers);
        if (valid && (int64_t)pos >= pairs) {
          bad = true;
          valid = false;
        }
        constexpr uint32_t kLow = kSlots - 1u;
        const bool done = valid && (pos | kLow) < end;   // its run of kSlots is complete after this round
        const bool merge = done && (pos & ~kLow) < old;  // ... and holds values of earlier rounds
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) {
          s_pos[tl] = end;
          if constexpr (kMaskRank) s_mask[tl] = 0u;
        }
        if (merge) s_buf[(pos & kLow) * npad + tl] = e_gid;
        __syncwarp();
        if (merge && (pos & kLow) == kLow) {
          uint32_t v[kSlots];
          bool whole = true;
#pragma unroll
          for (int q = 0; q < (int)kSlots; ++q) {
            v[q] = s_buf[q * npad + tl];
            whole &= v[q] != kNoValue;
          }
          uint32_t* dst = value + (pos & ~kLow);
          if (whole) {
            *reinterpret_cast<uint4*>(dst) = make_uint4(v[0], v[1], v[2], v[3]);
          } else {
#pragma unroll
            for (int q = 0; q < (int)kSlots; ++q)
              if (v[q] != kNoValue) dst[q] = v[q];
          }
        } else if (done && !merge) {
          value[pos] = e_gid;  // the run's lanes store together
        }
        __syncwarp();
        if (valid && !done) s_buf[(pos & kLow) * npad + tl] = e_gid;
      }
    }
    if (more && stager) {
      s_ex[buf ^ 1][threadIdx.x] = ent_next.x;
      s_ey[buf ^ 1][threadIdx.x] = ent_next.y;
      s_gid[buf ^ 1][threadIdx.x] = gid_next;
    }
    __syncthreads();
  }
  // the last, incomplete run of every tile's list
  for (int k = threadIdx.x; k < nt; k += kBinThreads) {
    const int kp = k + (k >> 5);
    const uint32_t p = s_pos[kp];
    uint32_t* dst = value + (p & ~(kSlots - 1u));
    for (uint32_t q = 0; q < (p & (kSlots - 1u)); ++q) {
      const uint32_t v = s_buf[q * npad + kp];
      if (v != kNoValue) dst[q] = v;
    }
  }
  if (bad) st->code = XG_ERR_CHECK;
}

// The work order (see k_bin_base): one item per thread; an item of bucket b lands at
// order_base[b] (advanced by one global atomic per bucket and CTA) plus its place among the
// CTA's items of that bucket.  The ranges k_bin_base wrote give the lengths it counted, so
// every position lies inside the array; a position outside it (ranges from another call)
// records XG_ERR_CHECK and is not written.
__global__ void __launch_bounds__(kOrderThreads) k_work_order(const uint2* __restrict__ range, int n_views,
                                                              int tiles_per_view, int tile_bits,
                                                              DevStatus* __restrict__ st,
                                                              uint32_t* __restrict__ order_base,
                                                              uint32_t* __restrict__ order) {
  __shared__ uint32_t s_cnt[kOrderBuckets], s_base[kOrderBuckets];
  const int items = n_views * tiles_per_view;
  for (int b = threadIdx.x; b < kOrderBuckets; b += kOrderThreads) s_cnt[b] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t le_mask = 0xffffffffu >> (31 - lane);  // lanes 0 .. lane
  const int w = (int)blockIdx.x * kOrderThreads + (int)threadIdx.x;
  int b = -1;
  if (w < items) {
    const int v = w / tiles_per_view, t = w - v * tiles_per_view;
    const uint2 r = range[((int64_t)v << tile_bits) + t];
    b = length_bucket(r.y - r.x);
  }
  // runs of consecutive lanes with the same bucket: a lane leads a run if its bucket differs
  // from the previous lane's; the leader reserves the run's places
  const int prev = __shfl_up_sync(0xffffffffu, b, 1);
  const uint32_t leads = __ballot_sync(0xffffffffu, lane == 0 || b != prev);
  const uint32_t after = leads & ~le_mask;
  const int run_end = after ? __ffs(after) - 1 : 32;
  const int leader = 31 - __clz(leads & le_mask);
  uint32_t local = 0u;
  if (b >= 0 && leader == lane) local = atomicAdd(&s_cnt[b], (uint32_t)(run_end - lane));
  local = __shfl_sync(0xffffffffu, local, leader) + (uint32_t)(lane - leader);
  __syncthreads();
  for (int k = threadIdx.x; k < kOrderBuckets; k += kOrderThreads) {
    const uint32_t c = s_cnt[k];
    s_base[k] = c ? atomicAdd(&order_base[k], c) : 0u;
  }
  __syncthreads();
  if (b >= 0) {
    const uint32_t at = s_base[b] + local;
    if (at < (uint32_t)items) {
      order[at] = (uint32_t)w;
    } else {
      st->code = XG_ERR_CHECK;
    }
  }
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

template <int WORDS, int DW, bool IOTA1>
cudaError_t scatter_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_radix_scatter<WORDS, DW, IOTA1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scatter_smem<WORDS>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_radix_scatter<WORDS, DW, IOTA1>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  return e;
}

// Dynamic shared memory of the pair scatter: a position, a lane mask and kSlots buffer
// slots per tile of a group.
size_t bin_scatter_smem(int group_tiles) { return (size_t)(kSlots + 2) * 4 * (size_t)bin_padded(group_tiles); }

// Dynamic shared memory of the scatter kernels, set once per process (the first call must
// not be inside a stream capture; frame creation makes it).
cudaError_t radix_prepare() {
  static cudaError_t once = [] {
    cudaError_t e = cudaSuccess;
    for (const void* k : {(const void*)k_bin_scatter<true, kMaskRankLaneEntries>,
                          (const void*)k_bin_scatter<false, kMatchLaneEntries>})
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bin_scatter_smem(kBinGroupTiles));
    if (e == cudaSuccess) e = scatter_attrs<2, 0, false>();
    if (e == cudaSuccess) e = scatter_attrs<2, 0, true>();
    if (e == cudaSuccess) e = scatter_attrs<2, 1, false>();  // instantiated by radix_pass<2>, unused
    if (e == cudaSuccess) e = scatter_attrs<3, 0, false>();
    if (e == cudaSuccess) e = scatter_attrs<3, 1, false>();
    return e;
  }();
  return once;
}

template <int WORDS>
cudaError_t radix_pass(xg_frame* f, const SortArrays<WORDS>& arr, int digit_word, int shift, uint32_t mask,
                       const SortGeom& geom, DevStatus* status, uint32_t* hist, cudaStream_t st, bool iota1,
                       uint32_t* key_span) {
  if (digit_word != 0) key_span = nullptr;  // the span is of the keys in word 0
  const cudaError_t prep = radix_prepare();
  if (prep != cudaSuccess) return prep;
  const int blocks = geom.segments * geom.per_seg;
  {
    Timed t(f, kRadixHist, st);
    k_radix_hist<<<blocks, kSortThreads, 0, st>>>(arr.in[digit_word], shift, mask, geom, hist, key_span);
  }
  if (geom.per_seg > kLocalPrefixBlocks) {
    Timed t(f, kRadixScan, st);
    k_radix_colscan<<<256, 256, 0, st>>>(hist, blocks, key_span, shift);
  }
  {
    Timed t(f, kRadixScatter, st);
    constexpr size_t smem = scatter_smem<WORDS>();
    if (digit_word == 0 && iota1 && WORDS == 2)
      k_radix_scatter<WORDS, 0, WORDS == 2><<<blocks, kSortThreads, smem, st>>>(arr, shift, mask, spin_limit(), status,
                                                                                 geom, hist, key_span);
    else if (digit_word == 0)
      k_radix_scatter<WORDS, 0, false><<<blocks, kSortThreads, smem, st>>>(arr, shift, mask, spin_limit(), status,
                                                                            geom, hist, key_span);
    else
      k_radix_scatter<WORDS, 1, false><<<blocks, kSortThreads, smem, st>>>(arr, shift, mask, spin_limit(), status,
                                                                            geom, hist, key_span);
  }
  return cudaGetLastError();
}

template cudaError_t radix_pass<2>(xg_frame*, const SortArrays<2>&, int, int, uint32_t, const SortGeom&, DevStatus*,
                                    uint32_t*, cudaStream_t, bool, uint32_t*);
template cudaError_t radix_pass<3>(xg_frame*, const SortArrays<3>&, int, int, uint32_t, const SortGeom&, DevStatus*,
                                    uint32_t*, cudaStream_t, bool, uint32_t*);

cudaError_t launch_bin_sort(xg_frame* f, cudaStream_t st) {
  const FramePtrs& p = f->p;
  // every binning starts from a clean code (a failed check of an earlier call does not stick)
  {
    Timed t(f, kMemset, st);
    cudaError_t e = cudaMemsetAsync(&p.status->code, 0, sizeof(p.status->code), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.key_span, 0, 2 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
  }
  // stage 1: every view's n entries, [v*n, (v+1)*n), sorted by the depth bits as a segment
  // of its own; words: depth bits, Gaussian.  The first pass reads the projection's depth
  // plane (t_z >= 0, whose float bits order like the values) and generates the Gaussian
  // index, the entry's position in its view.  Culled entries have key 0 and no pairs; the
  // first pass records the range of the other keys, and a later pass whose digits are the
  // same for all of them (t_z between 512 and 2048 mm: the top byte) does nothing.
  const SortGeom sg = sort_geom(f->n, f->n_views, f->sort_blocks);
  int cur = 0;
  for (int pass = 0; pass < f->entry_passes; ++pass) {
    SortArrays<2> arr;
    arr.in[0] = pass == 0 ? reinterpret_cast<const uint32_t*>(p.depth) : p.ent_depth[cur];
    arr.in[1] = pass == 0 ? nullptr : p.ent_gid[cur];
    arr.out[0] = p.ent_depth[cur ^ 1], arr.out[1] = p.ent_gid[cur ^ 1];
    const cudaError_t e = radix_pass<2>(f, arr, 0, 8 * pass, 255u, sg, p.status, p.hist, st, pass == 0, p.key_span);
    if (e != cudaSuccess) return e;
    cur ^= 1;
  }
  // the sorted entries' set is known on the device only (a pass may have been a no-op);
  // the counting pass writes the sorted rectangles into the other set's free planes
  const SortedPlanes sp = {p.ent_depth[0], p.ent_depth[1], p.ent_gid[0], p.ent_gid[1], p.key_span, f->entry_passes};
  // stages 2-4: counts per unit and tile, their prefixes and the ranges, the pairs
  const BinGeom g = {f->n, f->tiles_per_view, f->n_views, f->tiles_x, f->tiles_y, f->tile_bits,
                     f->bin_unit, f->bin_units, f->bin_rows, f->bin_groups};
  const unsigned ctas = (unsigned)((int64_t)f->n_views * f->bin_units * f->bin_groups);
  {
    Timed t(f, kBinCount, st);
    k_bin_count<<<ctas, kBinThreads, 0, st>>>(g, sp, p.count, p.rect, p.status, p.bin_hist);
  }
  {
    Timed t(f, kBinColscan, st);
    k_bin_colscan<<<(unsigned)((int64_t)f->n_views * ((f->tiles_per_view + 31) / 32)), 256, 0, st>>>(
        g, p.status, p.bin_hist, p.bin_total);
  }
  {
    Timed t(f, kBinBase, st);
    k_bin_base<<<1, 1024, 0, st>>>(g, f->cfg.pair_capacity, p.bin_total, p.status, p.range, p.order_base);
  }
  {
    Timed t(f, kBinScatter, st);
    const int group_tiles = f->bin_rows * f->tiles_x;
    if (group_tiles > kBinMaskRankTiles)
      k_bin_scatter<true, kMaskRankLaneEntries><<<ctas, kBinThreads, bin_scatter_smem(group_tiles), st>>>(
          g, sp, p.bin_hist, p.range, p.status, p.value);
    else
      k_bin_scatter<false, kMatchLaneEntries><<<ctas, kBinThreads, bin_scatter_smem(group_tiles), st>>>(
          g, sp, p.bin_hist, p.range, p.status, p.value);
  }
  {
    Timed t(f, kWorkOrder, st);
    const int64_t items = (int64_t)f->n_views * f->tiles_per_view;
    k_work_order<<<(unsigned)((items + kOrderThreads - 1) / kOrderThreads), kOrderThreads, 0, st>>>(
        p.range, f->n_views, (int)f->tiles_per_view, f->tile_bits, p.status, p.order_base, p.order);
  }
  return cudaGetLastError();
}

}  // namespace xg

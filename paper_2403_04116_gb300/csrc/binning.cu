// Tile binning and the depth-keyed radix sort (Sec. 3.2: Gaussians are assigned to the
// tiles their projection touches and sorted by depth).
//
//   count --scan--> offset --emit--> (tile key, depth key, Gaussian) pairs
//         --LSD radix sort, 8-bit digits, depth bytes first, then tile bytes--> sorted pairs
//         --ranges--> [start, end) per (view, tile)
//
// Every kernel here runs on a fixed grid of kSortBlocks CTAs that split the work into
// contiguous chunks computed on the device from the pair count, so the host never needs to
// know the count and the whole sequence can be captured in a CUDA graph.  There is no
// inter-CTA waiting: each scan is reduce / scan-of-partials / down-sweep in three launches.
#include "xg_internal.cuh"

namespace xg {

constexpr int kWarps = kSortThreads / 32;

__device__ __forceinline__ int64_t chunk_of(int64_t total) {
  // per-CTA chunk: ceil(total / kSortBlocks) rounded up to whole radix tiles
  const int64_t c = (total + kSortBlocks - 1) / kSortBlocks;
  return (c + kSortTile - 1) / kSortTile * kSortTile;
}

__device__ __forceinline__ int64_t pairs_of(const DevStatus* st) { return st->code == XG_OK ? st->pairs : 0; }

// exclusive scan of one value per thread across a 256-thread block; returns the block total
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* s_warp, T& total) {
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
    T w = lane < kWarps ? s_warp[lane] : T(0);
#pragma unroll
    for (int o = 1; o < kWarps; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kWarps) s_warp[lane] = w;
  }
  __syncthreads();
  const T before = warp > 0 ? s_warp[warp - 1] : T(0);
  total = s_warp[kWarps - 1];
  __syncthreads();
  return before + x - v;
}

// ------------------------------------------------------------------------------------------
// scan of the per-(view, Gaussian) tile counts
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) k_scan_reduce(const uint32_t* __restrict__ count, int64_t total,
                                                              unsigned long long* __restrict__ part) {
  __shared__ unsigned long long s_warp[kWarps];
  const int64_t chunk = chunk_of(total);
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(total, beg + chunk);
  unsigned long long acc = 0;
  for (int64_t i = beg + threadIdx.x; i < end; i += kSortThreads) acc += count[i];
  unsigned long long tot;
  block_exclusive_scan(acc, s_warp, tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_scan_top(unsigned long long* __restrict__ part, int64_t capacity, DevStatus* __restrict__ st) {
  if (threadIdx.x != 0) return;
  unsigned long long run = 0;
  for (int b = 0; b < kSortBlocks; ++b) {
    const unsigned long long c = part[b];
    part[b] = run;
    run += c;
  }
  st->scan_total = run;
  st->pairs = (long long)run;
  st->fwd_evaluated = st->fwd_contrib = st->bwd_evaluated = st->bwd_contrib = 0ull;
  st->code = run > (unsigned long long)capacity ? XG_ERR_CAPACITY : XG_OK;
}

__global__ void __launch_bounds__(kSortThreads) k_scan_down(const uint32_t* __restrict__ count, int64_t total,
                                                            const unsigned long long* __restrict__ part,
                                                            uint32_t* __restrict__ offset) {
  __shared__ unsigned long long s_warp[kWarps];
  const int64_t chunk = chunk_of(total);
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(total, beg + chunk);
  unsigned long long run = part[blockIdx.x];
  for (int64_t base = beg; base < end; base += kSortThreads) {
    const int64_t i = base + threadIdx.x;
    const unsigned long long c = i < end ? count[i] : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_scan(c, s_warp, tot);
    if (i < end) offset[i] = (uint32_t)(run + ex);
    run += tot;
  }
}

// ------------------------------------------------------------------------------------------
// emit one pair per touched tile
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_emit(const uint32_t* __restrict__ count, const uint32_t* __restrict__ offset,
                                              const ushort4* __restrict__ rect, const float* __restrict__ depth,
                                              int64_t n, int n_views, int tiles_x, int64_t tiles_per_view,
                                              int64_t capacity, DevStatus* __restrict__ st,
                                              uint32_t* __restrict__ key_tile,
                                              uint32_t* __restrict__ key_depth, uint32_t* __restrict__ value) {
  const int64_t vg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (vg >= (int64_t)n_views * n) return;
  if (st->code != XG_OK) return;
  const uint32_t cnt = count[vg];
  if (cnt == 0) return;
  const int v = (int)(vg / n);
  const uint32_t g = (uint32_t)(vg - (int64_t)v * n);
  const ushort4 r = rect[vg];
  const uint32_t dbits = __float_as_uint(depth[vg]);
  const uint32_t vbase = (uint32_t)(v * tiles_per_view);
  uint32_t o = offset[vg];
  if ((int64_t)o + cnt > capacity) {  // cannot happen when the scan is right
    st->code = XG_ERR_CHECK;
    return;
  }
  for (int ty = r.y; ty <= r.w; ++ty)
    for (int tx = r.x; tx <= r.z; ++tx) {
      key_tile[o] = vbase + (uint32_t)(ty * tiles_x + tx);
      key_depth[o] = dbits;
      value[o] = g;
      ++o;
    }
}

// ------------------------------------------------------------------------------------------
// LSD radix sort of (key_tile, key_depth, value) triples, one 8-bit digit per pass
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ word, int shift,
                                                             const DevStatus* __restrict__ st,
                                                             uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_h[kWarps][256];
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&s_h[0][0])[i] = 0;
  __syncthreads();
  const int64_t total = pairs_of(st);
  const int64_t chunk = chunk_of(total);
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(total, beg + chunk);
  for (int64_t i = beg + threadIdx.x; i < end; i += kSortThreads) atomicAdd(&s_h[warp][(word[i] >> shift) & 255u], 1u);
  __syncthreads();
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) c += s_h[w][threadIdx.x];
  hist[threadIdx.x * kSortBlocks + blockIdx.x] = c;
}

// exclusive scan over hist[256][kSortBlocks] in digit-major order (one CTA of 1024 threads)
__global__ void __launch_bounds__(1024) k_radix_scan(uint32_t* __restrict__ hist) {
  constexpr int kN = 256 * kSortBlocks;
  constexpr int kPer = (kN + 1023) / 1024;
  __shared__ uint32_t s_warp[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int beg = threadIdx.x * kPer;
  uint32_t local = 0;
  for (int i = 0; i < kPer; ++i)
    if (beg + i < kN) local += hist[beg + i];
  uint32_t x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  uint32_t run = (warp > 0 ? s_warp[warp - 1] : 0u) + x - local;
  for (int i = 0; i < kPer; ++i)
    if (beg + i < kN) {
      const uint32_t c = hist[beg + i];
      hist[beg + i] = run;
      run += c;
    }
}

// Stable scatter of one digit.  Each CTA walks its chunk in tiles of kSortTile keys; inside
// a tile, warp w owns keys [w*256, w*256+256) in 8 rounds of 32, ranks them with match_any,
// the tile is reordered by digit in shared memory and written out in digit runs.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t* __restrict__ in_tile, const uint32_t* __restrict__ in_depth, const uint32_t* __restrict__ in_val,
    uint32_t* __restrict__ out_tile, uint32_t* __restrict__ out_depth, uint32_t* __restrict__ out_val, int digit_word,
    int shift, DevStatus* __restrict__ st, const uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_tile[kSortTile], s_depth[kSortTile], s_val[kSortTile];
  __shared__ uint32_t s_wcnt[kWarps][256];
  __shared__ uint32_t s_bofs[256], s_tofs[256], s_tcnt[256];
  __shared__ uint32_t s_warp[kWarps];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t total = pairs_of(st);
  const int64_t chunk = chunk_of(total);
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(total, beg + chunk);
  if (beg >= end) return;
  s_bofs[tid] = hist[tid * kSortBlocks + blockIdx.x];
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s_wcnt[w][tid] = 0;
  __syncthreads();

  for (int64_t base = beg; base < end; base += kSortTile) {
    uint32_t kt[kSortItems], kd[kSortItems], kv[kSortItems], dig[kSortItems], rank[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      const int64_t i = base + warp * (32 * kSortItems) + k * 32 + lane;
      const bool valid = i < end;
      kt[k] = valid ? in_tile[i] : 0u;
      kd[k] = valid ? in_depth[i] : 0u;
      kv[k] = valid ? in_val[i] : 0u;
      dig[k] = valid ? (((digit_word ? kt[k] : kd[k]) >> shift) & 255u) : 256u;
      const uint32_t peers = __match_any_sync(0xffffffffu, dig[k]);
      rank[k] = valid ? s_wcnt[warp][dig[k]] + __popc(peers & lt_mask) : 0u;
      __syncwarp();
      if (valid && lane == __ffs(peers) - 1) s_wcnt[warp][dig[k]] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // digit `tid`: warp-exclusive prefixes and the tile's count
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = s_wcnt[w][tid];
      s_wcnt[w][tid] = run;
      run += c;
    }
    s_tcnt[tid] = run;
    uint32_t tile_total;
    const uint32_t tofs = block_exclusive_scan(run, s_warp, tile_total);
    s_tofs[tid] = tofs;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      if (dig[k] < 256u) {
        const uint32_t loc = s_tofs[dig[k]] + s_wcnt[warp][dig[k]] + rank[k];
        s_tile[loc] = kt[k];
        s_depth[loc] = kd[k];
        s_val[loc] = kv[k];
      }
    }
    __syncthreads();
    const int n_tile = (int)min((int64_t)kSortTile, end - base);
    for (int i = tid; i < n_tile; i += kSortThreads) {
      const uint32_t t = s_tile[i], dd = s_depth[i];
      const uint32_t d = ((digit_word ? t : dd) >> shift) & 255u;
      const uint32_t pos = s_bofs[d] + (uint32_t)i - s_tofs[d];
      if ((int64_t)pos >= total) {  // cannot happen when the histograms are right
        st->code = XG_ERR_CHECK;
        continue;
      }
      out_tile[pos] = t;
      out_depth[pos] = dd;
      out_val[pos] = s_val[i];
    }
    __syncthreads();
    s_bofs[tid] += s_tcnt[tid];
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s_wcnt[w][tid] = 0;
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// tile ranges in the sorted pairs
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_ranges(const uint32_t* __restrict__ key_tile, int64_t n_keys,
                                                DevStatus* __restrict__ st, uint2* __restrict__ range) {
  const int64_t total = pairs_of(st);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t t = key_tile[i];
    if ((int64_t)t >= n_keys) {  // cannot happen when emit and sort are right
      st->code = XG_ERR_CHECK;
      continue;
    }
    if (i == 0 || key_tile[i - 1] != t) range[t].x = (uint32_t)i;
    if (i == total - 1 || key_tile[i + 1] != t) range[t].y = (uint32_t)(i + 1);
  }
}

cudaError_t launch_bin_sort(xg_frame* f, cudaStream_t st) {
  const FramePtrs& p = f->p;
  const int64_t VN = (int64_t)f->n_views * f->n;
  {
    Timed t(f, kScanReduce, st);
    k_scan_reduce<<<kSortBlocks, kSortThreads, 0, st>>>(p.count, VN, p.scan_part);
  }
  {
    Timed t(f, kScanTop, st);
    k_scan_top<<<1, 32, 0, st>>>(p.scan_part, f->cfg.pair_capacity, p.status);
  }
  {
    Timed t(f, kScanDown, st);
    k_scan_down<<<kSortBlocks, kSortThreads, 0, st>>>(p.count, VN, p.scan_part, p.offset);
  }
  {
    Timed t(f, kEmit, st);
    k_emit<<<(unsigned)((VN + 255) / 256), 256, 0, st>>>(p.count, p.offset, p.rect, p.depth, f->n, f->n_views,
                                                         f->tiles_x, f->tiles_per_view, f->cfg.pair_capacity,
                                                         p.status, p.key_tile[0], p.key_depth[0], p.value[0]);
  }
  int cur = 0;
  for (int pass = 0; pass < f->sort_passes; ++pass) {
    const int digit_word = pass < 4 ? 0 : 1;
    const int shift = pass < 4 ? 8 * pass : 8 * (pass - 4);
    const uint32_t* word = digit_word ? p.key_tile[cur] : p.key_depth[cur];
    {
      Timed t(f, kRadixHist, st);
      k_radix_hist<<<kSortBlocks, kSortThreads, 0, st>>>(word, shift, p.status, p.hist);
    }
    {
      Timed t(f, kRadixScan, st);
      k_radix_scan<<<1, 1024, 0, st>>>(p.hist);
    }
    {
      Timed t(f, kRadixScatter, st);
      k_radix_scatter<<<kSortBlocks, kSortThreads, 0, st>>>(p.key_tile[cur], p.key_depth[cur], p.value[cur],
                                                            p.key_tile[cur ^ 1], p.key_depth[cur ^ 1],
                                                            p.value[cur ^ 1], digit_word, shift, p.status, p.hist);
    }
    cur ^= 1;
  }
  f->sorted_buf = cur;
  cudaError_t e;
  {
    Timed t(f, kMemset, st);
    e = cudaMemsetAsync(p.range, 0, sizeof(uint2) * (size_t)(f->n_views * f->tiles_per_view), st);
  }
  if (e != cudaSuccess) return e;
  {
    Timed t(f, kRanges, st);
    k_ranges<<<kSortBlocks * 4, 256, 0, st>>>(p.key_tile[cur], (int64_t)f->n_views * f->tiles_per_view, p.status,
                                               p.range);
  }
  return cudaGetLastError();
}

}  // namespace xg

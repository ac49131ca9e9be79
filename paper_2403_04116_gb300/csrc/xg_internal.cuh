// Internal declarations shared by the library's CUDA translation units.
//
// FP32 decision sequence.  Every operation that decides which tiles a Gaussian touches,
// the depth key, or whether a Gaussian contributes to a pixel is written with explicit
// round-to-nearest intrinsics (__fmul_rn, __fadd_rn, __fmaf_rn, __fdiv_rn, __fsqrt_rn),
// which the compiler never contracts or reorders.  The sequence is fixed and documented
// so that an independent FP32 re-implementation reproduces tile ids, sort keys, ranges,
// contributor counts and last-contributor positions bit for bit.
#pragma once

#include <cuda_runtime.h>
#include <algorithm>
#include <stdint.h>

#include "../../include/xg.h"

namespace xg {

constexpr int kMaxViews = 65535;  // views of a frame (a grid dimension of the projection)
// Grids are sized from the SM count of the device they run on (cudaDevAttrMultiProcessorCount
// of the current device, read once per device; 1 if the query fails, which shrinks grids
// but changes no result).
int device_sms();
constexpr int kSortCtasPerSM = 4;
constexpr int kMaxSortBlocks = kSortCtasPerSM * 256;  // bound for statically sized arrays
// grid of the scan and radix-sort passes: 4 CTAs per SM
inline int sort_blocks() {
  const int b = kSortCtasPerSM * device_sms();
  return b < kMaxSortBlocks ? b : kMaxSortBlocks;
}
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;         // keys per thread per radix tile
constexpr int kSortTile = kSortThreads * kSortItems;
// pair scatter: a CTA takes one unit of sorted entries and one group of tile rows whose
// tiles (at most kBinGroupTiles) keep their next output position in shared memory
constexpr int kBinThreads = 256;
constexpr int kBinGroupTiles = 2048;
// iteration limit of every spin-wait in a kernel; on expiry the kernel records
// XG_ERR_CHECK in the status word and returns
constexpr uint32_t kSpinLimit = 1u << 22;
// buckets of tile-list length that order the compositing work items (four per octave)
constexpr int kOrderBuckets = 129;
// The limit the kernels' first waits use: kSpinLimit, or the XG_SPIN_LIMIT environment
// variable (read once per process) to make waits expire for fault-injection tests.  Waits
// that drain copies in flight before a kernel returns always use kSpinLimit.
uint32_t spin_limit();

// Decision constants (float roundings of the paper-level values).
constexpr double kLn2D = 0.69314718055994530942;
constexpr float kLog2e = (float)1.44269504088896340736;
constexpr float kLn2Hi = (float)kLn2D;
constexpr float kLn2Lo = (float)(kLn2D - (double)(float)kLn2D);
constexpr float kSqrt2 = (float)1.41421356237309504880;
constexpr float kAlphaMin = (float)(1.0 / 255.0);
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kDilate = 0.3f;
constexpr float kRadiusMargin = 1.0009765625f;  // 1 + 2^-10

// Per-view camera table in the workspace (16 floats).
struct Camera {
  float c, s;        // cos, sin of the azimuth (rounded from double)
  float L;           // L_SO
  float fu, fv;      // focal lengths in pixels, L_SD / pitch
  float hw, hh;      // W/2 - 1/2, H/2 - 1/2: pixel x has centred coordinate x - hw
  float pad[9];
};
static_assert(sizeof(Camera) == 64, "camera record is 64 bytes");

struct DevStatus {
  int32_t code;
  uint32_t next_item;  // persistent compositing launches: the next work item (zeroed per launch)
  long long pairs;
  unsigned long long nonfinite;
  unsigned long long fwd_evaluated;   // (pixel, list entry) pairs evaluated by the last forward
  unsigned long long fwd_contrib;     // of which contributed
  unsigned long long bwd_evaluated;   // pairs re-evaluated by the last backward
  unsigned long long bwd_contrib;     // of which contributed
  unsigned long long scan_total;      // internal: total of the counts (before the capacity check)
};
static_assert(sizeof(DevStatus) == 64, "status is 64 bytes");

// ------------------------------------------------------------------------------------------
// exact FP32 helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsqrt(float a) { return __fsqrt_rn(a); }

// e^x: Cody-Waite reduction by ln 2, degree-6 Taylor polynomial on |r| <= ln2/2, times 2^k.
// k = rint(x log2 e) is the nearest integer (ties to even) to the exact product, taken from
// one fused multiply-add: m = x log2 e + 1.5 * 2^23 rounded once holds it in its last
// mantissa bits (|x log2 e| < 2^22), and k = m - 1.5 * 2^23 is exact.
constexpr float kRound = 12582912.0f;  // 1.5 * 2^23
__device__ __forceinline__ float xg_exp(float x) {
  x = fmaxf(x, -80.0f);
  const float k = fsub(ffma(x, kLog2e, kRound), kRound);
  float r = ffma(k, -kLn2Hi, x);
  r = ffma(k, -kLn2Lo, r);
  float p = ffma(r, (float)(1.0 / 720.0), (float)(1.0 / 120.0));
  p = ffma(p, r, (float)(1.0 / 24.0));
  p = ffma(p, r, (float)(1.0 / 6.0));
  p = ffma(p, r, 0.5f);
  p = ffma(p, r, 1.0f);
  p = ffma(p, r, 1.0f);
  return fmul(p, __int_as_float(((int)k + 127) << 23));
}

// Packed two-lane FP32 (the f32x2 instructions of sm_100 and later): each lane is rounded
// exactly as the scalar operation, so packed and scalar sequences give the same bits as
// long as no packed multiply feeds a packed add that the compiler may fuse with it.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// xg_exp of two values, lane for lane bit-identical to it: m and k as in xg_exp, one packed
// fused multiply-add and one packed add.  The bits of m are 0x4B400000 + k, and shifted
// left by 23 they are k << 23 (the constant's low nine bits are zero), so the scaling by
// 2^k is an integer add of those bits to the bits of the polynomial's value p: p lies in
// [0.70, 1.42] and -116 <= k <= 127 (x in [-80, 88], the domain of xg_exp's scale as
// well), so the result stays normal, and the product p * 2^k that xg_exp rounds is exact
// -- the same bits.
//
// xg_exp2v_core takes x as it is: its value is xg_exp's for x in [-80, 88] and meaningless
// below.  The compositing kernels call it directly, because they keep exp only where the
// exponent reaches the record's threshold (above -6) and discard the other lanes' values.
__device__ __forceinline__ float2 xg_exp2v_core(float2 x) {
  const float2 m = ffma2(x, f2(kLog2e), f2(kRound));
  const float2 k = fadd2(m, f2(-kRound));
  float2 r = ffma2(k, f2(-kLn2Hi), x);
  r = ffma2(k, f2(-kLn2Lo), r);
  float2 p = ffma2(r, f2((float)(1.0 / 720.0)), f2((float)(1.0 / 120.0)));
  p = ffma2(p, r, f2((float)(1.0 / 24.0)));
  p = ffma2(p, r, f2((float)(1.0 / 6.0)));
  p = ffma2(p, r, f2(0.5f));
  p = ffma2(p, r, f2(1.0f));
  p = ffma2(p, r, f2(1.0f));
  return make_float2(__uint_as_float(__float_as_uint(p.x) + (__float_as_uint(m.x) << 23)),
                     __uint_as_float(__float_as_uint(p.y) + (__float_as_uint(m.y) << 23)));
}
__device__ __forceinline__ float2 xg_exp2v(float2 x) {
  return xg_exp2v_core(make_float2(fmaxf(x.x, -80.0f), fmaxf(x.y, -80.0f)));
}

// ln x for finite x >= 1: x = m 2^e, m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s), s = (m-1)/(m+1).
__device__ __forceinline__ float xg_log_ge1(float x) {
  const unsigned b = __float_as_uint(x);
  int e = (int)(b >> 23) - 127;
  float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
  if (m > kSqrt2) {
    m = fmul(m, 0.5f);
    e += 1;
  }
  const float s = fdiv(fsub(m, 1.0f), fadd(m, 1.0f));
  const float s2 = fmul(s, s);
  float p = ffma(s2, (float)(2.0 / 9.0), (float)(2.0 / 7.0));
  p = ffma(p, s2, (float)(2.0 / 5.0));
  p = ffma(p, s2, (float)(2.0 / 3.0));
  p = ffma(p, s2, 2.0f);
  p = fmul(p, s);
  const float ef = (float)e;
  const float t = ffma(ef, kLn2Lo, p);
  return ffma(ef, kLn2Hi, t);
}

// ------------------------------------------------------------------------------------------
// frame
// ------------------------------------------------------------------------------------------
struct FramePtrs {
  DevStatus* status;
  Camera* cam;
  float4* rec;        // [V*n][2]
  float* depth;       // [V*n]
  ushort4* rect;      // [V*n]
  uint32_t* count;    // [V*n]
  uint32_t* ent_depth[2];  // stage-1 sort of the V*n entries (ping-pong): depth key, Gaussian;
  uint32_t* ent_gid[2];    // the first pass reads `depth` and generates the Gaussian index
  uint32_t* value;    // [capacity]: Gaussian index of every pair, in (tile, view, depth) order
  uint32_t* hist;     // [radix blocks + 1][256]: per-block digit counts (prefixes after a column scan)
  uint32_t* key_span; // [2]: the entry sort's key range over its nonzero keys (max, max of ~key)
  uint32_t* bin_hist;   // [V][J][T]: pairs of each unit of entries per tile, then their prefix
  uint32_t* bin_total;  // [T][V]: pairs per (tile, view)
  uint2* range;       // [V << tile_bits]
  uint32_t* order;    // [V*T] (view, tile) work items, longest tile lists first
  uint32_t* order_base;  // [kOrderBuckets]: first work-order position of each list-length bucket
  float* tfinal;      // [V*H*W]
  uint32_t* last;     // [V*H*W]
  float* grad2d;      // [V*n][8]
};

// Parameter groups of one Adam step, passed by value.
struct AdamGroups {
  xg_adam_group g[XG_ADAM_MAX_GROUPS];
  int count;
};

// Segments of a radix pass: `segments` runs of seg_len items, [s*seg_len, (s+1)*seg_len),
// each sorted on its own by per_seg CTAs (grid segments * per_seg).
struct SortGeom {
  int64_t seg_len;
  int32_t segments, per_seg;
};

// About `blocks` CTAs over `segments` runs of seg_len items.
inline SortGeom sort_geom(int64_t seg_len, int32_t segments, int32_t blocks) {
  SortGeom g;
  g.seg_len = seg_len;
  g.segments = segments;
  // no more CTAs per segment than it has radix tiles (the others would sort nothing)
  const int64_t tiles = (seg_len + kSortTile - 1) / kSortTile;
  g.per_seg = (int32_t)std::max<int64_t>(1, std::min<int64_t>((blocks + segments - 1) / segments, tiles));
  return g;
}

// Input and output arrays of one radix pass, passed by value.
template <int WORDS>
struct SortArrays {
  const uint32_t* in[WORDS];
  uint32_t* out[WORDS];
};

}  // namespace xg

namespace xg {
enum KernelId {
  kProject, kBinCount, kBinColscan, kBinBase, kBinScatter, kRadixHist, kRadixScan, kRadixScatter, kWorkOrder,
  kRenderFwd, kRenderBwd, kProjectBwd, kMemset, kNumKernels
};
struct TimingRec {
  int kid;
  cudaEvent_t a, b;
};
constexpr int kMaxTimingRecs = 2048;
}  // namespace xg

struct xg_frame {
  xg_config cfg;
  int64_t n;
  int32_t n_views;         // views of the current pass (the kernels' V)
  int32_t n_scan;          // views in the camera table
  int32_t views_per_pass;  // capacity of the per-pass arrays
  int32_t first_view;      // camera-table index of the current pass's view 0
  int32_t width, height;
  int32_t tiles_x, tiles_y;
  int64_t tiles_per_view;
  int32_t tile_bits;     // bits of a tile index within its view: pair key = view << tile_bits | tile
  int64_t range_keys;    // n_views << tile_bits: entries of the range array
  int32_t entry_passes;  // stage-1 passes: the 4 depth bytes
  int32_t bin_unit;      // E: sorted entries per unit of the pair scatter
  int32_t bin_units;     // J: units per view, ceil(n / E)
  int32_t bin_rows;      // R: tile rows per group (R * tiles_x <= kBinGroupTiles)
  int32_t bin_groups;    // G: ceil(tiles_y / R)
  int32_t sort_blocks;   // CTAs of a radix pass (4 per SM of the device the frame was made on)
  int32_t render_blocks[2];  // persistent compositing: blocks that fit at once (forward, backward)
  void* workspace;
  size_t workspace_bytes;
  xg_layout layout;
  xg::Camera* cam_all;  // camera table of all n_scan views; p.cam = cam_all + first_view
  xg::FramePtrs p;
  // optional per-kernel timing with CUDA events on the launch stream
  int timing;
  int nrec;
  int dropped;
  xg::TimingRec* recs;
  double acc_ms[xg::kNumKernels];
  long long acc_n[xg::kNumKernels];
};

namespace xg {
// Brackets one launch with timing events when the frame's timing is on.
struct Timed {
  xg_frame* f;
  cudaStream_t st;
  int slot;
  Timed(xg_frame* frame, int kid, cudaStream_t stream);  // frame may be NULL (not timed)
  ~Timed();
};

// launchers, one per translation unit
cudaError_t launch_project(xg_frame* f, const xg_gaussians* g, cudaStream_t st);
cudaError_t launch_bin_sort(xg_frame* f, cudaStream_t st);
cudaError_t launch_render_fwd(xg_frame* f, float* image, uint32_t* n_contrib, cudaStream_t st);
cudaError_t launch_render_bwd(xg_frame* f, const float* grad_image, cudaStream_t st);
// Dynamic shared memory of a compositing block of this configuration.
size_t render_smem_bytes(const xg_config* cfg);
// Shared-memory attributes and persistent grid sizes of the frame's compositing kernels
// (frame creation; outside any stream capture).
cudaError_t render_prepare(xg_frame* f);
cudaError_t launch_project_bwd(xg_frame* f, const xg_gaussians* g, const xg_grads* out, cudaStream_t st);
cudaError_t launch_loss_l1(const float* image, const float* target, int64_t count, float scale, float* grad,
                           float* loss, cudaStream_t st);
cudaError_t launch_exp_check(const float* x, float* ys, float* yp, int64_t n, cudaStream_t st);

// One LSD radix pass (histogram, digit scan where segments have many blocks, stable scatter;
// binning.cu) over WORDS arrays,
// the digit (arr.in[digit_word] >> shift) & mask (mask <= 255), every segment of `geom`
// sorted on its own.  `hist` holds (segments * per_seg + 1) * 256 words.  `f` may be NULL
// (no timing).
// With iota1 (WORDS == 2, digit word 0), word 1 is not read: each item's is its index within
// its segment.
// With key_span (digit word 0): the pass at shift 0 records the range of the nonzero keys
// there (key_span zeroed before it); a later pass whose digit, and every digit above it, is
// the same for all nonzero keys would move none of them and does nothing: its output arrays
// are not written, and the sorted arrays are the output of the last pass that ran (the
// caller finds which from the span).  Zero keys (entries with nothing to sort for) may then
// stand elsewhere than a full sort would put them; the order of the nonzero keys is that of
// the full sort.
template <int WORDS>
cudaError_t radix_pass(xg_frame* f, const SortArrays<WORDS>& arr, int digit_word, int shift, uint32_t mask,
                       const SortGeom& geom, DevStatus* status, uint32_t* hist, cudaStream_t st,
                       bool iota1 = false, uint32_t* key_span = nullptr);
// Sets the scatter kernels' shared-memory attributes (once per process); call outside
// stream capture before the first radix_pass.
cudaError_t radix_prepare();
}  // namespace xg

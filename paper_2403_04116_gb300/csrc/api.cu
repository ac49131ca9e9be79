// Host side of the C ABI declared in include/xg.h: argument checks, workspace layout, the
// FP32 camera table built from the scanner parameters (Sec. 3.3, Eq. 12), and the
// stream-ordered launches of each stage.
#include <algorithm>
#include <atomic>
#include <math.h>
#include <nvtx3/nvToolsExt.h>
#include <stdlib.h>
#include <string.h>

#include "xg_internal.cuh"

namespace xg {

int device_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
  if (dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

}  // namespace xg

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kMaxBlockSmem = 227 * 1024;  // dynamic shared memory one block may use

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool valid_tile(int t) { return t == 8 || t == 16 || t == 32; }

bool valid_batch(int b) { return b == 0 || b == 64 || b == 128 || b == 256 || b == 512; }

bool valid_config(const xg_config* cfg) {
  if (!cfg) return false;
  const int ppt = cfg->pixels_per_thread == 0 ? 2 : cfg->pixels_per_thread;
  return (ppt == 1 || ppt == 2 || ppt == 4) && valid_tile(cfg->tile_w) && valid_tile(cfg->tile_h) &&
         cfg->tile_h % (4 * ppt) == 0 && cfg->tile_w * cfg->tile_h <= 512 * ppt && valid_batch(cfg->batch) &&
         (cfg->persistent == 0 || cfg->persistent == 1) && xg::render_smem_bytes(cfg) <= kMaxBlockSmem &&
         isfinite(cfg->near_mm) && cfg->near_mm > 0.f && cfg->pair_capacity >= 1 &&
         cfg->pair_capacity < ((int64_t)1 << 31) && cfg->views_per_pass >= 0;
}

// Views rendered per pass: all of them unless the configuration asks for fewer.
int32_t pass_views(const xg_config* cfg, int32_t n_views) {
  return cfg->views_per_pass > 0 && cfg->views_per_pass < n_views ? cfg->views_per_pass : n_views;
}

bool valid_sizes(int64_t n, int32_t n_views, int32_t per_pass, int32_t W, int32_t H) {
  return n >= 1 && n < ((int64_t)1 << 31) && n_views >= 1 && n_views <= xg::kMaxViews && W >= 1 && W <= 4096 &&
         H >= 1 && H <= 4096 && (int64_t)per_pass * n < ((int64_t)1 << 40);
}

struct Sizes {
  int32_t tiles_x, tiles_y;
  int64_t tiles_per_view;
  int32_t tile_bits;   // bits of a tile index within its view: pair key = view << tile_bits | tile
  int64_t range_keys;  // n_views << tile_bits
  int32_t entry_passes;
  int32_t bin_unit, bin_units, bin_rows, bin_groups;  // E, J, R, G of the pair scatter
};

bool sizes_of(const xg_config* cfg, int64_t n, int64_t n_views, int32_t W, int32_t H, int sms, Sizes* s) {
  s->tiles_x = (W + cfg->tile_w - 1) / cfg->tile_w;
  s->tiles_y = (H + cfg->tile_h - 1) / cfg->tile_h;
  s->tiles_per_view = (int64_t)s->tiles_x * s->tiles_y;
  int bits = 0;
  while (((int64_t)1 << bits) < s->tiles_per_view) ++bits;
  s->range_keys = n_views << bits;
  if (s->range_keys >= ((int64_t)1 << 31)) return false;
  s->tile_bits = bits;
  s->entry_passes = 4;
  // Pair scatter: groups of at most kBinGroupTiles tiles (whole rows), and units of sorted
  // entries sized for about 16 CTAs (unit, group) per SM, fewer where the per-(unit, tile)
  // counts would pass 2^24 words; every unit lies inside one view.
  const int64_t T = s->tiles_per_view;
  s->bin_rows = std::max(1, std::min(s->tiles_y, xg::kBinGroupTiles / s->tiles_x));
  s->bin_groups = (s->tiles_y + s->bin_rows - 1) / s->bin_rows;
  const int64_t target = ((int64_t)sms * 16 + s->bin_groups - 1) / s->bin_groups;
  const int64_t units = std::max<int64_t>(n_views, std::min<int64_t>(target, ((int64_t)1 << 24) / T));
  int64_t E = (n_views * n + units - 1) / units;
  E = std::max<int64_t>(256, (E + 255) / 256 * 256);
  if (E >= ((int64_t)1 << 31)) return false;
  s->bin_unit = (int32_t)E;
  s->bin_units = (int32_t)((n + E - 1) / E);
  return true;
}

// Byte offsets of every array in the workspace, public and private, in allocation order.
struct Offsets {
  size_t status, cameras, records, depth, rect, count;
  size_t ent_depth[2], ent_gid[2], value, hist, key_span, bin_hist, bin_total, range, order, order_base, tfinal, last, grad2d;
  size_t total;
};

// Per-pass arrays are sized for V views; the camera table holds all n_scan views.
bool make_offsets(const xg_config* cfg, int64_t n, int32_t V, int32_t n_scan, int32_t W, int32_t H, int sms,
                  Sizes* s, Offsets* o) {
  if (!sizes_of(cfg, n, V, W, H, sms, s)) return false;
  const size_t sort_blocks = (size_t)std::min(xg::kSortCtasPerSM * sms, xg::kMaxSortBlocks);
  const size_t VN = (size_t)V * (size_t)n;
  const size_t cap = (size_t)cfg->pair_capacity;
  const size_t pix = (size_t)V * (size_t)W * (size_t)H;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  o->status = take(sizeof(xg::DevStatus));
  o->cameras = take(sizeof(xg::Camera) * (size_t)n_scan);
  o->records = take(32 * VN);
  o->depth = take(4 * VN);
  o->rect = take(8 * VN);
  o->count = take(4 * VN);
  for (int b = 0; b < 2; ++b) o->ent_depth[b] = take(4 * VN);
  for (int b = 0; b < 2; ++b) o->ent_gid[b] = take(4 * VN);
  o->value = take(4 * cap);
  // radix blocks of a pass of V' <= V views: V' * ceil(sort_blocks / V') < sort_blocks + V'
  o->hist = take(4 * 256 * (sort_blocks + (size_t)V + 1) + 8);
  o->key_span = o->hist + 4 * 256 * (sort_blocks + (size_t)V + 1);  // two words after the histograms
  o->bin_hist = take(4 * (size_t)V * (size_t)s->bin_units * (size_t)s->tiles_per_view);
  o->bin_total = take(4 * (size_t)V * (size_t)s->tiles_per_view);
  o->range = take(8 * (size_t)s->range_keys);
  o->order = take(4 * (size_t)V * (size_t)s->tiles_per_view);
  o->order_base = take(4 * (size_t)xg::kOrderBuckets);
  o->tfinal = take(4 * pix);
  o->last = take(4 * pix);
  o->grad2d = take(4 * 8 * VN);
  o->total = off;
  return true;
}

bool valid_view(const xg_view& w) {
  return isfinite(w.sod_mm) && w.sod_mm > 0 && isfinite(w.sdd_mm) && w.sdd_mm > 0 && isfinite(w.pitch_u_mm) &&
         w.pitch_u_mm > 0 && isfinite(w.pitch_v_mm) && w.pitch_v_mm > 0 && isfinite(w.angle_rad);
}

// Camera table of the frame's views (trigonometry in FP64, rounded once to FP32), copied to
// the workspace on `st`; the host staging buffer may be freed when the copy call returns.
cudaError_t upload_cameras(const xg_frame* f, const xg_view* views, cudaStream_t st) {
  xg::Camera* cams = (xg::Camera*)calloc((size_t)f->n_scan, sizeof(xg::Camera));
  if (!cams) return cudaErrorMemoryAllocation;
  for (int32_t v = 0; v < f->n_scan; ++v) {
    const xg_view& w = views[v];
    xg::Camera& c = cams[v];
    c.c = (float)cos(w.angle_rad);
    c.s = (float)sin(w.angle_rad);
    c.L = (float)w.sod_mm;
    c.fu = (float)(w.sdd_mm / w.pitch_u_mm);
    c.fv = (float)(w.sdd_mm / w.pitch_v_mm);
    c.hw = (float)f->width * 0.5f - 0.5f;
    c.hh = (float)f->height * 0.5f - 0.5f;
  }
  const cudaError_t e =
      cudaMemcpyAsync(f->cam_all, cams, sizeof(xg::Camera) * (size_t)f->n_scan, cudaMemcpyHostToDevice, st);
  free(cams);  // pageable source: the copy has been staged when cudaMemcpyAsync returns
  return e;
}

__global__ void k_iota(uint32_t* __restrict__ a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (uint32_t)i;
}

__global__ void k_copy_status(const xg::DevStatus* __restrict__ s, xg_device_status* __restrict__ out) {
  out->code = s->code;
  out->reserved = 0;
  out->pairs = s->pairs;
  out->nonfinite = (int64_t)s->nonfinite;
  out->fwd_evaluated = (int64_t)s->fwd_evaluated;
  out->fwd_contrib = (int64_t)s->fwd_contrib;
  out->bwd_evaluated = (int64_t)s->bwd_evaluated;
  out->bwd_contrib = (int64_t)s->bwd_contrib;
}

// An NVTX range around one C-ABI stage call (host side: it marks the enqueueing).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

}  // namespace

namespace xg {
Timed::Timed(xg_frame* frame, int kid, cudaStream_t stream) : f(frame), st(stream), slot(-1) {
  if (!f || !f->timing) return;
  if (f->nrec >= kMaxTimingRecs) {
    ++f->dropped;
    return;
  }
  slot = f->nrec++;
  f->recs[slot].kid = kid;
  cudaEventRecord(f->recs[slot].a, st);
}
Timed::~Timed() {
  if (slot >= 0) cudaEventRecord(f->recs[slot].b, st);
}
}  // namespace xg

extern "C" {

size_t xg_workspace_bytes(const xg_config* cfg, int64_t n, int32_t n_views, int32_t width, int32_t height) {
  if (!valid_config(cfg) || n_views < 1) return 0;
  const int32_t per_pass = pass_views(cfg, n_views);
  if (!valid_sizes(n, n_views, per_pass, width, height)) return 0;
  Sizes s;
  Offsets o;
  return make_offsets(cfg, n, per_pass, n_views, width, height, xg::device_sms(), &s, &o) ? o.total : 0;
}

xg_status xg_frame_create(xg_frame** out, const xg_config* cfg, int64_t n, const xg_view* views, int32_t n_views,
                          void* workspace, size_t workspace_bytes, void* stream) {
  if (!out) return XG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!valid_config(cfg) || !views || n_views < 1) return XG_ERR_INVALID_ARG;
  const int32_t W = views[0].width, H = views[0].height;
  const int32_t per_pass = pass_views(cfg, n_views);
  if (!valid_sizes(n, n_views, per_pass, W, H)) return XG_ERR_INVALID_ARG;
  for (int32_t v = 0; v < n_views; ++v) {
    const xg_view& w = views[v];
    if (w.width != W || w.height != H || !valid_view(w)) return XG_ERR_INVALID_ARG;
  }
  Sizes s;
  Offsets o;
  const int sms = xg::device_sms();
  if (!make_offsets(cfg, n, per_pass, n_views, W, H, sms, &s, &o)) return XG_ERR_INVALID_ARG;
  if (!workspace || ((uintptr_t)workspace % kAlign) != 0 || workspace_bytes < o.total) return XG_ERR_WORKSPACE;

  xg_frame* f = (xg_frame*)calloc(1, sizeof(xg_frame));
  if (!f) return XG_ERR_INVALID_ARG;
  f->cfg = *cfg;
  if (f->cfg.batch == 0) f->cfg.batch = 64;
  if (f->cfg.pixels_per_thread == 0) f->cfg.pixels_per_thread = 2;
  f->cfg.views_per_pass = per_pass;
  f->n = n;
  f->n_scan = n_views;
  f->views_per_pass = per_pass;
  f->first_view = 0;
  f->n_views = per_pass;
  f->width = W;
  f->height = H;
  f->tiles_x = s.tiles_x;
  f->tiles_y = s.tiles_y;
  f->tiles_per_view = s.tiles_per_view;
  f->tile_bits = s.tile_bits;
  f->range_keys = s.range_keys;
  f->entry_passes = s.entry_passes;
  f->bin_unit = s.bin_unit;
  f->bin_units = s.bin_units;
  f->bin_rows = s.bin_rows;
  f->bin_groups = s.bin_groups;
  f->sort_blocks = std::min(xg::kSortCtasPerSM * sms, xg::kMaxSortBlocks);
  f->workspace = workspace;
  f->workspace_bytes = workspace_bytes;

  char* base = (char*)workspace;
  xg::FramePtrs& p = f->p;
  p.status = (xg::DevStatus*)(base + o.status);
  f->cam_all = (xg::Camera*)(base + o.cameras);
  p.cam = f->cam_all;
  p.rec = (float4*)(base + o.records);
  p.depth = (float*)(base + o.depth);
  p.rect = (ushort4*)(base + o.rect);
  p.count = (uint32_t*)(base + o.count);
  for (int k = 0; k < 2; ++k) {
    p.ent_depth[k] = (uint32_t*)(base + o.ent_depth[k]);
    p.ent_gid[k] = (uint32_t*)(base + o.ent_gid[k]);
  }
  p.value = (uint32_t*)(base + o.value);
  p.hist = (uint32_t*)(base + o.hist);
  p.key_span = (uint32_t*)(base + o.key_span);
  p.bin_hist = (uint32_t*)(base + o.bin_hist);
  p.bin_total = (uint32_t*)(base + o.bin_total);
  p.range = (uint2*)(base + o.range);
  p.order = (uint32_t*)(base + o.order);
  p.order_base = (uint32_t*)(base + o.order_base);
  p.tfinal = (float*)(base + o.tfinal);
  p.last = (uint32_t*)(base + o.last);
  p.grad2d = (float*)(base + o.grad2d);

  xg_layout& L = f->layout;
  L.status = o.status;
  L.cameras = o.cameras;
  L.records = o.records;
  L.depth = o.depth;
  L.rect = o.rect;
  L.count = o.count;
  L.value = o.value;
  L.range = o.range;
  L.tfinal = o.tfinal;
  L.last = o.last;
  L.grad2d = o.grad2d;
  L.order = o.order;
  L.tiles_per_view = s.tiles_per_view;
  L.tiles_x = s.tiles_x;
  L.tiles_y = s.tiles_y;
  L.sort_passes = s.entry_passes;
  L.range_stride = 1 << s.tile_bits;

  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = xg::radix_prepare();  // kernel attributes, set outside any stream capture
  if (e == cudaSuccess) e = xg::render_prepare(f);
  if (e == cudaSuccess) e = upload_cameras(f, views, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.status, 0, sizeof(xg::DevStatus), st);
  if (e == cudaSuccess) {  // the work order before any binning: every (view, tile) once
    const int64_t items = (int64_t)per_pass * s.tiles_per_view;
    k_iota<<<(unsigned)std::min<int64_t>((items + 255) / 256, 4096), 256, 0, st>>>(p.order, items);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    free(f);
    return XG_ERR_CUDA;
  }
  *out = f;
  return XG_OK;
}

xg_status xg_frame_select_views(xg_frame* frame, int32_t first_view, int32_t* n_selected) {
  if (!frame || first_view < 0 || first_view >= frame->n_scan) return XG_ERR_INVALID_ARG;
  const int32_t left = frame->n_scan - first_view;
  frame->first_view = first_view;
  frame->n_views = left < frame->views_per_pass ? left : frame->views_per_pass;
  frame->p.cam = frame->cam_all + first_view;
  if (n_selected) *n_selected = frame->n_views;
  return XG_OK;
}

void xg_frame_destroy(xg_frame* frame) {
  if (!frame) return;
  if (frame->recs) {
    for (int i = 0; i < xg::kMaxTimingRecs; ++i) {
      cudaEventDestroy(frame->recs[i].a);
      cudaEventDestroy(frame->recs[i].b);
    }
    free(frame->recs);
  }
  free(frame);
}

xg_status xg_frame_set_timing(xg_frame* frame, int32_t enable) {
  if (!frame) return XG_ERR_INVALID_ARG;
  if (enable && !frame->recs) {
    xg::TimingRec* recs = (xg::TimingRec*)calloc(xg::kMaxTimingRecs, sizeof(xg::TimingRec));
    if (!recs) return XG_ERR_INVALID_ARG;
    for (int i = 0; i < xg::kMaxTimingRecs; ++i) {
      if (cudaEventCreate(&recs[i].a) != cudaSuccess || cudaEventCreate(&recs[i].b) != cudaSuccess) {
        for (int j = 0; j <= i; ++j) {
          if (recs[j].a) cudaEventDestroy(recs[j].a);
          if (recs[j].b) cudaEventDestroy(recs[j].b);
        }
        free(recs);
        return XG_ERR_CUDA;
      }
    }
    frame->recs = recs;
  }
  frame->timing = enable ? 1 : 0;
  return XG_OK;
}

xg_status xg_frame_read_timing(xg_frame* frame, xg_kernel_time* out, int32_t capacity, int32_t* count) {
  static const char* const names[xg::kNumKernels] = {
      "k_project", "k_bin_count", "k_bin_colscan", "k_bin_base", "k_bin_scatter", "k_radix_hist", "k_radix_colscan",
      "k_radix_scatter", "k_work_order", "k_render_fwd", "k_render_bwd", "k_project_bwd", "memset"};
  if (!frame || !count || (capacity > 0 && !out)) return XG_ERR_INVALID_ARG;
  if (frame->nrec > 0) {
    if (cudaEventSynchronize(frame->recs[frame->nrec - 1].b) != cudaSuccess) return XG_ERR_CUDA;
    for (int i = 0; i < frame->nrec; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, frame->recs[i].a, frame->recs[i].b) != cudaSuccess) return XG_ERR_CUDA;
      frame->acc_ms[frame->recs[i].kid] += ms;
      frame->acc_n[frame->recs[i].kid] += 1;
    }
  }
  int32_t k = 0;
  for (int kid = 0; kid < xg::kNumKernels; ++kid) {
    if (!frame->acc_n[kid]) continue;
    if (k < capacity) {
      memset(out[k].name, 0, sizeof out[k].name);
      strncpy(out[k].name, names[kid], sizeof out[k].name - 1);
      out[k].launches = frame->acc_n[kid];
      out[k].total_ms = frame->acc_ms[kid];
    }
    ++k;
  }
  *count = k < capacity ? k : capacity;
  frame->nrec = 0;
  frame->dropped = 0;
  memset(frame->acc_ms, 0, sizeof frame->acc_ms);
  memset(frame->acc_n, 0, sizeof frame->acc_n);
  return XG_OK;
}

xg_status xg_loss_l1(const float* image, const float* target, int64_t count, float scale, float* grad, float* loss,
                     void* stream) {
  if (!image || !target || !grad || !loss || count < 1) return XG_ERR_INVALID_ARG;
  return xg::launch_loss_l1(image, target, count, scale, grad, loss, (cudaStream_t)stream) == cudaSuccess
             ? XG_OK
             : XG_ERR_CUDA;
}

xg_status xg_exp_check(const float* x, float* y_scalar, float* y_packed, int64_t n, void* stream) {
  if (!x || !y_scalar || !y_packed || n < 1 || n > ((int64_t)1 << 38)) return XG_ERR_INVALID_ARG;
  return xg::launch_exp_check(x, y_scalar, y_packed, n, (cudaStream_t)stream) == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

static bool valid_gaussians(const xg_frame* f, const xg_gaussians* g) {
  return g && g->n == f->n && g->mean && g->scale && g->quat && g->opacity && g->intensity;
}

xg_status xg_project(xg_frame* frame, const xg_gaussians* g, void* stream) {
  const Range range("xg_project");
  if (!frame || !valid_gaussians(frame, g)) return XG_ERR_INVALID_ARG;
  return xg::launch_project(frame, g, (cudaStream_t)stream) == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

xg_status xg_bin_sort(xg_frame* frame, void* stream) {
  const Range range("xg_bin_sort");
  if (!frame) return XG_ERR_INVALID_ARG;
  return xg::launch_bin_sort(frame, (cudaStream_t)stream) == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

xg_status xg_render_fwd(xg_frame* frame, float* image, uint32_t* n_contrib, void* stream) {
  const Range range("xg_render_fwd");
  if (!frame || !image) return XG_ERR_INVALID_ARG;
  return xg::launch_render_fwd(frame, image, n_contrib, (cudaStream_t)stream) == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

xg_status xg_render_bwd(xg_frame* frame, const xg_gaussians* g, const float* grad_image, const xg_grads* out,
                        void* stream) {
  const Range range("xg_render_bwd");
  if (!frame || !valid_gaussians(frame, g) || !grad_image || !out || !out->mean || !out->scale || !out->quat ||
      !out->opacity || !out->intensity)
    return XG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (xg::launch_render_bwd(frame, grad_image, st) != cudaSuccess) return XG_ERR_CUDA;
  return xg::launch_project_bwd(frame, g, out, st) == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

xg_status xg_frame_read_status(const xg_frame* frame, xg_device_status* out, void* stream) {
  if (!frame || !out) return XG_ERR_INVALID_ARG;
  xg::DevStatus s;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&s, frame->p.status, sizeof s, cudaMemcpyDeviceToHost, st) != cudaSuccess) return XG_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return XG_ERR_CUDA;
  out->code = s.code;
  out->reserved = 0;
  out->pairs = s.pairs;
  out->nonfinite = (int64_t)s.nonfinite;
  out->fwd_evaluated = (int64_t)s.fwd_evaluated;
  out->fwd_contrib = (int64_t)s.fwd_contrib;
  out->bwd_evaluated = (int64_t)s.bwd_evaluated;
  out->bwd_contrib = (int64_t)s.bwd_contrib;
  return XG_OK;
}

xg_status xg_frame_copy_status(const xg_frame* frame, xg_device_status* out, void* stream) {
  if (!frame || !out || ((uintptr_t)out % 8) != 0) return XG_ERR_INVALID_ARG;
  k_copy_status<<<1, 1, 0, (cudaStream_t)stream>>>(frame->p.status, out);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

xg_status xg_frame_layout(const xg_frame* frame, xg_layout* out) {
  if (!frame || !out) return XG_ERR_INVALID_ARG;
  *out = frame->layout;
  return XG_OK;
}

const char* xg_status_str(xg_status s) {
  switch (s) {
    case XG_OK: return "ok";
    case XG_ERR_INVALID_ARG: return "invalid argument";
    case XG_ERR_CAPACITY: return "pair capacity exceeded";
    case XG_ERR_CUDA: return "CUDA error";
    case XG_ERR_WORKSPACE: return "workspace too small or misaligned";
    case XG_ERR_CHECK: return "device-side bounds check failed";
  }
  return "unknown status";
}

}  // extern "C"

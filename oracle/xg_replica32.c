/*
 * FP32 replica of the culling test, tile assignment, depth order and per-pixel blending
 * decisions of X-Gaussian's rasterizer (arXiv 2403.04116, Sec. 3.2, Eq. 7-10).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline call this file.  It shares no code with the CUDA library; it is a second,
 * independent implementation of the same documented FP32 operation sequence (every
 * operation IEEE round-to-nearest; fused multiply-adds only where written as fmaf; built
 * with -ffp-contract=off), so tile ids, sort keys, tile ranges, contributor counts and the
 * last-contributor positions must match the GPU bit for bit.  Its own correctness is
 * pinned against the FP64 oracle and against brute-force checks in the tests.
 *
 * Transcendentals used in a decision are computed here from basic operations:
 *   exp: k = the integer nearest x log2 e (from one fused multiply-add), Cody-Waite
 *        reduction by ln 2 (split into its float rounding and the float of the remainder),
 *        then the degree-6 Taylor polynomial of e^r, |r| <= ln2/2, scaled by 2^k;
 *   log: x = m 2^e with m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh((m-1)/(m+1)) by its odd
 *        series to s^9, plus e ln 2.
 * Readings of the paper used here: focal in pixels L_SD / pitch; pixel centres at
 * (x + 1/2, y + 1/2) with the principal point at (W/2, H/2), coordinates stored centred on
 * the principal point; 0.3 px^2 dilation of Sigma''; near plane; sigma = min(0.99, o e^p)
 * with sigma < 1/255 skipped; stop before T would drop below 1e-4; the tile footprint
 * radius sqrt(2 ln(255 o) lambda_max) (1 + 2^-10), which contains every pixel where sigma
 * can reach 1/255.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double sod, sdd, pitch_u, pitch_v, angle;
  int32_t width, height;
} xr_view;

#define LN2_D 0.69314718055994530942
static const float R_L2E = (float)1.44269504088896340736;
static const float R_LN2_HI = (float)LN2_D;
#define R_LN2_LO ((float)(LN2_D - (double)(float)LN2_D))
static const float R_SQRT2 = (float)1.41421356237309504880;
static const float R_ALPHA_MIN = (float)(1.0 / 255.0);
static const float R_ALPHA_MAX = 0.99f;
static const float R_T_MIN = 1e-4f;
static const float R_DILATE = 0.3f;
static const float R_RMARGIN = 1.0009765625f; /* 1 + 2^-10 */

static float bits_f(uint32_t b) {
  float f;
  memcpy(&f, &b, 4);
  return f;
}
static uint32_t f_bits(float f) {
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
}

float xr_exp(float x) {
  x = fmaxf(x, -80.0f);
  /* k: the integer nearest x log2 e (ties to even), rounded once from the exact product:
   * x log2 e + 1.5 * 2^23 in one fmaf keeps it in the last mantissa bits */
  float k = fmaf(x, R_L2E, 12582912.0f) - 12582912.0f;
  float r = fmaf(k, -R_LN2_HI, x);
  r = fmaf(k, -R_LN2_LO, r);
  float p = fmaf(r, (float)(1.0 / 720.0), (float)(1.0 / 120.0));
  p = fmaf(p, r, (float)(1.0 / 24.0));
  p = fmaf(p, r, (float)(1.0 / 6.0));
  p = fmaf(p, r, 0.5f);
  p = fmaf(p, r, 1.0f);
  p = fmaf(p, r, 1.0f);
  int ki = (int)k;
  return p * bits_f((uint32_t)(ki + 127) << 23);
}

/* natural log for finite x >= 1 */
float xr_log(float x) {
  uint32_t b = f_bits(x);
  int e = (int)(b >> 23) - 127;
  float m = bits_f((b & 0x7fffffu) | 0x3f800000u);
  if (m > R_SQRT2) {
    m = m * 0.5f;
    e += 1;
  }
  float s = (m - 1.0f) / (m + 1.0f);
  float s2 = s * s;
  float p = fmaf(s2, (float)(2.0 / 9.0), (float)(2.0 / 7.0));
  p = fmaf(p, s2, (float)(2.0 / 5.0));
  p = fmaf(p, s2, (float)(2.0 / 3.0));
  p = fmaf(p, s2, 2.0f);
  p = p * s;
  float ef = (float)e;
  float t = fmaf(ef, R_LN2_LO, p);
  return fmaf(ef, R_LN2_HI, t);
}

static int all_finite(const float* v, int k) {
  for (int i = 0; i < k; ++i)
    if (!isfinite(v[i])) return 0;
  return 1;
}

/*
 * Projection of every Gaussian under one view.
 *   rec[8n]: (u_x, u_y, -a/2, -b, -c/2 of the conic (a, b, c), opacity, intensity,
 *   -ln(255 opacity) - 1e-4), u centred on
 *   the principal point; the last field is the exponent below which sigma stays under 1/255
 *   with a margin (a skip test that never changes a decision)
 *   depth[n]: t_z;  rect[4n]: tile rectangle (x0, y0, x1, y1), inclusive;  count[n]: tiles touched
 * Everything is zero where count is zero.  Returns the number of Gaussians with a
 * non-finite attribute.
 */
int64_t xr_project(int64_t n, const float* mean, const float* scale, const float* quat, const float* opac,
                   const float* inten, const xr_view* v, float near_mm, int tile_w, int tile_h, float* rec,
                   float* depth, int32_t* rect, uint32_t* count) {
  const float s = (float)sin(v->angle), c = (float)cos(v->angle);
  const float L = (float)v->sod, fu = (float)(v->sdd / v->pitch_u), fv = (float)(v->sdd / v->pitch_v);
  const int W = v->width, H = v->height;
  const float hw = (float)W * 0.5f - 0.5f, hh = (float)H * 0.5f - 0.5f;
  int64_t nonfinite = 0;
  for (int64_t g = 0; g < n; ++g) {
    float* rg = rec + 8 * g;
    memset(rg, 0, 8 * sizeof(float));
    depth[g] = 0.0f;
    rect[4 * g + 0] = rect[4 * g + 1] = rect[4 * g + 2] = rect[4 * g + 3] = 0;
    count[g] = 0;
    float a[12] = {mean[g],         mean[n + g],     mean[2 * n + g], scale[g],
                   scale[n + g],    scale[2 * n + g], quat[g],        quat[n + g],
                   quat[2 * n + g], quat[3 * n + g], opac[g],        inten[g]};
    if (!all_finite(a, 12)) {
      ++nonfinite;
      continue;
    }
    float mx = a[0], my = a[1], mz = a[2], sx = a[3], sy = a[4], sz = a[5];
    float qw = a[6], qx = a[7], qy = a[8], qz = a[9], o = a[10], in = a[11];
    float qq = qw * qw;
    qq = fmaf(qx, qx, qq);
    qq = fmaf(qy, qy, qq);
    qq = fmaf(qz, qz, qq);
    if (!(qq > 0.0f)) continue;
    float inv = 1.0f / sqrtf(qq);
    float w = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float t;
    float R[3][3];
    t = yy + zz;
    R[0][0] = 1.0f - (t + t);
    t = xy - wz;
    R[0][1] = t + t;
    t = xz + wy;
    R[0][2] = t + t;
    t = xy + wz;
    R[1][0] = t + t;
    t = xx + zz;
    R[1][1] = 1.0f - (t + t);
    t = yz - wx;
    R[1][2] = t + t;
    t = xz - wy;
    R[2][0] = t + t;
    t = yz + wx;
    R[2][1] = t + t;
    t = xx + yy;
    R[2][2] = 1.0f - (t + t);
    float sc[3] = {sx, sy, sz};
    float M[3][3];
    for (int r = 0; r < 3; ++r)
      for (int k = 0; k < 3; ++k) M[r][k] = R[r][k] * sc[k];
    float S00 = fmaf(M[0][2], M[0][2], fmaf(M[0][1], M[0][1], M[0][0] * M[0][0]));
    float S01 = fmaf(M[0][2], M[1][2], fmaf(M[0][1], M[1][1], M[0][0] * M[1][0]));
    float S02 = fmaf(M[0][2], M[2][2], fmaf(M[0][1], M[2][1], M[0][0] * M[2][0]));
    float S11 = fmaf(M[1][2], M[1][2], fmaf(M[1][1], M[1][1], M[1][0] * M[1][0]));
    float S12 = fmaf(M[1][2], M[2][2], fmaf(M[1][1], M[2][1], M[1][0] * M[2][0]));
    float S22 = fmaf(M[2][2], M[2][2], fmaf(M[2][1], M[2][1], M[2][0] * M[2][0]));

    float tx = fmaf(c, my, (-s) * mx);
    float ty = -mz;
    float tz = fmaf(-s, my, (-c) * mx) + L;
    if (!(tz > near_mm)) continue;
    float iz = 1.0f / tz;
    float ax = tx * iz, ay = ty * iz;
    float ux = fu * ax, uy = fv * ay;
    /* rows of J W without the focal factors: v0 = W0 - ax W2, v1 = W1 - ay W2 */
    float v0x = fmaf(ax, c, -s), v0y = fmaf(ax, s, c);
    float v1x = ay * c, v1y = ay * s; /* v1z = -1 */
    float w00 = fmaf(S01, v0y, S00 * v0x);
    float w01 = fmaf(S11, v0y, S01 * v0x);
    float w02 = fmaf(S12, v0y, S02 * v0x);
    float q00 = fmaf(v0y, w01, v0x * w00);
    float q01 = fmaf(v1y, w01, v1x * w00) - w02;
    float w10 = fmaf(S01, v1y, S00 * v1x) - S02;
    float w11 = fmaf(S11, v1y, S01 * v1x) - S12;
    float w12 = fmaf(S12, v1y, S02 * v1x) - S22;
    float q11 = fmaf(v1y, w11, v1x * w10) - w12;
    float gu = fu * iz, gv = fv * iz;
    float A = fmaf(gu * gu, q00, R_DILATE);
    float B = (gu * gv) * q01;
    float C = fmaf(gv * gv, q11, R_DILATE);
    float det = fmaf(A, C, -(B * B));
    if (!(det > 0.0f)) continue;
    float idet = 1.0f / det;
    float ca = C * idet, cb = -(B * idet), cc = A * idet;
    if (!(o >= R_ALPHA_MIN)) continue;
    float mid = 0.5f * (A + C);
    float disc = fmaf(mid, mid, -det);
    float lam = mid + sqrtf(fmaxf(disc, 0.1f));
    float lg = xr_log(255.0f * o);
    float rad = sqrtf((lg + lg) * lam) * R_RMARGIN;
    float cx = ux + hw, cy = uy + hh;
    if (!(isfinite(rad) && isfinite(cx) && isfinite(cy))) continue;
    float x0 = fmaxf(ceilf(cx - rad), 0.0f), x1 = fminf(floorf(cx + rad), (float)(W - 1));
    float y0 = fmaxf(ceilf(cy - rad), 0.0f), y1 = fminf(floorf(cy + rad), (float)(H - 1));
    if (!(x0 <= x1 && y0 <= y1)) continue;
    int tx0 = (int)x0 / tile_w, tx1 = (int)x1 / tile_w, ty0 = (int)y0 / tile_h, ty1 = (int)y1 / tile_h;
    rg[0] = ux;
    rg[1] = uy;
    rg[2] = -0.5f * ca; /* the exponent's coefficients (-a/2, -b, -c/2) */
    rg[3] = -cb;
    rg[4] = -0.5f * cc;
    rg[5] = o;
    rg[6] = in;
    rg[7] = -lg - 1e-4f; /* exponent below which sigma < 1/255 for sure (the kernels' skip test) */
    depth[g] = tz;
    rect[4 * g + 0] = tx0;
    rect[4 * g + 1] = ty0;
    rect[4 * g + 2] = tx1;
    rect[4 * g + 3] = ty1;
    count[g] = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
  }
  return nonfinite;
}

typedef struct {
  uint32_t dbits;
  int64_t id;
} xr_item;

static int item_cmp(const void* pa, const void* pb) {
  const xr_item* a = (const xr_item*)pa;
  const xr_item* b = (const xr_item*)pb;
  if (a->dbits != b->dbits) return a->dbits < b->dbits ? -1 : 1;
  return (a->id < b->id) ? -1 : (a->id > b->id);
}

/*
 * Per-tile lists of one view: list[] holds Gaussian indices tile after tile (tile id
 * row-major), each tile ordered by (bits of t_z, index); range[2t], range[2t+1] is the
 * tile's [start, end) in list, [0, 0) for an empty tile.  Returns the list length, or -1
 * when memory runs out.  list must hold sum(count) entries.
 */
int64_t xr_bin(int64_t n, const float* depth, const int32_t* rect, const uint32_t* count, int tiles_x,
               int tiles_y, uint32_t* range, int32_t* list) {
  int64_t T = (int64_t)tiles_x * tiles_y;
  int64_t* cnt = (int64_t*)calloc((size_t)T + 1, sizeof(int64_t));
  if (!cnt) return -1;
  for (int64_t g = 0; g < n; ++g) {
    if (!count[g]) continue;
    for (int ty = rect[4 * g + 1]; ty <= rect[4 * g + 3]; ++ty)
      for (int tx = rect[4 * g + 0]; tx <= rect[4 * g + 2]; ++tx) cnt[(int64_t)ty * tiles_x + tx + 1]++;
  }
  for (int64_t t = 0; t < T; ++t) cnt[t + 1] += cnt[t];
  int64_t M = cnt[T];
  xr_item* items = (xr_item*)malloc(sizeof(xr_item) * (size_t)(M > 0 ? M : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(T > 0 ? T : 1));
  if (!items || !fill) {
    free(cnt);
    free(items);
    free(fill);
    return -1;
  }
  memcpy(fill, cnt, sizeof(int64_t) * (size_t)T);
  for (int64_t g = 0; g < n; ++g) {
    if (!count[g]) continue;
    for (int ty = rect[4 * g + 1]; ty <= rect[4 * g + 3]; ++ty)
      for (int tx = rect[4 * g + 0]; tx <= rect[4 * g + 2]; ++tx) {
        int64_t t = (int64_t)ty * tiles_x + tx;
        xr_item it = {f_bits(depth[g]), g};
        items[fill[t]++] = it;
      }
  }
  for (int64_t t = 0; t < T; ++t) {
    qsort(items + cnt[t], (size_t)(cnt[t + 1] - cnt[t]), sizeof(xr_item), item_cmp);
    if (cnt[t + 1] > cnt[t]) {
      range[2 * t] = (uint32_t)cnt[t];
      range[2 * t + 1] = (uint32_t)cnt[t + 1];
    } else {
      range[2 * t] = range[2 * t + 1] = 0;
    }
  }
  for (int64_t k = 0; k < M; ++k) list[k] = (int32_t)items[k].id;
  free(items);
  free(fill);
  free(cnt);
  return M;
}

/*
 * Blend every pixel of one view from the tile lists (Eq. 10 with the thresholds above).
 * Outputs W*H arrays: image, transmittance after the last contributor, contributor
 * count, and the 1-based position within the tile list of the last contributor (0: none).
 */
void xr_render(const float* rec, const uint32_t* range, const int32_t* list, const xr_view* v, int tile_w,
               int tile_h, float* image, float* tfinal, uint32_t* ncontrib, uint32_t* last) {
  const int W = v->width, H = v->height;
  const int tiles_x = (W + tile_w - 1) / tile_w;
  const float hw = (float)W * 0.5f - 0.5f, hh = (float)H * 0.5f - 0.5f;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      int64_t t = (int64_t)(y / tile_h) * tiles_x + x / tile_w;
      uint32_t b = range[2 * t], e = range[2 * t + 1];
      float px = (float)x - hw, py = (float)y - hh;
      float T = 1.0f, C = 0.0f;
      uint32_t nc = 0, lst = 0;
      for (uint32_t k = b; k < e; ++k) {
        const float* r = rec + 8 * (int64_t)list[k];
        float na = r[2], nb = r[3], nc2 = r[4];
        float dx = r[0] - px, dy = r[1] - py;
        /* dx (na dx + nb dy) + (nc dy) dy */
        float t = fmaf(na, dx, nb * dy);
        float p = fmaf(dx, t, (nc2 * dy) * dy);
        float ex = xr_exp(p);
        float al = fminf(R_ALPHA_MAX, r[5] * ex);
        if (al < R_ALPHA_MIN) continue;
        float Tn = T * (1.0f - al);
        if (Tn < R_T_MIN) break;
        C = fmaf(r[6], al * T, C);
        T = Tn;
        ++nc;
        lst = k - b + 1;
      }
      int64_t p = (int64_t)y * W + x;
      image[p] = C;
      tfinal[p] = T;
      ncontrib[p] = nc;
      last[p] = lst;
    }
}

/* element-wise wrappers so the tests can pin the two transcendentals */
void xr_exp_batch(const float* x, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = xr_exp(x[i]);
}
void xr_log_batch(const float* x, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = xr_log(x[i]);
}

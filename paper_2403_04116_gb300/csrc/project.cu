// Projection of 3-D Gaussians into cone-beam views, and its backward pass.
//
// k_project: Sec. 3.1 (Sigma = R S S^T R^T), Eq. 7 (t = M_ext mu, u = M_int t), Eq. 8-9
// (Sigma' = J W Sigma W^T J^T) and the 2-D covariance Sigma'' of Sec. 3.2, then the tile
// rectangle of the footprint.  One thread per (Gaussian, view): the five attribute planes
// are read with unit-stride loads (structure of arrays), the per-view camera is a broadcast.
//
// k_project_bwd: the chain rule back from the per-(view, Gaussian) sums the compositing
// backward pass writes (moments of dL/dpower over the pixel offsets, and dL/dintensity):
// first to dL/du, dL/dconic and dL/dopacity of each view (written back in place of the
// sums), then to mean, scale, quaternion, opacity and intensity; eight threads per Gaussian
// (one per warp of a block) sum its views, each every eighth view.
#include "xg_internal.cuh"

namespace xg {

__global__ void __launch_bounds__(256) k_project(const float* __restrict__ mean, const float* __restrict__ scale,
                                                 const float* __restrict__ quat, const float* __restrict__ opac,
                                                 const float* __restrict__ inten, int64_t n,
                                                 const Camera* __restrict__ cams, int W, int H, int tw_shift, int th_shift,
                                                 float near_mm, float4* __restrict__ rec, float* __restrict__ depth,
                                                 ushort4* __restrict__ rect, uint32_t* __restrict__ count,
                                                 DevStatus* __restrict__ status) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const int v = blockIdx.y;
  const int64_t vg = (int64_t)v * n + g;

  float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = make_float4(0.f, 0.f, 0.f, 0.f);
  float dz = 0.f;
  ushort4 rc = make_ushort4(0, 0, 0, 0);
  uint32_t cnt = 0;

  const float mx = mean[g], my = mean[n + g], mz = mean[2 * n + g];
  const float sx = scale[g], sy = scale[n + g], sz = scale[2 * n + g];
  const float qw = quat[g], qx = quat[n + g], qy = quat[2 * n + g], qz = quat[3 * n + g];
  const float o = opac[g], in = inten[g];
  const bool finite = isfinite(mx) && isfinite(my) && isfinite(mz) && isfinite(sx) && isfinite(sy) &&
                      isfinite(sz) && isfinite(qw) && isfinite(qx) && isfinite(qy) && isfinite(qz) &&
                      isfinite(o) && isfinite(in);
  if (!finite && v == 0) atomicAdd(&status->nonfinite, 1ull);

  do {
    if (!finite) break;
    float qq = fmul(qw, qw);
    qq = ffma(qx, qx, qq);
    qq = ffma(qy, qy, qq);
    qq = ffma(qz, qz, qq);
    if (!(qq > 0.0f)) break;
    const float inv = fdiv(1.0f, fsqrt(qq));
    const float w = fmul(qw, inv), x = fmul(qx, inv), y = fmul(qy, inv), z = fmul(qz, inv);
    const float xx = fmul(x, x), yy = fmul(y, y), zz = fmul(z, z);
    const float xy = fmul(x, y), xz = fmul(x, z), yz = fmul(y, z);
    const float wx = fmul(w, x), wy = fmul(w, y), wz = fmul(w, z);
    float t;
    float R[3][3];
    t = fadd(yy, zz);
    R[0][0] = fsub(1.0f, fadd(t, t));
    t = fsub(xy, wz);
    R[0][1] = fadd(t, t);
    t = fadd(xz, wy);
    R[0][2] = fadd(t, t);
    t = fadd(xy, wz);
    R[1][0] = fadd(t, t);
    t = fadd(xx, zz);
    R[1][1] = fsub(1.0f, fadd(t, t));
    t = fsub(yz, wx);
    R[1][2] = fadd(t, t);
    t = fsub(xz, wy);
    R[2][0] = fadd(t, t);
    t = fadd(yz, wx);
    R[2][1] = fadd(t, t);
    t = fadd(xx, yy);
    R[2][2] = fsub(1.0f, fadd(t, t));
    const float sc[3] = {sx, sy, sz};
    float M[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) M[r][k] = fmul(R[r][k], sc[k]);
    const float S00 = ffma(M[0][2], M[0][2], ffma(M[0][1], M[0][1], fmul(M[0][0], M[0][0])));
    const float S01 = ffma(M[0][2], M[1][2], ffma(M[0][1], M[1][1], fmul(M[0][0], M[1][0])));
    const float S02 = ffma(M[0][2], M[2][2], ffma(M[0][1], M[2][1], fmul(M[0][0], M[2][0])));
    const float S11 = ffma(M[1][2], M[1][2], ffma(M[1][1], M[1][1], fmul(M[1][0], M[1][0])));
    const float S12 = ffma(M[1][2], M[2][2], ffma(M[1][1], M[2][1], fmul(M[1][0], M[2][0])));
    const float S22 = ffma(M[2][2], M[2][2], ffma(M[2][1], M[2][1], fmul(M[2][0], M[2][0])));

    const Camera cam = cams[v];
    const float c = cam.c, s = cam.s;
    const float tx = ffma(c, my, fmul(-s, mx));
    const float ty = -mz;
    const float tz = fadd(ffma(-s, my, fmul(-c, mx)), cam.L);
    if (!(tz > near_mm)) break;
    const float iz = fdiv(1.0f, tz);
    const float ax = fmul(tx, iz), ay = fmul(ty, iz);
    const float ux = fmul(cam.fu, ax), uy = fmul(cam.fv, ay);
    // rows of J W without the focal factors: v0 = W0 - ax W2, v1 = W1 - ay W2 (v0z = 0, v1z = -1)
    const float v0x = ffma(ax, c, -s), v0y = ffma(ax, s, c);
    const float v1x = fmul(ay, c), v1y = fmul(ay, s);
    const float w00 = ffma(S01, v0y, fmul(S00, v0x));
    const float w01 = ffma(S11, v0y, fmul(S01, v0x));
    const float w02 = ffma(S12, v0y, fmul(S02, v0x));
    const float q00 = ffma(v0y, w01, fmul(v0x, w00));
    const float q01 = fsub(ffma(v1y, w01, fmul(v1x, w00)), w02);
    const float w10 = fsub(ffma(S01, v1y, fmul(S00, v1x)), S02);
    const float w11 = fsub(ffma(S11, v1y, fmul(S01, v1x)), S12);
    const float w12 = fsub(ffma(S12, v1y, fmul(S02, v1x)), S22);
    const float q11 = fsub(ffma(v1y, w11, fmul(v1x, w10)), w12);
    const float gu = fmul(cam.fu, iz), gv = fmul(cam.fv, iz);
    const float A = ffma(fmul(gu, gu), q00, kDilate);
    const float B = fmul(fmul(gu, gv), q01);
    const float C = ffma(fmul(gv, gv), q11, kDilate);
    const float det = ffma(A, C, -fmul(B, B));
    if (!(det > 0.0f)) break;
    const float idet = fdiv(1.0f, det);
    const float ca = fmul(C, idet), cb = -fmul(B, idet), cc = fmul(A, idet);
    if (!(o >= kAlphaMin)) break;
    const float mid = fmul(0.5f, fadd(A, C));
    const float disc = ffma(mid, mid, -det);
    const float lam = fadd(mid, fsqrt(fmaxf(disc, 0.1f)));
    const float lg = xg_log_ge1(fmul(255.0f, o));
    const float rad = fmul(fsqrt(fmul(fadd(lg, lg), lam)), kRadiusMargin);
    const float cx = fadd(ux, cam.hw), cy = fadd(uy, cam.hh);
    if (!(isfinite(rad) && isfinite(cx) && isfinite(cy))) break;
    const float x0 = fmaxf(ceilf(fsub(cx, rad)), 0.0f), x1 = fminf(floorf(fadd(cx, rad)), (float)(W - 1));
    const float y0 = fmaxf(ceilf(fsub(cy, rad)), 0.0f), y1 = fminf(floorf(fadd(cy, rad)), (float)(H - 1));
    if (!(x0 <= x1 && y0 <= y1)) break;
    // tile sizes are powers of two (8, 16 or 32) and the pixel indices non-negative
    const int tx0 = (int)x0 >> tw_shift, tx1 = (int)x1 >> tw_shift, ty0 = (int)y0 >> th_shift,
              ty1 = (int)y1 >> th_shift;
    // the exponent's coefficients: power = na dx^2 + nb dx dy + nc dy^2 with
    // (na, nb, nc) = (-a/2, -b, -c/2) of the conic (a, b, c) (exact halvings and negations)
    r0 = make_float4(ux, uy, fmul(-0.5f, ca), -cb);
    // the exponent below which the opacity stays under 1/255 for sure, with a margin far
    // above the error of the FP32 exp: the compositing kernels skip such pairs
    r1 = make_float4(fmul(-0.5f, cc), o, in, fsub(-lg, 1e-4f));
    dz = tz;
    rc = make_ushort4((unsigned short)tx0, (unsigned short)ty0, (unsigned short)tx1, (unsigned short)ty1);
    cnt = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
  } while (0);

  rec[2 * vg] = r0;
  rec[2 * vg + 1] = r1;
  depth[vg] = dz;
  rect[vg] = rc;
  count[vg] = cnt;
}

cudaError_t launch_project(xg_frame* f, const xg_gaussians* g, cudaStream_t st) {
  const int64_t n = f->n;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)f->n_views);
  Timed t(f, kProject, st);
  k_project<<<grid, 256, 0, st>>>(g->mean, g->scale, g->quat, g->opacity, g->intensity, n, f->p.cam, f->width,
                                  f->height, __builtin_ctz((unsigned)f->cfg.tile_w),
                                  __builtin_ctz((unsigned)f->cfg.tile_h), f->cfg.near_mm, f->p.rec, f->p.depth,
                                  f->p.rect, f->p.count, f->p.status);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// backward
// ------------------------------------------------------------------------------------------

// k_project_bwd: a block takes 32 Gaussians (one per lane) and its 8 warps split the views
// (warp w takes views w, w + 8, ...); the warps' partial sums meet in shared memory and
// warp 0 finishes the chain rule.  The kernel waits on its loads more than it computes, so
// it is compiled for 4 resident blocks per SM (64 registers).
constexpr int kPbGaussians = 32;
constexpr int kPbWarps = 8;

__global__ void __launch_bounds__(32 * kPbWarps, 4) k_project_bwd(const float* __restrict__ mean, const float* __restrict__ scale,
                                                     const float* __restrict__ quat, const float* __restrict__ opac,
                                                     int64_t n, int n_views,
                                                     const Camera* __restrict__ cams, float* __restrict__ g2d,
                                                     const DevStatus* __restrict__ status, float* __restrict__ g_mean,
                                                     float* __restrict__ g_scale, float* __restrict__ g_quat,
                                                     float* __restrict__ g_opac, float* __restrict__ g_inten) {
  // per warp and Gaussian: the partial sums over the warp's views (gS: 6 of the symmetric
  // 3x3, mean: 3, S_1, dL/dintensity), a padded column per Gaussian
  __shared__ float s_part[kPbWarps][11][kPbGaussians + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t g = (int64_t)blockIdx.x * kPbGaussians + lane;
  const bool live = g < n;
  float gm[3] = {0.f, 0.f, 0.f}, gsc[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
  float go = 0.f, gi = 0.f;
  float gSu[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dL/dSigma, upper triangle (symmetric)
  float s1 = 0.f;  // sum over views of S_1
  float w = 0.f, x = 0.f, y = 0.f, z = 0.f, inv = 0.f, R[3][3] = {}, M[3][3] = {};

  const int64_t gl = live ? g : 0;  // lanes past n load Gaussian 0 and store nothing
  const float mx = mean[gl], my = mean[n + gl], mz = mean[2 * n + gl];
  const float s3[3] = {scale[gl], scale[n + gl], scale[2 * n + gl]};
  const float q4[4] = {quat[gl], quat[n + gl], quat[2 * n + gl], quat[3 * n + gl]};
  const float qq = q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3];
  const bool usable = live && status->code == XG_OK && qq > 0.f && isfinite(qq) && isfinite(mx) && isfinite(my) &&
                      isfinite(mz) && isfinite(s3[0]) && isfinite(s3[1]) && isfinite(s3[2]);
  if (usable) {
    inv = rsqrtf(qq);
    w = q4[0] * inv, x = q4[1] * inv, y = q4[2] * inv, z = q4[3] * inv;
    R[0][0] = 1.f - 2.f * (y * y + z * z);
    R[0][1] = 2.f * (x * y - w * z);
    R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z);
    R[1][1] = 1.f - 2.f * (x * x + z * z);
    R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y);
    R[2][1] = 2.f * (y * z + w * x);
    R[2][2] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) M[r][k] = R[r][k] * s3[k];
    // Sigma = M M^T, symmetric: its 6 entries S[r][k], r <= k, in Su (row-major upper triangle)
    float Su[6];
#pragma unroll
    for (int r = 0, i = 0; r < 3; ++r)
#pragma unroll
      for (int k = r; k < 3; ++k, ++i) Su[i] = M[r][0] * M[k][0] + M[r][1] * M[k][1] + M[r][2] * M[k][2];
    auto S = [&](int r, int k) { return r <= k ? Su[r * 3 + k - (r * (r + 1)) / 2] : Su[k * 3 + r - (k * (k + 1)) / 2]; };
    // this warp's views: warp, warp + kPbWarps, ...
    for (int v = warp; v < n_views; v += kPbWarps) {
      const int64_t vg = (int64_t)v * n + g;
      // the compositing pass's sums over the view's pixels: S_x, S_y, S_xx, S_xy, S_yy, S_1
      // of dp = dL/dpower times (d, d d^T, 1), and dL/dintensity
      const float4 q0 = reinterpret_cast<const float4*>(g2d)[2 * vg];
      const float4 q1 = reinterpret_cast<const float4*>(g2d)[2 * vg + 1];
      s1 += q1.y;
      gi += q1.z;
      if (q0.x == 0.f && q0.y == 0.f && q0.z == 0.f && q0.w == 0.f && q1.x == 0.f && q1.y == 0.f) continue;
      const Camera cam = cams[v];
      const float c = cam.c, s = cam.s, fu = cam.fu, fv = cam.fv;
      const float tx = c * my - s * mx, ty = -mz, tz = -c * mx - s * my + cam.L;
      const float iz = 1.f / tz;
      const float ax = tx * iz, ay = ty * iz;
      const float gu = fu * iz, gv = fv * iz;
      const float T0[3] = {gu * (ax * c - s), gu * (ax * s + c), 0.f};
      const float T1[3] = {gv * (ay * c), gv * (ay * s), -gv};
      float ST0[3], ST1[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        ST0[r] = S(r, 0) * T0[0] + S(r, 1) * T0[1] + S(r, 2) * T0[2];
        ST1[r] = S(r, 0) * T1[0] + S(r, 1) * T1[1] + S(r, 2) * T1[2];
      }
      const float A = T0[0] * ST0[0] + T0[1] * ST0[1] + T0[2] * ST0[2] + kDilate;
      const float B = T1[0] * ST0[0] + T1[1] * ST0[1] + T1[2] * ST0[2];
      const float C = T1[0] * ST1[0] + T1[1] * ST1[1] + T1[2] * ST1[2] + kDilate;
      const float idet = 1.f / (A * C - B * B);
      const float ka = C * idet, kb = -B * idet, kc = A * idet;
      // power = -1/2 (a dx^2 + 2 b dx dy + c dy^2), d = u - p: dL/du = -K (S_x, S_y),
      // dL/d(a, b, c) = (-S_xx / 2, -S_xy, -S_yy / 2)
      const float gux = -(ka * q0.x + kb * q0.y), guy = -(kb * q0.x + kc * q0.y);
      const float ga = -0.5f * q0.z, gb = -q0.w, gc = -0.5f * q1.x;
      // the view's 2-D gradients replace the sums (dL/dopacity = S_1 / opacity)
      reinterpret_cast<float4*>(g2d)[2 * vg] = make_float4(gux, guy, ga, gb);
      reinterpret_cast<float4*>(g2d)[2 * vg + 1] = make_float4(gc, q1.y / opac[g], q1.z, 0.f);
      // conic K = Sigma''^-1; dL/dSigma'' = -K Gh K, Gh = [[ga, gb/2], [gb/2, gc]]
      const float hb = 0.5f * gb;
      const float KG00 = ka * ga + kb * hb, KG01 = ka * hb + kb * gc;
      const float KG10 = kb * ga + kc * hb, KG11 = kb * hb + kc * gc;
      const float g00 = -(KG00 * ka + KG01 * kb);
      const float g01 = -(KG00 * kb + KG01 * kc);
      const float g11 = -(KG10 * kb + KG11 * kc);
      // Sigma'' = T Sigma T^T + 0.3 I with rows T0, T1
#pragma unroll
      for (int r = 0, i = 0; r < 3; ++r)
#pragma unroll
        for (int k = r; k < 3; ++k, ++i)
          gSu[i] += g00 * T0[r] * T0[k] + g01 * (T0[r] * T1[k] + T1[r] * T0[k]) + g11 * T1[r] * T1[k];
      float gT0[3], gT1[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        gT0[r] = 2.f * (g00 * ST0[r] + g01 * ST1[r]);
        gT1[r] = 2.f * (g01 * ST0[r] + g11 * ST1[r]);
      }
      // T0 = (fu/tz)(W0 - ax W2), T1 = (fv/tz)(W1 - ay W2); W0 = (-s, c, 0), W1 = (0, 0, -1), W2 = (-c, -s, 0)
      const float fu2 = fu * iz * iz, fv2 = fv * iz * iz;
      const float gT0W2 = -c * gT0[0] - s * gT0[1];
      const float gT1W2 = -c * gT1[0] - s * gT1[1];
      float gtx = -fu2 * gT0W2;
      float gty = -fv2 * gT1W2;
      float gtz = -fu2 * (gT0[0] * (2.f * ax * c - s) + gT0[1] * (2.f * ax * s + c)) -
                  fv2 * (gT1[0] * (2.f * ay * c) + gT1[1] * (2.f * ay * s) - gT1[2]);
      // u = (fu tx/tz, fv ty/tz) (centred)
      gtx += gux * gu;
      gty += guy * gv;
      gtz -= (gux * fu * ax + guy * fv * ay) * iz;
      // t = W mu + (0, 0, L)
      gm[0] += -s * gtx - c * gtz;
      gm[1] += c * gtx - s * gtz;
      gm[2] += -gty;
    }
  }
  {
    const float part[11] = {gSu[0], gSu[1], gSu[2], gSu[3], gSu[4], gSu[5], gm[0], gm[1], gm[2], s1, gi};
#pragma unroll
    for (int k = 0; k < 11; ++k) s_part[warp][k][lane] = part[k];
  }
  __syncthreads();
  if (warp != 0 || !live) return;
  {
    float tot[11];
#pragma unroll
    for (int k = 0; k < 11; ++k) {
      tot[k] = 0.f;
#pragma unroll
      for (int j = 0; j < kPbWarps; ++j) tot[k] += s_part[j][k][lane];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) gSu[k] = tot[k];
    gm[0] = tot[6], gm[1] = tot[7], gm[2] = tot[8];
    s1 = tot[9];
    gi = tot[10];
  }
  if (usable) {
    const float gS[3][3] = {{gSu[0], gSu[1], gSu[2]}, {gSu[1], gSu[3], gSu[4]}, {gSu[2], gSu[4], gSu[5]}};
    // Sigma = M M^T, M = R S
    float gM[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) gM[r][k] = 2.f * (gS[r][0] * M[0][k] + gS[r][1] * M[1][k] + gS[r][2] * M[2][k]);
    float gR[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gsc[k] = gM[0][k] * R[0][k] + gM[1][k] * R[1][k] + gM[2][k] * R[2][k];
#pragma unroll
      for (int r = 0; r < 3; ++r) gR[r][k] = gM[r][k] * s3[k];
    }
    // dR/d(w, x, y, z) of the unit quaternion
    float gw = 2.f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
    float gx = 2.f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2.f * x * gR[1][1] - w * gR[1][2] +
                      z * gR[2][0] + w * gR[2][1] - 2.f * x * gR[2][2]);
    float gy = 2.f * (-2.f * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] -
                      w * gR[2][0] + z * gR[2][1] - 2.f * y * gR[2][2]);
    float gz = 2.f * (-2.f * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2.f * z * gR[1][1] +
                      y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
    const float dot = gw * w + gx * x + gy * y + gz * z;
    gq[0] = (gw - w * dot) * inv;
    gq[1] = (gx - x * dot) * inv;
    gq[2] = (gy - y * dot) * inv;
    gq[3] = (gz - z * dot) * inv;
    go = s1 / opac[g];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    g_mean[k * n + g] = gm[k];
    g_scale[k * n + g] = gsc[k];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) g_quat[k * n + g] = gq[k];
  g_opac[g] = go;
  g_inten[g] = gi;
}

cudaError_t launch_project_bwd(xg_frame* f, const xg_gaussians* g, const xg_grads* out, cudaStream_t st) {
  const int64_t n = f->n;
  Timed t(f, kProjectBwd, st);
  k_project_bwd<<<(unsigned)((n + kPbGaussians - 1) / kPbGaussians), 32 * kPbWarps, 0, st>>>(g->mean, g->scale, g->quat, g->opacity, n, f->n_views, f->p.cam,
                                                             f->p.grad2d, f->p.status, out->mean, out->scale,
                                                             out->quat, out->opacity, out->intensity);
  return cudaGetLastError();
}

}  // namespace xg

// FDK cone-beam reconstruction (Feldkamp, Davis, Kress) from a full circular scan, the
// downstream use of rendered projections in the paper (Sec. 4, Table 2), in the scanner
// geometry of Eq. 12:
//   1. P_w = P D / sqrt(D^2 + p^2 + zeta^2) with (p, zeta) the pixel centre scaled to the
//      plane through the rotation axis (tau = pitch L_SO / L_SD), D = L_SO;
//   2. Q = tau (h * P_w) along every detector row, h the ramp (Ram-Lak) kernel:
//      h[0] = 1 / (4 tau^2), h[n odd] = -1 / (pi^2 n^2 tau^2), h[n even] = 0;
//   3. f(mu) = (pi / V) sum_v U^2 Q_v(U t_x / tau + W/2 - 1/2, U t_y / tau + H/2 - 1/2),
//      U = D / t_z, t = M_ext mu, bilinear, zero outside the detector.
#include <math.h>

#include "xg_internal.cuh"

namespace xg {
namespace {

struct FdkCam {
  float c, s, D, inv_tau_u, inv_tau_v, cx, cy, tau_u;  // cx, cy = W/2 - 1/2, H/2 - 1/2
};

constexpr double kPi = 3.14159265358979323846;
constexpr int kFilterThreads = 256;
constexpr int kBpZ = 8;  // voxels along z per back-projection thread

// One CTA per (detector row, view): weight the row into shared memory (zero-padded by W on
// both sides), then Q[x] = tau (h0 P_w[x] + sum_{n odd} h[n] (P_w[x - n] + P_w[x + n])).
__global__ void __launch_bounds__(kFilterThreads) k_fdk_filter(const float* __restrict__ proj,
                                                               const FdkCam* __restrict__ cams,
                                                               const float* __restrict__ h_odd, int W, int H,
                                                               float tau_v, float* __restrict__ q) {
  extern __shared__ float s_row[];  // [3 W]
  const int y = blockIdx.x, v = blockIdx.y;
  const FdkCam cam = cams[v];
  const float zeta = ((float)y + 0.5f - 0.5f * (float)H) * tau_v;
  const float D2z2 = cam.D * cam.D + zeta * zeta;
  const float* row = proj + ((int64_t)v * H + y) * W;
  for (int x = threadIdx.x; x < 3 * W; x += blockDim.x) {
    const int k = x - W;
    float w = 0.f;
    if (k >= 0 && k < W) {
      const float p = ((float)k + 0.5f - 0.5f * (float)W) * cam.tau_u;
      w = row[k] * (cam.D * rsqrtf(D2z2 + p * p));
    }
    s_row[x] = w;
  }
  __syncthreads();
  const float h0 = 0.25f / (cam.tau_u * cam.tau_u);
  float* out = q + ((int64_t)v * H + y) * W;
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    const float* c = s_row + W + x;
    float acc = h0 * c[0];
    for (int m = 0, n = 1; n < W; ++m, n += 2) acc = fmaf(h_odd[m], c[-n] + c[n], acc);
    out[x] = cam.tau_u * acc;
  }
}

__device__ __forceinline__ float tap(const float* __restrict__ img, int W, int H, int x, int y) {
  return (x >= 0 && x < W && y >= 0 && y < H) ? __ldg(img + (int64_t)y * W + x) : 0.f;
}

// Thread = one (x, y) voxel column over kBpZ consecutive z; all views summed in registers.
__global__ void __launch_bounds__(256) k_fdk_backproject(const float* __restrict__ q, const FdkCam* __restrict__ cams,
                                                         int n_views, int W, int H, int nx, int ny, int nz,
                                                         float voxel, float scale, float* __restrict__ vol) {
  extern __shared__ FdkCam s_cam[];
  for (int i = threadIdx.x; i < n_views; i += blockDim.x) s_cam[i] = cams[i];
  __syncthreads();
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int k0 = blockIdx.y * kBpZ;
  if (col >= (int64_t)nx * ny) return;
  const int i = (int)(col % nx), j = (int)(col / nx);
  const float X = ((float)i + 0.5f - 0.5f * (float)nx) * voxel;
  const float Y = ((float)j + 0.5f - 0.5f * (float)ny) * voxel;
  float acc[kBpZ];
#pragma unroll
  for (int z = 0; z < kBpZ; ++z) acc[z] = 0.f;
  for (int v = 0; v < n_views; ++v) {
    const FdkCam cam = s_cam[v];
    const float tx = -cam.s * X + cam.c * Y;
    const float tz = cam.D - (cam.c * X + cam.s * Y);
    const float U = cam.D / tz;
    // indices beyond the detector sample zeros: clamp them so the conversions stay in range
    const float xi = fminf(fmaxf(U * tx * cam.inv_tau_u + cam.cx, -2.f), (float)W + 1.f);
    const float fxf = floorf(xi);
    const int x0 = (int)fxf;
    const float fx = xi - fxf;
    const float U2 = U * U;
    const float* img = q + (int64_t)v * H * W;
#pragma unroll
    for (int z = 0; z < kBpZ; ++z) {
      const int k = k0 + z;
      const float Z = ((float)k + 0.5f - 0.5f * (float)nz) * voxel;
      const float yi = fminf(fmaxf(U * (-Z) * cam.inv_tau_v + cam.cy, -2.f), (float)H + 1.f);
      const float fyf = floorf(yi);
      const int y0 = (int)fyf;
      const float fy = yi - fyf;
      const float top = (1.f - fx) * tap(img, W, H, x0, y0) + fx * tap(img, W, H, x0 + 1, y0);
      const float bot = (1.f - fx) * tap(img, W, H, x0, y0 + 1) + fx * tap(img, W, H, x0 + 1, y0 + 1);
      acc[z] = fmaf(U2, (1.f - fy) * top + fy * bot, acc[z]);
    }
  }
#pragma unroll
  for (int z = 0; z < kBpZ; ++z) {
    const int k = k0 + z;
    if (k < nz) vol[((int64_t)k * ny + j) * nx + i] = acc[z] * scale;
  }
}

struct FdkLayout {
  size_t cams, h_odd, q, total;
};

FdkLayout fdk_layout(int32_t V, int32_t W, int32_t H) {
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  FdkLayout l;
  l.cams = 0;
  l.h_odd = up(sizeof(FdkCam) * (size_t)V);
  l.q = l.h_odd + up(sizeof(float) * (size_t)(W / 2 + 1));
  l.total = l.q + up(sizeof(float) * (size_t)V * W * H);
  return l;
}

bool valid_volume(const xg_volume* vol) {
  return vol && vol->nx >= 1 && vol->ny >= 1 && vol->nz >= 1 && vol->nx <= 4096 && vol->ny <= 4096 &&
         vol->nz <= 4096 && isfinite(vol->voxel_mm) && vol->voxel_mm > 0;
}

}  // namespace
}  // namespace xg

extern "C" {

size_t xg_fdk_workspace_bytes(int32_t n_views, int32_t width, int32_t height) {
  if (n_views < 1 || n_views > 65536 || width < 1 || width > 4096 || height < 1 || height > 4096) return 0;
  return xg::fdk_layout(n_views, width, height).total;
}

xg_status xg_fdk(const xg_view* views, int32_t n_views, const float* projections, const xg_volume* vol,
                 float* volume, void* workspace, size_t workspace_bytes, void* stream) {
  if (!views || n_views < 1 || !projections || !xg::valid_volume(vol) || !volume) return XG_ERR_INVALID_ARG;
  const int32_t W = views[0].width, H = views[0].height;
  const size_t need = xg_fdk_workspace_bytes(n_views, W, H);
  if (need == 0) return XG_ERR_INVALID_ARG;
  const xg_view& w0 = views[0];
  if (!(isfinite(w0.sod_mm) && w0.sod_mm > 0 && isfinite(w0.sdd_mm) && w0.sdd_mm > 0 && isfinite(w0.pitch_u_mm) &&
        w0.pitch_u_mm > 0 && isfinite(w0.pitch_v_mm) && w0.pitch_v_mm > 0))
    return XG_ERR_INVALID_ARG;
  for (int32_t v = 0; v < n_views; ++v) {  // one scanner, only the angle changes
    const xg_view& w = views[v];
    if (w.width != W || w.height != H || w.sod_mm != w0.sod_mm || w.sdd_mm != w0.sdd_mm ||
        w.pitch_u_mm != w0.pitch_u_mm || w.pitch_v_mm != w0.pitch_v_mm || !isfinite(w.angle_rad))
      return XG_ERR_INVALID_ARG;
  }
  if (!workspace || ((uintptr_t)workspace % 256) != 0 || workspace_bytes < need) return XG_ERR_WORKSPACE;
  const xg::FdkLayout L = xg::fdk_layout(n_views, W, H);
  char* base = (char*)workspace;
  auto* cams = (xg::FdkCam*)(base + L.cams);
  auto* h_odd = (float*)(base + L.h_odd);
  auto* q = (float*)(base + L.q);
  cudaStream_t st = (cudaStream_t)stream;

  // camera constants (FP64, rounded once) and the odd ramp taps, staged through host memory
  const size_t host_bytes = sizeof(xg::FdkCam) * (size_t)n_views + sizeof(float) * (size_t)(W / 2 + 1);
  char* host = (char*)malloc(host_bytes);
  if (!host) return XG_ERR_INVALID_ARG;
  auto* hc = (xg::FdkCam*)host;
  auto* hh = (float*)(host + sizeof(xg::FdkCam) * (size_t)n_views);
  for (int32_t v = 0; v < n_views; ++v) {
    const xg_view& w = views[v];
    const double tu = w.pitch_u_mm * w.sod_mm / w.sdd_mm, tv = w.pitch_v_mm * w.sod_mm / w.sdd_mm;
    hc[v] = xg::FdkCam{(float)cos(w.angle_rad), (float)sin(w.angle_rad), (float)w.sod_mm, (float)(1.0 / tu),
                       (float)(1.0 / tv), (float)(0.5 * W - 0.5), (float)(0.5 * H - 0.5), (float)tu};
  }
  const double tau_u = views[0].pitch_u_mm * views[0].sod_mm / views[0].sdd_mm;
  const double tau_v = views[0].pitch_v_mm * views[0].sod_mm / views[0].sdd_mm;
  for (int m = 0; 2 * m + 1 < W; ++m) {
    const double n = 2.0 * m + 1.0;
    hh[m] = (float)(-1.0 / (xg::kPi * xg::kPi * n * n * tau_u * tau_u));
  }
  cudaError_t e = cudaMemcpyAsync(cams, host, sizeof(xg::FdkCam) * (size_t)n_views, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_odd, hh, sizeof(float) * (size_t)(W / 2 + 1), cudaMemcpyHostToDevice, st);
  free(host);  // pageable source: staged when cudaMemcpyAsync returns
  if (e != cudaSuccess) return XG_ERR_CUDA;

  const size_t filt_smem = sizeof(float) * 3 * (size_t)W;
  if (filt_smem > 48 * 1024) {
    e = cudaFuncSetAttribute(xg::k_fdk_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filt_smem);
    if (e != cudaSuccess) return XG_ERR_CUDA;
  }
  xg::k_fdk_filter<<<dim3((unsigned)H, (unsigned)n_views), xg::kFilterThreads, filt_smem, st>>>(
      projections, cams, h_odd, W, H, (float)tau_v, q);
  const int64_t cols = (int64_t)vol->nx * vol->ny;
  const size_t cam_smem = sizeof(xg::FdkCam) * (size_t)n_views;
  if (cam_smem > 48 * 1024) {
    if (cam_smem > 200 * 1024) return XG_ERR_INVALID_ARG;
    e = cudaFuncSetAttribute(xg::k_fdk_backproject, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cam_smem);
    if (e != cudaSuccess) return XG_ERR_CUDA;
  }
  const dim3 grid((unsigned)((cols + 255) / 256), (unsigned)((vol->nz + xg::kBpZ - 1) / xg::kBpZ));
  xg::k_fdk_backproject<<<grid, 256, cam_smem, st>>>(q, cams, n_views, W, H, vol->nx, vol->ny, vol->nz,
                                                      (float)vol->voxel_mm, (float)(xg::kPi / n_views), volume);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

}  // extern "C"

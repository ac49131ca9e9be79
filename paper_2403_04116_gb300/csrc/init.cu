// ACUI grid initialisation of the Gaussian centres (Sec. 3.3, Eq. 13): the points
// (n_1 S_1 d / M_1, n_2 S_2 d / M_2, n_3 S_3 d / M_3) with |n_i| <= floor(M_i / (2 d)) + 1,
// listed with n_1 slowest, each n_i ascending; each coordinate is formed in FP64 as
// ((n S) d) / M and rounded once to FP32.
#include <math.h>

#include "xg_internal.cuh"

namespace xg {
namespace {

struct AcuiAxis {
  double S, d, M;
  int32_t c;  // floor(M / (2 d)) + 1
};

__global__ void k_acui(AcuiAxis ax0, AcuiAxis ax1, AcuiAxis ax2, int64_t count, float* __restrict__ mean) {
  const int64_t k1 = 2 * ax1.c + 1, k2 = 2 * ax2.c + 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i2 = i % k2, i1 = (i / k2) % k1, i0 = i / (k1 * k2);
    const AcuiAxis* axes[3] = {&ax0, &ax1, &ax2};
    const int64_t idx[3] = {i0, i1, i2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double n = (double)(idx[a] - axes[a]->c);
      mean[a * count + i] = __double2float_rn(__ddiv_rn(__dmul_rn(__dmul_rn(n, axes[a]->S), axes[a]->d), axes[a]->M));
    }
  }
}

bool acui_axes(const double* size_mm, const int32_t* grid, double interval, AcuiAxis* ax, int64_t* count) {
  if (!size_mm || !grid || !(isfinite(interval) && interval > 0.0)) return false;
  int64_t n = 1;
  for (int a = 0; a < 3; ++a) {
    if (!(isfinite(size_mm[a]) && size_mm[a] > 0.0) || grid[a] < 1) return false;
    const double h = floor((double)grid[a] / (2.0 * interval));
    if (h > (double)(1 << 20)) return false;
    ax[a] = AcuiAxis{size_mm[a], interval, (double)grid[a], (int32_t)h + 1};
    n *= 2 * (int64_t)ax[a].c + 1;
    if (n >= ((int64_t)1 << 31)) return false;
  }
  *count = n;
  return true;
}

}  // namespace
}  // namespace xg

extern "C" {

int64_t xg_acui_count(const double size_mm[3], const int32_t grid[3], double interval) {
  xg::AcuiAxis ax[3];
  int64_t n = 0;
  return xg::acui_axes(size_mm, grid, interval, ax, &n) ? n : 0;
}

xg_status xg_acui_points(const double size_mm[3], const int32_t grid[3], double interval, float* mean,
                         int64_t capacity, void* stream) {
  xg::AcuiAxis ax[3];
  int64_t n = 0;
  if (!xg::acui_axes(size_mm, grid, interval, ax, &n) || !mean) return XG_ERR_INVALID_ARG;
  if (n > capacity) return XG_ERR_CAPACITY;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)xg::device_sms() * 16);
  xg::k_acui<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(ax[0], ax[1], ax[2], n, mean);
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

}  // extern "C"

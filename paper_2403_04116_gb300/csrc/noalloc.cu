// Allocation-free variant of the pair sort inside xg_bin_sort.
//
// Some callers cannot allocate device memory: plugins hosted by an application that owns
// the GPU's memory pool, and real-time pipelines that forbid allocation after start-up
// (cudaMalloc can synchronise the device and its latency is unbounded).  They can still
// sort (tile, depth, Gaussian) pairs with xg_sort_pairs_noalloc: the caller passes only
// the input and output arrays; the ping-pong buffers, the digit histograms and the pair
// count live in the file-scope device array below.  Every GPU that loads the library holds
// that array (about 12.6 MB) until the process exits.
#include <stddef.h>

#include <mutex>

#include "xg_internal.cuh"

namespace xg {

constexpr size_t kNoallocStatusBytes = 256;
constexpr size_t kNoallocHistBytes = (size_t)4 * 256 * (kMaxSortBlocks + 1);
constexpr size_t kNoallocBufBytes = (size_t)4 * XG_NOALLOC_MAX_PAIRS;
constexpr size_t kNoallocBytes = kNoallocStatusBytes + kNoallocHistBytes + 3 * kNoallocBufBytes;

// Shared by every call on a device; the last call's contents stay behind.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices];

// Device address of the scratch array on the current device.  In host code
// `g_noalloc_scratch` names a host-side stand-in, never pass it to a kernel.  Outside a
// stream capture the address is looked up on every call (cheap once the module is loaded),
// so a context torn down and created again by cudaDeviceReset, which may place the array
// elsewhere, never leaves a stale address behind; inside a capture, where the lookup could
// load the module, the address of the last call outside a capture on this device is used.
xg_status noalloc_scratch(cudaStream_t st, unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return XG_ERR_CUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return XG_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return XG_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  } else if (!g_noalloc_ptr[dev]) {
    return XG_ERR_CUDA;  // the first call on a device must come before any capture
  }
  *out = (unsigned char*)g_noalloc_ptr[dev];
  return XG_OK;
}

}  // namespace

// The status word the radix kernels read the pair count from; cleared on every call.
__global__ void k_noalloc_status(DevStatus* st, int64_t count) {
  if (threadIdx.x != 0) return;
  st->code = XG_OK;
  st->next_item = 0;
  st->pairs = count;
  st->nonfinite = 0;
  st->fwd_evaluated = st->fwd_contrib = st->bwd_evaluated = st->bwd_contrib = 0;
  st->scan_total = (unsigned long long)count;
}

}  // namespace xg

extern "C" xg_status xg_sort_pairs_noalloc(const uint32_t* key_tile, const uint32_t* key_depth, const uint32_t* value,
                                           int64_t count, int32_t tile_bits, uint32_t* out_key_tile,
                                           uint32_t* out_key_depth, uint32_t* out_value, void* stream) {
  using namespace xg;
  if (count < 0 || count > XG_NOALLOC_MAX_PAIRS || tile_bits < 0 || tile_bits > 32) return XG_ERR_INVALID_ARG;
  if (count > 0 && (!key_tile || !key_depth || !value || !out_key_tile || !out_key_depth || !out_value))
    return XG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  const xg_status s = noalloc_scratch(st, &base);
  if (s != XG_OK) return s;
  if (radix_prepare() != cudaSuccess) return XG_ERR_CUDA;
  if (count == 0) return XG_OK;
  DevStatus* status = (DevStatus*)base;
  uint32_t* hist = (uint32_t*)(base + kNoallocStatusBytes);
  uint32_t* tmp_tile = (uint32_t*)(base + kNoallocStatusBytes + kNoallocHistBytes);
  uint32_t* tmp_depth = tmp_tile + XG_NOALLOC_MAX_PAIRS;
  uint32_t* tmp_val = tmp_depth + XG_NOALLOC_MAX_PAIRS;

  k_noalloc_status<<<1, 32, 0, st>>>(status, count);
  const int passes = 4 + (tile_bits + 7) / 8;
  // alternate so that the last pass writes the caller's output
  const uint32_t* src[3] = {key_tile, key_depth, value};
  for (int pass = 0; pass < passes; ++pass) {
    const bool to_out = ((passes - 1 - pass) % 2) == 0;
    uint32_t* dst[3] = {to_out ? out_key_tile : tmp_tile, to_out ? out_key_depth : tmp_depth,
                        to_out ? out_value : tmp_val};
    const int digit_word = pass < 4 ? 0 : 1;
    const int shift = pass < 4 ? 8 * pass : 8 * (pass - 4);
    // words: 0 tile key, 1 depth key, 2 value
    SortArrays<3> arr;
    for (int w = 0; w < 3; ++w) {
      arr.in[w] = src[w];
      arr.out[w] = dst[w];
    }
    if (radix_pass<3>(nullptr, arr, digit_word ? 0 : 1, shift, 255u, sort_geom(count, 1, sort_blocks()), status, hist, st) !=
        cudaSuccess)
      return XG_ERR_CUDA;
    src[0] = dst[0];
    src[1] = dst[1];
    src[2] = dst[2];
  }
  return cudaGetLastError() == cudaSuccess ? XG_OK : XG_ERR_CUDA;
}

extern "C" xg_status xg_sort_pairs_noalloc_status(void* stream, int32_t* device_code) {
  using namespace xg;
  if (!device_code) return XG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  const xg_status s = noalloc_scratch(st, &base);
  if (s != XG_OK) return s;
  if (cudaStreamSynchronize(st) != cudaSuccess) return XG_ERR_CUDA;
  int32_t code = XG_OK;
  if (cudaMemcpy(&code, base + offsetof(DevStatus, code), sizeof code, cudaMemcpyDeviceToHost) != cudaSuccess)
    return XG_ERR_CUDA;
  *device_code = code;
  return XG_OK;
}

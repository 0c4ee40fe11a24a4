// Allocation-free column statistics of an 8-bit TF image: per column the sum
// of levels S_f and the exact Otsu threshold (Eq. 4), with the column
// histograms held in a fixed file-scope device array instead of context
// memory.  The paper has no counterpart of this entry point; it exists for
// callers that must not allocate device memory at all, such as a host
// framework that owns every byte of device memory and forbids allocation in
// its per-frame callbacks, or a real-time receive loop, where a cudaMalloc
// or cudaFree could synchronise the device and stall the other streams.
#include <cstdint>
#include <mutex>

#include "common.cuh"

// Column histograms of the last call: [RISE_NOALLOC_MAX_COLS][256] counts,
// 4 MiB.  Every GPU on which the library is loaded holds it until the
// process exits.  Host code must not pass this name to a kernel (on the host
// it is only a stand-in); the set-up below fetches its device address.
static __device__ __align__(256) uint32_t rise_noalloc_hist[RISE_NOALLOC_MAX_COLS * 256];

namespace rise {
namespace {

// Variant of the cluster histogram kernel for the 8-bit input: a block counts
// 64 columns of one band of rows in shared memory (level-major, so a warp's
// 32 lanes hit 32 banks), then adds its non-zero counts into the global
// histogram with atomics.  Bands are independent; no cluster is needed.
constexpr int NA_COLS = 64, NA_WARPS = 8, NA_UNROLL = 8;
constexpr int NA_SMEM = 256 * NA_COLS * (int)sizeof(uint32_t);   // 64 KB

__global__ void __launch_bounds__(32 * NA_WARPS, 2)
noalloc_hist_kernel(const uint8_t *__restrict__ img, int64_t T, int F, int64_t rows_per_band,
                    uint32_t *hist) {
  extern __shared__ uint32_t cnt[];   // [256 levels][64 column slots]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 256 * NA_COLS; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  // lane l reads columns 2l and 2l+1 of the block's 64; slot l and l+32
  const int c0 = blockIdx.x * NA_COLS + 2 * lane;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_band;
  const int64_t r1 = min(T, r0 + rows_per_band);
  const int64_t stride = (int64_t)NA_WARPS * F;
  int64_t r = r0 + warp;
  for (; r + (NA_UNROLL - 1) * NA_WARPS < r1; r += NA_UNROLL * NA_WARPS) {
    const uint8_t *p = img + r * F + c0;
    uint32_t w[NA_UNROLL];
#pragma unroll
    for (int u = 0; u < NA_UNROLL; ++u) w[u] = __ldg(reinterpret_cast<const uint16_t *>(p + u * stride));
#pragma unroll
    for (int u = 0; u < NA_UNROLL; ++u) {
      atomicAdd(&cnt[(w[u] & 0xffu) * NA_COLS + lane], 1u);
      atomicAdd(&cnt[(w[u] >> 8) * NA_COLS + lane + 32], 1u);
    }
  }
  for (; r < r1; r += NA_WARPS) {
    const uint32_t w = __ldg(reinterpret_cast<const uint16_t *>(img + r * F + c0));
    atomicAdd(&cnt[(w & 0xffu) * NA_COLS + lane], 1u);
    atomicAdd(&cnt[(w >> 8) * NA_COLS + lane + 32], 1u);
  }
  __syncthreads();
  for (int i = tid; i < 256 * NA_COLS; i += blockDim.x) {
    const uint32_t v = cnt[i];
    if (v) {
      const int level = i / NA_COLS, slot = i % NA_COLS;
      const int col = blockIdx.x * NA_COLS + 2 * (slot & 31) + (slot >> 5);
      atomicAdd(&hist[(size_t)col * 256 + level], v);
    }
  }
}

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_setup_mu;
uint32_t *g_scratch[NA_MAX_DEVICES];   // device address of rise_noalloc_hist, per device

// With device dev current: the device address of the scratch array and the
// shared-memory size of the histogram kernel.  Looked up on the first call
// on a device and again on every call whose stream is not capturing (a
// device reset gives the array a new address and clears the kernel's
// attribute); a capturing call reuses the last address, since the set-up
// calls are not stream work.
int setup_device(int dev, cudaStream_t s, uint32_t **out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;   // unknown: take the capturing branch
  }
  if (!g_scratch[dev] || cap == cudaStreamCaptureStatusNone) {
    uint32_t *p = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void **>(&p), rise_noalloc_hist) != cudaSuccess || !p)
      return RISE_ECUDA;
    if (cudaFuncSetAttribute(noalloc_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             NA_SMEM) != cudaSuccess)
      return RISE_ECUDA;
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return RISE_OK;
}

// True when p is device (or managed) memory of device dev.
bool on_device(const void *p, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace
}  // namespace rise

extern "C" int rise_column_stats_noalloc(const uint8_t *img_dev, int64_t T, int F,
                                         rise_colstat *cols_dev, void *cuda_stream) {
  using namespace rise;
  if (!img_dev || !cols_dev) return RISE_EINVAL;
  if (T < 1 || T > RISE_MAX_ROWS) return RISE_EINVAL;
  if (F < RISE_MIN_FFT || (F & (F - 1)) != 0) return RISE_EINVAL;
  if (F > RISE_NOALLOC_MAX_COLS) return RISE_ESCRATCH;
  if ((reinterpret_cast<uintptr_t>(img_dev) & 1u) || (reinterpret_cast<uintptr_t>(cols_dev) & 7u))
    return RISE_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RISE_ECUDA;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return RISE_EINVAL;
  if (!on_device(img_dev, dev) || !on_device(cols_dev, dev)) return RISE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  uint32_t *hist = nullptr;
  int rc = setup_device(dev, s, &hist);
  if (rc != RISE_OK) return rc;
  // the array keeps the previous call's counts: clear this call's columns
  if (cudaMemsetAsync(hist, 0, (size_t)F * 256 * sizeof(uint32_t), s) != cudaSuccess) return RISE_ECUDA;
  if (cudaMemsetAsync(cols_dev, 0, (size_t)F * sizeof(rise_colstat), s) != cudaSuccess) return RISE_ECUDA;
  // about four blocks per SM over all (column group, row band) pairs
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int gx = F / NA_COLS;
  int64_t bands = ((int64_t)4 * sms + gx - 1) / gx;
  int64_t rows = (T + bands - 1) / bands;
  if (rows < 64) rows = 64;
  bands = (T + rows - 1) / rows;
  noalloc_hist_kernel<<<dim3((unsigned)gx, (unsigned)bands), 32 * NA_WARPS, NA_SMEM, s>>>(img_dev, T, F, rows, hist);
  count_launches(1);
  if (cudaGetLastError() != cudaSuccess) return RISE_ECUDA;
  if (launch_column_otsu(hist, T, F, cols_dev, s) != cudaSuccess) return RISE_ECUDA;
  return RISE_OK;
}

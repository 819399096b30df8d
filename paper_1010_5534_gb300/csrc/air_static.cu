// air_static.cu -- band flux of a device-resident image, computed without
// allocating any memory.
//
// The regular render entry points grow a cudaMalloc'd workspace on first use.
// Some callers cannot allocate at the time they need the flux: a real-time or
// serving loop that must not stall the device (cudaFree synchronises it), a
// plugin inside a host application whose device memory is owned by the host's
// own pool, or code that runs where the CUDA runtime forbids allocation. This
// file gives them one entry point whose only scratch is a fixed array in the
// library's own device image, reserved when the library is loaded on a device
// and held until the process exits.
#include <cmath>
#include <mutex>

#include "air_handle.cuh"

namespace air {

constexpr int kStaticFluxBlocks = 1024;                         // partial sums per band
constexpr int64_t kStaticFluxMaxN = ((int64_t)1 << 31) - 1;     // pixels per call
constexpr int kStaticMaxDevices = 64;
// Pixel levels the flux accepts: an image of base n0 has levels 0..max_level
// with n0 << max_level <= 2^20, so no render produces a level above 20.
constexpr int kStaticMaxLevel = 20;

// [block][band] partial sums: 1024 x 64 doubles = 512 KiB per device.
static __device__ __align__(256) double g_flux_scratch[kStaticFluxBlocks * kMaxBands];

__global__ void __launch_bounds__(256) k_flux_static_partial(
    const float *__restrict__ I, int64_t stride, int n_bands, const int32_t *__restrict__ level,
    const uint8_t *__restrict__ is_leaf, int64_t n, double area0, int64_t per_block,
    double *__restrict__ scratch) {
  __shared__ double sh[256];
  const int64_t start = (int64_t)blockIdx.x * per_block;
  const int64_t end = min(n, start + per_block);
  for (int b = 0; b < n_bands; ++b) {
    double s = 0.0;
    for (int64_t k = start + threadIdx.x; k < end; k += blockDim.x) {
      if (is_leaf && !is_leaf[k]) continue;
      const int L = level ? level[k] : 0;
      // 4^-L as exponent bits for 0 <= L <= kStaticMaxLevel; a level outside
      // that range (a corrupt or stale entry) makes the band's flux NaN
      const double scale = (L >= 0 && L <= kStaticMaxLevel)
                               ? __longlong_as_double((long long)(1023 - 2 * L) << 52)
                               : __longlong_as_double(0x7ff8000000000000ll);
      s += (double)I[(int64_t)b * stride + k] * area0 * scale;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
      if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
      __syncthreads();
    }
    if (threadIdx.x == 0) scratch[(int64_t)blockIdx.x * kMaxBands + b] = sh[0];
    __syncthreads();
  }
}

// One thread per band adds the block partials in block order.
__global__ void k_flux_static_final(const double *__restrict__ scratch, int nblocks, int n_bands,
                                    double *__restrict__ flux) {
  const int b = threadIdx.x;
  if (b >= n_bands) return;
  double s = 0.0;
  for (int x = 0; x < nblocks; ++x) s += scratch[(int64_t)x * kMaxBands + b];
  flux[b] = s;
}

static std::mutex g_scratch_mu;
static double *g_scratch_ptr[kStaticMaxDevices];
static bool g_scratch_ready[kStaticMaxDevices];

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the array's name as a device pointer). The
// address is cached for the life of the process: after cudaDeviceReset (or a
// destroyed and re-created primary context) the module may load elsewhere, so
// this entry point must not be used across a device reset.
static air_status static_scratch(double **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kStaticMaxDevices) return set_error(AIR_ERR_ARG, "device ordinal %d not supported", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ready[dev]) {
    double *p = nullptr;
    e = cudaGetSymbolAddress((void **)&p, g_flux_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_flux_scratch)");
    g_scratch_ptr[dev] = p;
    g_scratch_ready[dev] = true;
  }
  *out = g_scratch_ptr[dev];
  return AIR_OK;
}

// Device (or managed) memory of device `dev`.
static bool on_device(const void *p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeDevice) return a.device == dev;
  return a.type == cudaMemoryTypeManaged;
}

}  // namespace air

extern "C" air_status air_band_flux_static(const float *intensity, int64_t stride, int32_t n_bands,
                                           const int32_t *level, const uint8_t *is_leaf, int64_t n,
                                           double area0, double *band_flux, void *stream) {
  using namespace air;
  if (!intensity || !band_flux) return set_error(AIR_ERR_ARG, "intensity and band_flux must not be NULL");
  if (n_bands < 1 || n_bands > kMaxBands)
    return set_error(AIR_ERR_ARG, "n_bands %d is outside [1, %d], the static scratch limit", n_bands, kMaxBands);
  if (n < 0 || n > kStaticFluxMaxN)
    return set_error(AIR_ERR_ARG, "n %lld is outside [0, %lld], the static scratch limit", (long long)n,
                     (long long)kStaticFluxMaxN);
  if (stride < n) return set_error(AIR_ERR_ARG, "stride %lld < n %lld", (long long)stride, (long long)n);
  // the last element read, (n_bands - 1) * stride + n - 1, must fit an int64
  if (n_bands > 1 && stride > (INT64_MAX - n) / (n_bands - 1))
    return set_error(AIR_ERR_ARG, "stride %lld overflows the index range for %d bands", (long long)stride, n_bands);
  if (!std::isfinite(area0) || !(area0 > 0.0)) return set_error(AIR_ERR_ARG, "area0 must be finite and > 0");
  int dev = -1;
  cudaError_t de = cudaGetDevice(&dev);
  if (de != cudaSuccess) return cuda_fail(de, "cudaGetDevice");
  if (!on_device(intensity, dev) || !on_device(band_flux, dev) || (level && !on_device(level, dev)) ||
      (is_leaf && !on_device(is_leaf, dev)))
    return set_error(AIR_ERR_ARG, "every array must be device memory of the current device (%d)", dev);
  double *scratch = nullptr;
  air_status s = static_scratch(&scratch);
  if (s != AIR_OK) return s;
  set_error(AIR_OK, "");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t per_block = (n + kStaticFluxBlocks - 1) / kStaticFluxBlocks;
  if (per_block < 2048) per_block = 2048;
  const int nblocks = (int)((n + per_block - 1) / per_block);
  if (nblocks > 0)
    k_flux_static_partial<<<nblocks, 256, 0, st>>>(intensity, stride, n_bands, level, is_leaf, n,
                                                   area0, per_block, scratch);
  k_flux_static_final<<<1, 64, 0, st>>>(scratch, nblocks, n_bands, band_flux);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "air_band_flux_static launch");
  return AIR_OK;
}

// Energy entry point that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need the
// energy: code running under a memory pool that forbids growth, inside a
// region where cudaMalloc would synchronise the device, or in a process whose
// allocator is owned by another framework.  adft_energy_static computes
// E = 1/2 tr(DJ) - 1/4 tr(DK) from caller-owned D, J and K using scratch that
// lives in this file as a fixed-size device array, so the call itself never
// allocates.  The array (ADFT_STATIC_MAX_NBF doubles) exists on every device
// that loads the library, until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "adft_internal.cuh"

namespace adft {

// One partial sum per row of the matrices.
static __device__ __align__(256) double g_row_partial[ADFT_STATIC_MAX_NBF];

// Row sums: block b reduces rows b, b + gridDim.x, ... into g_row_partial.
static __global__ void k_energy_rows(int n, const double* __restrict__ D, const double* __restrict__ J,
                                     const double* __restrict__ K, double* partial) {
  __shared__ double ws[32];
  for (int row = blockIdx.x; row < n; row += gridDim.x) {
    double s = 0.0;
    const long long o = (long long)row * n;
    for (int c = threadIdx.x; c < n; c += blockDim.x) s += D[o + c] * (0.5 * J[o + c] - 0.25 * K[o + c]);
    for (int k = 16; k > 0; k >>= 1) s += __shfl_down_sync(0xffffffffu, s, k);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      s = (threadIdx.x < (blockDim.x >> 5)) ? ws[threadIdx.x] : 0.0;
      for (int k = 16; k > 0; k >>= 1) s += __shfl_down_sync(0xffffffffu, s, k);
      if (threadIdx.x == 0) partial[row] = s;
    }
    __syncthreads();
  }
}

// Sum of the row partials in a fixed order (one block).
static __global__ void k_energy_total(int n, const double* __restrict__ partial, double* E) {
  __shared__ double ws[32];
  double s = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) s += partial[r];
  for (int k = 16; k > 0; k >>= 1) s += __shfl_down_sync(0xffffffffu, s, k);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? ws[threadIdx.x] : 0.0;
    for (int k = 16; k > 0; k >>= 1) s += __shfl_down_sync(0xffffffffu, s, k);
    if (threadIdx.x == 0) *E = s;
  }
}

// Device address of g_row_partial, looked up once per device.  In host code
// the name g_row_partial is only a host-side stand-in, never a device address.
static std::mutex g_static_mu;
static double* g_static_ptr[64];

static int static_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    set_error("adft_energy_static: no usable CUDA device");
    return ADFT_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_row_partial);
    if (e != cudaSuccess || !p) {
      set_error(std::string("adft_energy_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return ADFT_ERR_CUDA;
    }
    g_static_ptr[dev] = (double*)p;
  }
  *out = g_static_ptr[dev];
  return ADFT_OK;
}

}  // namespace adft

extern "C" int adft_energy_static(const double* D, const double* J, const double* K, int nbf, double* E,
                                  void* stream) {
  using namespace adft;
  if (!D || !J || !K || !E) { set_error("adft_energy_static: NULL argument"); return ADFT_ERR_ARG; }
  if (nbf <= 0 || nbf > ADFT_STATIC_MAX_NBF) {
    set_error("adft_energy_static: nbf must be in 1.." + std::to_string(ADFT_STATIC_MAX_NBF) +
              " (size of the built-in scratch)");
    return ADFT_ERR_ARG;
  }
  double* partial = nullptr;
  const int st = static_scratch(&partial);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = nbf < 4 * sms ? nbf : 4 * sms;
  // Launch errors are checked per launch with cudaPeekAtLastError: an error
  // that earlier, unrelated work left behind is neither reported as this
  // call's nor cleared.
  const cudaError_t before = cudaPeekAtLastError();
  k_energy_rows<<<blocks, 256, 0, s>>>(nbf, D, J, K, partial);
  cudaError_t e = cudaPeekAtLastError();
  if (e == cudaSuccess || e == before) {
    k_energy_total<<<1, 1024, 0, s>>>(nbf, partial, E);
    e = cudaPeekAtLastError();
  }
  if (e != cudaSuccess && e != before) {
    set_error(std::string("adft_energy_static: launch failed: ") + cudaGetErrorString(e));
    return ADFT_ERR_CUDA;
  }
  return ADFT_OK;
}

// ALU peak microbenchmark: the FP64 and FP32 fused multiply-add rates of the
// current device, measured with independent FMA chains on every SM.  These
// are the denominators of the ERI kernels' roofline (the ERI and digestion
// kernels are bound by plain FP64 / FP32 arithmetic, not by tensor cores or
// memory bandwidth).
#include <cuda_runtime.h>

#include <string>

#include "adft_internal.cuh"

namespace adft {

constexpr int PEAK_CHAINS = 8;   // independent accumulators per thread
constexpr int PEAK_UNROLL = 16;  // FMAs per chain per loop trip

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* sink, int iters, T a, T b) {
  T x[PEAK_CHAINS];
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = T(threadIdx.x) * T(1e-3) + T(c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PEAK_UNROLL; ++k)
#pragma unroll
      for (int c = 0; c < PEAK_CHAINS; ++c) x[c] = x[c] * a + b;
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) s += x[c];
  if (s == T(-1.2345)) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

}  // namespace adft

extern "C" int adft_alu_peak(int fp64, int iters, double* tflops, double* ms) {
  using namespace adft;
  if (!tflops || iters <= 0) { set_error("adft_alu_peak: tflops must be non-NULL and iters > 0"); return ADFT_ERR_ARG; }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
    set_error("adft_alu_peak: no CUDA device");
    return ADFT_ERR_CUDA;
  }
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_error("adft_alu_peak: event creation failed");
    return ADFT_ERR_CUDA;
  }
  float t = 0.0f;
  cudaError_t err = cudaSuccess;
  for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, 0);
    if (fp64) k_fma_peak<double><<<blocks, threads>>>(nullptr, iters, 0.999999999, 1e-9);
    else k_fma_peak<float><<<blocks, threads>>>(nullptr, iters, 0.9999f, 1e-5f);
    cudaEventRecord(e1, 0);
    err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    set_error(std::string("adft_alu_peak: ") + cudaGetErrorString(err));
    return ADFT_ERR_CUDA;
  }
  const double flops = 2.0 * (double)blocks * threads * PEAK_CHAINS * PEAK_UNROLL * (double)iters;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return ADFT_OK;
}

// FP32 instantiations of the J/K kernels (the single-precision band of the
// mixed-precision dispatcher, Sec. 1.2.2).
#include "adft_eri.cuh"

namespace adft {

cudaError_t launch_jk_fp32(int X, int Y, const JKLaunch& a, int grid, cudaStream_t s) {
  return dispatch_jk<float>(X, Y, a, grid, s, std::make_integer_sequence<int, NCLS * NCLS>{});
}

}  // namespace adft

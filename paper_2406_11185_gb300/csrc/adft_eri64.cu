// FP64 instantiations: J/K kernels of all class pairs and the Schwarz kernels.
#include "adft_eri.cuh"

namespace adft {

cudaError_t launch_jk_fp64(int X, int Y, const JKLaunch& a, int grid, cudaStream_t s) {
  return dispatch_jk<double>(X, Y, a, grid, s, std::make_integer_sequence<int, NCLS * NCLS>{});
}

cudaError_t launch_schwarz(int X, const BasisView& bv, int first, int n, double* Q, cudaStream_t s) {
  if (X < 0 || X >= NCLS) return cudaErrorInvalidValue;
  const int blocks = (n + JK_THREADS - 1) / JK_THREADS;
  const RtClass C = make_rt_class(cls_la(X), cls_lb(X), cls_la(X), cls_lb(X));
  if (blocks > 0) k_schwarz_generic<<<blocks, JK_THREADS, 0, s>>>(bv, C, first, n, Q);
  return cudaGetLastError();
}

}  // namespace adft

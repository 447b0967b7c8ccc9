// Class-pair ERI kernels (FP64 band), class pairs [(9, 0), (9, 1), (9, 2), (9, 3), (9, 4), (9, 5), (9, 6), (9, 7), (9, 8), (9, 9)]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel
// with the other groups; also the Schwarz-bound kernels.
#define ADFT_ERI_SCHWARZ
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<double, 9, 0>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 9, 1>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 9, 2>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 9, 3>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 9, 4>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 9, 5>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 9, 6>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 9, 7>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 9, 8>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 9, 9>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);

cudaError_t launch_schwarz(int X, const BasisView& bv, int first, int n, int maxp, double* part, double* Qmax,
                           cudaStream_t s) {
  if (X < 0 || X >= NCLS) return cudaErrorInvalidValue;
  if (n <= 0 || maxp <= 0) return cudaSuccess;
  const RtClass C = make_rt_class(cls_la(X), cls_lb(X), cls_la(X), cls_lb(X));
  const int nab = ncart(cls_la(X)) * ncart(cls_lb(X));
  const long long t1 = (long long)n * C.nchunk * maxp, t2 = (long long)n * nab;
  k_schwarz_part<<<(unsigned)((t1 + JK_THREADS - 1) / JK_THREADS), JK_THREADS, 0, s>>>(bv, C, first, n, maxp, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_schwarz_reduce<<<(unsigned)((t2 + 255) / 256), 256, 0, s>>>(bv, first, n, nab, maxp, part,
                                                                reinterpret_cast<unsigned long long*>(Qmax));
  return cudaGetLastError();
}

cudaError_t launch_prim_schwarz(int X, const BasisView& bv, int first, int n, const int* pp_pair, int npp_class,
                                double* Qp, cudaStream_t s) {
  if (X < 0 || X >= NCLS) return cudaErrorInvalidValue;
  const int blocks = (npp_class + JK_THREADS - 1) / JK_THREADS;
  const RtClass C = make_rt_class(cls_la(X), cls_lb(X), cls_la(X), cls_lb(X));
  if (blocks > 0 && n > 0) k_prim_schwarz<<<blocks, JK_THREADS, 0, s>>>(bv, C, first, n, pp_pair, Qp);
  return cudaGetLastError();
}

}  // namespace adft

// Class-pair ERI kernels (FP64 band), class pairs [(7, 0), (7, 1), (7, 2), (7, 3), (7, 4), (7, 5), (7, 6), (7, 7), (8, 0), (8, 1), (8, 2), (8, 3), (8, 4), (8, 5), (8, 6), (8, 7), (8, 8)]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel
// with the other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<double, 7, 0>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 7, 1>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 7, 2>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 7, 3>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 7, 4>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 7, 5>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 7, 6>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 7, 7>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 8, 0>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 8, 1>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 8, 2>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 8, 3>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 8, 4>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 8, 5>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 8, 6>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 8, 7>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 8, 8>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);

}  // namespace adft

// Class-pair ERI kernels (FP64 band), class pairs [(6, 0), (6, 1), (6, 2), (6, 3), (6, 4), (6, 5), (6, 6)]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel
// with the other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<double, 6, 0>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 6, 1>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 6, 2>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 6, 3>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 6, 4>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 6, 5>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 6, 6>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);

}  // namespace adft

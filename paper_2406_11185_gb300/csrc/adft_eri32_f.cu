// Class-pair ERI kernels (FP32 band), class pairs [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 1), (3, 2), (3, 3)]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel
// with the other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<float, 0, 0>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 1, 0>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 1, 1>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 2, 0>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 2, 1>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 2, 2>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 3, 0>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 3, 1>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 3, 2>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 3, 3>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);

}  // namespace adft

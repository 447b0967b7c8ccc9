// Class-pair ERI kernels (FP32 band), class pairs [(9, 0), (9, 1), (9, 2), (9, 3), (9, 4), (9, 5), (9, 6), (9, 7), (9, 8), (9, 9)]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel
// with the other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<float, 9, 0>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 9, 1>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 9, 2>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 9, 3>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 9, 4>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 9, 5>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 9, 6>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 9, 7>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 9, 8>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<float, 9, 9>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);

}  // namespace adft

// Class-pair ERI kernels (FP64 band), class pairs [(5, 0), (5, 1), (5, 2)]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel
// with the other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<double, 5, 0>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 5, 1>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 5, 2>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);

}  // namespace adft

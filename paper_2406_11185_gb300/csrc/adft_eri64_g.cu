// Class-pair ERI kernels (FP64 band), class pairs [(4, 0), (4, 1), (4, 2)]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel
// with the other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<double, 4, 0>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 4, 1>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);
template cudaError_t launch_one<double, 4, 2>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);

}  // namespace adft

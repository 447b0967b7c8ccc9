// Class-pair ERI kernels (FP32 band), class pairs [(5, 3)]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel
// with the other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<float, 5, 3>(const JKLaunch&, int, int, cudaStream_t, KernelInfo*);

}  // namespace adft

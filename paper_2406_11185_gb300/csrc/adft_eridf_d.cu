// Class-pair ERI kernels (double-float evaluation of the FP64 band), bra classes [5]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel with
// the other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<df, 5, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 5, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 5, 2>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 5, 3>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 5, 4>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 5, 5>(const JKLaunch&, int, cudaStream_t);

}  // namespace adft

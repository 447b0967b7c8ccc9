// Class-pair ERI kernels (double-float evaluation of the FP64 band), bra classes [6]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel with
// the other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<df, 6, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 6, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 6, 2>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 6, 3>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 6, 4>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 6, 5>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 6, 6>(const JKLaunch&, int, cudaStream_t);

}  // namespace adft

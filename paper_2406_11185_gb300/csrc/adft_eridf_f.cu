// Class-pair ERI kernels (double-float evaluation of the FP64 band), bra classes [0, 1, 2, 3]:
// explicit instantiations of the launchers of adft_eri.cuh, compiled in parallel with
// the other groups.
#include "adft_eri.cuh"

namespace adft {

template cudaError_t launch_one<df, 0, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 1, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 1, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 2, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 2, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 2, 2>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 3, 0>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 3, 1>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 3, 2>(const JKLaunch&, int, cudaStream_t);
template cudaError_t launch_one<df, 3, 3>(const JKLaunch&, int, cudaStream_t);

}  // namespace adft
